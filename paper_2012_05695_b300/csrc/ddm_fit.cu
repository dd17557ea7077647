// Fit of the radial structure functions (not in the paper): sample every curve at 64
// log-spaced lags, seed (heuristic or MLP), and Levenberg-Marquardt of
// D(lag) = A (1 - exp(-(lag / tau)^beta)) + B.  Two lags per lane; the features take one
// warp per curve, the fit one block of four warps per curve (one damping value per warp).
//
// Every warp reduction ends with a broadcast of lane 0's value, so all lanes hold
// bitwise-identical sums and take identical accept / reject decisions.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "ddm_internal.h"

namespace ddm {

ddm_status mlp_forward_raw(const ddm_mlp_s* m, const float* x, int B, float* o, cudaStream_t s);
int mlp_max_batch(const ddm_mlp_s* m);

namespace {

constexpr int kLags = DDM_FIT_LAGS;
constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ float warp_sum_bcast(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return __shfl_sync(0xffffffffu, v, 0);
}

// grid: ceil(n / kWarpsPerBlock); block: 32 * kWarpsPerBlock
__global__ void features_kernel(const float* __restrict__ Dr, int n, int N,
                                const int* __restrict__ lag_j, const float* __restrict__ lag_f,
                                float* __restrict__ x, float* __restrict__ p8) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= n) return;
    const float* d = Dr + (size_t)c * N;
    float y[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        const int j = lag_j[i];
        const int j1 = j + 1 < N ? j + 1 : N - 1;
        const float f = lag_f[i];
        y[h] = d[j] * (1.f - f) + d[j1] * f;
    }
    // plateau: mean of samples 56..63 (lanes 24..31, second half)
    float p = warp_sum_bcast(lane >= 24 ? y[1] : 0.f) * 0.125f;
    if (!(p > 0.f)) p = 1.f;
    x[(size_t)c * kLags + lane] = y[0] / p;
    x[(size_t)c * kLags + lane + 32] = y[1] / p;
    if (lane == 0) p8[c] = p;
}

struct Curve {
    float y[2], ll[2];
};

// residuals and Jacobian rows of the two lags of this lane at p = (A, B, ln tau, beta)
__device__ __forceinline__ void model_rows(const Curve& cv, const float p[4], float r[2],
                                           float J[2][4]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float lx = cv.ll[h] - p[2];
        const float s = expf(p[3] * lx);
        const float e = expf(-s);
        r[h] = p[0] * (1.f - e) + p[1] - cv.y[h];
        J[h][0] = 1.f - e;
        J[h][1] = 1.f;
        J[h][2] = -p[0] * p[3] * s * e;
        J[h][3] = p[0] * e * s * lx;
    }
}

__device__ __forceinline__ float cost_at(const Curve& cv, const float p[4]) {
    float r[2], J[2][4];
    model_rows(cv, p, r, J);
    return warp_sum_bcast(r[0] * r[0] + r[1] * r[1]);
}

// Solve (H + mu diag H) dp = -g by Cholesky of the Jacobi-scaled matrix
// S (H + mu diag H) S with S = diag(H)^(-1/2) (unit diagonal 1 + mu: better conditioned in
// FP32 when columns of J are nearly collinear); false if not positive definite / finite.
// The factor's pivots are kept as reciprocal square roots, so the dependent chain holds
// multiplications instead of divisions.
__device__ __forceinline__ bool solve4(const float H[10], const float g[4], float mu, float dp[4]) {
    // H packed: 00 10 11 20 21 22 30 31 32 33
    if (!(H[0] > 0.f && H[2] > 0.f && H[5] > 0.f && H[9] > 0.f)) return false;
    const float s0 = rsqrtf(H[0]), s1 = rsqrtf(H[2]), s2 = rsqrtf(H[5]), s3 = rsqrtf(H[9]);
    const float dg = 1.f + mu;
    const float a10 = H[1] * s1 * s0, a20 = H[3] * s2 * s0, a21 = H[4] * s2 * s1;
    const float a30 = H[6] * s3 * s0, a31 = H[7] * s3 * s1, a32 = H[8] * s3 * s2;
    const float b0 = -g[0] * s0, b1 = -g[1] * s1, b2 = -g[2] * s2, b3 = -g[3] * s3;
    const float i00 = rsqrtf(dg);                      // 1 / l00
    const float l10 = a10 * i00, l20 = a20 * i00, l30 = a30 * i00;
    const float d1 = dg - l10 * l10;
    if (!(d1 > 0.f)) return false;
    const float i11 = rsqrtf(d1);
    const float l21 = (a21 - l20 * l10) * i11, l31 = (a31 - l30 * l10) * i11;
    const float d2 = dg - l20 * l20 - l21 * l21;
    if (!(d2 > 0.f)) return false;
    const float i22 = rsqrtf(d2);
    const float l32 = (a32 - l30 * l20 - l31 * l21) * i22;
    const float d3 = dg - l30 * l30 - l31 * l31 - l32 * l32;
    if (!(d3 > 0.f)) return false;
    const float i33 = rsqrtf(d3);
    const float z0 = b0 * i00;
    const float z1 = (b1 - l10 * z0) * i11;
    const float z2 = (b2 - l20 * z0 - l21 * z1) * i22;
    const float z3 = (b3 - l30 * z0 - l31 * z1 - l32 * z2) * i33;
    const float e3 = z3 * i33;
    const float e2 = (z2 - l32 * e3) * i22;
    const float e1 = (z1 - l21 * e2 - l31 * e3) * i11;
    const float e0 = (z0 - l10 * e1 - l20 * e2 - l30 * e3) * i00;
    dp[0] = e0 * s0;
    dp[1] = e1 * s1;
    dp[2] = e2 * s2;
    dp[3] = e3 * s3;
    return isfinite(dp[0]) && isfinite(dp[1]) && isfinite(dp[2]) && isfinite(dp[3]);
}

// One damped trial at mu: pn = p + dp(mu) (beta clamped) with its residuals, Jacobian and
// cost; true if it lowers the cost.
struct Trial {
    float p[4], r[2], J[2][4], cost;
};

__device__ __forceinline__ bool lm_trial(const Curve& cv, const float p[4], const float H[10],
                                         const float g[4], float mu, float cost, Trial& t) {
    float dp[4];
    if (!solve4(H, g, mu, dp)) return false;
#pragma unroll
    for (int a = 0; a < 4; ++a) t.p[a] = p[a] + dp[a];
    t.p[3] = fminf(fmaxf(t.p[3], 0.05f), 3.f);
    model_rows(cv, t.p, t.r, t.J);
    t.cost = warp_sum_bcast(t.r[0] * t.r[0] + t.r[1] * t.r[1]);
    return isfinite(t.cost) && t.cost < cost;
}

constexpr int kTrials = 4;   // damping values tried side by side: one per warp of a curve's block

// what a warp's trial leaves for the other warps of the block
struct TrialShare {
    float p[kTrials][4];
    float cost[kTrials];
    int ok[kTrials];
    float rj[kTrials][32][10];   // per lane: r[2], J[2][4]
};

// LM from p (in/out); returns iterations, sets cost and flags.  Marquardt's rule: after a
// rejected step mu grows tenfold and the step is solved again, until a step lowers the
// cost or mu exceeds 1e12.  The kTrials warps of the block hold the same curve and compute
// the same normal equations; each round warp w tries the w-th of the consecutive values
// mu, 10 mu, ... and the first that lowers the cost is taken by all: the same trial the
// one-at-a-time loop accepts, with the same arithmetic, in fewer dependent rounds (the
// last iteration of a converged fit rejects every value up to 1e12).  The accepted
// trial's residuals and Jacobian serve the next iteration.  Block-uniform control flow.
__device__ int lm(const Curve& cv, float p[4], float& cost, int& flags, TrialShare& sh) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float r[2], J[2][4];
    model_rows(cv, p, r, J);
    cost = warp_sum_bcast(r[0] * r[0] + r[1] * r[1]);
    if (!isfinite(cost)) {
        flags = DDM_FIT_NONFINITE;
        return 0;
    }
    float mu = 1e-3f;
    flags = DDM_FIT_MAXITER;
    int it = 0;
    while (it < 100) {
        ++it;
        float H[10], g[4];
        {
            int k = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
#pragma unroll
                for (int b = 0; b <= a; ++b) H[k++] = warp_sum_bcast(J[0][a] * J[0][b] + J[1][a] * J[1][b]);
                g[a] = warp_sum_bcast(J[0][a] * r[0] + J[1][a] * r[1]);
            }
        }
        bool accepted = false, first_try = false, first_round = true;
        float dec = 0.f;
        // the first value is always tried; later ones only while mu <= 1e12
        while (!accepted && (first_round || !(mu > 1e12f))) {
            float mus[kTrials];
            mus[0] = mu;
#pragma unroll
            for (int k = 1; k < kTrials; ++k) mus[k] = mus[k - 1] * 10.f;
            float mw = mus[0];
#pragma unroll
            for (int k = 1; k < kTrials; ++k)
                if (w == k) mw = mus[k];
            const bool tried = (w == 0 && first_round) || !(mw > 1e12f);
            Trial t;
            const bool ok = tried && lm_trial(cv, p, H, g, mw, cost, t);
            if (ok) {
                if (lane == 0) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) sh.p[w][a] = t.p[a];
                    sh.cost[w] = t.cost;
                }
                sh.rj[w][lane][0] = t.r[0];
                sh.rj[w][lane][1] = t.r[1];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    sh.rj[w][lane][2 + a] = t.J[0][a];
                    sh.rj[w][lane][6 + a] = t.J[1][a];
                }
            }
            if (lane == 0) sh.ok[w] = ok ? 1 : 0;
            __syncthreads();
            int acc = -1;
#pragma unroll
            for (int k = kTrials - 1; k >= 0; --k)
                if (sh.ok[k]) acc = k;
            if (acc >= 0) {
                accepted = true;
                first_try = first_round && acc == 0;
#pragma unroll
                for (int k = 0; k < kTrials; ++k)
                    if (k == acc) mu = mus[k];
                const float ca = sh.cost[acc];
                dec = cost - ca;
                cost = ca;
#pragma unroll
                for (int a = 0; a < 4; ++a) p[a] = sh.p[acc][a];
                r[0] = sh.rj[acc][lane][0];
                r[1] = sh.rj[acc][lane][1];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    J[0][a] = sh.rj[acc][lane][2 + a];
                    J[1][a] = sh.rj[acc][lane][6 + a];
                }
            } else {
                mu = mus[kTrials - 1] * 10.f;
            }
            first_round = false;
            __syncthreads();   // shared slots read before the next round writes them
        }
        if (!accepted) {
            flags = DDM_FIT_CONVERGED;
            break;
        }
        mu = fmaxf(mu * 0.1f, 1e-12f);
        if (first_try && dec <= 1e-6f * cost) {
            flags = DDM_FIT_CONVERGED;
            break;
        }
    }
    return it;
}

__device__ void heuristic_seed(const Curve& cv, int lane, float p[4]) {
    const float target = 1.f - expf(-1.f);           // plateau of a normalised curve is 1
    const unsigned b0 = __ballot_sync(0xffffffffu, cv.y[0] >= target);
    const unsigned b1 = __ballot_sync(0xffffffffu, cv.y[1] >= target);
    int k = -1;
    if (b0) k = __ffs(b0) - 1;
    else if (b1) k = 32 + __ffs(b1) - 1;
    float ltau;
    const float ll_last = __shfl_sync(0xffffffffu, cv.ll[1], 31);
    const float ll_first = __shfl_sync(0xffffffffu, cv.ll[0], 0);
    if (k < 0) {
        ltau = ll_last;
    } else if (k == 0) {
        ltau = ll_first - logf(2.f);
    } else {
        const int km = k - 1;
        const float yk = __shfl_sync(0xffffffffu, k < 32 ? cv.y[0] : cv.y[1], k & 31);
        const float ykm = __shfl_sync(0xffffffffu, km < 32 ? cv.y[0] : cv.y[1], km & 31);
        const float llk = __shfl_sync(0xffffffffu, k < 32 ? cv.ll[0] : cv.ll[1], k & 31);
        const float llkm = __shfl_sync(0xffffffffu, km < 32 ? cv.ll[0] : cv.ll[1], km & 31);
        const float w = (yk != ykm) ? (target - ykm) / (yk - ykm) : 0.f;
        ltau = llkm + w * (llk - llkm);
    }
    (void)lane;
    p[0] = 1.f;
    p[1] = 0.f;
    p[2] = ltau;
    p[3] = 1.f;
}

// grid: n (one curve per block); block: 32 * kTrials
__global__ void __launch_bounds__(32 * kTrials) lm_kernel(const float* __restrict__ x, const float* __restrict__ p8,
                          const float* __restrict__ mlp_o, int n, int mode,
                          const float* __restrict__ lag_ll, float* __restrict__ params,
                          float* __restrict__ cost_out, int* __restrict__ iters_out,
                          int* __restrict__ flags_out) {
    __shared__ TrialShare sh;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x;
    if (c >= n) return;
    Curve cv;
    cv.y[0] = x[(size_t)c * kLags + lane];
    cv.y[1] = x[(size_t)c * kLags + lane + 32];
    cv.ll[0] = lag_ll[lane];
    cv.ll[1] = lag_ll[lane + 32];
    const float P8 = p8[c];
    float p[4], cost = 0.f;
    int flags = 0, it = 0;
    if (mode == DDM_FIT_LM) {
        heuristic_seed(cv, lane, p);
        it = lm(cv, p, cost, flags, sh);
    } else {
        const float o0 = mlp_o[(size_t)c * 4 + 0], o1 = mlp_o[(size_t)c * 4 + 1];
        const float o2 = mlp_o[(size_t)c * 4 + 2], o3 = mlp_o[(size_t)c * 4 + 3];
        const float A = expf(o0);
        p[0] = A;
        p[1] = A * o3;
        p[2] = o1;
        p[3] = 0.3f + 0.9f / (1.f + expf(-o2));
        cost = cost_at(cv, p);
        if (mode == DDM_FIT_MLP) {
            flags = DDM_FIT_MLP_ACCEPTED | (isfinite(cost) ? 0 : DDM_FIT_NONFINITE);
        } else if (isfinite(cost) && sqrtf(cost / (float)kLags) <= 1e-2f * fabsf(A)) {
            flags = DDM_FIT_CONVERGED | DDM_FIT_MLP_ACCEPTED;
        } else {
            // LM from the lower-cost seed: the network's or the heuristic one (a network
            // trained on another distribution then costs nothing, a good one saves iterations)
            float q[4] = {p[0], p[1], p[2], p[3]};
            float h[4];
            heuristic_seed(cv, lane, h);
            const bool from_heuristic = !(cost <= cost_at(cv, h));
            if (from_heuristic) {
#pragma unroll
                for (int a = 0; a < 4; ++a) q[a] = h[a];
            }
            it = lm(cv, q, cost, flags, sh);
            if ((flags & DDM_FIT_NONFINITE) && !from_heuristic) {
                heuristic_seed(cv, lane, q);
                it += lm(cv, q, cost, flags, sh);
                flags |= DDM_FIT_FALLBACK;
            }
            if (from_heuristic) flags |= DDM_FIT_SEED_HEURISTIC;
#pragma unroll
            for (int a = 0; a < 4; ++a) p[a] = q[a];
        }
    }
    if (threadIdx.x == 0) {
        params[(size_t)c * 4 + 0] = p[0] * P8;
        params[(size_t)c * 4 + 1] = expf(p[2]);
        params[(size_t)c * 4 + 2] = p[3];
        params[(size_t)c * 4 + 3] = p[1] * P8;
        if (cost_out) cost_out[c] = cost * P8 * P8;
        if (iters_out) iters_out[c] = it;
        if (flags_out) flags_out[c] = flags;
    }
}

}  // namespace

ddm_status make_fit_tables(ddm_plan_s* p) {
    const int N = p->d.N;
    if (N < 2) return DDM_OK;
    std::vector<int> j(kLags);
    std::vector<float> f(kLags), ll(kLags);
    for (int i = 0; i < kLags; ++i) {
        const double lam = std::exp((double)i * std::log((double)(N - 1)) / (double)(kLags - 1));
        int jj = (int)std::floor(lam);
        if (jj > N - 1) jj = N - 1;
        j[i] = jj;
        f[i] = (float)(lam - (double)jj);
        ll[i] = (float)std::log(lam);
    }
    if (cudaMalloc(&p->lag_j, sizeof(int) * kLags) != cudaSuccess ||
        cudaMalloc(&p->lag_f, sizeof(float) * kLags) != cudaSuccess ||
        cudaMalloc(&p->lag_ll, sizeof(float) * kLags) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_OOM;
    }
    if (cudaMemcpy(p->lag_j, j.data(), sizeof(int) * kLags, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->lag_f, f.data(), sizeof(float) * kLags, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->lag_ll, ll.data(), sizeof(float) * kLags, cudaMemcpyHostToDevice) != cudaSuccess)
        return DDM_ERR_CUDA;
    return DDM_OK;
}

ddm_status launch_features(const ddm_plan_s* p, const float* Dr, int n, float* x, float* p8,
                           cudaStream_t s) {
    const int blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
    features_kernel<<<blocks, 32 * kWarpsPerBlock, 0, s>>>(Dr, n, p->d.N, p->lag_j, p->lag_f, x, p8);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

ddm_status launch_fit(ddm_plan_s* p, const float* Dr, int n, int mode, const ddm_mlp_s* mlp,
                      float* params, float* cost, int* iters, int* flags, cudaStream_t s) {
    // scratch: x [n][64], p8 [n], o [n][4]
    const size_t need = (size_t)n * (kLags + 1 + 4) * sizeof(float);
    if (p->fit_scratch_bytes < need) {
        if (p->fit_scratch) cudaFree(p->fit_scratch);
        p->fit_scratch = nullptr;
        p->fit_scratch_bytes = 0;
        if (cudaMalloc(&p->fit_scratch, need) != cudaSuccess) {
            cudaGetLastError();
            return DDM_ERR_OOM;
        }
        p->fit_scratch_bytes = need;
    }
    float* x = p->fit_scratch;
    float* p8 = x + (size_t)n * kLags;
    float* o = p8 + n;
    ddm_status st = launch_features(p, Dr, n, x, p8, s);
    if (st != DDM_OK) return st;
    if (mode != DDM_FIT_LM) {
        const int mb = mlp_max_batch(mlp);
        for (int c0 = 0; c0 < n; c0 += mb) {
            const int b = (n - c0) < mb ? (n - c0) : mb;
            st = mlp_forward_raw(mlp, x + (size_t)c0 * kLags, b, o + (size_t)c0 * 4, s);
            if (st != DDM_OK) return st;
        }
    }
    lm_kernel<<<n, 32 * kTrials, 0, s>>>(x, p8, o, n, mode, p->lag_ll, params, cost, iters, flags);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace ddm

extern "C" {

ddm_status ddm_fit_features(ddm_plan p, const float* Dr, int n_curves, float* x, float* p8,
                            void* stream) {
    if (!p || !Dr || !x || !p8 || n_curves < 1) return DDM_ERR_INVALID_ARG;
    if (p->d.N < 2 || !p->lag_j) return DDM_ERR_INVALID_ARG;
    return ddm::launch_features(p, Dr, n_curves, x, p8, (cudaStream_t)stream);
}

ddm_status ddm_fit(ddm_plan p, const float* Dr, int n_curves, int mode, ddm_mlp mlp, float* params,
                   float* cost, int* iters, int* flags, void* stream) {
    if (!p || !Dr || !params || n_curves < 1) return DDM_ERR_INVALID_ARG;
    if (mode != DDM_FIT_LM && mode != DDM_FIT_MLP && mode != DDM_FIT_MLP_LM) return DDM_ERR_INVALID_ARG;
    if (mode != DDM_FIT_LM && !mlp) return DDM_ERR_INVALID_ARG;
    if (p->d.N < 2 || !p->lag_j) return DDM_ERR_INVALID_ARG;
    return ddm::launch_fit(p, Dr, n_curves, mode, mlp, params, cost, iters, flags, (cudaStream_t)stream);
}

}  // extern "C"
