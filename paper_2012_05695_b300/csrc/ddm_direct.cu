// The paper's WITHOUT_FT scheme on the GPU (Sec. 2, the comparison method of Figs. 1 and
// 3): for every wave vector, D(q, m) straight from Eq. 1,
//     D(q, m) = 1/(N - m) sum_{t=0}^{N-1-m} |F(q, t+m) - F(q, t)|^2 ,   m = 1 .. N-1,
// by explicit differences of the stored spectra, O(N^2) per wave vector (D(q, 0) = 0).
// It reads the same [t][q] spectrum as the WITH_FT time kernels and writes the same D, so
// the two schemes are compared on one GPU with identical inputs and outputs.
//
// Layout of the work.  A CTA of 256 threads copies the time sequences of QC consecutive
// stored wave vectors into shared memory (one sequence per group of TPQ = 256 / QC
// threads, padded by one element per R so that lanes R elements apart hit different
// banks).  The lags 1 .. N-1 are cut into blocks of R consecutive lags; a thread owns block
// b together with block nb - 1 - b, so that every thread sums about the same number of
// terms (block b has N - R (b + 1) full time steps, its partner the complement).  For one
// block the R lags share the time index t: g(t) is read once per step and a register
// window holds g(t + m0 .. t + m0 + R - 1), refilled one element per step in a circular
// order fixed at compile time (no register moves), so each step costs two shared loads and
// R complex differences.  The few terms past the last full chunk of R steps (the ragged
// edge of each lag's range) are summed by a plain loop.  Sums are FP32, per lag in time
// order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

constexpr int kDirectThreads = 256;
constexpr int kR = 16;                    // lags per block

struct DirArgs {
    int N;
    int nb;            // lag blocks, even (the last ones may hold lags >= N only)
    int pairs;         // nb / 2
    int QC;            // wave vectors per CTA
    int S;             // padded sequence stride (float2), odd
    int H, Wh, crop, kx0, nk;
    int64_t n_q, q0, q1;
    unsigned* status;
};

// storage index -> public q (the row of D), as in the WITH_FT time kernels: crop = 1 the
// low-frequency store (D rows in stored order), 2 a kx-column range [kx0, kx0 + nk)
__device__ __forceinline__ int64_t direct_public_q(int64_t s, int H, int Wh, int crop, int kx0, int nk) {
    if (crop == 1) return s;
    if (crop == 2) {
        const int64_t main = (int64_t)H * nk;
        if (s < main) {
            const int64_t ky = s / nk;
            return ky * (Wh + 1) + kx0 + (s - ky * nk);
        }
        return (s - main) * (Wh + 1) + Wh;
    }
    const int64_t main = (int64_t)H * Wh;
    if (s < main) {
        const int64_t ky = s / Wh;
        return ky * (Wh + 1) + (s - ky * Wh);
    }
    return (s - main) * (Wh + 1) + Wh;
}

// The accumulators are float2: the squares of the real and imaginary differences are
// summed in the two halves with paired FP32 instructions (sub2, fma2 of ddm_fft.cuh) and
// added when a lag is finished.

// padded shared-memory position of time index e: one gap per R elements
__host__ __device__ __forceinline__ int pidx(int e) { return e + e / kR; }

// Window of one lag block: w[r] = g(m0 + r) (zero past the sequence, for lags that do not
// exist: their block has no full step).
__device__ __forceinline__ void window_load(const float2* __restrict__ g, int N, int m0, float2 (&w)[kR]) {
#pragma unroll
    for (int r = 0; r < kR; ++r) w[r] = (m0 + r <= N) ? g[pidx(m0 + r)] : make_float2(0.f, 0.f);
}

// R steps t .. t + R - 1 of one lag block: acc[r] += |g(t' + m0 + r) - g(t')|^2 (the
// squares of the real and imaginary differences in the two halves of acc[r]).  On entry
// w[k] = g(t + m0 + k); on exit w[k] = g(t + R + m0 + k).  Every index read is <= N when
// t + R <= N - m0 - R + 1 (a full chunk), and g(N) = 0 is in the buffer.
__device__ __forceinline__ void block_chunk(const float2* __restrict__ g, int t, int m0, float2 (&w)[kR],
                                            float2 (&acc)[kR]) {
    // t is a multiple of R and m0 = 1 mod R (m0 = 1 + b R), so the padded positions of
    // t + s and of e0 + s, e0 = t + m0 + R, are the bases plus s (plus the gap at s = R - 1)
    const int gb = t + t / kR;
    const int e0 = t + m0 + kR;
    const int wb = e0 + e0 / kR;
#pragma unroll
    for (int s = 0; s < kR; ++s) {
        const float2 gt = g[gb + s];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const float2 d = sub2(w[(r + s) % kR], gt);
            acc[r] = fma2(d, d, acc[r]);
        }
        w[s] = g[wb + s + (s == kR - 1 ? 1 : 0)];   // = g(t + s + m0 + R): slot s next holds
                                                     // lag 0's sample of step t + R + s
    }
}

// The terms of each lag m0 + r with t in [t0, N - m0 - r) (the ragged edge), then the
// normalisation and the store of the block's lags that exist (m < N).
__device__ __forceinline__ float block_finish(const float2* __restrict__ g, int N, int m0, int t0,
                                              float2 (&acc)[kR], float* __restrict__ drow) {
    float chk = 0.f;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int m = m0 + r;
        if (m >= N) break;
        float a = acc[r].x + acc[r].y;
        for (int t = t0; t < N - m; ++t) {
            const float2 x = g[pidx(t + m)], y = g[pidx(t)];
            const float dx = x.x - y.x, dy = x.y - y.y;
            a = fmaf(dx, dx, fmaf(dy, dy, a));
        }
        const float d = a / (float)(N - m);
        chk = fmaf(d, 0.f, chk);
        drow[m] = d;
        acc[r] = make_float2(0.f, 0.f);
    }
    return chk;
}

// full chunks of R steps that every lag of the block starting at m0 has: t < N - m0 - R + 1
__device__ __forceinline__ int full_chunks(int N, int m0) {
    const int T = N - m0 - kR + 1;
    return T > 0 ? T / kR : 0;
}

__global__ void __launch_bounds__(kDirectThreads, 2)
direct_sf_kernel(const float2* __restrict__ spec, float* __restrict__ D, DirArgs a) {
    extern __shared__ float2 ser[];      // [QC][S]
    const int N = a.N, QC = a.QC, S = a.S;
    const int tpq = kDirectThreads / QC;
    const int c = threadIdx.x / tpq, tg = threadIdx.x % tpq;
    const int64_t qb = a.q0 + (int64_t)blockIdx.x * QC;

    // the QC sequences: coalesced reads of the [t][q] rows, zero past q1; g(N) = 0
    for (int k = threadIdx.x; k < (N + 1) * QC; k += kDirectThreads) {
        const int t = k / QC, cc = k % QC;
        const int64_t q = qb + cc;
        float2 v = make_float2(0.f, 0.f);
        if (t < N && q < a.q1) v = spec[(int64_t)t * a.n_q + q];
        ser[cc * S + pidx(t)] = v;
    }
    __syncthreads();

    const int64_t q = qb + c;
    if (q >= a.q1) return;
    const float2* g = ser + c * S;
    float* drow = D + direct_public_q(q, a.H, a.Wh, a.crop, a.kx0, a.nk) * (int64_t)N;
    if (tg == 0) drow[0] = 0.f;
    float chk = 0.f;
    float2 acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = make_float2(0.f, 0.f);
    float2 w[kR];
    for (int pi = tg; pi < a.pairs; pi += tpq) {
        // block b0 = pi, then its partner b1 = nb - 1 - pi, in one loop of K0 + K1 chunks:
        // K0 + K1 is the same for every pair (up to the blocks of lags >= N), so the lanes
        // of a warp stay together; each lane switches blocks at its own k
        const int m00 = 1 + pi * kR, m01 = 1 + (a.nb - 1 - pi) * kR;
        const int K0 = full_chunks(N, m00), K1 = full_chunks(N, m01);
        int side = -1, m0 = 0, Kc = 0, t = 0;
        while (true) {
            if (t == Kc * kR) {                          // this block's full chunks are done
                if (side >= 0) chk += block_finish(g, N, m0, t, acc, drow);
                if (side == 1) break;
                ++side;
                m0 = side ? m01 : m00;
                Kc = side ? K1 : K0;
                t = 0;
                window_load(g, N, m0, w);
                continue;
            }
            block_chunk(g, t, m0, w, acc);
            t += kR;
        }
    }
    if (chk != chk) atomicOr(a.status, 1u);
}

}  // namespace

// WITHOUT_FT D of the plan's stored wave vectors [q0, q1) from a [t][q] spectrum.
ddm_status launch_direct(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s) {
    const int N = p->d.N;
    DirArgs a{};
    a.N = N;
    int nb = (N - 1 + kR - 1) / kR;
    if (nb < 1) nb = 1;
    nb += nb & 1;
    a.nb = nb;
    a.pairs = nb / 2;
    int S = pidx(N) + 2;
    if ((S & 1) == 0) ++S;                                  // odd stride: groups on other banks
    a.S = S;
    // threads per wave vector: enough for every block pair, at most the whole CTA; wave
    // vectors per CTA limited by shared memory (two CTAs per SM up to N = 6000)
    int tpq = 1;
    while (tpq < a.pairs && tpq < kDirectThreads) tpq *= 2;
    int QC = kDirectThreads / tpq;
    const size_t max_smem = 110 * 1024;
    while (QC > 1 && (size_t)QC * S * sizeof(float2) > max_smem) QC /= 2;
    const size_t smem = (size_t)QC * S * sizeof(float2);
    if (smem > 227 * 1024) return DDM_ERR_UNSUPPORTED;
    a.QC = QC;
    a.H = p->d.H;
    a.Wh = p->Wh;
    a.crop = p->kc > 0 ? 1 : (p->nk > 0 ? 2 : 0);
    a.kx0 = p->kx0;
    a.nk = p->nk;
    a.n_q = p->n_q;
    a.q0 = p->q0;
    a.q1 = p->q1;
    a.status = p->dev_status;
    const int64_t nq = p->q1 - p->q0;
    const int64_t grid = (nq + QC - 1) / QC;
    if (grid <= 0) return DDM_OK;
    if (grid > 2147483647LL) return DDM_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(direct_sf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    direct_sf_kernel<<<(unsigned)grid, kDirectThreads, smem, s>>>(spec, D, a);
    if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    return DDM_OK;
}

}  // namespace ddm

extern "C" ddm_status ddm_temporal_sf_direct(ddm_plan p, const float* spectrum, float* D, void* stream) {
    if (!p || !spectrum || !D) return DDM_ERR_INVALID_ARG;
    if (p->d.precision == DDM_PREC_FP64) return DDM_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(spectrum) & 7) != 0 || (reinterpret_cast<uintptr_t>(D) & 3) != 0)
        return DDM_ERR_INVALID_ARG;
    return ddm::launch_direct(p, reinterpret_cast<const float2*>(spectrum), D, (cudaStream_t)stream);
}
