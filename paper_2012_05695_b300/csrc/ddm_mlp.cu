// The fit seed network: MLP 64 -> 128 -> 128 -> 128 -> 4, GELU (erf form) on the hidden
// layers, trained with Adam.  Not in the paper: it seeds the Levenberg-Marquardt fit of
// D(|q|, dt) (ddm_fit.cu), which has the final say.
//
// Precision: FP32 master weights, gradients and Adam moments; the weight matrices are
// used rounded to bfloat16 (a transposed bf16 copy, rebuilt after every Adam step);
// biases, activations and every accumulation are FP32.
//
// One CTA handles a chunk of kSB samples with all bf16 weights resident in shared memory
// (83 KB): forward, and for training the backward pass and the chunk's weight-gradient
// partials.  A second kernel sums the partials over chunks in chunk order (fixed order:
// bitwise reproducible), a third applies Adam.  The network is tiny (0.34 GFLOP per batch
// of 4096): CUDA cores, not tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "ddm_internal.h"

namespace ddm {
namespace {

constexpr int kIn = 64, kHid = 128, kOut = 4;
constexpr int kSB = 32;                       // samples per CTA
constexpr int kThreads = 128;
// flat FP32 parameter layout: per layer W [out][in] then b [out]
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + kHid * kIn;
constexpr int OFF_W2 = OFF_B1 + kHid, OFF_B2 = OFF_W2 + kHid * kHid;
constexpr int OFF_W3 = OFF_B2 + kHid, OFF_B3 = OFF_W3 + kHid * kHid;
constexpr int OFF_W4 = OFF_B3 + kHid, OFF_B4 = OFF_W4 + kOut * kHid;
constexpr int NPARAM = OFF_B4 + kOut;
static_assert(NPARAM == DDM_MLP_PARAMS, "parameter count");
// bf16 transposed weights: Wt [in][out]
constexpr int T1 = 0, T2 = T1 + kIn * kHid, T3 = T2 + kHid * kHid, T4 = T3 + kHid * kHid;
constexpr int NWT = T4 + kHid * kOut;
constexpr int NBIAS = 3 * kHid + kOut;

constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kInvSqrt2Pi = 0.39894228040143268f;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * kInvSqrt2)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * kInvSqrt2)) + z * expf(-0.5f * z * z) * kInvSqrt2Pi;
}

struct Smem {
    __nv_bfloat16 wt[NWT];
    float bias[NBIAS];
    float x[kSB][kIn];
    float z1[kSB][kHid], h1[kSB][kHid];
    float z2[kSB][kHid], h2[kSB][kHid];
    float z3[kSB][kHid], h3[kSB][kHid];
    float o[kSB][kOut];
    float d4[kSB][kOut];
    float lsum[kThreads];
};

// z[s][j] = b[j] + sum_k in[s][k] Wt[k][j] for the chunk's samples; thread j, all s.
template <int K>
__device__ __forceinline__ void dense_hidden(const float (*in)[K], const __nv_bfloat16* Wt,
                                             const float* b, float (*z)[kHid], float (*h)[kHid],
                                             int ns) {
    const int j = threadIdx.x;
    float acc[kSB];
#pragma unroll
    for (int s = 0; s < kSB; ++s) acc[s] = b[j];
    for (int k = 0; k < K; k += 4) {
        const float w0 = __bfloat162float(Wt[(k + 0) * kHid + j]);
        const float w1 = __bfloat162float(Wt[(k + 1) * kHid + j]);
        const float w2 = __bfloat162float(Wt[(k + 2) * kHid + j]);
        const float w3 = __bfloat162float(Wt[(k + 3) * kHid + j]);
#pragma unroll
        for (int s = 0; s < kSB; ++s) {
            const float4 a = *reinterpret_cast<const float4*>(&in[s][k]);
            acc[s] = fmaf(a.x, w0, acc[s]);
            acc[s] = fmaf(a.y, w1, acc[s]);
            acc[s] = fmaf(a.z, w2, acc[s]);
            acc[s] = fmaf(a.w, w3, acc[s]);
        }
    }
#pragma unroll
    for (int s = 0; s < kSB; ++s) {
        z[s][j] = acc[s];
        h[s][j] = (s < ns) ? gelu(acc[s]) : 0.f;
    }
}

// dIn[s][i] = (sum_j dOut[s][j] W[j][i]) * gelu'(zIn[s][i]), W[j][i] = Wt[i][j]; thread i.
// Lanes walk j in a rotated order so that their Wt reads fall in different banks.
__device__ __forceinline__ void back_hidden(const float (*dout)[kHid], const __nv_bfloat16* Wt,
                                            float (*zin)[kHid]) {
    const int i = threadIdx.x;
    const int lane = i & 31;
    float acc[kSB];
#pragma unroll
    for (int s = 0; s < kSB; ++s) acc[s] = 0.f;
    for (int jj = 0; jj < kHid; ++jj) {
        const int j = (jj + lane) & (kHid - 1);
        const float w = __bfloat162float(Wt[i * kHid + j]);
#pragma unroll
        for (int s = 0; s < kSB; ++s) acc[s] = fmaf(dout[s][j], w, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < kSB; ++s) zin[s][i] = acc[s] * gelu_grad(zin[s][i]);
}

// partial dW[o][i] = sum_s d[s][o] in[s][i] and db[o] = sum_s d[s][o] over the chunk;
// written in the master layout at part + off_w / off_b.
template <int IN, int OUT>
__device__ __forceinline__ void weight_grad(const float (*d)[OUT], const float (*in)[IN],
                                            float* part, int off_w, int off_b) {
    for (int i = threadIdx.x; i < IN; i += kThreads) {
        for (int o0 = 0; o0 < OUT; o0 += 8) {
            float acc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = 0.f;
#pragma unroll 4
            for (int s = 0; s < kSB; ++s) {
                const float a = in[s][i];
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    if (o0 + r < OUT) acc[r] = fmaf(d[s][o0 + r], a, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (o0 + r < OUT) part[off_w + (o0 + r) * IN + i] = acc[r];
        }
    }
    for (int o = threadIdx.x; o < OUT; o += kThreads) {
        float acc = 0.f;
        for (int s = 0; s < kSB; ++s) acc += d[s][o];
        part[off_b + o] = acc;
    }
}

// grid: ceil(B / kSB); block: kThreads; dynamic smem: sizeof(Smem)
template <bool TRAIN>
__global__ void __launch_bounds__(kThreads)
mlp_chunk_kernel(const float* __restrict__ x, const float* __restrict__ tgt, int B,
                 const float* __restrict__ w, const __nv_bfloat16* __restrict__ wt,
                 float* __restrict__ out, float* __restrict__ partials,
                 float* __restrict__ loss_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * kSB;
    const int ns = min(kSB, B - s0);
    {
        const uint4* src = reinterpret_cast<const uint4*>(wt);
        uint4* dst = reinterpret_cast<uint4*>(sm.wt);
        for (int k = tid; k < NWT / 8; k += kThreads) dst[k] = __ldg(src + k);
    }
    for (int k = tid; k < kHid; k += kThreads) {
        sm.bias[k] = w[OFF_B1 + k];
        sm.bias[kHid + k] = w[OFF_B2 + k];
        sm.bias[2 * kHid + k] = w[OFF_B3 + k];
    }
    if (tid < kOut) sm.bias[3 * kHid + tid] = w[OFF_B4 + tid];
    for (int k = tid; k < kSB * kIn; k += kThreads) {
        const int s = k / kIn, i = k - s * kIn;
        sm.x[s][i] = (s < ns) ? x[(size_t)(s0 + s) * kIn + i] : 0.f;
    }
    __syncthreads();
    dense_hidden<kIn>(sm.x, sm.wt + T1, sm.bias, sm.z1, sm.h1, ns);
    __syncthreads();
    dense_hidden<kHid>(sm.h1, sm.wt + T2, sm.bias + kHid, sm.z2, sm.h2, ns);
    __syncthreads();
    dense_hidden<kHid>(sm.h2, sm.wt + T3, sm.bias + 2 * kHid, sm.z3, sm.h3, ns);
    __syncthreads();
    {   // output layer: thread = (sample, output)
        const int s = tid / kOut, o = tid - s * kOut;
        float acc = sm.bias[3 * kHid + o];
        for (int k = 0; k < kHid; ++k) acc = fmaf(sm.h3[s][k], __bfloat162float(sm.wt[T4 + k * kOut + o]), acc);
        sm.o[s][o] = acc;
        if (!TRAIN && s < ns) out[(size_t)(s0 + s) * kOut + o] = acc;
        if (TRAIN) {
            // loss term and dL/do for this (sample, output); mean over the batch
            float l = 0.f, d = 0.f;
            if (s < ns) {
                const float t = tgt[(size_t)(s0 + s) * kOut + o];
                if (o == 2) {
                    const float sg = 1.f / (1.f + expf(-acc));
                    const float diff = 0.3f + 0.9f * sg - t;
                    l = diff * diff;
                    d = 2.f * diff / (float)B * 0.9f * sg * (1.f - sg);
                } else {
                    const float diff = acc - t;
                    l = diff * diff;
                    d = 2.f * diff / (float)B;
                }
            }
            sm.d4[s][o] = d;
            sm.lsum[tid] = l;
        }
    }
    if constexpr (TRAIN) {
        __syncthreads();
        float* part = partials + (size_t)blockIdx.x * NPARAM;
        if (tid == 0) {
            float l = 0.f;
            for (int k = 0; k < kThreads; ++k) l += sm.lsum[k];
            loss_part[blockIdx.x] = l / (float)B;
        }
        // layer 4: gradients, then delta3 into z3
        weight_grad<kHid, kOut>(sm.d4, sm.h3, part, OFF_W4, OFF_B4);
        {
            const int i = tid;
            float acc[kSB];
#pragma unroll
            for (int s = 0; s < kSB; ++s) {
                float a = 0.f;
#pragma unroll
                for (int o = 0; o < kOut; ++o)
                    a = fmaf(sm.d4[s][o], __bfloat162float(sm.wt[T4 + i * kOut + o]), a);
                acc[s] = a;
            }
#pragma unroll
            for (int s = 0; s < kSB; ++s) sm.z3[s][i] = acc[s] * gelu_grad(sm.z3[s][i]);
        }
        __syncthreads();
        weight_grad<kHid, kHid>(sm.z3, sm.h2, part, OFF_W3, OFF_B3);
        back_hidden(sm.z3, sm.wt + T3, sm.z2);
        __syncthreads();
        weight_grad<kHid, kHid>(sm.z2, sm.h1, part, OFF_W2, OFF_B2);
        back_hidden(sm.z2, sm.wt + T2, sm.z1);
        __syncthreads();
        weight_grad<kIn, kHid>(sm.z1, sm.x, part, OFF_W1, OFF_B1);
    }
}

// grad[p] = sum over chunks in chunk order; loss = sum of chunk losses in order
__global__ void mlp_reduce_kernel(const float* __restrict__ partials, int n_chunks,
                                  float* __restrict__ grad, const float* __restrict__ loss_part,
                                  float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) {
        float acc = 0.f;
        for (int c = 0; c < n_chunks; ++c) acc += partials[(size_t)c * NPARAM + p];
        grad[p] = acc;
    }
    if (p == 0 && loss) {
        float l = 0.f;
        for (int c = 0; c < n_chunks; ++c) l += loss_part[c];
        *loss = l;
    }
}

// index of master parameter p in the transposed bf16 copy, or -1 for a bias
__device__ __forceinline__ int wt_index(int p) {
    if (p < OFF_B1) { const int o = p / kIn, i = p - o * kIn; return T1 + i * kHid + o; }
    if (p < OFF_W2) return -1;
    if (p < OFF_B2) { const int q = p - OFF_W2, o = q / kHid, i = q - o * kHid; return T2 + i * kHid + o; }
    if (p < OFF_W3) return -1;
    if (p < OFF_B3) { const int q = p - OFF_W3, o = q / kHid, i = q - o * kHid; return T3 + i * kHid + o; }
    if (p < OFF_W4) return -1;
    if (p < OFF_B4) { const int q = p - OFF_W4, o = q / kHid, i = q - o * kHid; return T4 + i * kOut + o; }
    return -1;
}

__global__ void bf16_copy_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) {
        const int k = wt_index(p);
        if (k >= 0) wt[k] = __float2bfloat16_rn(w[p]);
    }
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, __nv_bfloat16* __restrict__ wt, float lr,
                            float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float gp = g[p];
    const float mp = 0.9f * m[p] + 0.1f * gp;
    const float vp = 0.999f * v[p] + 0.001f * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float wn = w[p] - lr * (mp * c1) / (sqrtf(vp * c2) + 1e-8f);
    w[p] = wn;
    const int k = wt_index(p);
    if (k >= 0) wt[k] = __float2bfloat16_rn(wn);
}

}  // namespace

ddm_status mlp_forward_raw(const ddm_mlp_s* m, const float* x, int B, float* o, cudaStream_t s);

}  // namespace ddm

struct ddm_mlp_s {
    int max_batch;
    int step;
    float* w;
    float* m;
    float* v;
    float* grad;
    float* partials;
    float* loss_part;
    __nv_bfloat16* wt;
};

namespace ddm {

int mlp_max_batch(const ddm_mlp_s* m) { return m->max_batch; }

ddm_status mlp_forward_raw(const ddm_mlp_s* m, const float* x, int B, float* o, cudaStream_t s) {
    const int chunks = (B + kSB - 1) / kSB;
    auto k = mlp_chunk_kernel<false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    k<<<chunks, kThreads, sizeof(Smem), s>>>(x, nullptr, B, m->w, m->wt, o, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace ddm

using namespace ddm;

namespace {

void free_mlp(ddm_mlp_s* m) {
    if (!m) return;
    cudaFree(m->w);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->partials);
    cudaFree(m->loss_part);
    cudaFree(m->wt);
    delete m;
}

ddm_status run_grad(ddm_mlp_s* m, const float* x, const float* t, int B, float* grad, float* loss,
                    cudaStream_t s) {
    const int chunks = (B + kSB - 1) / kSB;
    auto k = mlp_chunk_kernel<true>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    k<<<chunks, kThreads, sizeof(Smem), s>>>(x, t, B, m->w, m->wt, nullptr, m->partials, m->loss_part);
    if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    mlp_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(m->partials, chunks, grad, m->loss_part, loss);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace

extern "C" {

ddm_status ddm_mlp_create(ddm_mlp* out, int max_batch) {
    if (!out || max_batch < 1 || max_batch > (1 << 22)) return DDM_ERR_INVALID_ARG;
    *out = nullptr;
    ddm_mlp_s* m = new (std::nothrow) ddm_mlp_s();
    if (!m) return DDM_ERR_OOM;
    m->max_batch = max_batch;
    const int chunks = (max_batch + kSB - 1) / kSB;
    bool ok = cudaMalloc(&m->w, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->m, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->v, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->grad, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->partials, sizeof(float) * NPARAM * (size_t)chunks) == cudaSuccess &&
              cudaMalloc(&m->loss_part, sizeof(float) * chunks) == cudaSuccess &&
              cudaMalloc(&m->wt, sizeof(__nv_bfloat16) * NWT) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_mlp(m);
        return DDM_ERR_OOM;
    }
    cudaMemset(m->w, 0, sizeof(float) * NPARAM);
    cudaMemset(m->m, 0, sizeof(float) * NPARAM);
    cudaMemset(m->v, 0, sizeof(float) * NPARAM);
    cudaMemset(m->wt, 0, sizeof(__nv_bfloat16) * NWT);
    *out = m;
    return DDM_OK;
}

ddm_status ddm_mlp_destroy(ddm_mlp m) {
    free_mlp(m);
    return DDM_OK;
}

ddm_status ddm_mlp_set_weights(ddm_mlp m, const float* host_w) {
    if (!m || !host_w) return DDM_ERR_INVALID_ARG;
    if (cudaMemcpy(m->w, host_w, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m, 0, sizeof(float) * NPARAM) != cudaSuccess ||
        cudaMemset(m->v, 0, sizeof(float) * NPARAM) != cudaSuccess)
        return DDM_ERR_CUDA;
    m->step = 0;
    bf16_copy_kernel<<<(NPARAM + 255) / 256, 256>>>(m->w, m->wt);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return DDM_ERR_CUDA;
    return DDM_OK;
}

ddm_status ddm_mlp_get_weights(ddm_mlp m, float* host_w) {
    if (!m || !host_w) return DDM_ERR_INVALID_ARG;
    return cudaMemcpy(host_w, m->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess
               ? DDM_OK : DDM_ERR_CUDA;
}

ddm_status ddm_mlp_get_state(ddm_mlp m, float* host_state) {
    if (!m || !host_state) return DDM_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(host_state, m->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host_state + NPARAM, m->m, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host_state + 2 * NPARAM, m->v, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
        return DDM_ERR_CUDA;
    host_state[3 * NPARAM] = (float)m->step;
    return DDM_OK;
}

ddm_status ddm_mlp_set_state(ddm_mlp m, const float* host_state) {
    if (!m || !host_state) return DDM_ERR_INVALID_ARG;
    const float st = host_state[3 * NPARAM];
    if (!(st >= 0.f && st <= 16777216.f) || st != (float)(int)st) return DDM_ERR_INVALID_ARG;
    if (cudaMemcpy(m->w, host_state, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->m, host_state + NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->v, host_state + 2 * NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
        return DDM_ERR_CUDA;
    m->step = (int)st;
    bf16_copy_kernel<<<(NPARAM + 255) / 256, 256>>>(m->w, m->wt);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return DDM_ERR_CUDA;
    return DDM_OK;
}

ddm_status ddm_mlp_forward(ddm_mlp m, const float* x, int B, float* o, void* stream) {
    if (!m || !x || !o || B < 1 || B > m->max_batch) return DDM_ERR_INVALID_ARG;
    return mlp_forward_raw(m, x, B, o, (cudaStream_t)stream);
}

ddm_status ddm_mlp_grad(ddm_mlp m, const float* x, const float* t, int B, float* grad, float* loss,
                        void* stream) {
    if (!m || !x || !t || !grad || B < 1 || B > m->max_batch) return DDM_ERR_INVALID_ARG;
    return run_grad(m, x, t, B, grad, loss, (cudaStream_t)stream);
}

ddm_status ddm_mlp_train_step(ddm_mlp m, const float* x, const float* t, int B, float lr,
                              float* loss, void* stream) {
    if (!m || !x || !t || B < 1 || B > m->max_batch || !(lr > 0.f)) return DDM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ddm_status st = run_grad(m, x, t, B, m->grad, loss, s);
    if (st != DDM_OK) return st;
    m->step += 1;
    const double c1 = 1.0 / (1.0 - pow(0.9, m->step)), c2 = 1.0 / (1.0 - pow(0.999, m->step));
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(m->w, m->m, m->v, m->grad, m->wt, lr, (float)c1,
                                                   (float)c2);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // extern "C"
