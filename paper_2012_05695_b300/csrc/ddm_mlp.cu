// The fit seed network: MLP 64 -> 128 -> 128 -> 128 -> 4, GELU (erf form) on the hidden
// layers, trained with Adam.  Not in the paper: it seeds the Levenberg-Marquardt fit of
// D(|q|, dt) (ddm_fit.cu), which has the final say.
//
// Precision: FP32 master weights, gradients and Adam moments; the weight matrices are
// used rounded to bfloat16 (a transposed bf16 copy, rebuilt after every Adam step);
// biases, activations and every accumulation are FP32.
//
// Inference (ddm_mlp_forward, the fit's seeds) runs the three hidden layers on the
// 5th-generation tensor cores: tcgen05.mma (kind::f16, bf16 operands, FP32 accumulators in
// tensor memory), one CTA per 128 samples.  Each FP32 activation enters as three bf16 terms
// whose sum is exactly the activation (8 + 8 + 8 significand bits; for |h| >= 2^-103), so
// that every product is exact and the result is the FP32-activation network's to within FP32
// accumulation order.
//
// Training: one CTA handles a chunk of kSB samples with all bf16 weights resident in shared
// memory (83 KB): forward, backward pass and the chunk's weight-gradient partials on CUDA
// cores.  A second kernel sums the partials over chunks in chunk order (fixed order: bitwise
// reproducible), a third applies Adam.
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

// ---------------------------------------------------------------- tensor-core forward
// Operand images in shared memory: K-major, no swizzle.  A "core matrix" is 8 rows x 16 bytes
// (8 bf16 of one row per 16-byte line); the K/8 core matrices of one 8-row group lie 128 B
// apart (the descriptor's leading byte offset) and consecutive row groups K * 16 B apart (its
// stride byte offset).  Element (r, k) of an image with K columns:
__host__ __device__ constexpr int img_at(int r, int k, int K) {
    return (r >> 3) * (K * 8) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}
constexpr int kTM = 128;                                   // samples per CTA = MMA M = TMEM lanes
constexpr int kTcThreads = 512;                            // 4 lane quarters x 4 column groups
constexpr int kColGroups = kTcThreads / kTM;               // 32-column slices of an accumulator row
constexpr int IMG1 = 0, IMG2 = IMG1 + kHid * kIn, IMG3 = IMG2 + kHid * kHid;
constexpr int NIMG = IMG3 + kHid * kHid;                   // W1, W2, W3 as [out][in] images
// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B bf16 (bits
// 7-9 and 10-12 = 1), both K-major, N = 128 (bits 17-22 = N / 8), M = 128 (bits 24-28 = M / 16)
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                                ((uint32_t)(kTM >> 4) << 24);
constexpr uint32_t kTmemCols = 128;                        // one 128 x 128 FP32 accumulator
constexpr long long kMmaWaitCap = 4000000000LL;            // ~2 s of SM clocks

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: start, leading and stride byte offsets (16-byte units),
// descriptor version 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((smem_addr(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(kIdescBf16), "r"(accumulate) : "memory");
}
// arrive on the barrier once every tcgen05 operation this thread issued so far has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait_bounded(uint64_t* bar, uint32_t parity, long long cap = kMmaWaitCap) {
    const long long t0 = clock64();
    while (!bar_try_wait(bar, parity))
        if (clock64() - t0 > cap) return false;
    return true;
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_addr(slot)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t tmem) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
}
// An MMA batch that has not completed within the bound (block-uniform call): report it in
// the status word (bit 1), give the tensor cores one more bounded wait, then every thread
// is done with tensor memory and the caller may release it.
__device__ __forceinline__ void mma_give_up(unsigned* status, uint64_t* bar, uint32_t parity, long long cap) {
    if (threadIdx.x == 0) atomicOr(status, 2u);
    (void)bar_wait_bounded(bar, parity, cap);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
// 32 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes (one lane per
// thread); the wait sits in the same statement, so no use of r can precede it
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32]) {
    uint32_t u[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];\n tcgen05.wait::ld.sync.aligned;"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
          "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
          "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr) : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = __uint_as_float(u[j]);
}
// h = hi + mid + lo: hi is h with the low 16 bits of its FP32 pattern cleared (a bf16
// value), r = h - hi is exact and holds the remaining 16 significand bits, mid is r cleared
// the same way, and lo = r - mid, also exact, has at most 8 significant bits, so it is a
// bf16 value too whenever it is a normal FP32 number (|h| >= 2^-103; below that the upper
// half of its subnormal pattern drops less than 2^-133).  The upper halves of the three
// patterns are the bf16 terms; eight values of one row go out as one 16-byte line per term.
__device__ __forceinline__ void split_store8(const float (&h)[8], __nv_bfloat16* hi, __nv_bfloat16* mid,
                                             __nv_bfloat16* lo, int at) {
    uint32_t t[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        t[0][j] = __float_as_uint(h[j]) & 0xFFFF0000u;
        const float r = h[j] - __uint_as_float(t[0][j]);
        t[1][j] = __float_as_uint(r) & 0xFFFF0000u;
        t[2][j] = __float_as_uint(r - __uint_as_float(t[1][j]));
    }
    __nv_bfloat16* dst[3] = {hi, mid, lo};
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = __byte_perm(t[u][2 * j], t[u][2 * j + 1], 0x7632);
        *reinterpret_cast<uint4*>(dst[u] + at) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct TcSmem {
    __nv_bfloat16 w[NIMG];                 // 80 KB
    __nv_bfloat16 a[3][kTM * kHid];        // 96 KB: hi, mid, lo terms of the layer input
    float w4[kOut][kHid];                  // bf16-rounded output layer
    float bias[NBIAS];
    float red[kColGroups][kTM][kOut];      // output-layer partial sums per column group
    uint64_t bar;
    uint32_t tmem;
};

// grid: ceil(B / 128); block: 512; dynamic smem: sizeof(TcSmem).  Warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (the quarter a warp may access), i.e. samples s0 + 32 (w % 4) + lane, and
// columns 32 (w / 4) .. + 31 of each accumulator row: bias + GELU there, and the next layer's
// operand terms (or the output layer's partial sums) for those 32 columns.
__global__ void __launch_bounds__(kTcThreads, 1)
mlp_forward_tc_kernel(const float* __restrict__ x, int B, const float* __restrict__ w,
                      const __nv_bfloat16* __restrict__ wt, const __nv_bfloat16* __restrict__ wimg,
                      float* __restrict__ out, unsigned* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem& sm = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cg = warp >> 2;
    const int srow = 32 * quarter + lane;               // this thread's sample (TMEM lane)
    const int s0 = blockIdx.x * kTM;
    if (warp == 0) tmem_alloc(&sm.tmem);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(wimg);
        uint4* dst = reinterpret_cast<uint4*>(sm.w);
#pragma unroll
        for (int k = tid; k < NIMG / 8; k += kTcThreads) dst[k] = __ldg(src + k);
    }
    for (int k = tid; k < kOut * kHid; k += kTcThreads) {
        const int o = k / kHid, i = k - o * kHid;
        sm.w4[o][i] = __bfloat162float(wt[T4 + i * kOut + o]);
    }
    for (int k = tid; k < kHid; k += kTcThreads) {
        sm.bias[k] = w[OFF_B1 + k];
        sm.bias[kHid + k] = w[OFF_B2 + k];
        sm.bias[2 * kHid + k] = w[OFF_B3 + k];
    }
    if (tid < kOut) sm.bias[3 * kHid + tid] = w[OFF_B4 + tid];
    {   // the layer-1 operand (K = 64): thread (sample tid % 128, features 16 (tid / 128) ..
        // + 15); zero past the batch
        const int sl = tid & (kTM - 1), f0 = 16 * (tid >> 7);
        const bool valid = s0 + sl < B;
        const float* xr = x + (size_t)(valid ? s0 + sl : 0) * kIn + f0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = valid ? __ldg(xr + 8 * c + j) : 0.f;
            split_store8(h, sm.a[0], sm.a[1], sm.a[2], img_at(sl, f0 + 8 * c, kIn));
        }
    }
    proxy_fence();                      // generic-proxy stores -> the tensor cores' reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    float o[kOut] = {0.f, 0.f, 0.f, 0.f};
    int failed = -1;                    // layer whose MMA batch did not complete in time
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
        const int K = layer == 0 ? kIn : kHid;
        if (tid == 0) {
            const __nv_bfloat16* wl = sm.w + (layer == 0 ? IMG1 : layer == 1 ? IMG2 : IMG3);
            const uint32_t sbo = (uint32_t)K * 16;
#pragma unroll 1
            for (int kk = 0; kk < K / 16; ++kk) {
                const uint64_t bd = smem_desc(wl + kk * 128, 128, sbo);
#pragma unroll
                for (int u = 0; u < 3; ++u)
                    mma_bf16(tmem, smem_desc(sm.a[u] + kk * 128, 128, sbo), bd, (kk | u) != 0);
            }
            mma_commit(&sm.bar);
        }
        const bool done = bar_wait_bounded(&sm.bar, (uint32_t)(layer & 1));
        tc_fence_after();
        if (__syncthreads_or(done ? 0 : 1)) {
            failed = layer;
            break;
        }
        const float* bl = sm.bias + layer * kHid;
        {
            const int col0 = 32 * cg;
            float r[32];
            tmem_ld32(lane_base + col0, r);
#pragma unroll
            for (int j = 0; j < 32; ++j) r[j] = gelu(r[j] + bl[col0 + j]);
            if (layer < 2) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float h8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h8[j] = r[8 * c + j];
                    split_store8(h8, sm.a[0], sm.a[1], sm.a[2], img_at(srow, col0 + 8 * c, kHid));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
#pragma unroll
                    for (int q = 0; q < kOut; ++q) o[q] = fmaf(r[j], sm.w4[q][col0 + j], o[q]);
            }
        }
        proxy_fence();
        tc_fence_before();
        __syncthreads();                // every accumulator row read, next operand written
        tc_fence_after();
    }
    if (failed < 0) {
#pragma unroll
        for (int q = 0; q < kOut; ++q) sm.red[cg][srow][q] = o[q];
        __syncthreads();
        if (tid < kTM && s0 + tid < B) {
#pragma unroll
            for (int q = 0; q < kOut; ++q) {
                float acc = sm.bias[3 * kHid + q];
#pragma unroll
                for (int g = 0; g < kColGroups; ++g) acc += sm.red[g][tid][q];
                out[(size_t)(s0 + tid) * kOut + q] = acc;
            }
        }
    } else {
        mma_give_up(status, &sm.bar, (uint32_t)(failed & 1), kMmaWaitCap);
    }
    __syncwarp();
    if (warp == 0) tmem_free(tmem);
}

// Test hook for the bounded MMA wait and the give-up path above: one CTA takes tensor memory
// and an MMA barrier as the forward does, waits (bound: cap cycles) on a phase that no commit
// will complete (no MMA is issued), reports through the status word, waits once more and
// releases the tensor memory.
__global__ void __launch_bounds__(128) mlp_wait_selftest_kernel(unsigned* status, long long cap) {
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(&slot);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = slot;
    const bool done = bar_wait_bounded(&bar, 0u, cap);
    if (__syncthreads_or(done ? 0 : 1)) mma_give_up(status, &bar, 0u, cap);
    __syncwarp();
    if (warp == 0) tmem_free(tmem);
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
__global__ void __launch_bounds__(kThreads)
mlp_chunk_kernel(const float* __restrict__ x, const float* __restrict__ tgt, int B,
                 const float* __restrict__ w, const __nv_bfloat16* __restrict__ wt,
                 float* __restrict__ partials, float* __restrict__ loss_part) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
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
        {
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
    {
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

// index of master parameter p in the tensor-core operand images (W1..W3), or -1
__device__ __forceinline__ int img_index(int p) {
    if (p < OFF_B1) { const int o = p / kIn, i = p - o * kIn; return IMG1 + img_at(o, i, kIn); }
    if (p < OFF_W2) return -1;
    if (p < OFF_B2) { const int q = p - OFF_W2, o = q / kHid, i = q - o * kHid; return IMG2 + img_at(o, i, kHid); }
    if (p < OFF_W3) return -1;
    if (p < OFF_B3) { const int q = p - OFF_W3, o = q / kHid, i = q - o * kHid; return IMG3 + img_at(o, i, kHid); }
    return -1;
}

__device__ __forceinline__ void put_bf16(int p, float v, __nv_bfloat16* wt, __nv_bfloat16* wimg) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    const int k = wt_index(p);
    if (k >= 0) wt[k] = b;
    const int g = img_index(p);
    if (g >= 0) wimg[g] = b;
}

__global__ void bf16_copy_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wt,
                                 __nv_bfloat16* __restrict__ wimg) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) put_bf16(p, w[p], wt, wimg);
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, __nv_bfloat16* __restrict__ wt,
                            __nv_bfloat16* __restrict__ wimg, float lr, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float gp = g[p];
    const float mp = 0.9f * m[p] + 0.1f * gp;
    const float vp = 0.999f * v[p] + 0.001f * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float wn = w[p] - lr * (mp * c1) / (sqrtf(vp * c2) + 1e-8f);
    w[p] = wn;
    put_bf16(p, wn, wt, wimg);
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
    __nv_bfloat16* wimg;    // W1..W3 as tensor-core operand images
    unsigned* status;       // bit 1: a bounded wait gave up
};

namespace ddm {

int mlp_max_batch(const ddm_mlp_s* m) { return m->max_batch; }

cudaError_t launch_mlp_wait_selftest(unsigned* status, long long cap_cycles, cudaStream_t s) {
    mlp_wait_selftest_kernel<<<1, 128, 0, s>>>(status, cap_cycles);
    return cudaGetLastError();
}

ddm_status mlp_forward_raw(const ddm_mlp_s* m, const float* x, int B, float* o, cudaStream_t s) {
    auto k = mlp_forward_tc_kernel;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem)) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    k<<<(B + kTM - 1) / kTM, kTcThreads, sizeof(TcSmem), s>>>(x, B, m->w, m->wt, m->wimg, o, m->status);
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
    cudaFree(m->wimg);
    cudaFree(m->status);
    delete m;
}

ddm_status run_grad(ddm_mlp_s* m, const float* x, const float* t, int B, float* grad, float* loss,
                    cudaStream_t s) {
    const int chunks = (B + kSB - 1) / kSB;
    auto k = mlp_chunk_kernel;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    k<<<chunks, kThreads, sizeof(Smem), s>>>(x, t, B, m->w, m->wt, m->partials, m->loss_part);
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
              cudaMalloc(&m->wt, sizeof(__nv_bfloat16) * NWT) == cudaSuccess &&
              cudaMalloc(&m->wimg, sizeof(__nv_bfloat16) * NIMG) == cudaSuccess &&
              cudaMalloc(&m->status, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_mlp(m);
        return DDM_ERR_OOM;
    }
    cudaMemset(m->w, 0, sizeof(float) * NPARAM);
    cudaMemset(m->m, 0, sizeof(float) * NPARAM);
    cudaMemset(m->v, 0, sizeof(float) * NPARAM);
    cudaMemset(m->wt, 0, sizeof(__nv_bfloat16) * NWT);
    cudaMemset(m->wimg, 0, sizeof(__nv_bfloat16) * NIMG);
    cudaMemset(m->status, 0, sizeof(unsigned));
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
    bf16_copy_kernel<<<(NPARAM + 255) / 256, 256>>>(m->w, m->wt, m->wimg);
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
    bf16_copy_kernel<<<(NPARAM + 255) / 256, 256>>>(m->w, m->wt, m->wimg);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return DDM_ERR_CUDA;
    return DDM_OK;
}

ddm_status ddm_mlp_last_device_status(ddm_mlp m, ddm_status* out) {
    if (!m || !out) return DDM_ERR_INVALID_ARG;
    unsigned h = 0;
    if (cudaMemcpy(&h, m->status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(m->status, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    *out = (h & 2u) ? DDM_ERR_TIMEOUT : DDM_OK;
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
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(m->w, m->m, m->v, m->grad, m->wt, m->wimg, lr,
                                                   (float)c1, (float)c2);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // extern "C"
