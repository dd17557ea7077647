// Step one's column transform (Sec. 2) as DFT-as-GEMM on the 5th-generation tensor cores:
// the DDM_PREC_TC_TF32X3 tier, for frames of H = 512 rows.
//
// The 512-point DFT down every column factors as 512 = 16 x 32 (ky = j1 + 16 j2,
// k = k2 + 32 k1):
//     X[k2 + 32 k1] = sum_{j1} W16^{j1 k1} W512^{j1 k2} sum_{j2} W32^{j2 k2} x[j1 + 16 j2]
// Stage 1 is a GEMM of the data (rows (j1, c): 16 j1 x 16 columns c = 256 rows; K = the 32
// complex j2 as 64 real: re then im) with the real form of the 32-point DFT matrix (N = 64:
// re of the 32 outputs k2, then im); the twiddle W512^{j1 k2} is applied on the CUDA cores
// as the accumulators are read back; stage 2 is a GEMM of rows (k2, c) (512 rows, K = the 16
// complex j1 as 32 real) with the real 16-point DFT matrix (N = 32).
//
// Precision: tcgen05.mma kind::tf32 multiplies 19-bit (TF32) operands with FP32 accumulation,
// about 1e-3 relative on its own.  Each operand is split into two TF32 terms, a = a_hi + a_lo
// (a_hi = a rounded to TF32, a_lo = the remainder rounded to TF32: 22 significant bits), and
// every product is taken as a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped a_lo b_lo is
// ~2^-22 of the product): three MMAs per K step, FP32-class results.
//
// Work: a persistent CTA (one per SM: the operand images take 172 KB of shared memory) takes
// one (frame, 16-column block) at a time: loads and splits the block, stage 1 (2 M-tiles of
// 128 rows, 24 MMAs each), reads back, twiddles and splits, stage 2 (4 M-tiles, 12 MMAs
// each), reads back into an output tile and stores it in place; block 0 unpacks the DC /
// Nyquist column pair the row pass packed into column 0, as the CUDA-core column pass does.
// The MMA waits are bounded (about 2 s); a wait that gives up sets bit 2 of the plan's status
// word, gives the tensor cores one more bounded wait and ends the CTA.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

constexpr int kH = 512, kQC = 16, kThreads = 256;
constexpr int kRows1 = 16 * kQC;       // stage-1 rows (j1, c)
constexpr int kK1 = 64;                // 32 complex j2
constexpr int kN1 = 64;                // 32 complex k2
constexpr int kRows2 = 32 * kQC;       // stage-2 rows (k2, c)
constexpr int kK2 = 32;                // 16 complex j1
constexpr int kN2 = 32;                // 16 complex k1
constexpr uint32_t kTcCols = 256;      // stage-1 accumulators [0, 128), stage-2 [128, 256)
constexpr long long kWaitCap = 4000000000LL;

// shared memory (floats): two data images (hi, lo) of 256 x 64 = 512 x 32 floats, reused by
// both stages and, after stage 2, as the output tile [512][16] complex; the DFT matrix images
// (hi, lo) of both stages; the inter-stage twiddles W512^{j1 k2} [16][32]
constexpr int kImg = kRows1 * kK1;                      // 16384 floats = 64 KB
constexpr int kB1 = kN1 * kK1, kB2 = kN2 * kK2;
constexpr size_t OFF_A_HI = 0;
constexpr size_t OFF_A_LO = OFF_A_HI + (size_t)kImg * 4;
constexpr size_t OFF_B1_HI = OFF_A_LO + (size_t)kImg * 4;
constexpr size_t OFF_B1_LO = OFF_B1_HI + (size_t)kB1 * 4;
constexpr size_t OFF_B2_HI = OFF_B1_LO + (size_t)kB1 * 4;
constexpr size_t OFF_B2_LO = OFF_B2_HI + (size_t)kB2 * 4;
constexpr size_t OFF_TW = OFF_B2_LO + (size_t)kB2 * 4;
constexpr size_t SMEM_BYTES = OFF_TW + (size_t)16 * 32 * 8;
static_assert(kRows2 * kK2 == kImg, "both stages' data images have the same size");
static_assert(SMEM_BYTES + 1024 <= 232448, "one CTA per SM");

// Operand images in shared memory: K-major, no swizzle.  A core matrix is 8 rows x 16 bytes
// (4 TF32 of one row per 16-byte line); the core matrices of one 8-row group follow each
// other along K 128 B apart (the descriptor's leading byte offset) and consecutive 8-row
// groups K * 32 B apart (its stride byte offset).  Element (r, k) of an image with K columns:
__host__ __device__ constexpr int tf_at(int r, int k, int K) {
    return (r >> 3) * (K * 8) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// instruction descriptor of tcgen05.mma kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28
constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory matrix descriptor: start, leading and stride byte offsets (16-byte units),
// descriptor version 1 (bits 46-47), base offset 0, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, long long cap = kWaitCap) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
        if (ok) return true;
        if (clock64() - t0 > cap) return false;
    }
}
// 32 consecutive accumulator columns of this warp's 32 TMEM lanes, one lane per thread
__device__ __forceinline__ void ld32(uint32_t taddr, float (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];\n tcgen05.wait::ld.sync.aligned;"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
          "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]),
          "=f"(r[16]), "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]),
          "=f"(r[24]), "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]), "=f"(r[30]), "=f"(r[31])
        : "r"(taddr) : "memory");
}
// a = hi + lo, each exactly representable in TF32 (cvt.rna: low 13 mantissa bits zero)
__device__ __forceinline__ void split_tf32(float a, float& hi, float& lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(a));
    hi = __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(a - hi));
    lo = __uint_as_float(l);
}

struct TcTables {
    const float* b1_hi;      // stage-1 DFT matrix image (N1 x K1), hi and lo
    const float* b1_lo;
    const float* b2_hi;      // stage-2 DFT matrix image (N2 x K2)
    const float* b2_lo;
    const float2* tw;        // W512^{j1 k2}, [j1][k2]
};

__global__ void __launch_bounds__(kThreads, 1)
col_tc_kernel(float2* __restrict__ spec, int Wh, size_t frame_stride, int N, TcTables tb,
              unsigned* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* a_hi = reinterpret_cast<float*>(smem_raw + OFF_A_HI);
    float* a_lo = reinterpret_cast<float*>(smem_raw + OFF_A_LO);
    float* b1_hi = reinterpret_cast<float*>(smem_raw + OFF_B1_HI);
    float* b1_lo = reinterpret_cast<float*>(smem_raw + OFF_B1_LO);
    float* b2_hi = reinterpret_cast<float*>(smem_raw + OFF_B2_HI);
    float* b2_lo = reinterpret_cast<float*>(smem_raw + OFF_B2_LO);
    float2* tw = reinterpret_cast<float2*>(smem_raw + OFF_TW);
    float2* outt = reinterpret_cast<float2*>(smem_raw + OFF_A_HI);   // [ky][c], after stage 2
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(&tmem_slot)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = tid; k < kB1; k += kThreads) {
        b1_hi[k] = tb.b1_hi[k];
        b1_lo[k] = tb.b1_lo[k];
    }
    for (int k = tid; k < kB2; k += kThreads) {
        b2_hi[k] = tb.b2_hi[k];
        b2_lo[k] = tb.b2_lo[k];
    }
    for (int k = tid; k < 512; k += kThreads) tw[k] = tb.tw[k];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    const int quarter = warp & 3, half = warp >> 2;
    uint32_t phase = 0;
    bool failed = false;
    const int nblk = Wh / kQC;
    const int64_t items = (int64_t)nblk * N;

    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int bx = (int)(it % nblk);
        const int t = (int)(it / nblk);
        float2* base = spec + (size_t)t * frame_stride;
        // ---- the block [ky][c] (128-byte rows) into the stage-1 images: row (j1, c), K = j2
        // (real parts) then 32 + j2 (imaginary parts), ky = j1 + 16 j2
#pragma unroll 4
        for (int r = 0; r < (kH * kQC) / kThreads; ++r) {
            const int e = tid + kThreads * r;
            const int ky = e >> 4, c = e & 15;
            const float2 x = base[(size_t)ky * Wh + bx * kQC + c];
            const int j1 = ky & 15, j2 = ky >> 4;
            const int row = j1 * kQC + c;
            float h, l;
            split_tf32(x.x, h, l);
            a_hi[tf_at(row, j2, kK1)] = h;
            a_lo[tf_at(row, j2, kK1)] = l;
            split_tf32(x.y, h, l);
            a_hi[tf_at(row, 32 + j2, kK1)] = h;
            a_lo[tf_at(row, 32 + j2, kK1)] = l;
        }
        proxy_fence();                        // generic-proxy stores -> the tensor cores' reads
        fence_before();
        __syncthreads();
        fence_after();
        // ---- stage 1: two M-tiles of 128 rows, N = 64, K = 64 (8 steps of 8)
        if (tid == 0) {
            constexpr uint32_t id = idesc_tf32(128, kN1);
            const uint32_t sbo = kK1 * 32;
#pragma unroll 1
            for (int m = 0; m < 2; ++m) {
                const float* ah = a_hi + (size_t)(128 * m / 8) * (kK1 * 8);
                const float* al = a_lo + (size_t)(128 * m / 8) * (kK1 * 8);
#pragma unroll 1
                for (int kk = 0; kk < kK1 / 8; ++kk) {
                    const uint64_t bh = sdesc(b1_hi + kk * 64, 128, sbo), bl = sdesc(b1_lo + kk * 64, 128, sbo);
                    const uint64_t dh = sdesc(ah + kk * 64, 128, sbo), dl = sdesc(al + kk * 64, 128, sbo);
                    const uint32_t d = tmem + (uint32_t)(kN1 * m);
                    mma_tf32(d, dh, bh, id, kk != 0);
                    mma_tf32(d, dh, bl, id, 1);
                    mma_tf32(d, dl, bh, id, 1);
                }
            }
            mma_commit(&bar);
        }
        bool ok = bar_wait(&bar, phase);
        phase ^= 1u;
        fence_after();
        if (__syncthreads_or(ok ? 0 : 1)) { failed = true; break; }
        // ---- read back row (j1, c) = 128 half + lane of quarter: Y[k2] (32 re, then 32 im),
        // twiddle by W512^{j1 k2}, split into the stage-2 images: row (k2, c), K = j1, 16 + j1
        {
            const int row = 128 * half + 32 * quarter + lane;
            const int j1 = row / kQC, c = row % kQC;
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(kN1 * half);
            float re[32], im[32];
            ld32(taddr, re);
            ld32(taddr + 32, im);
            __syncthreads();                  // every stage-1 image read is done (MMAs waited)
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) {
                const float2 w = tw[j1 * 32 + k2];
                const float yr = re[k2] * w.x - im[k2] * w.y;
                const float yi = re[k2] * w.y + im[k2] * w.x;
                const int r2 = k2 * kQC + c;
                float h, l;
                split_tf32(yr, h, l);
                a_hi[tf_at(r2, j1, kK2)] = h;
                a_lo[tf_at(r2, j1, kK2)] = l;
                split_tf32(yi, h, l);
                a_hi[tf_at(r2, 16 + j1, kK2)] = h;
                a_lo[tf_at(r2, 16 + j1, kK2)] = l;
            }
        }
        proxy_fence();
        fence_before();
        __syncthreads();
        fence_after();
        // ---- stage 2: four M-tiles of 128 rows, N = 32, K = 32 (4 steps of 8)
        if (tid == 0) {
            constexpr uint32_t id = idesc_tf32(128, kN2);
            const uint32_t sbo = kK2 * 32;
#pragma unroll 1
            for (int m = 0; m < 4; ++m) {
                const float* ah = a_hi + (size_t)(128 * m / 8) * (kK2 * 8);
                const float* al = a_lo + (size_t)(128 * m / 8) * (kK2 * 8);
#pragma unroll 1
                for (int kk = 0; kk < kK2 / 8; ++kk) {
                    const uint64_t bh = sdesc(b2_hi + kk * 64, 128, sbo), bl = sdesc(b2_lo + kk * 64, 128, sbo);
                    const uint64_t dh = sdesc(ah + kk * 64, 128, sbo), dl = sdesc(al + kk * 64, 128, sbo);
                    const uint32_t d = tmem + 128u + (uint32_t)(kN2 * m);
                    mma_tf32(d, dh, bh, id, kk != 0);
                    mma_tf32(d, dh, bl, id, 1);
                    mma_tf32(d, dl, bh, id, 1);
                }
            }
            mma_commit(&bar);
        }
        ok = bar_wait(&bar, phase);
        phase ^= 1u;
        fence_after();
        if (__syncthreads_or(ok ? 0 : 1)) { failed = true; break; }
        // ---- read back: warp pair `half` takes M-tiles 2 half and 2 half + 1; row (k2, c)
        // holds X[k2 + 32 k1], k1 < 16 (16 re then 16 im) -> the output tile [ky][c]
        {
            float2 xv[2][16];
            int rows[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int m = 2 * half + s;
                rows[s] = 128 * m + 32 * quarter + lane;
                float r32[32];
                ld32(tmem + ((uint32_t)(32 * quarter) << 16) + 128u + (uint32_t)(kN2 * m), r32);
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) xv[s][k1] = make_float2(r32[k1], r32[16 + k1]);
            }
            __syncthreads();                  // the stage-2 images are no longer read
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int k2 = rows[s] / kQC, c = rows[s] % kQC;
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) outt[(k2 + 32 * k1) * kQC + c] = xv[s][k1];
            }
        }
        __syncthreads();
        // ---- the output tile back in place (128-byte rows); block 0 unpacks column 0 into
        // the DC column (kx = 0) and the Nyquist column (kx = W/2, after the main block)
#pragma unroll 4
        for (int r = 0; r < (kH * kQC) / kThreads; ++r) {
            const int e = tid + kThreads * r;
            const int ky = e >> 4, c = e & 15;
            const float2 z = outt[ky * kQC + c];
            if (bx == 0 && c == 0) {
                const float2 zr = outt[((kH - ky) & (kH - 1)) * kQC];
                base[(size_t)ky * Wh] = make_float2(0.5f * (z.x + zr.x), 0.5f * (z.y - zr.y));
                base[(size_t)kH * Wh + ky] = make_float2(0.5f * (z.y + zr.y), 0.5f * (zr.x - z.x));
            } else {
                base[(size_t)ky * Wh + bx * kQC + c] = z;
            }
        }
        fence_before();
        __syncthreads();                      // output tile and accumulators free
        fence_after();
    }
    if (failed) {
        if (tid == 0) atomicOr(status, 2u);
        (void)bar_wait(&bar, phase);          // a last bounded chance for the tensor cores
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols)
                     : "memory");
}

}  // namespace

// Tables of the tensor-core column pass (plan creation, double precision): the real forms
// of the 32- and 16-point DFT matrices as K-major TF32 images (hi and lo terms), and the
// twiddles W512^{j1 k2}.  Returns the host images concatenated: b1_hi, b1_lo, b2_hi, b2_lo
// (floats), then the twiddles (float2 as two floats).
void tc_column_tables(float* out) {
    auto tf32 = [](double v) -> float {   // round to nearest TF32 (ties away): 10 fraction bits
        float f = (float)v;
        uint32_t u;
        memcpy(&u, &f, 4);
        u = (u + 0x1000u) & ~0x1FFFu;
        float r;
        memcpy(&r, &u, 4);
        return r;
    };
    auto fill = [&](int n, int K, float* hi, float* lo) {   // n-point DFT, rows = outputs
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j) {
                const cx_cs cs = cx_cossin_frac((long)k * j % n, n);
                const double wr = cs.c, wi = -cs.s;            // exp(-2 pi i k j / n)
                const double vals[4][3] = {{(double)k, (double)j, wr},
                                           {(double)k, (double)(n + j), -wi},
                                           {(double)(n + k), (double)j, wi},
                                           {(double)(n + k), (double)(n + j), wr}};
                for (const auto& v : vals) {
                    const int r = (int)v[0], c = (int)v[1];
                    const float h = tf32(v[2]);
                    hi[tf_at(r, c, K)] = h;
                    lo[tf_at(r, c, K)] = tf32(v[2] - (double)h);
                }
            }
    };
    float* b1h = out;
    float* b1l = b1h + kB1;
    float* b2h = b1l + kB1;
    float* b2l = b2h + kB2;
    fill(32, kK1, b1h, b1l);
    fill(16, kK2, b2h, b2l);
    float* twf = b2l + kB2;
    for (int j1 = 0; j1 < 16; ++j1)
        for (int k2 = 0; k2 < 32; ++k2) {
            const cx_cs cs = cx_cossin_frac((long)j1 * k2 % 512, 512);
            twf[2 * (j1 * 32 + k2)] = (float)cs.c;
            twf[2 * (j1 * 32 + k2) + 1] = (float)-cs.s;
        }
}
size_t tc_column_table_floats() { return (size_t)2 * kB1 + 2 * kB2 + 2 * 512; }

bool tc_columns_supported(const ddm_plan_desc& d) {
    const bool pow2w = d.W >= 32 && d.W <= 1024 && (d.W & (d.W - 1)) == 0;
    return d.H == kH && pow2w && d.kmax == 0 && d.kx_begin == 0 && d.kx_end == 0 &&
           d.spatial_path == DDM_SPATIAL_TWO_PASS;
}

cudaError_t launch_cols_tc(const ddm_plan_s* p, float2* spec, cudaStream_t s) {
    const float* t = p->tc_tables;
    TcTables tb;
    tb.b1_hi = t;
    tb.b1_lo = tb.b1_hi + kB1;
    tb.b2_hi = tb.b1_lo + kB1;
    tb.b2_lo = tb.b2_hi + kB2;
    tb.tw = reinterpret_cast<const float2*>(tb.b2_lo + kB2);
    cudaError_t e = cudaFuncSetAttribute(col_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int64_t items = (int64_t)(p->Wh / kQC) * p->d.N;
    const int grid = (int)(items < p->n_sm ? items : p->n_sm);
    col_tc_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(spec, p->Wh, (size_t)p->n_q, p->d.N, tb, p->dev_status);
    return cudaGetLastError();
}

}  // namespace ddm
