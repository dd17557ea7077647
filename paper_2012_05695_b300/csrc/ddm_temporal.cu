// Step two of the method (Sec. 2, App. B): the structure function of every time
// sequence F(q, 0..N-1), FP32.
//
// For one wave vector q with time sequence g(t) (t < N, the time mean removed first: D
// depends only on differences, so any constant may be subtracted):
//   power terms (Eqs. B1, B3):  P1(m) = sum_{t < N-m} |g|^2 = S(N-1-m),
//                                P2(m) = sum_{t >= m} |g|^2  = S(N-1) - S(m-1),
//                                S = inclusive prefix sums of |g|^2;
//   cross term (Eq. B4): g zero-padded to M = 2L points, L = 2^ceil(log2 N) (so M is the
//   paper's N_2), transformed, squared in modulus, inverse-transformed:
//     C(m) = (1/M) sum_k |X(k)|^2 e^{+2 pi i k m / M} = sum_t g*(t) g(t + m), m < N;
//   D(m) = (P1(m) + P2(m) - 2 Re C(m)) / (N - m),  D(0) = 0.
// The M-point transform is never formed: its even bins are the L-point DFT of g and its
// odd bins the L-point DFT of g(t) e^{-i pi t / L}.  The inverse of the real power
// spectrum uses one L-point complex transform of Z(j) = |X(2j)|^2 + i |X(2j+1)|^2 and
//     Re C(m) = (1/4L) [ (a + c) + cos(pi m / L) (b + d) + sin(pi m / L) (a - c) ],
// z(m) = a + ib, z(L - m) = c + id, z = unnormalised inverse DFT of Z.
// The last kd lags (N - m <= kd pairs) are taken directly from Eq. 1 by differences
// instead: few terms, and no cancellation against the much larger power sums.
//
// Four kernel families share this arithmetic; each thread holds 32 samples of a transform in
// the cyclic layout (thread i of T holds t = i + T u; fewer below L = 32), and the
// mean-removed sequence waits in tensor memory (tcgen05.st / ld, 128 columns per thread)
// between the transforms, so every tile is read from global memory once (below L = 32 it is
// read again from L2):
//  * L = 512, 1024 (the production sizes): 512-thread CTAs split into four independent
//    groups of 128 threads, each owning QG = 128 / T consecutive stored wave vectors at a
//    time; the tile ([L frames][QG] complex) arrives by TMA bulk tensor copies, each group
//    synchronises on a named barrier of its own, so the groups drift apart and one group's
//    copy wait hides behind the others' transforms.  Two-pass transforms, the three of them
//    through one copy of the code; the next tile's copy is issued after the partner step and
//    the D rows leave shared memory by bulk async copies.
//  * L = 2048 .. 8192: 256-thread CTAs (512 at 8192), three-pass transforms, TMA tiles of
//    (threads per CTA) / T wave vectors (from a blocked copy [q/16][t][16] for large n_q).
//  * L = 16384: one wave vector per 512-thread CTA; its sequence arrives by TMA through a
//    ring of 16 stages; the three transforms through one copy of the code.
//  * L <= 256: 256-thread CTAs, each thread loads its own samples (every warp load covers
//    whole row segments F[t][q0 .. q0+QT) of the [t][q] spectrum); D rows stored by warps.
// From L = 512 on, every kernel also has an instance for N = L (a stack that fills the
// transform length, kd = min(32, N / 32) with it), in which every bound that depends on N is
// a compile-time constant; the launchers pick it whenever the plan's N and kd match.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

// ---- TMA (bulk tensor copies), bulk copies and mbarrier helpers, inline PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y),
        "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z),
        "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// shared -> global bulk copy (size and both addresses multiples of 16 bytes)
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk copies have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// this thread's bulk copies are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// A bounded wait on a tile barrier: about two seconds of polling (cap in SM clock cycles),
// then false.
constexpr long long kWaitCapCycles = 4000000000LL;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long cap = kWaitCapCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > cap) return false;
    }
    return true;
}

// Test hook for the bounded waits: one CTA arms a barrier for 16 bytes that no copy will
// deliver, waits on it with the given bound (the same routine every tile wait uses), and
// reports the give-up in the status word the way the time kernels do (bit 2).
__global__ void wait_selftest_kernel(unsigned* status, long long cap) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(&bar, 16u);
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, cap);
    if (__syncthreads_or(ok ? 0 : 1) && threadIdx.x == 0) atomicOr(status, 2u);
}
// true in every thread of the group of `nthreads` on named barrier `id` if pred holds in any
__device__ __forceinline__ bool group_any(bool pred, int id, int nthreads) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r) : "r"((uint32_t)pred), "r"(id), "r"(nthreads) : "memory");
    return r != 0;
}

// named barrier `id` over the threads of one group
template <int NTHREADS>
struct SyncGroup {
    int id;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NTHREADS) : "memory");
    }
};

struct TArgs {
    int N;            // frames
    int kd;           // directly evaluated trailing lags (<= 32, < N)
    int H, Wh;        // for the storage -> public q map
    int crop;         // stored order -> D row: 0 whole half plane, 1 low-frequency store
                      // (D rows in stored order), 2 kx-column range [kx0, kx0 + nk)
    int kx0, nk;
    int64_t n_q;      // stored wave vectors = spectrum frame stride
    int64_t q0, q1;   // stored wave vectors this launch covers: [q0, q1)
    int64_t n_tiles;  // tiles of [q0, q1) (of one group, L >= 512; of one CTA, L <= 256)
    int vec4;         // D rows 16-byte aligned (N % 4 == 0 and D aligned)
    int fix;          // FP64-fixup tier: lags 1..fix by direct differences (0 = off)
    int blocked;      // L >= 2048: the spectrum arrives as 16-wave-vector blocks [b][t][16]
                      // of the range [q0, q1) (block b = wave vectors q0 + 16 b ..)
    const float2* tw;
    const float2* tw2;
    const float* inv;
    unsigned* status;
};

// storage index -> public q = ky * (Wh + 1) + kx (Wh = W/2 is a power of two); with the
// low-frequency restriction (crop = 1) the stored order is the D order; a kx-column range
// (crop = 2) stores [ky][kx - kx0] and then, for kx0 = 0, the kx = W/2 column
__device__ __forceinline__ int public_q(int s, const TArgs& a) {
    if (a.crop == 1) return s;
    const int Wh = a.Wh;
    if (a.crop == 2) {
        const int main = a.H * a.nk;
        if (s < main) {
            const int ky = s / a.nk;
            return ky * (Wh + 1) + a.kx0 + (s - ky * a.nk);
        }
        return (s - main) * (Wh + 1) + Wh;
    }
    const int main = a.H * Wh;
    if (s < main) {
        const int ky = s / Wh;
        return ky * (Wh + 1) + (s - ky * Wh);
    }
    return (s - main) * (Wh + 1) + Wh;
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// =====================================================================================
// L >= 512: independent thread groups per CTA (NGROUPS of 512 / NGROUPS threads), tiles
// by TMA
// =====================================================================================
template <int LOG2L, int NGROUPS>
struct GShape {
    static constexpr int L = 1 << LOG2L;
    using S = FftShape<L>;
    static constexpr int P = S::P, T = S::T;
    static constexpr int NG = NGROUPS;        // groups per CTA
    static constexpr int GT = 512 / NG;       // threads per group
    static constexpr int NT = NG * GT;
    static constexpr int QG = GT / T;         // wave vectors per group tile
    static constexpr int IW = 32 / QG;        // threads of one wave vector in a warp
    static constexpr int NWG = GT / 32;       // warps per group
    static constexpr int KD = 32;             // most trailing lags taken by differences
    static constexpr int KT = (KD + T - 1) / T;   // trailing lags per thread
    static constexpr int G = P / T;           // rows of T frames per thread in the prefix sums
    static constexpr int DS = L + IW;         // D staging row stride (floats): conflict-free
    static constexpr int BOX_T = 256, NBOX = L / BOX_T;
    static constexpr int FIX_MAX = 8;
    // per-group buffers (bytes)
    //   xs:  the tile [t][QG] (TMA layout), then the padded transform exchange
    //   ab:  |X_odd|^2 ([m][QG] floats), then the padded |g|^2 / prefix-sum rows, then the
    //        D rows [QG][DS]
    //   red: row totals of the prefix sums; the mean's warp partials
    //   fix: warp partials of the FP64-fixup lags
    // (the mean-removed sequence and Re C live in tensor memory; |X_odd|^2 waits in shared
    // memory: parked in tensor memory it measured 2 % slower, 0.782 against 0.764 ms at
    // 512^2 x 1024)
    static constexpr size_t G_XS = (size_t)(L + L / T) * QG * sizeof(float2);
    static constexpr size_t G_AB = cmax(cmax((size_t)L * QG * sizeof(float), (size_t)QG * DS * sizeof(float)),
                                        (size_t)(L + L / T) * QG * sizeof(float));
    static constexpr size_t G_RED = (size_t)P * QG * sizeof(float);
    static constexpr size_t G_FIX = (size_t)FIX_MAX * NWG * QG * sizeof(float);
    static constexpr size_t OFF_TW = 0;
    static constexpr size_t OFF_TW2 = OFF_TW + (size_t)L * sizeof(float2);
    static constexpr size_t OFF_INV = OFF_TW2 + (size_t)L * sizeof(float2);
    static constexpr size_t OFF_XS = (OFF_INV + (size_t)L * sizeof(float) + 1023) & ~size_t(1023);
    static constexpr size_t OFF_AB = OFF_XS + NG * G_XS;
    static constexpr size_t OFF_RED = OFF_AB + NG * G_AB;
    static constexpr size_t OFF_FIX = OFF_RED + NG * G_RED;
    static constexpr size_t BYTES = OFF_FIX + NG * G_FIX;
    static_assert(L >= 512 && T >= 16 && QG * T == GT, "grouped kernel: L >= 512");
    static_assert(BYTES + 1024 <= 232448, "temporal kernel shared memory exceeds 227 KB");
    static_assert(G_XS % 1024 == 0, "TMA destinations stay 1024-byte aligned");
    static_assert((DS % 4) == 0 && (G_AB % 16) == 0, "D rows must be 16-byte aligned for bulk copies");
    static_assert((size_t)NWG * QG * sizeof(float2) <= G_RED, "mean partials must fit");
    static_assert(NG * GT == 512, "tensor-memory columns: four warps of 128 columns per lane quarter");
};

// ---- tensor memory as per-thread scratch of the grouped kernel.  Thread (warp w, lane l)
// owns TMEM lane 32 (w mod 4) + l; the four warps that share a lane quarter own 128 columns
// each (w / 4 selects them), so a 512-thread CTA uses all 512 columns.  Columns [0, 64) of
// a thread hold its mean-removed time sequence (re, im of its P = 32 samples, in u order),
// [64, 96) its 32 values of Re C.
constexpr uint32_t kSeqTmemCols = 512;
__device__ __forceinline__ void seq_tmem_alloc(uint32_t* slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "r"(kSeqTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void seq_tmem_free(uint32_t tmem) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSeqTmemCols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 consecutive columns of this thread's lane <- r (warp-wide: every lane stores its own)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&r)[32]) {
    __syncwarp();   // the warp-collective tcgen05 forms need a converged warp
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31, %32};"
        ::"r"(taddr), "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]),
          "f"(r[8]), "f"(r[9]), "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15]),
          "f"(r[16]), "f"(r[17]), "f"(r[18]), "f"(r[19]), "f"(r[20]), "f"(r[21]), "f"(r[22]), "f"(r[23]),
          "f"(r[24]), "f"(r[25]), "f"(r[26]), "f"(r[27]), "f"(r[28]), "f"(r[29]), "f"(r[30]), "f"(r[31])
        : "memory");
}
// every tcgen05.st of this thread has completed (before the same columns are read back)
__device__ __forceinline__ void tmem_st_wait() {
    __syncwarp();
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// r <- 32 consecutive columns of this thread's lane; the wait is in the same statement
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32]) {
    __syncwarp();
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
// 16-column forms, for kernels with less register room
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&r)[16]) {
    __syncwarp();
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16};"
        ::"r"(taddr), "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]),
          "f"(r[8]), "f"(r[9]), "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
    __syncwarp();
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];\n tcgen05.wait::ld.sync.aligned;"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
          "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
        : "r"(taddr) : "memory");
}
// the 32 complex samples of a thread in columns [0, 64), (re, im) of v[0], v[1], ...;
// moved in pieces of 32 columns, or of 16 (SMALL) where registers are short
template <bool SMALL = false>
__device__ __forceinline__ void tmem_st_seq(uint32_t taddr, const float2 (&v)[32]) {
    if constexpr (SMALL) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float r[16];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                r[2 * k] = v[8 * h + k].x;
                r[2 * k + 1] = v[8 * h + k].y;
            }
            tmem_st16(taddr + 16u * h, r);
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float r[32];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                r[2 * k] = v[16 * h + k].x;
                r[2 * k + 1] = v[16 * h + k].y;
            }
            tmem_st32(taddr + 32u * h, r);
        }
    }
}
template <bool SMALL = false>
__device__ __forceinline__ void tmem_ld_seq(uint32_t taddr, float2 (&v)[32]) {
    if constexpr (SMALL) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float r[16];
            tmem_ld16(taddr + 16u * h, r);
#pragma unroll
            for (int k = 0; k < 8; ++k) v[8 * h + k] = make_float2(r[2 * k], r[2 * k + 1]);
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float r[32];
            tmem_ld32(taddr + 32u * h, r);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[16 * h + k] = make_float2(r[2 * k], r[2 * k + 1]);
        }
    }
}

template <int NCOLS>
__device__ __forceinline__ void long_tmem_alloc(uint32_t* slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "n"(NCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOLS>
__device__ __forceinline__ void long_tmem_free(uint32_t tmem) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(NCOLS) : "memory");
}

// FULL: the instance for N = L (hence kd = T): every bound that depends on N is a
// compile-time constant, so the per-sample range tests fold away (512^2 x 1024:
// 0.761 -> 0.751 ms; 512^2 x 512: 0.363 -> 0.350 ms, bitwise the same D).
template <int LOG2L, int NGROUPS, bool FIXUP, bool FULL>
__global__ void __launch_bounds__(GShape<LOG2L, NGROUPS>::NT, 1)
temporal_sf_kernel(float* __restrict__ D, TArgs a, const __grid_constant__ CUtensorMap tmap) {
    using C = GShape<LOG2L, NGROUPS>;
    constexpr int L = C::L, P = C::P, T = C::T, QG = C::QG, NG = C::NG, GT = C::GT;
    constexpr int NWG = C::NWG, G = C::G, KT = C::KT, DS = C::DS, FM = C::FIX_MAX;
    static_assert(P == 32, "one thread holds 32 samples (64 tensor-memory columns)");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t tile_bar[NG];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int grp = tid / GT, tg = tid % GT;
    const int bar_id = 1 + grp;          // named barrier of this group (0 is __syncthreads)
    float2* tw = reinterpret_cast<float2*>(smem_raw + C::OFF_TW);
    float2* tw2 = reinterpret_cast<float2*>(smem_raw + C::OFF_TW2);
    float* inv = reinterpret_cast<float*>(smem_raw + C::OFF_INV);
    float2* xs = reinterpret_cast<float2*>(smem_raw + C::OFF_XS + grp * C::G_XS);
    float* ab = reinterpret_cast<float*>(smem_raw + C::OFF_AB + grp * C::G_AB);
    float* red = reinterpret_cast<float*>(smem_raw + C::OFF_RED + grp * C::G_RED);
    float2* red2 = reinterpret_cast<float2*>(red);
    float* fixw = reinterpret_cast<float*>(smem_raw + C::OFF_FIX + grp * C::G_FIX);
    uint64_t* bar = &tile_bar[grp];

    if (tg == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) seq_tmem_alloc(&tmem_slot);
    for (int k = tid; k < L; k += C::NT) {
        tw[k] = a.tw[k];
        tw2[k] = a.tw2[k];
        inv[k] = a.inv[k];
    }
    tc_fence_before();
    __syncthreads();   // the only CTA-wide barrier before the end: the groups run on their own
    tc_fence_after();
    // this thread's tensor-memory columns: the sequence at t_seq, Re C at t_rec, and at t_inv
    // the normalisations 1 / (N - m) of its lags m = i + T u (the same for every tile)
    const uint32_t t_seq = tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(warp >> 2) * 128u;
    const uint32_t t_rec = t_seq + 64u;
    const uint32_t t_inv = t_seq + 96u;

    const int ql = tg % QG;
    const int i = tg / QG;
    {
        float iv[P];
#pragma unroll
        for (int u = 0; u < P; ++u) iv[u] = inv[i + T * u];
        tmem_st32(t_inv, iv);
    }
    const int lane = tid & 31, wg = tg >> 5;
    const SyncGroup<GT> sync{bar_id};
    const AddrPaddedInterleaved<QG, T> xaddr{ql};
    const int N = FULL ? L : a.N;
    const int kd = FULL ? T : a.kd;
    const int64_t q0 = a.q0, q1 = a.q1;
    const int64_t gstride = (int64_t)gridDim.x * NG;
    bool timed_out = false;
    float chk = 0.f;                      // becomes NaN if any D value is not finite
    uint32_t phase = 0;

    // Copy group tile `t` ([t][QG] complex, zeros beyond N and n_q) into xs.
    // Precondition: every thread of the group is done with xs (a group barrier was passed).
    auto issue = [&](int64_t t) {
        if (tg == 0) {
            fence_proxy_async();
            mbar_expect_tx(bar, (uint32_t)(C::NBOX * C::BOX_T * QG * sizeof(float2)));
#pragma unroll
            for (int b = 0; b < C::NBOX; ++b)
                tma_load_2d(xs + b * C::BOX_T * QG, &tmap, (int)(2 * (q0 + t * QG)), b * C::BOX_T, bar);
        }
    };
    // Wait for the copy in flight; the decision to give up is the same in the whole group.
    auto wait = [&]() -> bool {
        const bool ok = mbar_wait_bounded(bar, phase);
        if (group_any(!ok, bar_id, GT)) return false;
        phase ^= 1u;
        return true;
    };

    // trailing lags of this thread: m = m0 + k T in [N - kd, N)
    const int m_lo = N - kd;
    const int m0 = m_lo + ((i - m_lo) % T + T) % T;
    // S(m - 1) and S(N - 1 - m) for m = i + T u sit at these padded positions + / - u (T + 1)
    const int base1 = i >= 1 ? i - 1 : -2;
    const int base2 = (N - 1 - i) + (N - 1 - i) / T;

    int64_t gt = (int64_t)blockIdx.x * NG + grp;
    if (gt < a.n_tiles) issue(gt);
    for (; gt < a.n_tiles; gt += gstride) {
        // (no L2 prefetch of later tiles: with several groups per SM their copies already
        // overlap the other groups' work, and prefetched lines measurably crowd the
        // current tiles out of L2 at 512x512x1024)
        if (!wait()) { timed_out = true; break; }

        // ---- the time sequence in the cyclic layout, and its mean
        float2 v[P];
        float2 part = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            v[u] = xs[(i + T * u) * QG + ql];
            part = cadd(part, v[u]);
        }
#pragma unroll
        for (int o = QG; o < 32; o <<= 1) {
            part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
            part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
        }
        if (lane < QG) red2[wg * QG + ql] = part;
        // the previous tile's D copies must have left ab before it is written again
        if (tg < QG) bulk_wait_read_all();
        sync();
        float2 mean = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NWG; ++w) mean = cadd(mean, red2[w * QG + ql]);
        {
            const float rn = 1.0f / (float)N;
            mean = make_float2(mean.x * rn, mean.y * rn);
        }
#pragma unroll
        for (int u = 0; u < P; ++u)
            if (i + T * u < N) v[u] = csub(v[u], mean);
        // the mean-removed sequence into tensor memory: the even-bin transform and the power
        // sums take it from there, so the tile is read from shared memory only this once
        tmem_st_seq(t_seq, v);

        // ---- from the tile while it is still in xs: the trailing lags by differences
        // (Eq. 1) and, in the FP64-fixup tier, the leading lags' partial sums (differences
        // do not depend on the mean)
        float tl[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int m = m0 + k * T;
            float acc = 0.f;
            if (m < N) {
                // four partial sums: the group waits at its next barrier for the thread with
                // the most pairs (kd of them), so its chain of dependent adds is kept short
                const int n = N - m;
                float a4[4] = {0.f, 0.f, 0.f, 0.f};
                int t = 0;
                for (; t + 4 <= n; t += 4) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        a4[j] += cabs2(csub(xs[(t + j + m) * QG + ql], xs[(t + j) * QG + ql]));
                }
                for (; t < n; ++t) a4[0] += cabs2(csub(xs[(t + m) * QG + ql], xs[t * QG + ql]));
                acc = ((a4[0] + a4[1]) + (a4[2] + a4[3])) * inv[m];
                chk = fmaf(acc, 0.f, chk);
            }
            tl[k] = acc;
        }
        if constexpr (FIXUP) {
            const int fix = a.fix;
            float fp[FM];
#pragma unroll
            for (int k = 0; k < FM; ++k) fp[k] = 0.f;
#pragma unroll 4
            for (int u = 0; u < P; ++u) {
                const int t = i + T * u;
                if (t < N) {
                    const float2 g0 = xs[t * QG + ql];
#pragma unroll
                    for (int k = 0; k < FM; ++k)
                        if (k < fix && t + k + 1 < N) fp[k] += cabs2(csub(xs[(t + k + 1) * QG + ql], g0));
                }
            }
#pragma unroll
            for (int k = 0; k < FM; ++k) {
#pragma unroll
                for (int o = QG; o < 32; o <<= 1) fp[k] += __shfl_xor_sync(0xffffffffu, fp[k], o);
                if (lane < QG) fixw[(k * NWG + wg) * QG + ql] = fp[k];
            }
        }

        // ---- odd bins: L-point DFT of g(t) e^{-i pi t / L}; |.|^2 parked in ab
#pragma unroll
        for (int u = 0; u < P; ++u) {
            v[u] = cmul(v[u], tw2[i + T * u]);
            if ((u & 7) == 7) hoist_fence();
        }
        sync();   // every read of the tile is done: xs becomes the exchange
        // ---- one copy of the transform's code for the three: pass 0 the odd bins (|.|^2 parked
        // in ab), pass 1 the even bins (g taken back from tensor memory), pass 2 the inverse of
        // Z = |X_even|^2 + i |X_odd|^2 as DFT(conj Z), the conjugate of the inverse (folded into
        // the partner step below); the FP64-fixup tier unrolls the three (1.20 -> 1.16 ms at
        // 512^2 x 1024: the loop costs it more than it saves)
#pragma unroll (FIXUP ? 3 : 1)
        for (int pass = 0; pass < 3; ++pass) {
            if (pass == 1) {
                tmem_st_wait();
                tmem_ld_seq(t_seq, v);
            } else if (pass == 2) {
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    v[u] = make_float2(cabs2(v[u]), -ab[(i + T * u) * QG + ql]);
                    if ((u & 7) == 7) hoist_fence();
                }
            }
            fft_cyclic<L, false>(v, i, xs, xaddr, tw, sync);
            if (pass == 0) {
#pragma unroll
                for (int u = 0; u < P; ++u) ab[(i + T * u) * QG + ql] = cabs2(v[u]);
            }
        }
        // ---- Re C(m) into tensor memory.  v = conj(z), z the unnormalised inverse DFT of Z:
        // the partner formula below is the one of the file header with z = conj(v),
        // z(L - m) = conj(xs[L - m])
#pragma unroll
        for (int u = 0; u < P; ++u) xs[(i + T * u) * QG + ql] = v[u];
        sync();
        {
            const float scale = 0.25f / (float)L;
            float rc[P];
#pragma unroll
            for (int u = 0; u < P; ++u) {
                const int m = i + T * u;
                const float2 y = v[u];
                const float2 yr = xs[((L - m) & (L - 1)) * QG + ql];
                const float2 w = tw2[m];                   // (cos(pi m/L), -sin(pi m/L))
                rc[u] = scale * ((y.x + yr.x) - w.x * (y.y + yr.y) - w.y * (y.x - yr.x));
                if ((u & 7) == 7) hoist_fence();
            }
            tmem_st32(t_rec, rc);
        }
        sync();   // partner reads done: xs is free

        // ---- the next tile's copy overlaps the power sums, the combination and the stores
        if (gt + gstride < a.n_tiles) issue(gt + gstride);

        // |g - mean|^2 (from tensor memory) into padded rows of ab (frame t at t + t / T):
        // both the cyclic writes here and the row-wise reads below are conflict-free
        tmem_ld_seq(t_seq, v);
#pragma unroll
        for (int u = 0; u < P; ++u) ab[(i + u * (T + 1)) * QG + ql] = cabs2(v[u]);
        sync();
        // ---- inclusive prefix sums S(t): thread i owns the rows r = i + T g of T frames
        float rowv[G][T];
        float racc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = i + T * g;
            float acc = 0.f;
#pragma unroll
            for (int jj = 0; jj < T; ++jj) {
                acc += ab[(r * (T + 1) + jj) * QG + ql];
                rowv[g][jj] = acc;
            }
            racc[g] = acc;
            if constexpr (G > 1) red[r * QG + ql] = acc;
        }
        float total = 0.f;
        float off[G];
#pragma unroll
        for (int g = 0; g < G; ++g) off[g] = 0.f;
        if constexpr (G == 1) {
            // one row per thread (rows in thread order): a shuffle scan within the warp (lanes
            // of one wave vector QG apart) and the warps' totals
            float incl = racc[0];
#pragma unroll
            for (int o = QG; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane >= 32 - QG) red[wg * QG + ql] = incl;
            sync();
            off[0] = incl - racc[0];
#pragma unroll
            for (int w = 0; w < NWG; ++w) {
                const float x = red[w * QG + ql];
                if (w < wg) off[0] += x;
                total += x;
            }
        } else {
            sync();
#pragma unroll
            for (int rp = 0; rp < P; ++rp) {
                const float x = red[rp * QG + ql];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (rp < i + T * g) off[g] += x;
                total += x;
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = i + T * g;
#pragma unroll
            for (int jj = 0; jj < T; ++jj) ab[(r * (T + 1) + jj) * QG + ql] = rowv[g][jj] + off[g];
        }
        sync();
        // FP64-fixup tier: lag m = i (1 <= i <= fix) summed over the group's warps in FP64
        float fixd = 0.f;
        const bool has_fix = FIXUP && a.fix > 0 && i >= 1 && i <= a.fix && i < N - kd;
        if (has_fix) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NWG; ++w) s += (double)fixw[((i - 1) * NWG + w) * QG + ql];
            fixd = (float)(s / (double)(N - i));
            chk = fmaf(fixd, 0.f, chk);
        }

        // ---- D(m) = (P1 + P2 - 2 Re C) / (N - m) for 0 < m < N - kd
        float dv[P];
        tmem_st_wait();
        tmem_ld32(t_rec, dv);                              // Re C(i + T u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float iv[16];
            tmem_ld16(t_inv + 16u * h, iv);                // 1 / (N - m)
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int u = 16 * h + k;
                const int m = i + T * u;
                float d = 0.f;
                if (m > 0 && m < N - kd) {
                    const float p1 = ab[(base2 - u * (T + 1)) * QG + ql];
                    const float p2 = total - ab[(base1 + u * (T + 1)) * QG + ql];
                    d = (p1 + p2 - 2.f * dv[u]) * iv[k];
                    chk = fmaf(d, 0.f, chk);
                }
                dv[u] = d;
                if ((u & 7) == 7) hoist_fence();
            }
        }
        sync();   // reads of S done: ab takes the D rows

        // ---- D rows [q][m] staged in ab, then copied out
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            if (m < N) ab[ql * DS + m] = dv[u];
        }
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int m = m0 + k * T;
            if (m < N) ab[ql * DS + m] = tl[k];
        }
        if (has_fix) ab[ql * DS + i] = fixd;
        if (a.vec4) fence_proxy_async();   // generic writes -> the bulk copies' reads
        sync();
        if (a.vec4) {
            if (tg < QG) {
                const int64_t sr = q0 + gt * QG + tg;
                if (sr < q1) {
                    float* drow = D + (int64_t)public_q((int)sr, a) * N;
                    bulk_store(drow, ab + tg * DS, (uint32_t)N * (uint32_t)sizeof(float));
                }
                bulk_commit();
            }
        } else {
#pragma unroll 1
            for (int r = 0; r < QG; ++r) {
                const int64_t sr = q0 + gt * QG + r;
                if (sr >= q1) break;
                float* drow = D + (int64_t)public_q((int)sr, a) * N;
                for (int m = tg; m < N; m += GT) drow[m] = ab[r * DS + m];
            }
        }
    }
    if (timed_out) {
        // a tile copy never completed: report it; give the outstanding copy a last bounded
        // chance to land before the CTA's shared memory goes away
        atomicOr(a.status, 2u);
        mbar_wait_bounded(bar, phase);
    }
    if (tg < QG) bulk_wait_all();
    if (chk != chk) atomicOr(a.status, 1u);
    // every group is done with tensor memory before it is released
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) seq_tmem_free(tmem_slot);
}

// =====================================================================================
// L = 2048 .. 8192 (N up to 8192): three-pass transforms; 256-thread CTAs, two per SM, at
// L = 2048, 4096; one 512-thread CTA per SM at L = 8192
// =====================================================================================
// A CTA owns QG = 256 / T wave vectors at a time (T = L / 32 threads each, 32 samples per
// thread).  Tiles arrive by TMA as above; the three transforms are fft_cyclic3 (32-point
// register DFT, handover exchange, inner two-pass T-point transform), whose output order
// is the permuted thread index sigma(i); the inverse runs with i = sigma(i) and leaves
// lag m = sigma(sigma(i)) + T u in thread i.  Prefix sums: thread i owns the chunk of 32
// consecutive frames starting at 32 i.  Small tables so that two CTAs share an SM: pass
// twiddles from a quarter-wave table; e^{-i pi t / L} for t = i + T u as e^{-i pi i / L}
// (one per thread) times e^{-i pi u / 32}; 1/(N - m) as a correctly rounded reciprocal.
// The next tile's copy is issued before the D rows are staged; the rows leave by bulk
// copies, as in the kernel above.
template <int LOG2L>
struct LShape {
    static constexpr int L = 1 << LOG2L;
    static constexpr int P = 32, T = L / P, R = T / P;
    static constexpr int NT = L >= 8192 ? 512 : 256;   // QG = 2 at L = 4096 and 8192
    static constexpr int CTAS_PER_SM = NT == 256 ? 2 : 1;
    static constexpr int QG = NT / T;             // wave vectors per tile
    static constexpr int NWG = NT / 32;
    static constexpr int PAD = (QG == 2) ? 4 : 2; // (T + PAD) * QG = 8 mod 16: handover reads spread
    static constexpr int DS = L + 32 / QG;        // D staging row stride (floats): rows of the
                                                  // QG wave vectors start on different banks
    static constexpr int BOX_T = 256, NBOX = L / BOX_T;
    static constexpr size_t XS_ELEMS = (size_t)P * (T + PAD) * QG > (size_t)L * QG
                                           ? (size_t)P * (T + PAD) * QG : (size_t)L * QG;
    static constexpr size_t OFF_TWQ = 0;                                        // L/4 entries
    static constexpr size_t OFF_TWI = OFF_TWQ + (size_t)(L / 4) * sizeof(float2);  // T entries
    static constexpr size_t OFF_CI = OFF_TWI + (size_t)T * sizeof(float2);         // T entries
    static constexpr size_t OFF_W64 = OFF_CI + (size_t)T * sizeof(float2);         // 32 entries
    static constexpr size_t OFF_XS = (OFF_W64 + 32 * sizeof(float2) + 1023) & ~size_t(1023);
    static constexpr size_t OFF_AB = OFF_XS + XS_ELEMS * sizeof(float2);
    // ab: the padded |g|^2 / prefix rows ((L + L/32) QG floats), then the D rows
    static constexpr size_t AB_FLOATS = cmax(cmax((size_t)L * QG, (size_t)QG * DS), (size_t)(L + L / P) * QG);
    static constexpr size_t OFF_RED = OFF_AB + AB_FLOATS * sizeof(float);
    static constexpr int FIX_MAX = 8;
    static constexpr size_t OFF_FIX = OFF_RED + (size_t)T * QG * sizeof(float);
    static constexpr size_t BYTES = OFF_FIX + (size_t)FIX_MAX * NWG * QG * sizeof(float);
    static_assert(T % P == 0 && QG * T == NT && QG >= 2, "long kernel: L = 2048 .. 8192");
    static_assert(CTAS_PER_SM * (BYTES + 1024) <= 233472, "shared memory per SM");
    static_assert(NT % 128 == 0, "tensor memory: 128 columns per warp, NT columns per CTA");
    static_assert((size_t)NWG * QG * 2 <= (size_t)T * QG, "mean partials must fit");
    static_assert((DS % 4) == 0 && (OFF_AB % 16) == 0, "D rows 16-byte aligned for bulk copies");
};

struct LTables {
    const float2* quarter;   // (cos, sin) of 2 pi k / L, k < L / 4
    const float2* inner;     // pass twiddles of the inner T-point transform
    const float2* ci;        // exp(-i pi i / L), i < T
    const float2* w64;       // exp(-i pi u / 32), u < 32
};

// FULL: the instance for N = L (hence kd = 32), as for the grouped kernel above (random
// spectrum, kernel alone: 512^2 x 2048 2.645 -> 2.535 ms, x 4096 5.754 -> 5.494 ms, FP64-fixup
// tier 7.33 -> 6.76 ms, x 8192 12.92 -> 12.54 ms; bitwise the same D).
template <int LOG2L, bool FIXUP, bool FULL>
__global__ void __launch_bounds__(LShape<LOG2L>::NT, LShape<LOG2L>::CTAS_PER_SM)
temporal_sf_long_kernel(float* __restrict__ D, TArgs a, const __grid_constant__ CUtensorMap tmap,
                        LTables tb) {
    using C = LShape<LOG2L>;
    constexpr int L = C::L, P = C::P, T = C::T, R = C::R, QG = C::QG, NT = C::NT, NWG = C::NWG;
    constexpr int DS = C::DS, PAD = C::PAD, FM = C::FIX_MAX;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t tile_bar;
    __shared__ uint32_t tmem_slot;
    float2* twq = reinterpret_cast<float2*>(smem_raw + C::OFF_TWQ);
    float2* twi = reinterpret_cast<float2*>(smem_raw + C::OFF_TWI);
    float2* ci = reinterpret_cast<float2*>(smem_raw + C::OFF_CI);
    float2* w64 = reinterpret_cast<float2*>(smem_raw + C::OFF_W64);
    float2* xs = reinterpret_cast<float2*>(smem_raw + C::OFF_XS);
    float* ab = reinterpret_cast<float*>(smem_raw + C::OFF_AB);
    float* xf = ab;                              // the padded |g|^2 / prefix rows
    float* red = reinterpret_cast<float*>(smem_raw + C::OFF_RED);
    float2* red2 = reinterpret_cast<float2*>(red);
    float* fixw = reinterpret_cast<float*>(smem_raw + C::OFF_FIX);

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&tile_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = tid; k < L / 4; k += NT) twq[k] = tb.quarter[k];
    for (int k = tid; k < T; k += NT) {
        twi[k] = tb.inner[k];
        ci[k] = tb.ci[k];
    }
    if (tid < 32) w64[tid] = tb.w64[tid];
    if (tid < 32) long_tmem_alloc<NT>(&tmem_slot);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int ql = tid % QG, i = tid / QG;
    const int lane = tid & 31, wg = tid >> 5;
    // tensor-memory columns of this thread (lane 32 (warp mod 4) + lane, 128 columns per warp
    // of a lane quarter): the mean-removed sequence, |X_odd|^2, Re C
    const uint32_t t_seq = tmem_slot + ((uint32_t)(32 * (wg & 3)) << 16) + (uint32_t)(wg >> 2) * 128u;
    const uint32_t t_odd = t_seq + 64u, t_rec = t_seq + 96u;
    const int s1 = fft3_sigma(i, P, R);          // forward output order
    const float2 c_i = ci[i];
    // Transform outputs come in the order s1 = sigma(i) (a warp's lanes 32 / R apart in
    // index); they go back to cyclic order (m = i + T u) through xs, index m at slot
    // m ^ ((m >> ZS) mod 8), which spreads both access patterns over the banks.
    constexpr int ZS = R >= 8 ? 4 : 3;
    auto zslot = [](int m) { return m ^ ((m >> ZS) & 7); };
    static_assert(((T >> ZS) & 7) == 0, "zslot(j + T u) = zslot(j) + T u");
    const int zs1 = zslot(s1), zsi = zslot(i);
    const TwiddleQuarter<L> tw1{twq};
    const int N = FULL ? L : a.N, kd = FULL ? 32 : a.kd;
    const int64_t q0 = a.q0, q1 = a.q1;
    bool timed_out = false;
    float chk = 0.f;
    uint32_t phase = 0;
    auto issue = [&](int64_t t) {
        if (tid == 0) {
            fence_proxy_async();
            mbar_expect_tx(&tile_bar, (uint32_t)(C::NBOX * C::BOX_T * QG * sizeof(float2)));
            const int64_t rel = t * QG;                    // first wave vector, relative to q0
#pragma unroll
            for (int b = 0; b < C::NBOX; ++b) {
                if (a.blocked)                             // [block][t][16]: x in the block, t, block
                    tma_load_3d(xs + b * C::BOX_T * QG, &tmap, (int)(2 * (rel & 15)), b * C::BOX_T,
                                (int)(rel >> 4), &tile_bar);
                else
                    tma_load_2d(xs + b * C::BOX_T * QG, &tmap, (int)(2 * (q0 + rel)), b * C::BOX_T, &tile_bar);
            }
        }
    };
    auto wait = [&]() -> bool {
        const bool ok = mbar_wait_bounded(&tile_bar, phase);
        if (__syncthreads_or(ok ? 0 : 1)) return false;
        phase ^= 1u;
        return true;
    };
    // trailing lag of this thread, if < N: the one it also holds in the combination's
    // (cyclic) order, m = i + T u
    const int m_lo = N - kd;
    const int m_tail = m_lo + ((i - m_lo) % T + T) % T;

    if ((int64_t)blockIdx.x < a.n_tiles) issue(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        if (!wait()) { timed_out = true; break; }
        // ---- time sequence (cyclic, thread i holds t = i + T u) and its mean
        float2 v[P];
        float2 part = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            v[u] = xs[(i + T * u) * QG + ql];
            part = cadd(part, v[u]);
        }
#pragma unroll
        for (int o = QG; o < 32; o <<= 1) {
            part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
            part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
        }
        if (lane < QG) red2[wg * QG + ql] = part;
        if (tid < QG) bulk_wait_read_all();                // the previous rows have left ab
        __syncthreads();
        float2 mean = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NWG; ++w) mean = cadd(mean, red2[w * QG + ql]);
        {
            const float rn = 1.0f / (float)N;
            mean = make_float2(mean.x * rn, mean.y * rn);
        }
#pragma unroll
        for (int u = 0; u < P; ++u)
            if (i + T * u < N) v[u] = csub(v[u], mean);
        // the mean-removed sequence into tensor memory: both forward transforms and the power
        // sums take it from there (so the tile is copied from global memory once, and the
        // registers are free for the sums below)
        tmem_st_seq<true>(t_seq, v);
        // ---- from the tile while it is still in xs: the trailing lag by differences (Eq. 1)
        // and, in the FP64-fixup tier, the leading lags' partial sums
        float tl = 0.f;
        if (m_tail < N) {
            for (int t = 0; t < N - m_tail; ++t)
                tl += cabs2(csub(xs[(t + m_tail) * QG + ql], xs[t * QG + ql]));
            tl *= __frcp_rn((float)(N - m_tail));
            chk = fmaf(tl, 0.f, chk);
        }
        if constexpr (FIXUP) {
            // FP64-fixup tier: sum over this thread's samples of |g(t+m) - g(t)|^2, m = 1..fix,
            // then over the lanes of the same wave vector in the warp
            const int fix = a.fix;
            float fp[FM];
#pragma unroll
            for (int k = 0; k < FM; ++k) fp[k] = 0.f;
#pragma unroll 4
            for (int u = 0; u < P; ++u) {
                const int t = i + T * u;
                if (t < N) {
                    const float2 g0 = xs[t * QG + ql];
#pragma unroll
                    for (int k = 0; k < FM; ++k)
                        if (k < fix && t + k + 1 < N) fp[k] += cabs2(csub(xs[(t + k + 1) * QG + ql], g0));
                }
            }
#pragma unroll
            for (int k = 0; k < FM; ++k) {
#pragma unroll
                for (int o = QG; o < 32; o <<= 1) fp[k] += __shfl_xor_sync(0xffffffffu, fp[k], o);
                if (lane < QG) fixw[(k * NWG + wg) * QG + ql] = fp[k];
            }
        }
        __syncthreads();                                   // every read of the tile is done
        // ---- pass 0, odd bins: DFT of g(t) e^{-i pi t / L}, |.|^2 parked in tensor memory;
        //      pass 1, even bins: DFT of g (from tensor memory).  One copy of the transform's
        //      code for both (the unrolled transform is most of the kernel's instructions).
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            tmem_st_wait();
            tmem_ld_seq<true>(t_seq, v);
            if (pass == 0) {
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    v[u] = cmul(cmul(v[u], c_i), w64[u]);          // zero past N stays zero
                    if ((u & 7) == 7) hoist_fence();
                }
            }
            fft_cyclic3<L, false, QG, PAD>(v, i, i, ql, xs, tw1, twi, SyncBlock{});
            if (pass == 0) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float o2[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) o2[k] = cabs2(v[16 * h + k]);
                    tmem_st16(t_odd + 16u * h, o2);
                }
            }
        }
        tmem_st_wait();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float o2[16];
            tmem_ld16(t_odd + 16u * h, o2);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[16 * h + k] = make_float2(cabs2(v[16 * h + k]), o2[k]);
        }
        // ---- inverse of Z = |X_even|^2 + i |X_odd|^2: input order s1, groups by i, output
        // order s1
        fft_cyclic3<L, true, QG, PAD, true>(v, s1, i, ql, xs, tw1, twi, SyncBlock{});
#pragma unroll
        for (int u = 0; u < P; ++u) xs[(zs1 + T * u) * QG + ql] = v[u];
        __syncthreads();
        {
            const float scale = 0.25f / (float)L;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float rc[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int u = 16 * h + k;
                    const int m = i + T * u;
                    const float2 z = xs[(zsi + T * u) * QG + ql];
                    const float2 zr = xs[zslot((L - m) & (L - 1)) * QG + ql];
                    const float2 w = cmul(c_i, w64[u]);    // e^{-i pi m / L}
                    rc[k] = scale * ((z.x + zr.x) + w.x * (z.y + zr.y) - w.y * (z.x - zr.x));
                    if ((k & 7) == 7) hoist_fence();
                }
                tmem_st16(t_rec + 16u * h, rc);
            }
        }
        __syncthreads();                                   // partner reads done: xs is free
        // ---- the next tile's copy overlaps the power sums, the combination and the stores
        if (tile + gridDim.x < a.n_tiles) issue(tile + gridDim.x);
        // |g - mean|^2 (from tensor memory) at padded positions t + t / 32 of ab (chunk-wise
        // reads below are conflict-free)
        tmem_ld_seq<true>(t_seq, v);                             // zero past N
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int t = i + T * u;
            xf[(t + (t >> 5)) * QG + ql] = cabs2(v[u]);
        }
        __syncthreads();
        // ---- inclusive prefix sums: thread i owns frames 32 i .. 32 i + 31; the offsets of
        // the chunks by a shuffle scan within the warp (lanes of one wave vector are QG apart)
        // and the warps' totals
        float rowv[P];
        float acc = 0.f;
#pragma unroll
        for (int jj = 0; jj < P; ++jj) {
            acc += xf[(i * (P + 1) + jj) * QG + ql];
            rowv[jj] = acc;
        }
        float incl = acc;
#pragma unroll
        for (int o = QG; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane >= 32 - QG) red[wg * QG + ql] = incl;     // the warp's last chunk of ql
        __syncthreads();
        float total = 0.f, off = incl - acc;
#pragma unroll
        for (int w = 0; w < NWG; ++w) {
            const float x = red[w * QG + ql];
            if (w < wg) off += x;
            total += x;
        }
#pragma unroll
        for (int jj = 0; jj < P; ++jj) xf[(i * (P + 1) + jj) * QG + ql] = rowv[jj] + off;
        __syncthreads();
        // FP64-fixup tier: lag m = i (1 <= i <= fix), held by this thread at u = 0, summed
        // over the warps in FP64
        float fixd = 0.f;
        const bool has_fix = FIXUP && a.fix > 0 && i >= 1 && i <= a.fix && i < N - kd;
        if (has_fix) {
            double sum = 0.0;
            for (int w = 0; w < NWG; ++w) sum += (double)fixw[((i - 1) * NWG + w) * QG + ql];
            fixd = (float)(sum / (double)(N - i));
            chk = fmaf(fixd, 0.f, chk);
        }
        // ---- D(m) = (P1 + P2 - 2 Re C) / (N - m) for 0 < m < N - kd, m = i + T u
        float dv[P];
        tmem_st_wait();
#pragma unroll
        for (int h = 0; h < 2; ++h) {                      // Re C(i + T u)
            float rc[16];
            tmem_ld16(t_rec + 16u * h, rc);
#pragma unroll
            for (int k = 0; k < 16; ++k) dv[16 * h + k] = rc[k];
        }
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            float d = 0.f;
            if (m > 0 && m < N - kd) {
                const int ta = N - 1 - m, tb2 = m - 1;
                const float p1 = xf[(ta + (ta >> 5)) * QG + ql];
                const float p2 = total - xf[(tb2 + (tb2 >> 5)) * QG + ql];
                d = __fdividef(p1 + p2 - 2.f * dv[u], (float)(N - m));   // within 2 ulp
                chk = fmaf(d, 0.f, chk);
            }
            dv[u] = d;
            if ((u & 7) == 7) hoist_fence();
        }
        __syncthreads();                                   // reads of S done: ab takes the D rows
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            if (m < N) ab[ql * DS + m] = dv[u];
        }
        if (m_tail < N) ab[ql * DS + m_tail] = tl;
        if (has_fix) ab[ql * DS + i] = fixd;
        if (a.vec4) fence_proxy_async();
        __syncthreads();
        if (a.vec4) {
            if (tid < QG) {
                const int64_t sr = q0 + tile * QG + tid;
                if (sr < q1) {
                    float* drow = D + (int64_t)public_q((int)sr, a) * N;
                    bulk_store(drow, ab + tid * DS, (uint32_t)N * (uint32_t)sizeof(float));
                }
                bulk_commit();
            }
        } else {
            for (int r = 0; r < QG; ++r) {
                const int64_t sr = q0 + tile * QG + r;
                if (sr >= q1) break;
                float* drow = D + (int64_t)public_q((int)sr, a) * N;
                for (int m = tid; m < N; m += NT) drow[m] = ab[r * DS + m];
            }
        }
    }
    if (timed_out) {
        if (tid == 0) atomicOr(a.status, 2u);
        mbar_wait_bounded(&tile_bar, phase);
    }
    if (tid < QG) bulk_wait_all();
    if (chk != chk) atomicOr(a.status, 1u);
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) long_tmem_free<NT>(tmem_slot);
}

// =====================================================================================
// L = 16384 (N up to 16384, M = 32768): one wave vector per 512-thread CTA.  Its time
// sequence (128 KB) and the transform's exchange (128 KB) cannot share shared memory: the
// sequence arrives by TMA in chunks of 256 frames (boxes of two neighbouring wave vectors,
// 16 bytes x 256 rows: the narrowest box a TMA row allows) through a ring of 16 stages,
// each thread takes its samples from there into registers and keeps the mean-removed
// sequence in tensor memory (then |X_odd|^2 and Re C: 128 columns per thread).  The first
// round of the next wave vector's chunks is issued as soon as the current one has been
// read, and lands while this one is transformed.  Shared memory holds the exchange, the
// ring, a 32-sample head and tail for the trailing lags and small twiddle tables (pass-1
// twiddles from two 2.5 KB tables, w^j = hi[j / 64] lo[j mod 64]).
// =====================================================================================
template <int L_>
struct TwiddleTwoLevel {
    static constexpr bool kEvenByProduct = true;
    const float2* lo;   // exp(-2 pi i b / L), b < 64
    const float2* hi;   // exp(-2 pi i 64 a / L), a < L / 64
    __device__ __forceinline__ float2 operator()(int k1, int i) const {
        const int j = (k1 * i) & (L_ - 1);
        return cmul(hi[j >> 6], lo[j & 63]);
    }
};

struct XLShape {
    static constexpr int LOG2L = 14, L = 1 << LOG2L;
    static constexpr int P = 32, T = L / P, R = T / P;
    static constexpr int NT = T, NWG = NT / 32;
    static constexpr int PAD = 0;                          // the handover's swizzle suffices
    static constexpr size_t OFF_LO = 0;                                      // 64
    static constexpr size_t OFF_HI = OFF_LO + 64 * sizeof(float2);           // L / 64
    static constexpr size_t OFF_TWI = OFF_HI + (size_t)(L / 64) * sizeof(float2);  // T (inner pass)
    static constexpr size_t OFF_W64 = OFF_TWI + (size_t)T * sizeof(float2);  // 32
    static constexpr size_t OFF_RED = OFF_W64 + 32 * sizeof(float2);         // NWG float2 + 2 NWG float
    static constexpr size_t OFF_XS = (OFF_RED + (size_t)NWG * 16 + 1023) & ~size_t(1023);
    static constexpr size_t XS_ELEMS = (size_t)P * (T + PAD);                // handover; >= L
    static constexpr size_t OFF_HT = OFF_XS + XS_ELEMS * sizeof(float2);    // 32 head + 32 tail
    // the TMA ring: NST stages of one box [256 frames][2 wave vectors] each
    static constexpr int BOX_T = 256, NCH = L / BOX_T, NST = 16, NROUND = NCH / NST;
    static constexpr uint32_t BOX_BYTES = BOX_T * 2 * sizeof(float2);
    static constexpr size_t OFF_RING = OFF_HT + 64 * sizeof(float2);
    static constexpr size_t BYTES = OFF_RING + (size_t)NST * BOX_BYTES;
    static_assert(NT == 2 * BOX_T && NST % 2 == 0 && NCH % NST == 0,
                  "thread i's sample t = i + T u sits in chunk (i / 256) + 2 u: round u / 8, "
                  "stage (i / 256) + 2 (u mod 8)");
    static_assert(NST == 2 * (P / NROUND), "a round holds 8 of each thread's 32 samples");
    static_assert(OFF_RING % 128 == 0, "TMA destinations 128-byte aligned");
    static_assert(XS_ELEMS >= (size_t)L && (size_t)(L + L / 32) * sizeof(float) <= XS_ELEMS * sizeof(float2),
                  "exchange holds the transform and the padded power sums");
    static_assert(BYTES + 1024 <= 233472, "one CTA per SM");
    static_assert(NT == 512, "tensor-memory columns: four warps of 128 columns per lane quarter");
};

struct XLTables {
    const float2* lo;
    const float2* hi;
    const float2* inner;     // pass twiddles of the inner T-point transform
    const float2* ci;        // exp(-i pi i / L), i < T
    const float2* w64;       // exp(-i pi u / 32), u < 32
};

// FULL: the instance for N = L (hence kd = 32), as for the grouped kernel above
// (256^2 x 16384 through ddm_temporal_sf, blocked copy included: 8.47 -> 7.62 ms; bitwise the
// same D).
template <bool FULL>
__global__ void __launch_bounds__(XLShape::NT, 1)
temporal_sf_xl_kernel(float* __restrict__ D, TArgs a, XLTables tb, const __grid_constant__ CUtensorMap tmap) {
    using C = XLShape;
    constexpr int L = C::L, P = C::P, T = C::T, R = C::R, NWG = C::NWG, NST = C::NST, BOX_T = C::BOX_T;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* lo = reinterpret_cast<float2*>(smem_raw + C::OFF_LO);
    float2* hi = reinterpret_cast<float2*>(smem_raw + C::OFF_HI);
    float2* twi = reinterpret_cast<float2*>(smem_raw + C::OFF_TWI);
    float2* w64 = reinterpret_cast<float2*>(smem_raw + C::OFF_W64);
    float2* red2 = reinterpret_cast<float2*>(smem_raw + C::OFF_RED);
    float* wsum = reinterpret_cast<float*>(smem_raw + C::OFF_RED + NWG * sizeof(float2));
    float2* xs = reinterpret_cast<float2*>(smem_raw + C::OFF_XS);
    float* xf = reinterpret_cast<float*>(xs);
    float2* head = reinterpret_cast<float2*>(smem_raw + C::OFF_HT);   // g(t), t < 32
    float2* tail = head + 32;                                          // g(N - 32 + t), t < 32
    float2* ring = reinterpret_cast<float2*>(smem_raw + C::OFF_RING);
    __shared__ uint32_t tmem_slot;
    __shared__ uint64_t ring_bar[C::NST];

    const int i = threadIdx.x;
    const int lane = i & 31, wg = i >> 5;
    if (wg == 0) seq_tmem_alloc(&tmem_slot);
    if (i == 0) {
        for (int st = 0; st < NST; ++st) mbar_init(&ring_bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = i; k < 64; k += C::NT) lo[k] = tb.lo[k];
    for (int k = i; k < L / 64; k += C::NT) hi[k] = tb.hi[k];
    for (int k = i; k < T; k += C::NT) twi[k] = tb.inner[k];
    if (i < 32) w64[i] = tb.w64[i];
    const float2 c_i = tb.ci[i];
    const int s1 = fft3_sigma(i, P, R);                    // transform output order
    // inverse output back to cyclic order through xs: index m at slot m ^ ((m >> 5) mod 16)
    auto zslot = [](int m) { return m ^ ((m >> 5) & 15); };
    static_assert(((T >> 5) & 15) == 0, "zslot(j + T u) = zslot(j) + T u");
    const int zs1 = zslot(s1), zsi = zslot(i);
    const TwiddleTwoLevel<L> tw1{lo, hi};
    const int N = FULL ? L : a.N, kd = FULL ? 32 : a.kd;
    const int m_lo = N - kd;
    const int m_tail = m_lo + ((i - m_lo) % T + T) % T;    // this thread's trailing lag, if < N
    float chk = 0.f;
    // the ring: chunk c (frames 256 c .. 256 c + 255) of a wave vector in stage c mod NST;
    // chunks from nch on hold no frame (N <= 256 nch) and are neither copied nor waited for
    const int nch = (N + BOX_T - 1) / BOX_T;
    bool timed_out = false;
    // copies of round r of stored wave vector `tile` (relative to q0); the box holds the
    // pair of wave vectors (2 k, 2 k + 1) that contains it (q0 and n_q are even)
    auto issue_round = [&](int64_t tile, int r) {
        fence_proxy_async();
        for (int st = 0; st < NST; ++st) {
            const int c = r * NST + st;
            if (c >= nch) break;
            mbar_expect_tx(&ring_bar[st], C::BOX_BYTES);
            if (a.blocked)
                tma_load_3d(ring + (size_t)st * BOX_T * 2, &tmap, (int)(2 * ((tile & 15) & ~1)), c * BOX_T,
                            (int)(tile >> 4), &ring_bar[st]);
            else
                tma_load_2d(ring + (size_t)st * BOX_T * 2, &tmap, (int)(2 * ((a.q0 + tile) & ~(int64_t)1)),
                            c * BOX_T, &ring_bar[st]);
        }
    };
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (i == 0 && blockIdx.x < a.n_tiles) issue_round(blockIdx.x, 0);
    // tensor-memory columns of this thread (lane 32 (warp mod 4) + lane, 128 columns per warp
    // of a lane quarter): the mean-removed sequence, |X_odd|^2, Re C
    const uint32_t t_seq = tmem_slot + ((uint32_t)(32 * (wg & 3)) << 16) + (uint32_t)(wg >> 2) * 128u;
    const uint32_t t_odd = t_seq + 64u, t_rec = t_seq + 96u;

    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int64_t sq = a.q0 + tile;                    // stored wave vector
        const int half = (int)(sq & 1);                    // its column in the ring's boxes
        const int hb = i / BOX_T;                          // thread i reads the chunks hb + 2 u
        // stage st completes once per round that uses it: ceil((nch - st) / NST) times per
        // wave vector, so its parity in round r follows from the wave vectors done before
        const uint32_t done = (uint32_t)((tile - blockIdx.x) / gridDim.x);
        uint32_t pending = 0, pending_par = 0;             // stages this thread gave up on
        __syncthreads();                                   // previous wave vector's reads done
        // ---- time sequence (thread i holds t = i + T u) from the ring, round by round (8 of
        // a thread's samples per round); its first and last 32 samples for the trailing lags;
        // its mean
        float2 v[P];
        float2 part = make_float2(0.f, 0.f);
        bool ok = true;
#pragma unroll
        for (int r = 0; r < C::NROUND; ++r) {
            if (r > 0) {
                // every thread is done with the previous round's stages before they refill
                if (__syncthreads_or(!ok)) break;
                if (i == 0) issue_round(tile, r);
            }
            // this thread's stages of the round: hb, hb + 2, ..., hb + 14 (chunks hb + 2 u)
#pragma unroll 1
            for (int st = hb; st < NST; st += 2) {
                if (r * NST + st >= nch) break;
                const uint32_t par = (done * (uint32_t)((nch - st + NST - 1) / NST) + (uint32_t)r) & 1u;
                if (!mbar_wait_bounded(&ring_bar[st], par)) {
                    ok = false;
                    pending |= 1u << st;
                    pending_par |= par << st;
                }
            }
            const float2* rb = ring + (size_t)(hb * BOX_T + (i & (BOX_T - 1))) * 2 + half;
#pragma unroll
            for (int k = 0; k < P / C::NROUND; ++k) {
                const int u = r * (P / C::NROUND) + k;
                const int t = i + T * u;                   // in chunk hb + 2 u = r NST + hb + 2 k
                v[u] = (ok && t < N) ? rb[(size_t)k * 2 * BOX_T * 2] : make_float2(0.f, 0.f);
                part = cadd(part, v[u]);
                if (t < 32) head[t] = v[u];
                if (t >= N - 32 && t < N) tail[t - (N - 32)] = v[u];
            }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
            part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
        }
        if (lane == 0) red2[wg] = part;
        // a copy that never landed ends the kernel for the whole CTA (status bit 2); the copies
        // this thread gave up on get a last bounded chance to land before the CTA's shared
        // memory goes away
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            for (int st = 0; st < NST; ++st)
                if ((pending >> st) & 1u) mbar_wait_bounded(&ring_bar[st], (pending_par >> st) & 1u);
            break;
        }
        // the ring is free: the next wave vector's first round lands while this one is
        // transformed
        if (i == 0 && tile + gridDim.x < a.n_tiles) issue_round(tile + gridDim.x, 0);
        float2 mean = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NWG; ++w) mean = cadd(mean, red2[w]);
        {
            const float rn = 1.0f / (float)N;
            mean = make_float2(mean.x * rn, mean.y * rn);
        }
#pragma unroll
        for (int u = 0; u < P; ++u)
            if (i + T * u < N) v[u] = csub(v[u], mean);
        // the mean-removed sequence into tensor memory: the even-bin transform and the power
        // sums take it from there instead of reading global memory again
        tmem_st_seq(t_seq, v);
        // ---- the three transforms through one copy of the code (the unrolled transform is
        // most of the kernel's instructions): pass 0, odd bins: DFT of g(t) e^{-i pi t / L},
        // |.|^2 parked in tensor memory; pass 1, even bins: DFT of g (from tensor memory);
        // pass 2, the inverse of Z = |X_even|^2 + i |X_odd|^2 as conj(DFT(conj Z)), fed in the
        // forward transforms' output order s1
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            if (pass == 0) {
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    v[u] = cmul(cmul(v[u], c_i), w64[u]);          // zero past N stays zero
                    if ((u & 7) == 7) hoist_fence();
                }
            } else if (pass == 1) {
                tmem_st_wait();
                tmem_ld_seq(t_seq, v);
            } else {
                float o2[P];
                tmem_st_wait();
                tmem_ld32(t_odd, o2);
#pragma unroll
                for (int u = 0; u < P; ++u) v[u] = make_float2(cabs2(v[u]), -o2[u]);
            }
            fft_cyclic3<L, false, 1, C::PAD, true>(v, pass == 2 ? s1 : i, i, 0, xs, tw1, twi, SyncBlock{});
            if (pass == 0) {
                float o2[P];
#pragma unroll
                for (int u = 0; u < P; ++u) o2[u] = cabs2(v[u]);
                tmem_st32(t_odd, o2);
            }
        }
#pragma unroll
        for (int u = 0; u < P; ++u) v[u].y = -v[u].y;   // conj: the inverse transform of Z
        // ---- Re C in cyclic order from the 2-for-1 split, into tensor memory
#pragma unroll
        for (int u = 0; u < P; ++u) xs[zs1 + T * u] = v[u];
        __syncthreads();
        {
            const float scale = 0.25f / (float)L;
            float rc[P];
#pragma unroll
            for (int u = 0; u < P; ++u) {
                const int m = i + T * u;
                const float2 z = xs[zsi + T * u];
                const float2 zr = xs[zslot((L - m) & (L - 1))];
                const float2 w = cmul(c_i, w64[u]);        // e^{-i pi m / L}
                rc[u] = scale * ((z.x + zr.x) + w.x * (z.y + zr.y) - w.y * (z.x - zr.x));
                if ((u & 7) == 7) hoist_fence();
            }
            tmem_st32(t_rec, rc);
        }
        __syncthreads();                                   // xs becomes the power sums
        // ---- |g - mean|^2 at padded positions t + t / 32, then the power sums of Eq. B1 as
        // a split scan: frames below h = 32 hc (hc = ceil(N / 64) chunks of 32) hold the
        // inclusive prefix sum, frames from h on the inclusive suffix sum, so that
        // P1(m) = S(N - m) and P2(m) = S(N) - S(m) are each read either directly or as S(N)
        // minus at most about half of it (no S(N) - S(m) cancellation at the largest lags,
        // where it grows like N / (N - m)).  Thread i owns frames 32 i .. 32 i + 31.
        tmem_ld_seq(t_seq, v);                             // zero past N
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int t = i + T * u;
            xf[t + (t >> 5)] = cabs2(v[u]);
        }
        __syncthreads();
        const int hc = (N + 63) / 64, h = 32 * hc;
        const bool fwd = i < hc;
        float acc = 0.f;
        if (fwd) {
#pragma unroll
            for (int jj = 0; jj < P; ++jj) acc += xf[i * (P + 1) + jj];
        } else {
#pragma unroll
            for (int jj = P - 1; jj >= 0; --jj) acc += xf[i * (P + 1) + jj];
        }
        const float acc_f = fwd ? acc : 0.f, acc_b = fwd ? 0.f : acc;
        float inc_f = acc_f, inc_b = acc_b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float yf = __shfl_up_sync(0xffffffffu, inc_f, o);
            const float yb = __shfl_down_sync(0xffffffffu, inc_b, o);
            if (lane >= o) inc_f += yf;
            if (lane + o < 32) inc_b += yb;
        }
        if (lane == 31) wsum[wg] = inc_f;
        if (lane == 0) wsum[NWG + wg] = inc_b;
        __syncthreads();
        float off = fwd ? inc_f - acc_f : inc_b - acc_b, total = 0.f;
#pragma unroll
        for (int w = 0; w < NWG; ++w) {
            const float xf_w = wsum[w], xb_w = wsum[NWG + w];
            if (fwd && w < wg) off += xf_w;
            if (!fwd && w > wg) off += xb_w;
            total += xf_w + xb_w;
        }
        if (fwd) {
#pragma unroll
            for (int jj = 0; jj < P; ++jj) {               // same order of additions as acc
                off += xf[i * (P + 1) + jj];
                xf[i * (P + 1) + jj] = off;
            }
        } else {
#pragma unroll
            for (int jj = P - 1; jj >= 0; --jj) {
                off += xf[i * (P + 1) + jj];
                xf[i * (P + 1) + jj] = off;
            }
        }
        // ---- the trailing lags by direct differences (Eq. 1): at most kd pairs each, from the
        // saved head and tail (t < N - m <= kd <= 32, t + m >= N - kd >= N - 32)
        float tl = 0.f;
        if (m_tail < N) {
            for (int t = 0; t < N - m_tail; ++t)
                tl += cabs2(csub(tail[t + m_tail - (N - 32)], head[t]));
            tl *= __frcp_rn((float)(N - m_tail));
            chk = fmaf(tl, 0.f, chk);
        }
        float rcv[P];
        tmem_st_wait();
        tmem_ld32(t_rec, rcv);                             // Re C(i + T u)
        __syncthreads();
        // ---- D(m) = (P1 + P2 - 2 Re C) / (N - m), m = i + T u, straight to global memory
        float* drow = D + (int64_t)public_q((int)sq, a) * N;
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            if (m >= N) break;
            float d = 0.f;
            if (m > 0 && m < m_lo) {
                // P1 = sum over t < N - m, P2 = sum over t >= m (Eq. B1)
                const int ta = N - 1 - m;
                const float p1 = ta < h ? xf[ta + (ta >> 5)] : total - xf[(ta + 1) + ((ta + 1) >> 5)];
                const float p2 = m >= h ? xf[m + (m >> 5)] : total - xf[(m - 1) + ((m - 1) >> 5)];
                d = __fdividef(p1 + p2 - 2.f * rcv[u], (float)(N - m));  // within 2 ulp
                chk = fmaf(d, 0.f, chk);
            } else if (m >= m_lo) {
                d = tl;                                    // m == m_tail
            }
            drow[m] = d;
        }
    }
    if (timed_out && i == 0) atomicOr(a.status, 2u);
    if (chk != chk) atomicOr(a.status, 1u);
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wg == 0) seq_tmem_free(tmem_slot);
}

// =====================================================================================
// L <= 256: one group per CTA, per-thread loads; two CTAs per SM
// =====================================================================================
// The first and last kd samples of each wave vector go through the exchange buffer before
// the transforms need it, and the trailing lags are taken from them there; the D rows are
// staged [q][m] and each warp copies whole rows out (lanes on consecutive lags).
template <int LOG2L>
struct TShape {
    static constexpr int L = 1 << LOG2L;
    using S = FftShape<L>;
    static constexpr int P = S::P, T = S::T;
    static constexpr int NT = 256;                         // threads per CTA
    static constexpr int QT = NT / T;                      // wave vectors per tile (>= 32)
    // most trailing lags taken by differences: the plan's kd = min(32, max(1, N / 32), N - 1)
    // never exceeds L / 32 (at least 1 where L >= 2); one lag per thread
    static constexpr int KD = L >= 32 ? L / 32 : (L >= 2 ? 1 : 0);
    static constexpr int KT = KD > 0 ? (KD + T - 1) / T : 0;
    static constexpr int DSTRIDE = L + 1;                  // D staging row stride
    static constexpr int RED = (P > 2 * T ? P : 2 * T);
    static constexpr size_t OFF_TW = 0;
    static constexpr size_t OFF_TW2 = OFF_TW + (T > 1 ? L : 0) * sizeof(float2);
    static constexpr size_t OFF_INV = OFF_TW2 + (size_t)L * sizeof(float2);
    static constexpr size_t OFF_XS = (OFF_INV + (size_t)L * sizeof(float) + 1023) & ~size_t(1023);
    static constexpr size_t OFF_AB = OFF_XS + (size_t)L * QT * sizeof(float2);
    static constexpr size_t OFF_MU = OFF_AB + (size_t)L * QT * sizeof(float);
    // at L = 64 the mean's partials and the prefix sums' row totals live in the upper half of
    // the exchange buffer (free in both phases: the power sums use its lower half as floats),
    // which makes room for a second CTA per SM (512^2 x 64: 0.114 -> 0.085 ms); at L = 32 the
    // same move measured slower than one CTA per SM with the registers of a whole SM half
    static constexpr bool RED_IN_XS = (L == 64);
    static constexpr size_t OFF_RED = RED_IN_XS ? OFF_XS + (size_t)L * QT * sizeof(float)
                                                : OFF_MU + (size_t)QT * sizeof(float2);
    static constexpr size_t BYTES = RED_IN_XS ? OFF_MU + (size_t)QT * sizeof(float2)
                                              : OFF_RED + (size_t)RED * QT * sizeof(float);
    static_assert(L <= 256 && QT >= 32, "per-thread-load kernel: L <= 256");
    static_assert(BYTES <= 232448, "temporal kernel shared memory exceeds 227 KB");
    static_assert((size_t)QT * DSTRIDE <= (size_t)2 * L * QT, "D staging must fit the exchange buffer");
    static_assert(2 * KD <= L, "the head and tail samples fit the exchange buffer");
    // two CTAs per SM where their shared memory allows (tensor memory: 256 columns each)
    static constexpr int CTAS_PER_SM = 2 * (BYTES + 1024) <= 233472 ? 2 : 1;
};

template <int LOG2L>
__global__ void __launch_bounds__(TShape<LOG2L>::NT, TShape<LOG2L>::CTAS_PER_SM)
temporal_sf_small_kernel(const float2* __restrict__ spec, float* __restrict__ D, TArgs a) {
    using C = TShape<LOG2L>;
    constexpr int L = C::L, P = C::P, T = C::T, NT = C::NT, QT = C::QT, KD = C::KD, KT = C::KT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw + C::OFF_TW);
    float2* tw2 = reinterpret_cast<float2*>(smem_raw + C::OFF_TW2);
    float* inv = reinterpret_cast<float*>(smem_raw + C::OFF_INV);
    float2* xs = reinterpret_cast<float2*>(smem_raw + C::OFF_XS);
    float* xf = reinterpret_cast<float*>(smem_raw + C::OFF_XS);     // same bytes as xs
    float* ab = reinterpret_cast<float*>(smem_raw + C::OFF_AB);
    float2* head = xs;                   // the first kd samples [t][QT], then the last kd,
    float2* tail = xs + KD * QT;         // while the exchange buffer is free
    float2* mu = reinterpret_cast<float2*>(smem_raw + C::OFF_MU);
    float* red = reinterpret_cast<float*>(smem_raw + C::OFF_RED);
    float2* red2 = reinterpret_cast<float2*>(smem_raw + C::OFF_RED);

    const int tid = threadIdx.x;
    // at P = 32 (L >= 32) every thread's mean-removed sequence waits in tensor memory for the
    // even-bin transform and the power sums (two fewer reads of the tile from L2); each of the
    // 8 warps owns 128 columns of its lane quarter, 256 per CTA
    constexpr bool STASH = (P == 32);
    __shared__ uint32_t tmem_slot;
    if constexpr (STASH) {
        if (tid < 32) long_tmem_alloc<NT>(&tmem_slot);
    }
    if constexpr (T > 1) {
        for (int k = tid; k < L; k += NT) tw[k] = a.tw[k];
    }
    for (int k = tid; k < L; k += NT) {
        tw2[k] = a.tw2[k];
        inv[k] = a.inv[k];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t t_seq = STASH ? tmem_slot + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) +
                                       (uint32_t)(tid >> 7) * 128u
                                 : 0u;

    const int ql = tid % QT;
    const int i = tid / QT;
    const int N = a.N;
    const int kd = a.kd;
    const int64_t q0 = a.q0, q1 = a.q1;
    const uint32_t nq32 = (uint32_t)a.n_q;   // N * n_q < 2^32 (checked at plan creation)
    const AddrInterleaved<QT> addr{ql};
    bool bad = false;

    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int64_t s = q0 + tile * QT + ql;
        const bool valid = s < q1;
        const float2* src = spec + (valid ? s : 0);

        // ---- prefetch the next tile of this CTA into L2: its DRAM fetch overlaps this tile
        {
            const int64_t sn = q0 + (tile + gridDim.x) * QT + ql;
            if (sn < q1) {
                const float2* pn = spec + sn;
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    const int t = i + T * u;
                    if (t < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(pn + (uint32_t)t * nq32));
                }
            }
        }

        // ---- load the time sequence (cyclic layout) and remove its mean
        float2 v[P];
        float2 part = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int t = i + T * u;
            v[u] = (valid && t < N) ? __ldg(src + (uint32_t)t * nq32) : make_float2(0.f, 0.f);
            part = cadd(part, v[u]);
        }
        red2[i * QT + ql] = part;
        __syncthreads();
        if (i == 0) {
            float2 sum = make_float2(0.f, 0.f);
            for (int ip = 0; ip < T; ++ip) sum = cadd(sum, red2[ip * QT + ql]);
            const float rn = 1.0f / (float)N;
            mu[ql] = make_float2(sum.x * rn, sum.y * rn);
        }
        __syncthreads();
        const float2 mean = mu[ql];
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int t = i + T * u;
            if (t < N) v[u] = csub(v[u], mean);
            if constexpr (KD > 0) {
                if (t < kd) head[t * QT + ql] = v[u];
                if (t >= N - kd && t < N) tail[(t - (N - kd)) * QT + ql] = v[u];
            }
        }
        if constexpr (STASH) tmem_st_seq<true>(t_seq, v);
        __syncthreads();   // head/tail visible; the mean buffer may be reused

        // ---- the last kd lags (N - m <= kd pairs) directly from Eq. 1, by differences of the
        // head and tail samples; kept in registers until the D rows are staged
        const int m_lo = (N - kd > 1) ? N - kd : 1;
        const int m_first = m_lo + ((i - m_lo) % T + T) % T;   // first lag >= m_lo owned by i
        float tl[KT > 0 ? KT : 1];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int m = m_first + k * T;
            float acc = 0.f;
            if (m < N) {
                const int base = m - (N - kd);
                for (int t = 0; t < N - m; ++t)
                    acc += cabs2(csub(tail[(t + base) * QT + ql], head[t * QT + ql]));
                acc *= inv[m];
            }
            tl[k] = acc;
        }
        if constexpr (KT > 0) __syncthreads();   // head and tail read: the transforms take xs

        // ---- odd bins: L-point DFT of g(t) e^{-i pi t / L}; |.|^2 parked in ab
#pragma unroll
        for (int u = 0; u < P; ++u) {
            v[u] = cmul(v[u], tw2[i + T * u]);
            if ((u & 7) == 7) hoist_fence();
        }
        fft_cyclic<L, false>(v, i, xs, addr, tw, SyncBlock{});
#pragma unroll
        for (int u = 0; u < P; ++u) ab[(i + T * u) * QT + ql] = cabs2(v[u]);

        // ---- even bins: L-point DFT of g (from tensor memory, or reloaded from L2 at P < 32)
        if constexpr (STASH) {
            tmem_st_wait();
            tmem_ld_seq<true>(t_seq, v);
        } else {
            const float2* src2 = opaque_ptr(src);
#pragma unroll
            for (int u = 0; u < P; ++u) {
                const int t = i + T * u;
                v[u] = (valid && t < N) ? csub(__ldg(src2 + (uint32_t)t * nq32), mean) : make_float2(0.f, 0.f);
            }
        }
        fft_cyclic<L, false>(v, i, xs, addr, tw, SyncBlock{});
#pragma unroll
        for (int u = 0; u < P; ++u) {
            v[u] = make_float2(cabs2(v[u]), ab[(i + T * u) * QT + ql]);
            if ((u & 7) == 7) hoist_fence();
        }

        // ---- inverse transform of Z = |X_even|^2 + i |X_odd|^2, then Re C(m) into ab
        fft_cyclic<L, true>(v, i, xs, addr, tw, SyncBlock{});
#pragma unroll
        for (int u = 0; u < P; ++u) xs[(i + T * u) * QT + ql] = v[u];
        __syncthreads();
        const float scale = 0.25f / (float)L;
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            const float2 z = v[u];
            const float2 zr = xs[((L - m) & (L - 1)) * QT + ql];
            const float2 w = tw2[m];                   // (cos(pi m/L), -sin(pi m/L))
            ab[m * QT + ql] = scale * ((z.x + zr.x) + w.x * (z.y + zr.y) - w.y * (z.x - zr.x));
            if ((u & 7) == 7) hoist_fence();
        }
        __syncthreads();   // partner reads done: the exchange buffer is free

        // ---- power terms: inclusive prefix sums S(t) of |g|^2.  Thread i owns the rows
        // r = i + T g of T consecutive t (at P = 32 |g|^2 comes from tensor memory through
        // the free exchange buffer [t][QT]; below that the tile is reloaded from L2), sums
        // them in registers, and adds the offset of the rows before it.
        if constexpr (STASH) {
            tmem_ld_seq<true>(t_seq, v);                   // zero past N and past q1
#pragma unroll
            for (int u = 0; u < P; ++u) xf[(i + T * u) * QT + ql] = cabs2(v[u]);
            __syncthreads();
        }
        const float2* src3 = opaque_ptr(src);
        constexpr int G = P / T;
        float rowv[G][T];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = i + T * g;
            float acc = 0.f;
#pragma unroll
            for (int jj = 0; jj < T; ++jj) {
                const int t = r * T + jj;
                if constexpr (STASH) {
                    acc += xf[t * QT + ql];
                } else {
                    if (valid && t < N) acc += cabs2(csub(__ldg(src3 + (uint32_t)t * nq32), mean));
                }
                rowv[g][jj] = acc;
            }
            red[r * QT + ql] = acc;
        }
        __syncthreads();
        float total = 0.f;
        float off[G];
#pragma unroll
        for (int g = 0; g < G; ++g) off[g] = 0.f;
#pragma unroll
        for (int rp = 0; rp < P; ++rp) {
            const float x = red[rp * QT + ql];
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (rp < i + T * g) off[g] += x;
            total += x;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = i + T * g;
#pragma unroll
            for (int jj = 0; jj < T; ++jj) xf[(r * T + jj) * QT + ql] = rowv[g][jj] + off[g];
        }
        __syncthreads();

        // ---- D(m) = (P1 + P2 - 2 Re C) / (N - m) for m < N - kd
        float dv[P];
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            float d = 0.f;
            if (m > 0 && m < N - kd) {
                const float p1 = xf[(N - 1 - m) * QT + ql];
                const float p2 = total - xf[(m - 1) * QT + ql];
                d = (p1 + p2 - 2.f * ab[m * QT + ql]) * inv[m];
            }
            dv[u] = d;
            if ((u & 7) == 7) hoist_fence();
        }
        __syncthreads();   // prefix reads done: the exchange buffer now stages D

        // ---- stage D as [q][m] (the trailing lags from registers), then each warp copies
        // whole rows out: lanes on consecutive lags
        constexpr int DS = C::DSTRIDE;
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            if (m < N) xf[ql * DS + m] = dv[u];
        }
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int m = m_first + k * T;
            if (m < N) xf[ql * DS + m] = tl[k];
        }
        __syncthreads();
        {
            const int64_t left = q1 - (q0 + tile * QT);
            const int nr = left < QT ? (int)left : QT;
            const int lane = tid & 31;
#pragma unroll 2
            for (int r = tid >> 5; r < nr; r += NT / 32) {
                float* drow = D + (int64_t)public_q((int)(q0 + tile * QT + r), a) * N;
                for (int m = lane; m < N; m += 32) {
                    const float d = xf[r * DS + m];
                    bad |= !isfinite(d);
                    drow[m] = d;
                }
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(a.status, 1u);
    if constexpr (STASH) {
        tmem_st_wait();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid < 32) long_tmem_free<NT>(tmem_slot);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// Corner turn of the stored wave vectors [q0, q1) into blocks of 16 contiguous over time:
// blk[(b N + t) 16 + c] = spec[t n_q + q0 + 16 b + c], zero past q1.  One block of 256 frames
// per CTA; reads and writes are 128-byte rows.
__global__ void __launch_bounds__(256)
blocked_copy_kernel(const float2* __restrict__ spec, float2* __restrict__ blk, int N, int64_t n_q,
                    int64_t q0, int64_t q1) {
    const int64_t b = blockIdx.x;
    const int t0 = blockIdx.y * 256;
    const int64_t qb = q0 + 16 * b;
    for (int idx = threadIdx.x; idx < 256 * 16; idx += 256) {
        const int t = t0 + (idx >> 4), c = idx & 15;
        if (t >= N) break;
        const int64_t q = qb + c;
        blk[(b * N + t) * 16 + c] = q < q1 ? __ldg(spec + (int64_t)t * n_q + q) : make_float2(0.f, 0.f);
    }
}

// 3D view of the blocked copy as float32 [nb][N][32]; boxes of 2 qg floats x 256 rows x 1
// block.
bool make_blocked_map(CUtensorMap* map, const float2* blk, int64_t nb, int N, int qg) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[3] = {32, (cuuint64_t)N, (cuuint64_t)nb};
    const cuuint64_t strides[2] = {32 * sizeof(float), (cuuint64_t)N * 32 * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * qg), 256, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(blk), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The blocked copy of [q0, q1) in the plan workspace (made here unless step one wrote it:
// pre), or nullptr when the plan does not use it (or has no workspace yet: the kernels then
// read the [t][q] spectrum).
float2* blocked_copy(const ddm_plan_s* p, const float2* spec, cudaStream_t s, bool pre, bool* ok) {
    *ok = true;
    if (!p->blocked || !p->workspace) return nullptr;
    float2* blk = reinterpret_cast<float2*>(static_cast<char*>(p->workspace) + p->blk_offset);
    if (pre) return blk;                               // step one wrote the blocks already
    const int64_t nb = (p->q1 - p->q0 + 15) / 16;
    dim3 grid((unsigned)nb, (unsigned)((p->d.N + 255) / 256));
    blocked_copy_kernel<<<grid, 256, 0, s>>>(spec, blk, p->d.N, p->n_q, p->q0, p->q1);
    *ok = cudaGetLastError() == cudaSuccess;
    return blk;
}

// 2D view of the spectrum as float32 [N][2 n_q]; boxes of 2 qg floats (qg complex) x 256
// rows; rows >= N and columns >= 2 n_q read as zero.
bool make_spectrum_map(CUtensorMap* map, const float2* spec, int64_t n_q, int N, int qg) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * n_q), (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * n_q * sizeof(float))};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * qg), 256};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(spec), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void fill_args(TArgs& a, const ddm_plan_s* p, float* D, int qt) {
    a.N = p->d.N;
    a.kd = p->kd;
    a.H = p->d.H;
    a.Wh = p->Wh;
    a.crop = p->kc > 0 ? 1 : (p->nk > 0 ? 2 : 0);
    a.kx0 = p->kx0;
    a.nk = p->nk;
    a.vec4 = (p->d.N % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
    a.blocked = 0;
    a.fix = (p->d.precision == DDM_PREC_FP32_FP64FIX) ? p->fix_lags : 0;
    a.n_q = p->n_q;
    a.q0 = p->q0;
    a.q1 = p->q1;
    a.n_tiles = (p->q1 - p->q0 + qt - 1) / qt;
    a.tw = p->tw_t;
    a.tw2 = p->tw2;
    a.inv = p->inv;
    a.status = p->dev_status;
}

template <int LOG2L, bool FIXUP, int NGROUPS>
ddm_status launch_grouped(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s) {
    using C = GShape<LOG2L, NGROUPS>;
    const bool full = p->d.N == C::L && p->kd == C::T;   // the FULL instance's premise
    if ((reinterpret_cast<uintptr_t>(spec) & 15) != 0) return DDM_ERR_INVALID_ARG;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if (!make_spectrum_map(&tmap, spec, p->n_q, p->d.N, C::QG)) return DDM_ERR_CUDA;
    TArgs a;
    fill_args(a, p, D, C::QG);
    auto k = full ? temporal_sf_kernel<LOG2L, NGROUPS, FIXUP, true> : temporal_sf_kernel<LOG2L, NGROUPS, FIXUP, false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    const int64_t ctas = (a.n_tiles + C::NG - 1) / C::NG;
    const int64_t grid = ctas < p->n_sm ? ctas : p->n_sm;
    k<<<(unsigned)grid, C::NT, C::BYTES, s>>>(D, a, tmap);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

template <int LOG2L, bool FIXUP>
ddm_status launch_long(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s, bool pre_blocked) {
    using C = LShape<LOG2L>;
    if ((reinterpret_cast<uintptr_t>(spec) & 15) != 0 || !p->tw_tin || !p->tw_long) return DDM_ERR_INVALID_ARG;
    bool ok = true;
    const float2* blk = blocked_copy(p, spec, s, pre_blocked, &ok);
    if (!ok) return DDM_ERR_CUDA;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if (blk ? !make_blocked_map(&tmap, blk, (p->q1 - p->q0 + 15) / 16, p->d.N, C::QG)
            : !make_spectrum_map(&tmap, spec, p->n_q, p->d.N, C::QG))
        return DDM_ERR_CUDA;
    TArgs a;
    fill_args(a, p, D, C::QG);
    a.blocked = blk != nullptr;
    const bool full = p->d.N == C::L && p->kd == 32;     // the FULL instance's premise
    auto k = full ? temporal_sf_long_kernel<LOG2L, FIXUP, true> : temporal_sf_long_kernel<LOG2L, FIXUP, false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return DDM_ERR_CUDA;
    LTables tb;
    tb.quarter = p->tw_long;                      // [L/4] quarter wave, then [T] ci, then [32] w64
    tb.ci = p->tw_long + p->L / 4;
    tb.w64 = p->tw_long + p->L / 4 + p->L / 32;
    tb.inner = p->tw_tin;
    const int64_t slots = (int64_t)C::CTAS_PER_SM * p->n_sm;
    const int64_t grid = a.n_tiles < slots ? a.n_tiles : slots;
    k<<<(unsigned)grid, C::NT, C::BYTES, s>>>(D, a, tmap, tb);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

ddm_status launch_xl(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s, bool pre_blocked) {
    using C = XLShape;
    if (!p->tw_tin || !p->tw_long || p->L != C::L) return DDM_ERR_INVALID_ARG;
    bool ok = true;
    const float2* blk = blocked_copy(p, spec, s, pre_blocked, &ok);
    if (!ok) return DDM_ERR_CUDA;
    if ((reinterpret_cast<uintptr_t>(blk ? blk : spec) & 15) != 0) return DDM_ERR_INVALID_ARG;
    CUtensorMap tmap;                             // boxes of 2 wave vectors x 256 frames
    memset(&tmap, 0, sizeof(tmap));
    if (blk ? !make_blocked_map(&tmap, blk, (p->q1 - p->q0 + 15) / 16, p->d.N, 2)
            : !make_spectrum_map(&tmap, spec, p->n_q, p->d.N, 2))
        return DDM_ERR_CUDA;
    TArgs a;
    fill_args(a, p, D, 1);
    a.blocked = blk != nullptr;
    const bool full = p->d.N == C::L && p->kd == 32;     // the FULL instance's premise
    auto k = full ? temporal_sf_xl_kernel<true> : temporal_sf_xl_kernel<false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return DDM_ERR_CUDA;
    XLTables tb;                                  // tw_long: [L/4] quarter, [T] ci, [32] w64, [64] lo, [L/64] hi
    tb.ci = p->tw_long + p->L / 4;
    tb.w64 = tb.ci + p->L / 32;
    tb.lo = tb.w64 + 32;
    tb.hi = tb.lo + 64;
    tb.inner = p->tw_tin;
    const int64_t grid = a.n_tiles < p->n_sm ? a.n_tiles : p->n_sm;
    k<<<(unsigned)grid, C::NT, C::BYTES, s>>>(D, a, tb, tmap);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

template <int LOG2L>
ddm_status launch_small(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s) {
    using C = TShape<LOG2L>;
    TArgs a;
    fill_args(a, p, D, C::QT);
    auto k = temporal_sf_small_kernel<LOG2L>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    if (C::CTAS_PER_SM > 1 &&
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return DDM_ERR_CUDA;
    const int64_t slots = (int64_t)C::CTAS_PER_SM * p->n_sm;
    const int64_t grid = a.n_tiles < slots ? a.n_tiles : slots;
    k<<<(unsigned)grid, C::NT, C::BYTES, s>>>(spec, D, a);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace

bool encode_f32_tensor_map(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                           const cuuint64_t* strides, const cuuint32_t* box) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || rank < 1 || rank > 5) return false;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_wait_selftest(unsigned* status, long long cap_cycles, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(status, cap_cycles);
    return cudaGetLastError();
}

ddm_status launch_temporal(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s, bool pre_blocked) {
    const bool fix = p->d.precision == DDM_PREC_FP32_FP64FIX;
    switch (ilog2(p->L)) {
        case 0: return launch_small<0>(p, spec, D, s);
        case 1: return launch_small<1>(p, spec, D, s);
        case 2: return launch_small<2>(p, spec, D, s);
        case 3: return launch_small<3>(p, spec, D, s);
        case 4: return launch_small<4>(p, spec, D, s);
        case 5: return launch_small<5>(p, spec, D, s);
        case 6: return launch_small<6>(p, spec, D, s);
        case 7: return launch_small<7>(p, spec, D, s);
        case 8: return launch_small<8>(p, spec, D, s);
        // groups per CTA.  Measured at 512x512x1024 (L = 1024) when each tile was copied three
        // times: 1 group of 512 threads (128-byte TMA rows, lockstep) 1.13 ms, 2 groups 1.05 ms,
        // 4 groups (32-byte rows) 1.15 ms.  With one copy per tile (tensor-memory stash) four
        // groups of 128 threads lead by about 1 % (0.773 against 0.781 ms); at L = 512 eight
        // groups of 64 do not (0.377 against 0.375 ms), four stay.
        case 9: return fix ? launch_grouped<9, true, 4>(p, spec, D, s) : launch_grouped<9, false, 4>(p, spec, D, s);
        case 10: return fix ? launch_grouped<10, true, 4>(p, spec, D, s) : launch_grouped<10, false, 4>(p, spec, D, s);
        case 11: return fix ? launch_long<11, true>(p, spec, D, s, pre_blocked) : launch_long<11, false>(p, spec, D, s, pre_blocked);
        case 12: return fix ? launch_long<12, true>(p, spec, D, s, pre_blocked) : launch_long<12, false>(p, spec, D, s, pre_blocked);
        case 13: return fix ? launch_long<13, true>(p, spec, D, s, pre_blocked) : launch_long<13, false>(p, spec, D, s, pre_blocked);
        case 14: return fix ? DDM_ERR_UNSUPPORTED : launch_xl(p, spec, D, s, pre_blocked);
        default: return DDM_ERR_UNSUPPORTED;
    }
}

}  // namespace ddm
