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
// Corner turn: a CTA owns QT consecutive stored wave vectors; each warp load instruction
// reads whole 128-byte row segments F[t][q0 .. q0+QT) of the [t][q] spectrum, and the
// thread mapping (q fastest, then transform thread i) turns them into per-q sequences
// in registers (thread i of q holds t = i + T u).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

// ---- TMA (bulk tensor copies) and mbarrier helpers, inline PTX
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
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"(map), "r"(x),
                 "r"(y) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// A bounded wait on the tile barrier: about two seconds of polling, then false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 4000000000LL) return false;
    }
    return true;
}

template <int LOG2L>
struct TShape {
    static constexpr int L = 1 << LOG2L;
    using S = FftShape<L>;
    static constexpr int P = S::P, T = S::T;
    static constexpr int NT = (T == 32) ? 512 : 256;      // threads per CTA
    static constexpr int QT = NT / T;                      // wave vectors per tile
    static constexpr int KD = (L / 2 < 32) ? L / 2 : 32;  // max directly evaluated lags
    // D staging row stride: conflict-free writes from the cyclic layout, and 16-byte
    // aligned rows (float4 stores) when QT == 16
    static constexpr int DSTRIDE = L + (QT >= 32 ? 1 : (QT == 16 ? 4 : 32 / QT));
    static constexpr int RED = (P > 2 * T ? P : 2 * T);
    // tiles of 16 wave vectors and L >= 256 frames arrive by TMA: boxes of 16 complex x 256
    // frames (32 KB) straight into the exchange buffer, which has the same [t][16] layout
    static constexpr bool USE_TMA = (QT == 16) && (L >= 256);
    static constexpr int BOX_T = 256;
    static constexpr int NBOX = L / BOX_T;
    static constexpr int FIX_MAX = 8;             // most leading lags the FP64 fixup redoes
    // shared memory carve-up (bytes)
    static constexpr size_t OFF_TW = 0;
    static constexpr size_t OFF_TW2 = OFF_TW + (T > 1 ? L : 0) * sizeof(float2);
    static constexpr size_t OFF_INV = OFF_TW2 + (size_t)L * sizeof(float2);
    static constexpr size_t OFF_XS = (OFF_INV + (size_t)L * sizeof(float) + 1023) & ~size_t(1023);
    static constexpr size_t OFF_AB = OFF_XS + (size_t)L * QT * sizeof(float2);
    static constexpr size_t OFF_HT = OFF_AB + (size_t)L * QT * sizeof(float);
    static constexpr size_t OFF_MU = OFF_HT + (size_t)2 * (KD > 0 ? KD : 1) * QT * sizeof(float2);
    static constexpr size_t OFF_RED = OFF_MU + (size_t)QT * sizeof(float2);
    static constexpr size_t BYTES = OFF_RED + (size_t)RED * QT * sizeof(float);
    static_assert(BYTES <= 232448, "temporal kernel shared memory exceeds 227 KB");
    static_assert((size_t)QT * DSTRIDE <= (size_t)2 * L * QT, "D staging must fit the exchange buffer");
};

struct TArgs {
    int N;            // frames
    int kd;           // directly evaluated trailing lags (<= KD, < N)
    int H, Wh, lwh;   // for the storage -> public q map (lwh = log2 Wh)
    int64_t n_q;      // stored wave vectors = spectrum frame stride
    int64_t n_tiles;
    int vec4;         // D rows 16-byte aligned (N % 4 == 0 and D aligned): float4 stores
    int fix;          // FP64-fixup tier: lags 1..fix by direct differences (0 = off)
    const float2* tw;
    const float2* tw2;
    const float* inv;
    unsigned* status;
};

// storage index -> public q = ky * (Wh + 1) + kx (Wh = W/2 is a power of two)
__device__ __forceinline__ int public_q(int s, int H, int Wh, int lwh) {
    const int main = H << lwh;
    if (s < main) return (s >> lwh) * (Wh + 1) + (s & (Wh - 1));
    return (s - main) * (Wh + 1) + Wh;
}

template <int LOG2L, bool FIXUP>
__global__ void __launch_bounds__(TShape<LOG2L>::NT, TShape<LOG2L>::NT == 512 ? 1 : 2)
temporal_sf_kernel(const float2* __restrict__ spec, float* __restrict__ D, TArgs a,
                   const __grid_constant__ CUtensorMap tmap) {
    using C = TShape<LOG2L>;
    constexpr int L = C::L, P = C::P, T = C::T, NT = C::NT, QT = C::QT, KD = C::KD;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw + C::OFF_TW);
    float2* tw2 = reinterpret_cast<float2*>(smem_raw + C::OFF_TW2);
    float* inv = reinterpret_cast<float*>(smem_raw + C::OFF_INV);
    float2* xs = reinterpret_cast<float2*>(smem_raw + C::OFF_XS);
    float* xf = reinterpret_cast<float*>(smem_raw + C::OFF_XS);     // same bytes as xs
    float* ab = reinterpret_cast<float*>(smem_raw + C::OFF_AB);
    float2* head = reinterpret_cast<float2*>(smem_raw + C::OFF_HT);
    float2* tail = head + (KD > 0 ? KD : 1) * QT;
    float2* mu = reinterpret_cast<float2*>(smem_raw + C::OFF_MU);
    float* red = reinterpret_cast<float*>(smem_raw + C::OFF_RED);
    float2* red2 = reinterpret_cast<float2*>(smem_raw + C::OFF_RED);

    const int tid = threadIdx.x;
    __shared__ uint64_t tile_bar;
    uint32_t bar_phase = 0;
    if constexpr (C::USE_TMA) {
        if (tid == 0) {
            mbar_init(&tile_bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    if constexpr (T > 1) {
        for (int k = tid; k < L; k += NT) tw[k] = a.tw[k];
    }
    for (int k = tid; k < L; k += NT) {
        tw2[k] = a.tw2[k];
        inv[k] = a.inv[k];
    }
    __syncthreads();

    const int ql = tid % QT;
    const int i = tid / QT;
    const int N = a.N;
    const int kd = a.kd;
    const int64_t nq = a.n_q;
    const uint32_t nq32 = (uint32_t)nq;   // N * n_q < 2^32 (checked at plan creation)
    const AddrInterleaved<QT> addr{ql};
    bool bad = false;
    bool timed_out = false;
    // Copy tile `tl` into xs ([t][16] complex, zeros beyond N and n_q) and wait for it.
    // Precondition: every thread is done with xs (a barrier was just passed).
    auto load_tile = [&](int64_t tl) -> bool {
        if (tid == 0) {
            fence_proxy_async();
            mbar_expect_tx(&tile_bar, (uint32_t)(C::NBOX * C::BOX_T * QT * sizeof(float2)));
#pragma unroll
            for (int b = 0; b < C::NBOX; ++b)
                tma_load_2d(xs + b * C::BOX_T * QT, &tmap, (int)(2 * tl * QT), b * C::BOX_T, &tile_bar);
        }
        const bool ok = mbar_wait_bounded(&tile_bar, bar_phase);
        bar_phase ^= 1u;
        // the decision to give up must be the same in every thread (barriers follow)
        return __syncthreads_or(ok ? 0 : 1) == 0;
    };

    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int64_t s = tile * QT + ql;
        const bool valid = s < nq;
        const float2* src = spec + (valid ? s : 0);

        // ---- prefetch the next tile of this CTA into L2: its DRAM fetch overlaps this tile
        if constexpr (C::USE_TMA) {
            const int64_t tn = tile + gridDim.x;
            if (tid < C::NBOX && tn < a.n_tiles)
                tma_prefetch_2d(&tmap, (int)(2 * tn * QT), tid * C::BOX_T);
        } else {
            const int64_t sn = (tile + gridDim.x) * QT + ql;
            if (sn < nq) {
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
        if constexpr (C::USE_TMA) {
            if (!load_tile(tile)) { timed_out = true; break; }
#pragma unroll
            for (int u = 0; u < P; ++u) {
                v[u] = xs[(i + T * u) * QT + ql];
                part = cadd(part, v[u]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < P; ++u) {
                const int t = i + T * u;
                v[u] = (valid && t < N) ? __ldg(src + (uint32_t)t * nq32) : make_float2(0.f, 0.f);
                part = cadd(part, v[u]);
            }
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
            if (t < kd) head[t * QT + ql] = v[u];
            if (t >= N - kd && t < N) tail[(t - (N - kd)) * QT + ql] = v[u];
        }
        __syncthreads();   // head/tail visible; the mean buffer may be reused

        // ---- odd bins: L-point DFT of g(t) e^{-i pi t / L}; |.|^2 parked in ab
#pragma unroll
        for (int u = 0; u < P; ++u) {
            v[u] = cmul(v[u], tw2[i + T * u]);
            if ((u & 7) == 7) hoist_fence();
        }
        fft_cyclic<L, false>(v, i, xs, addr, tw, SyncBlock{});
#pragma unroll
        for (int u = 0; u < P; ++u) ab[(i + T * u) * QT + ql] = cabs2(v[u]);

        // ---- even bins: L-point DFT of g (reloaded; the tile is still in L2)
        if constexpr (C::USE_TMA) {
            if (!load_tile(tile)) { timed_out = true; break; }
#pragma unroll
            for (int u = 0; u < P; ++u) {
                const int t = i + T * u;
                v[u] = (t < N) ? csub(xs[t * QT + ql], mean) : make_float2(0.f, 0.f);
            }
            __syncthreads();   // tile read: the exchange buffer is reused by the transform
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
        // r = i + T g of T consecutive t (reloaded from L2; each load instruction still
        // covers whole 128-byte segments), sums them in registers, and adds the offset of
        // the rows before it.
        const float2* src3 = opaque_ptr(src);
        constexpr int G = P / T;
        float rowv[G][T];
        if constexpr (C::USE_TMA) {
            if (!load_tile(tile)) { timed_out = true; break; }
        }
        // FP64-fixup tier (tile in shared memory): over its rows each thread also sums
        // |F(t+m) - F(t)|^2 for m = 1..fix, the direct, cancellation-free form of Eq. 1,
        // keeping F(t .. t+FIX_MAX) in a sliding register window
        constexpr int FM = C::FIX_MAX;
        const int fix = (FIXUP && C::USE_TMA) ? a.fix : 0;
        float fixp[FM];
#pragma unroll
        for (int k = 0; k < FM; ++k) fixp[k] = 0.f;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = i + T * g;
            float acc = 0.f;
            float2 win[FM + 1];
            if constexpr (FIXUP && C::USE_TMA) {
                if (fix > 0) {
#pragma unroll
                    for (int k = 0; k < FM; ++k) {
                        const int tk = r * T + k;
                        win[k] = tk < N ? xs[tk * QT + ql] : make_float2(0.f, 0.f);
                    }
                }
            }
#pragma unroll
            for (int jj = 0; jj < T; ++jj) {
                const int t = r * T + jj;
                float e = 0.f;
                if constexpr (FIXUP && C::USE_TMA) {
                    if (fix > 0) {
                        win[FM] = (t + FM < N) ? xs[(t + FM) * QT + ql] : make_float2(0.f, 0.f);
#pragma unroll
                        for (int m = 1; m <= FM; ++m)
                            if (m <= fix && t + m < N) fixp[m - 1] += cabs2(csub(win[m], win[0]));
                        if (t < N) e = cabs2(csub(win[0], mean));
#pragma unroll
                        for (int k = 0; k < FM; ++k) win[k] = win[k + 1];
                    } else {
                        if (t < N) e = cabs2(csub(xs[t * QT + ql], mean));
                    }
                } else if constexpr (C::USE_TMA) {
                    if (t < N) e = cabs2(csub(xs[t * QT + ql], mean));
                } else {
                    if (valid && t < N) e = cabs2(csub(__ldg(src3 + (uint32_t)t * nq32), mean));
                }
                acc += e;
                rowv[g][jj] = acc;
            }
            red[r * QT + ql] = acc;
        }
        __syncthreads();
        // the tile has been read: the upper half of the exchange buffer takes the fixup partials
        float* fixpart = xf + (size_t)L * QT;                  // [m][i][ql]
        if (FIXUP && fix > 0) {
#pragma unroll
            for (int k = 0; k < FM; ++k)
                if (k < fix) fixpart[(k * T + i) * QT + ql] = fixp[k];
        }
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
        // partials of lag m = i + 1 summed in FP64 over the T threads of each sequence;
        // D(m) parked in the row-total buffer (free now) until the D rows are staged
        if (FIXUP && fix > 0 && i < fix && i + 1 < N) {
            double sum = 0.0;
            for (int ip = 0; ip < T; ++ip) sum += (double)fixpart[(i * T + ip) * QT + ql];
            red[i * QT + ql] = (float)(sum / (double)(N - 1 - i));
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

        // ---- stage D as [q][m]; the last kd lags (N - m <= kd pairs) come directly from
        // Eq. 1 by differences of the stored head and tail samples
        constexpr int DS = C::DSTRIDE;
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int m = i + T * u;
            if (m < N) xf[ql * DS + m] = dv[u];
        }
        {
            const int m_lo = (N - kd > 1) ? N - kd : 1;
            int m = m_lo + ((i - m_lo) % T + T) % T;     // first lag >= m_lo owned by i
            for (; m < N; m += T) {
                float acc = 0.f;
                const int base = m - (N - kd);
                for (int t = 0; t < N - m; ++t)
                    acc += cabs2(csub(tail[(t + base) * QT + ql], head[t * QT + ql]));
                xf[ql * DS + m] = acc * inv[m];
            }
        }
        if (FIXUP && fix > 0 && i < fix && i + 1 < N - kd) xf[ql * DS + i + 1] = red[i * QT + ql];
        __syncthreads();
        if (QT == 16 && a.vec4) {
            const int n4 = N >> 2;
            const int total4 = QT * n4;
            for (int f = tid; f < total4; f += NT) {
                const int r = f / n4, j = f - r * n4;
                const int64_t sr = tile * QT + r;
                if (sr >= nq) break;
                const float4 d = *reinterpret_cast<const float4*>(xf + r * DS + 4 * j);
                bad |= !(isfinite(d.x) && isfinite(d.y) && isfinite(d.z) && isfinite(d.w));
                float* drow = D + (int64_t)public_q((int)sr, a.H, a.Wh, a.lwh) * N;
                reinterpret_cast<float4*>(drow)[j] = d;
            }
        } else {
            for (int r = 0; r < QT; ++r) {
                const int64_t sr = tile * QT + r;
                if (sr >= nq) break;
                float* drow = D + (int64_t)public_q((int)sr, a.H, a.Wh, a.lwh) * N;
                for (int m = tid; m < N; m += NT) {
                    const float d = xf[r * DS + m];
                    bad |= !isfinite(d);
                    drow[m] = d;
                }
            }
        }
        __syncthreads();
    }
    if (timed_out) {
        // a tile copy never completed: report it; give an outstanding copy a last bounded
        // chance to land before the CTA's shared memory goes away
        atomicOr(a.status, 2u);
        mbar_wait_bounded(&tile_bar, bar_phase);
    }
    if (bad) atomicOr(a.status, 1u);
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

// 2D view of the spectrum as float32 [N][2 n_q]; boxes of 32 floats (16 complex) x 256 rows;
// rows >= N and columns >= 2 n_q read as zero.
bool make_spectrum_map(CUtensorMap* map, const float2* spec, int64_t n_q, int N) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * n_q), (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * n_q * sizeof(float))};
    const cuuint32_t box[2] = {32, 256};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(spec), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int LOG2L, bool FIXUP>
ddm_status launch_t(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s) {
    using C = TShape<LOG2L>;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if constexpr (C::USE_TMA) {
        if ((reinterpret_cast<uintptr_t>(spec) & 15) != 0) return DDM_ERR_INVALID_ARG;
        if (!make_spectrum_map(&tmap, spec, p->n_q, p->d.N)) return DDM_ERR_CUDA;
    }
    TArgs a;
    a.N = p->d.N;
    a.kd = p->kd;
    a.H = p->d.H;
    a.Wh = p->Wh;
    a.lwh = ilog2(p->Wh);
    a.vec4 = (p->d.N % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
    a.fix = (p->d.precision == DDM_PREC_FP32_FP64FIX) ? p->fix_lags : 0;
    a.n_q = p->n_q;
    a.n_tiles = (p->n_q + C::QT - 1) / C::QT;
    a.tw = p->tw_t;
    a.tw2 = p->tw2;
    a.inv = p->inv;
    a.status = p->dev_status;
    auto k = temporal_sf_kernel<LOG2L, FIXUP>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    const int64_t grid = a.n_tiles < p->n_sm ? a.n_tiles : p->n_sm;
    k<<<(unsigned)grid, C::NT, C::BYTES, s>>>(spec, D, a, tmap);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace

ddm_status launch_temporal(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s) {
    const bool fix = p->d.precision == DDM_PREC_FP32_FP64FIX;
    switch (ilog2(p->L)) {
        case 0: return launch_t<0, false>(p, spec, D, s);
        case 1: return launch_t<1, false>(p, spec, D, s);
        case 2: return launch_t<2, false>(p, spec, D, s);
        case 3: return launch_t<3, false>(p, spec, D, s);
        case 4: return launch_t<4, false>(p, spec, D, s);
        case 5: return launch_t<5, false>(p, spec, D, s);
        case 6: return launch_t<6, false>(p, spec, D, s);
        case 7: return launch_t<7, false>(p, spec, D, s);
        case 8: return launch_t<8, false>(p, spec, D, s);
        case 9: return fix ? launch_t<9, true>(p, spec, D, s) : launch_t<9, false>(p, spec, D, s);
        case 10: return fix ? launch_t<10, true>(p, spec, D, s) : launch_t<10, false>(p, spec, D, s);
        default: return DDM_ERR_UNSUPPORTED;
    }
}

}  // namespace ddm
