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
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

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
    // shared memory carve-up (bytes)
    static constexpr size_t OFF_TW = 0;
    static constexpr size_t OFF_TW2 = OFF_TW + (T > 1 ? L : 0) * sizeof(float2);
    static constexpr size_t OFF_INV = OFF_TW2 + (size_t)L * sizeof(float2);
    static constexpr size_t OFF_XS = (OFF_INV + (size_t)L * sizeof(float) + 15) & ~size_t(15);
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

template <int LOG2L>
__global__ void __launch_bounds__(TShape<LOG2L>::NT, TShape<LOG2L>::NT == 512 ? 1 : 2)
temporal_sf_kernel(const float2* __restrict__ spec, float* __restrict__ D, TArgs a) {
    using C = TShape<LOG2L>;
    constexpr int L = C::L, P = C::P, T = C::T, NT = C::NT, QT = C::QT, KD = C::KD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
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

    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int64_t s = tile * QT + ql;
        const bool valid = s < nq;
        const float2* src = spec + (valid ? s : 0);

        // ---- prefetch the next tile of this CTA into L2: its DRAM fetch overlaps this tile
        {
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
        const float2* src2 = opaque_ptr(src);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int t = i + T * u;
            v[u] = (valid && t < N) ? csub(__ldg(src2 + (uint32_t)t * nq32), mean) : make_float2(0.f, 0.f);
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
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = i + T * g;
            float acc = 0.f;
#pragma unroll
            for (int jj = 0; jj < T; ++jj) {
                const int t = r * T + jj;
                float e = 0.f;
                if (valid && t < N) e = cabs2(csub(__ldg(src3 + (uint32_t)t * nq32), mean));
                acc += e;
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
    if (bad) atomicOr(a.status, 1u);
}

template <int LOG2L>
ddm_status launch_t(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s) {
    using C = TShape<LOG2L>;
    TArgs a;
    a.N = p->d.N;
    a.kd = p->kd;
    a.H = p->d.H;
    a.Wh = p->Wh;
    a.lwh = ilog2(p->Wh);
    a.vec4 = (p->d.N % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
    a.n_q = p->n_q;
    a.n_tiles = (p->n_q + C::QT - 1) / C::QT;
    a.tw = p->tw_t;
    a.tw2 = p->tw2;
    a.inv = p->inv;
    a.status = p->dev_status;
    auto k = temporal_sf_kernel<LOG2L>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    const int64_t grid = a.n_tiles < p->n_sm ? a.n_tiles : p->n_sm;
    k<<<(unsigned)grid, C::NT, C::BYTES, s>>>(spec, D, a);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace

ddm_status launch_temporal(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s) {
    switch (ilog2(p->L)) {
        case 0: return launch_t<0>(p, spec, D, s);
        case 1: return launch_t<1>(p, spec, D, s);
        case 2: return launch_t<2>(p, spec, D, s);
        case 3: return launch_t<3>(p, spec, D, s);
        case 4: return launch_t<4>(p, spec, D, s);
        case 5: return launch_t<5>(p, spec, D, s);
        case 6: return launch_t<6>(p, spec, D, s);
        case 7: return launch_t<7>(p, spec, D, s);
        case 8: return launch_t<8>(p, spec, D, s);
        case 9: return launch_t<9>(p, spec, D, s);
        case 10: return launch_t<10>(p, spec, D, s);
        default: return DDM_ERR_UNSUPPORTED;
    }
}

}  // namespace ddm
