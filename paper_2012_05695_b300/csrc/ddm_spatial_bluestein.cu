// Step one (Sec. 2) for frame sides that are not powers of two (e.g. a 600 x 800 camera),
// and for power-of-two sides of 2048 (the same 2048-point transform without the chirp):
// the n-point DFTs of the rows and columns by Bluestein's chirp-z identity,
//     X[k] = conj(c_k) sum_j (z_j conj(c_j)) c_{k-j},   c_j = exp(i pi j^2 / n),
// a cyclic convolution of length M = 2^ceil(log2(2n - 1)) done with the power-of-two
// transforms of ddm_fft.cuh: a = z conj(c) zero-padded to M, A = DFT_M(a), A * F with
// F = DFT_M(c placed circularly) / M (a plan table), y = inverse DFT_M, X[k] = y[k] conj(c_k).
// Everything around the transform is as in the power-of-two kernels (ddm_spatial.cu): two
// real rows per complex row transform, the Nyquist value packed into slot 0, the column
// pass in place with the packed DC / Nyquist column unpacked by the block that holds it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

template <int M>
struct BShape {
    static constexpr int P = 32, T = M / P;
    static constexpr int NT = 256;
    static constexpr int QT = NT / T;                      // transforms per CTA
    static constexpr bool THREE = M >= 2048;               // three-pass transform
    static constexpr int PAD = THREE ? ((QT == 2) ? 4 : 2) : 0;
    // exchange elements: the transforms' scratch, also the staging and the partner step
    static constexpr size_t X_TWO = T > 1 ? (size_t)(M + M / T) * QT     // AddrPaddedInterleaved
                                          : (size_t)M * QT;              // (M = 32: no exchange)
    static constexpr size_t X_THREE = (size_t)P * (T + PAD) * QT > (size_t)M * QT
                                          ? (size_t)P * (T + PAD) * QT : (size_t)M * QT;
    static constexpr size_t XE = THREE ? X_THREE : X_TWO;
    // row stride of the staged rows and of the output X of transform ql (at ql WS + k):
    // WS = 32 / QT (mod 16) float2 (odd when QT >= 32), so that a warp's QT x (32 / QT) lanes
    // fall on distinct bank pairs
    static constexpr int WS_MOD = QT >= 32 ? 1 : 32 / QT;
    static constexpr int ws(int W) { return W + ((WS_MOD - W % 16) % 16 + 16) % 16; }
    static_assert(M >= 32 && M <= 2048 && QT * T == NT, "Bluestein lengths 3 .. 1024");
};

// The cyclic convolution at the heart of Bluestein's identity, on QT transforms held in
// the cyclic layout (thread i of transform ql holds a[i + T u]).  Returns the logical index
// li of the result: the thread then holds y[li + T u].
// DIRECT (a power-of-two side of M = 2048 points): the forward transform alone, no chirp.
template <int M, bool DIRECT, typename Sync>
__device__ __forceinline__ int bluestein_core(float2 (&v)[32], int i, int ql, float2* xs,
                                              const ddm_bluestein& b, const float2* filt,
                                              const float2* tw, Sync sync) {
    using C = BShape<M>;
    constexpr int T = C::T, QT = C::QT;
    if constexpr (DIRECT) {
        static_assert(C::THREE, "direct transforms only at M = 2048");
        const TwiddleTable tw1{tw, T};
        fft_cyclic3<M, false, QT, C::PAD>(v, i, i, ql, xs, tw1, b.twin, sync);
        return fft3_sigma(i, 32, T / 32);
    } else if constexpr (!C::THREE) {
        const AddrPaddedInterleaved<QT, T> addr{ql};
        fft_cyclic<M, false>(v, i, xs, addr, tw, sync);
#pragma unroll
        for (int u = 0; u < 32; ++u) v[u] = cmul(v[u], filt[i + T * u]);
        fft_cyclic<M, true>(v, i, xs, addr, tw, sync);
        return i;
    } else {
        constexpr int R = T / 32;
        const TwiddleTable tw1{tw, T};
        fft_cyclic3<M, false, QT, C::PAD>(v, i, i, ql, xs, tw1, b.twin, sync);
        const int s1 = fft3_sigma(i, 32, R);
#pragma unroll
        for (int u = 0; u < 32; ++u) v[u] = cmul(v[u], filt[s1 + T * u]);
        fft_cyclic3<M, true, QT, C::PAD, true>(v, s1, i, ql, xs, tw1, b.twin, sync);
        return s1;
    }
}

// ------------------------------------------------------------------ rows (W not 2^k)
// grid: (ceil(H/2 / QT), N); block: 256.  CTA: QT row pairs of one frame.
template <int M, bool DIRECT, typename In>
__global__ void __launch_bounds__(256, 2)
row_bluestein_kernel(const In* __restrict__ frames, float2* __restrict__ spec, int H, int W,
                     size_t frame_stride, int subtract_ref, ddm_bluestein b) {
    using C = BShape<M>;
    constexpr int T = C::T, QT = C::QT, NT = C::NT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* xs = reinterpret_cast<float2*>(smem_raw);
    float2* chirp = xs + C::XE;                            // W entries
    float2* filt = chirp + 1024;                           // M entries
    float2* tw = filt + M;                                 // M entries (pass twiddles)

    const int tid = threadIdx.x;
    if constexpr (!DIRECT)
        for (int k = tid; k < W; k += NT) chirp[k] = b.chirp[k];
    for (int k = tid; k < M; k += NT) {
        if constexpr (!DIRECT) filt[k] = b.filt[k];
        if constexpr (C::T > 1) tw[k] = b.tw[k];         // M = 32: one thread per transform
    }
    const int t = blockIdx.y;
    const int pair0 = blockIdx.x * QT;
    const int npairs = min(QT, H / 2 - pair0);
    // the CTA's rows, frame 0 subtracted in integers, staged as floats [pair][W] complex
    const In* src = frames + ((size_t)t * H + 2 * pair0) * W;
    const In* ref = frames + (size_t)(2 * pair0) * W;
    float2* stage = xs;                                    // QT * WS complex <= exchange size
    const int WS = C::ws(W);
#pragma unroll 4
    for (int e = tid; e < npairs * W; e += NT) {
        const int q = e / W, x = e - q * W;
        const size_t ia = (size_t)(2 * q) * W + x, ib = ia + W;
        float a, bb;
        if constexpr (sizeof(In) == 2) {
            a = (float)((int)src[ia] - (subtract_ref ? (int)ref[ia] : 0));
            bb = (float)((int)src[ib] - (subtract_ref ? (int)ref[ib] : 0));
        } else {
            a = subtract_ref ? (float)src[ia] - (float)ref[ia] : (float)src[ia];
            bb = subtract_ref ? (float)src[ib] - (float)ref[ib] : (float)src[ib];
        }
        stage[q * WS + x] = make_float2(a, bb);
    }
    __syncthreads();
    const int ql = tid % QT, i = tid / QT;
    const bool active = ql < npairs;
    float2 v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int n = i + T * u;
        const float2 z = (active && n < W) ? stage[ql * WS + n] : make_float2(0.f, 0.f);
        v[u] = (DIRECT || n >= W) ? z : cmul_conj(z, chirp[n]);
    }
    __syncthreads();                                       // staging read: the exchange reuses it
    const int li = bluestein_core<M, DIRECT>(v, i, ql, xs, b, filt, tw, SyncBlock{});
    // X[k] = y[k] conj(c_k), k < W, into row ql for the two-real-rows unpacking
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int k = li + T * u;
        if (k < W) xs[ql * WS + k] = DIRECT ? v[u] : cmul_conj(v[u], chirp[k]);
    }
    __syncthreads();
    const int Wh = W / 2;
    for (int e = tid; e < npairs * Wh; e += NT) {
        const int q = e / Wh, k = e - q * Wh;
        float2* outa = spec + (size_t)t * frame_stride + (size_t)(2 * (pair0 + q)) * Wh;
        float2* outb = outa + Wh;
        const float2 z = xs[q * WS + k];
        if (k == 0) {
            const float2 zn = xs[q * WS + Wh];
            outa[0] = make_float2(z.x, zn.x);
            outb[0] = make_float2(z.y, zn.y);
        } else {
            const float2 zr = xs[q * WS + W - k];
            outa[k] = make_float2(0.5f * (z.x + zr.x), 0.5f * (z.y - zr.y));
            outb[k] = make_float2(0.5f * (z.y + zr.y), 0.5f * (zr.x - z.x));
        }
    }
}

// --------------------------------------------------------------- columns (H not 2^k)
// grid: (ceil(Wh / QT), N); block: 256.  In place, QT stored columns of one frame.
template <int M, bool DIRECT>
__global__ void __launch_bounds__(256, 2)
col_bluestein_kernel(float2* __restrict__ spec, int H, int Wh, size_t frame_stride, ddm_bluestein b,
                     SpecOut out) {
    using C = BShape<M>;
    constexpr int T = C::T, QT = C::QT, NT = C::NT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* xs = reinterpret_cast<float2*>(smem_raw);
    float2* chirp = xs + C::XE;
    float2* filt = chirp + 1024;
    float2* tw = filt + M;

    const int tid = threadIdx.x;
    if constexpr (!DIRECT)
        for (int k = tid; k < H; k += NT) chirp[k] = b.chirp[k];
    for (int k = tid; k < M; k += NT) {
        if constexpr (!DIRECT) filt[k] = b.filt[k];
        if constexpr (C::T > 1) tw[k] = b.tw[k];         // M = 32: one thread per transform
    }
    __syncthreads();
    const int ql = tid % QT, i = tid / QT;
    const int kx = blockIdx.x * QT + ql;
    const bool valid = kx < Wh;
    const int t = blockIdx.y;
    float2* base = spec + (size_t)t * frame_stride;
    float2 v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int y = i + T * u;
        const float2 z = (valid && y < H) ? base[(size_t)y * Wh + kx] : make_float2(0.f, 0.f);
        v[u] = (DIRECT || y >= H) ? z : cmul_conj(z, chirp[y]);
    }
    const int li = bluestein_core<M, DIRECT>(v, i, ql, xs, b, filt, tw, SyncBlock{});
    if constexpr (!DIRECT) {
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int k = li + T * u;
            if (k < H) v[u] = cmul_conj(v[u], chirp[k]);
        }
    }
    if (blockIdx.x != 0) {
        if (valid) {
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int ky = li + T * u;
                if (ky < H) out.put(base, t, (int64_t)ky * Wh + kx, v[u]);
            }
        }
        return;
    }
    // the block holding kx = 0 unpacks the packed DC / Nyquist column (partner ky <-> H - ky)
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int ky = li + T * u;
        if (ky < H) xs[ky * QT + ql] = v[u];
    }
    __syncthreads();
    if (!valid) return;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int ky = li + T * u;
        if (ky >= H) continue;
        if (ql != 0) {
            out.put(base, t, (int64_t)ky * Wh + kx, v[u]);
        } else {
            const float2 c = v[u];
            const float2 cr = xs[(ky == 0 ? 0 : H - ky) * QT];
            out.put(base, t, (int64_t)ky * Wh, make_float2(0.5f * (c.x + cr.x), 0.5f * (c.y - cr.y)));
            out.put(base, t, (int64_t)H * Wh + ky, make_float2(0.5f * (c.y + cr.y), 0.5f * (cr.x - c.x)));
        }
    }
}

template <int M>
size_t bluestein_smem() {
    return sizeof(float2) * (BShape<M>::XE + 1024 + 2 * (size_t)M);
}

template <int M, typename In, bool DIRECT = false>
cudaError_t rows_t(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    using C = BShape<M>;
    auto k = row_bluestein_kernel<M, DIRECT, In>;
    const size_t smem = bluestein_smem<M>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p->d.H / 2 + C::QT - 1) / C::QT, p->d.N);
    k<<<grid, C::NT, smem, s>>>((const In*)frames, spec, p->d.H, p->d.W, (size_t)p->n_q, p->d.subtract_ref,
                                 p->blue_w);
    return cudaGetLastError();
}

template <int M, bool DIRECT = false>
cudaError_t cols_t(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out) {
    using C = BShape<M>;
    auto k = col_bluestein_kernel<M, DIRECT>;
    const size_t smem = bluestein_smem<M>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p->Wh + C::QT - 1) / C::QT, p->d.N);
    k<<<grid, C::NT, smem, s>>>(spec, p->d.H, p->Wh, (size_t)p->n_q, p->blue_h, out);
    return cudaGetLastError();
}

template <typename In>
cudaError_t rows_dispatch(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    if (p->blue_w.M == p->blue_w.n) return p->blue_w.M == 2048 ? rows_t<2048, In, true>(p, frames, spec, s)
                                                                : cudaErrorInvalidValue;
    switch (p->blue_w.M) {
        case 32: return rows_t<32, In>(p, frames, spec, s);
        case 64: return rows_t<64, In>(p, frames, spec, s);
        case 128: return rows_t<128, In>(p, frames, spec, s);
        case 256: return rows_t<256, In>(p, frames, spec, s);
        case 512: return rows_t<512, In>(p, frames, spec, s);
        case 1024: return rows_t<1024, In>(p, frames, spec, s);
        case 2048: return rows_t<2048, In>(p, frames, spec, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_rows_bluestein(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    return p->d.dtype == DDM_IN_U16 ? rows_dispatch<uint16_t>(p, frames, spec, s)
                                    : rows_dispatch<float>(p, frames, spec, s);
}

cudaError_t launch_cols_bluestein(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out) {
    if (p->blue_h.M == p->blue_h.n) return p->blue_h.M == 2048 ? cols_t<2048, true>(p, spec, s, out)
                                                                : cudaErrorInvalidValue;
    switch (p->blue_h.M) {
        case 32: return cols_t<32>(p, spec, s, out);
        case 64: return cols_t<64>(p, spec, s, out);
        case 128: return cols_t<128>(p, spec, s, out);
        case 256: return cols_t<256>(p, spec, s, out);
        case 512: return cols_t<512>(p, spec, s, out);
        case 1024: return cols_t<1024>(p, spec, s, out);
        case 2048: return cols_t<2048>(p, spec, s, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ddm
