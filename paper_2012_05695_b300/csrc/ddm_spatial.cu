// Step one of the method (Sec. 2): the real-to-complex 2D DFT of every frame, FP32.
//
// Row pass: two real rows a, b form one complex row z = a + i b; an L = W point FFT
// gives Z, and A[k] = (Z[k] + conj Z[W-k]) / 2, B[k] = (Z[k] - conj Z[W-k]) / (2i) for
// k = 0..W/2.  A[0] and A[W/2] are real, so a row is stored as W/2 complex values with
// the Nyquist value in the imaginary part of slot 0.
// Column pass: an H-point FFT down every stored column.  Column 0 holds
// c[y] = A_y[0] + i A_y[W/2], two real columns, and is unpacked with the same identity
// into the kx = 0 and kx = W/2 spectra.
//
// Spectrum layout per frame (complex64): [ky][kx] for kx < W/2, then the kx = W/2
// column [ky]; frame stride H * (W/2 + 1).  The row pass writes in place of the final
// spectrum and the column pass transforms it in place.
//
// Frame 0 is subtracted from every frame first (exact for uint16): D depends only on
// differences between frames, and removing the static image keeps the FP32 transform's
// rounding relative to the changing part of the signal.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

template <typename In>
__device__ __forceinline__ float pixel_diff(const In* f, const In* r, size_t idx, bool sub);
template <>
__device__ __forceinline__ float pixel_diff<uint16_t>(const uint16_t* f, const uint16_t* r,
                                                     size_t idx, bool sub) {
    const int a = (int)__ldg(f + idx);
    return (float)(sub ? a - (int)__ldg(r + idx) : a);
}
template <>
__device__ __forceinline__ float pixel_diff<float>(const float* f, const float* r, size_t idx,
                                                  bool sub) {
    const float a = __ldg(f + idx);
    return sub ? a - __ldg(r + idx) : a;
}

constexpr int kRowThreads = 256;

// grid: (H/2 / pairs_per_block, N); block: kRowThreads.  W = L points per row.
template <int W, typename In>
__global__ void __launch_bounds__(kRowThreads)
row_r2c_kernel(const In* __restrict__ frames, float2* __restrict__ spec, int H,
               size_t frame_stride, int subtract_ref, const float2* __restrict__ tw_g) {
    using S = FftShape<W>;
    constexpr int P = S::P, T = S::T;
    constexpr int PAIRS = kRowThreads / T;             // row pairs per block
    constexpr int STRIDE = AddrPadded<W>::stride();
    extern __shared__ float2 smem[];
    float2* tw = smem;                                  // W entries (T > 1)
    float2* xs = smem + (T > 1 ? W : 0);                // PAIRS * STRIDE

    const int tid = threadIdx.x;
    if constexpr (T > 1) {
        for (int k = tid; k < W; k += kRowThreads) tw[k] = tw_g[k];
    }
    const int i = tid % T;
    const int j = tid / T;
    const int pair = blockIdx.x * PAIRS + j;
    const int t = blockIdx.y;
    const bool active = (2 * pair + 1) < H;
    const In* f = frames + (size_t)t * H * W;
    const size_t ra = (size_t)(2 * pair) * W, rb = ra + W;

    float2 v[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
        const int x = i + T * u;
        if (active) {
            v[u].x = pixel_diff<In>(f, frames, ra + x, subtract_ref);
            v[u].y = pixel_diff<In>(f, frames, rb + x, subtract_ref);
        } else {
            v[u] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();   // twiddle table ready
    AddrPadded<W> addr{j * STRIDE};
    fft_cyclic<W, false>(v, i, xs, addr, tw, SyncBlock{});

    // split the two real rows: needs Z[W - k]
#pragma unroll
    for (int u = 0; u < P; ++u) xs[addr(i + T * u)] = v[u];
    __syncthreads();
    if (active) {
        float2* outa = spec + (size_t)t * frame_stride + (size_t)(2 * pair) * (W / 2);
        float2* outb = outa + W / 2;
#pragma unroll
        for (int u = 0; u < (P + 1) / 2; ++u) {
            const int k = i + T * u;
            if (k >= W / 2) break;
            const float2 z = xs[addr(k)];
            if (k == 0) {
                const float2 zn = xs[addr(W / 2)];
                outa[0] = make_float2(z.x, zn.x);        // A[0], A[W/2] (both real)
                outb[0] = make_float2(z.y, zn.y);        // B[0], B[W/2]
            } else {
                const float2 zr = xs[addr(W - k)];
                outa[k] = make_float2(0.5f * (z.x + zr.x), 0.5f * (z.y - zr.y));
                outb[k] = make_float2(0.5f * (z.y + zr.y), 0.5f * (zr.x - z.x));
            }
        }
    }
}

// grid: (Wh / QC, N); block: QC * T threads.  H = L points per column, QC columns.
template <int H, int QC>
__global__ void __launch_bounds__(QC * FftShape<H>::T, (QC * FftShape<H>::T) >= 512 ? 1 : (QC * FftShape<H>::T) >= 256 ? 2 : 4)
col_c2c_kernel(float2* __restrict__ spec, int Wh, size_t frame_stride,
               const float2* __restrict__ tw_g) {
    using S = FftShape<H>;
    constexpr int P = S::P, T = S::T, NT = QC * T;
    extern __shared__ float2 smem[];
    float2* tw = smem;                                   // H entries (T > 1)
    float2* xs = smem + (T > 1 ? H : 0);                 // H * QC

    const int tid = threadIdx.x;
    if constexpr (T > 1) {
        for (int k = tid; k < H; k += NT) tw[k] = tw_g[k];
    }
    const int ql = tid % QC;
    const int i = tid / QC;
    const int kx = blockIdx.x * QC + ql;
    const int t = blockIdx.y;
    float2* base = spec + (size_t)t * frame_stride;
    // 32-bit element offsets (a frame holds < 2^32 elements): cheap strided addressing
    const uint32_t off0 = (uint32_t)(i * Wh + kx), step = (uint32_t)(T * Wh);

    float2 v[P];
#pragma unroll
    for (int u = 0; u < P; ++u) v[u] = base[off0 + (uint32_t)u * step];
    __syncthreads();
    AddrInterleaved<QC> addr{ql};
    fft_cyclic<H, false>(v, i, xs, addr, tw, SyncBlock{});

    base = opaque_ptr(base);
    if (blockIdx.x != 0) {
#pragma unroll
        for (int u = 0; u < P; ++u) base[off0 + (uint32_t)u * step] = v[u];
        return;
    }
    // block 0 holds the packed DC/Nyquist column in ql = 0: unpack it
#pragma unroll
    for (int u = 0; u < P; ++u) xs[addr(i + T * u)] = v[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < P; ++u) {
        const int ky = i + T * u;
        if (ql != 0) {
            base[(size_t)ky * Wh + kx] = v[u];
        } else {
            const float2 c = v[u];
            const float2 cr = xs[addr((H - ky) & (H - 1))];
            // F0 = (C[ky] + conj C[-ky]) / 2 ; FN = (C[ky] - conj C[-ky]) / (2i)
            base[(size_t)ky * Wh] = make_float2(0.5f * (c.x + cr.x), 0.5f * (c.y - cr.y));
            base[(size_t)H * Wh + ky] = make_float2(0.5f * (c.y + cr.y), 0.5f * (cr.x - c.x));
        }
    }
}

template <int W, typename In>
cudaError_t launch_rows(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    using S = FftShape<W>;
    constexpr int PAIRS = kRowThreads / S::T;
    const int H = p->d.H, N = p->d.N;
    const int pairs = H / 2;
    dim3 grid((pairs + PAIRS - 1) / PAIRS, N);
    const size_t smem = sizeof(float2) * ((S::T > 1 ? W : 0) + (size_t)PAIRS * AddrPadded<W>::stride());
    auto k = row_r2c_kernel<W, In>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, kRowThreads, smem, s>>>((const In*)frames, spec, H, spectrum_frame_stride(p),
                                      p->d.subtract_ref, p->tw_row);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_cols(const ddm_plan_s* p, float2* spec, cudaStream_t s) {
    using S = FftShape<H>;
    const int Wh = p->Wh, N = p->d.N;
    const size_t frame_stride = spectrum_frame_stride(p);
    auto go = [&](auto qc_tag) -> cudaError_t {
        constexpr int QC = decltype(qc_tag)::value;
        dim3 grid(Wh / QC, N);
        const size_t smem = sizeof(float2) * ((S::T > 1 ? H : 0) + (size_t)H * QC);
        auto k = col_c2c_kernel<H, QC>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, QC * S::T, smem, s>>>(spec, Wh, frame_stride, p->tw_col);
        return cudaGetLastError();
    };
    if (Wh >= 16) return go(std::integral_constant<int, 16>{});
    if (Wh == 8) return go(std::integral_constant<int, 8>{});
    if (Wh == 4) return go(std::integral_constant<int, 4>{});
    if (Wh == 2) return go(std::integral_constant<int, 2>{});
    return go(std::integral_constant<int, 1>{});
}

template <typename In>
cudaError_t dispatch_rows(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    switch (p->d.W) {
        case 2: return launch_rows<2, In>(p, frames, spec, s);
        case 4: return launch_rows<4, In>(p, frames, spec, s);
        case 8: return launch_rows<8, In>(p, frames, spec, s);
        case 16: return launch_rows<16, In>(p, frames, spec, s);
        case 32: return launch_rows<32, In>(p, frames, spec, s);
        case 64: return launch_rows<64, In>(p, frames, spec, s);
        case 128: return launch_rows<128, In>(p, frames, spec, s);
        case 256: return launch_rows<256, In>(p, frames, spec, s);
        case 512: return launch_rows<512, In>(p, frames, spec, s);
        case 1024: return launch_rows<1024, In>(p, frames, spec, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_cols(const ddm_plan_s* p, float2* spec, cudaStream_t s) {
    switch (p->d.H) {
        case 2: return launch_cols<2>(p, spec, s);
        case 4: return launch_cols<4>(p, spec, s);
        case 8: return launch_cols<8>(p, spec, s);
        case 16: return launch_cols<16>(p, spec, s);
        case 32: return launch_cols<32>(p, spec, s);
        case 64: return launch_cols<64>(p, spec, s);
        case 128: return launch_cols<128>(p, spec, s);
        case 256: return launch_cols<256>(p, spec, s);
        case 512: return launch_cols<512>(p, spec, s);
        case 1024: return launch_cols<1024>(p, spec, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t spectrum_frame_stride(const ddm_plan_s* p) { return (size_t)p->n_q; }

ddm_status launch_spatial(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    cudaError_t e = (p->d.dtype == DDM_IN_U16) ? dispatch_rows<uint16_t>(p, frames, spec, s)
                                               : dispatch_rows<float>(p, frames, spec, s);
    if (e != cudaSuccess) return DDM_ERR_CUDA;
    e = dispatch_cols(p, spec, s);
    return e == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace ddm
