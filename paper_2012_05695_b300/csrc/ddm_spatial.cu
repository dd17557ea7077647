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
#include <string.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

// shared-memory address and bounded mbarrier wait (about two seconds of polling, then false),
// for the staged copies of this file's kernels
__device__ __forceinline__ uint32_t cvta_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init_s(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cvta_smem(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait_s(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(cvta_smem(bar)), "r"(parity) : "memory");
        if (ok) return true;
        if (clock64() - t0 > 4000000000LL) return false;
    }
}

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
// COLRANGE: a kx-column range plan, whose output goes to the range's own store (SpecOut
// put_col) and whose grid starts at column block bx0.
// TMA: the block's H x QC values arrive by TMA copies (3-D tensor map over the row output as
// float32 [N][H][2 Wh], boxes of 256 rows x 2 QC floats) into the exchange region, in its
// [row][QC] layout, instead of per-thread strided loads.  At H = 512 the TMA instance asks for
// three CTAs per SM (80 registers): with the loads gone its registers allow it, and three
// CTAs hide the copies better than two (512x512x1024 step one 0.655 -> 0.622 ms).  At
// H = 1024 the block is 8 columns (256 threads, 72 KB), three CTAs per SM, in place of one
// 512-thread CTA of 16 columns (1024x1024x512 step one 1.60 -> 1.31 ms); at H = 256 six
// 128-thread CTAs per SM instead of four (256x256x1024 0.20 -> 0.195 ms).
template <int H, int QC, bool COLRANGE, bool TMA = false>
__global__ void __launch_bounds__(QC * FftShape<H>::T, (QC * FftShape<H>::T) >= 512 ? 1 : (QC * FftShape<H>::T) >= 256 ? (TMA && (H == 512 || H == 1024) ? 3 : 2) : (TMA && H == 256 ? 6 : 4))
col_c2c_kernel(float2* __restrict__ spec, int Wh, size_t frame_stride,
               const float2* __restrict__ tw_g, SpecOut out, int bx0,
               const __grid_constant__ CUtensorMap tmap, unsigned* status) {
    using S = FftShape<H>;
    constexpr int P = S::P, T = S::T, NT = QC * T;
    extern __shared__ __align__(1024) float2 smem[];
    float2* tw = smem;                                   // H entries (T > 1)
    float2* xs = smem + (T > 1 ? H : 0);                 // H * QC

    const int tid = threadIdx.x;
    const int ql = tid % QC;
    const int i = tid / QC;
    const int bx = COLRANGE ? (int)blockIdx.x + bx0 : (int)blockIdx.x;   // column block
    const int kx = bx * QC + ql;
    const int t = blockIdx.y;
    float2* base = spec + (size_t)t * frame_stride;
    // 32-bit element offsets (a frame holds < 2^32 elements): cheap strided addressing
    const uint32_t off0 = (uint32_t)(i * Wh + kx), step = (uint32_t)(T * Wh);

    float2 v[P];
    if constexpr (TMA) {
        static_assert(H % 256 == 0 && (QC * 8) % 16 == 0 && ((T > 1 ? H : 0) * 8) % 128 == 0,
                      "TMA staging: boxes of 256 rows, 16-byte rows, 128-byte aligned destinations");
        __shared__ uint64_t bar;
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cvta_smem(&bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cvta_smem(&bar)),
                         "r"((uint32_t)(H * QC * sizeof(float2))) : "memory");
#pragma unroll
            for (int b = 0; b < H / 256; ++b)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4}], [%5];"
                    ::"r"(cvta_smem(xs + (size_t)b * 256 * QC)), "l"(&tmap), "r"(2 * bx * QC), "r"(b * 256),
                    "r"(t), "r"(cvta_smem(&bar)) : "memory");
        }
        if constexpr (T > 1) {
            for (int k = tid; k < H; k += NT) tw[k] = tw_g[k];
        }
        __syncthreads();                                 // the twiddles; the barrier is armed
        const bool ok = mbar_wait_s(&bar, 0);
#pragma unroll
        for (int u = 0; u < P; ++u) v[u] = ok ? xs[(i + T * u) * QC + ql] : make_float2(0.f, 0.f);
        if (!ok) {
            // report it (status bit 2); the copies get a last bounded chance to land before
            // the region becomes the exchange
            if (tid == 0) atomicOr(status, 2u);
            mbar_wait_s(&bar, 0);
        }
    } else {
        if constexpr (T > 1) {
            for (int k = tid; k < H; k += NT) tw[k] = tw_g[k];
        }
#pragma unroll
        for (int u = 0; u < P; ++u) v[u] = base[off0 + (uint32_t)u * step];
    }
    __syncthreads();
    AddrInterleaved<QC> addr{ql};
    fft_cyclic<H, false>(v, i, xs, addr, tw, SyncBlock{});

    base = opaque_ptr(base);
    if (bx != 0) {
        if constexpr (COLRANGE) {
            // row ky = i + T u of column kx in the range's store [ky][kx - kx0]
            float2* cb = out.col + (size_t)t * (size_t)out.n_qc + (size_t)(kx - out.kx0);
            const uint32_t c0 = (uint32_t)(i * out.nk), cstep = (uint32_t)(T * out.nk);
#pragma unroll
            for (int u = 0; u < P; ++u) cb[c0 + (uint32_t)u * cstep] = v[u];
        } else if (!out.blk) {
#pragma unroll
            for (int u = 0; u < P; ++u) base[off0 + (uint32_t)u * step] = v[u];
        } else {
#pragma unroll
            for (int u = 0; u < P; ++u) out.put(base, t, off0 + (uint32_t)u * step, v[u]);
        }
        return;
    }
    // block 0 holds the packed DC/Nyquist column in ql = 0: unpack it
#pragma unroll
    for (int u = 0; u < P; ++u) xs[addr(i + T * u)] = v[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < P; ++u) {
        const int ky = i + T * u;
        auto put = [&](int64_t q, float2 val) {
            if constexpr (COLRANGE) out.put_col(t, q, val);
            else out.put(base, t, q, val);
        };
        if (ql != 0) {
            put((int64_t)ky * Wh + kx, v[u]);
        } else {
            const float2 c = v[u];
            const float2 cr = xs[addr((H - ky) & (H - 1))];
            // F0 = (C[ky] + conj C[-ky]) / 2 ; FN = (C[ky] - conj C[-ky]) / (2i)
            put((int64_t)ky * Wh, make_float2(0.5f * (c.x + cr.x), 0.5f * (c.y - cr.y)));
            put((int64_t)H * Wh + ky, make_float2(0.5f * (c.y + cr.y), 0.5f * (cr.x - c.x)));
        }
    }
}

// Low-frequency restriction (Sec. 3): H-point FFTs down the columns kx = 0..kc of the
// row-pass output [N][H][kc + 1]; only ky' = 0..kc and -kc..-1 are kept, written to the
// cropped spectrum [N][(2 kc + 1)(kc + 1)] (rows in that ky' order, kx inner).
// grid: (ceil((kc + 1) / QC), N); block: QC * T threads.
template <int H, int QC>
__global__ void __launch_bounds__(QC * FftShape<H>::T)
col_crop_kernel(const float2* __restrict__ inter, float2* __restrict__ spec, int kc,
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
    const int cols = kc + 1;
    const int kx = blockIdx.x * QC + ql;
    const bool valid = kx <= kc;
    const int t = blockIdx.y;
    const float2* src = inter + (size_t)t * H * cols + (valid ? kx : 0);
    float2 v[P];
#pragma unroll
    for (int u = 0; u < P; ++u)
        v[u] = valid ? __ldg(src + (size_t)(i + T * u) * cols) : make_float2(0.f, 0.f);
    __syncthreads();
    AddrInterleaved<QC> addr{ql};
    fft_cyclic<H, false>(v, i, xs, addr, tw, SyncBlock{});
    if (!valid) return;                                  // after the transform's last barrier
    float2* dst = spec + (size_t)t * (size_t)(2 * kc + 1) * cols + kx;
#pragma unroll
    for (int u = 0; u < P; ++u) {
        const int ky = i + T * u;
        const int r = ky <= kc ? ky : (ky >= H - kc ? ky - H + 2 * kc + 1 : -1);
        if (r >= 0) dst[(size_t)r * cols] = v[u];
    }
}

template <int H>
cudaError_t launch_cols_crop(const ddm_plan_s* p, float2* spec, cudaStream_t s) {
    using S = FftShape<H>;
    constexpr int QC = 16;
    const int kc = p->kc;
    dim3 grid((kc + 1 + QC - 1) / QC, p->d.N);
    const size_t smem = sizeof(float2) * ((S::T > 1 ? H : 0) + (size_t)H * QC);
    auto k = col_crop_kernel<H, QC>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, QC * S::T, smem, s>>>(p->crop_inter, spec, kc, p->tw_col);
    return cudaGetLastError();
}

cudaError_t dispatch_cols_crop(const ddm_plan_s* p, float2* spec, cudaStream_t s) {
    switch (p->d.H) {
        case 4: return launch_cols_crop<4>(p, spec, s);
        case 8: return launch_cols_crop<8>(p, spec, s);
        case 16: return launch_cols_crop<16>(p, spec, s);
        case 32: return launch_cols_crop<32>(p, spec, s);
        case 64: return launch_cols_crop<64>(p, spec, s);
        case 128: return launch_cols_crop<128>(p, spec, s);
        case 256: return launch_cols_crop<256>(p, spec, s);
        case 512: return launch_cols_crop<512>(p, spec, s);
        case 1024: return launch_cols_crop<1024>(p, spec, s);
        default: return cudaErrorInvalidValue;
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
cudaError_t launch_cols(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out) {
    using S = FftShape<H>;
    const int Wh = p->Wh, N = p->d.N;
    const size_t frame_stride = spectrum_frame_stride(p);
    auto go = [&](auto qc_tag) -> cudaError_t {
        constexpr int QC = decltype(qc_tag)::value;
        // a kx-column range transforms only its own column blocks
        const int nblk = p->nk > 0 ? p->nk / QC : Wh / QC, bx0 = p->nk > 0 ? p->kx0 / QC : 0;
        dim3 grid(nblk, N);
        const size_t smem = sizeof(float2) * ((S::T > 1 ? H : 0) + (size_t)H * QC);
        auto k = p->nk > 0 ? col_c2c_kernel<H, QC, true> : col_c2c_kernel<H, QC, false>;
        CUtensorMap tmap;
        memset(&tmap, 0, sizeof(tmap));
        if constexpr ((QC == 16 || (H == 1024 && QC == 8)) && H % 256 == 0) {
            // TMA staging: 16-byte rows and frames (Wh, frame stride even), aligned spectrum
            const cuuint64_t dims[3] = {(cuuint64_t)(2 * Wh), (cuuint64_t)H, (cuuint64_t)N};
            const cuuint64_t strides[2] = {(cuuint64_t)Wh * sizeof(float2), (cuuint64_t)frame_stride * sizeof(float2)};
            const cuuint32_t box[3] = {(cuuint32_t)(2 * QC), 256u, 1u};
            if (Wh % 2 == 0 && frame_stride % 2 == 0 && reinterpret_cast<uintptr_t>(spec) % 16 == 0 &&
                encode_f32_tensor_map(&tmap, spec, 3, dims, strides, box))
                k = p->nk > 0 ? col_c2c_kernel<H, QC, true, true> : col_c2c_kernel<H, QC, false, true>;
        }
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        k<<<grid, QC * S::T, smem, s>>>(spec, Wh, frame_stride, p->tw_col, out, bx0, tmap, p->dev_status);
        return cudaGetLastError();
    };
    if (H == 1024 && Wh >= 16) return go(std::integral_constant<int, 8>{});   // 3 CTAs per SM
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

cudaError_t dispatch_cols(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out = {}) {
    switch (p->d.H) {
        case 2: return launch_cols<2>(p, spec, s, out);
        case 4: return launch_cols<4>(p, spec, s, out);
        case 8: return launch_cols<8>(p, spec, s, out);
        case 16: return launch_cols<16>(p, spec, s, out);
        case 32: return launch_cols<32>(p, spec, s, out);
        case 64: return launch_cols<64>(p, spec, s, out);
        case 128: return launch_cols<128>(p, spec, s, out);
        case 256: return launch_cols<256>(p, spec, s, out);
        case 512: return launch_cols<512>(p, spec, s, out);
        case 1024: return launch_cols<1024>(p, spec, s, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t spectrum_frame_stride(const ddm_plan_s* p) { return (size_t)(p->nk > 0 ? p->full_nq : p->n_q); }

bool fused_spatial_supported(const ddm_plan_s* p);
ddm_status launch_spatial_fused(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s);
bool rows_bulk_supported(const ddm_plan_s* p, const void* frames);
cudaError_t launch_rows_bulk(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s);

// Path: Bluestein transforms where a side is not a power of two; DDM_SPATIAL_FUSED (cluster
// kernel) where supported and asked for; otherwise the
// row pass (bulk-staged where rows allow it) followed by the column pass.
ddm_status launch_spatial(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s,
                          float2* blk_out, bool* wrote_blocked) {
    if (wrote_blocked) *wrote_blocked = false;
    const SpecOut out{blk_out, p->d.N, p->q0, p->q1};
    if (p->nk > 0) {
        // kx-column range: every row into the whole-plane row output in the workspace, then
        // the range's column blocks into the range's own store `spec`
        if (!p->workspace) return DDM_ERR_NO_WORKSPACE;
        float2* inter = reinterpret_cast<float2*>(static_cast<char*>(p->workspace) + p->inter_offset);
        cudaError_t e = rows_bulk_supported(p, frames)
                            ? launch_rows_bulk(p, frames, inter, s)
                            : ((p->d.dtype == DDM_IN_U16) ? dispatch_rows<uint16_t>(p, frames, inter, s)
                                                          : dispatch_rows<float>(p, frames, inter, s));
        if (e != cudaSuccess) return DDM_ERR_CUDA;
        SpecOut cout{nullptr, p->d.N, p->q0, p->q1};
        cout.col = spec;
        cout.n_qc = p->n_q;
        cout.H = p->d.H;
        cout.Wh = p->Wh;
        cout.kx0 = p->kx0;
        cout.nk = p->nk;
        return dispatch_cols(p, inter, s, cout) == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
    }
    if (p->kc > 0) {
        // low-frequency restriction: bulk-staged row pass into the intermediate, then the
        // cropping column pass
        if (!rows_bulk_supported(p, frames)) return DDM_ERR_UNSUPPORTED;
        if (launch_rows_bulk(p, frames, spec, s) != cudaSuccess) return DDM_ERR_CUDA;
        return dispatch_cols_crop(p, spec, s) == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
    }
    if (p->blue_w.M > 0 || p->blue_h.M > 0 || p->mix_w.n > 0 || p->mix_h.n > 0) {
        // a side that is not a power of two, or of 2048: mixed-radix, Bluestein (or
        // 2048-point) rows or the power-of-two row pass, then mixed-radix, Bluestein (or
        // 2048-point) columns or the power-of-two column pass
        cudaError_t e;
        if (p->mix_w.n > 0)
            e = launch_rows_mixed(p, frames, spec, s);
        else if (p->blue_w.M > 0)
            e = launch_rows_bluestein(p, frames, spec, s);
        else if (rows_bulk_supported(p, frames))
            e = launch_rows_bulk(p, frames, spec, s);
        else
            e = (p->d.dtype == DDM_IN_U16) ? dispatch_rows<uint16_t>(p, frames, spec, s)
                                           : dispatch_rows<float>(p, frames, spec, s);
        if (e != cudaSuccess) return DDM_ERR_CUDA;
        e = p->mix_h.n > 0 ? launch_cols_mixed(p, spec, s, out)
            : p->blue_h.M > 0 ? launch_cols_bluestein(p, spec, s, out) : dispatch_cols(p, spec, s, out);
        if (e == cudaSuccess && wrote_blocked) *wrote_blocked = blk_out != nullptr;
        return e == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
    }
    if (p->d.spatial_path == DDM_SPATIAL_FUSED && fused_spatial_supported(p) &&
        (reinterpret_cast<uintptr_t>(frames) & 15) == 0)
        return launch_spatial_fused(p, frames, spec, s);
    cudaError_t e;
    if (p->d.precision == DDM_PREC_TC_TF32X3) {
        // the column transform on the tensor cores, in place (a blocked copy, if the time
        // kernels want one, is then made by step two)
        e = rows_bulk_supported(p, frames) ? launch_rows_bulk(p, frames, spec, s)
            : ((p->d.dtype == DDM_IN_U16) ? dispatch_rows<uint16_t>(p, frames, spec, s)
                                          : dispatch_rows<float>(p, frames, spec, s));
        if (e != cudaSuccess) return DDM_ERR_CUDA;
        return launch_cols_tc(p, spec, s) == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
    }
    if (rows_bulk_supported(p, frames))
        e = launch_rows_bulk(p, frames, spec, s);
    else
        e = (p->d.dtype == DDM_IN_U16) ? dispatch_rows<uint16_t>(p, frames, spec, s)
                                       : dispatch_rows<float>(p, frames, spec, s);
    if (e != cudaSuccess) return DDM_ERR_CUDA;
    e = dispatch_cols(p, spec, s, out);
    if (e == cudaSuccess && wrote_blocked) *wrote_blocked = blk_out != nullptr;
    return e == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace ddm

// =====================================================================================
// Fused one-pass step one for square frames (side S <= 512): a cluster of CL CTAs owns
// one frame at a time (persistent over frames).  CTAs of 256 threads and ~68 KB of shared
// memory, so that two or three share an SM and hide each other's waits (512 x 512: a
// 16-CTA cluster, which needs the non-portable cluster size).  CTA r of the cluster
//   1. bulk-copies its S/CL consecutive rows of frame t into shared memory (one 1-D
//      cp.async.bulk per 16 KB, mbarrier with a bounded wait) and subtracts frame 0
//      (read through L2, where it stays: every cluster uses it);
//   2. transforms its rows (two real rows per complex FFT) and splits them;
//   3. writes every output value straight into the shared memory of the CTA that owns
//      its column block (distributed shared memory, st.shared::cluster), cluster barrier;
//   4. transforms its S/2/CL columns (column 0 of CTA 0 holds the packed DC / Nyquist
//      pair and is unpacked) and stores 256-byte row segments of the [t][q] spectrum.
// No intermediate spectrum ever goes through HBM.
// =====================================================================================
namespace ddm {
namespace {


__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_cluster_f2(uint32_t local_addr, uint32_t rank, float2 v) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(remote), "f"(v.x), "f"(v.y) : "memory");
}

template <int S, int CL>
struct FusedShape {
    static constexpr int T = FftShape<S>::T, P = FftShape<S>::P;
    static constexpr int RH = S / CL;            // rows per CTA
    static constexpr int PAIRS = RH / 2;         // row pairs per CTA
    static constexpr int CW = S / 2 / CL;        // stored columns per CTA
    static constexpr int NT = PAIRS * T;         // threads
    static_assert(CW * T == NT, "row and column phases use the same threads");
    static constexpr int XELEMS = PAIRS * S;     // complex elements of the shared region
    static_assert(XELEMS == CW * S, "region holds the CTA's rows and its columns");
    static constexpr size_t BYTES = sizeof(float2) * (size_t)XELEMS + (T > 1 ? sizeof(float2) * S : 0);
};

template <int S, int CL, typename In>
__global__ void __launch_bounds__(FusedShape<S, CL>::NT, FusedShape<S, CL>::NT <= 256 ? 2 : 1)
fused_r2c_kernel(const In* __restrict__ frames, float2* __restrict__ spec, int N, int subtract_ref,
                 const float2* __restrict__ tw_g, int n_clusters, unsigned* status) {
    using C = FusedShape<S, CL>;
    constexpr int T = C::T, P = C::P, NT = C::NT, CW = C::CW, RH = C::RH;
    constexpr int Wh = S / 2;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);
    float2* tw = X + C::XELEMS;
    __shared__ uint64_t bar;
    const int tid = threadIdx.x;
    const uint32_t rank = (CL > 1) ? cluster_rank() : 0u;
    const int cluster = blockIdx.x / CL;
    if (tid == 0) {
        mbar_init_s(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if constexpr (T > 1) {
        for (int k = tid; k < S; k += NT) tw[k] = tw_g[k];
    }
    __syncthreads();
    uint32_t phase = 0;
    bool timeout = false;
    // row phase mapping: transform j (row pair), thread i; column phase: column c, thread ic
    const int i = tid % T, j = tid / T;
    const int c = tid % CW, ic = tid / CW;
    constexpr uint32_t kRowBytes = S * sizeof(In);
    constexpr uint32_t kBytes = RH * kRowBytes;
    constexpr uint32_t kChunk = kBytes < 16384u ? kBytes : 16384u;

    for (int t = cluster; t < N; t += n_clusters) {
        const In* rows = frames + ((size_t)t * S + (size_t)rank * RH) * S;
        // ---- 1. rows of frame t -> shared memory (bulk copies), frame 0 via L2
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cvta_smem(&bar)),
                         "r"(kBytes) : "memory");
            for (uint32_t off = 0; off < kBytes; off += kChunk)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    ::"r"(cvta_smem(reinterpret_cast<unsigned char*>(X) + off)),
                    "l"(reinterpret_cast<const unsigned char*>(rows) + off), "r"(kChunk),
                    "r"(cvta_smem(&bar)) : "memory");
        }
        if (t + n_clusters < N && tid == 0) {
            const In* nxt = frames + ((size_t)(t + n_clusters) * S + (size_t)rank * RH) * S;
            for (uint32_t off = 0; off < kBytes; off += kChunk)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                                 reinterpret_cast<const unsigned char*>(nxt) + off), "r"(kChunk) : "memory");
        }
        if (!mbar_wait_s(&bar, phase)) timeout = true;   // keep going: every barrier must match
        phase ^= 1u;
        const In* stage = reinterpret_cast<const In*>(X);
        const In* ref = frames + (size_t)rank * RH * S;
        float2 v[P];
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int x = i + T * u;
            const int ra = (2 * j) * S + x, rb = ra + S;
            float a, b;
            if constexpr (sizeof(In) == 2) {
                a = (float)((int)stage[ra] - (subtract_ref ? (int)__ldg(ref + ra) : 0));
                b = (float)((int)stage[rb] - (subtract_ref ? (int)__ldg(ref + rb) : 0));
            } else {
                a = subtract_ref ? (float)stage[ra] - (float)__ldg(ref + ra) : (float)stage[ra];
                b = subtract_ref ? (float)stage[rb] - (float)__ldg(ref + rb) : (float)stage[rb];
            }
            v[u] = make_float2(a, b);
        }
        __syncthreads();   // staging read: the region becomes the row exchange buffer

        // ---- 2. row transforms (z = row a + i row b), then split into the two rows
        const AddrSwizzled<S> raddr{j * S};
        fft_cyclic<S, false>(v, i, X, raddr, tw, SyncBlock{});
#pragma unroll
        for (int u = 0; u < P; ++u) X[raddr(i + T * u)] = v[u];
        __syncthreads();
        float2 outa[P / 2], outb[P / 2];
#pragma unroll
        for (int u = 0; u < P / 2; ++u) {
            const int k = i + T * u;                      // k < S/2
            const float2 z = X[raddr(k)];
            if (k == 0) {
                const float2 zn = X[raddr(S / 2)];
                outa[u] = make_float2(z.x, zn.x);         // A[0], A[S/2] (both real)
                outb[u] = make_float2(z.y, zn.y);
            } else {
                const float2 zr = X[raddr(S - k)];
                outa[u] = make_float2(0.5f * (z.x + zr.x), 0.5f * (z.y - zr.y));
                outb[u] = make_float2(0.5f * (z.y + zr.y), 0.5f * (zr.x - z.x));
            }
        }
        // ---- 3. every CTA is done with its region; scatter (row y, kx) to kx's owner
        if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();
        const int ya = rank * RH + 2 * j, yb = ya + 1;
#pragma unroll
        for (int u = 0; u < P / 2; ++u) {
            const int k = i + T * u;
            const uint32_t dst = (uint32_t)(k / CW);
            const int col = k - (int)dst * CW;
            if constexpr (CL > 1) {
                st_cluster_f2(cvta_smem(X + ya * CW + col), dst, outa[u]);
                st_cluster_f2(cvta_smem(X + yb * CW + col), dst, outb[u]);
            } else {
                X[ya * CW + col] = outa[u];
                X[yb * CW + col] = outb[u];
            }
        }
        if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();

        // ---- 4. column transforms of this CTA's CW stored columns
        float2 w[P];
#pragma unroll
        for (int u = 0; u < P; ++u) w[u] = X[(ic + T * u) * CW + c];
        __syncthreads();
        const AddrInterleaved<CW> caddr{c};
        fft_cyclic<S, false>(w, ic, X, caddr, tw, SyncBlock{});
        const int kx = rank * CW + c;
        float2* fr = spec + (size_t)t * (size_t)(S * (Wh + 1));
        if (rank == 0) {
            // column 0 holds the packed DC / Nyquist pair: needs C[-ky]
#pragma unroll
            for (int u = 0; u < P; ++u)
                if (c == 0) X[ic + T * u] = w[u];
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int ky = ic + T * u;
            if (rank == 0 && c == 0) {
                const float2 cc = w[u];
                const float2 cr = X[(S - ky) & (S - 1)];
                fr[(size_t)ky * Wh] = make_float2(0.5f * (cc.x + cr.x), 0.5f * (cc.y - cr.y));
                fr[(size_t)S * Wh + ky] = make_float2(0.5f * (cc.y + cr.y), 0.5f * (cr.x - cc.x));
            } else {
                fr[(size_t)ky * Wh + kx] = w[u];
            }
        }
        __syncthreads();   // the region is rewritten by the next frame's copy
    }
    if (timeout && tid == 0) atomicOr(status, 2u);
    if constexpr (CL > 1) cluster_sync_all();   // no CTA leaves while a peer may still write
}

template <int S, int CL, typename In>
cudaError_t launch_fused(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    using C = FusedShape<S, CL>;
    auto k = fused_r2c_kernel<S, CL, In>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
    if (e != cudaSuccess) return e;
    if (CL > 8) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = C::BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int max_clusters = 0;
    cfg.gridDim = dim3(CL * 1024);
    e = cudaOccupancyMaxActiveClusters(&max_clusters, (void*)k, &cfg);
    if (e != cudaSuccess || max_clusters < 1) {
        cudaGetLastError();
        max_clusters = p->n_sm / CL;
    }
    const int n_clusters = max_clusters < p->d.N ? max_clusters : p->d.N;
    cfg.gridDim = dim3(CL * n_clusters);
    return cudaLaunchKernelEx(&cfg, k, (const In*)frames, spec, p->d.N, p->d.subtract_ref,
                              (const float2*)p->tw_col, n_clusters, p->dev_status);
}

template <typename In>
cudaError_t dispatch_fused(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    switch (p->d.H) {
        case 64: return launch_fused<64, 1, In>(p, frames, spec, s);
        case 128: return launch_fused<128, 2, In>(p, frames, spec, s);
        case 256: return launch_fused<256, 4, In>(p, frames, spec, s);
        case 512: return launch_fused<512, 16, In>(p, frames, spec, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

namespace {

// ---- row pass with bulk-staged input -------------------------------------------------
// A CTA owns PAIRS consecutive row pairs of one frame.  Those rows, and the same rows of
// frame 0, are contiguous in memory: two cp.async.bulk copies bring them into shared
// memory (mbarrier with a bounded wait) instead of 2-byte scattered loads, and the region
// then serves as the transform's exchange buffer (XOR-swizzled, no padding).  Rows of 128
// bytes or more are staged one copy per row with a 16-byte pad after each, so that the two
// row pairs a warp reads sit on different banks.  Up to ~70 KB per CTA, three CTAs per SM
// (37 KB and five at 512-pixel rows).
template <int W, typename In>
struct RowBulkShape {
    static constexpr int T = FftShape<W>::T, P = FftShape<W>::P;
    static constexpr int BYTES_ROW = W * (int)sizeof(In);
    static constexpr int PAD = (BYTES_ROW >= 128 && BYTES_ROW % 128 == 0) ? 16 : 0;
    static constexpr int ROW_STRIDE = BYTES_ROW + PAD;                   // staged row pitch
    static constexpr int P1 = 256 / T;
    static constexpr int P2 = 16384 / BYTES_ROW > 0 ? 16384 / BYTES_ROW : 1;
    static constexpr int PAIRS0 = (P1 < P2 ? P1 : P2) < 1 ? 1 : (P1 < P2 ? P1 : P2);
    // 512-pixel rows: 8 row pairs per 128-thread CTA, five CTAs per SM (37 KB each) hide the
    // staging wait better than 16 pairs at three per SM (512x512x1024 step one 0.683 ->
    // 0.666 ms); the other widths keep the larger CTA (256 columns: 0.203 against 0.222 ms)
    static constexpr int PAIRS = (W == 512 && PAIRS0 > 8) ? 8 : PAIRS0;
    static constexpr int MIN_CTAS = W == 512 ? 5 : 3;
    static constexpr int NT = PAIRS * T;
    static constexpr size_t STAGE = (size_t)2 * 2 * PAIRS * ROW_STRIDE;  // frame rows + frame-0 rows
    static constexpr size_t XCH = (size_t)PAIRS * W * sizeof(float2);
    static constexpr size_t XBYTES = STAGE > XCH ? STAGE : XCH;
    static constexpr size_t BYTES = XBYTES + (T > 1 ? W * sizeof(float2) : 0);
};

template <int W, typename In>
__global__ void __launch_bounds__(RowBulkShape<W, In>::NT, RowBulkShape<W, In>::MIN_CTAS)
row_bulk_kernel(const In* __restrict__ frames, float2* __restrict__ spec, int H, size_t frame_stride,
                int subtract_ref, const float2* __restrict__ tw_g, unsigned* status, int kc) {
    using C = RowBulkShape<W, In>;
    constexpr int T = C::T, P = C::P, PAIRS = C::PAIRS, NT = C::NT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);
    float2* tw = reinterpret_cast<float2*>(smem_raw + C::XBYTES);
    __shared__ uint64_t bar;
    const int tid = threadIdx.x;
    const int t = blockIdx.y;
    const int pair0 = blockIdx.x * PAIRS;
    const int npairs = min(PAIRS, H / 2 - pair0);
    const uint32_t bytes = (uint32_t)(2 * npairs) * C::BYTES_ROW;
    const In* src = frames + ((size_t)t * H + 2 * pair0) * W;
    const In* ref = frames + (size_t)(2 * pair0) * W;
    unsigned char* stage_f = smem_raw;
    unsigned char* stage_r = smem_raw + (size_t)2 * PAIRS * C::ROW_STRIDE;
    if (tid == 0) {
        mbar_init_s(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cvta_smem(&bar)),
                     "r"(subtract_ref ? 2 * bytes : bytes) : "memory");
        if constexpr (C::PAD == 0) {
            for (uint32_t off = 0; off < bytes; off += 16384u) {
                const uint32_t n = bytes - off < 16384u ? bytes - off : 16384u;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    ::"r"(cvta_smem(stage_f + off)), "l"(reinterpret_cast<const unsigned char*>(src) + off),
                    "r"(n), "r"(cvta_smem(&bar)) : "memory");
                if (subtract_ref)
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                        ::"r"(cvta_smem(stage_r + off)), "l"(reinterpret_cast<const unsigned char*>(ref) + off),
                        "r"(n), "r"(cvta_smem(&bar)) : "memory");
            }
        }
    }
    if constexpr (C::PAD != 0) {
        // one row per thread: the barrier expects the bytes before any copy is issued
        __syncthreads();
        for (int r = tid; r < 2 * npairs; r += NT) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"(cvta_smem(stage_f + (size_t)r * C::ROW_STRIDE)),
                "l"(reinterpret_cast<const unsigned char*>(src) + (size_t)r * C::BYTES_ROW),
                "r"((uint32_t)C::BYTES_ROW), "r"(cvta_smem(&bar)) : "memory");
            if (subtract_ref)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    ::"r"(cvta_smem(stage_r + (size_t)r * C::ROW_STRIDE)),
                    "l"(reinterpret_cast<const unsigned char*>(ref) + (size_t)r * C::BYTES_ROW),
                    "r"((uint32_t)C::BYTES_ROW), "r"(cvta_smem(&bar)) : "memory");
        }
    }
    if constexpr (T > 1) {
        for (int k = tid; k < W; k += NT) tw[k] = tw_g[k];
    }
    __syncthreads();                                   // barrier initialised, twiddles in place
    const bool ok = mbar_wait_s(&bar, 0);
    const int i = tid % T, j = tid / T;
    const bool active = j < npairs;
    const In* fa = reinterpret_cast<const In*>(stage_f + (size_t)(2 * j) * C::ROW_STRIDE);
    const In* fb = reinterpret_cast<const In*>(stage_f + (size_t)(2 * j + 1) * C::ROW_STRIDE);
    const In* ra = reinterpret_cast<const In*>(stage_r + (size_t)(2 * j) * C::ROW_STRIDE);
    const In* rb = reinterpret_cast<const In*>(stage_r + (size_t)(2 * j + 1) * C::ROW_STRIDE);
    float2 v[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
        const int x = i + T * u;
        float a = 0.f, b = 0.f;
        if (active) {
            if constexpr (sizeof(In) == 2) {
                a = (float)((int)fa[x] - (subtract_ref ? (int)ra[x] : 0));
                b = (float)((int)fb[x] - (subtract_ref ? (int)rb[x] : 0));
            } else {
                a = subtract_ref ? (float)fa[x] - (float)ra[x] : (float)fa[x];
                b = subtract_ref ? (float)fb[x] - (float)rb[x] : (float)fb[x];
            }
        }
        v[u] = make_float2(a, b);
    }
    __syncthreads();                                   // staging read: region becomes the exchange
    const AddrSwizzled<W> addr{j * W};
    fft_cyclic<W, false>(v, i, X, addr, tw, SyncBlock{});
    static_assert(P >= 2 && 32 % T == 0, "row pairs: P >= 2 points per thread, T | 32");
    // The split into the two real rows pairs X[k] with X[W - k].  Thread i holds X[i + T u];
    // for k = i + T u, X[W - k] sits in thread (T - i) % T of the same transform (the same
    // warp: T divides 32) at u' = P - 1 - u (i > 0) or (P - u) % P (i = 0), so it comes by a
    // shuffle, with no shared-memory round trip and no block barrier.
    {
        // kc > 0 (low-frequency restriction): rows of kx = 0..kc, no Nyquist packing
        const int rowlen = kc > 0 ? kc + 1 : W / 2;
        const int lane = tid & 31;
        const int src = lane - i + ((T - i) & (T - 1));
        float2* outa = spec + (size_t)t * frame_stride + (size_t)(2 * (pair0 + j)) * rowlen;
        float2* outb = outa + rowlen;
#pragma unroll
        for (int u = 0; u < (P + 1) / 2; ++u) {
            const float2 send = (i == 0) ? v[(P - u) & (P - 1)] : v[P - 1 - u];
            float2 zr;
            zr.x = __shfl_sync(0xffffffffu, send.x, src);
            zr.y = __shfl_sync(0xffffffffu, send.y, src);
            const int k = i + T * u;
            if (!active || k >= rowlen) continue;
            const float2 z = v[u];
            if (k == 0) {
                const float2 nyq = v[P / 2];                      // X[W / 2]: thread 0, u = P / 2
                outa[0] = make_float2(z.x, kc > 0 ? 0.f : nyq.x);
                outb[0] = make_float2(z.y, kc > 0 ? 0.f : nyq.y);
            } else {
                outa[k] = make_float2(0.5f * (z.x + zr.x), 0.5f * (z.y - zr.y));
                outb[k] = make_float2(0.5f * (z.y + zr.y), 0.5f * (zr.x - z.x));
            }
        }
    }
    if (!ok && tid == 0) atomicOr(status, 2u);
}

template <int W, typename In>
cudaError_t launch_rows_bulk_t(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    using C = RowBulkShape<W, In>;
    auto k = row_bulk_kernel<W, In>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dim3 grid((p->d.H / 2 + C::PAIRS - 1) / C::PAIRS, p->d.N);
    // full: the spectrum itself, frame stride n_q; low-frequency restriction: the plan's
    // intermediate [N][H][kc + 1]
    const bool crop = p->kc > 0;
    float2* out = crop ? p->crop_inter : spec;
    const size_t fstride = crop ? (size_t)p->d.H * (size_t)(p->kc + 1) : spectrum_frame_stride(p);
    k<<<grid, C::NT, C::BYTES, s>>>((const In*)frames, out, p->d.H, fstride, p->d.subtract_ref,
                                     p->tw_row, p->dev_status, p->kc);
    return cudaGetLastError();
}

template <typename In>
cudaError_t dispatch_rows_bulk(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    switch (p->d.W) {
        case 4: return launch_rows_bulk_t<4, In>(p, frames, spec, s);
        case 8: return launch_rows_bulk_t<8, In>(p, frames, spec, s);
        case 16: return launch_rows_bulk_t<16, In>(p, frames, spec, s);
        case 32: return launch_rows_bulk_t<32, In>(p, frames, spec, s);
        case 64: return launch_rows_bulk_t<64, In>(p, frames, spec, s);
        case 128: return launch_rows_bulk_t<128, In>(p, frames, spec, s);
        case 256: return launch_rows_bulk_t<256, In>(p, frames, spec, s);
        case 512: return launch_rows_bulk_t<512, In>(p, frames, spec, s);
        case 1024: return launch_rows_bulk_t<1024, In>(p, frames, spec, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// rows of W * sizeof(In) >= 16 bytes, frames 16-byte aligned: bulk-staged row pass
bool rows_bulk_supported(const ddm_plan_s* p, const void* frames) {
    const int esize = p->d.dtype == DDM_IN_U16 ? 2 : 4;
    return p->d.W * esize >= 16 && (reinterpret_cast<uintptr_t>(frames) & 15) == 0;
}

cudaError_t launch_rows_bulk(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    return p->d.dtype == DDM_IN_U16 ? dispatch_rows_bulk<uint16_t>(p, frames, spec, s)
                                    : dispatch_rows_bulk<float>(p, frames, spec, s);
}

bool fused_spatial_supported(const ddm_plan_s* p) {
    return p->d.H == p->d.W && (p->d.H == 64 || p->d.H == 128 || p->d.H == 256 || p->d.H == 512);
}

ddm_status launch_spatial_fused(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    cudaError_t e = (p->d.dtype == DDM_IN_U16) ? dispatch_fused<uint16_t>(p, frames, spec, s)
                                               : dispatch_fused<float>(p, frames, spec, s);
    return e == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace ddm
