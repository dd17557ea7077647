// Step one (Sec. 2) for frame sides n = P T with P, T of the form 2^a 3^b 5^c (common camera
// sides: 384, 480, 540, 600, 640, 720, 768, 800, 900, 960, 1000, 1080, 1200, 1280, 1440, 1536,
// 1600, 1920, 2000): a two-pass mixed-radix
// transform instead of Bluestein's, about 6x less arithmetic at n = 800.  T threads per transform, P points per
// thread in the cyclic layout (thread i holds x[i + T u], u < P):
//   pass 1: the P-point DFT over u (dft_mix), the twiddle w_n^{i k1} (host table, double
//           precision), one shared-memory exchange;
//   pass 2: thread j < P takes k1 = j and does the T-point DFT over i; it then holds
//           X[j + P k2], k2 < T (threads j >= P idle in this pass).
// The row and column kernels around it are those of the Bluestein path (two real rows per
// complex row transform with the Nyquist value in slot 0; columns in place, the packed DC /
// Nyquist column unpacked by the block that holds it).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// A bounded wait on an mbarrier phase: about two seconds of polling (SM clock cycles), then
// false.
__device__ __forceinline__ bool mbar_wait_bounded_m(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
        if (ok) return true;
        if (clock64() - t0 > 4000000000LL) return false;
    }
}

// exchange row stride: the smallest r >= T with r QT = QT (mod 16), so that in pass 2 the
// QT-lane groups of consecutive k1 tile the 16 bank pairs (8-byte elements)
constexpr int mixed_row(int T, int QT) {
    int r = T;
    while ((r * QT - QT) % 16 != 0) ++r;
    return r;
}

template <int P_, int T_, int NT_ = 256>
struct MShape {
    static constexpr int P = P_, T = T_, N = P * T;
    static constexpr int NT = NT_;
    static constexpr int QT = NT / T;                       // transforms per CTA
    static constexpr int ROW = mixed_row(T, QT);            // exchange row of one k1
    static constexpr size_t XCH = (size_t)P * ROW * QT;     // (k1 ROW + i) QT + ql
    // row stride of the staged input and of the output X (transform ql at ql WS + k): 4 mod 16
    // float2, so that the lanes of a warp (a few transforms x a few consecutive indices) fall
    // on distinct bank pairs
    static constexpr int WS = N + ((4 - N % 16) + 16) % 16;
    static constexpr size_t STG = (size_t)QT * WS;
    static constexpr size_t OUT = STG;
    static constexpr size_t XE = XCH > STG ? (XCH > OUT ? XCH : OUT) : (STG > OUT ? STG : OUT);
    static constexpr size_t BYTES = sizeof(float2) * (XE + (size_t)N);
    // bulk staging of uint16 rows (row kernel): the 2 QT rows of the frame and the same rows
    // of frame 0, each at a pitch of its bytes plus a 16-byte pad, inside the exchange region
    static constexpr int RAW_PITCH = ((N * 2 + 15) / 16) * 16 + 16;
    static constexpr bool BULK_FITS = (N * 2) % 16 == 0 && (size_t)4 * QT * RAW_PITCH <= XE * sizeof(float2);
    // TMA staging of QT columns (column kernel): NBOX boxes of BOXR rows x QT complex (QT even:
    // 16-byte multiples), landing [row][QT] in the exchange region, each box at a 128-byte
    // aligned shared-memory address
    static constexpr int NBOX = (N + 255) / 256, BOXR = (N + NBOX - 1) / NBOX;
    static constexpr bool TMA_FITS = QT % 2 == 0 && (BOXR * QT) % 16 == 0 && (size_t)NBOX * BOXR * QT <= XE;
    static_assert(P <= 40 && T <= 50 && QT >= 1, "mixed-radix shapes");
    static_assert(P <= T, "pass 2 gives each k1 < P its own thread: P <= T");
};

// QT interleaved transforms; thread (ql, i) with i < T.  live: the thread is one of the
// T QT threads that carry a transform (the CTA may have a few spare threads).  Returns with
// thread (ql, j), j < P, holding X[j + P k2] in w[k2].
template <int P, int T, int NT = 256>
__device__ __forceinline__ void fft_mixed(float2 (&v)[P], float2 (&w)[T], int i, int ql, bool live,
                                          float2* xs, const float2* tw) {
    using C = MShape<P, T, NT>;
    dft_mix<P, false>(v);
    if (live) {
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const float2 a = k1 == 0 ? v[k1] : cmul(v[k1], tw[k1 * T + i]);
            xs[(k1 * C::ROW + i) * C::QT + ql] = a;
        }
    }
    __syncthreads();
    if (live && i < P) {
#pragma unroll
        for (int ip = 0; ip < T; ++ip) w[ip] = xs[(i * C::ROW + ip) * C::QT + ql];
        dft_mix<T, false>(w);
    }
    __syncthreads();                                        // exchange read: xs is free
}

// ---------------------------------------------------------------- rows (W = P T)
// grid: (ceil(H/2 / QT), N); block: 256.  CTA: QT row pairs of one frame.
// four consecutive pixels by one 8-byte (uint16) or 16-byte (float) load
__device__ __forceinline__ void load4(const uint16_t* p, float (&f)[4]) {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    f[0] = (float)(r.x & 0xffffu);
    f[1] = (float)(r.x >> 16);
    f[2] = (float)(r.y & 0xffffu);
    f[3] = (float)(r.y >> 16);
}
__device__ __forceinline__ void load4(const float* p, float (&f)[4]) {
    const float4 r = __ldg(reinterpret_cast<const float4*>(p));
    f[0] = r.x;
    f[1] = r.y;
    f[2] = r.z;
    f[3] = r.w;
}

// STAGE: 0 one pixel per load; 1 four pixels per load (frames aligned to four pixels);
// 2 (uint16 frames, 16-byte aligned rows) each row of the CTA and of frame 0 by one
// cp.async.bulk copy into shared memory, converted from there straight into registers
template <int P, int T, typename In, int STAGE>
__global__ void __launch_bounds__(256)
row_mixed_kernel(const In* __restrict__ frames, float2* __restrict__ spec, int H, size_t frame_stride,
                 int subtract_ref, const float2* __restrict__ tw_g, unsigned* status) {
    using C = MShape<P, T>;
    constexpr int W = C::N, QT = C::QT, NT = C::NT, WS = C::WS;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* xs = reinterpret_cast<float2*>(smem_raw);
    float2* tw = xs + C::XE;
    const int tid = threadIdx.x;
    const int t = blockIdx.y;
    const int pair0 = blockIdx.x * QT;
    const int npairs = min(QT, H / 2 - pair0);
    const In* src = frames + ((size_t)t * H + 2 * pair0) * W;
    const In* ref = frames + (size_t)(2 * pair0) * W;
    const int ql = tid % QT, i = tid / QT;
    const bool live = i < T;
    const bool active = live && ql < npairs;
    float2 v[P], w[T];
    if constexpr (STAGE == 2) {
        static_assert(sizeof(In) == 2 && C::BULK_FITS, "bulk staging: uint16 rows of 16-byte multiples");
        constexpr int RP = C::RAW_PITCH;
        constexpr uint32_t ROWB = (uint32_t)W * 2u;
        __shared__ uint64_t bar;
        unsigned char* rawf = smem_raw;                               // rows of this frame
        unsigned char* rawr = smem_raw + (size_t)2 * QT * RP;         // the same rows of frame 0
        const uint32_t nrows = (uint32_t)(2 * npairs);
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)),
                         "r"((subtract_ref ? 2u : 1u) * nrows * ROWB) : "memory");
        }
        for (int k = tid; k < W; k += NT) tw[k] = tw_g[k];
        __syncthreads();                                   // the barrier expects the bytes
        for (uint32_t r = tid; r < nrows; r += NT) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"(smem_addr(rawf + (size_t)r * RP)), "l"(src + (size_t)r * W), "r"(ROWB),
                "r"(smem_addr(&bar)) : "memory");
            if (subtract_ref)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    ::"r"(smem_addr(rawr + (size_t)r * RP)), "l"(ref + (size_t)r * W), "r"(ROWB),
                    "r"(smem_addr(&bar)) : "memory");
        }
        const bool ok = mbar_wait_bounded_m(&bar, 0);
        // rows 2 ql and 2 ql + 1 as the real and imaginary parts; integer differences below
        // 2^16 are exact in float, as on the other staging paths
        const uint16_t* fa = reinterpret_cast<const uint16_t*>(rawf + (size_t)(2 * ql) * RP);
        const uint16_t* ra = reinterpret_cast<const uint16_t*>(rawr + (size_t)(2 * ql) * RP);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int x = i + T * u;
            float a = 0.f, b = 0.f;
            if (active && ok) {
                a = (float)((int)fa[x] - (subtract_ref ? (int)ra[x] : 0));
                b = (float)((int)fa[RP / 2 + x] - (subtract_ref ? (int)ra[RP / 2 + x] : 0));
            }
            v[u] = make_float2(a, b);
        }
        if (!ok) {
            // report it (status bit 2); the copies get a last bounded chance to land before
            // the region becomes the exchange
            if (tid == 0) atomicOr(status, 2u);
            mbar_wait_bounded_m(&bar, 0);
        }
        __syncthreads();                                   // staging read: xs becomes the exchange
    } else {
        for (int k = tid; k < W; k += NT) tw[k] = tw_g[k];
        if constexpr (STAGE == 1) {
            // four pixels of rows 2q and 2q + 1 per thread and iteration: a warp moves 256 B (uint16)
            // or 512 B (float) of each row per load, enough bytes in flight to cover HBM latency.  The
            // 32 B of four staged pairs go out as two 16 B halves; a quad whose 32 B chunk lies at an
            // odd multiple of 128 B writes its upper half first, so that each store by a warp meets all
            // 32 banks.  The differences of integers below 2^16 are exact in float, as on the scalar path.
            static_assert(W % 4 == 0 && WS % 4 == 0, "vector staging: W and WS multiples of 4");
            constexpr int W4 = W / 4;
#pragma unroll 4
            for (int e = tid; e < npairs * W4; e += NT) {
                const int q = e / W4, x4 = e - q * W4, x = 4 * x4;
                const size_t ia = (size_t)(2 * q) * W + x, ib = ia + W;
                float a[4], b[4];
                load4(src + ia, a);
                load4(src + ib, b);
                if (subtract_ref) {
                    float ra[4], rb[4];
                    load4(ref + ia, ra);
                    load4(ref + ib, rb);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        a[j] -= ra[j];
                        b[j] -= rb[j];
                    }
                }
                const float4 lo = make_float4(a[0], b[0], a[1], b[1]), hi = make_float4(a[2], b[2], a[3], b[3]);
                float4* dst = reinterpret_cast<float4*>(xs + q * WS + x);
                const int h = ((q * (WS / 4) + x4) >> 2) & 1;
                dst[h] = h ? hi : lo;
                dst[1 - h] = h ? lo : hi;
            }
        } else {
#pragma unroll 4
            for (int e = tid; e < npairs * W; e += NT) {        // 4 iterations of loads in flight
                const int q = e / W, x = e - q * W;
                const size_t ia = (size_t)(2 * q) * W + x, ib = ia + W;
                float a, b;
                if constexpr (sizeof(In) == 2) {
                    a = (float)((int)__ldg(src + ia) - (subtract_ref ? (int)__ldg(ref + ia) : 0));
                    b = (float)((int)__ldg(src + ib) - (subtract_ref ? (int)__ldg(ref + ib) : 0));
                } else {
                    a = subtract_ref ? __ldg(src + ia) - __ldg(ref + ia) : __ldg(src + ia);
                    b = subtract_ref ? __ldg(src + ib) - __ldg(ref + ib) : __ldg(src + ib);
                }
                xs[q * WS + x] = make_float2(a, b);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < P; ++u) v[u] = active ? xs[ql * WS + i + T * u] : make_float2(0.f, 0.f);
        __syncthreads();                                        // staging read: xs becomes the exchange
    }
    fft_mixed<P, T>(v, w, i, ql, live, xs, tw);
    if (live && i < P) {
#pragma unroll
        for (int k2 = 0; k2 < T; ++k2) xs[ql * WS + i + P * k2] = w[k2];
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

// ------------------------------------------------------------- columns (H = P T)
// grid: (ceil(Wh / QT), N); block: NTC (256, or 512 for the wide shapes: 12 columns of T = 40
// threads, 96-byte row segments).  In place, QT stored columns of one frame.  TMA: the CTA's
// H x QT block arrives by TMA copies (tensor map over the spectrum as float32
// [N][H][2 Wh], boxes of BOXR rows x 2 QT floats) instead of per-thread strided loads.
template <int P, int T, int NTC, bool TMA>
__global__ void __launch_bounds__(NTC)
col_mixed_kernel(float2* __restrict__ spec, int Wh, size_t frame_stride, const float2* __restrict__ tw_g,
                 SpecOut out, const __grid_constant__ CUtensorMap tmap, unsigned* status) {
    using C = MShape<P, T, NTC>;
    constexpr int H = C::N, QT = C::QT, NT = C::NT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* xs = reinterpret_cast<float2*>(smem_raw);
    float2* tw = xs + C::XE;
    const int tid = threadIdx.x;
    const int ql = tid % QT, i = tid / QT;
    const bool live = i < T;
    const int kx = blockIdx.x * QT + ql;
    const bool valid = live && kx < Wh;
    float2* base = spec + (size_t)blockIdx.y * frame_stride;
    float2 v[P], w[T];
    if constexpr (TMA) {
        static_assert(C::TMA_FITS, "TMA staging: QT even, the staged rows fit the exchange region");
        __shared__ uint64_t bar;
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)),
                         "r"((uint32_t)(C::NBOX * C::BOXR * QT * sizeof(float2))) : "memory");
#pragma unroll
            for (int b = 0; b < C::NBOX; ++b)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4}], [%5];"
                    ::"r"(smem_addr(xs + (size_t)b * C::BOXR * QT)), "l"(&tmap), "r"(2 * (int)blockIdx.x * QT),
                    "r"(b * C::BOXR), "r"((int)blockIdx.y), "r"(smem_addr(&bar)) : "memory");
        }
        for (int k = tid; k < H; k += NT) tw[k] = tw_g[k];
        __syncthreads();                                   // the twiddles; the barrier is armed
        const bool ok = mbar_wait_bounded_m(&bar, 0);
#pragma unroll
        for (int u = 0; u < P; ++u) v[u] = (valid && ok) ? xs[(i + T * u) * QT + ql] : make_float2(0.f, 0.f);
        if (!ok) {
            // report it (status bit 2); the copies get a last bounded chance to land before the
            // region becomes the exchange
            if (tid == 0) atomicOr(status, 2u);
            mbar_wait_bounded_m(&bar, 0);
        }
        __syncthreads();                                   // staging read: xs becomes the exchange
    } else {
        for (int k = tid; k < H; k += NT) tw[k] = tw_g[k];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < P; ++u) v[u] = valid ? base[(size_t)(i + T * u) * Wh + kx] : make_float2(0.f, 0.f);
    }
    fft_mixed<P, T, NTC>(v, w, i, ql, live, xs, tw);
    const bool holds = live && i < P;                       // holds X[i + P k2], k2 < T
    const int t = blockIdx.y;
    if (blockIdx.x != 0) {
        if (holds && kx < Wh) {
#pragma unroll
            for (int k2 = 0; k2 < T; ++k2) out.put(base, t, (int64_t)(i + P * k2) * Wh + kx, w[k2]);
        }
        return;
    }
    // the block holding kx = 0 unpacks the packed DC / Nyquist column (partner ky <-> H - ky)
    if (holds) {
#pragma unroll
        for (int k2 = 0; k2 < T; ++k2) xs[(i + P * k2) * QT + ql] = w[k2];
    }
    __syncthreads();
    if (!holds || kx >= Wh) return;
#pragma unroll
    for (int k2 = 0; k2 < T; ++k2) {
        const int ky = i + P * k2;
        if (ql != 0) {
            out.put(base, t, (int64_t)ky * Wh + kx, w[k2]);
        } else {
            const float2 c = w[k2];
            const float2 cr = xs[(ky == 0 ? 0 : H - ky) * QT];
            out.put(base, t, (int64_t)ky * Wh, make_float2(0.5f * (c.x + cr.x), 0.5f * (c.y - cr.y)));
            out.put(base, t, (int64_t)H * Wh + ky, make_float2(0.5f * (c.y + cr.y), 0.5f * (cr.x - c.x)));
        }
    }
}

template <int P, int T, typename In>
cudaError_t rows_t(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    using C = MShape<P, T>;
    // vector staging needs the frames 4-pixel aligned (every row offset is: W is a multiple of
    // 4); bulk staging uint16 frames 16-byte aligned with rows of a multiple of 16 bytes
    const uintptr_t a = reinterpret_cast<uintptr_t>(frames);
    const bool vec = a % (4 * sizeof(In)) == 0;
    auto k = vec ? row_mixed_kernel<P, T, In, 1> : row_mixed_kernel<P, T, In, 0>;
    if constexpr (sizeof(In) == 2 && C::BULK_FITS) {
        if (a % 16 == 0) k = row_mixed_kernel<P, T, In, 2>;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
    if (e != cudaSuccess) return e;
    dim3 grid((p->d.H / 2 + C::QT - 1) / C::QT, p->d.N);
    k<<<grid, C::NT, C::BYTES, s>>>((const In*)frames, spec, p->d.H, (size_t)p->n_q, p->d.subtract_ref,
                                     p->mix_w.tw, p->dev_status);
    return cudaGetLastError();
}

template <int P, int T, int NTC = 256>
cudaError_t cols_t(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out) {
    using C = MShape<P, T, NTC>;
    auto k = col_mixed_kernel<P, T, NTC, false>;
    // the TMA path needs 16-byte rows and frames (Wh and n_q even) and an aligned spectrum;
    // it is taken for the 256-thread shapes (600x800x3000 step one 4.75 -> 4.28 ms), not for
    // the 512-thread ones (1080x1920x256 2.21 -> 2.24 ms)
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if constexpr (C::TMA_FITS && NTC == 256) {
        const cuuint64_t dims[3] = {(cuuint64_t)(2 * p->Wh), (cuuint64_t)C::N, (cuuint64_t)p->d.N};
        const cuuint64_t strides[2] = {(cuuint64_t)p->Wh * sizeof(float2), (cuuint64_t)p->n_q * sizeof(float2)};
        const cuuint32_t box[3] = {(cuuint32_t)(2 * C::QT), (cuuint32_t)C::BOXR, 1};
        if (p->Wh % 2 == 0 && p->n_q % 2 == 0 && reinterpret_cast<uintptr_t>(spec) % 16 == 0 &&
            encode_f32_tensor_map(&tmap, spec, 3, dims, strides, box))
            k = col_mixed_kernel<P, T, NTC, true>;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
    if (e != cudaSuccess) return e;
    dim3 grid((p->Wh + C::QT - 1) / C::QT, p->d.N);
    k<<<grid, C::NT, C::BYTES, s>>>(spec, p->Wh, (size_t)p->n_q, p->mix_h.tw, out, tmap, p->dev_status);
    return cudaGetLastError();
}

// the shapes built: side -> (P, T)
template <typename In>
cudaError_t rows_dispatch(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    switch (p->d.W) {
        case 384: return rows_t<12, 32, In>(p, frames, spec, s);
        case 480: return rows_t<15, 32, In>(p, frames, spec, s);
        case 540: return rows_t<18, 30, In>(p, frames, spec, s);
        case 600: return rows_t<24, 25, In>(p, frames, spec, s);
        case 640: return rows_t<20, 32, In>(p, frames, spec, s);
        case 720: return rows_t<24, 30, In>(p, frames, spec, s);
        case 768: return rows_t<24, 32, In>(p, frames, spec, s);
        case 800: return rows_t<25, 32, In>(p, frames, spec, s);
        case 900: return rows_t<30, 30, In>(p, frames, spec, s);
        case 960: return rows_t<30, 32, In>(p, frames, spec, s);
        case 1000: return rows_t<25, 40, In>(p, frames, spec, s);
        case 1080: return rows_t<27, 40, In>(p, frames, spec, s);
        case 1200: return rows_t<30, 40, In>(p, frames, spec, s);
        case 1280: return rows_t<32, 40, In>(p, frames, spec, s);
        case 1440: return rows_t<30, 48, In>(p, frames, spec, s);
        case 1536: return rows_t<32, 48, In>(p, frames, spec, s);
        case 1600: return rows_t<32, 50, In>(p, frames, spec, s);
        case 1920: return rows_t<40, 48, In>(p, frames, spec, s);
        case 2000: return rows_t<40, 50, In>(p, frames, spec, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// (P, T) of a side built with the mixed-radix kernels, or (0, 0)
void mixed_shape(int n, int* P, int* T) {
    switch (n) {
        case 384: *P = 12; *T = 32; return;
        case 480: *P = 15; *T = 32; return;
        case 540: *P = 18; *T = 30; return;
        case 600: *P = 24; *T = 25; return;
        case 640: *P = 20; *T = 32; return;
        case 720: *P = 24; *T = 30; return;
        case 768: *P = 24; *T = 32; return;
        case 800: *P = 25; *T = 32; return;
        case 900: *P = 30; *T = 30; return;
        case 960: *P = 30; *T = 32; return;
        case 1000: *P = 25; *T = 40; return;
        case 1080: *P = 27; *T = 40; return;
        case 1200: *P = 30; *T = 40; return;
        case 1280: *P = 32; *T = 40; return;
        case 1440: *P = 30; *T = 48; return;
        case 1536: *P = 32; *T = 48; return;
        case 1600: *P = 32; *T = 50; return;
        case 1920: *P = 40; *T = 48; return;
        case 2000: *P = 40; *T = 50; return;
        default: *P = 0; *T = 0; return;
    }
}

cudaError_t launch_rows_mixed(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s) {
    return p->d.dtype == DDM_IN_U16 ? rows_dispatch<uint16_t>(p, frames, spec, s)
                                    : rows_dispatch<float>(p, frames, spec, s);
}

cudaError_t launch_cols_mixed(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out) {
    switch (p->d.H) {
        case 384: return cols_t<12, 32>(p, spec, s, out);
        case 480: return cols_t<15, 32>(p, spec, s, out);
        case 540: return cols_t<18, 30>(p, spec, s, out);
        case 600: return cols_t<24, 25>(p, spec, s, out);
        case 640: return cols_t<20, 32>(p, spec, s, out);
        case 720: return cols_t<24, 30>(p, spec, s, out);
        case 768: return cols_t<24, 32>(p, spec, s, out);
        case 800: return cols_t<25, 32>(p, spec, s, out);
        case 900: return cols_t<30, 30>(p, spec, s, out);
        case 960: return cols_t<30, 32>(p, spec, s, out);
        case 1000: return cols_t<25, 40, 512>(p, spec, s, out);
        case 1080: return cols_t<27, 40, 512>(p, spec, s, out);
        case 1200: return cols_t<30, 40, 512>(p, spec, s, out);
        case 1280: return cols_t<32, 40, 512>(p, spec, s, out);
        case 1440: return cols_t<30, 48>(p, spec, s, out);
        case 1536: return cols_t<32, 48>(p, spec, s, out);
        case 1600: return cols_t<32, 50>(p, spec, s, out);
        case 1920: return cols_t<40, 48, 512>(p, spec, s, out);
        case 2000: return cols_t<40, 50>(p, spec, s, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ddm
