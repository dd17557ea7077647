// The FP64 tier (DDM_PREC_FP64): the whole structure-function path in double precision on
// the GPU, the reference tier of a precision sweep.  Same scheme as the FP32 kernels
// (Sec. 2 step one; App. B step two: the 2L-point transform of the zero-padded sequence as
// its even and odd bins, the inverse of the real spectrum by the 2-for-1 packing, power sums
// as prefix sums), written plainly: one radix-2 Stockham FFT in shared memory per transform,
// twiddles from a table built on the host in double precision.  B300's FP64 rate (about
// 1/64 of FP32) sets the speed, not the code's finesse.
//
// Spectrum workspace: complex128 [N][H][W/2 + 1] (public wave-vector order, q = ky (W/2 + 1)
// + kx), written by the row pass and transformed in place by the column pass.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddm_internal.h"

namespace ddm {
namespace {

constexpr int kFp64Threads = 512;

__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double zabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }

// Stockham radix-2 FFT of n = 2^k points (unnormalised; forward exp(-2 pi i jk / n), inverse
// the conjugate), ping-ponging between x and y; returns the buffer that holds the result.
// tw[r] = exp(-2 pi i r / n_tab) for r < n_tab / 2, n_tab a power of two >= n.
// Stage with half-span l and stride m (l m = n / 2): butterfly (j, k), j < l, k < m, maps
// x[k + j m], x[k + j m + l m] to y[k + 2 j m] = a + b, y[k + 2 j m + m] = w^j (a - b),
// w = exp(-/+ i pi / l).
__device__ double2* fft_stockham(double2* x, double2* y, int n, bool inv, const double2* tw, int n_tab) {
    for (int l = n >> 1, m = 1; l >= 1; l >>= 1, m <<= 1) {
        const int step = n_tab / (2 * l);                 // pi j / l = 2 pi (j step) / n_tab
        for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const int j = b / m, k = b - j * m;
            double2 w = tw[j * step];
            if (inv) w.y = -w.y;
            const double2 c0 = x[k + j * m], c1 = x[k + j * m + l * m];
            y[k + 2 * j * m] = zadd(c0, c1);
            y[k + 2 * j * m + m] = zmul(w, zsub(c0, c1));
        }
        __syncthreads();
        double2* t = x;
        x = y;
        y = t;
    }
    return x;
}

// ---- step one, rows: grid (H, N), one row of one frame per CTA; kx = 0 .. W/2 kept
template <typename In>
__global__ void __launch_bounds__(kFp64Threads)
fp64_rows_kernel(const In* __restrict__ frames, double2* __restrict__ spec, int H, int W,
                 int subtract_ref, const double2* __restrict__ tw_g, int n_tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* tw = reinterpret_cast<double2*>(smem_raw);
    double2* xa = tw + n_tab / 2;
    double2* xb = xa + W;
    for (int r = threadIdx.x; r < n_tab / 2; r += blockDim.x) tw[r] = tw_g[r];
    const int y = blockIdx.x, t = blockIdx.y;
    const In* row = frames + ((size_t)t * H + y) * W;
    const In* ref = frames + (size_t)y * W;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        double v = (double)row[x];
        if (subtract_ref) v -= (double)ref[x];            // exact: integers or floats in double
        xa[x] = make_double2(v, 0.0);
    }
    __syncthreads();
    const double2* X = fft_stockham(xa, xb, W, false, tw, n_tab);
    const int Wq = W / 2 + 1;
    double2* out = spec + ((size_t)t * H + y) * Wq;
    for (int k = threadIdx.x; k < Wq; k += blockDim.x) out[k] = X[k];
}

// ---- step one, columns: grid (W/2 + 1, N), one column of one frame per CTA, in place
__global__ void __launch_bounds__(kFp64Threads)
fp64_cols_kernel(double2* __restrict__ spec, int H, int Wq, const double2* __restrict__ tw_g, int n_tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* tw = reinterpret_cast<double2*>(smem_raw);
    double2* xa = tw + n_tab / 2;
    double2* xb = xa + H;
    for (int r = threadIdx.x; r < n_tab / 2; r += blockDim.x) tw[r] = tw_g[r];
    const int kx = blockIdx.x, t = blockIdx.y;
    double2* col = spec + (size_t)t * H * Wq + kx;
    for (int y = threadIdx.x; y < H; y += blockDim.x) xa[y] = col[(size_t)y * Wq];
    __syncthreads();
    const double2* X = fft_stockham(xa, xb, H, false, tw, n_tab);
    for (int ky = threadIdx.x; ky < H; ky += blockDim.x) col[(size_t)ky * Wq] = X[ky];
}

// ---- step two: one wave vector at a time per CTA (persistent over q)
// shared memory: tw [n_tab/2] | A [L] | B [L] | park [L] doubles | scan [NT/32] doubles;
// half[t] = exp(-i pi t / L), t < L, read from global memory (L2)
__global__ void __launch_bounds__(kFp64Threads)
fp64_temporal_kernel(const double2* __restrict__ spec, float* __restrict__ D, int N, int L, int64_t n_q,
                     const double2* __restrict__ tw_g, int n_tab, const double2* __restrict__ half,
                     unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* tw = reinterpret_cast<double2*>(smem_raw);
    double2* A = tw + n_tab / 2;
    double2* B = A + L;
    double* park = reinterpret_cast<double*>(B + L);
    double* wsum = park + L;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wg = tid >> 5;
    for (int r = tid; r < n_tab / 2; r += nt) tw[r] = tw_g[r];
    __syncthreads();
    bool bad = false;
    for (int64_t q = blockIdx.x; q < n_q; q += gridDim.x) {
        const double2* x = spec + q;                      // x(t) = x[t * n_q]
        // even bins: DFT_L of x (zero beyond N)
        for (int t = tid; t < L; t += nt) A[t] = t < N ? x[(int64_t)t * n_q] : make_double2(0.0, 0.0);
        __syncthreads();
        double2* Xe = fft_stockham(A, B, L, false, tw, n_tab);
        for (int k = tid; k < L; k += nt) park[k] = zabs2(Xe[k]);
        __syncthreads();
        // odd bins: DFT_L of x(t) exp(-i pi t / L)
        for (int t = tid; t < L; t += nt)
            A[t] = t < N ? zmul(x[(int64_t)t * n_q], __ldg(half + t)) : make_double2(0.0, 0.0);
        __syncthreads();
        double2* Xo = fft_stockham(A, B, L, false, tw, n_tab);
        // Z = |X_even|^2 + i |X_odd|^2, unnormalised inverse
        for (int k = tid; k < L; k += nt) Xo[k] = make_double2(park[k], zabs2(Xo[k]));
        __syncthreads();
        double2* z = fft_stockham(Xo, Xo == A ? B : A, L, true, tw, n_tab);
        // Re C(m), m < L, from the 2-for-1 packing: into park
        const double scale = 0.25 / (double)L;
        for (int m = tid; m < L; m += nt) {
            const double2 zm = z[m], zr = z[(L - m) & (L - 1)];
            const double2 w = __ldg(half + m);            // exp(-i pi m / L)
            park[m] = scale * ((zm.x + zr.x) + w.x * (zm.y + zr.y) - w.y * (zm.x - zr.x));
        }
        __syncthreads();
        // prefix sums S(k) = sum_{t < k} |x(t)|^2, k = 0 .. N, in the buffer z does not use
        double* S = reinterpret_cast<double*>(z == A ? B : A);
        const int per = (N + nt - 1) / nt, t0 = tid * per, t1 = min(N, t0 + per);
        double acc = 0.0;
        for (int t = t0; t < t1; ++t) acc += zabs2(x[(int64_t)t * n_q]);
        double incl = acc;
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[wg] = incl;
        __syncthreads();
        double off = incl - acc;
        for (int w = 0; w < wg; ++w) off += wsum[w];
        if (tid == 0) S[0] = 0.0;
        for (int t = t0; t < t1; ++t) {
            off += zabs2(x[(int64_t)t * n_q]);
            S[t + 1] = off;
        }
        __syncthreads();
        // D(m) = (S(N - m) + S(N) - S(m) - 2 Re C(m)) / (N - m), Eqs. B1-B2
        float* drow = D + q * (int64_t)N;
        const double total = S[N];
        for (int m = tid; m < N; m += nt) {
            double d = 0.0;
            if (m > 0) d = (S[N - m] + (total - S[m]) - 2.0 * park[m]) / (double)(N - m);
            if (!(d == d)) bad = true;
            drow[m] = (float)d;
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, 1u);
}

size_t fp64_temporal_smem(int L, int n_tab) {
    return sizeof(double2) * ((size_t)n_tab / 2 + 2 * (size_t)L) + sizeof(double) * ((size_t)L + kFp64Threads / 32);
}

}  // namespace

bool fp64_supported(const ddm_plan_desc& d) {
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    int L = 1;
    while (L < d.N) L *= 2;
    int n_tab = d.W > d.H ? d.W : d.H;
    if (L > n_tab) n_tab = L;
    return pow2(d.H) && pow2(d.W) && d.kmax == 0 && d.q_begin == 0 && d.q_end == 0 &&
           fp64_temporal_smem(L, n_tab) <= 232448;
}

ddm_status launch_fp64(const ddm_plan_s* p, const void* frames, void* workspace, float* D, cudaStream_t s) {
    const int H = p->d.H, W = p->d.W, N = p->d.N, L = p->L, Wq = W / 2 + 1;
    const int n_tab = p->fp64_ntab;
    double2* spec = reinterpret_cast<double2*>(workspace);
    const size_t smem_rows = sizeof(double2) * ((size_t)n_tab / 2 + 2 * (size_t)W);
    const size_t smem_cols = sizeof(double2) * ((size_t)n_tab / 2 + 2 * (size_t)H);
    const size_t smem_t = fp64_temporal_smem(L, n_tab);
    cudaError_t e;
    if (p->d.dtype == DDM_IN_U16) {
        e = cudaFuncSetAttribute(fp64_rows_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows);
        if (e == cudaSuccess)
            fp64_rows_kernel<uint16_t><<<dim3(H, N), kFp64Threads, smem_rows, s>>>(
                (const uint16_t*)frames, spec, H, W, p->d.subtract_ref, p->tw64, n_tab);
    } else {
        e = cudaFuncSetAttribute(fp64_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows);
        if (e == cudaSuccess)
            fp64_rows_kernel<float><<<dim3(H, N), kFp64Threads, smem_rows, s>>>(
                (const float*)frames, spec, H, W, p->d.subtract_ref, p->tw64, n_tab);
    }
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    if (cudaFuncSetAttribute(fp64_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    fp64_cols_kernel<<<dim3(Wq, N), kFp64Threads, smem_cols, s>>>(spec, H, Wq, p->tw64, n_tab);
    if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    if (cudaFuncSetAttribute(fp64_temporal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    const int64_t grid = p->n_q < p->n_sm ? p->n_q : p->n_sm;
    fp64_temporal_kernel<<<(unsigned)grid, kFp64Threads, smem_t, s>>>(spec, D, N, L, p->n_q, p->tw64, n_tab,
                                                                      p->tw64_half, p->dev_status);
    return cudaGetLastError() == cudaSuccess ? DDM_OK : DDM_ERR_CUDA;
}

}  // namespace ddm
