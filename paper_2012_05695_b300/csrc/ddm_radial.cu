// Radial (azimuthal) average of D over |q| bins (not in the paper; the analysis step that
// turns D(q, dt) into D(|q|, dt)).
//
// Weights: stored wave vectors cover the half plane kx = 0 .. W/2; a mode with
// 0 < kx < W/2 stands for itself and its mirror -q (same bin, same D), so it counts twice.
//
// Two kernels, both with a fixed summation order (bitwise reproducible run to run):
//  * partial sums: a CTA takes one chunk (<= 64 consecutive entries of one bin's ascending
//    wave-vector list) and streams those whole D rows, each thread owning four consecutive
//    lags (one 16-byte load per row: a warp reads 512 contiguous bytes), four rows in
//    flight, summing the rows in list order;
//  * reduction: each bin's chunk sums added in chunk order, then divided by the bin's mode
//    count (or left as sums for a caller that adds several wave-vector ranges).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddm_internal.h"

namespace ddm {
namespace {

constexpr int kPartThreads = 256;   // x 4 lags = 1024 lags per CTA
constexpr int kReduceThreads = 256;

__device__ __forceinline__ float weight_of(int e) { return (e & 1) ? 2.f : 1.f; }

// grid: (n_chunks, ceil(N / 1024)); block: kPartThreads.
__global__ void __launch_bounds__(kPartThreads)
radial_partial_kernel(const float* __restrict__ D, float* __restrict__ part, int N,
                      const int* __restrict__ chunk_start, const int* __restrict__ bin_q, int vec4) {
    const int c = blockIdx.x;
    const int m0 = (blockIdx.y * kPartThreads + threadIdx.x) * 4;
    if (m0 >= N) return;
    const int beg = chunk_start[c], end = chunk_start[c + 1];
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (vec4) {   // N % 4 == 0 and D 16-byte aligned: m0 + 4 <= N
        int e = beg;
        for (; e + 4 <= end; e += 4) {
            const int q0 = bin_q[e], q1 = bin_q[e + 1], q2 = bin_q[e + 2], q3 = bin_q[e + 3];
            const float4 x0 = __ldg(reinterpret_cast<const float4*>(D + (int64_t)(q0 >> 1) * N + m0));
            const float4 x1 = __ldg(reinterpret_cast<const float4*>(D + (int64_t)(q1 >> 1) * N + m0));
            const float4 x2 = __ldg(reinterpret_cast<const float4*>(D + (int64_t)(q2 >> 1) * N + m0));
            const float4 x3 = __ldg(reinterpret_cast<const float4*>(D + (int64_t)(q3 >> 1) * N + m0));
            const float w0 = weight_of(q0), w1 = weight_of(q1), w2 = weight_of(q2), w3 = weight_of(q3);
            acc[0] = fmaf(w0, x0.x, acc[0]); acc[1] = fmaf(w0, x0.y, acc[1]);
            acc[2] = fmaf(w0, x0.z, acc[2]); acc[3] = fmaf(w0, x0.w, acc[3]);
            acc[0] = fmaf(w1, x1.x, acc[0]); acc[1] = fmaf(w1, x1.y, acc[1]);
            acc[2] = fmaf(w1, x1.z, acc[2]); acc[3] = fmaf(w1, x1.w, acc[3]);
            acc[0] = fmaf(w2, x2.x, acc[0]); acc[1] = fmaf(w2, x2.y, acc[1]);
            acc[2] = fmaf(w2, x2.z, acc[2]); acc[3] = fmaf(w2, x2.w, acc[3]);
            acc[0] = fmaf(w3, x3.x, acc[0]); acc[1] = fmaf(w3, x3.y, acc[1]);
            acc[2] = fmaf(w3, x3.z, acc[2]); acc[3] = fmaf(w3, x3.w, acc[3]);
        }
        for (; e < end; ++e) {
            const int q = bin_q[e];
            const float4 x = __ldg(reinterpret_cast<const float4*>(D + (int64_t)(q >> 1) * N + m0));
            const float w = weight_of(q);
            acc[0] = fmaf(w, x.x, acc[0]); acc[1] = fmaf(w, x.y, acc[1]);
            acc[2] = fmaf(w, x.z, acc[2]); acc[3] = fmaf(w, x.w, acc[3]);
        }
        *reinterpret_cast<float4*>(part + (int64_t)c * N + m0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    } else {
        for (int e = beg; e < end; ++e) {
            const int q = bin_q[e];
            const float* row = D + (int64_t)(q >> 1) * N + m0;
            const float w = weight_of(q);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (m0 + j < N) acc[j] = fmaf(w, __ldg(row + j), acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (m0 + j < N) part[(int64_t)c * N + m0 + j] = acc[j];
    }
}

// grid: (n_bins, ceil(N / kReduceThreads)); block: kReduceThreads.
__global__ void __launch_bounds__(kReduceThreads)
radial_reduce_kernel(const float* __restrict__ part, float* __restrict__ Dr, int N,
                     const int* __restrict__ bin_chunk, const int* __restrict__ bin_count,
                     int normalise) {
    const int b = blockIdx.x;
    const int m = blockIdx.y * kReduceThreads + threadIdx.x;
    if (m >= N) return;
    float s = 0.f;
    for (int c = bin_chunk[b]; c < bin_chunk[b + 1]; ++c) s += part[(int64_t)c * N + m];
    const int cnt = bin_count[b];
    Dr[(int64_t)b * N + m] = !normalise ? s : (cnt > 0 ? s / (float)cnt : 0.f);
}

}  // namespace

ddm_status launch_radial(const ddm_plan_s* p, const float* D, float* Dr, int* counts, bool normalise,
                         cudaStream_t s) {
    const int n_bins = p->d.n_bins, N = p->d.N;
    if (p->n_chunks > 0) {
        const int vec4 = (N % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
        dim3 g1(p->n_chunks, (N + 4 * kPartThreads - 1) / (4 * kPartThreads));
        radial_partial_kernel<<<g1, kPartThreads, 0, s>>>(D, p->radial_part, N, p->chunk_start, p->bin_q,
                                                          vec4);
        if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    }
    dim3 g2(n_bins, (N + kReduceThreads - 1) / kReduceThreads);
    radial_reduce_kernel<<<g2, kReduceThreads, 0, s>>>(p->radial_part, Dr, N, p->bin_chunk, p->bin_count,
                                                       normalise ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    if (counts) {
        if (cudaMemcpyAsync(counts, p->bin_count, sizeof(int) * (size_t)n_bins,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return DDM_ERR_CUDA;
    }
    return DDM_OK;
}

}  // namespace ddm
