// Radial (azimuthal) average of D over |q| bins (not in the paper; the analysis step that
// turns D(q, dt) into D(|q|, dt)).  Deterministic: every lane sums its wave vectors of
// the bin in a fixed order, then a fixed xor-butterfly of warp shuffles combines lanes.
//
// Weights: stored wave vectors cover the half plane kx = 0 .. W/2; a mode with
// 0 < kx < W/2 stands for itself and its mirror -q (same bin, same D), so it counts twice.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddm_internal.h"

namespace ddm {
namespace {

constexpr int kLagsPerWarp = 8;     // 32 bytes of one D row per lane per wave vector
constexpr int kWarps = 8;

// grid: (n_bins, ceil(N / (kLagsPerWarp * kWarps))); block: 32 * kWarps.
__global__ void __launch_bounds__(32 * kWarps)
radial_kernel(const float* __restrict__ D, float* __restrict__ Dr, int N, int Wh,
              const int* __restrict__ bin_start, const int* __restrict__ bin_q,
              const int* __restrict__ bin_count, int normalise) {
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int m0 = (blockIdx.y * kWarps + warp) * kLagsPerWarp;
    if (m0 >= N) return;
    const int beg = bin_start[b], end = bin_start[b + 1];
    const bool vec = (N % 4) == 0 && (m0 + kLagsPerWarp) <= N &&
                     (reinterpret_cast<uintptr_t>(D) & 15) == 0;
    float acc[kLagsPerWarp];
#pragma unroll
    for (int j = 0; j < kLagsPerWarp; ++j) acc[j] = 0.f;
    for (int e = beg + lane; e < end; e += 32) {
        const int q = bin_q[e];
        const int kx = q % (Wh + 1);
        const float w = (kx == 0 || kx == Wh) ? 1.f : 2.f;
        const float* row = D + (int64_t)q * N + m0;
        if (vec) {
            const float4 x0 = __ldg(reinterpret_cast<const float4*>(row));
            const float4 x1 = __ldg(reinterpret_cast<const float4*>(row) + 1);
            acc[0] = fmaf(w, x0.x, acc[0]); acc[1] = fmaf(w, x0.y, acc[1]);
            acc[2] = fmaf(w, x0.z, acc[2]); acc[3] = fmaf(w, x0.w, acc[3]);
            acc[4] = fmaf(w, x1.x, acc[4]); acc[5] = fmaf(w, x1.y, acc[5]);
            acc[6] = fmaf(w, x1.z, acc[6]); acc[7] = fmaf(w, x1.w, acc[7]);
        } else {
#pragma unroll
            for (int j = 0; j < kLagsPerWarp; ++j)
                if (m0 + j < N) acc[j] = fmaf(w, __ldg(row + j), acc[j]);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int j = 0; j < kLagsPerWarp; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], off);
    }
    if (lane < kLagsPerWarp && m0 + lane < N) {
        const int c = bin_count[b];
        float val = 0.f;
#pragma unroll
        for (int j = 0; j < kLagsPerWarp; ++j)
            if (j == lane) val = acc[j];
        Dr[(int64_t)b * N + m0 + lane] = !normalise ? val : (c > 0 ? val / (float)c : 0.f);
    }
}

}  // namespace

ddm_status launch_radial(const ddm_plan_s* p, const float* D, float* Dr, int* counts, bool normalise,
                         cudaStream_t s) {
    const int n_bins = p->d.n_bins, N = p->d.N;
    dim3 grid(n_bins, (N + kLagsPerWarp * kWarps - 1) / (kLagsPerWarp * kWarps));
    radial_kernel<<<grid, 32 * kWarps, 0, s>>>(D, Dr, N, p->Wh, p->bin_start, p->bin_q,
                                               p->bin_count, normalise ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    if (counts) {
        if (cudaMemcpyAsync(counts, p->bin_count, sizeof(int) * (size_t)n_bins,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return DDM_ERR_CUDA;
    }
    return DDM_OK;
}

}  // namespace ddm
