// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ddm.h"

// Bluestein tables of one non-power-of-two transform length n (M = 2^ceil(log2(2n - 1))):
// chirp c_j = exp(i pi (j^2 mod 2n) / n), j < n; filter F = DFT_M(c circularly placed) / M;
// pass twiddles of M (and of its inner M/32 transform when M >= 2048).
struct ddm_bluestein {
    int n = 0, M = 0;
    float2* chirp = nullptr;
    float2* filt = nullptr;
    float2* tw = nullptr;
    float2* twin = nullptr;
};

// Mixed-radix transform of a side n = P T (P, T of the form 2^a 3^b 5^c): pass twiddles
// tw[k1 T + i] = exp(-2 pi i i k1 / n), k1 < P, i < T.
struct ddm_mixed {
    int n = 0, P = 0, T = 0;
    float2* tw = nullptr;
};

struct ddm_plan_s {
    ddm_plan_desc d;
    int L;              // transform length in time: smallest power of two >= N (M = 2L)
    int Wh;             // W / 2
    int64_t n_q;        // H * (W/2 + 1)
    int64_t q0, q1;     // stored wave vectors covered by step two and the radial stage
    int kc;             // low-frequency restriction: kmax (0 = full half plane)
    int kx0, nk;        // kx-column range [kx0, kx0 + nk) (nk = 0: every column); its store
                        // is [N][n_q], n_q = H nk (+ H for the kx = W/2 column when kx0 = 0)
    int64_t full_nq;    // H (W/2 + 1): frame stride of step one's whole-plane row output
    size_t inter_offset = 0;   // kx-column range: byte offset of that row output in the
                               // workspace (after the range's own store)
    ddm_bluestein blue_w, blue_h;   // rows / columns of non-power-of-two length
    ddm_mixed mix_w, mix_h;         // rows / columns of a mixed-radix side (before Bluestein)
    double2* tw64 = nullptr;        // FP64 tier: exp(-2 pi i r / fp64_ntab), r < fp64_ntab / 2
    double2* tw64_half = nullptr;   // FP64 tier: exp(-i pi t / L), t < L
    int fp64_ntab = 0;
    bool blocked = false;           // L >= 2048, large n_q: time kernels read a blocked copy of
                                    // [q0, q1) (16 wave vectors contiguous over time) made in the
                                    // workspace at byte offset blk_offset
    size_t blk_offset = 0;
    float2* crop_inter; // kc > 0: row-pass output [N][H][kc + 1]
    int device;
    int n_sm;
    int kd;             // number of trailing lags evaluated by direct differences
    int fix_lags;       // leading lags recomputed by direct differences (FP64FIX tier)
    // device tables owned by the plan
    float2* tw_row;     // pass twiddles of the W-point row transform
    float2* tw_col;     // pass twiddles of the H-point column transform
    float2* tw_t;       // pass twiddles of the L-point time transform
    float2* tw_tin;     // L >= 2048: pass twiddles of the inner L/32-point transform
    float2* tw_long;    // L >= 2048: (cos, sin) 2 pi k / L for k < L/4; exp(-i pi i / L) for
                        // i < L/32; exp(-i pi u / 32) for u < 32
    float2* tw2;        // exp(-i pi t / L), t < L
    float* inv;         // 1 / (N - m), m < N; 0 at m = 0
    float* tc_tables = nullptr;     // DDM_PREC_TC_TF32X3: DFT matrix images and twiddles of
                                    // the tensor-core column pass (tc_column_tables)
    int* bin_start;     // [n_bins + 1] CSR offsets into bin_q
    int* bin_q;         // per bin, ascending: (public q << 1) | (q stands for itself and -q)
    int* bin_count;     // [n_bins] full-plane modes per bin
    int max_bin_items;
    int n_chunks;       // radial partial sums: runs of <= 64 consecutive entries of one bin
    int* chunk_start;   // [n_chunks + 1] offsets into bin_q
    int* bin_chunk;     // [n_bins + 1] CSR offsets into the chunks
    float* radial_part; // [n_chunks][N] partial sums
    int* lag_j;         // fit: integer part of the 64 log lags
    float* lag_f;       // fit: fractional part
    float* lag_ll;      // fit: ln(lag)
    float* fit_scratch; // fit: features, plateaus, MLP outputs (grown on demand)
    size_t fit_scratch_bytes;
    unsigned* dev_status;   // kernel-reported status word
    cudaEvent_t stats_ev[3] = {nullptr, nullptr, nullptr};   // step-one / step-two timing
    bool stats_recorded = false;
    void* workspace;
    size_t ws_bytes;
    bool ws_owned;
};

namespace ddm {

// storage index of the spectrum: the first H*Wh entries of a frame are kx < W/2
// ([ky][kx]); the last H entries are the kx = W/2 column ([ky]).
size_t spectrum_frame_stride(const ddm_plan_s* p);   // complex elements per frame

// blk_out: write the column pass's output straight into the plan's blocked copy (when the
// chosen kernels can; *wrote_blocked tells) instead of in place
ddm_status launch_spatial(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s,
                          float2* blk_out = nullptr, bool* wrote_blocked = nullptr);
// pre_blocked: the plan's blocked copy already holds the spectrum (no corner-turn pass)
ddm_status launch_temporal(const ddm_plan_s* p, const float2* spec, float* D, cudaStream_t s,
                           bool pre_blocked = false);
// Where a column pass writes the spectrum entry (frame t, stored wave vector q): in place in
// the [t][q] spectrum (blk == nullptr), or into the blocked copy [b][t][16] of the range
// [q0, q1) that the long time kernels read (entries outside the range are not written).
// Or, for a kx-column range, into the range's store [t][n_qc] (entries of other columns
// are not written): stored index ky nk + (kx - kx0), then the kx = W/2 column (kx0 = 0).
struct SpecOut {
    float2* blk;
    int N;
    int64_t q0, q1;
    float2* col = nullptr;
    int64_t n_qc = 0;
    int H = 0, Wh = 0, kx0 = 0, nk = 0;
#ifdef __CUDACC__
    // the kx-column range store (its own kernel instances: the check stays out of the others)
    __device__ __forceinline__ void put_col(int t, int64_t q, float2 v) const {
        const int64_t main = (int64_t)H * Wh;
        int64_t cs;
        if (q < main) {
            const int64_t ky = q / Wh, kx = q - ky * Wh;
            if (kx < kx0 || kx >= kx0 + nk) return;
            cs = ky * nk + (kx - kx0);
        } else {
            if (kx0 != 0) return;
            cs = (int64_t)H * nk + (q - main);
        }
        col[(int64_t)t * n_qc + cs] = v;
    }
    __device__ __forceinline__ void put(float2* frame, int t, int64_t q, float2 v) const {
        if (!blk) {
            frame[q] = v;
            return;
        }
        const int64_t r = q - q0;
        if (r < 0 || q >= q1) return;
        blk[((r >> 4) * N + t) * 16 + (r & 15)] = v;
    }
#endif
};

// A TMA tensor map of float32 elements (no swizzle, zero fill out of bounds, 256-byte L2
// promotion): dims innermost first, strides in bytes of dimensions 1 .. rank - 1 (multiples
// of 16), box extents in elements.  False if the driver's encoder is missing or refuses.
bool encode_f32_tensor_map(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                           const cuuint64_t* strides, const cuuint32_t* box);
bool fp64_supported(const ddm_plan_desc& d);
bool tc_columns_supported(const ddm_plan_desc& d);
void tc_column_tables(float* out);
size_t tc_column_table_floats();
cudaError_t launch_cols_tc(const ddm_plan_s* p, float2* spec, cudaStream_t s);
ddm_status launch_fp64(const ddm_plan_s* p, const void* frames, void* workspace, float* D, cudaStream_t s);
void mixed_shape(int n, int* P, int* T);
cudaError_t launch_rows_mixed(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s);
cudaError_t launch_cols_mixed(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out);
cudaError_t launch_wait_selftest(unsigned* status, long long cap_cycles, cudaStream_t s);
cudaError_t launch_mlp_wait_selftest(unsigned* status, long long cap_cycles, cudaStream_t s);
cudaError_t launch_rows_bluestein(const ddm_plan_s* p, const void* frames, float2* spec, cudaStream_t s);
cudaError_t launch_cols_bluestein(const ddm_plan_s* p, float2* spec, cudaStream_t s, SpecOut out);
ddm_status launch_radial(const ddm_plan_s* p, const float* D, float* Dr, int* counts, bool normalise,
                         cudaStream_t s);

int ilog2(int v);
ddm_status make_fit_tables(ddm_plan_s* p);

}  // namespace ddm
