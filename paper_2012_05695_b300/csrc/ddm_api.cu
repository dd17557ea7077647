// C ABI of the library: plan life cycle, validation, tables, and the entry points of
// include/ddm.h.  No exception crosses this boundary; every failure is a status code.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ddm_fft.cuh"
#include "ddm_internal.h"

namespace ddm {

int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

constexpr int kRadialChunk = 64;   // wave vectors per radial partial sum

constexpr int kMaxSide = 2048;         // powers of two; mixed-radix sides up to 2000; others up to 1022
constexpr int kMaxFrames = 16384;
// stored wave vectors from which the time kernels read a blocked copy (measured: at L = 16384
// 512x512 gains 1.11x with the copy included; at L = 4096 512x512 (131584) loses 1.3x, while
// 600x800 (240600) gains 1.10x and 1024x1024 1.5x)
constexpr int64_t kBlockedMinQ16k = 100000;
constexpr int64_t kBlockedMinQ = 200000;

// floor(n_bins * |q| / (pi sqrt 2)) with |q| = 2 pi sqrt((ky/H)^2 + (kx/W)^2):
// the largest b with (b H W)^2 <= 2 n_bins^2 (ky^2 W^2 + kx^2 H^2), in exact integers.
int radial_bin(int ky_signed, int kx_signed, int H, int W, int n_bins) {
    typedef unsigned __int128 u128;
    const u128 ky2 = (u128)((int64_t)ky_signed * ky_signed), kx2 = (u128)((int64_t)kx_signed * kx_signed);
    const u128 K = ky2 * (u128)W * (u128)W + kx2 * (u128)H * (u128)H;
    const u128 rhs = (u128)2 * (u128)n_bins * (u128)n_bins * K;
    const u128 hw2 = (u128)H * W * (u128)H * W;
    // upper estimate then step down; b <= n_bins * sqrt(2) / 2 * sqrt(2) ~ n_bins
    int64_t lo = 0, hi = (int64_t)2 * n_bins + 2;
    while (lo < hi) {          // largest b with b^2 hw2 <= rhs
        const int64_t mid = (lo + hi + 1) / 2;
        if ((u128)mid * (u128)mid * hw2 <= rhs) lo = mid; else hi = mid - 1;
    }
    return (int)std::min<int64_t>(lo, n_bins - 1);
}

template <typename T>
ddm_status upload(T** dst, const std::vector<T>& host) {
    *dst = nullptr;
    if (host.empty()) return DDM_OK;
    if (cudaMalloc((void**)dst, sizeof(T) * host.size()) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return DDM_ERR_OOM;
    }
    if (cudaMemcpy(*dst, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return DDM_ERR_CUDA;
    return DDM_OK;
}

void free_plan(ddm_plan_s* p) {
    if (!p) return;
    for (cudaEvent_t& e : p->stats_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(p->tw_row);
    cudaFree(p->tw_col);
    cudaFree(p->tw_t);
    cudaFree(p->tw_tin);
    cudaFree(p->mix_w.tw);
    cudaFree(p->mix_h.tw);
    cudaFree(p->tw64);
    cudaFree(p->tw64_half);
    for (ddm_bluestein* b : {&p->blue_w, &p->blue_h}) {
        cudaFree(b->chirp);
        cudaFree(b->filt);
        cudaFree(b->tw);
        cudaFree(b->twin);
    }
    cudaFree(p->tw_long);
    cudaFree(p->tc_tables);
    cudaFree(p->tw2);
    cudaFree(p->inv);
    cudaFree(p->bin_start);
    cudaFree(p->bin_q);
    cudaFree(p->bin_count);
    cudaFree(p->chunk_start);
    cudaFree(p->bin_chunk);
    cudaFree(p->radial_part);
    cudaFree(p->crop_inter);
    cudaFree(p->lag_j);
    cudaFree(p->lag_f);
    cudaFree(p->lag_ll);
    cudaFree(p->fit_scratch);
    cudaFree(p->dev_status);
    if (p->ws_owned) cudaFree(p->workspace);
    delete p;
}

std::vector<float2> pass_twiddles(int L);

// Bluestein tables for length n, built in double precision: the chirp's angle reduced
// exactly (j^2 mod 2n in integers), the filter's DFT by a plain O(M^2) sum in double.
ddm_status make_bluestein(ddm_bluestein* b, int n) {
    int M = 32;                                          // the register FFTs' smallest shape
    while (M < 2 * n - 1) M *= 2;
    b->n = n;
    b->M = M;
    std::vector<double> cr(n), ci(n);
    for (int j = 0; j < n; ++j) {
        const long r = (long)((long long)j * j % (2LL * n));
        const cx_cs cs = cx_cossin_frac(r, 2L * n);      // angle 2 pi r / 2n = pi r / n
        cr[j] = cs.c;
        ci[j] = cs.s;
    }
    std::vector<double> pr(M, 0.0), pi(M, 0.0);          // c placed circularly: c_{-m} = c_m
    for (int j = 0; j < n; ++j) {
        pr[j] = cr[j];
        pi[j] = ci[j];
        if (j > 0) {
            pr[M - j] = cr[j];
            pi[M - j] = ci[j];
        }
    }
    std::vector<float2> chirp(n), filt(M);
    for (int j = 0; j < n; ++j) chirp[j] = make_float2((float)cr[j], (float)ci[j]);
    std::vector<double> wc(M), ws(M);                    // cos / sin of 2 pi r / M
    for (int r = 0; r < M; ++r) {
        const cx_cs w = cx_cossin_frac(r, M);
        wc[r] = w.c;
        ws[r] = w.s;
    }
    for (int k = 0; k < M; ++k) {
        double sr = 0.0, si = 0.0;
        for (int m = 0, r = 0; m < M; ++m, r = (r + k) & (M - 1)) {   // r = k m mod M
            sr += pr[m] * wc[r] + pi[m] * ws[r];                        // times exp(-2 pi i r / M)
            si += pi[m] * wc[r] - pr[m] * ws[r];
        }
        filt[k] = make_float2((float)(sr / M), (float)(si / M));
    }
    ddm_status st = upload(&b->chirp, chirp);
    if (st == DDM_OK) st = upload(&b->filt, filt);
    if (st == DDM_OK && M >= 64) st = upload(&b->tw, pass_twiddles(M));
    if (st == DDM_OK && M >= 2048) st = upload(&b->twin, pass_twiddles(M / 32));
    return st;
}

// A side of a mixed-radix shape n = P T: the pass twiddles, built in double precision.
ddm_status make_mixed(ddm_mixed* m, int n) {
    int P = 0, T = 0;
    mixed_shape(n, &P, &T);
    if (P == 0) return DDM_ERR_UNSUPPORTED;
    m->n = n;
    m->P = P;
    m->T = T;
    std::vector<float2> tw((size_t)n);
    for (int k1 = 0; k1 < P; ++k1)
        for (int i = 0; i < T; ++i) {
            const cx_cs cs = cx_cossin_frac((long)((long)i * k1 % n), n);
            tw[(size_t)k1 * T + i] = make_float2((float)cs.c, (float)-cs.s);
        }
    return upload(&m->tw, tw);
}

// A power-of-two side of 2048 points: the Bluestein kernels' three-pass transform alone.
ddm_status make_direct(ddm_bluestein* b, int n) {
    b->n = n;
    b->M = n;
    ddm_status st = upload(&b->tw, pass_twiddles(n));
    if (st == DDM_OK) st = upload(&b->twin, pass_twiddles(n / 32));
    return st;
}

std::vector<float2> pass_twiddles(int L) {
    std::vector<float2> t;
    if (L >= 64) {
        t.resize(L);
        host_pass_twiddles(L, t.data());
    }
    return t;
}

bool kx_ranged(const ddm_plan_desc& d) { return d.kx_begin != 0 || d.kx_end != 0; }

size_t stored_wave_vectors(const ddm_plan_desc& d) {
    if (d.kmax > 0) return (size_t)(2 * d.kmax + 1) * (size_t)(d.kmax + 1);
    if (kx_ranged(d))
        return (size_t)d.H * (size_t)(d.kx_end - d.kx_begin) + (d.kx_begin == 0 ? (size_t)d.H : 0);
    return (size_t)d.H * (size_t)(d.W / 2 + 1);
}

// kx-column range: step one's whole-plane row output, after the range's store
size_t row_output_bytes(const ddm_plan_desc& d) {
    if (!kx_ranged(d)) return 0;
    return (size_t)d.H * (size_t)(d.W / 2 + 1) * (size_t)d.N * sizeof(float2);
}

size_t spectrum_bytes(const ddm_plan_desc& d) {
    const size_t nq = stored_wave_vectors(d);
    const size_t elem = d.precision == DDM_PREC_FP64 ? 2 * sizeof(double) : sizeof(float2);
    const size_t b = nq * (size_t)d.N * elem;
    return (b + 255) & ~(size_t)255;
}

// Bytes of the blocked copy of the plan's wave-vector range (16 per block, N frames each).
size_t blocked_bytes(const ddm_plan_desc& d) {
    const int64_t nq = (int64_t)stored_wave_vectors(d);
    const bool ranged = d.q_begin != 0 || d.q_end != 0;
    const int64_t n = ranged ? d.q_end - d.q_begin : nq;
    return (size_t)((n + 15) / 16) * (size_t)d.N * 16 * sizeof(float2);
}

// The time kernels for L >= 2048 read a blocked copy when the [t][q] spectrum's row stride
// (n_q * 8 bytes) makes a tile touch too many scattered DRAM pages, and the workspace limit
// allows the extra copy.
bool spectrum_blocked(const ddm_plan_desc& d) {
    const int L = 1 << ilog2(d.N);
    if (L < 2048 || d.precision == DDM_PREC_FP64 || kx_ranged(d)) return false;
    if ((int64_t)stored_wave_vectors(d) < (L == 16384 ? kBlockedMinQ16k : kBlockedMinQ)) return false;
    if (d.max_workspace_bytes != 0 && spectrum_bytes(d) + blocked_bytes(d) > d.max_workspace_bytes)
        return false;
    return true;
}

size_t workspace_bytes(const ddm_plan_desc& d) {
    return spectrum_bytes(d) + (spectrum_blocked(d) ? blocked_bytes(d) : 0) + row_output_bytes(d);
}

ddm_status validate(const ddm_plan_desc* d) {
    if (!d) return DDM_ERR_INVALID_ARG;
    if (d->H < 2 || d->W < 2 || d->H % 2 != 0 || d->W % 2 != 0) return DDM_ERR_INVALID_ARG;
    if (d->H > kMaxSide || d->W > kMaxSide) return DDM_ERR_UNSUPPORTED;
    {   // above 1024 pixels: powers of two, or a side the mixed-radix kernels are built for
        int P = 0, T = 0;
        mixed_shape(d->H, &P, &T);
        if (!is_pow2(d->H) && d->H > 1024 && P == 0) return DDM_ERR_UNSUPPORTED;
        mixed_shape(d->W, &P, &T);
        if (!is_pow2(d->W) && d->W > 1024 && P == 0) return DDM_ERR_UNSUPPORTED;
    }
    if (d->N < 1) return DDM_ERR_INVALID_ARG;
    if (d->N > kMaxFrames) return DDM_ERR_UNSUPPORTED;
    if (d->dtype != DDM_IN_U16 && d->dtype != DDM_IN_F32) return DDM_ERR_INVALID_ARG;
    if (d->precision != DDM_PREC_FP32 && d->precision != DDM_PREC_FP32_FP64FIX &&
        d->precision != DDM_PREC_FP64 && d->precision != DDM_PREC_TC_TF32X3)
        return DDM_ERR_INVALID_ARG;
    if (d->precision == DDM_PREC_TC_TF32X3 && !tc_columns_supported(*d)) return DDM_ERR_UNSUPPORTED;
    if (d->precision == DDM_PREC_FP32_FP64FIX) {
        // built for the time transforms whose tiles arrive whole in shared memory
        const int Lf = 1 << ilog2(d->N);
        if (Lf < 512 || Lf > 8192) return DDM_ERR_UNSUPPORTED;
        if (d->fix_lags > 8) return DDM_ERR_UNSUPPORTED;
    }
    if (d->subtract_ref != 0 && d->subtract_ref != 1) return DDM_ERR_INVALID_ARG;
    if (d->n_bins < 0 || d->n_bins > (1 << 20)) return DDM_ERR_INVALID_ARG;
    if (d->fix_lags < 0) return DDM_ERR_INVALID_ARG;
    if (d->spatial_path != DDM_SPATIAL_TWO_PASS && d->spatial_path != DDM_SPATIAL_FUSED)
        return DDM_ERR_INVALID_ARG;
    const int L = 1 << ilog2(d->N);
    if (d->M != 0) {
        if ((int64_t)d->M < 2 * (int64_t)d->N - 1) return DDM_ERR_INVALID_ARG;
        if (d->M != 2 * L) return DDM_ERR_UNSUPPORTED;
    }
    if (d->kmax < 0) return DDM_ERR_INVALID_ARG;
    if (d->kmax > 0 && (d->kmax % 2 == 0 || d->kmax >= d->H / 2 || d->kmax >= d->W / 2))
        return DDM_ERR_INVALID_ARG;
    if (d->kmax > 0 && (!is_pow2(d->H) || !is_pow2(d->W) || d->H > 1024 || d->W > 1024))
        return DDM_ERR_UNSUPPORTED;
    if (d->q_begin != 0 || d->q_end != 0) {
        const int64_t nq = (int64_t)stored_wave_vectors(*d);
        if (d->q_begin < 0 || d->q_begin % 64 != 0 || d->q_end <= d->q_begin || d->q_end > nq)
            return DDM_ERR_INVALID_ARG;
    }
    if (kx_ranged(*d)) {
        const int Wh = d->W / 2;
        if (d->kx_begin < 0 || d->kx_begin % 16 != 0 || d->kx_end % 16 != 0 ||
            d->kx_end <= d->kx_begin || d->kx_end > Wh)
            return DDM_ERR_INVALID_ARG;
        if (!is_pow2(d->H) || !is_pow2(d->W) || d->W < 32 || d->H > 1024 || d->W > 1024 ||
            d->kmax != 0 || d->q_begin != 0 || d->q_end != 0 || d->precision == DDM_PREC_FP64 ||
            d->spatial_path != DDM_SPATIAL_TWO_PASS)
            return DDM_ERR_UNSUPPORTED;
    }
    if (d->precision == DDM_PREC_FP64 && !fp64_supported(*d)) return DDM_ERR_UNSUPPORTED;
    if (d->max_workspace_bytes != 0 && workspace_bytes(*d) > d->max_workspace_bytes)
        return DDM_ERR_OOM;
    return DDM_OK;
}

bool check_plan(ddm_plan p) { return p != nullptr; }

ddm_status ensure_workspace(ddm_plan_s* p) {
    if (p->workspace) return DDM_OK;
    const size_t need = workspace_bytes(p->d);
    if (cudaMalloc(&p->workspace, need) != cudaSuccess) {
        cudaGetLastError();
        p->workspace = nullptr;
        return DDM_ERR_OOM;
    }
    p->ws_bytes = need;
    p->ws_owned = true;
    return DDM_OK;
}

}  // namespace
}  // namespace ddm

using namespace ddm;

extern "C" {

int ddm_abi_version(void) { return DDM_ABI_VERSION; }

size_t ddm_plan_desc_size(void) { return sizeof(ddm_plan_desc); }

const char* ddm_status_string(ddm_status s) {
    switch (s) {
        case DDM_OK: return "ok";
        case DDM_ERR_INVALID_ARG: return "invalid argument";
        case DDM_ERR_UNSUPPORTED: return "unsupported by this library";
        case DDM_ERR_OOM: return "out of device memory or over the workspace limit";
        case DDM_ERR_CUDA: return "CUDA runtime error";
        case DDM_ERR_TIMEOUT: return "bounded device wait timed out";
        case DDM_ERR_NUMERIC: return "non-finite value in a kernel";
        case DDM_ERR_NO_WORKSPACE: return "no workspace";
        default: return "unknown status";
    }
}

ddm_status ddm_plan_desc_init(ddm_plan_desc* desc, int H, int W, int N) {
    if (!desc) return DDM_ERR_INVALID_ARG;
    memset(desc, 0, sizeof(*desc));
    desc->H = H;
    desc->W = W;
    desc->N = N;
    desc->dtype = DDM_IN_U16;
    desc->precision = DDM_PREC_FP32;
    desc->subtract_ref = 1;
    return DDM_OK;
}

ddm_status ddm_plan_create(ddm_plan* out, const ddm_plan_desc* desc) {
    if (!out) return DDM_ERR_INVALID_ARG;
    *out = nullptr;
    const ddm_status v = validate(desc);
    if (v != DDM_OK) return v;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    ddm_plan_s* p = new (std::nothrow) ddm_plan_s();
    if (!p) return DDM_ERR_OOM;
    p->d = *desc;
    p->device = dev;
    p->L = 1 << ilog2(desc->N);
    p->Wh = desc->W / 2;
    p->kc = desc->kmax;
    p->kx0 = kx_ranged(*desc) ? desc->kx_begin : 0;
    p->nk = kx_ranged(*desc) ? desc->kx_end - desc->kx_begin : 0;
    p->full_nq = (int64_t)desc->H * (desc->W / 2 + 1);
    p->n_q = (int64_t)stored_wave_vectors(*desc);
    p->inter_offset = spectrum_bytes(*desc);
    const bool ranged = desc->q_begin != 0 || desc->q_end != 0;
    p->q0 = ranged ? desc->q_begin : 0;
    p->q1 = ranged ? desc->q_end : p->n_q;
    p->blocked = spectrum_blocked(*desc);
    p->blk_offset = spectrum_bytes(*desc);
    // trailing lags taken by differences: the FFT route's FP32 error in D(m) grows like
    // N / (N - m), so the last N / 32 lags (at most 32, at least 1) go by differences and
    // the factor stays below 32 at every N
    p->kd = std::min(std::min(32, std::max(1, desc->N / 32)), desc->N - 1);
    p->fix_lags = desc->fix_lags > 0 ? desc->fix_lags : 8;
    if (cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return DDM_ERR_CUDA;
    }
    ddm_status st = DDM_OK;
    // pass twiddles of the three transform lengths
    const bool pow2_w = is_pow2(desc->W), pow2_h = is_pow2(desc->H);
    if (st == DDM_OK && pow2_w && desc->W <= 1024) st = upload(&p->tw_row, pass_twiddles(desc->W));
    if (st == DDM_OK && pow2_h && desc->H <= 1024) st = upload(&p->tw_col, pass_twiddles(desc->H));
    // Bluestein tables: rows when W is not a power of two; columns when either side is not
    // (the power-of-two column kernel takes whole blocks of 16 stored columns).  Sides of
    // 2048: the same kernels' 2048-point transform alone (no chirp).
    // mixed-radix kernels first for the sides they are built for (mixed_shape)
    int mP = 0, mT = 0;
    mixed_shape(desc->W, &mP, &mT);
    const bool mix_w = mP > 0;
    mixed_shape(desc->H, &mP, &mT);
    const bool mix_h = mP > 0;
    if (st == DDM_OK && mix_w) st = make_mixed(&p->mix_w, desc->W);
    else if (st == DDM_OK && !pow2_w) st = make_bluestein(&p->blue_w, desc->W);
    if (st == DDM_OK && desc->W == 2048) st = make_direct(&p->blue_w, 2048);
    if (st == DDM_OK && desc->H == 2048) st = make_direct(&p->blue_h, 2048);
    else if (st == DDM_OK && !(pow2_w && pow2_h)) {
        if (mix_h) st = make_mixed(&p->mix_h, desc->H);
        else st = make_bluestein(&p->blue_h, desc->H);
    }
    if (st == DDM_OK) st = upload(&p->tw_t, pass_twiddles(p->L));
    if (st == DDM_OK && p->L >= 2048) st = upload(&p->tw_tin, pass_twiddles(p->L / 32));
    if (st == DDM_OK && p->L >= 2048) {
        const int L = p->L, Tl = L / 32;
        std::vector<float2> t;
        for (int k = 0; k < L / 4; ++k) {
            const cx_cs cs = cx_cossin_frac(k, L);
            t.push_back(make_float2((float)cs.c, (float)cs.s));
        }
        for (int i = 0; i < Tl; ++i) {
            const cx_cs cs = cx_cossin_frac(i, 2L * L);
            t.push_back(make_float2((float)cs.c, (float)-cs.s));
        }
        for (int u = 0; u < 32; ++u) {
            const cx_cs cs = cx_cossin_frac(u, 64);
            t.push_back(make_float2((float)cs.c, (float)-cs.s));
        }
        // two-level pass-1 twiddles of the L = 16384 kernel: exp(-2 pi i b / L), b < 64, and
        // exp(-2 pi i 64 a / L), a < L / 64
        for (int b = 0; b < 64; ++b) {
            const cx_cs cs = cx_cossin_frac(b, L);
            t.push_back(make_float2((float)cs.c, (float)-cs.s));
        }
        for (int a2 = 0; a2 < L / 64; ++a2) {
            const cx_cs cs = cx_cossin_frac(64L * a2, L);
            t.push_back(make_float2((float)cs.c, (float)-cs.s));
        }
        st = upload(&p->tw_long, t);
    }
    // exp(-i pi t / L) and 1/(N - m)
    if (st == DDM_OK) {
        std::vector<float2> tw2(p->L);
        std::vector<float> inv(p->L, 0.f);
        for (int t = 0; t < p->L; ++t) {
            const cx_cs cs = cx_cossin_frac(t, (long)2 * p->L);
            tw2[t] = make_float2((float)cs.c, (float)-cs.s);
        }
        for (int m = 1; m < desc->N; ++m) inv[m] = (float)(1.0 / (double)(desc->N - m));
        st = upload(&p->tw2, tw2);
        if (st == DDM_OK) st = upload(&p->inv, inv);
    }
    // radial bins: CSR of public q per bin (ascending), full-plane counts, over the stored
    // wave vectors of the plan's range
    if (st == DDM_OK && desc->n_bins > 0) {
        const int H = desc->H, W = desc->W, Wh = p->Wh, nb = desc->n_bins;
        // D row of (ky, kx) and its stored index: the full half plane (D row ky*(Wh+1)+kx;
        // stored main block then the kx = W/2 column) or the cropped window (both in the
        // window's order)
        // (a kx-column range: the range's columns, D rows in the whole plane's order)
        const int KC = p->kc;
        const int rows = KC > 0 ? 2 * KC + 1 : H, cols = KC > 0 ? KC + 1 : Wh + 1;
        const int64_t n_rows_d = (int64_t)rows * cols;      // D rows indexed below
        std::vector<int> bin_of((size_t)n_rows_d, -1);
        std::vector<int> count(nb, 0), start(nb + 1, 0);
        for (int r = 0; r < rows; ++r) {
            const int ys = KC > 0 ? (r <= KC ? r : r - (2 * KC + 1)) : (r > H / 2 ? r - H : r);
            for (int kx = 0; kx < cols; ++kx) {
                int64_t stored;
                if (KC > 0) {
                    stored = (int64_t)r * cols + kx;
                } else if (p->nk > 0) {
                    if (kx < Wh && (kx < p->kx0 || kx >= p->kx0 + p->nk)) continue;
                    if (kx == Wh && p->kx0 != 0) continue;
                    stored = kx < Wh ? (int64_t)r * p->nk + (kx - p->kx0) : (int64_t)H * p->nk + r;
                } else {
                    stored = kx < Wh ? (int64_t)r * Wh + kx : (int64_t)H * Wh + r;
                }
                if (stored < p->q0 || stored >= p->q1) continue;
                const int b = radial_bin(ys, kx, H, W, nb);
                bin_of[(size_t)r * cols + kx] = b;
                count[b] += (kx == 0 || (KC == 0 && kx == Wh)) ? 1 : 2;
                start[b + 1] += 1;
            }
        }
        for (int b = 0; b < nb; ++b) start[b + 1] += start[b];
        std::vector<int> items((size_t)start[nb] > 0 ? (size_t)start[nb] : 1), fill(start.begin(), start.end() - 1);
        for (int64_t q = 0; q < n_rows_d; ++q) {
            if (bin_of[q] < 0) continue;
            const int kx = (int)(q % cols);
            const bool single = kx == 0 || (KC == 0 && kx == Wh);
            items[fill[bin_of[q]]++] = (int)(q << 1) | (single ? 0 : 1);
        }
        // chunks of <= kRadialChunk entries, never crossing a bin
        std::vector<int> cstart, bchunk(nb + 1, 0);
        for (int b = 0; b < nb; ++b) {
            bchunk[b] = (int)cstart.size();
            for (int e = start[b]; e < start[b + 1]; e += kRadialChunk) cstart.push_back(e);
        }
        bchunk[nb] = (int)cstart.size();
        cstart.push_back(start[nb]);
        p->n_chunks = bchunk[nb];
        st = upload(&p->bin_start, start);
        if (st == DDM_OK) st = upload(&p->bin_q, items);
        if (st == DDM_OK) st = upload(&p->bin_count, count);
        if (st == DDM_OK) st = upload(&p->chunk_start, cstart);
        if (st == DDM_OK) st = upload(&p->bin_chunk, bchunk);
        if (st == DDM_OK && p->n_chunks > 0) {
            if (cudaMalloc(&p->radial_part, sizeof(float) * (size_t)p->n_chunks * desc->N) != cudaSuccess) {
                cudaGetLastError();
                st = DDM_ERR_OOM;
            }
        }
    }
    if (st == DDM_OK && p->kc > 0) {
        const size_t bytes = sizeof(float2) * (size_t)desc->N * desc->H * (size_t)(p->kc + 1);
        if (cudaMalloc(&p->crop_inter, bytes) != cudaSuccess) {
            cudaGetLastError();
            st = DDM_ERR_OOM;
        }
    }
    if (st == DDM_OK && desc->precision == DDM_PREC_FP64) {
        // FP64 tier: exp(-2 pi i r / n_tab), r < n_tab / 2, n_tab = max(W, H, L); and
        // exp(-i pi t / L), t < L
        int n_tab = desc->W > desc->H ? desc->W : desc->H;
        if (p->L > n_tab) n_tab = p->L;
        p->fp64_ntab = n_tab;
        std::vector<double2> t64(n_tab / 2 > 0 ? n_tab / 2 : 1), h64(p->L);
        for (int r = 0; r < n_tab / 2; ++r) {
            const cx_cs cs = cx_cossin_frac(r, n_tab);
            t64[r] = make_double2(cs.c, -cs.s);
        }
        if (n_tab < 2) t64[0] = make_double2(1.0, 0.0);
        for (int t = 0; t < p->L; ++t) {
            const cx_cs cs = cx_cossin_frac(t, 2L * p->L);
            h64[t] = make_double2(cs.c, -cs.s);
        }
        st = upload(&p->tw64, t64);
        if (st == DDM_OK) st = upload(&p->tw64_half, h64);
    }
    if (st == DDM_OK && desc->precision == DDM_PREC_TC_TF32X3) {
        std::vector<float> t(tc_column_table_floats());
        tc_column_tables(t.data());
        st = upload(&p->tc_tables, t);
    }
    if (st == DDM_OK) st = make_fit_tables(p);
    if (st == DDM_OK) {
        if (cudaMalloc(&p->dev_status, sizeof(unsigned)) != cudaSuccess ||
            cudaMemset(p->dev_status, 0, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            st = DDM_ERR_CUDA;
        }
    }
    if (st != DDM_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return DDM_OK;
}

ddm_status ddm_plan_destroy(ddm_plan p) {
    free_plan(p);
    return DDM_OK;
}

ddm_status ddm_plan_workspace_size(ddm_plan p, size_t* bytes) {
    if (!check_plan(p) || !bytes) return DDM_ERR_INVALID_ARG;
    *bytes = workspace_bytes(p->d);
    return DDM_OK;
}

ddm_status ddm_plan_set_workspace(ddm_plan p, void* dev_ptr, size_t bytes) {
    if (!check_plan(p) || !dev_ptr) return DDM_ERR_INVALID_ARG;
    if (bytes < workspace_bytes(p->d) || (reinterpret_cast<uintptr_t>(dev_ptr) & 255) != 0)
        return DDM_ERR_INVALID_ARG;
    if (p->ws_owned) cudaFree(p->workspace);
    p->workspace = dev_ptr;
    p->ws_bytes = bytes;
    p->ws_owned = false;
    return DDM_OK;
}

ddm_status ddm_plan_n_q(ddm_plan p, int64_t* n_q) {
    if (!check_plan(p) || !n_q) return DDM_ERR_INVALID_ARG;
    *n_q = p->n_q;
    return DDM_OK;
}

ddm_status ddm_plan_enable_stats(ddm_plan p, int on) {
    if (!check_plan(p)) return DDM_ERR_INVALID_ARG;
    for (cudaEvent_t& e : p->stats_ev) {
        if (on && !e && cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
            return DDM_ERR_CUDA;
        }
        if (!on && e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    }
    p->stats_recorded = false;
    return DDM_OK;
}

ddm_status ddm_plan_stats(ddm_plan p, float* step_one_ms, float* step_two_ms) {
    if (!check_plan(p) || !step_one_ms || !step_two_ms) return DDM_ERR_INVALID_ARG;
    if (!p->stats_recorded) return DDM_ERR_INVALID_ARG;
    if (cudaEventSynchronize(p->stats_ev[2]) != cudaSuccess ||
        cudaEventElapsedTime(step_one_ms, p->stats_ev[0], p->stats_ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(step_two_ms, p->stats_ev[1], p->stats_ev[2]) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    return DDM_OK;
}

ddm_status ddm_selftest_bounded_wait(long long cap_cycles) {
    if (cap_cycles < 1000) cap_cycles = 1000;
    if (cap_cycles > 4000000000LL) cap_cycles = 4000000000LL;
    unsigned* word = nullptr;   // [0]: the tile-barrier wait, [1]: the MMA-barrier wait
    if (cudaMalloc(&word, 2 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    unsigned h[2] = {0, 0};
    bool ok = cudaMemset(word, 0, 2 * sizeof(unsigned)) == cudaSuccess &&
              launch_wait_selftest(word, cap_cycles, nullptr) == cudaSuccess &&
              launch_mlp_wait_selftest(word + 1, cap_cycles, nullptr) == cudaSuccess &&
              cudaMemcpy(h, word, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(word);
    if (!ok) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    return ((h[0] & 2u) && (h[1] & 2u)) ? DDM_ERR_TIMEOUT : DDM_OK;
}

ddm_status ddm_plan_last_device_status(ddm_plan p, ddm_status* out) {
    if (!check_plan(p) || !out) return DDM_ERR_INVALID_ARG;
    unsigned h = 0;
    if (cudaMemcpy(&h, p->dev_status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(p->dev_status, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    *out = (h & 2u) ? DDM_ERR_TIMEOUT : (h & 1u) ? DDM_ERR_NUMERIC : DDM_OK;
    return DDM_OK;
}

ddm_status ddm_spatial_fft(ddm_plan p, const void* frames, float* spectrum, void* stream) {
    if (!check_plan(p) || !frames || !spectrum) return DDM_ERR_INVALID_ARG;
    if (p->d.precision == DDM_PREC_FP64) return DDM_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(spectrum) & 7) != 0) return DDM_ERR_INVALID_ARG;
    if (p->nk > 0) {                       // the whole-plane row output lives in the workspace
        const ddm_status st = ensure_workspace(p);
        if (st != DDM_OK) return st;
    }
    return launch_spatial(p, frames, reinterpret_cast<float2*>(spectrum), (cudaStream_t)stream);
}

ddm_status ddm_temporal_sf(ddm_plan p, const float* spectrum, float* D, void* stream) {
    if (!check_plan(p) || !spectrum || !D) return DDM_ERR_INVALID_ARG;
    if (p->d.precision == DDM_PREC_FP64) return DDM_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(spectrum) & 7) != 0 || (reinterpret_cast<uintptr_t>(D) & 3) != 0)
        return DDM_ERR_INVALID_ARG;
    if (p->blocked) {                      // the blocked copy lives in the workspace
        const ddm_status st = ensure_workspace(p);
        if (st != DDM_OK) return st;
    }
    return launch_temporal(p, reinterpret_cast<const float2*>(spectrum), D, (cudaStream_t)stream);
}

ddm_status ddm_structure_function(ddm_plan p, const void* frames, float* D, void* stream) {
    if (!check_plan(p) || !frames || !D) return DDM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(D) & 3) != 0) return DDM_ERR_INVALID_ARG;
    ddm_status st = ensure_workspace(p);
    if (st != DDM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool stats = p->stats_ev[0] != nullptr;
    p->stats_recorded = false;   // until this call's three events are on the stream
    if (stats && cudaEventRecord(p->stats_ev[0], s) != cudaSuccess) return DDM_ERR_CUDA;
    if (p->d.precision == DDM_PREC_FP64) {
        // one launch sequence: step one and step two are not separated in the stats
        st = launch_fp64(p, frames, p->workspace, D, s);
        if (st == DDM_OK && stats)
            st = (cudaEventRecord(p->stats_ev[1], s) == cudaSuccess &&
                  cudaEventRecord(p->stats_ev[2], s) == cudaSuccess) ? DDM_OK : DDM_ERR_CUDA;
        p->stats_recorded = stats && st == DDM_OK;
        return st;
    }
    float2* spec = reinterpret_cast<float2*>(p->workspace);
    // plans whose long time kernels read a blocked copy: step one's column pass writes it
    // directly (no corner-turn pass); the last block's entries past q1 are zeroed for the
    // tiles that read them
    float2* blk = nullptr;
    if (p->blocked) {
        blk = reinterpret_cast<float2*>(static_cast<char*>(p->workspace) + p->blk_offset);
        const int64_t n = p->q1 - p->q0, nb = (n + 15) / 16;
        if (n % 16 != 0 &&
            cudaMemsetAsync(blk + (size_t)(nb - 1) * p->d.N * 16, 0, sizeof(float2) * (size_t)p->d.N * 16, s) !=
                cudaSuccess)
            return DDM_ERR_CUDA;
    }
    bool wrote_blocked = false;
    st = launch_spatial(p, frames, spec, s, blk, &wrote_blocked);
    if (st != DDM_OK) return st;
    if (stats && cudaEventRecord(p->stats_ev[1], s) != cudaSuccess) return DDM_ERR_CUDA;
    st = launch_temporal(p, spec, D, s, wrote_blocked);
    if (st == DDM_OK && stats && cudaEventRecord(p->stats_ev[2], s) != cudaSuccess) return DDM_ERR_CUDA;
    p->stats_recorded = stats && st == DDM_OK;
    return st;
}

ddm_status ddm_azimuthal_average(ddm_plan p, const float* D, float* Dr, int* counts,
                                 void* stream) {
    if (!check_plan(p) || !D || !Dr) return DDM_ERR_INVALID_ARG;
    if (p->d.n_bins <= 0) return DDM_ERR_INVALID_ARG;
    return launch_radial(p, D, Dr, counts, true, (cudaStream_t)stream);
}

ddm_status ddm_azimuthal_sums(ddm_plan p, const float* D, float* sums, int* counts, void* stream) {
    if (!check_plan(p) || !D || !sums || !counts) return DDM_ERR_INVALID_ARG;
    if (p->d.n_bins <= 0) return DDM_ERR_INVALID_ARG;
    return launch_radial(p, D, sums, counts, false, (cudaStream_t)stream);
}

}  // extern "C"
