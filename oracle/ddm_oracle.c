/*
 * FP64 CPU oracle for the DDM image structure function (Norouzisadeh, Cerchiari,
 * Croccolo, "Increased performance in DDM analysis by calculating structure functions
 * through Fourier transform in time", arXiv 2012.05695).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or includes
 * this file; it shares no code, header, table or constant with the CUDA path.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Everything is plain, slow and in double precision:
 *   ddmo_dft2            naive separable 2D DFT of every frame (the F_xy of Eq. 1),
 *                        unnormalised (the FFT-library convention the paper used, Sec. 2)
 *   ddmo_sf_direct       Eq. 1 read as d(m) = 1/(N-m) sum_{n=m}^{N-1} |F(I_n) - F(I_{n-m})|^2,
 *                        computed by differences of the stored transforms (the paper's
 *                        WITHOUT_FT scheme, Sec. 2), d(0) = 0
 *   ddmo_sf_wk           the paper's WITH_FT route (App. B): zero-pad to M, DFT in time,
 *                        squared modulus, inverse DFT, ramp 1/(N-m) for d_c, recursion
 *                        Eq. B3 for d_a, d = d_a - d_c.  Naive DFTs, no FFT.  Self-check only.
 *   ddmo_radial_bins     |q| bin of every DFT index (radial average, a build decision)
 *   ddmo_radial_average  mean of D over the full-plane modes of each bin
 *
 * Conventions: q = (ky, kx) row-major, ky = 0..H-1, kx = 0..W-1 in DFT order; a
 * "time sequence" (Sec. 2) is F(q, t) for t = 0..N-1.  F arrays are [N][H][n_kx]
 * (frame-major), D arrays are [nq][N] (lag contiguous).
 *
 * Parity pins live in tests/test_oracle_*.py (Parseval, Hermitian symmetry, closed forms,
 * brute force by differencing images first, D-level Parseval in exact integers, ...).
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DDMO_OK 0
#define DDMO_EINVAL 1
#define DDMO_ENOMEM 2

static const double TWO_PI = 6.283185307179586476925286766559;

/* cos/sin of 2*pi*j/L for j = 0..L-1; the exponent index is reduced modulo L in
 * integers before the lookup, so no large angle ever reaches cos/sin. */
static int make_twiddles(int L, double** c, double** s) {
    *c = (double*)malloc(sizeof(double) * (size_t)L);
    *s = (double*)malloc(sizeof(double) * (size_t)L);
    if (!*c || !*s) { free(*c); free(*s); return DDMO_ENOMEM; }
    for (int j = 0; j < L; ++j) {
        double a = TWO_PI * (double)j / (double)L;
        (*c)[j] = cos(a);
        (*s)[j] = sin(a);
    }
    return DDMO_OK;
}

static double load_pixel(const void* frames, int dtype, size_t i) {
    switch (dtype) {
        case 0: return (double)((const uint16_t*)frames)[i];
        case 1: return (double)((const float*)frames)[i];
        default: return ((const double*)frames)[i];
    }
}

static int clamp_threads(int nthreads) {
    if (nthreads < 1) return 1;
    if (nthreads > 256) return 256;
    return nthreads;
}

/* ------------------------------------------------------------------------------------ */
/* 2D DFT: F(ky,kx,t) = sum_y e^{-2 pi i ky y / H} sum_x e^{-2 pi i kx x / W} I_t(y,x)    */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    const void* frames; int dtype; int N, H, W;
    const int* kx; int n_kx;
    const double *cw, *sw, *ch, *sh;
    double *F_re, *F_im;
    int t_begin, t_end;
} dft2_job;

static void* dft2_worker(void* arg) {
    dft2_job* j = (dft2_job*)arg;
    const int H = j->H, W = j->W, K = j->n_kx;
    double* r_re = (double*)malloc(sizeof(double) * (size_t)H * K);
    double* r_im = (double*)malloc(sizeof(double) * (size_t)H * K);
    if (!r_re || !r_im) { free(r_re); free(r_im); return (void*)1; }
    for (int t = j->t_begin; t < j->t_end; ++t) {
        const size_t base = (size_t)t * H * W;
        /* transform along x for the requested kx only */
        for (int y = 0; y < H; ++y) {
            for (int c = 0; c < K; ++c) {
                const int kx = j->kx[c];
                double acc_re = 0.0, acc_im = 0.0;
                for (int x = 0; x < W; ++x) {
                    const double v = load_pixel(j->frames, j->dtype, base + (size_t)y * W + x);
                    const int e = (int)(((int64_t)kx * x) % W);
                    acc_re += v * j->cw[e];
                    acc_im -= v * j->sw[e];
                }
                r_re[(size_t)y * K + c] = acc_re;
                r_im[(size_t)y * K + c] = acc_im;
            }
        }
        /* transform along y for every ky */
        for (int ky = 0; ky < H; ++ky) {
            for (int c = 0; c < K; ++c) {
                double acc_re = 0.0, acc_im = 0.0;
                for (int y = 0; y < H; ++y) {
                    const int e = (int)(((int64_t)ky * y) % H);
                    const double a = r_re[(size_t)y * K + c], b = r_im[(size_t)y * K + c];
                    /* (a + ib)(cos - i sin) */
                    acc_re += a * j->ch[e] + b * j->sh[e];
                    acc_im += b * j->ch[e] - a * j->sh[e];
                }
                const size_t o = ((size_t)t * H + ky) * K + c;
                j->F_re[o] = acc_re;
                j->F_im[o] = acc_im;
            }
        }
    }
    free(r_re); free(r_im);
    return NULL;
}

int ddmo_dft2(const void* frames, int dtype, int N, int H, int W,
              const int* kx_sel, int n_kx, double* F_re, double* F_im, int nthreads) {
    if (!frames || !F_re || !F_im || N < 1 || H < 1 || W < 1 || dtype < 0 || dtype > 2)
        return DDMO_EINVAL;
    int* all = NULL;
    if (!kx_sel) {
        all = (int*)malloc(sizeof(int) * (size_t)W);
        if (!all) return DDMO_ENOMEM;
        for (int i = 0; i < W; ++i) all[i] = i;
        kx_sel = all; n_kx = W;
    }
    for (int i = 0; i < n_kx; ++i)
        if (kx_sel[i] < 0 || kx_sel[i] >= W) { free(all); return DDMO_EINVAL; }
    double *cw, *sw, *ch, *sh;
    if (make_twiddles(W, &cw, &sw)) { free(all); return DDMO_ENOMEM; }
    if (make_twiddles(H, &ch, &sh)) { free(all); free(cw); free(sw); return DDMO_ENOMEM; }
    nthreads = clamp_threads(nthreads);
    if (nthreads > N) nthreads = N;
    pthread_t th[256];
    dft2_job jobs[256];
    int rc = DDMO_OK;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = (dft2_job){frames, dtype, N, H, W, kx_sel, n_kx, cw, sw, ch, sh, F_re, F_im,
                             (int)((int64_t)N * i / nthreads), (int)((int64_t)N * (i + 1) / nthreads)};
        pthread_create(&th[i], NULL, dft2_worker, &jobs[i]);
    }
    for (int i = 0; i < nthreads; ++i) {
        void* ret = NULL;
        pthread_join(th[i], &ret);
        if (ret) rc = DDMO_ENOMEM;
    }
    free(all); free(cw); free(sw); free(ch); free(sh);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Eq. 1, direct differences: D(q,m) = 1/(N-m) sum_{t=0}^{N-1-m} |F(q,t+m) - F(q,t)|^2   */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    const double *F_re, *F_im; int N; long nq; double* D; long q_begin, q_end; int M;
} sf_job;

static void* sf_direct_worker(void* arg) {
    sf_job* j = (sf_job*)arg;
    const int N = j->N;
    const long nq = j->nq;
    for (long q = j->q_begin; q < j->q_end; ++q) {
        double* d = j->D + (size_t)q * N;
        d[0] = 0.0;
        for (int m = 1; m < N; ++m) {
            double acc = 0.0;
            for (int t = 0; t + m < N; ++t) {
                const double dr = j->F_re[(size_t)(t + m) * nq + q] - j->F_re[(size_t)t * nq + q];
                const double di = j->F_im[(size_t)(t + m) * nq + q] - j->F_im[(size_t)t * nq + q];
                acc += dr * dr + di * di;
            }
            d[m] = acc / (double)(N - m);
        }
    }
    return NULL;
}

/* ------------------------------------------------------------------------------------ */
/* App. B route: d = d_a - d_c.                                                           */
/*   d_c(m) = 2 Re c(m) / (N-m),  c = IDFT_M(|DFT_M(x zero-padded to M)|^2), first N lags */
/*   d_a by the recursion Eq. B3:                                                         */
/*   d_a(N-n-1) = n/(n+1) d_a(N-n) + (|x_n|^2 + |x_{N-n-1}|^2)/(n+1),  n = 0..N-1          */
/* ------------------------------------------------------------------------------------ */
static void* sf_wk_worker(void* arg) {
    sf_job* j = (sf_job*)arg;
    const int N = j->N, M = j->M;
    const long nq = j->nq;
    double *cm, *sm;
    if (make_twiddles(M, &cm, &sm)) return (void*)1;
    double* x_re = (double*)malloc(sizeof(double) * (size_t)M);
    double* x_im = (double*)malloc(sizeof(double) * (size_t)M);
    double* P = (double*)malloc(sizeof(double) * (size_t)M);
    double* da = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    if (!x_re || !x_im || !P || !da) {
        free(cm); free(sm); free(x_re); free(x_im); free(P); free(da);
        return (void*)1;
    }
    for (long q = j->q_begin; q < j->q_end; ++q) {
        /* time sequence of wave vector q, zero-padded to M support points */
        for (int t = 0; t < M; ++t) {
            x_re[t] = (t < N) ? j->F_re[(size_t)t * nq + q] : 0.0;
            x_im[t] = (t < N) ? j->F_im[(size_t)t * nq + q] : 0.0;
        }
        /* power spectrum of the padded sequence */
        for (int k = 0; k < M; ++k) {
            double ar = 0.0, ai = 0.0;
            for (int t = 0; t < M; ++t) {
                const int e = (int)(((int64_t)k * t) % M);
                ar += x_re[t] * cm[e] + x_im[t] * sm[e];
                ai += x_im[t] * cm[e] - x_re[t] * sm[e];
            }
            P[k] = ar * ar + ai * ai;
        }
        /* d_a by the recursion Eq. B3; the n = 0 step multiplies d_a(N) by zero */
        da[N] = 0.0;
        for (int n = 0; n < N; ++n) {
            const double pn = x_re[n] * x_re[n] + x_im[n] * x_im[n];
            const double pr = x_re[N - n - 1] * x_re[N - n - 1] + x_im[N - n - 1] * x_im[N - n - 1];
            da[N - n - 1] = ((double)n / (double)(n + 1)) * da[N - n] + (pn + pr) / (double)(n + 1);
        }
        double* d = j->D + (size_t)q * N;
        for (int m = 0; m < N; ++m) {
            /* real part of the inverse transform (1/M) sum_k P(k) e^{+2 pi i k m / M} */
            double cr = 0.0;
            for (int k = 0; k < M; ++k) {
                const int e = (int)(((int64_t)k * m) % M);
                cr += P[k] * cm[e];
            }
            cr /= (double)M;
            const double dc = 2.0 * cr / (double)(N - m);
            d[m] = da[m] - dc;
        }
    }
    free(cm); free(sm); free(x_re); free(x_im); free(P); free(da);
    return NULL;
}

static int run_sf(void* (*fn)(void*), const double* F_re, const double* F_im, int N, long nq,
                  int M, double* D, int nthreads) {
    nthreads = clamp_threads(nthreads);
    if (nthreads > nq) nthreads = (int)nq;
    if (nthreads < 1) return DDMO_OK;
    pthread_t th[256];
    sf_job jobs[256];
    int rc = DDMO_OK;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = (sf_job){F_re, F_im, N, nq, D, nq * i / nthreads, nq * (i + 1) / nthreads, M};
        pthread_create(&th[i], NULL, fn, &jobs[i]);
    }
    for (int i = 0; i < nthreads; ++i) {
        void* ret = NULL;
        pthread_join(th[i], &ret);
        if (ret) rc = DDMO_ENOMEM;
    }
    return rc;
}

int ddmo_sf_direct(const double* F_re, const double* F_im, int N, long nq, double* D, int nthreads) {
    if (!F_re || !F_im || !D || N < 1 || nq < 0) return DDMO_EINVAL;
    return run_sf(sf_direct_worker, F_re, F_im, N, nq, 0, D, nthreads);
}

int ddmo_sf_wk(const double* F_re, const double* F_im, int N, long nq, int M, double* D, int nthreads) {
    if (!F_re || !F_im || !D || N < 1 || nq < 0 || M < N) return DDMO_EINVAL;
    return run_sf(sf_wk_worker, F_re, F_im, N, nq, M, D, nthreads);
}

/* ------------------------------------------------------------------------------------ */
/* Radial bins.  |q| = 2 pi sqrt((ky'/H)^2 + (kx'/W)^2) rad/px with signed ky', kx' in    */
/* (-L/2, L/2]; n_bins uniform bins over [0, q_c], q_c = pi sqrt(2) (Nyquist corner);     */
/* b = min(floor(|q| n_bins / q_c), n_bins - 1).                                          */
/* floor(|q| n_bins / q_c) = floor(n_bins sqrt(2 K) / (H W)), K = ky'^2 W^2 + kx'^2 H^2,  */
/* evaluated exactly in integers: the largest b with (b H W)^2 <= 2 n_bins^2 K.           */
/* ------------------------------------------------------------------------------------ */
static int signed_index(int k, int L) { return (k > L / 2) ? k - L : k; }

int ddmo_radial_bins(int H, int W, int n_bins, int* bin) {
    if (H < 1 || W < 1 || n_bins < 1 || !bin || H > 65536 || W > 65536) return DDMO_EINVAL;
    for (int ky = 0; ky < H; ++ky) {
        for (int kx = 0; kx < W; ++kx) {
            const __int128 ys = signed_index(ky, H), xs = signed_index(kx, W);
            const __int128 K = ys * ys * (__int128)W * W + xs * xs * (__int128)H * H;
            const __int128 rhs = (__int128)2 * n_bins * n_bins * K;
            const __int128 hw = (__int128)H * W;
            /* largest b >= 0 with (b*hw)^2 <= rhs, found by stepping from a float guess */
            long b = (long)floor(sqrt((double)rhs) / (double)hw);
            if (b < 0) b = 0;
            while (b > 0 && (__int128)b * b * hw * hw > rhs) --b;
            while ((__int128)(b + 1) * (b + 1) * hw * hw <= rhs) ++b;
            if (b > n_bins - 1) b = n_bins - 1;
            bin[(size_t)ky * W + kx] = (int)b;
        }
    }
    return DDMO_OK;
}

/* D: [H*W][N] full plane (q = ky*W + kx).  Dr: [n_bins][N] mean over the modes in each
 * bin (0 for an empty bin); counts: [n_bins] number of modes. */
int ddmo_radial_average(const double* D, int H, int W, int N, int n_bins, double* Dr, long* counts) {
    if (!D || !Dr || !counts || N < 1) return DDMO_EINVAL;
    int* bin = (int*)malloc(sizeof(int) * (size_t)H * W);
    if (!bin) return DDMO_ENOMEM;
    int rc = ddmo_radial_bins(H, W, n_bins, bin);
    if (rc) { free(bin); return rc; }
    memset(Dr, 0, sizeof(double) * (size_t)n_bins * N);
    memset(counts, 0, sizeof(long) * (size_t)n_bins);
    for (size_t q = 0; q < (size_t)H * W; ++q) {
        const int b = bin[q];
        counts[b] += 1;
        for (int m = 0; m < N; ++m) Dr[(size_t)b * N + m] += D[q * N + m];
    }
    for (int b = 0; b < n_bins; ++b)
        if (counts[b] > 0)
            for (int m = 0; m < N; ++m) Dr[(size_t)b * N + m] /= (double)counts[b];
    free(bin);
    return DDMO_OK;
}
