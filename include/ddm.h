/*
 * ddm.h -- C ABI of the B300 (sm_103a) DDM structure-function library.
 *
 * Computes the image structure function of Differential Dynamic Microscopy,
 *
 *     D(q, m) = 1/(N - m) * sum_{t=0}^{N-1-m} |F(q, t+m) - F(q, t)|^2 ,   m = 0 .. N-1,
 *
 * (Eq. 1 of Norouzisadeh, Cerchiari, Croccolo, arXiv 2012.05695, read with the lag index
 * on both frames), where F(q, t) is the unnormalised 2D DFT of frame t (Sec. 2).  The lags
 * are obtained as in the paper's WITH_FT scheme (Sec. 2, App. B): per wave vector, the
 * power terms come from running sums of |F|^2 (Eqs. B1, B3) and the cross term from the
 * autocorrelation obtained by zero-padding the time sequence to N_2 = 2^(ceil(log2 N) + 1)
 * points (Eq. B4), a transform in time, the squared modulus and an inverse transform.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Frames are row-major [N][H][W] (uint16 or float32).  Wave vectors are stored on the
 *    real-to-complex half plane: q = ky * (W/2 + 1) + kx with ky = 0..H-1 (DFT order,
 *    ky >= H/2 means negative) and kx = 0..W/2; n_q = H * (W/2 + 1).  D(-q) = D(q).
 *  * D is float32 [n_q][N] (lag contiguous), D[q][0] = 0 exactly.
 *  * All array pointers are DEVICE pointers owned by the caller unless stated otherwise;
 *    `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  * Calls are asynchronous on `stream`.  Argument errors are returned synchronously and
 *    nothing is enqueued.  Errors found by a kernel (a non-finite intermediate) are
 *    recorded in a plan status word readable with ddm_plan_last_device_status() after the
 *    stream has been synchronised.  No C++ exception crosses this boundary.
 *  * A plan may be used from one host thread at a time; different plans are independent.
 */
#ifndef DDM_B300_H
#define DDM_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDM_ABI_VERSION 5

typedef enum ddm_status {
    DDM_OK = 0,
    DDM_ERR_INVALID_ARG = 1,   /* bad pointer, size or descriptor field */
    DDM_ERR_UNSUPPORTED = 2,   /* legal request this library does not implement */
    DDM_ERR_OOM = 3,           /* device allocation failed or exceeds max_workspace_bytes */
    DDM_ERR_CUDA = 4,          /* a CUDA runtime call failed (no device, launch error) */
    DDM_ERR_TIMEOUT = 5,       /* a bounded device wait (tile copy) gave up */
    DDM_ERR_NUMERIC = 6,       /* a kernel met a non-finite value */
    DDM_ERR_NO_WORKSPACE = 7   /* reserved */
} ddm_status;

typedef enum ddm_dtype { DDM_IN_U16 = 0, DDM_IN_F32 = 1 } ddm_dtype;

/* Arithmetic of the structure-function path. */
typedef enum ddm_precision {
    DDM_PREC_FP32 = 0,   /* FP32 transforms, prefix and suffix sums and combination */
    DDM_PREC_FP32_FP64FIX = 1, /* as FP32, plus: lags 1..fix_lags recomputed by direct
                                 differences (Eq. 1), FP32 over each thread's 32 frames and
                                 FP64 across threads: no cancellation against the power
                                 sums.  Implemented for 257 <= N <= 8192, fix_lags <= 8 */
    DDM_PREC_FP64 = 2,   /* everything in FP64 on the GPU (the precision sweep's reference
                            tier; D is still written as float32): spatial and time
                            transforms, power sums and combination.  About 1/64 of the
                            FP32 rate.  Implemented for power-of-two sides, N <= 4096, kmax = 0,
                            the whole wave-vector range, ddm_structure_function only
                            (ddm_spatial_fft / ddm_temporal_sf / the static entry return
                            DDM_ERR_UNSUPPORTED: the spectrum workspace is complex128) */
    DDM_PREC_TC_TF32X3 = 3 /* as DDM_PREC_FP32, but step one's column transform runs on the
                              tensor cores as DFT-as-GEMM (512 = 16 x 32: two GEMM stages of
                              tcgen05.mma kind::tf32, every operand split into two TF32 terms,
                              three products per term pair, FP32 accumulation).  Implemented
                              for H = 512 and power-of-two W of 32 .. 1024, whole plane, two-
                              pass step one (DDM_ERR_UNSUPPORTED otherwise) */
} ddm_precision;

/* Kernels of step one.  Both give the same spectrum (to FP32 rounding). */
typedef enum ddm_spatial_path {
    DDM_SPATIAL_TWO_PASS = 0,  /* row pass (rows staged by bulk copies) then column pass;
                                  the spectrum makes one extra round trip through HBM */
    DDM_SPATIAL_FUSED = 1      /* square frames 64..512: one frame per thread-block cluster,
                                  rows exchanged through distributed shared memory; other
                                  shapes fall back to the two-pass kernels */
} ddm_spatial_path;

typedef struct ddm_plan_desc {
    int H, W;          /* frame height and width in pixels, even: powers of two 2..2048
                          by radix-2 register FFTs; the sides 384, 480, 540, 600, 640,
                          720, 768, 800, 900, 960, 1000, 1080, 1200, 1280, 1440, 1536,
                          1600, 1920, 2000 by two-pass
                          mixed-radix (2, 3, 5) transforms; other even sides (6 .. 1022)
                          by Bluestein's chirp-z transform (a cyclic convolution of length
                          max(32, 2^ceil(log2(2n - 1))) <= 2048); odd sides
                          DDM_ERR_INVALID_ARG, other sides above 1024
                          DDM_ERR_UNSUPPORTED */
    int N;             /* number of frames, 1 .. 16384 */
    int dtype;         /* ddm_dtype */
    int precision;     /* ddm_precision */
    int M;             /* temporal pad length; 0 = N_2 of Eq. B4.  Any M >= 2N-1 gives
                          the same D (App. B); the library accepts 0 or N_2 and returns
                          DDM_ERR_INVALID_ARG for M < 2N-1, DDM_ERR_UNSUPPORTED otherwise */
    int n_bins;        /* radial bins for ddm_azimuthal_average (0 = no radial stage) */
    int subtract_ref;  /* 1: subtract frame 0 from every frame before the spatial
                          transform (exact in integers for uint16; D is unchanged by it) */
    int fix_lags;      /* DDM_PREC_FP32_FP64FIX: number of leading lags recomputed (0 = 8,
                          at most 8) */
    size_t max_workspace_bytes; /* 0 = no limit; else plan creation fails with
                                   DDM_ERR_OOM if the workspace would exceed it */
    int spatial_path;  /* ddm_spatial_path: which step-one kernels run */
    int64_t q_begin;   /* stored wave vectors [q_begin, q_end) (storage order of the
                          spectrum) that step two and the radial stage cover; 0, 0 = all.
                          Splits one stack across GPUs: every rank runs step one in full,
                          step two on its own range (D rows of other wave vectors are
                          left untouched), and ddm_azimuthal_sums() over its range; the
                          ranks' sums and counts add up to those of the whole plane.
                          q_begin must be a multiple of 64, q_begin < q_end <= n_q;
                          DDM_ERR_INVALID_ARG otherwise */
    int64_t q_end;
    int kmax;          /* low-frequency restriction (Sec. 3): 0 = every wave vector; else only
                          wave vectors with |ky'| <= kmax and 0 <= kx <= kmax (ky' the signed
                          row frequency) are kept, in a cropped spectrum store
                          [N][n_q], n_q = (2 kmax + 1)(kmax + 1), stored order
                          ky' = 0..kmax, -kmax..-1 (outer) by kx = 0..kmax (inner); D rows
                          follow the same order.  kmax must be odd and below H/2 and W/2
                          (DDM_ERR_INVALID_ARG otherwise); the library crops only frames
                          whose sides are powers of two (DDM_ERR_UNSUPPORTED otherwise).
                          The plan then also owns an
                          intermediate of N * H * (kmax + 1) complex64 for step one */
    int kx_begin;      /* kx-column range [kx_begin, kx_end) of one rank's share of a stack
                          split across GPUs by columns of the half plane (0, 0 = every
                          column).  Step one transforms every row (it needs all of them)
                          but only the range's columns; its spectrum store holds just the
                          range: [N][n_q], n_q = H (kx_end - kx_begin), stored [ky][kx -
                          kx_begin], followed -- for the range that starts at kx_begin = 0 --
                          by the H entries of the kx = W/2 column (n_q += H).  Step two, the
                          radial stage and D rows work on that store; D rows keep the
                          whole plane's public order q = ky (W/2 + 1) + kx, so every D
                          argument is [H (W/2 + 1)][N] (rows of other columns untouched),
                          and the ranks' D rows together are the whole plan's, bitwise.  kx_begin and kx_end multiples of 16,
                          0 <= kx_begin < kx_end <= W/2 (DDM_ERR_INVALID_ARG otherwise);
                          power-of-two sides 32 .. 1024, DDM_PREC_FP32 or _FP64FIX, no kmax,
                          no q_begin/q_end, two-pass step one (DDM_ERR_UNSUPPORTED
                          otherwise).  The workspace then also holds step one's row-pass
                          output for the whole plane (N H (W/2 + 1) complex64) */
    int kx_end;
} ddm_plan_desc;

typedef struct ddm_plan_s* ddm_plan;

/* Library version of this header's ABI. */
int ddm_abi_version(void);

/* sizeof(ddm_plan_desc) in this library: a binding checks its mirror of the struct against it. */
size_t ddm_plan_desc_size(void);

/* Static, never NULL. */
const char* ddm_status_string(ddm_status s);

/* Fill *desc with defaults for an H x W x N stack (uint16, FP32 tier, M = N_2,
 * n_bins = 0, subtract_ref = 1). */
ddm_status ddm_plan_desc_init(ddm_plan_desc* desc, int H, int W, int N);

/* Validate *desc and create a plan on the current CUDA device.  The plan owns host
 * metadata, small device tables (twiddles, radial bin map) and -- unless a workspace is
 * attached with ddm_plan_set_workspace() before the first call that needs it -- the
 * spectrum workspace.  *out is NULL on failure. */
ddm_status ddm_plan_create(ddm_plan* out, const ddm_plan_desc* desc);

/* Release everything the plan owns.  NULL is accepted.  The caller must make sure no
 * work enqueued with the plan is still running. */
ddm_status ddm_plan_destroy(ddm_plan p);

/* Bytes of device workspace ddm_structure_function needs: the spectrum store (n_q * N
 * complex64, complex128 for DDM_PREC_FP64, 256-byte aligned), plus, for time transforms of
 * L >= 2048 points on many wave vectors (n_q >= 200000, or >= 100000 at L = 16384) when
 * max_workspace_bytes leaves room, a blocked copy of the spectrum (16 wave vectors
 * contiguous over time) that the time kernels read.  ddm_temporal_sf uses the workspace
 * for that copy too (allocating it if none is attached). */
ddm_status ddm_plan_workspace_size(ddm_plan p, size_t* bytes);

/* Attach a caller-owned device workspace of at least ddm_plan_workspace_size() bytes,
 * 256-byte aligned.  Frees a workspace the plan allocated itself.  The caller keeps
 * ownership and must keep it alive while work is enqueued. */
ddm_status ddm_plan_set_workspace(ddm_plan p, void* dev_ptr, size_t bytes);

/* n_q = H * (W/2 + 1), the number of stored wave vectors ((2 kmax + 1)(kmax + 1) for a
 * plan with the low-frequency restriction). */
ddm_status ddm_plan_n_q(ddm_plan p, int64_t* n_q);

/* Kernel-detected status of the last completed calls on this plan (DDM_OK,
 * DDM_ERR_NUMERIC, or DDM_ERR_TIMEOUT if a tile copy did not complete within its bounded
 * wait); reading it resets it to DDM_OK.  Synchronise the stream first. */
ddm_status ddm_plan_last_device_status(ddm_plan p, ddm_status* out);

/* Per-stage timing (the paper's per-task time breakdown, Sec. 2): with stats enabled,
 * ddm_structure_function records CUDA events on its stream before step one, between the
 * steps and after step two; ddm_plan_stats waits for the last call's events and returns the
 * two stage times in milliseconds (the FP64 tier reports both steps as step one).
 * DDM_ERR_INVALID_ARG if no call has been recorded since stats were enabled. */
ddm_status ddm_plan_enable_stats(ddm_plan p, int on);
ddm_status ddm_plan_stats(ddm_plan p, float* step_one_ms, float* step_two_ms);

/* Test hook for the bounded device waits (no plan needed, current device, synchronous):
 * launches one CTA that arms a tile barrier for bytes no copy will deliver and waits on it
 * with the same bounded routine the time kernels use, and one CTA that holds tensor memory
 * and waits on an MMA barrier no commit will complete with the routine and give-up path of
 * the MLP's tensor-core forward (it then releases the tensor memory); each gives up after
 * cap_cycles SM clock cycles (clamped to 1e3 .. 4e9).  Returns DDM_ERR_TIMEOUT when both
 * bounds fired and were reported through status words (the expected outcome), DDM_OK if a
 * wait had completed (never, unless a bound is broken), DDM_ERR_CUDA on a launch or copy
 * failure. */
ddm_status ddm_selftest_bounded_wait(long long cap_cycles);

/* ---- the hot path ---------------------------------------------------------------- */

/* Step one of Sec. 2: the real-to-complex 2D DFT of every frame (after subtracting
 * frame 0 when desc.subtract_ref is set).
 *   frames   [N][H][W] uint16 or float32 (desc.dtype), device
 *   spectrum [N][n_q] complex64 (interleaved re, im), device, written
 * Unnormalised: F(ky, kx) = sum_{y,x} I(y, x) exp(-2 pi i (ky y / H + kx x / W)). */
ddm_status ddm_spatial_fft(ddm_plan p, const void* frames, float* spectrum, void* stream);

/* Step two of Sec. 2 with the App. B scheme, on a spectrum laid out as
 * ddm_spatial_fft writes it:
 *   spectrum [N][n_q] complex64, device, read only
 *   D        [n_q][N] float32, device, written
 * Per wave vector q: remove the time mean of F(q, .) (D is unchanged by any constant),
 * P1(m) = sum_{t < N-m} |F|^2 and P2(m) = sum_{t >= m} |F|^2 (Eqs. B1, B3), Re C(m) by the
 * zero-padded transform in time (Eq. B4), D = (P1 + P2 - 2 Re C) / (N - m).
 * Performance note: a power-of-two N >= 512 fills the transform length exactly and runs a
 * kernel instance with N fixed at compile time (the same D, 1-10 % faster). */
ddm_status ddm_temporal_sf(ddm_plan p, const float* spectrum, float* D, void* stream);

/* The paper's WITHOUT_FT scheme (Sec. 2; the comparison method of its Figs. 1 and 3) on
 * the GPU: D(q, m) = 1/(N - m) sum_{t < N-m} |F(q, t+m) - F(q, t)|^2 straight from Eq. 1,
 * by explicit differences of the stored spectra, O(N^2) per wave vector in FP32 (sums per
 * lag in time order).  Same input layout, output layout, wave-vector range (q_begin/q_end),
 * low-frequency store (kmax) and status reporting as ddm_temporal_sf, so the two schemes
 * can be timed against each other on one spectrum:
 *   spectrum [N][n_q] complex64, device, read only (as ddm_spatial_fft writes it)
 *   D        [n_q][N] float32, device, written (D[q][0] = 0)
 * DDM_ERR_UNSUPPORTED for DDM_PREC_FP64 plans (complex128 spectra). */
ddm_status ddm_temporal_sf_direct(ddm_plan p, const float* spectrum, float* D, void* stream);

/* Both steps: frames [N][H][W] -> D [n_q][N].  Uses the plan's workspace for the
 * spectrum (allocated on first use if none is attached). */
ddm_status ddm_structure_function(ddm_plan p, const void* frames, float* D, void* stream);

/* Radial (azimuthal) average over |q| bins -- not in the paper.
 *   D      [n_q][N] float32, device (as written above)
 *   Dr     [n_bins][N] float32, device, written: mean of D over the FULL-plane modes of
 *          each bin (half-plane modes with 0 < kx < W/2 count twice); 0 for empty bins.
 *          A plan restricted to a wave-vector range averages over that range only
 *   counts [n_bins] int32, device, written (may be NULL): full-plane modes per bin
 * Bins: |q| = 2 pi sqrt((ky'/H)^2 + (kx'/W)^2) rad/px (signed ky', kx'), n_bins uniform
 * bins over [0, pi sqrt 2], b = min(floor(|q| n_bins / (pi sqrt 2)), n_bins - 1), the floor
 * evaluated exactly in integers.  Summation order is fixed: results are bitwise
 * reproducible run to run.  Needs desc.n_bins > 0. */
ddm_status ddm_azimuthal_average(ddm_plan p, const float* D, float* Dr, int* counts,
                                 void* stream);

/* The radial stage before its division, for combining ranks that split a stack by
 * wave-vector range (ddm_plan_desc.q_begin/q_end):
 *   D      [n_q][N] float32, device (rows of the plan's range are read)
 *   sums   [n_bins][N] float32, device, written: sum over the plan's stored wave vectors in
 *          each bin of w_q D(q, m), w_q = 2 for 0 < kx < W/2, else 1
 *   counts [n_bins] int32, device, written: sum of w_q over the same wave vectors
 * Adding every rank's sums and counts and dividing (0 for empty bins) gives
 * ddm_azimuthal_average of the whole plane up to the order of the FP32 additions.  Same
 * fixed summation order per plan as ddm_azimuthal_average.  Needs desc.n_bins > 0. */
ddm_status ddm_azimuthal_sums(ddm_plan p, const float* D, float* sums, int* counts,
                              void* stream);

/* ---- fit of D(|q|, dt) (not in the paper: the analysis step that follows it) ---------- */

/* Model D(lag) = A (1 - exp(-(lag / tau)^beta)) + B, fitted per curve at the 64 log-spaced
 * lags lag_i = exp(i ln(N-1) / 63), i = 0..63 (curves sampled by linear interpolation
 * between neighbouring integer lags).  Needs N >= 2. */
#define DDM_FIT_LAGS 64
#define DDM_MLP_PARAMS 41860   /* 64 -> 128 -> 128 -> 128 -> 4, weights then bias per layer */

typedef enum ddm_fit_mode {
    DDM_FIT_LM = 0,        /* Levenberg-Marquardt from a heuristic seed */
    DDM_FIT_MLP = 1,       /* MLP prediction only */
    DDM_FIT_MLP_LM = 2     /* MLP seed; kept if its RMS residual / A <= 1e-2, else LM from
                              the lower-cost of the MLP and the heuristic seed (and from the
                              heuristic seed if LM from the MLP seed diverges) */
} ddm_fit_mode;

/* ddm_fit flags per curve */
#define DDM_FIT_CONVERGED 1
#define DDM_FIT_MAXITER 2
#define DDM_FIT_NONFINITE 4
#define DDM_FIT_MLP_ACCEPTED 8
#define DDM_FIT_FALLBACK 16
#define DDM_FIT_SEED_HEURISTIC 32   /* MLP_LM: LM started from the heuristic seed, whose cost
                                       was below the network's */

typedef struct ddm_mlp_s* ddm_mlp;

/* Features of curves for the MLP: the 64 log-lag samples divided by their plateau
 * p8 = mean of the last 8 samples (1 if p8 <= 0).
 *   Dr [n_curves][N] float32 device (e.g. ddm_azimuthal_average's output; N = plan's N)
 *   x  [n_curves][64] float32 device, written;  p8 [n_curves] float32 device, written */
ddm_status ddm_fit_features(ddm_plan p, const float* Dr, int n_curves, float* x, float* p8,
                            void* stream);

/* Fit every curve of Dr [n_curves][N].  mlp may be NULL for DDM_FIT_LM.
 *   params [n_curves][4] float32 (A, tau, beta, B);  cost [n_curves] float32 (sum of squared
 *   residuals at the 64 lags);  iters [n_curves] int32 (LM iterations, 0 if none);
 *   flags [n_curves] int32 (DDM_FIT_*).  cost, iters, flags may be NULL.
 * LM (FP32, one warp per curve): p = (A, B, ln tau, beta) on the curve divided by p8,
 * analytic Jacobian, damping (J^T J + lam diag J^T J) dp = -J^T r, lam from 1e-3, /10 on
 * an accepted step, x10 on a rejected one (stop above 1e12), beta clamped to [0.05, 3],
 * stop when a step accepted at its first trial lowers the cost by less than 1e-6 of it,
 * at most 100 iterations.  Scratch (features, MLP outputs) is taken from the plan's workspace if it is
 * large enough, else allocated by the plan on first use (n_curves * 276 bytes). */
ddm_status ddm_fit(ddm_plan p, const float* Dr, int n_curves, int mode, ddm_mlp mlp,
                   float* params, float* cost, int* iters, int* flags, void* stream);

/* MLP 64 -> 128 -> 128 -> 128 -> 4 with GELU (erf form) on the hidden layers.  FP32 master
 * weights, Adam state and gradients on the device; the weight matrices are used rounded to
 * bfloat16, biases and accumulation in FP32.  Head: A = p8 exp(o0), tau = exp(o1),
 * beta = 0.3 + 0.9 sigmoid(o2), B = A o3.  max_batch bounds every batch passed later. */
ddm_status ddm_mlp_create(ddm_mlp* out, int max_batch);
ddm_status ddm_mlp_destroy(ddm_mlp m);
/* Host arrays of DDM_MLP_PARAMS floats; set resets the Adam state and step count. */
ddm_status ddm_mlp_set_weights(ddm_mlp m, const float* host_w);
ddm_status ddm_mlp_get_weights(ddm_mlp m, float* host_w);
/* Training checkpoint: a host array of DDM_MLP_STATE_FLOATS floats holding the FP32 master
 * weights, Adam's first and second moments (DDM_MLP_PARAMS each, in that order) and the
 * Adam step count (an integer stored as a float, 0 .. 2^24).  get synchronises the device;
 * set restores all of it, so training resumed from a checkpoint takes exactly the steps
 * the uninterrupted run would have taken. */
#define DDM_MLP_STATE_FLOATS (3 * DDM_MLP_PARAMS + 1)
ddm_status ddm_mlp_get_state(ddm_mlp m, float* host_state);
ddm_status ddm_mlp_set_state(ddm_mlp m, const float* host_state);
/* x [B][64] device -> o [B][4] device (raw outputs, before the head); any alignment.  The
 * hidden layers run on the tensor cores (tcgen05.mma, bf16 operands, FP32 accumulation in
 * tensor memory), one CTA per 128 samples; each FP32 activation enters as three bf16 terms
 * that sum to it exactly, so the result is the FP32-activation network's up to FP32 rounding.  The MMA
 * waits are bounded (about 2 s); one that gives up leaves o unwritten for that CTA's samples
 * and is reported by ddm_mlp_last_device_status(). */
ddm_status ddm_mlp_forward(ddm_mlp m, const float* x, int B, float* o, void* stream);
/* DDM_ERR_TIMEOUT in *out if a bounded wait of a forward pass gave up since the last call,
 * else DDM_OK; synchronises the device and clears the word. */
ddm_status ddm_mlp_last_device_status(ddm_mlp m, ddm_status* out);
/* Loss = mean over the batch of (o0 - t0)^2 + (o1 - t1)^2 + (beta - t2)^2 + (o3 - t3)^2,
 * t [B][4] device targets (ln(A/p8), ln tau, beta, B/A).  grad [DDM_MLP_PARAMS] device and
 * loss [1] device are written (loss may be NULL).  Summation order is fixed. */
ddm_status ddm_mlp_grad(ddm_mlp m, const float* x, const float* t, int B, float* grad,
                        float* loss, void* stream);
/* ddm_mlp_grad followed by one Adam step (b1 0.9, b2 0.999, eps 1e-8) at rate lr. */
ddm_status ddm_mlp_train_step(ddm_mlp m, const float* x, const float* t, int B, float lr,
                              float* loss, void* stream);

/* ---- allocation-free variant (the paper has no counterpart) -------------------------- */

/* Size of the library's own device scratch used by ddm_structure_function_static:
 * 64 MiB, held on every GPU that loads this library until the process exits. */
#define DDM_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* Same result as ddm_structure_function, for callers that must not allocate device
 * memory when they ask for D -- a host whose own pool allocator already owns the device
 * memory, or a no-allocation hot loop.  The plan is created beforehand (plan creation
 * does allocate its small tables); this call allocates nothing, needs no workspace and
 * keeps the spectrum in the library's fixed device scratch instead.
 *   frames [N][H][W] uint16 or float32 (desc.dtype), device;  D [n_q][N] float32, device.
 * Limits and behaviour:
 *   - the spectrum, n_q * N * 8 bytes, must fit DDM_STATIC_SCRATCH_BYTES, else
 *     DDM_ERR_UNSUPPORTED is returned and nothing is enqueued;
 *   - the plan's device must be the current device, else DDM_ERR_INVALID_ARG;
 *   - the first call in a CUDA context (on each device, and again after that device has
 *     been reset) looks up the scratch's device address in that context and caches it;
 *     make that first call before capturing any stream;
 *   - with stats enabled (ddm_plan_enable_stats), ddm_plan_stats reports this call's two
 *     step times, as it does for ddm_structure_function;
 *   - all calls share the one scratch: calls whose work overlaps on the GPU (different
 *     streams, no ordering between them) race and give wrong results; calls ordered on
 *     one stream are safe.  Nothing in the scratch needs to start at zero. */
ddm_status ddm_structure_function_static(ddm_plan p, const void* frames, float* D, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DDM_B300_H */
