"""FP64 CPU oracle for the DDM structure function of arXiv 2012.05695.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product library never does, and the two
share no code.  The arithmetic lives in ``ddm_oracle.c`` (plain double precision C, built
with gcc by :func:`build`); this module only marshals numpy arrays.

What it computes (paper passages in brackets):

* :func:`dft2` -- the unnormalised 2D DFT F_xy of every frame [Eq. 1, Sec. 2], by a naive
  separable sum, optionally restricted to a few kx columns (all ky kept).
* :func:`sf_direct` -- Eq. 1 read as d(m) = 1/(N-m) sum_n |F(I_n) - F(I_{n-m})|^2 by
  differences of the stored transforms [Eq. 1, Sec. 2]; d(0) = 0.
* :func:`sf_wk` -- the paper's Fourier-transform-in-time route [App. B, Eqs. B1-B4] with
  naive DFTs, the recursion Eq. B3 for d_a and the reading d = d_a - d_c.  Used only to
  check the oracle against itself by a second route.
* :func:`radial_bins` / :func:`radial_average` -- mean of D over |q| bins (not in the paper;
  a uniform binning over [0, pi*sqrt(2)] rad/px).
* :func:`plateau_scale` -- s_q = 2 var_t F(q, .), the large-lag plateau of D used as the
  error scale: err = max |D - D_oracle| / s_q.
* :mod:`oracle.fit` -- FP64 model, Levenberg-Marquardt fit and MLP forward/backward/Adam.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_LIB_DIR, "libddm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ddm_oracle.c into oracle/_build/libddm_oracle.so (gcc, -O2, IEEE math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.ddmo_dft2.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ip, ctypes.c_int, dp, dp, ctypes.c_int]
        lib.ddmo_sf_direct.argtypes = [dp, dp, ctypes.c_int, ctypes.c_long, dp, ctypes.c_int]
        lib.ddmo_sf_wk.argtypes = [dp, dp, ctypes.c_int, ctypes.c_long, ctypes.c_int, dp,
                                   ctypes.c_int]
        lib.ddmo_radial_bins.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip]
        lib.ddmo_radial_average.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, dp, lp]
        for f in ("ddmo_dft2", "ddmo_sf_direct", "ddmo_sf_wk", "ddmo_radial_bins",
                  "ddmo_radial_average"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def _ptr(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def dft2(frames: np.ndarray, kx_sel=None, nthreads=None) -> np.ndarray:
    """Unnormalised 2D DFT of every frame.

    frames: [N, H, W] uint16 / float32 / float64.  kx_sel: optional list of kx columns
    (0 <= kx < W); all ky are always computed.  Returns complex128 [N, H, n_kx] with
    F[t, ky, j] = sum_{y,x} I_t(y, x) exp(-2 pi i (ky y / H + kx_sel[j] x / W)).
    """
    lib = _load()
    a = np.ascontiguousarray(frames)
    if a.ndim != 3:
        raise ValueError("frames must be [N, H, W]")
    code = {np.dtype(np.uint16): 0, np.dtype(np.float32): 1, np.dtype(np.float64): 2}.get(a.dtype)
    if code is None:
        a = a.astype(np.float64)
        code = 2
    N, H, W = a.shape
    if kx_sel is None:
        kx = None
        K = W
    else:
        kx = np.ascontiguousarray(np.asarray(kx_sel, dtype=np.int32))
        K = int(kx.size)
    re = np.empty((N, H, K), np.float64)
    im = np.empty((N, H, K), np.float64)
    rc = lib.ddmo_dft2(a.ctypes.data_as(ctypes.c_void_p), code, N, H, W,
                       None if kx is None else _ptr(kx, ctypes.c_int), K, _ptr(re), _ptr(im),
                       _threads(nthreads))
    _check(rc, "dft2")
    return re + 1j * im


def _split(F):
    F = np.asarray(F)
    if F.ndim < 2:
        raise ValueError("F must be [N, ...]")
    N = F.shape[0]
    flat = F.reshape(N, -1)
    re = np.ascontiguousarray(flat.real, dtype=np.float64)
    im = np.ascontiguousarray(flat.imag, dtype=np.float64)
    return N, flat.shape[1], re, im, F.shape[1:]


def sf_direct(F: np.ndarray, nthreads=None) -> np.ndarray:
    """Eq. 1 by differences: F [N, ...] complex -> D [..., N] float64, D[..., 0] = 0."""
    lib = _load()
    N, nq, re, im, qshape = _split(F)
    D = np.empty((nq, N), np.float64)
    _check(lib.ddmo_sf_direct(_ptr(re), _ptr(im), N, nq, _ptr(D), _threads(nthreads)), "sf_direct")
    return D.reshape(*qshape, N)


def sf_wk(F: np.ndarray, M: int | None = None, nthreads=None) -> np.ndarray:
    """App. B route (pad to M, DFT in time, |.|^2, inverse DFT, Eq. B3 recursion).

    M defaults to the paper's N_2 = 2^(ceil(log2 N) + 1) (Eq. B4).
    """
    lib = _load()
    N, nq, re, im, qshape = _split(F)
    if M is None:
        M = pad_length_paper(N)
    D = np.empty((nq, N), np.float64)
    _check(lib.ddmo_sf_wk(_ptr(re), _ptr(im), N, nq, int(M), _ptr(D), _threads(nthreads)), "sf_wk")
    return D.reshape(*qshape, N)


def pad_length_paper(N: int) -> int:
    """Eq. B4: log2 N_2 = ceil(log2 N) + 1."""
    c = 0
    while (1 << c) < N:
        c += 1
    return 1 << (c + 1)


def radial_bins(H: int, W: int, n_bins: int) -> np.ndarray:
    """int32 [H, W] bin of every DFT index (exact integer evaluation of the floor)."""
    lib = _load()
    b = np.empty((H, W), np.int32)
    _check(lib.ddmo_radial_bins(H, W, n_bins, _ptr(b, ctypes.c_int)), "radial_bins")
    return b


def radial_average(D_full: np.ndarray, n_bins: int):
    """D_full: [H, W, N] over the full plane -> (Dr [n_bins, N], counts [n_bins])."""
    lib = _load()
    H, W, N = D_full.shape
    d = np.ascontiguousarray(D_full, dtype=np.float64)
    Dr = np.empty((n_bins, N), np.float64)
    counts = np.empty((n_bins,), np.int64)
    _check(lib.ddmo_radial_average(_ptr(d), H, W, N, n_bins, _ptr(Dr),
                                   _ptr(counts, ctypes.c_long)), "radial_average")
    return Dr, counts


def plateau_scale(F: np.ndarray) -> np.ndarray:
    """s_q = 2 var_t F(q, .) = 2 <|F - <F>_t|^2>_t for F [N, ...]; returns [...]."""
    F = np.asarray(F, dtype=np.complex128)
    mu = F.mean(axis=0)
    return 2.0 * np.mean(np.abs(F - mu) ** 2, axis=0)


def half_plane_columns(W: int):
    """kx = 0 .. W//2, the columns a real-to-complex transform keeps."""
    return list(range(W // 2 + 1))


def structure_function(frames: np.ndarray, kx_sel=None, nthreads=None):
    """Oracle D for the given frames: returns (D [H, n_kx, N], s_q [H, n_kx]).

    kx_sel defaults to the half plane kx = 0..W/2 (D(-q) = D(q) for real frames).
    """
    N, H, W = frames.shape
    if kx_sel is None:
        kx_sel = half_plane_columns(W)
    F = dft2(frames, kx_sel, nthreads)
    D = sf_direct(F, nthreads)
    return D, plateau_scale(F)


TOLERANCE = 1e-4        # |D - D_oracle| relative to the wave vector's plateau
STATIC_REL = 1e-12      # s_q below this fraction of the largest plateau: a static mode
STATIC_BOUND = 1e-6     # a static mode must have |D| <= STATIC_BOUND * max s_q


def scaled_error(D_test, D_ref, s_q):
    """The precision metric: max over q, m of |D_test - D_ref| / s_q, with s_q = 2 var_t F(q)
    the large-lag plateau of each wave vector.

    Static modes -- s_q < STATIC_REL * max s_q, whose whole time variation is far below
    what FP32 arithmetic on the plane resolves (e.g. the DC mode of a field whose mean never
    changes, where only the input's own rounding moves) -- are judged on the global scale
    instead: they must have |D_test| <= STATIC_BOUND * max s_q.  Each of them enters the
    maximum as TOLERANCE * |D_test| / (STATIC_BOUND * max s_q), so that a result <= TOLERANCE
    means every mode passed its own rule.
    """
    s = np.asarray(s_q, dtype=np.float64)
    smax = float(np.max(s)) if s.size else 0.0
    Dt = np.asarray(D_test, np.float64)
    diff = np.abs(Dt - np.asarray(D_ref, np.float64))
    if diff.size == 0:
        return 0.0
    if smax <= 0.0:                        # every mode static at zero: compare absolutely
        return float(np.max(diff))
    static = s < STATIC_REL * smax
    scale = np.where(static, 1.0, s)
    err = diff / scale[..., None]
    if np.any(static):
        err_static = TOLERANCE * np.abs(Dt) / (STATIC_BOUND * smax)
        err = np.where(static[..., None], err_static, err)
    return float(np.max(err))
