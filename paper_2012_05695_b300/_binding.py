"""ctypes binding of the C ABI in include/ddm.h (argument marshalling only).

Every entry point keeps its C name.  Arrays are torch CUDA tensors (PyTorch provides the
device memory and streams); the binding checks shape, dtype, device and contiguity, passes
raw pointers, and turns a non-OK status into :class:`DDMError`.  There is no fallback: if
the shared library is missing this module raises on first use.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libddm_b300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ddm.h")

DDM_OK = 0
DDM_ERR_INVALID_ARG = 1
DDM_ERR_UNSUPPORTED = 2
DDM_ERR_OOM = 3
DDM_ERR_CUDA = 4
DDM_ERR_TIMEOUT = 5
DDM_ERR_NUMERIC = 6
DDM_ERR_NO_WORKSPACE = 7

DDM_IN_U16 = 0
DDM_IN_F32 = 1
DDM_PREC_FP32 = 0
DDM_PREC_FP32_FP64FIX = 1
DDM_PREC_FP64 = 2
DDM_PREC_TC_TF32X3 = 3

DDM_SPATIAL_TWO_PASS = 0
DDM_SPATIAL_FUSED = 1

DDM_FIT_LM = 0
DDM_FIT_MLP = 1
DDM_FIT_MLP_LM = 2
DDM_FIT_CONVERGED = 1
DDM_FIT_MAXITER = 2
DDM_FIT_NONFINITE = 4
DDM_FIT_MLP_ACCEPTED = 8
DDM_FIT_FALLBACK = 16
DDM_FIT_SEED_HEURISTIC = 32
DDM_FIT_LAGS = 64
DDM_MLP_PARAMS = 41860
DDM_MLP_STATE_FLOATS = 3 * DDM_MLP_PARAMS + 1


class DDMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class ddm_plan_desc(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int), ("W", ctypes.c_int), ("N", ctypes.c_int),
        ("dtype", ctypes.c_int), ("precision", ctypes.c_int), ("M", ctypes.c_int),
        ("n_bins", ctypes.c_int), ("subtract_ref", ctypes.c_int), ("fix_lags", ctypes.c_int),
        ("max_workspace_bytes", ctypes.c_size_t),
        ("spatial_path", ctypes.c_int),
        ("q_begin", ctypes.c_int64), ("q_end", ctypes.c_int64),
        ("kmax", ctypes.c_int),
        ("kx_begin", ctypes.c_int), ("kx_end", ctypes.c_int),
    ]


_lib = None


def lib():
    """Load libddm_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, c_int, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    sigs = {
        "ddm_abi_version": (c_int, []),
        "ddm_plan_desc_size": (ctypes.c_size_t, []),
        "ddm_status_string": (ctypes.c_char_p, [st]),
        "ddm_plan_desc_init": (st, [ctypes.POINTER(ddm_plan_desc), c_int, c_int, c_int]),
        "ddm_plan_create": (st, [ctypes.POINTER(vp), ctypes.POINTER(ddm_plan_desc)]),
        "ddm_plan_destroy": (st, [vp]),
        "ddm_plan_workspace_size": (st, [vp, ctypes.POINTER(ctypes.c_size_t)]),
        "ddm_plan_set_workspace": (st, [vp, vp, ctypes.c_size_t]),
        "ddm_plan_n_q": (st, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ddm_plan_last_device_status": (st, [vp, ctypes.POINTER(ctypes.c_int)]),
        "ddm_selftest_bounded_wait": (st, [ctypes.c_longlong]),
        "ddm_plan_enable_stats": (st, [vp, c_int]),
        "ddm_plan_stats": (st, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        "ddm_mlp_get_state": (st, [vp, vp]),
        "ddm_mlp_set_state": (st, [vp, vp]),
        "ddm_spatial_fft": (st, [vp, vp, vp, vp]),
        "ddm_temporal_sf": (st, [vp, vp, vp, vp]),
        "ddm_temporal_sf_direct": (st, [vp, vp, vp, vp]),
        "ddm_structure_function": (st, [vp, vp, vp, vp]),
        "ddm_azimuthal_average": (st, [vp, vp, vp, vp, vp]),
        "ddm_azimuthal_sums": (st, [vp, vp, vp, vp, vp]),
        "ddm_structure_function_static": (st, [vp, vp, vp, vp]),
        "ddm_fit_features": (st, [vp, vp, c_int, vp, vp, vp]),
        "ddm_fit": (st, [vp, vp, c_int, c_int, vp, vp, vp, vp, vp, vp]),
        "ddm_mlp_create": (st, [ctypes.POINTER(vp), c_int]),
        "ddm_mlp_destroy": (st, [vp]),
        "ddm_mlp_set_weights": (st, [vp, vp]),
        "ddm_mlp_get_weights": (st, [vp, vp]),
        "ddm_mlp_forward": (st, [vp, vp, c_int, vp, vp]),
        "ddm_mlp_last_device_status": (st, [vp, ctypes.POINTER(ctypes.c_int)]),
        "ddm_mlp_grad": (st, [vp, vp, vp, c_int, vp, vp, vp]),
        "ddm_mlp_train_step": (st, [vp, vp, vp, c_int, ctypes.c_float, vp, vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if L.ddm_plan_desc_size() != ctypes.sizeof(ddm_plan_desc):
        raise RuntimeError("ddm_plan_desc layout of the binding does not match the library")
    _lib = L
    return L


def header_functions(path: str = HEADER):
    """Names of the functions include/ddm.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ddm_[a-z0-9_]+)\s*\(", text)))


def status_string(s: int) -> str:
    try:
        return lib().ddm_status_string(int(s)).decode()
    except Exception:
        return "status %d" % int(s)


def selftest_bounded_wait(cap_cycles: int) -> int:
    """Run the library's bounded-wait test hook; returns the status (DDM_ERR_TIMEOUT
    expected)."""
    return int(lib().ddm_selftest_bounded_wait(int(cap_cycles)))


def _check(status: int, where: str):
    if status != DDM_OK:
        raise DDMError(status, where)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dev_ptr(t, what, dtype, numel):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{what} must hold {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def spectrum_index_map(H: int, W: int):
    """(ky, kx) of every stored spectrum slot of one frame, as lists.

    The first H * (W/2) slots are kx < W/2 in [ky][kx] order; the last H slots are the
    kx = W/2 column in ky order.
    """
    Wh = W // 2
    ky = [s // Wh for s in range(H * Wh)] + list(range(H))
    kx = [s % Wh for s in range(H * Wh)] + [Wh] * H
    return ky, kx


class Plan:
    """A ddm_plan with torch-tensor marshalling."""

    def __init__(self, H: int, W: int, N: int, dtype: str = "u16", n_bins: int = 0,
                 precision: int = DDM_PREC_FP32, subtract_ref: int = 1, M: int = 0,
                 fix_lags: int = 0, max_workspace_bytes: int = 0, spatial_path: int = 0,
                 q_begin: int = 0, q_end: int = 0, kmax: int = 0, kx_begin: int = 0, kx_end: int = 0):
        L = lib()
        d = ddm_plan_desc()
        _check(L.ddm_plan_desc_init(ctypes.byref(d), H, W, N), "ddm_plan_desc_init")
        d.dtype = {"u16": DDM_IN_U16, "f32": DDM_IN_F32}[dtype]
        d.n_bins = n_bins
        d.precision = precision
        d.subtract_ref = subtract_ref
        d.M = M
        d.fix_lags = fix_lags
        d.max_workspace_bytes = max_workspace_bytes
        d.spatial_path = spatial_path
        d.q_begin = q_begin
        d.q_end = q_end
        d.kmax = kmax
        d.kx_begin = kx_begin
        d.kx_end = kx_end
        self.desc = d
        self.H, self.W, self.N, self.n_bins = H, W, N, n_bins
        self.kmax = kmax
        self.kx_begin, self.kx_end = kx_begin, kx_end
        self.dtype = dtype
        h = ctypes.c_void_p()
        _check(L.ddm_plan_create(ctypes.byref(h), ctypes.byref(d)), "ddm_plan_create")
        self._h = h
        nq = ctypes.c_int64()
        _check(L.ddm_plan_n_q(h, ctypes.byref(nq)), "ddm_plan_n_q")
        self.n_q = int(nq.value)
        # rows of D: the stored wave vectors, except for a kx-column range, whose rows keep
        # the whole half plane's order (its D is the whole plane's size)
        self.d_rows = H * (W // 2 + 1) if kx_end > 0 else self.n_q

    @property
    def handle(self):
        return self._h

    def wave_vectors(self):
        """(ky, kx) of every stored wave vector, in the spectrum store's order, ky in 0..H-1
        (numpy int arrays of length n_q).  For the whole plane and the cropped store this is
        also the order of D's rows; a kx-column range writes D rows ky (W/2 + 1) + kx."""
        import numpy as np
        if self.kmax > 0:
            k = self.kmax
            r = np.arange(2 * k + 1)
            kys = np.where(r <= k, r, r - (2 * k + 1)) % self.H
            ky = np.repeat(kys, k + 1)
            kx = np.tile(np.arange(k + 1), 2 * k + 1)
            return ky, kx
        if self.kx_end > 0:
            nk = self.kx_end - self.kx_begin
            ky = np.repeat(np.arange(self.H), nk)
            kx = np.tile(np.arange(self.kx_begin, self.kx_end), self.H)
            if self.kx_begin == 0:
                ky = np.concatenate([ky, np.arange(self.H)])
                kx = np.concatenate([kx, np.full(self.H, self.W // 2)])
            return ky, kx
        q = np.arange(self.n_q)
        return q // (self.W // 2 + 1), q % (self.W // 2 + 1)

    def _frames(self, frames):
        import torch
        dt = torch.uint16 if self.dtype == "u16" else torch.float32
        return _dev_ptr(frames, "frames", dt, self.N * self.H * self.W)

    def workspace_size(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().ddm_plan_workspace_size(self._h, ctypes.byref(b)), "ddm_plan_workspace_size")
        return int(b.value)

    def set_workspace(self, ws):
        import torch
        if ws.dtype != torch.uint8 or not ws.is_cuda:
            raise TypeError("workspace must be a CUDA uint8 tensor")
        _check(lib().ddm_plan_set_workspace(self._h, ctypes.c_void_p(ws.data_ptr()), ws.numel()),
               "ddm_plan_set_workspace")
        self._ws = ws

    def spatial_fft(self, frames, spectrum, stream=None):
        import torch
        _check(lib().ddm_spatial_fft(self._h, self._frames(frames),
                                     _dev_ptr(spectrum, "spectrum", torch.float32, 2 * self.N * self.n_q),
                                     _stream_ptr(stream)), "ddm_spatial_fft")

    def temporal_sf(self, spectrum, D, stream=None):
        import torch
        _check(lib().ddm_temporal_sf(self._h,
                                     _dev_ptr(spectrum, "spectrum", torch.float32, 2 * self.N * self.n_q),
                                     _dev_ptr(D, "D", torch.float32, self.d_rows * self.N),
                                     _stream_ptr(stream)), "ddm_temporal_sf")

    def temporal_sf_direct(self, spectrum, D, stream=None):
        """The WITHOUT_FT scheme (explicit frame differences, O(N^2) per wave vector) on the
        same spectrum and output layout as temporal_sf."""
        import torch
        _check(lib().ddm_temporal_sf_direct(self._h,
                                            _dev_ptr(spectrum, "spectrum", torch.float32, 2 * self.N * self.n_q),
                                            _dev_ptr(D, "D", torch.float32, self.d_rows * self.N),
                                            _stream_ptr(stream)), "ddm_temporal_sf_direct")

    def structure_function(self, frames, D, stream=None):
        import torch
        _check(lib().ddm_structure_function(self._h, self._frames(frames),
                                            _dev_ptr(D, "D", torch.float32, self.d_rows * self.N),
                                            _stream_ptr(stream)), "ddm_structure_function")

    def azimuthal_average(self, D, Dr, counts=None, stream=None):
        import torch
        cp = ctypes.c_void_p(0) if counts is None else _dev_ptr(counts, "counts", torch.int32, self.n_bins)
        _check(lib().ddm_azimuthal_average(self._h, _dev_ptr(D, "D", torch.float32, self.d_rows * self.N),
                                           _dev_ptr(Dr, "Dr", torch.float32, self.n_bins * self.N),
                                           cp, _stream_ptr(stream)), "ddm_azimuthal_average")

    def azimuthal_sums(self, D, sums, counts, stream=None):
        import torch
        _check(lib().ddm_azimuthal_sums(self._h, _dev_ptr(D, "D", torch.float32, self.d_rows * self.N),
                                        _dev_ptr(sums, "sums", torch.float32, self.n_bins * self.N),
                                        _dev_ptr(counts, "counts", torch.int32, self.n_bins),
                                        _stream_ptr(stream)), "ddm_azimuthal_sums")

    def fit_features(self, Dr, n_curves, x, p8, stream=None):
        import torch
        _check(lib().ddm_fit_features(self._h, _dev_ptr(Dr, "Dr", torch.float32, n_curves * self.N),
                                      n_curves, _dev_ptr(x, "x", torch.float32, n_curves * DDM_FIT_LAGS),
                                      _dev_ptr(p8, "p8", torch.float32, n_curves),
                                      _stream_ptr(stream)), "ddm_fit_features")

    def fit(self, Dr, n_curves, mode, mlp, params, cost=None, iters=None, flags=None, stream=None):
        import torch

        def opt(t, what, dt):
            return ctypes.c_void_p(0) if t is None else _dev_ptr(t, what, dt, n_curves)
        _check(lib().ddm_fit(self._h, _dev_ptr(Dr, "Dr", torch.float32, n_curves * self.N), n_curves,
                             int(mode), None if mlp is None else mlp.handle,
                             _dev_ptr(params, "params", torch.float32, 4 * n_curves),
                             opt(cost, "cost", torch.float32), opt(iters, "iters", torch.int32),
                             opt(flags, "flags", torch.int32), _stream_ptr(stream)), "ddm_fit")

    def enable_stats(self, on: bool = True):
        _check(lib().ddm_plan_enable_stats(self._h, 1 if on else 0), "ddm_plan_enable_stats")

    def stats(self):
        """(step one ms, step two ms) of the last structure_function call."""
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(lib().ddm_plan_stats(self._h, ctypes.byref(a), ctypes.byref(b)), "ddm_plan_stats")
        return a.value, b.value

    def last_device_status(self) -> int:
        s = ctypes.c_int()
        _check(lib().ddm_plan_last_device_status(self._h, ctypes.byref(s)), "ddm_plan_last_device_status")
        return int(s.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ddm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class MLP:
    """ddm_mlp: the fit seed network (device weights, Adam state)."""

    def __init__(self, max_batch: int = 4096):
        h = ctypes.c_void_p()
        _check(lib().ddm_mlp_create(ctypes.byref(h), int(max_batch)), "ddm_mlp_create")
        self._h = h
        self.max_batch = int(max_batch)

    @property
    def handle(self):
        return self._h

    def set_weights(self, w):
        import numpy as np
        a = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        if a.size != DDM_MLP_PARAMS:
            raise ValueError("weights must hold %d floats" % DDM_MLP_PARAMS)
        _check(lib().ddm_mlp_set_weights(self._h, a.ctypes.data_as(ctypes.c_void_p)), "ddm_mlp_set_weights")

    def get_weights(self):
        import numpy as np
        a = np.empty(DDM_MLP_PARAMS, np.float32)
        _check(lib().ddm_mlp_get_weights(self._h, a.ctypes.data_as(ctypes.c_void_p)), "ddm_mlp_get_weights")
        return a

    def get_state(self):
        """Training checkpoint: weights, Adam moments and step count (host float32 array)."""
        import numpy as np
        a = np.empty(DDM_MLP_STATE_FLOATS, np.float32)
        _check(lib().ddm_mlp_get_state(self._h, a.ctypes.data_as(ctypes.c_void_p)), "ddm_mlp_get_state")
        return a

    def set_state(self, state):
        import numpy as np
        a = np.ascontiguousarray(np.asarray(state, dtype=np.float32))
        if a.size != DDM_MLP_STATE_FLOATS:
            raise ValueError("state must hold %d floats" % DDM_MLP_STATE_FLOATS)
        _check(lib().ddm_mlp_set_state(self._h, a.ctypes.data_as(ctypes.c_void_p)), "ddm_mlp_set_state")

    def forward(self, x, B, o, stream=None):
        import torch
        _check(lib().ddm_mlp_forward(self._h, _dev_ptr(x, "x", torch.float32, B * DDM_FIT_LAGS), int(B),
                                     _dev_ptr(o, "o", torch.float32, B * 4), _stream_ptr(stream)),
               "ddm_mlp_forward")

    def last_device_status(self) -> int:
        """DDM_ERR_TIMEOUT if a bounded MMA wait of a forward pass gave up since the last
        call, else DDM_OK (synchronises; clears the word)."""
        out = ctypes.c_int()
        _check(lib().ddm_mlp_last_device_status(self._h, ctypes.byref(out)), "ddm_mlp_last_device_status")
        return int(out.value)

    def grad(self, x, t, B, grad, loss=None, stream=None):
        import torch
        lp = ctypes.c_void_p(0) if loss is None else _dev_ptr(loss, "loss", torch.float32, 1)
        _check(lib().ddm_mlp_grad(self._h, _dev_ptr(x, "x", torch.float32, B * DDM_FIT_LAGS),
                                  _dev_ptr(t, "t", torch.float32, B * 4), int(B),
                                  _dev_ptr(grad, "grad", torch.float32, DDM_MLP_PARAMS), lp,
                                  _stream_ptr(stream)), "ddm_mlp_grad")

    def train_step(self, x, t, B, lr, loss=None, stream=None):
        import torch
        lp = ctypes.c_void_p(0) if loss is None else _dev_ptr(loss, "loss", torch.float32, 1)
        _check(lib().ddm_mlp_train_step(self._h, _dev_ptr(x, "x", torch.float32, B * DDM_FIT_LAGS),
                                        _dev_ptr(t, "t", torch.float32, B * 4), int(B), float(lr), lp,
                                        _stream_ptr(stream)), "ddm_mlp_train_step")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ddm_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
