"""The C-ABI library loads, exports every symbol include/ddm.h declares, and validates
arguments on the host (no device needed for any of these)."""
import ctypes
import subprocess

import pytest

import paper_2012_05695_b300 as ddm
from paper_2012_05695_b300 import _binding as B
from conftest import cuda_available


def test_library_is_in_tree_and_loads():
    L = ddm.lib()
    assert L.ddm_abi_version() == 5
    assert ddm.LIB_PATH.endswith("paper_2012_05695_b300/_lib/libddm_b300.so")


def test_every_header_function_is_exported():
    names = ddm.header_functions()
    assert len(names) >= 13
    L = ddm.lib()
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", ddm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported


def test_status_strings():
    for s in range(8):
        assert ddm.status_string(s)
    assert ddm.status_string(0) == "ok"
    assert "unknown" in ddm.status_string(99)


def _desc(H=8, W=8, N=4):
    d = B.ddm_plan_desc()
    assert ddm.lib().ddm_plan_desc_init(ctypes.byref(d), H, W, N) == 0
    return d


def test_desc_init_defaults():
    d = _desc(16, 32, 10)
    assert (d.H, d.W, d.N, d.dtype, d.precision, d.M, d.n_bins, d.subtract_ref) == \
        (16, 32, 10, 0, 0, 0, 0, 1)
    assert ddm.lib().ddm_plan_desc_init(None, 1, 1, 1) == B.DDM_ERR_INVALID_ARG


@pytest.mark.parametrize("field,value,status", [
    ("H", 3, B.DDM_ERR_INVALID_ARG),
    ("H", 21, B.DDM_ERR_INVALID_ARG),             # odd sides: rows are transformed in pairs
    ("W", 7, B.DDM_ERR_INVALID_ARG),
    ("W", 1030, B.DDM_ERR_UNSUPPORTED),           # above 1024
    ("H", 1100, B.DDM_ERR_UNSUPPORTED),           # above 1024, not a mixed-radix side
    ("W", 1700, B.DDM_ERR_UNSUPPORTED),
    ("W", 0, B.DDM_ERR_INVALID_ARG),
    ("H", 4096, B.DDM_ERR_UNSUPPORTED),
    ("N", 0, B.DDM_ERR_INVALID_ARG),
    ("N", 16385, B.DDM_ERR_UNSUPPORTED),
    ("dtype", 7, B.DDM_ERR_INVALID_ARG),
    ("precision", 9, B.DDM_ERR_INVALID_ARG),
    ("precision", 4, B.DDM_ERR_INVALID_ARG),
    ("precision", 3, B.DDM_ERR_UNSUPPORTED),      # tensor-core column pass: H = 512 only
    ("precision", 1, B.DDM_ERR_UNSUPPORTED),      # FP64 fixup needs N >= 257
    ("M", 6, B.DDM_ERR_INVALID_ARG),          # M < 2N - 1 wraps around (App. B)
    ("M", 7, B.DDM_ERR_UNSUPPORTED),          # legal pad length, not the one built
    ("subtract_ref", 2, B.DDM_ERR_INVALID_ARG),
    ("n_bins", -1, B.DDM_ERR_INVALID_ARG),
    ("max_workspace_bytes", 16, B.DDM_ERR_OOM),
    ("spatial_path", 7, B.DDM_ERR_INVALID_ARG),
    ("q_begin", 32, B.DDM_ERR_INVALID_ARG),       # range start not a multiple of 64
    ("q_end", 41, B.DDM_ERR_INVALID_ARG),         # past n_q = 8 * 5 = 40
    ("q_begin", -64, B.DDM_ERR_INVALID_ARG),
    ("kmax", 2, B.DDM_ERR_INVALID_ARG),           # the cropped window needs kmax odd
    ("kmax", 5, B.DDM_ERR_INVALID_ARG),           # and below H/2 = W/2 = 4
    ("kmax", -1, B.DDM_ERR_INVALID_ARG),
])
def test_plan_create_validates_before_touching_the_device(field, value, status):
    d = _desc(8, 8, 4)
    setattr(d, field, value)
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == status
    assert not h.value


def test_plan_desc_layout_matches_the_header():
    """The ctypes mirror of ddm_plan_desc has the C layout (its size is the library's
    sizeof), and ddm_plan_desc_init zeroes the optional fields."""
    d = _desc(16, 16, 8)
    assert (d.q_begin, d.q_end, d.kmax) == (0, 0, 0)
    assert ctypes.sizeof(B.ddm_plan_desc) == ddm.lib().ddm_plan_desc_size()
    assert B.ddm_plan_desc.q_begin.offset % 8 == 0
    d.q_begin, d.q_end = 64, 32      # empty range
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == B.DDM_ERR_INVALID_ARG


def test_null_arguments():
    L = ddm.lib()
    d = _desc()
    assert L.ddm_plan_create(None, ctypes.byref(d)) == B.DDM_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L.ddm_plan_create(ctypes.byref(h), None) == B.DDM_ERR_INVALID_ARG
    assert L.ddm_plan_destroy(None) == 0
    nul = ctypes.c_void_p(0)
    assert L.ddm_structure_function(nul, nul, nul, nul) == B.DDM_ERR_INVALID_ARG
    assert L.ddm_spatial_fft(nul, nul, nul, nul) == B.DDM_ERR_INVALID_ARG
    assert L.ddm_temporal_sf(nul, nul, nul, nul) == B.DDM_ERR_INVALID_ARG
    assert L.ddm_azimuthal_average(nul, nul, nul, nul, nul) == B.DDM_ERR_INVALID_ARG
    sz = ctypes.c_size_t()
    assert L.ddm_plan_workspace_size(nul, ctypes.byref(sz)) == B.DDM_ERR_INVALID_ARG


@pytest.mark.skipif(cuda_available(), reason="checks the no-device path")
def test_valid_plan_without_device_is_a_cuda_error():
    d = _desc(8, 8, 4)
    h = ctypes.c_void_p()
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == B.DDM_ERR_CUDA
    assert not h.value


@pytest.mark.parametrize("H,W", [(1080, 1280), (1200, 1024), (2048, 1280), (1280, 1022), (1080, 1920),
                                 (1536, 1600), (2000, 1440)])
def test_mixed_radix_sides_above_1024_pass_validation(H, W):
    """The mixed-radix sides above 1024 (1080 = 27 x 40 ... 2000 = 40 x 50) are built; without
    a device the plan gets as far as the first CUDA call."""
    d = _desc(H, W, 4)
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == B.DDM_ERR_CUDA
    assert not h.value


def test_low_frequency_window_needs_power_of_two_sides():
    d = _desc(600, 800, 4)
    d.kmax = 31
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == B.DDM_ERR_UNSUPPORTED
    assert not h.value


def test_fp64_fixup_tier_stops_at_8192_frames():
    d = _desc(8, 8, 9000)
    d.precision = B.DDM_PREC_FP32_FP64FIX
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == B.DDM_ERR_UNSUPPORTED
    assert not h.value


@pytest.mark.parametrize("H,W,N,kmax,status", [
    (8, 8, 5000, 0, B.DDM_ERR_UNSUPPORTED),        # FP64 tier: N <= 4096
    (8, 12, 16, 0, B.DDM_ERR_UNSUPPORTED),         # FP64 tier: power-of-two sides
    (16, 16, 16, 3, B.DDM_ERR_UNSUPPORTED),        # FP64 tier: the full half plane
])
def test_fp64_tier_limits(H, W, N, kmax, status):
    d = _desc(H, W, N)
    d.precision = B.DDM_PREC_FP64
    d.kmax = kmax
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == status
    assert not h.value


@pytest.mark.parametrize("H,W,kx0,kx1,extra,status", [
    (64, 64, 8, 32, {}, B.DDM_ERR_INVALID_ARG),           # not whole blocks of 16 columns
    (64, 64, 0, 48, {}, B.DDM_ERR_INVALID_ARG),           # beyond W/2
    (64, 64, 16, 16, {}, B.DDM_ERR_INVALID_ARG),          # empty
    (64, 64, -16, 16, {}, B.DDM_ERR_INVALID_ARG),
    (64, 64, 16, 32, {"kmax": 7}, B.DDM_ERR_UNSUPPORTED),
    (64, 64, 16, 32, {"q_begin": 0, "q_end": 64}, B.DDM_ERR_UNSUPPORTED),
    (64, 64, 16, 32, {"precision": B.DDM_PREC_FP64}, B.DDM_ERR_UNSUPPORTED),
    (64, 64, 16, 32, {"spatial_path": B.DDM_SPATIAL_FUSED}, B.DDM_ERR_UNSUPPORTED),
    (96, 96, 0, 16, {}, B.DDM_ERR_UNSUPPORTED),           # the power-of-two column pass only
    (64, 16, 0, 8, {}, B.DDM_ERR_INVALID_ARG),
])
def test_kx_column_range_validation(H, W, kx0, kx1, extra, status):
    d = _desc(H, W, 100)
    d.kx_begin, d.kx_end = kx0, kx1
    for k, v in extra.items():
        setattr(d, k, v)
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == status
    assert not h.value


@pytest.mark.skipif(cuda_available(), reason="checks the no-device path")
def test_kx_column_range_passes_validation():
    d = _desc(64, 512, 100)
    d.kx_begin, d.kx_end = 96, 256
    h = ctypes.c_void_p(123)
    assert ddm.lib().ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == B.DDM_ERR_CUDA
