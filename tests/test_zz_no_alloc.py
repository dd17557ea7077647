"""ddm_structure_function_static: the allocation-free entry point for callers that must
not allocate device memory when they ask for D (their device memory is owned by another
pool allocator, or the call sits in a no-allocation loop).  It keeps the spectrum in the
library's own fixed device scratch; its D must match ddm_structure_function's.

Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import TOL, to_device

pytestmark = pytest.mark.gpu


def _call_static(plan, frames_dev, D_dev):
    import torch
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    return ddm.lib().ddm_structure_function_static(
        plan.handle, ctypes.c_void_p(frames_dev.data_ptr()), ctypes.c_void_p(D_dev.data_ptr()),
        stream)


@pytest.mark.parametrize("H,W,N,dtype", [(64, 64, 128, "f32"), (128, 64, 200, "u16")])
def test_static_matches_allocating_entry_point_twice(H, W, N, dtype):
    import torch
    if dtype == "f32":
        stacks = [synth.ou_stack(H, W, N, 0.5, synth.gaussian_spectrum(0.3), 0.01, s) for s in (3, 4)]
    else:
        stacks = [synth.blob_stack(H, W, N, 90, 2.0, 0.2, s) for s in (3, 4)]
    plan = ddm.Plan(H, W, N, dtype=dtype)
    for frames in stacks:                       # two calls in a row, different stacks
        f = to_device(frames)
        D_ref = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
        plan.structure_function(f, D_ref)
        D = torch.full((plan.n_q * N,), float("nan"), dtype=torch.float32, device="cuda")
        assert _call_static(plan, f, D) == 0
        torch.cuda.synchronize()
        s_q = oracle.plateau_scale(oracle.dft2(frames, oracle.half_plane_columns(W)))
        got = D.cpu().numpy().reshape(H, W // 2 + 1, N)
        want = D_ref.cpu().numpy().reshape(H, W // 2 + 1, N)
        assert oracle.scaled_error(got, want, s_q) <= TOL
    assert plan.last_device_status() == 0


def test_static_rejects_a_spectrum_larger_than_the_scratch():
    import torch
    H = W = 256
    N = 1024                                     # 33024 * 1024 * 8 B > 64 MiB
    plan = ddm.Plan(H, W, N, dtype="u16")
    assert plan.n_q * N * 8 > 64 * 1024 * 1024     # DDM_STATIC_SCRATCH_BYTES
    f = torch.zeros(N * H * W, dtype=torch.uint16, device="cuda")
    D = torch.full((16,), 7.0, device="cuda")    # never written: the call is refused
    assert _call_static(plan, f, D) == ddm._binding.DDM_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.all(D == 7.0)
