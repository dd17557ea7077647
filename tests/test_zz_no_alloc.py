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


def test_static_call_records_its_own_stage_times():
    import torch
    H, W, N = 64, 64, 128
    frames = synth.ou_stack(H, W, N, 0.5, synth.gaussian_spectrum(0.3), 0.01, 5)
    plan = ddm.Plan(H, W, N, dtype="f32")
    plan.enable_stats(True)
    f = to_device(frames)
    D = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
    assert _call_static(plan, f, D) == 0        # no allocating call on this plan before
    one, two = plan.stats()
    assert one > 0.0 and two > 0.0
    plan.close()


_RESET_SCRIPT = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2012_05695_b300 import _binding as B
import synth
L = B.lib()
rt = ctypes.CDLL("libcudart.so.13")      # the runtime the library is linked against
vp = ctypes.c_void_p

def malloc(n):
    p = vp()
    assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(n)) == 0
    return p

def run(frames):
    N, H, W = frames.shape
    d = B.ddm_plan_desc()
    assert L.ddm_plan_desc_init(ctypes.byref(d), H, W, N) == 0
    d.dtype = B.DDM_IN_F32
    h = vp()
    assert L.ddm_plan_create(ctypes.byref(h), ctypes.byref(d)) == 0
    nq = ctypes.c_int64()
    assert L.ddm_plan_n_q(h, ctypes.byref(nq)) == 0
    n_d = nq.value * N * 4
    f, d1, d2 = malloc(frames.nbytes), malloc(n_d), malloc(n_d)
    assert rt.cudaMemcpy(f, frames.ctypes.data_as(vp), ctypes.c_size_t(frames.nbytes), 1) == 0
    assert L.ddm_structure_function(h, f, d1, None) == 0
    assert L.ddm_structure_function_static(h, f, d2, None) == 0
    assert rt.cudaDeviceSynchronize() == 0
    out = [np.empty(nq.value * N, np.float32) for _ in range(2)]
    for o, src in zip(out, (d1, d2)):
        assert rt.cudaMemcpy(o.ctypes.data_as(vp), src, ctypes.c_size_t(n_d), 2) == 0
    st = ctypes.c_int()
    assert L.ddm_plan_last_device_status(h, ctypes.byref(st)) == 0 and st.value == 0
    for p in (f, d1, d2):
        assert rt.cudaFree(p) == 0
    assert L.ddm_plan_destroy(h) == 0
    return out

stacks = [synth.ou_stack(64, 64, 128, 0.5, synth.gaussian_spectrum(0.3), 0.01, s) for s in (7, 8)]
res = run(stacks[0])
# a device reset destroys this process's context; the library's module, and with it the
# static scratch, is loaded again at a possibly different address in the next context
assert rt.cudaDeviceReset() == 0
res += run(stacks[1])
np.save(sys.argv[2], np.stack(res))
print("ok")
"""


def test_static_scratch_address_follows_a_device_reset(tmp_path):
    """A caller may reset its device between calls (ending its own CUDA context); the next
    static call must look the scratch up again in the new context.  Run in a child process
    so that the reset cannot touch this test process's own context."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = tmp_path / "d.npy"
    r = subprocess.run([sys.executable, "-c", _RESET_SCRIPT, root, str(out)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.load(out)
    for k, seed in enumerate((7, 8)):
        frames = synth.ou_stack(64, 64, 128, 0.5, synth.gaussian_spectrum(0.3), 0.01, seed)
        s_q = oracle.plateau_scale(oracle.dft2(frames, oracle.half_plane_columns(64)))
        want = got[2 * k].reshape(64, 33, 128)
        static = got[2 * k + 1].reshape(64, 33, 128)
        assert oracle.scaled_error(static, want, s_q) <= TOL
