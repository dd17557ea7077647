"""The FP64 tier against the FP64 oracle: the whole path in double precision on the GPU,
D written as float32, so the error is float32's rounding of D, far below the FP32 tier's."""
import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import gpu_structure_function, to_device

pytestmark = pytest.mark.gpu

TOL64 = 1e-6          # |D - D_oracle| / s_q: float32 rounding of D (2^-24 D, D up to a few s_q)


def _frames(N, H, W, dtype, seed):
    if dtype == "u16":
        return synth.blob_stack(H, W, N, max(1, H * W // 90), 2.0, 0.2, seed)
    return synth.ou_stack(H, W, N, 0.5, synth.gaussian_spectrum(0.3), 0.01, seed)


@pytest.mark.parametrize("H,W,N,dtype", [
    (2, 2, 1, "f32"), (8, 8, 3, "f32"), (16, 32, 100, "u16"), (64, 64, 128, "f32"),
    (32, 16, 1000, "u16"), (16, 8, 4096, "f32"), (4, 1024, 5, "u16"),
])
def test_fp64_tier_matches_oracle(H, W, N, dtype):
    frames = _frames(N, H, W, dtype, seed=5 * N + W)
    D, plan, _ = gpu_structure_function(frames, precision=ddm.DDM_PREC_FP64)
    assert plan.last_device_status() == 0
    D_ref, s_q = oracle.structure_function(frames)
    assert np.all(D[..., 0] == 0)
    err = oracle.scaled_error(D, D_ref, s_q)
    assert err <= TOL64, err


def test_fp64_tier_is_more_accurate_than_fp32():
    frames = synth.blobs_512x512x1024(seed=1, N=600, H=32, W=32)
    D64, _, _ = gpu_structure_function(frames, precision=ddm.DDM_PREC_FP64)
    D32, _, _ = gpu_structure_function(frames)
    D_ref, s_q = oracle.structure_function(frames)
    e64, e32 = oracle.scaled_error(D64, D_ref, s_q), oracle.scaled_error(D32, D_ref, s_q)
    assert e64 <= TOL64 and e64 < e32 / 10, (e64, e32)


def test_fp64_tier_takes_only_the_whole_path():
    import torch
    plan = ddm.Plan(8, 8, 16, dtype="f32", precision=ddm.DDM_PREC_FP64)
    frames = to_device(_frames(16, 8, 8, "f32", 0))
    spec = torch.empty(2 * 16 * plan.n_q, device="cuda")
    with pytest.raises(ddm.DDMError):
        plan.spatial_fft(frames, spec)
    D = torch.empty(plan.n_q * 16, device="cuda")
    with pytest.raises(ddm.DDMError):
        plan.temporal_sf(spec, D)
