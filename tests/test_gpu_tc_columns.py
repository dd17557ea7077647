"""The tensor-core DFT-as-GEMM column pass of step one (DDM_PREC_TC_TF32X3: 512 = 16 x 32,
tcgen05.mma kind::tf32 with two-term operand splits) against the oracle's DFT, frame by
frame, and the structure function it feeds against the oracle and the FP32 tier."""
import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import TOL, storage_to_plane, to_device

pytestmark = pytest.mark.gpu


def _frames(N, H, W, dtype, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    if dtype == "u16":
        return rng.integers(0, 4096, (N, H, W), dtype=np.uint16)
    return (rng.normal(0, 1, (N, H, W)) * 100.0 + 5.0).astype(np.float32)


@pytest.mark.parametrize("W,N,dtype", [(512, 3, "u16"), (512, 5, "f32"), (32, 4, "f32"),
                                       (1024, 2, "u16"), (256, 33, "u16")])
def test_tc_column_pass_matches_oracle_dft(W, N, dtype):
    """Every frame's half-plane spectrum within 1e-5 of its largest value (the FP32 column
    pass's bar), including the DC / Nyquist columns unpacked from column 0."""
    import torch
    H = 512
    frames = _frames(N, H, W, dtype, seed=W + N)
    plan = ddm.Plan(H, W, N, dtype=dtype, precision=ddm.DDM_PREC_TC_TF32X3)
    spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device="cuda")
    plan.spatial_fft(to_device(frames), spec)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    s = spec.cpu().numpy().view(np.complex64).reshape(N, plan.n_q).astype(np.complex128)
    F = storage_to_plane(s, H, W)
    diff = frames.astype(np.float64) - frames[0].astype(np.float64)[None]
    ref = oracle.dft2(diff, oracle.half_plane_columns(W))
    for t in range(1, N):
        scale = max(np.max(np.abs(ref[t])), 1e-30)
        err = np.max(np.abs(F[t] - ref[t])) / scale
        assert err <= 1e-5, (t, err)
    assert np.all(np.abs(F[0]) <= 1e-6 * max(np.max(np.abs(ref)), 1.0))


def test_tc_tier_structure_function_blobs_512x512x1024_sampled():
    """The benchmark stack through the tensor-core tier: D on sampled columns against the
    oracle (1e-4 of each plateau), and all of D against the FP32 tier."""
    import torch
    frames = synth.blobs_512x512x1024(seed=0)
    N, H, W = frames.shape
    f = to_device(frames)
    tc = ddm.Plan(H, W, N, dtype="u16", precision=ddm.DDM_PREC_TC_TF32X3)
    fp = ddm.Plan(H, W, N, dtype="u16")
    Dt = torch.empty(tc.n_q * N, device="cuda")
    Df = torch.empty(fp.n_q * N, device="cuda")
    tc.structure_function(f, Dt)
    fp.structure_function(f, Df)
    torch.cuda.synchronize()
    assert tc.last_device_status() == 0
    cols = [0, 3, 256]
    D_or, s_q = oracle.structure_function(frames, kx_sel=cols)
    got = Dt.view(H, W // 2 + 1, N)[:, cols, :].cpu().numpy()
    assert oracle.scaled_error(got, D_or, s_q) <= TOL
    want = Df.view(H, W // 2 + 1, N)[:, cols, :].cpu().numpy()
    assert oracle.scaled_error(got, want, s_q) <= 2 * TOL
