"""The precision sweep workload at full size: 1024x1024 float32 frames, N = 4096, Fourier-mode
Ornstein-Uhlenbeck dynamics with S(q) = 1 / max(q, 0.02)^2 and D0 log-uniform in [0.01, 1]
(the 4096-frame stacks of the paper's Sec. 2 at its 1024^2 size, Fig. 3).  Every precision
tier of ddm_structure_function against the FP64 oracle on sampled columns kx = 0, 1, 257
and W/2 with every ky and every lag: FP32 and FP32 + FP64 fixup within 1e-4 of each wave
vector's plateau, the FP64 tier within 1e-6.  The stack's DC mode never changes (its OU
rate is 0): its plateau is the input's own float32 rounding, ~1e-15 of the largest, a
static mode judged on the global scale; every tier also matches the oracle on static modes
to 1e-10 of the largest plateau."""
import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import TOL, oracle_columns_of_device_stack

pytestmark = pytest.mark.gpu

TIERS = [("fp32", ddm.DDM_PREC_FP32, TOL), ("fp32_fp64fix", ddm.DDM_PREC_FP32_FP64FIX, TOL),
         ("fp64", ddm.DDM_PREC_FP64, 1e-6)]


def test_precision_sweep_1024x1024x4096():
    import torch
    frames = synth.ou_precision_sweep_1024x1024x4096(seed=0)
    N, H, W = frames.shape
    cols = [0, 1, 257, W // 2]
    F = oracle_columns_of_device_stack(frames, cols)
    D_or = oracle.sf_direct(F)
    s_q = oracle.plateau_scale(F)
    errs = {}
    for name, prec, tol in TIERS:
        plan = ddm.Plan(H, W, N, dtype="f32", precision=prec)
        D = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
        plan.structure_function(frames, D)
        torch.cuda.synchronize()
        got = D.view(H, W // 2 + 1, N)[:, cols, :].cpu().numpy()
        errs[name] = oracle.scaled_error(got, D_or, s_q)
        static = s_q < oracle.STATIC_REL * np.max(s_q)
        if np.any(static):
            glob = float(np.max(np.abs(got - D_or)[static])) / float(np.max(s_q))
            assert glob <= 1e-10, (name, glob)
        assert plan.last_device_status() == 0, name
        assert np.all(got[..., 0] == 0)
        plan.close()
        del D
        torch.cuda.empty_cache()
    for name, _, tol in TIERS:
        assert errs[name] <= tol, errs
