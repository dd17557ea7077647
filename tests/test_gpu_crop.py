"""Low-frequency restriction (Sec. 3: the analysis limited to low-frequency wave vectors,
with a smaller store of the images' transforms): kmax keeps |ky'| <= kmax, 0 <= kx <= kmax.
Checked against the FP64 oracle at the kept modes, against the whole-plane plan, and for
the radial average over the kept window."""
import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import TOL, to_device
from paper_2012_05695_b300 import partition

pytestmark = pytest.mark.gpu


def _frames(N, H, W, dtype, seed):
    if dtype == "u16":
        return synth.blob_stack(H, W, N, n_particles=30, sigma_px=1.5, D0=0.4, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(100.0, 3.0, (N, H, W)).astype(np.float32)


def _run(plan, frames):
    import torch
    D = torch.empty(plan.n_q * plan.N, device="cuda")
    plan.structure_function(to_device(frames), D)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    return D


@pytest.mark.parametrize("H,W,N,kmax,dtype", [
    (32, 32, 50, 1, "f32"), (32, 64, 100, 7, "u16"), (64, 64, 128, 15, "f32"),
    (64, 32, 600, 15, "u16"),            # L = 1024: grouped TMA kernel on the cropped store
    (128, 128, 300, 31, "u16"),          # L = 512
])
def test_cropped_store_matches_oracle(H, W, N, kmax, dtype):
    frames = _frames(N, H, W, dtype, seed=H + W + N + kmax)
    plan = ddm.Plan(H, W, N, dtype=dtype, kmax=kmax)
    assert plan.n_q == (2 * kmax + 1) * (kmax + 1)
    D = _run(plan, frames).cpu().numpy().reshape(plan.n_q, N)
    D_ref, s_q = oracle.structure_function(frames, kx_sel=list(range(kmax + 1)))
    ky, kx = plan.wave_vectors()
    assert np.all(D[:, 0] == 0)
    assert oracle.scaled_error(D, D_ref[ky, kx], s_q[ky, kx]) <= TOL


def test_cropped_store_agrees_with_the_whole_plane_plan():
    """Same row transforms; at kx >= 1 also the same column transforms (bitwise); the
    kx = 0 column is transformed directly instead of packed with the Nyquist column."""
    H, W, N, kmax = 64, 64, 200, 15
    frames = _frames(N, H, W, "u16", seed=3)
    crop = ddm.Plan(H, W, N, dtype="u16", kmax=kmax)
    full = ddm.Plan(H, W, N, dtype="u16")
    Dc = _run(crop, frames).cpu().numpy().reshape(crop.n_q, N)
    Df = _run(full, frames).cpu().numpy().reshape(H, W // 2 + 1, N)
    ky, kx = crop.wave_vectors()
    ref = Df[ky, kx]
    inner = kx >= 1
    np.testing.assert_array_equal(Dc[inner], ref[inner])
    scale = np.maximum(np.max(np.abs(ref), axis=1, keepdims=True), 1e-30)
    assert np.max(np.abs(Dc[~inner] - ref[~inner]) / scale[~inner]) <= 1e-5


def test_cropped_radial_average_and_ranges():
    """The radial stage averages the full-plane modes of the kept window; range plans of
    the cropped store give the same D rows and add up to the same radial sums."""
    import torch
    H, W, N, kmax, nb = 64, 64, 96, 15, 12
    frames = _frames(N, H, W, "f32", seed=9)
    plan = ddm.Plan(H, W, N, dtype="f32", kmax=kmax, n_bins=nb)
    D = _run(plan, frames)
    Dr = torch.empty(nb * N, device="cuda")
    cnt = torch.empty(nb, dtype=torch.int32, device="cuda")
    plan.azimuthal_average(D, Dr, cnt)
    torch.cuda.synchronize()
    # reference: mean over the window's full-plane modes of the oracle's D
    D_ref, _ = oracle.structure_function(frames, kx_sel=list(range(kmax + 1)))
    bins = oracle.radial_bins(H, W, nb)
    ky, kx = plan.wave_vectors()
    sums = np.zeros((nb, N))
    counts = np.zeros(nb, np.int64)
    for q in range(plan.n_q):
        w = 1 if kx[q] == 0 else 2
        sums[bins[ky[q], kx[q]]] += w * D_ref[ky[q], kx[q]]
        counts[bins[ky[q], kx[q]]] += w
    np.testing.assert_array_equal(cnt.cpu().numpy(), counts)
    ref = partition.merge_radial(sums, counts)
    got = Dr.cpu().numpy().reshape(nb, N)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    # two ranges of the cropped store
    Dh = D.cpu().numpy().reshape(plan.n_q, N)
    tot = torch.zeros(nb * N, dtype=torch.float64, device="cuda")
    ctot = torch.zeros(nb, dtype=torch.int64, device="cuda")
    for q0, q1 in partition.q_ranges(plan.n_q, 2):
        part = ddm.Plan(H, W, N, dtype="f32", kmax=kmax, n_bins=nb, q_begin=q0, q_end=q1)
        Dp = torch.full((part.n_q * N,), float("nan"), device="cuda")
        part.structure_function(to_device(frames), Dp)
        s = torch.empty(nb * N, device="cuda")
        c = torch.empty(nb, dtype=torch.int32, device="cuda")
        part.azimuthal_sums(Dp, s, c)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(Dp.cpu().numpy().reshape(part.n_q, N)[q0:q1], Dh[q0:q1])
        tot += s.double()
        ctot += c.long()
    np.testing.assert_array_equal(ctot.cpu().numpy(), counts)
    merged = partition.merge_radial(tot.view(nb, N), ctot).float().cpu().numpy()
    np.testing.assert_allclose(merged, got, rtol=2e-6, atol=1e-6 * float(np.abs(got).max()))
