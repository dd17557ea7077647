"""The WITHOUT_FT scheme on the GPU (ddm_temporal_sf_direct: Eq. 1 by explicit differences
of the stored spectra, the paper's comparison method of Sec. 2) against the FP64 oracle,
and against the WITH_FT time kernels on the same spectrum."""
import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import TOL, plane_to_storage, to_device

pytestmark = pytest.mark.gpu


def _spectrum_and_reference(H, W, N, seed):
    frames = synth.ou_stack(H, W, N, 0.3, synth.gaussian_spectrum(0.8), 0.05, seed=seed)
    frames = frames + np.float32(3.0)
    F = oracle.dft2(frames, oracle.half_plane_columns(W)).astype(np.complex64)
    D_ref = oracle.sf_direct(F.astype(np.complex128))
    s_q = oracle.plateau_scale(F.astype(np.complex128))
    return F, D_ref, s_q


def _run(plan, F, H, W, direct=True):
    import torch
    N = F.shape[0]
    spec = torch.from_numpy(plane_to_storage(F, H, W).view(np.float32).ravel().copy()).cuda()
    D = torch.full((plan.n_q * N,), float("nan"), dtype=torch.float32, device="cuda")
    if direct:
        plan.temporal_sf_direct(spec, D)
    else:
        plan.temporal_sf(spec, D)
    torch.cuda.synchronize()
    return D


# N = 1, 2, 3: fewer lags than one block; 17, 33: a block of one lag; 100, 1000: ragged
# edges; 128, 1024: whole blocks; 2049, 4100: several block pairs per thread, fewer wave
# vectors per CTA
@pytest.mark.parametrize("N", [1, 2, 3, 16, 17, 33, 100, 128, 1000, 1024, 2049, 4100])
def test_direct_matches_oracle(N):
    H, W = 4, 8                       # n_q = 20: two CTAs of 8 wave vectors and a ragged one
    F, D_ref, s_q = _spectrum_and_reference(H, W, N, seed=100 + N)
    plan = ddm.Plan(H, W, N, dtype="f32")
    D = _run(plan, F, H, W).cpu().numpy().reshape(H, W // 2 + 1, N)
    assert np.all(np.isfinite(D))
    assert np.all(D[..., 0] == 0)
    if N > 1:
        assert oracle.scaled_error(D, D_ref, s_q) <= TOL
    assert plan.last_device_status() == 0


def test_direct_long_stack_matches_oracle():
    """N = 16384 (the paper's longest stacks): one wave vector per CTA, two block pairs per
    thread."""
    H, W, N = 4, 4, 16384
    F, D_ref, s_q = _spectrum_and_reference(H, W, N, seed=7)
    plan = ddm.Plan(H, W, N, dtype="f32")
    D = _run(plan, F, H, W).cpu().numpy().reshape(H, W // 2 + 1, N)
    assert oracle.scaled_error(D, D_ref, s_q) <= TOL


@pytest.mark.parametrize("N", [300, 1024, 3000])
def test_direct_equals_fourier_route(N):
    """Both schemes on one spectrum: the same D to the tolerance (the paper's premise that
    WITH_FT and WITHOUT_FT compute the same structure function, Sec. 2)."""
    H, W = 16, 16
    F, D_ref, s_q = _spectrum_and_reference(H, W, N, seed=N)
    plan = ddm.Plan(H, W, N, dtype="f32")
    Dd = _run(plan, F, H, W, direct=True).cpu().numpy().reshape(H, W // 2 + 1, N)
    Df = _run(plan, F, H, W, direct=False).cpu().numpy().reshape(H, W // 2 + 1, N)
    assert oracle.scaled_error(Dd, Df, s_q) <= 2 * TOL
    assert oracle.scaled_error(Dd, D_ref, s_q) <= TOL


def test_direct_on_a_range_and_on_the_cropped_store():
    """A wave-vector range writes exactly the range's D rows, bitwise those of the whole
    plan; the low-frequency store (kmax) gives its window's D."""
    import torch
    H, W, N = 32, 32, 500
    F, D_ref, s_q = _spectrum_and_reference(H, W, N, seed=3)
    full = ddm.Plan(H, W, N, dtype="f32")
    Dfull = _run(full, F, H, W).cpu().numpy()
    part = ddm.Plan(H, W, N, dtype="f32", q_begin=64, q_end=300)
    Dpart = _run(part, F, H, W).cpu().numpy().reshape(full.n_q, N)
    ky, kx = ddm.spectrum_index_map(H, W)
    rows = [ky[s] * (W // 2 + 1) + kx[s] for s in range(64, 300)]
    np.testing.assert_array_equal(Dpart[rows], Dfull.reshape(full.n_q, N)[rows])
    other = np.setdiff1d(np.arange(full.n_q), rows)
    assert np.all(np.isnan(Dpart[other]))          # untouched
    # cropped store: the spectrum is cropped by the plan's own step one
    frames = synth.ou_stack(H, W, N, 0.3, synth.gaussian_spectrum(0.8), 0.05, seed=4)
    crop = ddm.Plan(H, W, N, dtype="f32", kmax=7)
    spec = torch.empty(2 * N * crop.n_q, device="cuda")
    crop.spatial_fft(to_device(frames), spec)
    D = torch.empty(crop.n_q * N, device="cuda")
    crop.temporal_sf_direct(spec, D)
    Dt = torch.empty(crop.n_q * N, device="cuda")
    crop.temporal_sf(spec, Dt)
    torch.cuda.synchronize()
    ky, kx = crop.wave_vectors()
    Fo = oracle.dft2(frames, list(range(8)))                 # [N, H, 8]
    Fq = Fo[:, ky, kx]                                       # [N, n_q] in the store's order
    s_c = oracle.plateau_scale(Fq)
    D_c = oracle.sf_direct(Fq)
    got = D.cpu().numpy().reshape(crop.n_q, N)
    assert oracle.scaled_error(got, D_c, s_c) <= TOL
    assert oracle.scaled_error(got, Dt.cpu().numpy().reshape(crop.n_q, N), s_c) <= 2 * TOL


def test_direct_blobs_512x512x1024_sampled_columns():
    """The benchmark stack at full size, through the launch configuration the crossover
    sweep times: every wave vector against the WITH_FT result, two kx columns against the
    oracle."""
    import torch
    frames = synth.blobs_512x512x1024(seed=0)
    N, H, W = frames.shape
    plan = ddm.Plan(H, W, N, dtype="u16")
    spec = torch.empty(2 * N * plan.n_q, device="cuda")
    plan.spatial_fft(to_device(frames), spec)
    Dd = torch.empty(plan.n_q * N, device="cuda")
    Df = torch.empty(plan.n_q * N, device="cuda")
    plan.temporal_sf_direct(spec, Dd)
    plan.temporal_sf(spec, Df)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    cols = [1, 131]
    D_or, s_q = oracle.structure_function(frames, kx_sel=cols)
    Dd3 = Dd.view(H, W // 2 + 1, N)
    got = Dd3[:, cols, :].cpu().numpy()
    assert oracle.scaled_error(got, D_or, s_q) <= TOL
    # all wave vectors: direct vs Fourier route, on each q's plateau s_q = 2 var_t F (the
    # error scale of the oracle comparisons, computed here from the same spectrum)
    Fs = spec.view(N, plan.n_q, 2).double()
    s_st = 2.0 * ((Fs - Fs.mean(dim=0)) ** 2).sum(dim=-1).mean(dim=0)      # storage order
    ky, kx = ddm.spectrum_index_map(H, W)
    rows = torch.tensor(ky, device="cuda") * (W // 2 + 1) + torch.tensor(kx, device="cuda")
    s_pub = torch.empty_like(s_st)
    s_pub[rows] = s_st
    s_pub = torch.clamp(s_pub, min=1e-12 * s_pub.max().item())
    dd, df = Dd.view(plan.n_q, N).double(), Df.view(plan.n_q, N).double()
    rel = ((dd - df).abs() / s_pub[:, None]).max().item()
    assert rel <= 2 * TOL, rel
