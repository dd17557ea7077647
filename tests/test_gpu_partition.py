"""A stack split by stored wave-vector range on the GPU: every range plan's D rows are
bitwise those of the whole-plane plan (each wave vector's arithmetic does not depend on
its neighbours), rows outside the range are left untouched, and the ranges' radial sums
add up to the whole plane's radial average."""
import numpy as np
import pytest

import paper_2012_05695_b300 as ddm
import synth
from paper_2012_05695_b300 import partition
from gpu_helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W,N,parts,dtype", [
    (32, 32, 600, 2, "u16"),      # L = 1024: grouped TMA kernel, ragged last tile
    (64, 64, 128, 3, "f32"),      # L = 128: per-thread-load kernel
    (16, 64, 300, 4, "f32"),      # L = 512
])
def test_range_plans_match_the_whole_plane_plan(H, W, N, parts, dtype):
    import torch
    rng = np.random.Generator(np.random.PCG64(H * W + N))
    if dtype == "u16":
        frames = synth.blob_stack(H, W, N, n_particles=40, sigma_px=2.0, D0=0.3, seed=5)
    else:
        frames = rng.normal(0, 1, (N, H, W)).astype(np.float32)
    nb = 9
    f = to_device(frames)
    full = ddm.Plan(H, W, N, dtype=dtype, n_bins=nb)
    nq = full.n_q
    D_full = torch.empty(nq * N, device="cuda")
    Dr_full = torch.empty(nb * N, device="cuda")
    c_full = torch.empty(nb, dtype=torch.int32, device="cuda")
    full.structure_function(f, D_full)
    full.azimuthal_average(D_full, Dr_full, c_full)
    ky, kx = (np.asarray(a) for a in ddm.spectrum_index_map(H, W))
    public = ky * (W // 2 + 1) + kx                    # D row of every stored index
    sums = torch.zeros(nb * N, dtype=torch.float64, device="cuda")
    counts = torch.zeros(nb, dtype=torch.int64, device="cuda")
    for q0, q1 in partition.q_ranges(nq, parts):
        plan = ddm.Plan(H, W, N, dtype=dtype, n_bins=nb, q_begin=q0, q_end=q1)
        D = torch.full((nq * N,), float("nan"), device="cuda")
        plan.structure_function(f, D)
        s = torch.empty(nb * N, device="cuda")
        c = torch.empty(nb, dtype=torch.int32, device="cuda")
        plan.azimuthal_sums(D, s, c)
        torch.cuda.synchronize()
        Dh = D.cpu().numpy().reshape(nq, N)
        Dfh = D_full.cpu().numpy().reshape(nq, N)
        rows = public[q0:q1]
        np.testing.assert_array_equal(Dh[rows], Dfh[rows])
        others = np.setdiff1d(np.arange(nq), rows)
        assert np.all(np.isnan(Dh[others]))
        sums += s.double()
        counts += c.long()
        plan.close()
    np.testing.assert_array_equal(counts.cpu().numpy(), c_full.cpu().numpy())
    Dr = partition.merge_radial(sums.view(nb, N), counts).float().cpu().numpy()
    ref = Dr_full.cpu().numpy().reshape(nb, N)
    np.testing.assert_allclose(Dr, ref, rtol=2e-6, atol=1e-6 * float(np.abs(ref).max()))
    full.close()


@pytest.mark.parametrize("H,W,N,parts,dtype", [
    (32, 64, 600, 2, "u16"),      # W/2 = 32: two column blocks; L = 1024 grouped TMA kernel
    (64, 128, 300, 4, "f32"),     # four ranks of one block each; L = 512
    (32, 512, 1024, 3, "u16"),    # uneven ranges of 5 and 6 blocks (the bench's 512 columns)
    (16, 64, 130, 2, "f32"),      # L = 256: per-thread-load kernel
    (16, 32, 2100, 1, "f32"),     # one range of all columns; L = 4096 three-pass kernel
])
def test_kx_range_plans_match_the_whole_plane_plan(H, W, N, parts, dtype):
    """An emulation on one GPU of a stack split by kx columns: every rank's plan transforms
    all rows and only its columns; the union of the ranks' D rows is bitwise the whole
    plan's D, rows of other columns are untouched, the stores hold exactly the range's
    columns of the whole spectrum, and the ranks' radial sums add up to the whole plane's
    radial average."""
    import torch
    if dtype == "u16":
        frames = synth.blob_stack(H, W, N, n_particles=40, sigma_px=2.0, D0=0.3, seed=7)
    else:
        frames = np.random.Generator(np.random.PCG64(H + W + N)).normal(0, 1, (N, H, W)).astype(np.float32)
    nb = 9
    f = to_device(frames)
    full = ddm.Plan(H, W, N, dtype=dtype, n_bins=nb)
    nq = full.n_q
    spec_full = torch.empty(2 * N * nq, device="cuda")
    full.spatial_fft(f, spec_full)
    D_full = torch.empty(nq * N, device="cuda")
    full.temporal_sf(spec_full, D_full)
    Dr_full = torch.empty(nb * N, device="cuda")
    c_full = torch.empty(nb, dtype=torch.int32, device="cuda")
    full.azimuthal_average(D_full, Dr_full, c_full)
    Dd_full = torch.empty(nq * N, device="cuda")
    full.temporal_sf_direct(spec_full, Dd_full)
    torch.cuda.synchronize()
    ky_s, kx_s = (np.asarray(a) for a in ddm.spectrum_index_map(H, W))
    Sf = spec_full.cpu().numpy().view(np.complex64).reshape(N, nq)
    Sf_plane = np.zeros((N, H, W // 2 + 1), np.complex64)
    Sf_plane[:, ky_s, kx_s] = Sf
    Dfh = D_full.cpu().numpy().reshape(nq, N)
    sums = torch.zeros(nb * N, dtype=torch.float64, device="cuda")
    counts = torch.zeros(nb, dtype=torch.int64, device="cuda")
    D_union = np.full((nq, N), np.nan, np.float32)
    for kx0, kx1 in partition.kx_ranges(W, parts):
        plan = ddm.Plan(H, W, N, dtype=dtype, n_bins=nb, kx_begin=kx0, kx_end=kx1)
        assert plan.n_q == H * (kx1 - kx0) + (H if kx0 == 0 else 0)
        ky, kx = plan.wave_vectors()
        rows = ky * (W // 2 + 1) + kx
        # step one alone: the range's store is the whole spectrum's columns, bitwise
        spec = torch.empty(2 * N * plan.n_q, device="cuda")
        plan.spatial_fft(f, spec)
        D = torch.full((nq * N,), float("nan"), device="cuda")
        plan.structure_function(f, D)
        Dd = torch.full((nq * N,), float("nan"), device="cuda")
        plan.temporal_sf_direct(spec, Dd)
        s = torch.empty(nb * N, device="cuda")
        c = torch.empty(nb, dtype=torch.int32, device="cuda")
        plan.azimuthal_sums(D, s, c)
        torch.cuda.synchronize()
        assert plan.last_device_status() == 0
        np.testing.assert_array_equal(spec.cpu().numpy().view(np.complex64).reshape(N, plan.n_q),
                                      Sf_plane[:, ky, kx])
        Dh = D.cpu().numpy().reshape(nq, N)
        np.testing.assert_array_equal(Dh[rows], Dfh[rows])
        others = np.setdiff1d(np.arange(nq), rows)
        assert np.all(np.isnan(Dh[others]))
        np.testing.assert_array_equal(Dd.cpu().numpy().reshape(nq, N)[rows],
                                      Dd_full.cpu().numpy().reshape(nq, N)[rows])
        assert np.all(np.isnan(D_union[rows]))           # ranges are disjoint
        D_union[rows] = Dh[rows]
        sums += s.double()
        counts += c.long()
        plan.close()
    np.testing.assert_array_equal(D_union, Dfh)          # the ranges cover the half plane
    np.testing.assert_array_equal(counts.cpu().numpy(), c_full.cpu().numpy())
    Dr = partition.merge_radial(sums.view(nb, N), counts).float().cpu().numpy()
    ref = Dr_full.cpu().numpy().reshape(nb, N)
    np.testing.assert_allclose(Dr, ref, rtol=2e-6, atol=1e-6 * np.abs(ref).max())

