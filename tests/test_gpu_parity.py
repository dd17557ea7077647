"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bar: |D_gpu - D_oracle| / s_q <= 1e-4 with s_q = 2 var_t F(q, .) (the per-q plateau), and
for the spatial stage max |F_gpu - F_oracle| / max |F_oracle| per frame <= 1e-5.
"""
import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import (TOL, gpu_structure_function, plane_to_storage, storage_to_plane,
                         to_device)

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _frames(N, H, W, dtype, seed):
    if dtype == "u16":
        return synth.blob_stack(H, W, N, max(1, H * W // 90), 2.0, 0.2, seed)
    return synth.ou_stack(H, W, N, 0.5, synth.gaussian_spectrum(0.3), 0.01, seed)


# ------------------------------------------------------------------ step one alone
@pytest.mark.parametrize("H,W,N,dtype", [
    (2, 2, 1, "f32"), (8, 16, 3, "u16"), (16, 8, 2, "f32"), (64, 64, 8, "f32"),
    (64, 64, 8, "u16"), (32, 128, 5, "u16"), (512, 512, 4, "u16"), (1024, 1024, 2, "f32"),
    (4, 1024, 2, "u16"), (1024, 4, 2, "f32"),
])
def test_spatial_fft_matches_oracle_dft(H, W, N, dtype):
    import torch
    frames = _frames(N, H, W, dtype, seed=H + W + N)
    plan = ddm.Plan(H, W, N, dtype=dtype)
    spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device="cuda")
    plan.spatial_fft(to_device(frames), spec)
    torch.cuda.synchronize()
    s = spec.cpu().numpy().view(np.complex64).reshape(N, plan.n_q).astype(np.complex128)
    F = storage_to_plane(s, H, W)
    diff = frames.astype(np.float64) - frames[0].astype(np.float64)[None]
    ref = oracle.dft2(diff, oracle.half_plane_columns(W))
    for t in range(N):
        scale = max(np.max(np.abs(ref[t])), 1e-30)
        err = np.max(np.abs(F[t] - ref[t])) / scale
        assert err <= 1e-5, (t, err)
    assert np.all(F[0] == 0)         # frame 0 minus itself


@pytest.mark.parametrize("S,N,dtype", [(64, 5, "f32"), (128, 3, "u16"), (256, 4, "f32"),
                                       (512, 3, "u16"), (512, 40, "u16")])
def test_spatial_fft_fused_cluster_path_matches_oracle(S, N, dtype):
    """The cluster kernel (rows exchanged through distributed shared memory)."""
    import torch
    frames = _frames(N, S, S, dtype, seed=S + N)
    plan = ddm.Plan(S, S, N, dtype=dtype, spatial_path=ddm._binding.DDM_SPATIAL_FUSED)
    spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device="cuda")
    plan.spatial_fft(to_device(frames), spec)
    torch.cuda.synchronize()
    F = storage_to_plane(spec.cpu().numpy().view(np.complex64).reshape(N, plan.n_q).astype(np.complex128), S, S)
    diff = frames.astype(np.float64) - frames[0].astype(np.float64)[None]
    ref = oracle.dft2(diff, oracle.half_plane_columns(S))
    for t in range(N):
        scale = max(np.max(np.abs(ref[t])), 1e-30)
        assert np.max(np.abs(F[t] - ref[t])) / scale <= 1e-5, t
    assert plan.last_device_status() == 0


@pytest.mark.parametrize("H,W,N,dtype", [(512, 512, 4, "u16"), (256, 64, 3, "f32"), (600, 800, 2, "u16"),
                                         (1024, 256, 2, "f32")])
def test_spatial_fft_unaligned_spectrum_matches_aligned(H, W, N, dtype):
    """A caller's spectrum that is 8-byte but not 16-byte aligned takes the column passes'
    per-thread loads instead of their TMA staging (which needs 16-byte rows and base); both
    do the same arithmetic, so the spectra agree bit for bit."""
    import torch
    frames = to_device(_frames(N, H, W, dtype, seed=H + W))
    plan = ddm.Plan(H, W, N, dtype=dtype)
    n = 2 * N * plan.n_q
    aligned = torch.empty(n, dtype=torch.float32, device="cuda")
    buf = torch.empty(n + 2, dtype=torch.float32, device="cuda")
    shifted = buf[2:]
    assert aligned.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 8
    plan.spatial_fft(frames, aligned)
    plan.spatial_fft(frames, shifted)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    assert torch.equal(aligned, shifted)


def test_spatial_fft_without_reference_subtraction():
    import torch
    H, W, N = 64, 32, 3
    frames = _frames(N, H, W, "u16", seed=5)
    plan = ddm.Plan(H, W, N, dtype="u16", subtract_ref=0)
    spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device="cuda")
    plan.spatial_fft(to_device(frames), spec)
    torch.cuda.synchronize()
    F = storage_to_plane(spec.cpu().numpy().view(np.complex64).reshape(N, plan.n_q), H, W)
    ref = oracle.dft2(frames, oracle.half_plane_columns(W))
    assert np.max(np.abs(F - ref)) / np.max(np.abs(ref)) <= 1e-5


# ------------------------------------------------------------------ step two alone
@pytest.mark.parametrize("N", [1, 2, 3, 5, 17, 33, 64, 100, 128, 255, 256, 511, 1000, 1024,
                               1025, 1500, 2048, 2049, 3000, 4096, 5000, 8192, 8193,
                               12000, 16384])
def test_temporal_matches_oracle(N):
    """Oracle spectrum in, oracle D out: isolates the time-sequence stage."""
    import torch
    H, W = 4, 8                       # n_q = 20: one full tile plus a ragged one
    frames = synth.ou_stack(H, W, N, 0.3, synth.gaussian_spectrum(0.8), 0.05, seed=N)
    frames = frames + np.float32(3.0)           # a static offset the mean removal must absorb
    F = oracle.dft2(frames, oracle.half_plane_columns(W))       # [N, H, W/2+1]
    F32 = F.astype(np.complex64)
    D_ref = oracle.sf_direct(F32.astype(np.complex128))         # what the input implies
    plan = ddm.Plan(H, W, N, dtype="f32")
    spec = torch.from_numpy(plane_to_storage(F32, H, W).view(np.float32).ravel().copy()).cuda()
    D = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
    plan.temporal_sf(spec, D)
    torch.cuda.synchronize()
    D = D.cpu().numpy().reshape(H, W // 2 + 1, N)
    s_q = oracle.plateau_scale(F32.astype(np.complex128))
    if N == 1:
        assert np.all(D == 0)
        return
    assert np.all(D[..., 0] == 0)
    assert oracle.scaled_error(D, D_ref, s_q) <= TOL


@pytest.mark.parametrize("H,W,N,dtype,kw", [
    (16, 16, 3000, "u16", {}),                               # L = 4096, many tiles
    (32, 16, 2000, "f32", {"q_begin": 64, "q_end": 200}),    # L = 2048, a wave-vector range
    (32, 32, 2500, "u16", {"kmax": 7}),                      # L = 4096 on the cropped store
    (16, 16, 6000, "u16", {}),                               # L = 8192, one 512-thread CTA per SM
    (8, 16, 16384, "u16", {}),                               # L = 16384: one wave vector per CTA
    (16, 16, 10000, "f32", {"q_begin": 64, "q_end": 140}),   # L = 16384 on a wave-vector range
])
def test_long_sequences_end_to_end(H, W, N, dtype, kw):
    """N above 1024: the three-pass time transforms, from frames to D."""
    import torch
    if dtype == "u16":
        frames = synth.blob_stack(H, W, N, n_particles=8, sigma_px=1.5, D0=0.3, seed=N)
    else:
        frames = synth.ou_stack(H, W, N, 0.2, synth.gaussian_spectrum(0.7), 0.05, seed=N)
    plan = ddm.Plan(H, W, N, dtype=dtype, **kw)
    D = torch.full((plan.n_q * N,), float("nan"), device="cuda")
    plan.structure_function(to_device(frames), D)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    D = D.cpu().numpy().reshape(plan.n_q, N)
    ky, kx = plan.wave_vectors()
    kmax = kw.get("kmax", 0)
    D_ref, s_q = oracle.structure_function(frames, kx_sel=list(range(kmax + 1)) if kmax else None)
    rows = np.arange(plan.n_q)
    if "q_begin" in kw:               # stored range -> D rows
        sky, skx = (np.asarray(a) for a in ddm.spectrum_index_map(H, W))
        st = np.arange(kw["q_begin"], kw["q_end"])
        rows = sky[st] * (W // 2 + 1) + skx[st]
    Dt, Dr, sq = D[rows], D_ref[ky[rows], kx[rows]], s_q[ky[rows], kx[rows]]
    assert np.all(Dt[:, 0] == 0)
    assert oracle.scaled_error(Dt, Dr, sq) <= TOL


def test_temporal_many_tiles_random_spectrum():
    """A spectrum of independent random walks over many tiles (n_q = 16 * 33)."""
    import torch
    H, W, N = 16, 64, 1024
    rng = _rng(77)
    n_q = H * (W // 2 + 1)
    steps = rng.standard_normal((N, n_q)) + 1j * rng.standard_normal((N, n_q))
    walk = np.cumsum(steps, axis=0) * 0.05 + (rng.standard_normal(n_q) * 40)[None]
    F32 = walk.astype(np.complex64)
    plan = ddm.Plan(H, W, N, dtype="f32")
    spec = torch.from_numpy(F32.view(np.float32).ravel().copy()).cuda()
    D = torch.empty(n_q * N, dtype=torch.float32, device="cuda")
    plan.temporal_sf(spec, D)
    torch.cuda.synchronize()
    # storage order -> plane order for the comparison
    ky, kx = ddm.spectrum_index_map(H, W)
    pub = np.asarray(ky) * (W // 2 + 1) + np.asarray(kx)
    D = D.cpu().numpy().reshape(n_q, N)
    Fpub = np.zeros_like(F32)
    Fpub[:, pub] = F32
    D_ref = oracle.sf_direct(Fpub.astype(np.complex128))
    s_q = oracle.plateau_scale(Fpub.astype(np.complex128))
    assert oracle.scaled_error(D, D_ref, s_q) <= TOL


# ------------------------------------------------------------------ end to end
@pytest.mark.parametrize("H,W,N,dtype", [
    (2, 2, 1, "f32"), (2, 2, 2, "u16"), (8, 8, 3, "f32"), (16, 32, 100, "u16"),
    (64, 64, 128, "f32"), (64, 64, 64, "u16"), (128, 256, 37, "u16"), (32, 16, 1024, "f32"),
])
def test_structure_function_matches_oracle(H, W, N, dtype):
    frames = _frames(N, H, W, dtype, seed=7 * N + H)
    D, _, _ = gpu_structure_function(frames)
    D_ref, s_q = oracle.structure_function(frames)
    assert np.all(D[..., 0] == 0)
    assert oracle.scaled_error(D, D_ref, s_q) <= TOL


@pytest.mark.parametrize("seed", [0, 1])
def test_ou_64x64x128(seed):
    """The small OU workload: 64x64 float32 frames, N = 128, all lags."""
    frames = synth.ou_64x64x128(seed)
    D, _, _ = gpu_structure_function(frames)
    D_ref, s_q = oracle.structure_function(frames)
    assert oracle.scaled_error(D, D_ref, s_q) <= TOL


def test_blobs_512x512x1024_sampled_columns():
    """Full-size 512x512 uint16 stack, N = 1024, in the benchmark's launch configuration;
    the oracle checks every ky and every lag of a sample of kx columns."""
    frames = synth.blobs_512x512x1024(seed=0)
    D, _, _ = gpu_structure_function(frames)
    cols = [0, 1, 2, 3, 64, 127, 128, 200, 255, 256]
    D_ref, s_q = oracle.structure_function(frames, kx_sel=cols)
    err = oracle.scaled_error(D[:, cols, :], D_ref, s_q)
    assert err <= TOL, err


# ------------------------------------------------------------------ radial average
def _symmetric_plane(H, W, N, seed):
    R = _rng(seed).random((H, W, N)) * 10 + 1
    mirror = R[(-np.arange(H)) % H][:, (-np.arange(W)) % W]
    return 0.5 * (R + mirror)


@pytest.mark.parametrize("H,W,N,nb", [(8, 16, 5, 7), (64, 64, 16, 46), (512, 512, 8, 362),
                                      (16, 4, 3, 2), (32, 32, 9, 1)])
def test_radial_average_matches_oracle(H, W, N, nb):
    import torch
    Dfull = _symmetric_plane(H, W, N, seed=H * W + nb)
    half = np.ascontiguousarray(Dfull[:, : W // 2 + 1, :]).astype(np.float32)
    # the oracle averages the full plane (same float32 values the device sees)
    Dr_ref, cnt_ref = oracle.radial_average(Dfull.astype(np.float32).astype(np.float64), nb)
    plan = ddm.Plan(H, W, N, dtype="f32", n_bins=nb)
    Dr = torch.empty(nb * N, dtype=torch.float32, device="cuda")
    cnt = torch.empty(nb, dtype=torch.int32, device="cuda")
    plan.azimuthal_average(torch.from_numpy(half.ravel()).cuda(), Dr, cnt)
    torch.cuda.synchronize()
    assert np.array_equal(cnt.cpu().numpy(), cnt_ref)
    np.testing.assert_allclose(Dr.cpu().numpy().reshape(nb, N), Dr_ref, rtol=1e-5, atol=0)


def test_radial_average_is_bitwise_deterministic():
    import torch
    H, W, N, nb = 512, 512, 64, 362
    half = _symmetric_plane(H, W, N, 3)[:, : W // 2 + 1].astype(np.float32)
    plan = ddm.Plan(H, W, N, dtype="f32", n_bins=nb)
    D = torch.from_numpy(np.ascontiguousarray(half).ravel()).cuda()
    outs = []
    for _ in range(3):
        Dr = torch.empty(nb * N, dtype=torch.float32, device="cuda")
        plan.azimuthal_average(D, Dr)
        outs.append(Dr.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_radial_end_to_end_ou_64x64x128():
    import torch
    frames = synth.ou_64x64x128(2)
    nb = 46
    D, plan, D_dev = gpu_structure_function(frames, n_bins=nb)
    Dr = torch.empty(nb * 128, dtype=torch.float32, device="cuda")
    plan.azimuthal_average(D_dev, Dr)
    torch.cuda.synchronize()
    F = oracle.dft2(frames)
    D_full = oracle.sf_direct(F)                    # [H, W, N], full plane
    Dr_ref, counts = oracle.radial_average(D_full, nb)
    s_full = oracle.plateau_scale(F)
    s_bin, _ = oracle.radial_average(np.repeat(s_full[:, :, None], 1, axis=2), nb)
    got = Dr.cpu().numpy().reshape(nb, 128)
    nz = counts > 0
    err = np.max(np.abs(got[nz] - Dr_ref[nz]) / s_bin[nz])
    assert err <= TOL, err


# ------------------------------------------------------------------ plumbing
def test_nonfinite_input_sets_device_status():
    import torch
    H, W, N = 8, 8, 4
    frames = _frames(N, H, W, "f32", 1)
    frames[2, 3, 3] = np.nan
    D, plan, _ = gpu_structure_function(frames)
    assert plan.last_device_status() == ddm._binding.DDM_ERR_NUMERIC
    assert plan.last_device_status() == 0            # reading resets it
    good = _frames(N, H, W, "f32", 2)
    Dd = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
    plan.structure_function(to_device(good), Dd)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0


def test_caller_workspace_and_limit():
    import torch
    H, W, N = 16, 16, 8
    frames = _frames(N, H, W, "u16", 4)
    plan = ddm.Plan(H, W, N)
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device="cuda")
    plan.set_workspace(ws)
    D = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
    plan.structure_function(to_device(frames), D)
    torch.cuda.synchronize()
    D_ref, s_q = oracle.structure_function(frames)
    assert oracle.scaled_error(D.cpu().numpy().reshape(H, W // 2 + 1, N), D_ref, s_q) <= TOL
    with pytest.raises(ddm.DDMError) as e:
        ddm.Plan(H, W, N, max_workspace_bytes=1024)
    assert e.value.status == ddm._binding.DDM_ERR_OOM


def test_side_stream():
    import torch
    H, W, N = 32, 32, 16
    frames = _frames(N, H, W, "u16", 9)
    plan = ddm.Plan(H, W, N)
    s = torch.cuda.Stream()
    f = to_device(frames)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        D = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
        plan.structure_function(f, D, stream=s)
    s.synchronize()
    D_ref, s_q = oracle.structure_function(frames)
    assert oracle.scaled_error(D.cpu().numpy().reshape(H, W // 2 + 1, N), D_ref, s_q) <= TOL


# ------------------------------------------------------------------ FP64-fixup tier
@pytest.mark.parametrize("N", [300, 1024, 2000, 4096, 6000])
def test_fp64_fixup_tier_small_lags_relative_to_D(N):
    """Slow dynamics: D(1) is ~1e-5 of the plateau, so P1 + P2 - 2 Re C cancels most of
    its FP32 digits.  The fixup tier recomputes lags 1..8 by direct differences (FP64
    across threads) and must match the FP64 oracle relative to D itself; the whole D
    stays within the usual plateau-relative tolerance."""
    import torch
    H = W = 16
    frames = synth.ou_stack(H, W, N, 1e-4, synth.gaussian_spectrum(0.5), 1e-3, seed=N,
                            dtype=np.float32) + np.float32(5.0)
    D_ref, s_q = oracle.structure_function(frames)
    errs = {}
    for prec in (ddm.DDM_PREC_FP32, ddm.DDM_PREC_FP32_FP64FIX):
        D, plan, _ = gpu_structure_function(frames, precision=prec)
        assert oracle.scaled_error(D, D_ref, s_q) <= TOL
        ref = D_ref[..., 1:9]
        big = ref > 1e-9 * np.max(ref)
        errs[prec] = float(np.max(np.abs(D[..., 1:9] - ref)[big] / ref[big]))
    assert errs[ddm.DDM_PREC_FP32_FP64FIX] <= 2e-5, errs
    assert errs[ddm.DDM_PREC_FP32_FP64FIX] < errs[ddm.DDM_PREC_FP32], errs
    print(f"\nsmall-lag error relative to D, N={N}: FP32 {errs[ddm.DDM_PREC_FP32]:.2e}, "
          f"FP32+FP64 fixup {errs[ddm.DDM_PREC_FP32_FP64FIX]:.2e}")


def test_fp64_fixup_tier_blobs_512x512x1024_sampled():
    frames = synth.blobs_512x512x1024(seed=3)
    D, _, _ = gpu_structure_function(frames, precision=ddm.DDM_PREC_FP32_FP64FIX)
    cols = [1, 100, 256]
    D_ref, s_q = oracle.structure_function(frames, kx_sel=cols)
    assert oracle.scaled_error(D[:, cols, :], D_ref, s_q) <= TOL
    ref = D_ref[..., 1:9]
    err = np.max(np.abs(D[:, cols, 1:9] - ref) / ref)
    assert err <= 2e-5, err


@pytest.mark.parametrize("S,N,kw", [
    (640, 2048, {}),
    (640, 4096, {"precision": ddm.DDM_PREC_FP32_FP64FIX}),
    (640, 3000, {"q_begin": 1024, "q_end": 200000}),
    (512, 16384, {}),
])
def test_temporal_blocked_copy_matches_oracle(S, N, kw):
    """n_q = 205440 (640 x 640) at L = 2048 .. 4096 and 131584 (512 x 512) at L = 16384: the
    long time kernels read a blocked copy of the spectrum (16 wave vectors contiguous over
    time).  Random spectrum drawn on the device, checked on sampled wave vectors at block
    edges, inside blocks and at the range ends."""
    import torch
    H = W = S
    plan = ddm.Plan(H, W, N, dtype="f32", **kw)
    nq = plan.n_q
    g = torch.Generator(device="cuda")
    g.manual_seed(N)
    spec = torch.randn(2 * N * nq, generator=g, device="cuda") + 0.5
    D = torch.full((nq * N,), float("nan"), device="cuda")
    plan.temporal_sf(spec, D)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    q0, q1 = kw.get("q_begin", 0), kw.get("q_end", nq)
    cand = [q0, q0 + 1, q0 + 15, q0 + 16, q0 + 17, q0 + 31, q0 + 1000, (q0 + q1) // 2, q1 - 17, q1 - 2, q1 - 1]
    s = np.array(sorted(set(c for c in cand if q0 <= c < q1)))
    F = spec.view(N, nq, 2)[:, torch.from_numpy(s).cuda(), :].cpu().numpy().astype(np.float64)
    F = F[..., 0] + 1j * F[..., 1]                      # [N, len(s)]
    D_ref = oracle.sf_direct(F)                          # [len(s), N]
    sky, skx = (np.asarray(a) for a in ddm.spectrum_index_map(H, W))
    rows = sky[s] * (W // 2 + 1) + skx[s]
    Dg = D.view(nq, N)[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.all(Dg[:, 0] == 0)
    assert oracle.scaled_error(Dg, D_ref, oracle.plateau_scale(F)) <= TOL


@pytest.mark.parametrize("H,W,N,dtype,kw", [
    (512, 1024, 2048, "u16", {}),                                  # power-of-two columns
    (1022, 400, 2048, "f32", {}),                                  # Bluestein rows and columns
    (512, 1024, 2048, "u16", {"q_begin": 64, "q_end": 200007}),    # range ending mid-block
])
def test_structure_function_blocked_write_matches_oracle(H, W, N, dtype, kw):
    """n_q >= 200000 at L = 2048: step one's column pass writes the time kernels' blocked
    copy directly (no corner-turn pass).  Random frames; the oracle on sampled (ky, kx)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(H + W + N))
    if dtype == "u16":
        frames = rng.integers(1800, 2201, size=(N, H, W), dtype=np.uint16)
    else:
        frames = rng.uniform(-1.0, 1.0, size=(N, H, W)).astype(np.float32)
    plan = ddm.Plan(H, W, N, dtype=dtype, **kw)
    D = torch.full((plan.n_q * N,), float("nan"), device="cuda")
    plan.structure_function(to_device(frames), D)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    Wq = W // 2 + 1
    kx_sel = [0, 1, 7, W // 2]
    ky_sel = [0, 1, H // 2 - 1, H // 2, H - 1]
    F = oracle.dft2(frames, kx_sel)[:, ky_sel, :]                  # [N, 5, 4]
    D_ref = oracle.sf_direct(F)                                    # [5, 4, N]
    s_q = oracle.plateau_scale(F)
    Dg = D.view(plan.n_q, N).cpu().numpy()
    sky, skx = (np.asarray(a) for a in ddm.spectrum_index_map(H, W))
    stored = {(int(a), int(b)): s for s, (a, b) in enumerate(zip(sky, skx))}
    q0, q1 = kw.get("q_begin", 0), kw.get("q_end", plan.n_q)
    checked = 0
    for a, ky in enumerate(ky_sel):
        for b, kx in enumerate(kx_sel):
            if not (q0 <= stored[(ky, kx)] < q1):
                continue
            row = Dg[ky * Wq + kx]
            assert row[0] == 0
            err = np.max(np.abs(row - D_ref[a, b])) / s_q[a, b]
            assert err <= TOL, (ky, kx, err)
            checked += 1
    assert checked >= 5
