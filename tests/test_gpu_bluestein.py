"""Frame sides that are not powers of two (step one of Sec. 2 by the mixed-radix kernels for
384, 480, 540, 600, 640, 720, 768, 800, 900, 960, 1000 and by Bluestein's chirp-z transform
otherwise) and sides of 2048, against the FP64 oracle, through the C ABI.

Shapes cover every convolution length the kernels are built for (M = 64 .. 2048), a
power-of-two side beside a non-power-of-two one in both orders, ragged row-pair and
column blocks, and the 600 x 800 camera shape at its full stack length.
"""
import numpy as np
import pytest

import oracle
import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import TOL, gpu_structure_function, storage_to_plane, to_device

pytestmark = pytest.mark.gpu


def _frames(N, H, W, dtype, seed):
    if dtype == "u16":
        return synth.blob_stack(H, W, N, max(1, H * W // 90), 2.0, 0.2, seed)
    return synth.ou_stack(H, W, N, 0.5, synth.gaussian_spectrum(0.3), 0.01, seed)


@pytest.mark.parametrize("H,W,N,dtype", [
    (8, 12, 3, "f32"),         # M = 32: one thread per transform, no exchange
    (6, 10, 2, "u16"),
    (14, 16, 3, "f32"),        # columns M = 32, power-of-two rows
    (18, 22, 3, "f32"),        # M = 64 both ways
    (100, 64, 4, "u16"),       # columns M = 256, power-of-two rows
    (64, 100, 3, "f32"),       # rows M = 256, power-of-two columns through Bluestein (M = 128)
    (30, 1000, 2, "f32"),      # rows M = 2048 (three-pass), columns M = 64
    (998, 34, 2, "u16"),       # rows M = 128, columns M = 2048
    (250, 250, 3, "f32"),      # M = 512
    (512, 600, 2, "u16"),      # columns of a power-of-two side at M = 1024
    (600, 800, 3, "u16"),      # the camera shape: M = 2048 both ways
    (1000, 1022, 2, "u16"),
    (480, 640, 2, "f32"),      # mixed-radix sides (P T = 15 32, 20 32)
    (720, 960, 2, "u16"),      # (24 30, 30 32)
    (800, 600, 2, "f32"),      # (25 32 columns, 24 25 rows)
    (600, 512, 2, "u16"),      # mixed columns beside power-of-two rows
    (64, 960, 3, "f32"),       # mixed rows beside Bluestein columns (M = 128)
    (384, 768, 2, "u16"),      # (12 32, 24 32)
    (540, 900, 2, "f32"),      # (18 30, 30 30)
    (2048, 2048, 2, "u16"),    # 2048-pixel sides: the 2048-point transform without the chirp
    (2048, 64, 2, "f32"),
    (64, 2048, 3, "u16"),
    (600, 2048, 2, "u16"),
    (1080, 1280, 2, "u16"),    # (27 40 columns, 32 40 rows)
    (1200, 1024, 2, "f32"),    # (30 40) columns beside power-of-two rows
    (2048, 1280, 2, "u16"),    # 2048-point columns beside mixed rows
    (1280, 1022, 2, "f32"),    # Bluestein rows (M = 2048) beside mixed columns
    (1080, 1920, 2, "u16"),    # full HD: (27 40 columns, 40 48 rows)
    (1920, 1080, 2, "f32"),    # and turned: (40 48 columns, 27 40 rows)
    (1536, 1536, 2, "u16"),    # (32 48)
    (1600, 2000, 2, "f32"),    # (32 50 columns, 40 50 rows)
    (2048, 1440, 2, "u16"),    # 2048-point columns beside (30 48) rows
])
def test_spatial_fft_non_power_of_two_matches_oracle_dft(H, W, N, dtype):
    import torch
    frames = _frames(N, H, W, dtype, seed=H + 3 * W + N)
    plan = ddm.Plan(H, W, N, dtype=dtype)
    spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device="cuda")
    plan.spatial_fft(to_device(frames), spec)
    torch.cuda.synchronize()
    s = spec.cpu().numpy().view(np.complex64).reshape(N, plan.n_q).astype(np.complex128)
    F = storage_to_plane(s, H, W)
    diff = frames.astype(np.float64) - frames[0].astype(np.float64)[None]
    ref = oracle.dft2(diff, oracle.half_plane_columns(W))
    for t in range(1, N):
        scale = max(np.max(np.abs(ref[t])), 1e-30)
        err = np.max(np.abs(F[t] - ref[t])) / scale
        assert err <= 1e-5, (t, err)
    assert np.all(np.abs(F[0]) == 0)          # frame 0 minus itself


def test_spatial_fft_non_power_of_two_without_reference_subtraction():
    import torch
    H, W, N = 24, 40, 2
    frames = _frames(N, H, W, "f32", seed=5)
    plan = ddm.Plan(H, W, N, dtype="f32", subtract_ref=0)
    spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device="cuda")
    plan.spatial_fft(to_device(frames), spec)
    torch.cuda.synchronize()
    s = spec.cpu().numpy().view(np.complex64).reshape(N, plan.n_q).astype(np.complex128)
    F = storage_to_plane(s, H, W)
    ref = oracle.dft2(frames.astype(np.float64), oracle.half_plane_columns(W))
    for t in range(N):
        assert np.max(np.abs(F[t] - ref[t])) / np.max(np.abs(ref[t])) <= 1e-5


@pytest.mark.parametrize("H,W,dtype,sub", [
    (600, 800, "u16", 1), (480, 640, "f32", 1), (540, 900, "u16", 0), (384, 1000, "f32", 0),
])
def test_mixed_rows_unaligned_frames_match_aligned(H, W, dtype, sub):
    """The row kernels stage uint16 rows by bulk copies when the frames are 16-byte aligned
    (and a row is a multiple of 16 bytes), four pixels per load when the frames pointer is
    aligned to four pixels, and one pixel per load otherwise; frames one and four elements
    past an aligned allocation take the other paths.  All do the same arithmetic, so their
    spectra agree bit for bit, and all match the oracle's DFT."""
    import torch
    N = 3
    frames = _frames(N, H, W, dtype, seed=W + 7 * sub)
    plan = ddm.Plan(H, W, N, dtype=dtype, subtract_ref=sub)
    inputs = [to_device(frames)]
    # uint16: bulk (16-byte aligned), four-pixel (8-byte aligned) and one-pixel staging;
    # float32: four-pixel (16-byte aligned) and one-pixel staging
    for shift in ((1, 4) if dtype == "u16" else (1,)):
        host = np.empty(frames.size + shift, dtype=frames.dtype)
        host[shift:] = frames.ravel()
        shifted = to_device(host)[shift:]
        align = 4 * shifted.element_size() if shift == 1 else 16
        assert shifted.data_ptr() % align != 0
        inputs.append(shifted)
    specs = []
    for f in inputs:
        spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device="cuda")
        plan.spatial_fft(f, spec)
        specs.append(spec)
    torch.cuda.synchronize()
    for sp in specs[1:]:
        assert torch.equal(specs[0], sp)
    s = specs[0].cpu().numpy().view(np.complex64).reshape(N, plan.n_q).astype(np.complex128)
    F = storage_to_plane(s, H, W)
    x = frames.astype(np.float64)
    if sub:
        x = x - x[0][None]
    ref = oracle.dft2(x, oracle.half_plane_columns(W))
    for t in range(1 if sub else 0, N):
        assert np.max(np.abs(F[t] - ref[t])) / np.max(np.abs(ref[t])) <= 1e-5, t


@pytest.mark.parametrize("H,W,N,dtype", [
    (8, 12, 3, "f32"), (6, 10, 1, "u16"), (12, 8, 50, "u16"),
    (18, 22, 40, "f32"), (48, 80, 64, "u16"), (100, 64, 33, "u16"), (64, 100, 20, "f32"),
    (250, 250, 100, "f32"), (600, 800, 16, "u16"), (2048, 64, 40, "u16"), (16, 2048, 33, "f32"),
    (480, 640, 12, "f32"), (720, 96, 30, "u16"), (1080, 1280, 6, "u16"), (1080, 1920, 4, "u16"),
])
def test_structure_function_non_power_of_two_matches_oracle(H, W, N, dtype):
    frames = _frames(N, H, W, dtype, seed=11 * N + H)
    D, _, _ = gpu_structure_function(frames)
    D_ref, s_q = oracle.structure_function(frames)
    assert np.all(D[..., 0] == 0)
    assert oracle.scaled_error(D, D_ref, s_q) <= TOL


@pytest.mark.parametrize("H,W,N,nb", [(48, 80, 5, 30), (600, 800, 4, 500), (100, 64, 3, 40)])
def test_radial_average_non_power_of_two_matches_oracle(H, W, N, nb):
    import torch
    rng = np.random.Generator(np.random.PCG64(H * W + nb))
    R = rng.random((H, W, N)) * 10 + 1
    Dfull = 0.5 * (R + R[(-np.arange(H)) % H][:, (-np.arange(W)) % W])
    half = np.ascontiguousarray(Dfull[:, : W // 2 + 1, :]).astype(np.float32)
    Dr_ref, cnt_ref = oracle.radial_average(Dfull.astype(np.float32).astype(np.float64), nb)
    plan = ddm.Plan(H, W, N, dtype="f32", n_bins=nb)
    Dr = torch.empty(nb * N, dtype=torch.float32, device="cuda")
    cnt = torch.empty(nb, dtype=torch.int32, device="cuda")
    plan.azimuthal_average(torch.from_numpy(half.ravel()).cuda(), Dr, cnt)
    torch.cuda.synchronize()
    assert np.array_equal(cnt.cpu().numpy(), cnt_ref)
    np.testing.assert_allclose(Dr.cpu().numpy().reshape(nb, N), Dr_ref, rtol=1e-5, atol=0)


def test_two_species_600x800x3000_sampled_columns():
    """The camera workload at full size (600 x 800 uint16, N = 3000: a 4096-point time
    transform), two Brownian species and an illumination drift; every ky and every lag of a
    sample of kx columns against the oracle."""
    frames = synth.blobs_two_species_600x800(seed=0)
    D, _, _ = gpu_structure_function(frames)
    cols = [0, 1, 2, 5, 133, 267, 399, 400]
    D_ref, s_q = oracle.structure_function(frames, kx_sel=cols)
    err = oracle.scaled_error(D[:, cols, :], D_ref, s_q)
    assert err <= TOL, err
