"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: closed forms, exact
integer identities, a library FFT as a special case of the DFT definition, and brute
force that differences the images *before* transforming them (Eq. 1 as printed:
the transform of a difference) while the oracle transforms first and differences after.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------- DFT pins
def test_dft_matches_library_fft2():
    """The unnormalised 2D DFT equals numpy's FFT (an independent implementation)."""
    a = _rng(1).standard_normal((3, 12, 10))
    F = oracle.dft2(a)
    ref = np.fft.fft2(a)
    assert np.max(np.abs(F - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dft_column_selection_and_uint16():
    a = _rng(2).integers(0, 4096, size=(2, 8, 16), dtype=np.uint16)
    cols = [0, 3, 8, 15]
    F = oracle.dft2(a, cols)
    ref = np.fft.fft2(a.astype(np.float64))[:, :, cols]
    assert np.max(np.abs(F - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dft_parseval_and_hermitian():
    a = _rng(3).standard_normal((2, 9, 14))
    F = oracle.dft2(a)
    H, W = 9, 14
    lhs = np.sum(np.abs(F) ** 2, axis=(1, 2))
    rhs = H * W * np.sum(a ** 2, axis=(1, 2))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)
    # F(-q) = conj F(q) for real frames
    neg = F[:, (-np.arange(H)) % H][:, :, (-np.arange(W)) % W]
    assert np.max(np.abs(neg - np.conj(F))) <= 1e-11 * np.max(np.abs(F))


def test_dft_delta_and_cosine():
    H, W = 8, 12
    delta = np.zeros((1, H, W))
    delta[0, 0, 0] = 3.0
    np.testing.assert_allclose(oracle.dft2(delta)[0], 3.0 + 0j, atol=1e-14)
    y, x = np.mgrid[0:H, 0:W]
    ky, kx = 2, 5
    cosine = np.cos(2 * np.pi * (ky * y / H + kx * x / W))[None]
    F = oracle.dft2(cosine)[0]
    expect = np.zeros((H, W), complex)
    expect[ky, kx] = H * W / 2
    expect[-ky % H, -kx % W] = H * W / 2
    assert np.max(np.abs(F - expect)) < 1e-11


# ------------------------------------------------------------- structure-function pins
def _bruteforce_difference_first(frames):
    """Eq. 1 as printed: the DFT of the difference image, squared, averaged over pairs.

    Pure Python sums; only for tiny stacks.
    """
    N, H, W = frames.shape
    D = np.zeros((H, W, N))
    for m in range(1, N):
        for ky, kx in itertools.product(range(H), range(W)):
            acc = 0.0
            for t in range(N - m):
                s = 0j
                for y in range(H):
                    for x in range(W):
                        diff = float(frames[t + m, y, x]) - float(frames[t, y, x])
                        s += diff * complex(math.cos(-2 * math.pi * (ky * y / H + kx * x / W)),
                                            math.sin(-2 * math.pi * (ky * y / H + kx * x / W)))
                acc += abs(s) ** 2
            D[ky, kx, m] = acc / (N - m)
    return D


def test_structure_function_bruteforce_tiny():
    frames = _rng(4).integers(0, 50, size=(6, 3, 4)).astype(np.float64)
    D = oracle.sf_direct(oracle.dft2(frames))
    ref = _bruteforce_difference_first(frames)
    assert np.max(np.abs(D - ref)) <= 1e-10 * np.max(ref)


def test_static_stack_gives_zero():
    frame = _rng(5).integers(0, 4096, size=(1, 8, 8)).astype(np.uint16)
    frames = np.repeat(frame, 9, axis=0)
    D = oracle.sf_direct(oracle.dft2(frames))
    assert np.all(D == 0.0)


def test_d_level_parseval_exact_integers():
    """sum over the full plane of D(q, m) = H W / (N - m) sum_t sum_x (I_{t+m} - I_t)^2."""
    N, H, W = 7, 6, 10
    frames = _rng(6).integers(0, 4096, size=(N, H, W), dtype=np.uint16)
    D = oracle.sf_direct(oracle.dft2(frames))          # [H, W, N]
    I = frames.astype(np.int64)
    for m in range(1, N):
        exact = int(np.sum((I[m:] - I[:-m]) ** 2))     # exact in int64
        rhs = H * W * exact / (N - m)
        assert abs(np.sum(D[:, :, m]) - rhs) <= 1e-12 * rhs
    assert np.all(D[:, :, 0] == 0)


def test_periodic_translation_closed_form():
    """I_t = roll(I_0, v t): D = 2 |F_0(q)|^2 (1 - cos(2 pi (ky vy / H + kx vx / W) m))."""
    N, H, W = 8, 8, 12
    vy, vx = 1, 2
    base = _rng(7).standard_normal((H, W))
    frames = np.stack([np.roll(base, (vy * t, vx * t), axis=(0, 1)) for t in range(N)])
    D = oracle.sf_direct(oracle.dft2(frames))
    F0 = np.fft.fft2(base)
    ky = np.arange(H)[:, None]
    kx = np.arange(W)[None, :]
    for m in range(N):
        phase = 2 * np.pi * (ky * vy / H + kx * vx / W) * m
        expect = 2 * np.abs(F0) ** 2 * (1 - np.cos(phase))
        assert np.max(np.abs(D[:, :, m] - expect)) <= 1e-10 * np.max(np.abs(F0) ** 2)


def test_lag_zero_is_zero_and_lag_range():
    frames = _rng(8).standard_normal((5, 4, 4))
    D = oracle.sf_direct(oracle.dft2(frames))
    assert D.shape == (4, 4, 5)
    assert np.all(D[..., 0] == 0)


def test_single_frame():
    frames = _rng(9).standard_normal((1, 4, 6))
    D = oracle.sf_direct(oracle.dft2(frames))
    assert D.shape == (4, 6, 1) and np.all(D == 0)


# --------------------------------------------------------- App. B route vs Eq. 1 route
@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 13, 16])
def test_wk_route_equals_direct(N):
    """Eq. B1-B4: the padded-FFT-in-time route reproduces Eq. 1 to rounding."""
    frames = _rng(10 + N).standard_normal((N, 4, 6)) + 3.0
    F = oracle.dft2(frames)
    D1 = oracle.sf_direct(F)
    D2 = oracle.sf_wk(F)                       # M = 2^(ceil(log2 N) + 1)
    s = np.max(np.abs(F) ** 2)
    assert np.max(np.abs(D1 - D2)) <= 1e-11 * s


@pytest.mark.parametrize("M_of", [lambda N: 2 * N - 1, lambda N: 2 * N, lambda N: 3 * N])
def test_wk_route_any_pad_at_least_2n_minus_1(M_of):
    N = 9
    frames = _rng(30).standard_normal((N, 3, 5))
    F = oracle.dft2(frames)
    D1 = oracle.sf_direct(F)
    D2 = oracle.sf_wk(F, M=M_of(N))
    assert np.max(np.abs(D1 - D2)) <= 1e-11 * np.max(np.abs(F) ** 2)


def test_wk_route_without_padding_is_wrong():
    """Without the zero-padding of Eq. B4 the circular wrap corrupts d_c (App. B)."""
    N = 8
    frames = _rng(31).standard_normal((N, 3, 5))
    F = oracle.dft2(frames)
    D1 = oracle.sf_direct(F)
    D2 = oracle.sf_wk(F, M=N)
    assert np.max(np.abs(D1 - D2)) > 1e-2 * np.max(np.abs(D1))


def test_wk_constant_sequence():
    """A constant time sequence c: D = 0 on both routes."""
    frames = np.repeat(_rng(32).standard_normal((1, 4, 4)), 6, axis=0)
    F = oracle.dft2(frames)
    s = np.max(np.abs(F) ** 2)
    assert np.max(np.abs(oracle.sf_wk(F))) <= 1e-11 * s
    assert np.all(oracle.sf_direct(F) == 0)


def test_pad_length_rule():
    """Eq. B4: log2 N2 = ceil(log2 N) + 1."""
    assert [oracle.pad_length_paper(n) for n in (1, 2, 3, 4, 5, 1000, 1024, 1025, 3000)] == \
        [2, 4, 8, 8, 16, 2048, 2048, 4096, 8192]


# ------------------------------------------------------------------- OU statistical pin
def test_ou_closed_form_statistics():
    """E[D(q, m)] = H W (2 S(q) (1 - exp(-D0 q^2 m)) + 2 sigma^2) for the OU generator.

    Averaged over the independent modes of the open half plane (0 < kx < W/2) and
    four seeds; the mean ratio D / E[D] must be 1 within 5 standard errors.
    """
    H = W = 32
    N = 96
    D0, width, sigma = 0.5, 0.3, 0.05
    cols = list(range(1, W // 2))
    ratios = {m: [] for m in (1, 3, 10, 30)}
    qmag = synth.q_magnitude(H, W)[:, cols]
    S = np.exp(-qmag ** 2 / (2 * width ** 2))
    for seed in range(4):
        frames = synth.ou_stack(H, W, N, D0, synth.gaussian_spectrum(width), sigma, seed,
                                dtype=np.float64)
        D = oracle.sf_direct(oracle.dft2(frames, cols))
        for m in ratios:
            expect = H * W * (2 * S * (1 - np.exp(-D0 * qmag ** 2 * m)) + 2 * sigma ** 2)
            ratios[m].append((D[:, :, m] / expect).ravel())
    for m, r in ratios.items():
        r = np.concatenate(r)
        se = np.std(r) / math.sqrt(r.size)
        assert abs(np.mean(r) - 1.0) < 5 * se, (m, np.mean(r), se)


def test_plateau_scale_matches_ou_plateau():
    """s_q = 2 var_t F -> 2 H W (S + sigma^2) for the OU generator (statistical)."""
    H = W = 32
    N = 256
    frames = synth.ou_stack(H, W, N, 2.0, synth.gaussian_spectrum(0.5), 0.1, 3, np.float64)
    cols = list(range(1, W // 2))
    s = oracle.plateau_scale(oracle.dft2(frames, cols))
    q = synth.q_magnitude(H, W)[:, cols]
    expect = 2 * H * W * (np.exp(-q ** 2 / 0.5) + 0.01)
    r = (s / expect).ravel()
    assert abs(np.mean(r) - 1) < 5 * np.std(r) / math.sqrt(r.size) + 0.02


# ------------------------------------------------------------------------ radial pins
@pytest.mark.parametrize("H,W,nb", [(64, 64, 46), (16, 24, 7), (9, 15, 5), (512, 512, 362)])
def test_radial_bins_bruteforce(H, W, nb):
    b = oracle.radial_bins(H, W, nb)
    qc = math.pi * math.sqrt(2.0)
    checked = 0
    for ky in range(0, H, max(1, H // 40)):
        for kx in range(0, W, max(1, W // 40)):
            ys = ky - H if ky > H // 2 else ky
            xs = kx - W if kx > W // 2 else kx
            q = 2 * math.pi * math.sqrt((ys / H) ** 2 + (xs / W) ** 2)
            v = q * nb / qc
            if abs(v - round(v)) < 1e-9:
                continue            # on a bin edge: only the exact evaluation decides
            assert b[ky, kx] == min(int(math.floor(v)), nb - 1)
            checked += 1
    assert checked > 0
    counts = np.bincount(b.ravel(), minlength=nb)
    assert counts.sum() == H * W
    # symmetric under q -> -q
    assert np.array_equal(b, b[(-np.arange(H)) % H][:, (-np.arange(W)) % W])


def test_radial_average_constant_and_counts():
    H, W, N, nb = 12, 10, 4, 6
    D = np.full((H, W, N), 2.5)
    Dr, counts = oracle.radial_average(D, nb)
    assert counts.sum() == H * W
    assert np.all(Dr[counts > 0] == 2.5) and np.all(Dr[counts == 0] == 0)
    # a D that equals the bin index averages to the bin index
    b = oracle.radial_bins(H, W, nb)
    Dr2, _ = oracle.radial_average(np.repeat(b[:, :, None].astype(float), N, axis=2), nb)
    nz = counts > 0
    np.testing.assert_array_equal(Dr2[nz], np.repeat(np.arange(nb)[nz, None], N, axis=1))


def test_scaled_error_metric():
    s = np.array([1.0, 4.0])
    D = np.zeros((2, 3))
    D2 = D.copy()
    D2[1, 2] = 2e-4
    assert oracle.scaled_error(D2, D, s) == pytest.approx(5e-5)


def test_scaled_error_static_modes_on_the_global_scale():
    """A mode whose plateau is below 1e-12 of the largest is static: it passes when
    |D| <= 1e-6 of the largest plateau, whatever the reference says, and enters the metric
    scaled so that the 1e-4 bar means exactly that."""
    s = np.array([2.0, 1e-13, 0.5])
    D_ref = np.zeros((3, 4))
    D = D_ref.copy()
    D[1, 3] = 1e-6 * 2.0                     # exactly the static bound
    assert oracle.scaled_error(D, D_ref, s) == pytest.approx(oracle.TOLERANCE)
    D[1, 3] = 3e-6 * 2.0
    assert oracle.scaled_error(D, D_ref, s) == pytest.approx(3 * oracle.TOLERANCE)
    D[1, 3] = 0.0
    D_ref[1, 1] = 5.0                        # a static mode's reference plays no part
    assert oracle.scaled_error(D, D_ref, s) == 0.0
    D[2, 0] = 1e-5                           # an ordinary mode: relative to its own plateau
    assert oracle.scaled_error(D, D_ref, s) == pytest.approx(2e-5)
    # a plateau of exactly 1e-12 of the largest is not static
    assert oracle.scaled_error(np.array([[0.0, 0.0], [0.0, 1e-16]]), np.zeros((2, 2)),
                               np.array([1.0, 1e-12])) == pytest.approx(1e-4)


def test_ou_torch_generator_closed_form_statistics():
    """The torch rendering of the OU law (used for the 1024x1024x4096 precision sweep, run
    here on the CPU) obeys the same closed form E[D] = H W (2 S (1 - e^{-D0 q^2 m}) +
    2 sigma^2) within 5 standard errors, and its log-uniform D0 lies in [0.01, 1]."""
    H = W = 32
    N = 96
    D0, width, sigma = 0.5, 0.3, 0.05
    cols = list(range(1, W // 2))
    ratios = {m: [] for m in (1, 3, 10, 30)}
    qmag = synth.q_magnitude(H, W)[:, cols]
    S = np.exp(-qmag ** 2 / (2 * width ** 2))
    for seed in range(4):
        frames = synth.ou_stack_torch(H, W, N, D0, synth.gaussian_spectrum(width), sigma, seed,
                                      device="cpu").numpy()
        D = oracle.sf_direct(oracle.dft2(frames, cols))
        for m in ratios:
            expect = H * W * (2 * S * (1 - np.exp(-D0 * qmag ** 2 * m)) + 2 * sigma ** 2)
            ratios[m].append((D[:, :, m] / expect).ravel())
    for m, r in ratios.items():
        r = np.concatenate(r)
        se = np.std(r) / math.sqrt(r.size)
        assert abs(np.mean(r) - 1.0) < 5 * se, (m, np.mean(r), se)
    rng = np.random.Generator(np.random.PCG64(1))
    d0s = [synth.log_uniform_d0()(rng) for _ in range(200)]
    assert 0.01 <= min(d0s) and max(d0s) <= 1.0 and min(d0s) < 0.03 and max(d0s) > 0.3
