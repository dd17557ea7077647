"""Pins of the FP64 fit oracle (oracle/fit.py) against independent facts."""
import math

import numpy as np
import pytest

from oracle import fit as F


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_log_lags_geometric_from_1_to_N_minus_1():
    lam = F.log_lags(1024)
    assert lam.size == 64
    assert lam[0] == pytest.approx(1.0, abs=1e-15)
    assert lam[-1] == pytest.approx(1023.0, rel=1e-13)
    ratios = lam[1:] / lam[:-1]
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-12)


def test_sampling_is_exact_for_linear_curves():
    N = 300
    m = np.arange(N, dtype=np.float64)
    D = np.stack([3.0 * m + 2.0, -0.5 * m])
    y = F.sample_log_lags(D)
    lam = F.log_lags(N)
    np.testing.assert_allclose(y[0], 3.0 * lam + 2.0, rtol=1e-13)
    np.testing.assert_allclose(y[1], -0.5 * lam, rtol=1e-13)


def test_gelu_is_x_times_normal_cdf_and_grad_matches_fd():
    from scipy.stats import norm
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(F.gelu(z), z * norm.cdf(z), atol=1e-15)
    h = 1e-6
    fd = (F.gelu(z + h) - F.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(F.gelu_grad(z), fd, atol=1e-8)


def test_bf16_rounding_matches_torch():
    import torch
    x = np.concatenate([_rng(1).standard_normal(1000).astype(np.float32),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(F.bf16_round(x), ref)


def test_adam_two_steps_by_hand():
    w, g = np.array([1.0]), np.array([0.5])
    m = v = np.zeros(1)
    w1, m1, v1 = F.adam_step(w, g, m, v, 1, lr=0.1)
    # m = 0.05, v = 0.00025, mhat = 0.5, vhat = 0.25 -> w = 1 - 0.1 * 0.5 / (0.5 + 1e-8)
    assert w1[0] == pytest.approx(1 - 0.1 * 0.5 / (0.5 + 1e-8), rel=1e-14)
    w2, _, _ = F.adam_step(w1, np.array([-1.0]), m1, v1, 2, lr=0.1)
    m2 = 0.9 * 0.05 - 0.1
    v2 = 0.999 * 0.00025 + 0.001
    expect = w1[0] - 0.1 * (m2 / (1 - 0.81)) / (math.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    assert w2[0] == pytest.approx(expect, rel=1e-13)


def test_mlp_gradient_matches_central_differences():
    rng = _rng(3)
    w = rng.standard_normal(F.N_PARAMS) * 0.1
    x = rng.standard_normal((5, 64))
    t = rng.standard_normal((5, 4))
    loss, g = F.loss_and_grad(w, x, t, bf16=False)
    idx = rng.choice(F.N_PARAMS, 200, replace=False)
    h = 1e-6
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (F.loss_and_grad(wp, x, t, bf16=False)[0] - F.loss_and_grad(wm, x, t, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_mlp_parameter_count_and_layout():
    assert F.N_PARAMS == 41860
    layers = F.unpack(np.arange(F.N_PARAMS, dtype=np.float64))
    assert [W.shape for W, _ in layers] == [(128, 64), (128, 128), (128, 128), (4, 128)]
    assert layers[0][1][0] == 128 * 64            # b1 follows W1


@pytest.mark.parametrize("A,tau,beta,B", [(1.0, 20.0, 1.0, 0.1), (5e8, 3.0, 0.7, 1e7),
                                          (2.0, 300.0, 0.9, 0.0), (1.0, 1.5, 1.2, 0.5)])
def test_lm_recovers_noiseless_parameters(A, tau, beta, B):
    lam = F.log_lags(1024)
    y = F.model(lam, A, tau, beta, B)
    p0 = F.heuristic_seed(lam, y)
    p, cost, it, flags = F.lm_fit(lam, y, p0)
    phys = F.params_to_physical(p)
    np.testing.assert_allclose(phys, [A, tau, beta, B], rtol=1e-6, atol=1e-9 * A)
    assert flags & F.FLAG_CONVERGED and it < 100


def test_lm_cost_never_increases_and_seed_is_in_range():
    lam = F.log_lags(512)
    rng = _rng(9)
    for _ in range(20):
        A, tau, beta, B = 10 ** rng.uniform(-1, 3), 10 ** rng.uniform(0, 2.5), rng.uniform(0.5, 1.1), 0.0
        y = F.model(lam, A, tau, beta, B) * (1 + 0.01 * rng.standard_normal(lam.size))
        p0 = F.heuristic_seed(lam, y)
        assert 0.2 * tau <= math.exp(p0[2]) <= 5 * tau or tau > 300
        f0 = F.model(lam, p0[0], math.exp(p0[2]), p0[3], p0[1])
        c0 = float(np.sum((f0 - y) ** 2))
        _, cost, _, _ = F.lm_fit(lam, y, p0)
        assert cost <= c0
