"""Fit stage on the GPU (LM kernel, MLP kernels) vs the FP64 fit oracle, and what the
trained network gains over the heuristic seed."""
import math

import numpy as np
import pytest

import paper_2012_05695_b300 as ddm
import synth
from oracle import fit as F
from paper_2012_05695_b300 import _binding as B

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _fit(plan, D, mode, mlp=None):
    import torch
    n = D.shape[0]
    params = torch.empty(n * 4, device="cuda")
    cost = torch.empty(n, device="cuda")
    iters = torch.empty(n, dtype=torch.int32, device="cuda")
    flags = torch.empty(n, dtype=torch.int32, device="cuda")
    plan.fit(_cuda(D.reshape(-1)), n, mode, mlp, params, cost, iters, flags)
    torch.cuda.synchronize()
    return (params.cpu().numpy().reshape(n, 4).astype(np.float64), cost.cpu().numpy().astype(np.float64),
            iters.cpu().numpy(), flags.cpu().numpy())


def test_features_match_oracle():
    import torch
    N, n = 777, 37
    D, _ = synth.stretched_exp_curves(n, N, 1)
    plan = ddm.Plan(8, 8, N, dtype="f32")
    x = torch.empty(n * 64, device="cuda")
    p8 = torch.empty(n, device="cuda")
    plan.fit_features(_cuda(D.reshape(-1)), n, x, p8)
    torch.cuda.synchronize()
    y = F.sample_log_lags(D.astype(np.float64))
    xr, pr = F.features(y)
    np.testing.assert_allclose(p8.cpu().numpy(), pr, rtol=2e-6)
    np.testing.assert_allclose(x.cpu().numpy().reshape(n, 64), xr, rtol=2e-6, atol=1e-7)


def test_lm_matches_oracle_on_noiseless_curves():
    """Noiseless curves at integer lags; both sides fit the same log-lag samples (linear
    interpolation between integer lags), so the FP32 kernel must land on the FP64
    oracle's optimum."""
    N = 1024
    lam_int = np.arange(N, dtype=np.float64)
    truth = np.array([[1.0, 20.0, 1.0, 0.1], [5e8, 3.0, 0.7, 1e7], [2.0, 150.0, 0.9, 0.0],
                      [1e4, 1.5, 1.1, 5e3], [300.0, 60.0, 0.6, 30.0]])
    D = np.stack([F.model(np.maximum(lam_int, 1e-9), *t) for t in truth]).astype(np.float32)
    D[:, 0] = 0
    plan = ddm.Plan(8, 8, N, dtype="f32")
    params, cost, iters, flags = _fit(plan, D, B.DDM_FIT_LM)
    assert np.all(flags & B.DDM_FIT_CONVERGED), flags
    lam = F.log_lags(N)
    y = F.sample_log_lags(D.astype(np.float64))
    ref = np.stack([F.params_to_physical(F.lm_fit(lam, y[c], F.heuristic_seed(lam, y[c]))[0])
                    for c in range(len(truth))])
    err = np.abs(params - ref) / (np.abs(ref) + 1e-3 * ref[:, :1])
    assert np.max(err) <= 2e-3, (params, ref, err)


def test_lm_matches_oracle_on_noisy_curves():
    """Same curves, same algorithm, per curve: the FP32 kernel's final cost is within 1e-4
    of the FP64 oracle's optimum, and each of its parameters (A, B, ln tau, beta) sits within
    5 % of that parameter's standard error at the oracle's optimum (sigma^2 (J^T J)^-1,
    sigma^2 = cost / (64 - 4)): the FP32 arithmetic moves the fit by far less than the
    data's own noise determines it."""
    N, n = 1024, 64
    D, labels = synth.stretched_exp_curves(n, N, 2)
    plan = ddm.Plan(8, 8, N, dtype="f32")
    params, cost, iters, flags = _fit(plan, D, B.DDM_FIT_LM)
    assert np.all(flags & B.DDM_FIT_CONVERGED), flags
    lam = F.log_lags(N)
    y = F.sample_log_lags(D.astype(np.float64))
    for c in range(n):
        p, co, it, fl = F.lm_fit(lam, y[c], F.heuristic_seed(lam, y[c]))
        assert fl & F.FLAG_CONVERGED
        assert cost[c] <= co * (1 + 1e-4) + 1e-12 * y[c, -1] ** 2, (c, cost[c], co)
        _, J = F._model_and_jac(lam, p)
        se = np.sqrt(np.diag(np.linalg.inv(J.T @ J)) * co / (F.N_LAGS - 4))
        A, tau, beta, Bb = params[c]
        got = np.array([A, Bb, math.log(tau), beta])
        dev = np.abs(got - p)
        assert np.all(dev <= 0.05 * se + 1e-5 * np.abs(p)), (c, got, p, se)


def test_mlp_forward_matches_oracle():
    import torch
    w = synth.mlp_init(5)
    rng = np.random.Generator(np.random.PCG64(5))
    Bn = 77
    x = rng.uniform(0, 1.2, (Bn, 64)).astype(np.float32)
    mlp = ddm.MLP(128)
    mlp.set_weights(w)
    o = torch.empty(Bn * 4, device="cuda")
    mlp.forward(_cuda(x.reshape(-1)), Bn, o)
    torch.cuda.synchronize()
    ref, _ = F.mlp_forward(w.astype(np.float64), x.astype(np.float64), bf16=True)
    got = o.cpu().numpy().reshape(Bn, 4)
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))
    np.testing.assert_array_equal(mlp.get_weights(), w)


@pytest.mark.parametrize("Bn", [1, 127, 128, 129, 300, 4096])
def test_mlp_forward_tensor_cores_ragged_batches(Bn):
    """The forward runs 128 samples per CTA on the tensor cores: batches below, at and just
    past one CTA's tile, and the training batch, against the oracle (FP32 activations)."""
    import torch
    w = synth.mlp_init(8)
    rng = np.random.Generator(np.random.PCG64(Bn))
    x = rng.uniform(0, 1.2, (Bn, 64)).astype(np.float32)
    mlp = ddm.MLP(4096)
    mlp.set_weights(w)
    o = torch.full((Bn * 4,), float("nan"), device="cuda")
    mlp.forward(_cuda(x.reshape(-1)), Bn, o)
    assert mlp.last_device_status() == B.DDM_OK
    ref, _ = F.mlp_forward(w.astype(np.float64), x.astype(np.float64), bf16=True)
    got = o.cpu().numpy().reshape(Bn, 4)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_mlp_forward_unaligned_pointers_and_trained_weights():
    """Inputs and outputs one float past an aligned allocation; weights changed by Adam steps
    (the tensor-core operand images are rebuilt with every step)."""
    import torch
    w = synth.mlp_init(9)
    rng = np.random.Generator(np.random.PCG64(9))
    Bn = 200
    x = rng.uniform(0, 1.2, (Bn, 64)).astype(np.float32)
    t = rng.uniform(0, 1, (Bn, 4)).astype(np.float32)
    mlp = ddm.MLP(Bn)
    mlp.set_weights(w)
    xd, td = _cuda(x.reshape(-1)), _cuda(t.reshape(-1))
    for _ in range(3):
        mlp.train_step(xd, td, Bn, 1e-2)
    wk = mlp.get_weights().astype(np.float64)
    assert np.max(np.abs(wk - w)) > 1e-3
    xb = torch.empty(Bn * 64 + 1, device="cuda")
    xb[1:] = xd
    ob = torch.full((Bn * 4 + 1,), float("nan"), device="cuda")
    mlp.forward(xb[1:], Bn, ob[1:])
    assert mlp.last_device_status() == B.DDM_OK
    ref, _ = F.mlp_forward(wk, x.astype(np.float64), bf16=True)
    got = ob[1:].cpu().numpy().reshape(Bn, 4)
    assert np.isnan(ob[0].item())
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_mlp_forward_agrees_with_training_forward():
    """The loss that the training kernel (CUDA cores) computes equals the loss of the
    tensor-core forward's outputs."""
    import torch
    w = synth.mlp_init(10)
    rng = np.random.Generator(np.random.PCG64(10))
    Bn = 512
    x = rng.uniform(0, 1.2, (Bn, 64)).astype(np.float32)
    t = np.stack([rng.normal(0, 1, Bn), rng.uniform(0, 6, Bn), rng.uniform(0.5, 1.1, Bn),
                  rng.uniform(0, 0.5, Bn)], axis=1).astype(np.float32)
    mlp = ddm.MLP(Bn)
    mlp.set_weights(w)
    g = torch.empty(B.DDM_MLP_PARAMS, device="cuda")
    loss = torch.empty(1, device="cuda")
    mlp.grad(_cuda(x.reshape(-1)), _cuda(t.reshape(-1)), Bn, g, loss)
    o = torch.empty(Bn * 4, device="cuda")
    mlp.forward(_cuda(x.reshape(-1)), Bn, o)
    oo = o.cpu().numpy().reshape(Bn, 4).astype(np.float64)
    sig = 1.0 / (1.0 + np.exp(-oo[:, 2]))
    yhat = np.stack([oo[:, 0], oo[:, 1], 0.3 + 0.9 * sig, oo[:, 3]], axis=1)
    l_tc = float(np.sum((yhat - t) ** 2) / Bn)
    assert float(loss.item()) == pytest.approx(l_tc, rel=1e-5)


def test_mlp_gradient_matches_oracle():
    import torch
    w = synth.mlp_init(6)
    rng = np.random.Generator(np.random.PCG64(6))
    Bn = 100                                   # 4 chunks, the last one ragged
    x = rng.uniform(0, 1.2, (Bn, 64)).astype(np.float32)
    t = np.stack([rng.normal(0, 1, Bn), rng.uniform(0, 6, Bn), rng.uniform(0.5, 1.1, Bn),
                  rng.uniform(0, 0.5, Bn)], axis=1).astype(np.float32)
    mlp = ddm.MLP(256)
    mlp.set_weights(w)
    g = torch.empty(B.DDM_MLP_PARAMS, device="cuda")
    loss = torch.empty(1, device="cuda")
    mlp.grad(_cuda(x.reshape(-1)), _cuda(t.reshape(-1)), Bn, g, loss)
    torch.cuda.synchronize()
    lref, gref = F.loss_and_grad(w.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - gref)) <= 1e-4 * np.max(np.abs(gref))


def test_adam_step_matches_oracle():
    import torch
    w = synth.mlp_init(7)
    rng = np.random.Generator(np.random.PCG64(7))
    Bn = 64
    x = rng.uniform(0, 1.2, (Bn, 64)).astype(np.float32)
    t = rng.uniform(0, 1, (Bn, 4)).astype(np.float32)
    mlp = ddm.MLP(Bn)
    mlp.set_weights(w)
    lr = 1e-3
    mlp.train_step(_cuda(x.reshape(-1)), _cuda(t.reshape(-1)), Bn, lr)
    torch.cuda.synchronize()
    w1 = mlp.get_weights().astype(np.float64)
    _, g = F.loss_and_grad(w.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    wr, _, _ = F.adam_step(w.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))     # sign of tiny gradients is rounding noise
    np.testing.assert_allclose(w1[big], wr[big], rtol=0, atol=1e-6)


def test_trained_mlp_seed_gains_over_heuristic_seed():
    """Train on 16k curves with the GPU kernels, then fit 2k held-out curves: LM seeded by
    the network needs fewer iterations than LM from the heuristic seed, at no cost in fit
    quality.  The numbers are printed for the record."""
    import torch
    N = 1024
    Dtr, ltr = synth.stretched_exp_curves(16384, N, 10)
    Dte, lte = synth.stretched_exp_curves(2048, N, 11)
    plan = ddm.Plan(8, 8, N, dtype="f32")
    # features of the training curves on the device, targets from the labels
    x = torch.empty(16384 * 64, device="cuda")
    p8 = torch.empty(16384, device="cuda")
    plan.fit_features(_cuda(Dtr.reshape(-1)), 16384, x, p8)
    torch.cuda.synchronize()
    p8h = p8.cpu().numpy().astype(np.float64)
    tgt = F.targets(ltr, p8h).astype(np.float32)
    t_dev = _cuda(tgt.reshape(-1))
    mlp = ddm.MLP(4096)
    mlp.set_weights(synth.mlp_init(0))
    loss = torch.empty(1, device="cuda")
    losses = []
    rng = np.random.Generator(np.random.PCG64(0))
    for step in range(3000):
        b = int(rng.integers(0, 4))
        lr = 2e-3 if step < 2000 else 5e-4
        mlp.train_step(x[b * 4096 * 64:(b + 1) * 4096 * 64], t_dev[b * 4096 * 4:(b + 1) * 4096 * 4],
                       4096, lr, loss)
        if step % 500 == 0 or step == 2999:
            losses.append(float(loss.item()))
    assert losses[-1] < 0.2 * losses[0], losses
    pl, cl, il, fl = _fit(plan, Dte, B.DDM_FIT_LM)
    pm, cm, im, fm = _fit(plan, Dte, B.DDM_FIT_MLP_LM, mlp)
    ok_l = (fl & B.DDM_FIT_CONVERGED) > 0
    ok_m = (fm & B.DDM_FIT_CONVERGED) > 0
    ratio = cm / np.maximum(cl, 1e-30)
    print(f"\ntrain loss {losses[0]:.3f} -> {losses[-1]:.4f}; held-out 2048 curves: "
          f"LM iters mean {il.mean():.2f}, MLP+LM iters mean {im.mean():.2f}; "
          f"converged {ok_l.mean():.4f} vs {ok_m.mean():.4f}; "
          f"MLP accepted without LM {np.mean((fm & B.DDM_FIT_MLP_ACCEPTED) > 0):.3f}; "
          f"cost ratio median {np.median(ratio):.4f}, p99 {np.quantile(ratio, 0.99):.3f}")
    assert im.mean() < 0.7 * il.mean()
    assert ok_m.mean() >= ok_l.mean() - 0.01
    assert np.median(ratio) <= 1.02


def test_seed_network_trained_on_pipeline_curves_gains_on_held_out_stacks():
    """The learned fit stage on this pipeline's own structure functions (the polydisperse
    blob workload, reduced: 60 training and 8 held-out 512x512x1024 stacks, log-normal D0):
    each stack through ddm_structure_function and the radial average, the identifiable
    curves inside the inscribed Nyquist circle labelled by LM, the network trained with the
    library's kernels.  On the held-out stacks' identifiable curves LM seeded by the network
    needs fewer iterations than LM from the heuristic seed; where LM ran it reaches plain
    LM's final cost, and curves that kept the network's parameters met the acceptance rule
    (RMS residual <= 1e-2 A, checked here from the returned cost and A); over all their curves
    it needs no more iterations.  The numbers are printed for the record."""
    import torch
    from paper_2012_05695_b300 import seed_training as st
    H = W = 512
    N, nb, n_keep = 1024, 362, 256
    plan = ddm.Plan(H, W, N, dtype="u16", n_bins=nb)
    D = torch.empty(plan.d_rows * N, device="cuda")
    Dr = torch.empty(nb * N, device="cuda")

    def curves(seeds):
        return torch.cat([st.stack_curves(plan, synth.polydisperse_blobs_512x512x1024(sd), n_keep, None, D, Dr)
                          for sd in seeds]).contiguous()

    x, t, keep = st.labelled_features(plan, curves(range(1000, 1060)))
    mlp = ddm.MLP(2048)
    mlp.set_weights(synth.mlp_init(0))
    loss0, loss1 = st.train(mlp, x, t, 3000, 2048, seed=0)
    held = curves(range(2000, 2008))
    res = st.compare(plan, held, mlp)
    ident = res["identifiable"]
    prm, cost, _, flags = st.fit_curves(plan, held, B.DDM_FIT_MLP_LM, mlp)
    acc = (flags & B.DDM_FIT_MLP_ACCEPTED) > 0               # cost and A in the curve's units
    assert np.all(np.sqrt(cost[acc] / 64) <= 1e-2 * np.abs(prm[acc, 0]) * (1 + 1e-5))
    print(f"\nlabelled {int(keep.sum())} of {keep.size}; loss {loss0:.2f} -> {loss1:.4f}; "
          f"held-out all: LM {res['lm_iters_mean']:.2f} vs MLP+LM {res['mlp_lm_iters_mean']:.2f} iters; "
          f"identifiable ({ident['curves']}): {ident['lm_iters_mean']:.2f} vs {ident['mlp_lm_iters_mean']:.2f}, "
          f"LM fallback {ident['lm_fallback_rate']:.3f}, LM-run cost within 1e-3 "
          f"{ident['lm_run_cost_within_1e-3']:.4f}, accepted cost ratio median {ident['accepted_cost_ratio_median']}")
    assert loss1 < 0.1 * loss0
    assert ident["curves"] >= 300
    assert ident["mlp_lm_iters_mean"] <= 0.92 * ident["lm_iters_mean"]
    assert ident["lm_run_cost_within_1e-3"] >= 0.99
    assert res["mlp_lm_iters_mean"] <= res["lm_iters_mean"]
    assert res["mlp_lm_converged"] >= res["lm_converged"] - 0.01
    mlp.close()
    plan.close()


def test_training_resumes_from_a_checkpoint_bitwise():
    """Checkpoint after 3 Adam steps, restore into a fresh network, take 4 more steps in each:
    the weights and the Adam state agree bit for bit with the uninterrupted run."""
    import torch
    w = synth.mlp_init(11)
    rng = np.random.Generator(np.random.PCG64(11))
    Bn, lr = 128, 2e-3
    xs = [_cuda(rng.uniform(0, 1.2, Bn * 64).astype(np.float32)) for _ in range(7)]
    ts = [_cuda(rng.uniform(0, 1, Bn * 4).astype(np.float32)) for _ in range(7)]
    a = ddm.MLP(Bn)
    a.set_weights(w)
    for k in range(3):
        a.train_step(xs[k], ts[k], Bn, lr)
    state = a.get_state()
    assert state[-1] == 3.0
    b = ddm.MLP(Bn)
    b.set_state(state)
    for k in range(3, 7):
        a.train_step(xs[k], ts[k], Bn, lr)
        b.train_step(xs[k], ts[k], Bn, lr)
    torch.cuda.synchronize()
    sa, sb = a.get_state(), b.get_state()
    assert sa[-1] == sb[-1] == 7.0
    assert np.array_equal(sa, sb)
    with pytest.raises(ValueError):
        b.set_state(state[:-1])
    bad = state.copy()
    bad[-1] = 2.5                                   # step count must be an integer
    with pytest.raises(ddm.DDMError):
        b.set_state(bad)
