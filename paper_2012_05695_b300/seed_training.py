"""Training and judging the fit's seed network on structure functions this pipeline computes.

The seed network (64 -> 128 -> 128 -> 128 -> 4, the library's ddm_mlp) maps a radial curve
D_r(|q|, lag), sampled at 64 log-spaced lags and divided by its plateau, to the parameters
(A, tau, beta, B) of D = A (1 - exp(-(lag / tau)^beta)) + B; ddm_fit in DDM_FIT_MLP_LM mode
starts Levenberg-Marquardt from it (LM stays the fallback and the judge).  The network is
an amortised fit: its labels are the LM optima of the training curves, so it learns where
LM ends.  Training data are this pipeline's own radial curves of seeded synthetic stacks:
each stack goes through ddm_structure_function and ddm_azimuthal_average, the curves whose
bins lie inside the inscribed Nyquist circle are kept, LM (from its heuristic seed) labels
them, and the network trains on them with the library's own forward, backward and Adam
kernels (ddm_mlp_train_step).

Everything here orchestrates calls of the C ABI through the binding; the only arithmetic on
the host is turning fit labels into the network's regression targets (the inverse of the
head that include/ddm.h documents) and the bookkeeping of the comparison.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B


def head_targets(params, p8):
    """Fit labels (A, tau, beta, B) -> the seed network's regression targets
    (ln(A/p8), ln tau, beta, B/A): the inverse of the head A = p8 e^{o0}, tau = e^{o1},
    B = A o3 that include/ddm.h documents (beta is regressed through its sigmoid)."""
    params = np.asarray(params, dtype=np.float64)
    p8 = np.asarray(p8, dtype=np.float64)
    A, tau, beta, Bv = (params[:, k] for k in range(4))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.stack([np.log(A / p8), np.log(tau), beta, Bv / A], axis=1)


def stack_curves(plan, frames, n_keep, stream=None, D=None, Dr=None):
    """The radial curves of one stack through the library: structure function, radial
    average; returns the first n_keep bins' curves [n_keep][N] (a device tensor)."""
    import torch
    N = plan.N
    if D is None:
        D = torch.empty(plan.d_rows * N, dtype=torch.float32, device=frames.device)
    if Dr is None:
        Dr = torch.empty(plan.n_bins * N, dtype=torch.float32, device=frames.device)
    plan.structure_function(frames, D, stream)
    plan.azimuthal_average(D, Dr, None, stream)
    return Dr.view(plan.n_bins, N)[:n_keep].clone()


def fit_curves(plan, curves, mode, mlp=None, stream=None):
    """ddm_fit on curves [n][N] (device): host arrays params [n][4], cost, iterations, flags."""
    import torch
    n = curves.shape[0]
    dev = curves.device
    prm = torch.empty(n * 4, device=dev)
    cost = torch.empty(n, device=dev)
    its = torch.empty(n, dtype=torch.int32, device=dev)
    flg = torch.empty(n, dtype=torch.int32, device=dev)
    plan.fit(curves.view(-1), n, mode, mlp, prm, cost, its, flg, stream)
    torch.cuda.synchronize()
    return (prm.cpu().numpy().reshape(n, 4).astype(np.float64), cost.cpu().numpy().astype(np.float64),
            its.cpu().numpy(), flg.cpu().numpy())


def identifiable(params, flags, iters, N):
    """Curves whose LM optimum is determined by the data: converged in fewer than 100
    iterations to finite parameters, A > 0, a decay time inside the analysed lags
    (0.5 <= tau <= N) and a noise floor at most 5 times the amplitude (|B/A| <= 5).
    Outside that (the lowest |q|, whose decay lies beyond the last lag; the highest, where
    the Poisson floor drowns the particles' signal) the optimum wanders along a flat valley
    and its parameters are no label to learn."""
    A, tau, Bv = params[:, 0], params[:, 1], params[:, 3]
    ok = ((flags & B.DDM_FIT_CONVERGED) > 0) & (iters < 100) & np.all(np.isfinite(params), axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        ok &= (A > 0) & (tau >= 0.5) & (tau <= N) & (np.abs(Bv / A) <= 5.0)
    return ok


def labelled_features(plan, curves, stream=None):
    """Features x [n][64] and targets t [n][4] (device tensors) of the curves whose LM fit
    from the heuristic seed is identifiable (see identifiable); returns (x, t, kept mask)."""
    import torch
    n = curves.shape[0]
    dev = curves.device
    x = torch.empty(n * 64, device=dev)
    p8 = torch.empty(n, device=dev)
    plan.fit_features(curves.view(-1), n, x, p8, stream)
    params, _, iters, flags = fit_curves(plan, curves, B.DDM_FIT_LM, None, stream)
    p8h = p8.cpu().numpy().astype(np.float64)
    tg = head_targets(params, p8h)
    keep = identifiable(params, flags, iters, plan.N) & (p8h > 0)
    with np.errstate(invalid="ignore"):
        keep &= np.all(np.isfinite(tg), axis=1) & np.all(np.abs(tg) < 50, axis=1)
    idx = torch.from_numpy(np.nonzero(keep)[0]).to(dev)
    xk = x.view(n, 64)[idx].contiguous()
    tk = torch.from_numpy(tg[keep].astype(np.float32)).to(dev).contiguous()
    return xk, tk, keep


def train(mlp, x, t, steps, batch, seed=0, lr=2e-3, lr_late=5e-4, late_frac=0.75, stream=None):
    """Adam steps of the library's training kernel on random batches of (x, t) (device
    tensors [n][64], [n][4], n >= batch); returns the first and last batch losses."""
    import torch
    n = x.shape[0]
    if n < batch:
        raise ValueError(f"{n} training curves < batch {batch}")
    rng = np.random.Generator(np.random.PCG64(seed))
    loss = torch.empty(1, device=x.device)
    xb = torch.empty(batch * 64, device=x.device)
    tb = torch.empty(batch * 4, device=x.device)
    first = None
    for k in range(steps):
        sel = torch.from_numpy(rng.choice(n, size=batch, replace=False)).to(x.device)
        xb.copy_(x[sel].view(-1))
        tb.copy_(t[sel].view(-1))
        mlp.train_step(xb, tb, batch, lr if k < late_frac * steps else lr_late, loss, stream)
        if k == 0:
            first = float(loss.item())
    return first, float(loss.item())


def compare(plan, curves, mlp, stream=None, subsets=True):
    """Plain LM against LM seeded by the network on the same curves: mean iterations,
    converged fraction, the fraction whose network parameters were kept without LM
    (mlp_accepted) and its complement, the LM fallback rate; the fraction where LM started
    from the heuristic seed because it cost less (seed_heuristic) or restarted from it after
    the network's seed diverged (restarted); the final cost of MLP+LM relative to plain LM
    (median, 99th percentile, and the fraction within 1e-3 of plain LM's cost or better),
    separately for the curves where LM ran and for those that kept the network's
    parameters (which stop at the acceptance residual, not at LM's optimum)."""
    pl, cl, il, fl = fit_curves(plan, curves, B.DDM_FIT_LM, None, stream)
    pm, cm, im, fm = fit_curves(plan, curves, B.DDM_FIT_MLP_LM, mlp, stream)
    out = _summary(cl, il, fl, cm, im, fm)
    if subsets:
        # the curves whose plain-LM optimum is identifiable (the network's domain) and the rest
        ok = identifiable(pl, fl, il, plan.N)
        out["identifiable"] = _summary(cl[ok], il[ok], fl[ok], cm[ok], im[ok], fm[ok])
        out["not_identifiable"] = _summary(cl[~ok], il[~ok], fl[~ok], cm[~ok], im[~ok], fm[~ok])
    return out


def _summary(cl, il, fl, cm, im, fm):
    if il.size == 0:
        return {"curves": 0}
    ratio = cm / np.maximum(cl, 1e-30)
    acc = (fm & B.DDM_FIT_MLP_ACCEPTED) > 0
    return {
        "curves": int(il.size),
        "lm_iters_mean": float(il.mean()), "mlp_lm_iters_mean": float(im.mean()),
        "lm_converged": float(np.mean((fl & B.DDM_FIT_CONVERGED) > 0)),
        "mlp_lm_converged": float(np.mean((fm & B.DDM_FIT_CONVERGED) > 0)),
        "mlp_accepted": float(np.mean((fm & B.DDM_FIT_MLP_ACCEPTED) > 0)),
        "lm_fallback_rate": float(np.mean((fm & B.DDM_FIT_MLP_ACCEPTED) == 0)),
        "seed_heuristic": float(np.mean((fm & B.DDM_FIT_SEED_HEURISTIC) > 0)),
        "restarted": float(np.mean((fm & B.DDM_FIT_FALLBACK) > 0)),
        "cost_ratio_median": float(np.median(ratio)),
        "cost_ratio_p99": float(np.quantile(ratio, 0.99)),
        "cost_within_1e-3": float(np.mean(ratio <= 1.0 + 1e-3)),
        # curves where LM ran after the network's seed: they should reach plain LM's optimum
        "lm_run_cost_within_1e-3": float(np.mean(ratio[~acc] <= 1.0 + 1e-3)) if np.any(~acc) else None,
        # curves whose network parameters were kept (RMS residual <= 1e-2 A): their cost
        # relative to plain LM's optimum
        "accepted_cost_ratio_median": float(np.median(ratio[acc])) if np.any(acc) else None,
    }
