"""FP64 oracle of the fit stage (not in the paper: the analysis that follows D(|q|, dt)).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  Plain numpy in double precision,
one curve at a time, written from these definitions:

* log lags: lambda_i = exp(i ln(N-1) / 63), i = 0..63; a curve D_r(m), m = 0..N-1, is
  sampled at lambda_i by linear interpolation between the two neighbouring lags.
* model: D(lambda) = A (1 - exp(-(lambda / tau)^beta)) + B.
* Levenberg-Marquardt on p = (A, B, ln tau, beta), residual r = model - y, cost = sum r^2,
  analytic Jacobian, Marquardt damping (J^T J + lam diag(J^T J)) dp = -J^T r, lam starts at
  1e-3, /10 on an accepted step, x10 on a rejected one; beta is clamped to [0.05, 3];
  stop when a step accepted at its first trial (no rejection in that iteration) lowers the
  cost by less than tol * cost, when lam exceeds 1e12, or after 100 iterations.
* heuristic seed: plateau p8 = mean of the last 8 samples, A0 = p8, B0 = 0, beta0 = 1,
  tau0 = the lag where y first reaches (1 - 1/e) p8 (log-linear interpolation; lambda_0 / 2
  if already reached, lambda_63 if never).
* MLP 64 -> 128 -> 128 -> 128 -> 4, GELU (erf form) after the three hidden layers.  Input
  x = y / p8.  Head: A = p8 exp(o0), tau = exp(o1), beta = 0.3 + 0.9 sigmoid(o2), B = A o3.
  Loss = mean over the batch of (o0 - ln(A/p8))^2 + (o1 - ln tau)^2 + (beta - beta*)^2
  + (o3 - B/A)^2 against label parameters.  Weight matrices are used rounded to bfloat16
  (round to nearest even); biases, activations and accumulation in full precision.
* Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps),
  b1 = 0.9, b2 = 0.999, eps = 1e-8, on FP32 master weights.
"""
from __future__ import annotations

import math

import numpy as np

N_LAGS = 64
LAYERS = [(64, 128), (128, 128), (128, 128), (128, 4)]      # (fan_in, fan_out)
N_PARAMS = sum(i * o + o for i, o in LAYERS)                  # 41860
FLAG_CONVERGED, FLAG_MAXITER, FLAG_NONFINITE = 1, 2, 4


# ----------------------------------------------------------------------------- sampling
def log_lags(N: int, n: int = N_LAGS) -> np.ndarray:
    if N < 2:
        raise ValueError("need at least two lags")
    return np.exp(np.arange(n) * (math.log(N - 1) / (n - 1)))


def sample_log_lags(Dr: np.ndarray) -> np.ndarray:
    """Dr [n_curves, N] -> y [n_curves, 64] by linear interpolation at the log lags."""
    Dr = np.asarray(Dr, dtype=np.float64)
    N = Dr.shape[-1]
    lam = log_lags(N)
    j = np.floor(lam).astype(np.int64)
    j = np.minimum(j, N - 1)
    frac = lam - j
    j1 = np.minimum(j + 1, N - 1)
    return Dr[..., j] * (1.0 - frac) + Dr[..., j1] * frac


def plateau(y: np.ndarray) -> np.ndarray:
    return np.mean(np.asarray(y, np.float64)[..., -8:], axis=-1)


# ----------------------------------------------------------------------------- model
def model(lam, A, tau, beta, B):
    return A * (1.0 - np.exp(-np.power(lam / tau, beta))) + B


def _model_and_jac(lam, p):
    A, B, ltau, beta = p
    lx = np.log(lam) - ltau
    s = np.exp(beta * lx)
    e = np.exp(-s)
    f = A * (1.0 - e) + B
    J = np.empty((lam.size, 4))
    J[:, 0] = 1.0 - e
    J[:, 1] = 1.0
    J[:, 2] = -A * beta * s * e
    J[:, 3] = A * e * s * lx
    return f, J


def heuristic_seed(lam, y):
    y = np.asarray(y, np.float64)
    p8 = float(np.mean(y[-8:]))
    target = (1.0 - math.exp(-1.0)) * p8
    idx = np.nonzero(y >= target)[0]
    if idx.size == 0:
        tau = float(lam[-1])
    elif idx[0] == 0:
        tau = float(lam[0]) / 2.0
    else:
        k = int(idx[0])
        y0, y1 = y[k - 1], y[k]
        w = (target - y0) / (y1 - y0) if y1 != y0 else 0.0
        tau = math.exp(math.log(lam[k - 1]) + w * (math.log(lam[k]) - math.log(lam[k - 1])))
    return np.array([p8, 0.0, math.log(tau), 1.0])


def lm_fit(lam, y, p0, max_iter=100, tol=1e-10):
    """Levenberg-Marquardt from p0 = (A, B, ln tau, beta).

    Returns (p, cost, iterations, flags)."""
    lam = np.asarray(lam, np.float64)
    y = np.asarray(y, np.float64)
    p = np.array(p0, dtype=np.float64)
    f, J = _model_and_jac(lam, p)
    r = f - y
    cost = float(r @ r)
    if not np.isfinite(cost):
        return p, cost, 0, FLAG_NONFINITE
    mu = 1e-3
    flags = FLAG_MAXITER
    it = 0
    while it < max_iter:
        it += 1
        g = J.T @ r
        Hm = J.T @ J
        accepted = False
        first_try = True
        while True:
            Ad = Hm + mu * np.diag(np.diag(Hm))
            try:
                dp = np.linalg.solve(Ad, -g)
            except np.linalg.LinAlgError:
                dp = np.full(4, np.nan)
            pn = p + dp
            pn[3] = min(max(pn[3], 0.05), 3.0)
            fn, Jn = _model_and_jac(lam, pn)
            rn = fn - y
            cn = float(rn @ rn)
            if np.isfinite(cn) and cn < cost:
                accepted = True
                break
            mu *= 10.0
            first_try = False
            if mu > 1e12:
                break
        if not accepted:
            flags = FLAG_CONVERGED
            break
        dec = cost - cn
        p, f, J, r, cost = pn, fn, Jn, rn, cn
        mu = max(mu / 10.0, 1e-12)
        if first_try and dec <= tol * cost:
            flags = FLAG_CONVERGED
            break
    return p, cost, it, flags


def params_to_physical(p):
    """(A, B, ln tau, beta) -> (A, tau, beta, B)."""
    A, B, ltau, beta = p
    return np.array([A, math.exp(ltau), beta, B])


# ----------------------------------------------------------------------------- MLP
def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(w: np.ndarray):
    """Flat parameter vector -> [(W [out, in], b [out]), ...]."""
    out, k = [], 0
    for fi, fo in LAYERS:
        W = w[k:k + fi * fo].reshape(fo, fi)
        k += fi * fo
        b = w[k:k + fo]
        k += fo
        out.append((W, b))
    return out


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def features(y):
    y = np.asarray(y, np.float64)
    p8 = plateau(y)
    p8 = np.where(p8 > 0, p8, 1.0)
    return y / p8[..., None], p8


def mlp_forward(w, x, bf16=True):
    """x [B, 64] -> (o [B, 4], cache).  Weight matrices rounded to bf16 if bf16."""
    layers = unpack(np.asarray(w, np.float64))
    h = np.asarray(x, np.float64)
    cache = [h]
    for li, (W, b) in enumerate(layers):
        Wq = bf16_round(W) if bf16 else W
        z = h @ Wq.T + b
        if li < len(layers) - 1:
            cache.append(z)
            h = gelu(z)
            cache.append(h)
        else:
            h = z
    return h, cache


def head(o, p8):
    """Raw outputs -> physical (A, tau, beta, B)."""
    A = p8 * np.exp(o[:, 0])
    tau = np.exp(o[:, 1])
    beta = 0.3 + 0.9 / (1.0 + np.exp(-o[:, 2]))
    B = A * o[:, 3]
    return np.stack([A, tau, beta, B], axis=1)


def targets(params_phys, p8):
    """Label (A, tau, beta, B) -> regression targets (ln(A/p8), ln tau, beta, B/A)."""
    A, tau, beta, B = (params_phys[:, k] for k in range(4))
    return np.stack([np.log(A / p8), np.log(tau), beta, B / A], axis=1)


def loss_and_grad(w, x, t, bf16=True):
    """Mean-squared loss of the head against targets t and its gradient w.r.t. w."""
    o, cache = mlp_forward(w, x, bf16)
    Bn = x.shape[0]
    sig = 1.0 / (1.0 + np.exp(-o[:, 2]))
    yhat = np.stack([o[:, 0], o[:, 1], 0.3 + 0.9 * sig, o[:, 3]], axis=1)
    diff = yhat - t
    loss = float(np.sum(diff * diff) / Bn)
    d = 2.0 * diff / Bn
    d[:, 2] *= 0.9 * sig * (1.0 - sig)
    layers = unpack(np.asarray(w, np.float64))
    grads = []
    delta = d                                   # dL/do
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        Wq = bf16_round(W) if bf16 else W
        h_in = cache[0] if li == 0 else cache[2 * li]
        gW = delta.T @ h_in
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            z_prev = cache[2 * li - 1]
            delta = (delta @ Wq) * gelu_grad(z_prev)
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in reversed(grads)])
    return loss, g


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
