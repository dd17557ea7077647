"""Seeded synthetic image stacks shaped like the paper's DDM workloads.

The paper measured 16-bit microscopy image sets of up to 2^14 frames (Sec. 2); those sets
are not available, so these generators stand in for them.  This module is shared by the
oracle side and the CUDA side as *input only*: it holds none of the structure-function
arithmetic.  Random numbers are drawn here, on the host from numpy's PCG64, except in the
``*_torch`` generators, which draw them with torch's seeded generator on the device that
renders the stack (for stacks too large to render on the host).

Two families:

* :func:`ou_stack` -- a real random field whose every Fourier mode is an independent complex
  Ornstein-Uhlenbeck process with rate Gamma(q) = D0 q^2 and stationary power S(q), plus
  white pixel noise sigma.  For the unnormalised spatial DFT it gives
  E[D(q, dt)] = H W (2 S(q) (1 - exp(-Gamma(q) dt)) + 2 sigma^2), which the oracle tests use.
* :func:`blob_stack` -- Brownian Gaussian particles on a periodic field, a background that
  makes the frame mean ``mean``, Poisson shot noise, clamping to 12 bits, uint16 output.
  Options cover two species, a log-normal spread of D0 and a slow illumination drift.

|q| is in rad/px: q = 2 pi sqrt((ky'/H)^2 + (kx'/W)^2) with signed DFT indices ky', kx'.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np


def q_magnitude(H: int, W: int) -> np.ndarray:
    """|q| [H, W] in rad/px for DFT indices in numpy order."""
    ky = np.fft.fftfreq(H) * 2.0 * np.pi
    kx = np.fft.fftfreq(W) * 2.0 * np.pi
    return np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


def gaussian_spectrum(width: float):
    """S(q) = exp(-q^2 / (2 width^2))."""
    return lambda q: np.exp(-(q ** 2) / (2.0 * width ** 2))


def power_law_spectrum(q_cut: float = 0.02):
    """S(q) = 1 / max(q, q_cut)^2."""
    return lambda q: 1.0 / np.maximum(q, q_cut) ** 2


def ou_stack(H: int, W: int, N: int, D0: float, spectrum, sigma: float, seed: int,
             dtype=np.float32) -> np.ndarray:
    """Fourier-mode Ornstein-Uhlenbeck stack, [N, H, W] of ``dtype``.

    G(k, 0) ~ CN(0, S); G(k, t+1) = e^{-Gamma} G(k, t) + sqrt(S (1 - e^{-2 Gamma})) xi_t with
    E|xi|^2 = 1, independently for every k; the frame is sqrt(2) Re(IDFT_ortho(G_t)) plus
    N(0, sigma^2) pixel noise.  D0 may be a float or a callable ``rng -> float``.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0x0A1])))
    if callable(D0):
        D0 = float(D0(rng))
    q = q_magnitude(H, W)
    S = np.asarray(spectrum(q), dtype=np.float64)
    gamma = D0 * q ** 2
    decay = np.exp(-gamma)
    drive = np.sqrt(S * (1.0 - np.exp(-2.0 * gamma)))

    def cnormal():
        return (rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))) / math.sqrt(2.0)

    G = np.sqrt(S) * cnormal()
    out = np.empty((N, H, W), dtype=dtype)
    for t in range(N):
        if t > 0:
            G = decay * G + drive * cnormal()
        field = math.sqrt(2.0) * np.fft.ifft2(G, norm="ortho").real
        if sigma > 0:
            field = field + sigma * rng.standard_normal((H, W))
        out[t] = field.astype(dtype)
    return out


def ou_stack_torch(H: int, W: int, N: int, D0, spectrum, sigma: float, seed: int,
                   device="cuda"):
    """The law of :func:`ou_stack`, drawn with torch's generator and rendered on ``device``
    (a CUDA device for stacks too large to render on the host in reasonable time, e.g.
    1024x1024x4096 float32 = 17 GB).  Returns a float32 torch tensor [N, H, W].

    Same recursion: G(k, 0) ~ CN(0, S); G(k, t+1) = e^{-Gamma} G(k, t) +
    sqrt(S (1 - e^{-2 Gamma})) xi_t, E|xi|^2 = 1; frame = sqrt(2) Re(IDFT_ortho(G_t)) +
    N(0, sigma^2).  Modes are carried in complex64 and the inverse transform is torch's
    (an input generator only; it is not part of the structure-function path).  D0 may be a
    float or a callable ``numpy_rng -> float`` (drawn from PCG64 seeded by ``seed``).
    """
    import torch
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0x0A2])))
    if callable(D0):
        D0 = float(D0(rng))
    q = q_magnitude(H, W)
    S = np.asarray(spectrum(q), dtype=np.float64)
    gamma = D0 * q ** 2
    decay = torch.from_numpy(np.exp(-gamma).astype(np.float32)).to(device)
    drive = torch.from_numpy(np.sqrt(S * (1.0 - np.exp(-2.0 * gamma))).astype(np.float32)).to(device)
    amp = torch.from_numpy(np.sqrt(S).astype(np.float32)).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 7919 + 17)

    def cnormal():
        z = torch.randn((2, H, W), generator=g, device=device, dtype=torch.float32) / math.sqrt(2.0)
        return torch.complex(z[0], z[1])

    G = amp * cnormal()
    out = torch.empty((N, H, W), dtype=torch.float32, device=device)
    for t in range(N):
        if t > 0:
            G = decay * G + drive * cnormal()
        field = math.sqrt(2.0) * torch.fft.ifft2(G, norm="ortho").real
        if sigma > 0:
            field = field + sigma * torch.randn((H, W), generator=g, device=device, dtype=torch.float32)
        out[t] = field
    return out


def log_uniform_d0(lo: float = 0.01, hi: float = 1.0):
    """A D0 drawn log-uniformly in [lo, hi] from the generator's own numpy stream."""
    return lambda rng: float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def ou_precision_sweep_1024x1024x4096(seed: int = 0, N: int = 4096, H: int = 1024, W: int = 1024,
                                      device="cuda"):
    """The precision-sweep stack: 1024x1024 float32, N = 4096, OU Fourier modes with
    S(q) = 1 / max(q, 0.02)^2, D0 log-uniform in [0.01, 1] (once per stack), no pixel noise;
    rendered on ``device`` (torch tensor)."""
    return ou_stack_torch(H, W, N, log_uniform_d0(0.01, 1.0), power_law_spectrum(0.02), 0.0, seed,
                          device=device)


def ou_params(D0: float, spectrum_width: float):
    """Parameters of the small OU workload: 64x64 float32, N = 128."""
    return dict(D0=D0, spectrum=gaussian_spectrum(spectrum_width))


def _profile(H_or_W: int, centres: np.ndarray, sigma: float, reach: int) -> tuple:
    """Sparse periodic 1D Gaussian profiles: rows, columns and values for every particle.

    The profile of a particle at u0 is exp(-d(u, u0)^2 / (2 sigma^2)) for the periodic
    (minimum-image) distance d <= reach pixels, and zero further away.
    """
    P = centres.shape[0]
    base = np.floor(centres).astype(np.int64)
    offs = np.arange(-reach, reach + 1, dtype=np.int64)
    idx = base[:, None] + offs[None, :]
    d = idx.astype(np.float64) - centres[:, None]
    vals = np.exp(-(d ** 2) / (2.0 * sigma ** 2))
    vals[np.abs(d) > reach] = 0.0
    rows = np.repeat(np.arange(P), offs.size)
    return rows, np.mod(idx, H_or_W).ravel(), vals.ravel()


def blob_stack(H: int, W: int, N: int, n_particles: int, sigma_px: float, D0, seed: int,
               mean: float = 2000.0, amplitude: float = 1000.0, max_count: int = 4095,
               drift: float = 0.0, threads: int | None = None) -> np.ndarray:
    """Brownian Gaussian-blob stack with Poisson noise, [N, H, W] uint16.

    D0: a float (one species), or an array of per-particle D0 (px^2/frame).  Each frame
    step moves every particle by N(0, 2 D0) px per axis, with periodic wrap.  The
    expected frame is bg + amplitude * sum_p g_y(p) g_x(p) with bg chosen so the mean is
    ``mean``; drift multiplies frame t by 1 + drift * t / (N - 1) (illumination ramp);
    counts are Poisson, clamped to ``max_count``.
    """
    ss = np.random.SeedSequence([int(seed), 0xB10B])
    rng = np.random.Generator(np.random.PCG64(ss.spawn(1)[0]))
    P = int(n_particles)
    d0 = np.broadcast_to(np.asarray(D0, dtype=np.float64), (P,)).copy()
    start = rng.uniform(0.0, 1.0, size=(P, 2)) * np.array([H, W], dtype=np.float64)
    steps = rng.standard_normal((N, P, 2)) * np.sqrt(2.0 * d0)[None, :, None]
    steps[0] = 0.0
    pos = start[None] + np.cumsum(steps, axis=0)
    pos[..., 0] = np.mod(pos[..., 0], H)
    pos[..., 1] = np.mod(pos[..., 1], W)
    reach = int(math.ceil(4.0 * sigma_px))
    bg = mean - P * amplitude * (2.0 * math.pi * sigma_px ** 2) / float(H * W)
    frame_seeds = ss.spawn(N + 1)[1:]
    out = np.empty((N, H, W), dtype=np.uint16)

    def render(t):
        ry, cy, vy = _profile(H, pos[t, :, 0], sigma_px, reach)
        rx, cx, vx = _profile(W, pos[t, :, 1], sigma_px, reach)
        Gy = np.zeros((P, H), np.float32)
        Gx = np.zeros((P, W), np.float32)
        np.add.at(Gy, (ry, cy), vy.astype(np.float32))
        np.add.at(Gx, (rx, cx), vx.astype(np.float32))
        lam = (amplitude * (Gy.T @ Gx)).astype(np.float64) + bg
        if drift:
            lam *= 1.0 + drift * t / max(N - 1, 1)
        np.maximum(lam, 0.0, out=lam)
        r = np.random.Generator(np.random.PCG64(frame_seeds[t]))
        counts = r.poisson(lam)
        np.minimum(counts, max_count, out=counts)
        out[t] = counts.astype(np.uint16)

    n_threads = threads or min(16, os.cpu_count() or 1)
    if n_threads <= 1 or N < 4:
        for t in range(N):
            render(t)
    else:
        with ThreadPoolExecutor(max_workers=n_threads) as ex:
            list(ex.map(render, range(N)))
    return out


def blob_stack_torch(H: int, W: int, N: int, n_particles: int, sigma_px: float, D0, seed: int,
                     mean: float = 2000.0, amplitude: float = 1000.0, max_count: int = 4095,
                     drift: float = 0.0, device="cuda", chunk: int = 32):
    """The law of :func:`blob_stack` (Brownian Gaussian blobs on a periodic field, Poisson
    counts clamped to ``max_count``, uint16), drawn with torch's seeded generator and rendered
    on ``device``: the 200 training stacks of 512x512x1024 that the seed network learns from
    take minutes each on the host and milliseconds here.  Returns a uint16 tensor [N, H, W].

    Same model: start positions uniform on the field, steps N(0, 2 D0) px per axis per frame
    (D0 a float or a per-particle array), periodic wrap; the expected frame is
    bg + amplitude sum_p g(y - y_p) g(x - x_p) with g the Gaussian of ``sigma_px`` at the
    minimum-image distance, cut at 4 sigma (rounded up to whole pixels), bg making the
    mean ``mean``; ``drift`` multiplies frame t by 1 + drift t / (N - 1); Poisson counts.
    """
    import torch
    P = int(n_particles)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 0xB10B)
    d0 = torch.as_tensor(np.broadcast_to(np.asarray(D0, dtype=np.float64), (P,)).copy(), device=device)
    dims = torch.tensor([H, W], dtype=torch.float64, device=device)
    start = torch.rand((P, 2), generator=g, device=device, dtype=torch.float64) * dims
    reach = int(math.ceil(4.0 * sigma_px))
    bg = mean - P * amplitude * (2.0 * math.pi * sigma_px ** 2) / float(H * W)
    ys = torch.arange(H, device=device, dtype=torch.float64)
    xs = torch.arange(W, device=device, dtype=torch.float64)
    out = torch.empty((N, H, W), dtype=torch.int16, device=device)
    pos = start.clone()
    step_sd = torch.sqrt(2.0 * d0)[:, None]

    def profile(centres, coords, L):
        # centres are wrapped into [0, L) in float64 (trajectories wander far); the
        # minimum-image distance and the Gaussian in float32 (|d| < L: ~1e-5 px of rounding)
        c32 = centres.float()
        d = torch.remainder(coords.float()[None, None, :] - c32[:, :, None] + L / 2.0, float(L)) - L / 2.0
        v = torch.exp(-(d * d) * (1.0 / (2.0 * sigma_px ** 2)))
        return torch.where(d.abs() <= reach, v, torch.zeros_like(v))

    for t0 in range(0, N, chunk):
        n = min(chunk, N - t0)
        steps = torch.randn((n, P, 2), generator=g, device=device, dtype=torch.float64) * step_sd
        if t0 == 0:
            steps[0] = 0.0
        traj = torch.remainder(pos[None] + torch.cumsum(steps, dim=0), dims)
        pos = traj[-1].clone()
        gy = profile(traj[..., 0], ys, H)                 # [n, P, H]
        gx = profile(traj[..., 1], xs, W)                 # [n, P, W]
        lam = amplitude * torch.bmm(gy.transpose(1, 2), gx) + bg
        if drift:
            tt = torch.arange(t0, t0 + n, device=device, dtype=torch.float32)
            lam = lam * (1.0 + drift * tt / max(N - 1, 1))[:, None, None]
        lam = torch.clamp(lam, min=0.0)
        counts = torch.clamp(torch.poisson(lam, generator=g), max=float(max_count))
        out[t0:t0 + n] = counts.to(torch.int16)
    return out.view(torch.uint16)


def polydisperse_blobs_512x512x1024(seed: int, N: int = 1024, H: int = 512, W: int = 512,
                                    device="cuda"):
    """The learned-stage workload: 512x512 uint16, N = 1024, 3000 blobs (sigma 2 px) with
    log-normal D0 (median 0.2 px^2/frame, sigma_ln 0.5), mean 2000, Poisson; rendered on
    ``device`` (seeds 1000-1199 train the seed network, 2000-2019 are held out)."""
    d0 = lognormal_d0(3000, 0.2, 0.5, seed)
    return blob_stack_torch(H, W, N, 3000, 2.0, d0, seed, device=device)


def lognormal_d0(n: int, median: float, sigma_ln: float, seed: int) -> np.ndarray:
    """Per-particle D0 drawn log-normally (polydisperse sample)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0x1D0])))
    return median * np.exp(sigma_ln * rng.standard_normal(n))


def two_species_d0(n: int, d_a: float, d_b: float) -> np.ndarray:
    """Half the particles with D0 = d_a, half with d_b."""
    d = np.full(n, d_a, dtype=np.float64)
    d[n // 2:] = d_b
    return d


# Workloads named by what they are, with their sizes.
def ou_64x64x128(seed: int = 0) -> np.ndarray:
    """64x64 float32, N = 128, D0 = 0.5, S = exp(-q^2 / (2 * 0.3^2)), sigma = 0.01."""
    return ou_stack(64, 64, 128, 0.5, gaussian_spectrum(0.3), 0.01, seed)


def blobs_two_species_600x800(seed: int = 0, N: int = 3000, H: int = 600, W: int = 800) -> np.ndarray:
    """600x800 uint16, N = 3000: 4000 blobs (sigma 2 px), half with D0 = 0.05 and half with
    D0 = 0.8 px^2/frame, mean 2000, Poisson, a 1 % linear illumination drift over the stack."""
    return blob_stack(H, W, N, 4000, 2.0, two_species_d0(4000, 0.05, 0.8), seed, drift=0.01)


def blobs_512x512x1024(seed: int = 0, N: int = 1024, H: int = 512, W: int = 512) -> np.ndarray:
    """512x512 uint16, N = 1024, 3000 blobs (sigma 2 px), D0 = 0.2, mean 2000, Poisson."""
    return blob_stack(H, W, N, 3000, 2.0, 0.2, seed)


# Fit-stage data: curves of known parameters, and initial network weights.
def stretched_exp_curves(n: int, N: int, seed: int, noise_rel: float = 0.01,
                         log10_tau=(0.3, 2.6), log10_b_over_a=None):
    """n curves D(m), m = 0..N-1, with D(0) = 0 and, for m >= 1,
    D(m) = A (1 - exp(-(m / tau)^beta)) + B times (1 + noise_rel * N(0, 1)).

    A = s * 10^U(-0.3, 0.3) with a per-curve scale s = 10^U(2, 9); tau = 10^U(log10_tau);
    beta = U(0.5, 1.1); B = A * U(0, 0.5), or A * 10^U(log10_b_over_a) when given.
    Returns (D [n, N] float32, labels [n, 4] as (A, tau, beta, B) float64).
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0xF17])))
    scale = 10.0 ** rng.uniform(2, 9, n)
    A = scale * 10.0 ** rng.uniform(-0.3, 0.3, n)
    tau = 10.0 ** rng.uniform(log10_tau[0], log10_tau[1], n)
    beta = rng.uniform(0.5, 1.1, n)
    if log10_b_over_a is None:
        B = A * rng.uniform(0.0, 0.5, n)
    else:
        B = A * 10.0 ** rng.uniform(log10_b_over_a[0], log10_b_over_a[1], n)
    m = np.arange(N, dtype=np.float64)[None, :]
    D = A[:, None] * (1.0 - np.exp(-np.power(m / tau[:, None], beta[:, None]))) + B[:, None]
    D *= 1.0 + noise_rel * rng.standard_normal(D.shape)
    D[:, 0] = 0.0
    return D.astype(np.float32), np.stack([A, tau, beta, B], axis=1)


def mlp_init(seed: int) -> np.ndarray:
    """Initial weights of the 64-128-128-128-4 network: uniform(+-sqrt(6 / fan_in)) per
    weight matrix (He), zero biases; flat [W1, b1, W2, b2, W3, b3, W4, b4], float32."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0x3A1])))
    parts = []
    for fi, fo in [(64, 128), (128, 128), (128, 128), (128, 4)]:
        lim = math.sqrt(6.0 / fi)
        parts.append(rng.uniform(-lim, lim, fi * fo))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)
