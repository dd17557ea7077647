"""One stack split across ranks, with no exchange of spectra.

Every wave vector's time analysis is independent of every other (Sec. 2), so step two
needs no exchange.  Two ways to cut the half plane:

* by kx columns (``kx_ranges``): rank r creates its plan with ``kx_begin, kx_end =
  kx_ranges(W, R)[r]``; step one transforms every row (each rank reads all frames) but
  only the rank's own columns, into a store that holds just those columns, and step two
  runs on it.  Step one's column pass is split as well as step two.
* by stored wave-vector range (``q_ranges``): ``q_begin, q_end = q_ranges(n_q, R)[r]``;
  step one runs in full on every rank (rows are stored ky-major, so a range of stored
  wave vectors needs every column) and step two on the range.

Either way ``Plan.azimuthal_sums`` gives the rank's share of the radial stage, and the only
collective is the sum of those shares, [n_bins][N] floats and [n_bins] counts, after which
each rank divides.  This module holds that host logic; it does no arithmetic of the method
itself.
"""
from __future__ import annotations

RANGE_ALIGN = 64   # the library's alignment rule for q_begin


def q_ranges(n_q: int, parts: int, align: int = RANGE_ALIGN):
    """Split stored wave vectors [0, n_q) into `parts` contiguous ranges whose starts are
    multiples of `align`, as even as that allows.  Returns [(q_begin, q_end), ...]."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    blocks = -(-n_q // align)
    if parts > blocks:
        raise ValueError(f"{parts} ranges of >= {align} wave vectors do not fit n_q = {n_q}")
    out = []
    for r in range(parts):
        b0 = (blocks * r) // parts
        b1 = (blocks * (r + 1)) // parts
        out.append((b0 * align, min(b1 * align, n_q)))
    return out


KX_ALIGN = 16      # the library's alignment rule for kx_begin / kx_end (column blocks)


def kx_ranges(W: int, parts: int, align: int = KX_ALIGN):
    """Split the half plane's columns kx = 0 .. W/2 - 1 into `parts` contiguous ranges of
    whole blocks of `align` columns, as even as that allows; the range that starts at 0
    also carries the kx = W/2 column (the library adds it).  Returns [(kx_begin, kx_end)]."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    Wh = W // 2
    if Wh % align != 0:
        raise ValueError(f"W/2 = {Wh} is not a multiple of {align}")
    blocks = Wh // align
    if parts > blocks:
        raise ValueError(f"{parts} ranges of >= {align} columns do not fit W/2 = {Wh}")
    out = []
    for r in range(parts):
        b0 = (blocks * r) // parts
        b1 = (blocks * (r + 1)) // parts
        out.append((b0 * align, b1 * align))
    return out


def merge_radial(sums, counts):
    """D_r from the radial sums and counts added over all ranks: sums / counts per bin,
    0 for empty bins.  numpy arrays or torch tensors ([n_bins, N] and [n_bins])."""
    try:
        import torch
        if isinstance(sums, torch.Tensor):
            c = counts.to(sums.dtype).unsqueeze(-1)
            return torch.where(c > 0, sums / torch.clamp(c, min=1), torch.zeros_like(sums))
    except ImportError:   # pragma: no cover - torch is part of the environment
        pass
    import numpy as np
    c = np.asarray(counts, dtype=np.float64)[:, None]
    s = np.asarray(sums)
    return np.where(c > 0, s / np.maximum(c, 1), 0.0).astype(s.dtype)


def allreduce_radial(sums, counts, group=None):
    """Sum every rank's radial sums and counts in place (torch.distributed, any backend)
    and return D_r on every rank."""
    import torch.distributed as dist
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return merge_radial(sums, counts)
