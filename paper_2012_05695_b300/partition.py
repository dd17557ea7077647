"""One stack split across ranks by stored wave-vector range.

Every wave vector's time analysis is independent of every other (Sec. 2), so step two
needs no exchange: rank r creates its plan with ``q_begin, q_end = q_ranges(n_q, R)[r]``,
runs step one in full (each rank holds the whole spectrum) and step two on its range, and
``Plan.azimuthal_sums`` gives its share of the radial stage.  The only collective is the
sum of those shares, [n_bins][N] floats and [n_bins] counts, after which each rank divides.
This module holds that host logic; it does no arithmetic of the method itself.
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
