"""Host side of splitting one stack across ranks by stored wave-vector range: the range
split, and the merge of the ranks' radial sums, pinned against the oracle's radial average
of the whole plane (numpy and a two-rank gloo all-reduce on CPU)."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2012_05695_b300 import partition, spectrum_index_map

H, W, N, NB = 16, 16, 24, 7


@pytest.mark.parametrize("n_q,parts", [(40, 1), (544, 2), (131584, 8), (2112, 3), (64 * 5 + 1, 6)])
def test_q_ranges_cover_aligned_and_balanced(n_q, parts):
    r = partition.q_ranges(n_q, parts)
    assert len(r) == parts
    assert r[0][0] == 0 and r[-1][1] == n_q
    for (a, b), (c, _) in zip(r, r[1:]):
        assert b == c                                   # contiguous, disjoint
    for a, b in r:
        assert a % partition.RANGE_ALIGN == 0 and b > a
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 2 * partition.RANGE_ALIGN


def test_q_ranges_rejects_too_many_parts():
    with pytest.raises(ValueError):
        partition.q_ranges(100, 3)


def _half_plane_D():
    """Oracle D over the half plane kx = 0..W/2 of a small OU stack, and the full plane."""
    frames = synth.ou_stack(H, W, N, 0.5, synth.gaussian_spectrum(0.3), 0.05, seed=3)
    F = oracle.dft2(frames)                      # [N, H, W]
    D_full = oracle.sf_direct(F)                 # [H, W, N]
    return D_full[:, : W // 2 + 1, :], D_full


def _partial_sums(D_half, q0, q1):
    """Radial sums and counts over stored wave vectors [q0, q1), weights 2 for 0 < kx < W/2."""
    bins = oracle.radial_bins(H, W, NB)
    ky, kx = spectrum_index_map(H, W)
    sums = np.zeros((NB, N))
    counts = np.zeros(NB, np.int64)
    for s in range(q0, q1):
        w = 1 if kx[s] in (0, W // 2) else 2
        b = bins[ky[s], kx[s]]
        sums[b] += w * D_half[ky[s], kx[s]]
        counts[b] += w
    return sums, counts


def test_merged_partial_sums_equal_the_whole_plane_average():
    D_half, D_full = _half_plane_D()
    Dr_ref, cnt_ref = oracle.radial_average(D_full, NB)
    n_q = H * (W // 2 + 1)
    parts = [_partial_sums(D_half, a, b) for a, b in partition.q_ranges(n_q, 2)]
    sums = sum(p[0] for p in parts)
    counts = sum(p[1] for p in parts)
    np.testing.assert_array_equal(counts, cnt_ref)
    np.testing.assert_allclose(partition.merge_radial(sums, counts), Dr_ref, rtol=1e-12, atol=1e-12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        D_half, D_full = _half_plane_D()
        q0, q1 = partition.q_ranges(H * (W // 2 + 1), world)[rank]
        s, c = _partial_sums(D_half, q0, q1)
        Dr = partition.allreduce_radial(torch.from_numpy(s), torch.from_numpy(c))
        np.save(os.path.join(out_dir, f"dr{rank}.npy"), Dr.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_allreduce_of_radial_sums(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    _, D_full = _half_plane_D()
    Dr_ref, _ = oracle.radial_average(D_full, NB)
    for r in range(world):
        np.testing.assert_allclose(np.load(tmp_path / f"dr{r}.npy"), Dr_ref, rtol=1e-12, atol=1e-12)


def test_kx_ranges_cover_the_columns_in_aligned_blocks():
    from paper_2012_05695_b300 import partition
    for W, parts in [(32, 1), (512, 2), (512, 3), (512, 8), (1024, 7), (256, 8)]:
        r = partition.kx_ranges(W, parts)
        assert len(r) == parts and r[0][0] == 0 and r[-1][1] == W // 2
        for (a, b), (c, _) in zip(r, r[1:]):
            assert b == c
        for a, b in r:
            assert a % 16 == 0 and b % 16 == 0 and b > a
        sizes = [b - a for a, b in r]
        assert max(sizes) - min(sizes) <= 16
    with pytest.raises(ValueError):
        partition.kx_ranges(256, 9)      # 8 blocks of 16 columns
    with pytest.raises(ValueError):
        partition.kx_ranges(40, 1)       # W/2 = 20 is not whole blocks


def _kx_rank_main(rank, world, port, out_dir):
    """One rank of a stack split by kx columns: the oracle D of its columns only (plus the
    kx = W/2 column on the rank whose range starts at 0), its radial sums, the gloo sum."""
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Hk, Wk, Nk = 16, 64, 24
        frames = synth.ou_stack(Hk, Wk, Nk, 0.5, synth.gaussian_spectrum(0.3), 0.05, seed=4)
        kx0, kx1 = partition.kx_ranges(Wk, world)[rank]
        cols = list(range(kx0, kx1)) + ([Wk // 2] if kx0 == 0 else [])
        D = oracle.sf_direct(oracle.dft2(frames, cols))          # [H, len(cols), N]
        bins = oracle.radial_bins(Hk, Wk, NB)
        s = np.zeros((NB, Nk))
        c = np.zeros(NB, np.int64)
        for j, kx in enumerate(cols):
            w = 1 if kx in (0, Wk // 2) else 2
            for ky in range(Hk):
                s[bins[ky, kx]] += w * D[ky, j]
                c[bins[ky, kx]] += w
        Dr = partition.allreduce_radial(torch.from_numpy(s), torch.from_numpy(c))
        np.save(os.path.join(out_dir, f"kxdr{rank}.npy"), Dr.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_kx_column_split(tmp_path):
    """The kx-column split's host logic on two gloo ranks: each rank's columns (the ranges
    of kx_ranges, the kx = W/2 column with the first) give radial sums whose all-reduce is
    the oracle's whole-plane radial average."""
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_kx_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    frames = synth.ou_stack(16, 64, 24, 0.5, synth.gaussian_spectrum(0.3), 0.05, seed=4)
    Dr_ref, _ = oracle.radial_average(oracle.sf_direct(oracle.dft2(frames)), NB)
    for r in range(world):
        np.testing.assert_allclose(np.load(tmp_path / f"kxdr{r}.npy"), Dr_ref, rtol=1e-12, atol=1e-12)
