"""bench.py's multi-rank arithmetic on CPU ranks (gloo, world size 2): every rank sees the
slowest rank's time, and the reported throughput is the whole job's."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist)     # rank 1 is the slow one
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(repr(ms))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert float((tmp_path / f"r{r}.txt").read_text()) == 150.0


def test_single_rank_and_throughput():
    assert bench.max_over_ranks(12.5) == 12.5
    # two ranks, 1024 frames each, 10 steps in 20 ms -> 1,024,000 frames/s for the job
    assert bench.job_throughput(2, 1024, 10, 20.0) == pytest.approx(1.024e6)
    assert bench.job_throughput(1, 1024, 10, 20.0) == pytest.approx(5.12e5)


def test_fit_label_targets_invert_the_network_head():
    """The bench trains the seed network on targets it derives from fit labels; they must be
    the inverse of the head (oracle.fit.head): targets(head(o)) = (o0, o1, beta(o2), o3)."""
    import numpy as np
    from oracle import fit as F
    rng = np.random.Generator(np.random.PCG64(4))
    o = np.stack([rng.normal(0, 1, 500), rng.normal(1, 2, 500), rng.normal(0, 2, 500),
                  rng.normal(0, 0.5, 500)], axis=1)
    p8 = rng.uniform(0.1, 10, 500)
    phys = F.head(o, p8)
    t = bench.head_targets(phys, p8)
    np.testing.assert_allclose(t[:, [0, 1, 3]], o[:, [0, 1, 3]], rtol=0, atol=1e-12)
    np.testing.assert_allclose(t[:, 2], phys[:, 2], rtol=0, atol=0)


def test_traffic_is_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    """The bench line's roofline `traffic` comes from the committed ncu summary only while
    that summary's source hash is the hash of the step-two sources being built; any edit of
    those sources turns it into null."""
    csrc = tmp_path / "paper_2012_05695_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "ddm_temporal.cu").write_text("// kernel v1\n")
    (csrc / "ddm_fft.cuh").write_text("// fft\n")
    (csrc / "ddm_internal.h").write_text("// internal\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "temporal_sf_512x512x1024.md"
    prof.write_text(f"# t\n\nsource_sha256_16: {bench.kernel_source_hash()}\n"
                    "dram_bytes_per_launch: 1586487552\n")
    assert bench.profiled_traffic() == 1586487552.0
    (csrc / "ddm_temporal.cu").write_text("// kernel v2\n")
    assert bench.profiled_traffic() is None
    prof.unlink()
    assert bench.profiled_traffic() is None
