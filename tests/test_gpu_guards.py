"""Guard bands around every output of the C ABI, complete coverage of what each call must
write, and the bounded device wait giving up with DDM_ERR_TIMEOUT.

Each output buffer sits between two guard zones filled with a NaN bit pattern no kernel
writes; after the call the zones must be intact and the output region must hold no guard
word where the call is documented to write (every stored spectrum entry; every D row of
the plan's wave-vector range; every radial bin; every fitted curve).
"""
import numpy as np
import pytest

import paper_2012_05695_b300 as ddm
import synth
from gpu_helpers import to_device

pytestmark = pytest.mark.gpu

GUARD = 4096                    # floats on each side (16 KB: keeps 16-byte alignment)
SENTINEL = np.int32(0x7FC0DEAD)  # a quiet-NaN payload


def _guarded(n):
    import torch
    buf = torch.empty(n + 2 * GUARD, dtype=torch.float32, device="cuda")
    buf.view(torch.int32).fill_(int(SENTINEL))
    return buf, buf[GUARD:GUARD + n]


def _inner_after(buf, n):
    import torch
    torch.cuda.synchronize()
    b = buf.view(torch.int32).cpu().numpy()
    assert np.all(b[:GUARD] == SENTINEL), "write below the output"
    assert np.all(b[GUARD + n:] == SENTINEL), "write past the output"
    return b[GUARD:GUARD + n]


def _frames(N, H, W, dtype, seed):
    if dtype == "u16":
        return synth.blob_stack(H, W, N, max(1, H * W // 90), 2.0, 0.2, seed)
    return synth.ou_stack(H, W, N, 0.4, synth.gaussian_spectrum(0.5), 0.02, seed)


CASES = [
    (64, 64, 100, "f32", {}),                               # 512-point time kernel (N > 64)
    (16, 32, 37, "u16", {}),                                # short kernel, ragged tile
    (32, 32, 300, "u16", {"kmax": 7}),                      # cropped store
    (16, 16, 2000, "f32", {"q_begin": 64, "q_end": 140}),   # three-pass kernel on a range
    (8, 12, 9, "f32", {}),                                  # Bluestein M = 32
    (30, 100, 5, "u16", {}),                                # Bluestein rows and columns
    (8, 16, 9000, "u16", {}),                               # 16384-point time kernel
]


@pytest.mark.parametrize("H,W,N,dtype,kw", CASES)
def test_outputs_stay_inside_their_buffers(H, W, N, dtype, kw):
    import torch
    nb = 7
    frames = to_device(_frames(N, H, W, dtype, seed=H * W + N))
    plan = ddm.Plan(H, W, N, dtype=dtype, n_bins=nb, **kw)
    nq = plan.n_q
    # step one: every stored spectrum entry of every frame
    sbuf, spec = _guarded(2 * N * nq)
    plan.spatial_fft(frames, spec)
    inner = _inner_after(sbuf, 2 * N * nq)
    assert not np.any(inner == SENTINEL)
    # step two: the D rows of the plan's wave-vector range, nothing else
    dbuf, D = _guarded(nq * N)
    plan.temporal_sf(spec, D)
    inner = _inner_after(dbuf, nq * N).reshape(nq, N)
    rows = np.arange(nq)
    if "q_begin" in kw:
        sky, skx = (np.asarray(a) for a in ddm.spectrum_index_map(H, W))
        st = np.arange(kw["q_begin"], kw["q_end"])
        rows = sky[st] * (W // 2 + 1) + skx[st]
        others = np.setdiff1d(np.arange(nq), rows)
        assert np.all(inner[others] == SENTINEL), "rows outside the range were written"
    assert not np.any(inner[rows] == SENTINEL)
    assert plan.last_device_status() == 0
    # the radial stage: every bin, every lag, and the counts
    rbuf, Dr = _guarded(nb * N)
    cbuf, cnt = _guarded(nb)
    plan.azimuthal_average(D, Dr, cnt.view(torch.int32))
    assert not np.any(_inner_after(rbuf, nb * N) == SENTINEL)
    assert not np.any(_inner_after(cbuf, nb) == SENTINEL)


def test_fit_outputs_stay_inside_their_buffers():
    import torch
    n, N = 37, 512
    curves = synth.stretched_exp_curves(n, N, seed=3)[0].astype(np.float32)
    plan = ddm.Plan(16, 16, N, dtype="f32", n_bins=n)
    Dr = torch.from_numpy(np.ascontiguousarray(curves).ravel()).cuda()
    pbuf, params = _guarded(4 * n)
    cbuf, cost = _guarded(n)
    ibuf, iters = _guarded(n)
    fbuf, flags = _guarded(n)
    plan.fit(Dr, n, ddm._binding.DDM_FIT_LM, None, params, cost, iters.view(torch.int32),
             flags.view(torch.int32))
    for buf, size in ((pbuf, 4 * n), (cbuf, n), (ibuf, n), (fbuf, n)):
        assert not np.any(_inner_after(buf, size) == SENTINEL)


@pytest.mark.parametrize("cap", [1000, 2_000_000])
def test_bounded_wait_gives_up_with_timeout(cap):
    """A tile barrier armed for bytes no copy delivers, and an MMA barrier no commit
    completes (in a CTA holding tensor memory): both waits must give up after their bound
    and report DDM_ERR_TIMEOUT through the status words, the tensor memory is released, and
    the context stays usable (the tensor-core forward still runs afterwards)."""
    import torch
    assert ddm.selftest_bounded_wait(cap) == ddm._binding.DDM_ERR_TIMEOUT
    x = torch.ones(1024, device="cuda")
    assert float(x.sum().item()) == 1024.0
    mlp = ddm.MLP(256)
    mlp.set_weights(synth.mlp_init(1))
    o = torch.full((256 * 4,), float("nan"), device="cuda")
    mlp.forward(torch.rand(256 * 64, device="cuda"), 256, o)
    assert mlp.last_device_status() == ddm._binding.DDM_OK
    assert bool(torch.isfinite(o).all())


def test_plan_stats_time_both_steps():
    import torch
    H, W, N = 128, 128, 512
    frames = to_device(_frames(N, H, W, "u16", 3))
    plan = ddm.Plan(H, W, N, dtype="u16")
    D = torch.empty(plan.n_q * N, device="cuda")
    with pytest.raises(ddm.DDMError):
        plan.enable_stats(True)
        plan.stats()                                  # nothing recorded yet
    plan.structure_function(frames, D)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    plan.structure_function(frames, D)
    e.record()
    one, two = plan.stats()
    torch.cuda.synchronize()
    total = s.elapsed_time(e)
    assert one > 0 and two > 0
    assert one + two <= total * 1.05 + 0.05
    assert one + two >= total * 0.5
    plan.enable_stats(False)
