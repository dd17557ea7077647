"""The device renderings of the synthetic workloads (used where the host would take minutes
per stack) against the host generators of the same law, through the oracle's D.  Run on
the CPU: torch renders on any device."""
import numpy as np

import oracle
import synth


def _radial_D(frames, nb):
    D = oracle.sf_direct(oracle.dft2(frames))
    return oracle.radial_average(D, nb)[0]


def test_blob_torch_generator_matches_the_host_generator():
    """Six stacks from each generator (independent seeds), 64x64x128, 90 blobs, D0 = 0.2:
    the seed-averaged radial D agrees bin by bin within 10 % and on average within 3 % at
    lags 1, 4, 16 and 64 (a wrong step size, blob width, amplitude or background shows up
    as a lag- or q-dependent ratio far from 1)."""
    H = W = 64
    N, nb = 128, 23
    Rt, Rn = [], []
    for s in range(6):
        Rt.append(_radial_D(synth.blob_stack_torch(H, W, N, 90, 2.0, 0.2, s, device="cpu").numpy(), nb))
        Rn.append(_radial_D(synth.blob_stack(H, W, N, 90, 2.0, 0.2, 100 + s), nb))
    Rt, Rn = np.mean(Rt, axis=0), np.mean(Rn, axis=0)
    for m in (1, 4, 16, 64):
        r = Rt[2:16, m] / Rn[2:16, m]
        assert np.all(np.abs(r - 1) < 0.10), (m, r)
        assert abs(r.mean() - 1) < 0.03, (m, r.mean())


def test_blob_torch_generator_counts_and_drift():
    fr = synth.blob_stack_torch(32, 48, 40, 30, 2.0, 0.5, 1, device="cpu", drift=0.05).numpy()
    assert fr.dtype == np.uint16 and fr.shape == (40, 32, 48)
    assert fr.max() <= 4095
    m0, m1 = fr[:5].mean(), fr[-5:].mean()
    assert abs(m0 - 2000) < 40 and abs(m1 / m0 - 1.05) < 0.02     # the 5 % illumination ramp
    a = synth.blob_stack_torch(32, 48, 10, 30, 2.0, 0.5, 7, device="cpu").numpy()
    b = synth.blob_stack_torch(32, 48, 10, 30, 2.0, 0.5, 7, device="cpu").numpy()
    np.testing.assert_array_equal(a, b)                           # seeded
