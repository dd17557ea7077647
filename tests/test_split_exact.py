"""The tensor-core forward of the seed network feeds each FP32 activation h to a bf16 MMA as
three terms, each the upper 16 bits of an FP32 pattern: hi = h with the low 16 bits cleared,
mid = the same of the FP32 remainder r = h - hi, lo = r - mid.  The claim behind its parity:
for |h| >= 2^-103 the three sum to h exactly (lo then has at most 8 significant bits and is a
normal number), so every product with a bf16 weight is exact in FP32; below that the dropped
subnormal bits of lo are worth less than 2^-133.  Checked here on the host, bit for bit."""
import numpy as np


MASK = np.uint32(0xFFFF0000)


def _split(h):
    """The three bf16 terms the MMA receives (upper 16 bits of each FP32 pattern)."""
    h = np.asarray(h, np.float32)
    hi = (h.view(np.uint32) & MASK).view(np.float32)
    r = (h - hi).astype(np.float32)
    mid = (r.view(np.uint32) & MASK).view(np.float32)
    lo = ((r - mid).astype(np.float32).view(np.uint32) & MASK).view(np.float32)
    return hi, mid, lo


def test_three_bf16_terms_sum_exactly():
    rng = np.random.Generator(np.random.PCG64(17))
    mant = rng.uniform(1.0, 2.0, 200_000)
    expo = rng.integers(-103, 127, 200_000)
    sign = rng.choice([-1.0, 1.0], 200_000)
    h = (sign * mant * np.exp2(expo)).astype(np.float32)
    h = np.concatenate([h, np.float32([0.0, -0.0, 1.0, -1.0, 3.0e38, 2.0 ** -103, 65504.0])])
    hi, mid, lo = _split(h)
    s = hi.astype(np.float64) + mid.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(s, h.astype(np.float64))


def test_tiny_activations_lose_less_than_2_to_minus_133():
    rng = np.random.Generator(np.random.PCG64(19))
    h = (rng.uniform(1.0, 2.0, 50_000) * np.exp2(rng.integers(-126, -103, 50_000))).astype(np.float32)
    hi, mid, lo = _split(h)
    s = hi.astype(np.float64) + mid.astype(np.float64) + lo.astype(np.float64)
    assert np.max(np.abs(s - h.astype(np.float64))) < 2.0 ** -133


def test_products_with_bf16_weights_are_exact_in_fp32():
    rng = np.random.Generator(np.random.PCG64(18))
    h = rng.normal(0, 3, 50_000).astype(np.float32)
    w = rng.normal(0, 0.2, 50_000).astype(np.float32)
    w = (w.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)   # a bf16 weight
    for t in _split(h):
        p32 = (t * w).astype(np.float32)
        assert np.array_equal(p32.astype(np.float64), t.astype(np.float64) * w.astype(np.float64))
