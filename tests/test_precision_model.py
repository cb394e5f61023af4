"""The arithmetic of the BF16 precision pattern, pinned on the CPU.

Every operand x of a tensor-core product is split x = hi + lo with
hi = bf16(x) and lo = bf16(x - hi) (round to nearest even, 8 significant bits),
and a product a*b is formed as hi_a*hi_b + hi_a*lo_b + lo_a*hi_b.

Split: with 2^e <= |x| < 2^(e+1), r = x - hi is exact and |r| <= 2^(e-8); if
|r| = 2^(e-8) then lo = r exactly, else r lies below 2^(e-8) and rounding it to
8 significant bits errs by at most 2^(e-17).  So |x - hi - lo| <= 2^-17 |x|, and
|lo| <= 2^-8 |x|.  Product: the partial products of bf16 values are exact in
FP32 (8 + 8 significant bits); the dropped lo_a*lo_b is at most 2^-16 |a||b|
and the two split errors add at most 2^-17 |a||b| each, so the three-term
product misses a*b by at most 2^-15 |a||b|.  These are the bounds the BF16
tolerances are derived from; the test also shows they are nearly attained.
"""
import numpy as np


def bf16_rn(x):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = bf16_rn(x)
    lo = bf16_rn((x - hi).astype(np.float32))
    return hi, lo


def samples(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-30, 30, n)
    sign = rng.choice([-1.0, 1.0], n)
    return (sign * mant * 2.0 ** expo).astype(np.float32)


def test_rounding_helper_matches_known_bfloat16_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties to even gives 1
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 3.0e38], np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 * 2.0 ** -7, 1.0, -2.5, np.float32(3.0e38)], np.float64)
    got = bf16_rn(x).astype(np.float64)
    assert np.all(np.abs(got[:5] - want[:5]) == 0), got
    assert np.isfinite(got[5]) and abs(got[5] - 3.0e38) <= 2.0 ** -8 * 3.0e38
    # every result has at most 8 significant bits
    assert np.all((bf16_rn(samples(1000, 0)).view(np.uint32) & 0xFFFF) == 0)


def test_split_error_bound_and_that_it_is_nearly_attained():
    x = samples(200000, 1)
    hi, lo = split(x)
    rel = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -17
    assert rel.max() > 2.0 ** -18  # nearly attained
    # the first rounding alone is within half an ulp of 8 significant bits
    assert (np.abs(x - hi) / np.abs(x)).max() <= 2.0 ** -8
    assert (np.abs(lo) / np.abs(x)).max() <= 2.0 ** -8


def test_compensated_product_error_bound():
    a, b = samples(200000, 2), samples(200000, 3)
    ah, al = split(a)
    bh, bl = split(b)
    # each partial product of bf16 values is exact in FP32
    for p, q in ((ah, bh), (ah, bl), (al, bh)):
        assert np.all((p.astype(np.float32) * q.astype(np.float32)).astype(np.float64)
                      == p.astype(np.float64) * q.astype(np.float64))
    approx = (ah.astype(np.float64) * bh + ah.astype(np.float64) * bl + al.astype(np.float64) * bh)
    exact = a.astype(np.float64) * b.astype(np.float64)
    rel = np.abs(approx - exact) / np.abs(exact)
    assert rel.max() <= 2.0 ** -15
    assert rel.max() > 2.0 ** -16
    # plain bf16 (hi only) loses far more: about 2^-8
    rel_hi = np.abs(ah.astype(np.float64) * bh - exact) / np.abs(exact)
    assert rel_hi.max() > 2.0 ** -9
