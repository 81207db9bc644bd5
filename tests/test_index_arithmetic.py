"""The integrator divides flat indices by a run-time row length without the integer divide: for
e < d^2 (the LU's trailing block, the Jacobian's species block), q = e / d is the high word of
e * m with m = ceil(2^32 / d) formed in 32 bits as (2^32 - 1) / d + 1 (which wraps to 0 for
d = 1, where only e = 0 occurs).  Exact while e * d < 2^32, i.e. for d up to 1625.  The identity
is checked here for every (d, e) with d < 64 (the mechanisms in use), in the kernel's unsigned
32-bit arithmetic, and at the edge of the bound."""
import numpy as np


def _magic(d):
    return np.uint32((0xFFFFFFFF // d + 1) & 0xFFFFFFFF)


def _umulhi(a, b):
    return np.uint32((int(a) * int(b)) >> 32)


def test_multiply_high_division_is_exact_for_every_index():
    for d in range(1, 64):
        m = _magic(d)
        e = np.arange(d * d, dtype=np.uint64)
        q = ((e * np.uint64(m)) >> np.uint64(32)).astype(np.int64)
        assert np.array_equal(q, (e // d).astype(np.int64)), d
        assert np.array_equal(e.astype(np.int64) - q * d, (e % d).astype(np.int64)), d


def test_exactness_bound_and_wrap():
    # the error term of the round-up reciprocal stays below 1/d while e * d < 2^32: d = 1625 is
    # the largest row length with d^3 < 2^32; check the largest indices there and a sample below
    assert 1625 ** 3 < 2 ** 32 < 1626 ** 3
    rng = np.random.default_rng(0)
    for d in (1625, 1024, 1000, 777, 170):
        m = _magic(d)
        for e in list(range(d * d - 64, d * d)) + list(rng.integers(0, d * d, 2000)):
            q = int(_umulhi(e, m))
            assert q == e // d, (d, e)
    assert _magic(1) == 0 and _umulhi(0, _magic(1)) == 0
    # powers of two: the magic number is 2^32 / d exactly
    for k in range(1, 6):
        assert int(_magic(2 ** k)) == 2 ** 32 // 2 ** k
