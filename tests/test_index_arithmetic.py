"""The integrator divides flat indices by a run-time row length without the integer divide: for
e < d^2 and d < 64 (the LU's trailing block and the Jacobian's species block, at most 63 rows:
62 species plus temperature), q = e / d is the high word of e * m with m = ceil(2^32 / d) formed
in 32 bits as (2^32 - 1) / d + 1 (which wraps to 0 for d = 1, where only e = 0 occurs).  The
identity is checked here for every (d, e) those loops can see, in the kernel's unsigned 32-bit
arithmetic, together with the bound that makes it exact (e * d < 2^32)."""
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
    # the error term of the round-up reciprocal stays below 1/d while e * d < 2^32
    assert 63 * 63 * 63 < 2 ** 32
    assert _magic(1) == 0 and _umulhi(0, _magic(1)) == 0
    # powers of two: the magic number is 2^32 / d exactly
    for k in range(1, 6):
        assert int(_magic(2 ** k)) == 2 ** 32 // 2 ** k
