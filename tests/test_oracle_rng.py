"""Pins of the oracle's counter-based generator against a library routine.

numpy.random.Philox is Philox4x64-10 (Salmon et al., SC'11); a generator built
with counter c yields, as its first block, the Philox function of counter c+1.
"""
import numpy as np
import pytest

MASK = (1 << 64) - 1


def numpy_block(ctr, key):
    ctr_int = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    prev = (ctr_int - 1) % (1 << 256)
    words = [(prev >> (64 * i)) & MASK for i in range(4)]
    bg = np.random.Philox(key=np.array([int(key[0]), int(key[1])], dtype=np.uint64),
                          counter=np.array(words, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


@pytest.mark.parametrize("ctr,key", [
    ([1, 0, 0, 0], [0, 0]),
    ([5, 3, 17, 0], [12345, 0]),
    ([4, 2**40 + 7, 123456789, 9], [2**63 + 11, 0]),
    ([2, MASK, MASK, MASK], [MASK, MASK]),
    ([0, 1, 0, 0], [0xDEADBEEF, 0xCAFEBABE]),
])
def test_philox_matches_numpy(orc, ctr, key):
    got = [int(v) for v in orc.philox4x64(ctr, key)]
    assert got == numpy_block(ctr, key)


def test_philox_many_counters(orc):
    r = np.random.default_rng(7)
    for _ in range(200):
        ctr = [int(v) for v in r.integers(1, 2**63, size=4, dtype=np.int64)]
        key = [int(v) for v in r.integers(0, 2**63, size=2, dtype=np.int64)]
        assert [int(v) for v in orc.philox4x64(ctr, key)] == numpy_block(ctr, key)


def test_u01_is_top_53_bits(orc):
    for x in [0, 1, 2**11 - 1, 2**11, MASK, 0x8000000000000000, 123456789123456789]:
        assert orc.u01(x) == (x >> 11) / 2.0**53
    assert orc.u01(MASK) < 1.0


def test_below_is_multiply_high(orc):
    r = np.random.default_rng(3)
    for _ in range(500):
        x = int(r.integers(0, 2**63)) * 2 + int(r.integers(0, 2))
        m = int(r.integers(1, 2**31))
        assert orc.below(x, m) == (x * m) >> 64
    assert orc.below(MASK, 7) == 6
    assert orc.below(0, 7) == 0
