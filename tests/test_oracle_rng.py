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


def test_draws_of_the_method_use_their_documented_counters(orc):
    """Every random draw of the method is one Philox4x64-10 block with key
    (seed, 0), its words turned into 53-bit uniforms (top bits) or into an
    index by a multiply-high: the initial velocity of clone c at site
    s = y nx + x is amp (2u - 1) from words 0 and 1 of counter (5, c, s, 0);
    the App. D weight alpha_n of slot s at iteration j is word 0 of
    (4, j, s, n); the AMS survivor of killed trajectory k at iteration j is
    the r-th of the N - |K| others, r = word 0 of (3, j, k, 0) times
    (N - |K|) over 2^64.  Checked against numpy's Philox."""
    def u01(w):
        return (w >> 11) / 2.0**53

    nx, ny, seed, clone, amp = 16, 8, 99, 3, 0.01
    c = orc.cfg(nx, ny, tau=0.6)
    _, ux, uy = orc.macro(c, orc.init(c, seed, clone, amp))
    for x, y in [(0, 0), (5, 3), (15, 7), (9, 1)]:
        b = numpy_block([5, clone, y * nx + x, 0], [seed, 0])
        assert abs(ux[y, x] - amp * (2 * u01(b[0]) - 1)) < 1e-15
        assert abs(uy[y, x] - amp * (2 * u01(b[1]) - 1)) < 1e-15
    alpha = orc.perturb_alphas(9, 3, 5, 4)
    for n in range(4):
        assert alpha[n] == u01(numpy_block([4, 3, 5, n], [9, 0])[0])
    Q = np.arange(8.0)  # trajectory 0 is killed; the survivor is one of 1..7
    for it in range(6):
        _, surv, _ = orc.ams_select(Q, 77, it)
        assert surv[0] == 1 + ((numpy_block([3, it, 0, 0], [77, 0])[0] * 7) >> 64)
