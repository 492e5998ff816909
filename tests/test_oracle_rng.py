"""Pins for the oracle's random-number layer: Philox4x32-10, the (0,1) uniform,
the fixed-point -log(u) of Eq. sampling, and Lemire's bounded integers."""
import math
import os

import mpmath
import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_uniform_exact_and_open():
    # (2j+1) 2^-53 for j = the top 52 bits of hi:lo
    assert oracle.uniform(0, 0) == 2.0 ** -53
    assert oracle.uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.uniform(0, 0x80000000) == 0.5 + 2.0 ** -53
    rng = np.random.default_rng(0)
    for lo, hi in rng.integers(0, 2 ** 32, size=(200, 2), dtype=np.uint64):
        j = ((int(hi) << 32) | int(lo)) >> 12
        assert oracle.uniform(int(lo), int(hi)) == (2 * j + 1) / 2.0 ** 53


def test_log_tables_match_300_bit_arithmetic():
    L = oracle.lib()
    mpmath.mp.prec = 300
    for i in range(128):
        r = L.orc_recip(i)
        # reciprocal of the centre 1 + (2i+1)/256 of the i-th sub-interval, x1024, rounded
        assert r == int(mpmath.nint(mpmath.mpf(1024) / (1 + mpmath.mpf(2 * i + 1) / 256)))
        exact = mpmath.log(mpmath.mpf(1024) / r) * mpmath.mpf(2) ** 62
        assert L.orc_logr_q62(i) == int(mpmath.nint(exact))
    assert L.orc_ln2_q62() == int(mpmath.nint(mpmath.log(2) * mpmath.mpf(2) ** 62))


def _edge_js():
    js = [0, 1, 2, 3, (1 << 52) - 1, (1 << 52) - 2, (1 << 51), (1 << 51) - 1]
    for n in range(0, 53):
        x = 1 << n                      # x = 2j+1 near powers of two
        for d in (-3, -1, 1, 3):
            if 1 <= x + d < (1 << 53) and (x + d) % 2 == 1:
                js.append((x + d - 1) // 2)
    for i in range(128):                # table sub-interval edges at top binade
        M = (1 << 52) + (i << 45)
        for d in (-1, 1):
            x = M + d
            if x % 2 == 1:
                js.append((x - 1) // 2)
    return js


def test_neglog_accuracy_against_300_bit_log():
    """The Q58 fixed-point value is within 4 units (2^-56) of -ln(u); the double returned is
    that value rounded once to nearest, so within half an ulp more."""
    L = oracle.lib()
    mpmath.mp.prec = 200
    rng = np.random.default_rng(1)
    js = _edge_js() + [int(v) for v in rng.integers(0, 1 << 52, size=4000, dtype=np.uint64)]
    # also concentrate on small u (large E) and u near 1 (small E)
    js += [int(v) >> int(s) for v, s in zip(rng.integers(0, 1 << 52, size=1000, dtype=np.uint64),
                                               rng.integers(0, 52, size=1000))]
    worst = 0.0
    for j in js:
        u = mpmath.mpf(2 * j + 1) / mpmath.mpf(2) ** 53
        exact = -mpmath.log(u)
        q = L.orc_neglog_q58(j)
        err_q = abs(mpmath.mpf(q) / mpmath.mpf(2) ** 58 - exact) * mpmath.mpf(2) ** 58
        worst = max(worst, float(err_q))
        assert err_q <= 4, (j, q, exact)          # 4 units of 2^-58
        got = oracle.neglog(j)
        assert got == math.ldexp(float(q), -58)   # one round-to-nearest
        assert got > 0.0
        assert abs(mpmath.mpf(got) - exact) <= math.ulp(got) / 2 + 2.0 ** -55
    assert worst <= 4


def test_neglog_is_exponential():
    # E = -log(u) of a uniform is Exp(1): check mean / variance / tail on 2e5 draws
    rng = np.random.default_rng(2)
    js = rng.integers(0, 1 << 52, size=200_000, dtype=np.uint64)
    E = np.array([oracle.neglog(int(j)) for j in js])
    n = E.size
    assert abs(E.mean() - 1.0) < 4 / math.sqrt(n)
    assert abs(E.var() - 1.0) < 4 * math.sqrt(8 / n)
    assert abs((E > 3.0).mean() - math.exp(-3.0)) < 4 * math.sqrt(math.exp(-3.0) / n)


def test_lemire_is_uniform_and_bounded():
    L = oracle.lib()
    from scipy import stats
    s = 7
    draws = np.array([L.orc_lemire_draw(5, 0, e, 3, s, 0) for e in range(70_000)])
    assert draws.min() >= 0 and draws.max() < s
    cnt = np.bincount(draws, minlength=s)
    assert stats.chisquare(cnt).pvalue > 1e-4
    # a range that forces rejections often: s = 2^31 + 1 (reject probability ~ 1/2)
    big = (1 << 31) + 1
    d2 = np.array([L.orc_lemire_draw(5, 0, e, 3, big, 0) for e in range(20_000)])
    assert d2.max() < big
    assert abs(d2.mean() / big - 0.5) < 4 * math.sqrt(1 / 12 / d2.size)
