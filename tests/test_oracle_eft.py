"""Pins of the oracle's error-free transformations and normalisation.

TwoSum: s = RN(a+b) and a + b = s + e exactly, for every pair of doubles.
TwoProd: p = RN(a*b) and a*b = p + e exactly, whenever e is not below the
normal range.  VecSum normalisation: the exact sum is kept and the output is a
nonoverlapping expansion in decreasing magnitude.  All checked with exact
rational arithmetic (fractions.Fraction) on random and edge-case doubles.
"""
from fractions import Fraction

import numpy as np

from helpers import is_nonoverlapping

EDGE = [0.0, -0.0, 1.0, -1.0, 0.5, 3.0, 1.0 / 3.0, 2.0 ** -1022, 5e-324, -5e-324, 3 * 2.0 ** -1074,
        2.0 ** 1000, -(2.0 ** 1000), 2.0 ** 53, 2.0 ** 53 + 2, 1 + 2.0 ** -52, 1 - 2.0 ** -53, 2.0 ** -60,
        2.0 ** 60, 1e300, -1e-300, 0.1, 0.7]


def _pairs(rng, n):
    a = np.ldexp(rng.uniform(-1, 1, n), rng.integers(-500, 501, n))
    b = np.ldexp(rng.uniform(-1, 1, n), rng.integers(-500, 501, n))
    # near cancellation, equal exponents, and half-ulp ties
    k = n // 4
    b[:k] = -a[:k] * (1 + np.ldexp(rng.uniform(-1, 1, k), -40))
    b[k:2 * k] = np.ldexp(a[k:2 * k], -53)
    b[2 * k:3 * k] = a[2 * k:3 * k] * rng.uniform(0.5, 2, k)
    ea = np.array(EDGE)
    A, B = np.meshgrid(ea, ea)
    return np.concatenate([a, A.ravel()]), np.concatenate([b, B.ravel()])


def test_two_sum_exact(orc):
    rng = np.random.default_rng(11)
    a, b = _pairs(rng, 60000)
    s, e, _, _ = orc.eft(a, b)
    assert np.array_equal(s, a + b)
    for x, y, sx, ex in zip(a.tolist(), b.tolist(), s.tolist(), e.tolist()):
        assert Fraction(x) + Fraction(y) == Fraction(sx) + Fraction(ex)


def test_two_prod_exact(orc):
    rng = np.random.default_rng(12)
    a, b = _pairs(rng, 60000)
    _, _, p, f = orc.eft(a, b)
    assert np.array_equal(p, a * b)
    checked = 0
    for x, y, px, fx in zip(a.tolist(), b.tolist(), p.tolist(), f.tolist()):
        prod = Fraction(x) * Fraction(y)
        if prod != 0 and abs(prod) < Fraction(2) ** -969:
            continue            # the error term would be subnormal: not representable
        if abs(px) == float("inf"):
            continue
        assert prod == Fraction(px) + Fraction(fx)
        checked += 1
    assert checked > 50000


def test_normalize_exact_and_nonoverlapping(orc):
    rng = np.random.default_rng(13)
    rows = []
    for m in range(1, 24):
        for _ in range(300):
            v = np.ldexp(rng.uniform(-1, 1, m), rng.integers(-80, 81, m))
            if m > 2 and rng.uniform() < 0.5:      # planted cancellations
                v[1] = -v[0] * (1 + 2.0 ** -45)
                v[-1] = -v[-2]
            row = np.zeros(24)
            row[:m] = v
            rows.append(row)
    V = np.array(rows)
    out, ln = orc.normalize_rows(V)
    assert orc.lib().orc_error_flag() == 0
    for r in range(V.shape[0]):
        ex = sum((Fraction(x) for x in V[r].tolist()), Fraction(0))
        got = sum((Fraction(x) for x in out[r, :ln[r]].tolist()), Fraction(0))
        assert ex == got
        comp = out[r, :ln[r]]
        assert np.all(comp != 0)
        assert is_nonoverlapping(list(comp))
        assert np.all(np.abs(comp[1:]) <= np.abs(comp[:-1]))


def test_exact_sum_rows_greedy_rounding(orc):
    """Superaccumulator: limb k is RN(exact - limbs before it), checked with Fractions."""
    rng = np.random.default_rng(14)
    V = np.ldexp(rng.uniform(-1, 1, (400, 40)), rng.integers(-300, 301, (400, 40)))
    V[::3, 1] = -V[::3, 0]
    V[::5, :20] = np.ldexp(V[::5, :20], -60)
    out = orc.exact_sum_rows(V, 4)
    for r in range(V.shape[0]):
        ex = sum((Fraction(x) for x in V[r].tolist()), Fraction(0))
        for k in range(4):
            want = float(ex)            # Fraction -> float is correctly rounded (ties to even)
            assert out[r, k] == want, (r, k)
            ex -= Fraction(want)
