"""Pins of the oracle's multi-component operations against exact rationals.

Each real operation is "exact result rounded to L limbs", so its relative error
is below 2^(2-53L) (add, sub, mul) and 2^(4-53L) (long division), also under
cancellation.  Complex operations follow Eq. (1) (4M), Eq. (2) (3M), the
reciprocal (a - bi)/(a^2 + b^2) and cabs1; their bounds are stated per test.
"""
from fractions import Fraction

import numpy as np
import pytest

from helpers import frac_col, is_nonoverlapping, rand_limbs

N = 1500


def _inputs(L, rng):
    a = rand_limbs(L, N, rng)
    b = rand_limbs(L, N, rng)
    k = N // 5
    b[:, :k] = -a[:, :k]                                  # exact cancellation
    b[0, k:2 * k] = -a[0, k:2 * k]                        # cancellation of the leading limbs
    return a, b


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_real_ops(orc, L, op):
    rng = np.random.default_rng(100 + L)
    a, b = _inputs(L, rng)
    if op == "div":
        b[0, b[0] == 0] = 1.0
    code = {"add": orc.OP_ADD, "sub": orc.OP_SUB, "mul": orc.OP_MUL, "div": orc.OP_DIV}[op]
    z = orc.real_op(code, a, b)
    bound = Fraction(2) ** ((4 if op == "div" else 2) - 53 * L)
    worst = Fraction(0)
    for j in range(N):
        x, y, r = frac_col(a, j), frac_col(b, j), frac_col(z, j)
        ex = {"add": x + y, "sub": x - y, "mul": x * y, "div": x / y if y != 0 else None}[op]
        if ex == 0:
            assert r == 0
            continue
        rel = abs(r - ex) / abs(ex)
        worst = max(worst, rel)
        assert rel <= bound, (op, L, j, float(rel))
        assert is_nonoverlapping(list(z[:, j]))
    assert worst > 0        # the test exercises rounding, not only exact cases


def _cinputs(L, rng, n=600):
    x = np.stack([rand_limbs(L, n, rng, -8, 8), rand_limbs(L, n, rng, -8, 8)])
    y = np.stack([rand_limbs(L, n, rng, -8, 8), rand_limbs(L, n, rng, -8, 8)])
    y[:, :, :50] = x[:, :, :50]
    return x, y


def _cval(z, j):
    return frac_col(z[0], j), frac_col(z[1], j)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_complex_products(orc, L):
    rng = np.random.default_rng(200 + L)
    x, y = _cinputs(L, rng)
    z4 = orc.cplx_op(orc.COP_MUL4M, x, y)
    z3 = orc.cplx_op(orc.COP_MUL3M, x, y)
    u = Fraction(2) ** (-53 * L)
    for j in range(x.shape[2]):
        ar, ai = _cval(x, j)
        br, bi = _cval(y, j)
        re, im = ar * br - ai * bi, ar * bi + ai * br
        r4, i4 = _cval(z4, j)
        # Eq. (1): two roundings per product and one per sum
        assert abs(r4 - re) <= 16 * u * (abs(ar * br) + abs(ai * bi))
        assert abs(i4 - im) <= 16 * u * (abs(ar * bi) + abs(ai * br))
        r3, i3 = _cval(z3, j)
        # Eq. (2): Re as 4M; Im carries the (|Re a|+|Im a|)(|Re b|+|Im b|) scale of the 3M form
        assert abs(r3 - re) <= 16 * u * (abs(ar * br) + abs(ai * bi))
        assert abs(i3 - im) <= 64 * u * (abs(ar) + abs(ai)) * (abs(br) + abs(bi))


@pytest.mark.parametrize("L", [2, 3, 4])
def test_complex_inv_div_abs1(orc, L):
    rng = np.random.default_rng(300 + L)
    x, y = _cinputs(L, rng)
    zi = orc.cplx_op(orc.COP_INV, y)
    zd = orc.cplx_op(orc.COP_DIV, x, y)
    za = orc.cplx_op(orc.COP_ABS1, x)
    u = Fraction(2) ** (-53 * L)
    for j in range(x.shape[2]):
        ar, ai = _cval(x, j)
        br, bi = _cval(y, j)
        d = br * br + bi * bi
        ir, ii = br / d, -bi / d
        gr, gi = _cval(zi, j)
        mag = abs(ir) + abs(ii)
        assert abs(gr - ir) <= 64 * u * mag and abs(gi - ii) <= 64 * u * mag
        qr, qi = (ar * br + ai * bi) / d, (ai * br - ar * bi) / d
        gr, gi = _cval(zd, j)
        mag = (abs(ar) + abs(ai)) * (abs(br) + abs(bi)) / d
        assert abs(gr - qr) <= 64 * u * mag and abs(gi - qi) <= 64 * u * mag
        ab = abs(ar) + abs(ai)
        ga, gz = _cval(za, j)
        assert gz == 0 and abs(ga - ab) <= 4 * u * ab


def test_special_values(orc):
    for L in (2, 3, 4):
        a = np.zeros((L, 4))
        a[0] = [1.0, -3.0, 0.5, 7.0]
        a[1, 1] = 2.0 ** -60
        one = np.zeros((L, 4))
        one[0] = 1.0
        zero = np.zeros((L, 4))
        assert np.array_equal(orc.real_op(orc.OP_MUL, a, one), a)
        assert np.array_equal(orc.real_op(orc.OP_ADD, a, zero), a)
        assert np.array_equal(orc.real_op(orc.OP_SUB, a, a), zero)
        assert np.array_equal(orc.real_op(orc.OP_DIV, a, one), a)
        # (1 + 2^-100) - 1 = 2^-100 exactly (DD has the bits; TD/QD too)
        p = np.zeros((L, 1))
        p[0, 0], p[1, 0] = 1.0, 2.0 ** -100
        m = np.zeros((L, 1))
        m[0, 0] = 1.0
        r = orc.real_op(orc.OP_SUB, p, m)
        assert r[0, 0] == 2.0 ** -100 and np.all(r[1:, 0] == 0)
