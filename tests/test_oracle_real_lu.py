"""Pins of the oracle's real LU and solve (one plane per limb): the real
multi-component LU that the complex one builds on (Sec. 1, Sec. 3).

* n <= 8: pivots equal those of exact rational GEPP with the |a| key (the
  complex exact GEPP on the matrix with zero imaginary part, whose cabs1 key
  is |a|); the solution is within kappa * c * n * u of the exact one.
* Known factors A = P^T L U (dyadic): pivots, L and U bit for bit, and
  A x = b, A^T y = c solved exactly for dyadic x, y.
* Random n up to 96: normwise backward error with the exact residual
  <= 16 n u.
* Real inputs through the complex oracle: the same pivots, factors within the
  GEPP rounding bound (the two differ only in how the reciprocal is rounded).
* A zero column: info = first zero pivot, as in exact GEPP.
"""
from fractions import Fraction

import numpy as np
import pytest

from helpers import U_EXP
from lu_cases import known_factor_case_real
from oracle import exact
from paper_2403_16013_gb300 import inputs


def _real(n, L, seed):
    return np.ascontiguousarray(inputs.gaussian_matrix(n, L, seed=seed)[0])


def _embed(Ar):
    """[L, cols, rows] real planes -> [2, L, cols, rows] complex with Im = 0."""
    return np.ascontiguousarray(np.stack([Ar, np.zeros_like(Ar)]))


def _frac_vec(x, col=0):
    L, n = x.shape[0], x.shape[2]
    return [sum((Fraction(float(x[l, col, i])) for l in range(L)), Fraction(0)) for i in range(n)]


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_real_small_exact_gepp(orc, L, n):
    Ar = _real(n, L, 140 + n + L)
    LU, ipiv, info, gap = orc.dgetrf(Ar)
    M = exact.matrix(_embed(Ar))
    eLU, eipiv, einfo, _ = exact.gepp(M)
    assert info == einfo == 0
    assert list(ipiv) == eipiv
    xr = np.arange(1, n + 1)
    b = inputs.exact_rhs(_embed(Ar), xr, np.zeros(n, np.int64), L_out=4)
    bL = np.ascontiguousarray(inputs.truncate_limbs(b, L)[0])
    x = orc.dgetrs(LU, ipiv, bL)
    ex = [z[0] for z in exact.solve(M, [(v, Fraction(0)) for v in _frac_vec(bL)])]
    got = _frac_vec(x)
    u = Fraction(2) ** -U_EXP[L]
    inv_cols = [exact.solve(M, [(Fraction(int(i == j)), Fraction(0)) for i in range(n)]) for j in range(n)]
    nrm = lambda rows: max(sum(exact.cabs1(z) for z in r) for r in rows)
    kappa = nrm(M) * nrm([[inv_cols[j][i] for j in range(n)] for i in range(n)])
    xnorm = max(abs(e) for e in ex)
    err = max(abs(g - e) for g, e in zip(got, ex))
    assert err <= 64 * n * kappa * u * xnorm


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("n", [1, 7, 24])
def test_real_known_factor_exact(orc, L, n):
    A, ipiv_ref, packed, xv = known_factor_case_real(n, L, seed=170 + n)
    LU, ipiv, info, _ = orc.dgetrf(A)
    assert info == 0
    assert np.array_equal(ipiv, ipiv_ref)
    assert np.array_equal(LU, packed)
    M = [[Fraction(float(A[0, j, i])) for j in range(n)] for i in range(n)]
    # A x = b and A^T y = c for dyadic x, y: b, c exact in the leading limb
    for trans in ("N", "T"):
        rhs = []
        for i in range(n):
            s = sum((M[i][j] if trans == "N" else M[j][i]) * int(xv[j]) for j in range(n))
            assert float(s) == s
            rhs.append(float(s))
        B = np.zeros((L, 1, n))
        B[0, 0] = rhs
        x = orc.dgetrs(LU, ipiv, B, trans)
        assert np.array_equal(x[0, 0], xv.astype(float)), trans
        assert np.all(x[1:] == 0)


def _backward_error_real(orc, Ar, x, b):
    A, X, Bc = _embed(Ar), _embed(x), _embed(b)
    R = orc.exact_residual(A, X, Bc, Lr=1)
    r = np.abs(R[0, 0, 0])
    anorm = np.abs(Ar[0]).sum(axis=0).max()
    xnorm = np.abs(x[0, 0]).max()
    return r.max() / (anorm * xnorm)


@pytest.mark.parametrize("L,n", [(2, 96), (3, 64), (4, 40)])
def test_real_backward_error_random(orc, L, n):
    Ar = _real(n, L, 15)
    xr = np.ones(n, np.int64)
    b = np.ascontiguousarray(inputs.truncate_limbs(inputs.exact_rhs(_embed(Ar), xr, np.zeros(n, np.int64),
                                                                     L_out=4), L)[0])
    LU, ipiv, info, _ = orc.dgetrf(Ar)
    x = orc.dgetrs(LU, ipiv, b)
    assert _backward_error_real(orc, Ar, x, b) <= 16 * n * 2.0 ** -U_EXP[L]
    assert np.abs(x[0, 0] - 1).max() < 1e6 * n * 2.0 ** -U_EXP[L]
    # the planted one-ulp error in a factor is caught
    LU[0, 5, 9] = np.nextafter(LU[0, 5, 9], np.inf)
    xbad = orc.dgetrs(LU, ipiv, b)
    assert _backward_error_real(orc, Ar, xbad, b) > 16 * n * 2.0 ** -U_EXP[L]


@pytest.mark.parametrize("L", [2, 3, 4])
def test_real_agrees_with_complex_oracle_on_real_inputs(orc, L):
    n = 48
    Ar = _real(n, L, 21)
    LUr, ipr, infor, _ = orc.dgetrf(Ar)
    LUc, ipc, infoc, _ = orc.zgetrf(_embed(Ar))
    assert infor == infoc == 0
    assert np.array_equal(ipr, ipc)
    assert np.all(LUc[1] == 0)                       # the complex path keeps Im exactly zero
    diff = np.abs((LUr - LUc[0]).sum(axis=0)).max()
    assert diff <= 2.0 ** 10 * n * 2.0 ** -U_EXP[L] * np.abs(Ar[0]).max() * max(1.0, np.abs(LUc[0, 0]).max())


def test_real_zero_column_info(orc):
    n, L = 12, 2
    Ar = _real(n, L, 22)
    Ar[:, 4, :] = 0.0
    LU, ipiv, info, _ = orc.dgetrf(Ar)
    eLU, eipiv, einfo, _ = exact.gepp(exact.matrix(_embed(Ar)))
    assert info == einfo == 5
    assert list(ipiv) == eipiv
