"""Pins of the oracle's LU, solve, ZGEMM and adjoint (Sec. 2.1, Sec. 3, Sec. 4).

* n <= 8: pivots equal those of exact rational GEPP with the cabs1 key; the
  computed solution is within kappa * c * n * u of the exact one.
* Known factors A = P^T L U (dyadic): pivots, L and U reproduced bit for bit,
  and A x = b, A^H y = c solved exactly for dyadic x.
* Random n up to 96: normwise backward error with the exact residual
  <= 16 n u (u = 2^-104, 2^-157, 2^-209).
* ZGEMM 4M and 3M (Eq. 3) against exact entries, with the componentwise 4M
  bound and the normwise 3M bound; 3M and 4M agree within the sum of bounds.
* Adjoint: lambda = A^{-H} xbar and Abar = -lambda x^H against exact rationals.
* The per-step pivot-key gap the oracle records equals exact GEPP's; an
  exact tie gives 0 and a constructed gap its value.
* The exact P A - L U checker (orc_exact_entries in L U mode) gives 0 on
  known factors and exactly the planted change after a one-ulp edit.
"""
from fractions import Fraction

import numpy as np
import pytest

from helpers import U_EXP
from lu_cases import known_factor_case
from oracle import exact
from paper_2403_16013_gb300 import inputs


def _frac_planes(X, col=0):
    L, n = X.shape[1], X.shape[3]
    return [(sum((Fraction(float(X[0, l, col, i])) for l in range(L)), Fraction(0)),
             sum((Fraction(float(X[1, l, col, i])) for l in range(L)), Fraction(0))) for i in range(n)]


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_small_exact_gepp(orc, L, n):
    A = inputs.gaussian_matrix(n, L, seed=40 + n + L)
    LU, ipiv, info, gap = orc.zgetrf(A)
    M = exact.matrix(A)
    eLU, eipiv, einfo, egaps = exact.gepp(M)
    assert info == einfo == 0
    assert list(ipiv) == eipiv
    xr, xi = inputs.ones_x_true(n)
    b = inputs.exact_rhs(A, xr, xi, L_out=4)
    bL = inputs.truncate_limbs(b, L)
    x = orc.zgetrs(LU, ipiv, bL)
    ex = exact.solve(M, _frac_planes(bL))
    got = _frac_planes(x)
    u = Fraction(2) ** -U_EXP[L]
    # kappa_inf(A) from the exact inverse
    inv_cols = [exact.solve(M, [(Fraction(int(i == j)), Fraction(0)) for i in range(n)]) for j in range(n)]
    nrm = lambda rows: max(sum(exact.cabs1(z) for z in r) for r in rows)
    kappa = nrm(M) * nrm([[inv_cols[j][i] for j in range(n)] for i in range(n)])
    xnorm = max(exact.cabs1(z) for z in ex)
    err = max(exact.cabs1(exact.csub(g, e)) for g, e in zip(got, ex))
    assert err <= 64 * n * kappa * u * xnorm


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("n", [1, 7, 24])
def test_known_factor_exact(orc, L, n):
    A, ipiv_ref, packed, xr, xi = known_factor_case(n, L, seed=70 + n)
    LU, ipiv, info, _ = orc.zgetrf(A)
    assert info == 0
    assert np.array_equal(ipiv, ipiv_ref)
    assert np.array_equal(LU, packed)
    b = inputs.exact_rhs(A, xr, xi, L_out=L)
    assert np.all(b[:, 1:] == 0)                 # dyadic b fits in the leading limb
    x = orc.zgetrs(LU, ipiv, b, "N")
    assert np.array_equal(x[0, 0, 0], xr.astype(float)) and np.array_equal(x[1, 0, 0], xi.astype(float))
    assert np.all(x[:, 1:] == 0)
    # A^H y = c with c = A^H y_true for dyadic y_true: compute c exactly via Fractions
    M = exact.matrix(A)
    y_true = [(Fraction(int(a)), Fraction(int(c))) for a, c in zip(xr[::-1], xi[::-1])]
    c = []
    for j in range(n):
        s = (Fraction(0), Fraction(0))
        for i in range(n):
            p = exact.cmul(exact.conj(M[i][j]), y_true[i])
            s = (s[0] + p[0], s[1] + p[1])
        c.append(s)
    C = np.zeros((2, L, 1, n))
    for i, (re, im) in enumerate(c):
        assert float(re) == re and float(im) == im
        C[0, 0, 0, i], C[1, 0, 0, i] = float(re), float(im)
    y = orc.zgetrs(LU, ipiv, C, "C")
    assert [(Fraction(y[0, 0, 0, i]), Fraction(y[1, 0, 0, i])) for i in range(n)] == y_true


def _backward_error(orc, A, x, b):
    R = orc.exact_residual(A, x, b, Lr=1)
    r = np.abs(R[0, 0, 0]) + np.abs(R[1, 0, 0])
    Ah = np.abs(A[0, 0]) + np.abs(A[1, 0])          # [cols, rows]
    anorm = Ah.sum(axis=0).max()
    xnorm = (np.abs(x[0, 0, 0]) + np.abs(x[1, 0, 0])).max()
    return r.max() / (anorm * xnorm)


@pytest.mark.parametrize("L,n", [(2, 96), (3, 64), (4, 40)])
def test_backward_error_random(orc, L, n):
    A = inputs.gaussian_matrix(n, L, seed=5)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    LU, ipiv, info, gap = orc.zgetrf(A)
    x = orc.zgetrs(LU, ipiv, b)
    eta = _backward_error(orc, A, x, b)
    assert eta <= 16 * n * 2.0 ** -U_EXP[L]
    # forward error against x_true (well-conditioned random matrix)
    fe = max(np.abs(x[0, 0, 0] - 1).max(), np.abs(x[1, 0, 0] - 1).max())
    assert fe < 1e6 * n * 2.0 ** -U_EXP[L]


def test_backward_error_detects_planted_mistake(orc):
    """A perturbed factor (one limb off by an ulp) is caught by the residual check."""
    L, n = 2, 32
    A = inputs.gaussian_matrix(n, L, seed=6)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    LU, ipiv, info, _ = orc.zgetrf(A)
    LU[0, 0, 5, 9] = np.nextafter(LU[0, 0, 5, 9], np.inf)
    x = orc.zgetrs(LU, ipiv, b)
    assert _backward_error(orc, A, x, b) > 16 * n * 2.0 ** -U_EXP[L]


@pytest.mark.parametrize("L", [2, 3, 4])
def test_zgemm_4m_3m_against_exact(orc, L):
    m, n, k = 9, 7, 13
    A = inputs.gaussian_matrix(k, L, seed=8, rows=m)
    B = inputs.gaussian_matrix(n, L, seed=9, rows=k)
    Cin = inputs.gaussian_matrix(n, L, seed=10, rows=m)
    C4 = orc.zgemm(A, B, method="4m")
    C3 = orc.zgemm(A, B, method="3m")
    D4 = orc.zgemm(A, B, Cin, method="4m")
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    ex = orc.exact_entries(A, B, rows, cols)
    exd = orc.exact_entries(A, B, rows, cols, C=Cin, sign=-1)
    u = 2.0 ** (-53 * L)
    absA = np.abs(A[:, 0])            # [2, k, m]
    absB = np.abs(B[:, 0])            # [2, n, k]
    for s, (i, j) in enumerate(zip(rows, cols)):
        rr = absA[0, :, i] @ absB[0, j, :] + absA[1, :, i] @ absB[1, j, :]
        ri = absA[0, :, i] @ absB[1, j, :] + absA[1, :, i] @ absB[0, j, :]
        s3 = (absA[0, :, i] + absA[1, :, i]) @ (absB[0, j, :] + absB[1, j, :])
        e_re = sum(Fraction(v) for v in ex[s, 0])
        e_im = sum(Fraction(v) for v in ex[s, 1])
        g = lambda C, c: sum(Fraction(float(C[c, l, j, i])) for l in range(L))
        tol4_re, tol4_im = 4 * (k + 2) * u * rr * 1.01, 4 * (k + 2) * u * ri * 1.01
        assert abs(float(g(C4, 0) - e_re)) <= tol4_re
        assert abs(float(g(C4, 1) - e_im)) <= tol4_im
        assert abs(float(g(C3, 0) - e_re)) <= tol4_re
        tol3 = 8 * (k + 4) * u * s3 * 1.01
        assert abs(float(g(C3, 1) - e_im)) <= tol3
        assert abs(float(g(C3, 1) - g(C4, 1))) <= tol3 + tol4_im
        d_re = sum(Fraction(v) for v in exd[s, 0])
        cre = sum(Fraction(float(Cin[0, l, j, i])) for l in range(L))
        assert abs(float(g(D4, 0) - d_re)) <= tol4_re + 4 * u * abs(float(cre))


@pytest.mark.parametrize("L", [2, 4])
def test_adjoint_exact(orc, L):
    n = 6
    A = inputs.gaussian_matrix(n, L, seed=21)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    LU, ipiv, info, _ = orc.zgetrf(A)
    x = orc.zgetrs(LU, ipiv, b)
    cvec = inputs.complex_gaussian_vector(n, L, seed=22)
    lam, Abar = orc.adjoint(LU, ipiv, x, cvec)
    M = exact.matrix(A)
    lam_ex = exact.solve_adjoint(M, _frac_planes(cvec))
    xs = _frac_planes(x)
    u = 2.0 ** -U_EXP[L]
    scale = max(float(exact.cabs1(z)) for z in lam_ex)
    got = _frac_planes(lam)
    assert max(float(exact.cabs1(exact.csub(g, e))) for g, e in zip(got, lam_ex)) <= 1e4 * u * scale
    xsc = max(float(exact.cabs1(z)) for z in xs)
    for i in range(n):
        for j in range(n):
            want = exact.cmul(lam_ex[i], exact.conj(xs[j]))
            want = (-want[0], -want[1])
            g = (sum(Fraction(float(Abar[0, l, j, i])) for l in range(L)),
                 sum(Fraction(float(Abar[1, l, j, i])) for l in range(L)))
            assert float(exact.cabs1(exact.csub(g, want))) <= 1e4 * u * scale * xsc


def test_zero_pivot_info(orc):
    n, L = 5, 2
    A = inputs.gaussian_matrix(n, L, seed=3)
    A[:, :, 2, :] = 0.0                     # column 2 identically zero -> info = 3
    LU, ipiv, info, _ = orc.zgetrf(A)
    assert info == 3
    M = exact.matrix(A)
    _, eipiv, einfo, _ = exact.gepp(M)
    assert einfo == 3 and list(ipiv) == eipiv


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("n", [2, 5, 8])
def test_pivot_gap_against_exact(orc, L, n):
    """The oracle's per-step gap between the two largest pivot keys equals the
    exact rational GEPP's relative gap (k1 - k2) / k1 to binary64 resolution,
    at every step of the elimination (1 where fewer than two candidates)."""
    A = inputs.gaussian_matrix(n, L, seed=140 + n + L)
    _, ipiv, _, gap = orc.zgetrf(A)
    _, eipiv, _, egaps = exact.gepp(exact.matrix(A))
    assert list(ipiv) == eipiv
    for k in range(n):
        assert abs(gap[k] - float(egaps[k])) <= 2.0 ** -50, (k, gap[k], float(egaps[k]))
    assert gap[n - 1] == 1.0


@pytest.mark.parametrize("L", [2, 4])
def test_pivot_gap_tie_and_clear_gap(orc, L):
    """Constructed first columns: an exact tie of the two largest cabs1 keys
    (1 + 2i and -2 + 1i, both 3) gives gap 0 and the lower row; keys 4 and 3
    give gap exactly 1/4; a zero column gives gap 1 (k1 = 0)."""
    n = 5
    A = inputs.gaussian_matrix(n, L, seed=150)
    A[:, :, 0, :] = 0.0
    col = [(0.5, 0.25), (1.0, 2.0), (0.25, -0.5), (-2.0, 1.0), (0.0, 1.0)]
    for i, (re, im) in enumerate(col):
        A[0, 0, 0, i], A[1, 0, 0, i] = re, im
    _, ipiv, _, gap = orc.zgetrf(A)
    assert ipiv[0] == 2 and gap[0] == 0.0           # tie: rows 1 and 3, the lower index wins
    col = [(0.5, 0.25), (3.0, -1.0), (0.25, -0.5), (-2.0, 1.0), (0.0, 1.0)]
    for i, (re, im) in enumerate(col):
        A[0, 0, 0, i], A[1, 0, 0, i] = re, im
    _, ipiv, _, gap = orc.zgetrf(A)
    assert ipiv[0] == 2 and gap[0] == 0.25           # keys 4 (row 1) and 3 (row 3)
    A[:, :, 0, :] = 0.0
    _, ipiv, info, gap = orc.zgetrf(A)
    assert info == 1 and ipiv[0] == 1 and gap[0] == 1.0


@pytest.mark.parametrize("L", [2, 4])
def test_exact_entries_lower_unit_known_factors(orc, L):
    """orc_exact_entries in its L U mode (unit lower L, upper U, both read from
    one packed array): on known factors with P A = L U exactly it returns 0
    at every position; after a one-ulp change of one entry of L (or of U) it
    returns exactly the change times the matching row of U (column of L) at
    the affected positions and 0 elsewhere."""
    from fractions import Fraction
    n = 12
    A, ipiv, packed, _, _ = known_factor_case(n, L, seed=160)
    P = np.arange(n)
    for k, p in enumerate(ipiv - 1):
        P[k], P[p] = P[p], P[k]
    PA = np.ascontiguousarray(A[:, :, :, P])
    rows, cols = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    d = orc.exact_entries(packed, packed, rows, cols, C=PA, sign=-1, lu=True)
    assert np.all(d == 0.0)

    def check(LU, expect):
        d = orc.exact_entries(LU, LU, rows, cols, C=PA, sign=-1, lu=True)
        for s, (i, j) in enumerate(zip(rows, cols)):
            want = expect.get((int(i), int(j)), (Fraction(0), Fraction(0)))
            got = tuple(sum((Fraction(float(v)) for v in d[s, c]), Fraction(0)) for c in range(2))
            assert got == want, (i, j, got, want)

    # L entry (r, q), r > q, raised by one ulp (real): P A - L U changes by -delta U[q, c] for c >= q
    r, q = 9, 4
    LU = packed.copy()
    old = LU[0, 0, q, r]
    LU[0, 0, q, r] = np.nextafter(old, np.inf)
    delta = Fraction(float(LU[0, 0, q, r])) - Fraction(float(old))
    assert delta != 0
    expect = {(r, c): (-delta * Fraction(float(packed[0, 0, c, q])), -delta * Fraction(float(packed[1, 0, c, q])))
              for c in range(q, n)}
    check(LU, expect)
    # U entry (q, c0), imaginary part, raised by one ulp: changes -L[i, q] * i delta for i >= q (L[q, q] = 1)
    q, c0 = 3, 8
    LU = packed.copy()
    old = LU[1, 0, c0, q]
    LU[1, 0, c0, q] = np.nextafter(old, np.inf)
    delta = Fraction(float(LU[1, 0, c0, q])) - Fraction(float(old))
    expect = {}
    for i in range(q, n):
        lr = Fraction(1) if i == q else Fraction(float(packed[0, 0, q, i]))
        li = Fraction(0) if i == q else Fraction(float(packed[1, 0, q, i]))
        expect[(i, c0)] = (li * delta, -lr * delta)   # -(lr + i li)(i delta) = li delta - i lr delta
    check(LU, expect)
