"""Pins of the seeded inputs: canonical limbs, exact right-hand sides (checked
against the oracle's superaccumulator residual and exact rationals), and the
ill-conditioned A = Q1 diag(sigma) Q2^H former (checked against exact rationals)."""
from fractions import Fraction

import numpy as np

from helpers import is_nonoverlapping
from oracle import exact
from paper_2403_16013_gb300 import inputs


def test_canonical_limbs():
    for gen in (lambda: inputs.uniform_matrix(16, 4, 0), lambda: inputs.gaussian_matrix(16, 4, 1),
                lambda: inputs.spread_matrix(16, 16, 4, 2), lambda: inputs.paper_matrix(16, 3, 3)):
        A = gen()
        for c in range(2):
            for j in range(A.shape[2]):
                for i in range(A.shape[3]):
                    assert is_nonoverlapping(list(A[c, :, j, i]))


def test_seeded_reproducible():
    assert np.array_equal(inputs.gaussian_matrix(8, 2, 5), inputs.gaussian_matrix(8, 2, 5))
    assert not np.array_equal(inputs.gaussian_matrix(8, 2, 5), inputs.gaussian_matrix(8, 2, 6))


def test_exact_rhs_against_fractions_and_oracle(orc):
    n, L = 12, 3
    A = inputs.spread_matrix(n, n, L, seed=7)
    xr, xi = inputs.paper_x_true(n)
    b = inputs.exact_rhs(A, xr, xi, L_out=4)
    M = exact.matrix(A)
    for i in range(n):
        s = (Fraction(0), Fraction(0))
        for j in range(n):
            p = exact.cmul(M[i][j], (Fraction(int(xr[j])), Fraction(int(xi[j]))))
            s = (s[0] + p[0], s[1] + p[1])
        for c in range(2):
            rem = s[c]
            for l in range(4):
                want = float(rem)
                assert b[c, l, 0, i] == want
                rem -= Fraction(want)
    X = inputs.int_vector_planes(xr, xi, 1)
    R = orc.exact_residual(A, X, b, Lr=1)
    tail = np.abs(b[:, 3, 0, :])
    assert np.all(np.abs(R[:, 0, 0, :]) <= tail * 2.0 ** -52 + 1e-300)


def test_ill_conditioned_former_against_exact(orc):
    n, h = 6, 2
    V1 = inputs.householder_vectors(n, h, seed=3)
    V2 = inputs.householder_vectors(n, h, seed=4)
    r = inputs.geometric_ratio(n, decades=10.0)
    A = orc.make_ill_conditioned(4, n, V1, V2, r)

    def reflect_left(M, v):
        vv = [(Fraction(v[0, i]), Fraction(v[1, i])) for i in range(n)]
        w = Fraction(2) / sum(a * a + b * b for a, b in vv)
        for s in range(n):
            d = (Fraction(0), Fraction(0))
            for i in range(n):
                p = exact.cmul(exact.conj(vv[i]), M[i][s])
                d = (d[0] + p[0], d[1] + p[1])
            for i in range(n):
                p = exact.cmul(vv[i], d)
                M[i][s] = (M[i][s][0] - w * p[0], M[i][s][1] - w * p[1])

    def conjT(M):
        return [[exact.conj(M[j][i]) for j in range(n)] for i in range(n)]

    S = [[(Fraction(r) ** i if i == j else Fraction(0), Fraction(0)) for j in range(n)] for i in range(n)]
    # A = Q1 S Q2^H with Q = H_1 ... H_h:  (S Q2^H) = (Q2 S^H)^H
    T = conjT(S)
    for j in range(h - 1, -1, -1):
        reflect_left(T, V2[j])
    T = conjT(T)
    for j in range(h - 1, -1, -1):
        reflect_left(T, V1[j])
    u = 2.0 ** -209
    for i in range(n):
        for j in range(n):
            g = exact.element(A, i, j)
            e = T[i][j]
            assert abs(float(g[0] - e[0])) <= 1e3 * u and abs(float(g[1] - e[1])) <= 1e3 * u
