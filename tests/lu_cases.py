"""Constructed LU test cases with known answers (no multi-component arithmetic).

``known_factor_case`` builds A = P^T L U exactly: L unit lower with real dyadic
multipliers |l_ij| <= 1/2, U upper with small complex dyadic entries and
diagonal entries c * 2^t, c in {1, i, 1+i, 1-i}, so that 1/u_kk is dyadic.  In
exact partial pivoting on cabs1 the pivot at step k is the unique candidate
whose multiplier is 1, so the pivots are fixed by P, and every intermediate
value of the elimination is a short dyadic rational: an implementation whose
operations are exact whenever the result is representable must return L and U
bit for bit.  A dyadic x_true then gives an exactly representable b = A x_true.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def known_factor_case(n: int, L: int, seed: int):
    rng = np.random.default_rng(seed)
    Lm = [[(Fraction(0), Fraction(0))] * n for _ in range(n)]
    Um = [[(Fraction(0), Fraction(0))] * n for _ in range(n)]
    for i in range(n):
        Lm[i][i] = (Fraction(1), Fraction(0))
        for j in range(i):
            num = int(rng.integers(-4, 5))
            Lm[i][j] = (Fraction(num, 8), Fraction(0))           # |l| <= 1/2
        t = int(rng.integers(-2, 3))
        c = [(1, 0), (0, 1), (1, 1), (1, -1)][int(rng.integers(0, 4))]
        Um[i][i] = (Fraction(c[0]) * Fraction(2) ** t, Fraction(c[1]) * Fraction(2) ** t)
        for j in range(i + 1, n):
            Um[i][j] = (Fraction(int(rng.integers(-16, 17)), 4), Fraction(int(rng.integers(-16, 17)), 4))
    LU = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            s = (Fraction(0), Fraction(0))
            for k in range(min(i, j) + 1):
                p = _cmul(Lm[i][k], Um[k][j])
                s = (s[0] + p[0], s[1] + p[1])
            LU[i][j] = s
    sigma = rng.permutation(n)                   # row t of L U goes to row sigma[t] of A
    A = np.zeros((2, L, n, n))
    for t in range(n):
        for j in range(n):
            re, im = LU[t][j]
            assert float(re) == re and float(im) == im
            A[0, 0, j, sigma[t]] = float(re)
            A[1, 0, j, sigma[t]] = float(im)
    cur = list(range(n))
    ipiv = []
    for k in range(n):
        p = cur.index(int(sigma[k]), k)
        ipiv.append(p + 1)
        cur[k], cur[p] = cur[p], cur[k]
    packed = np.zeros((2, L, n, n))
    for i in range(n):
        for j in range(n):
            v = Lm[i][j] if i > j else Um[i][j]
            packed[0, 0, j, i] = float(v[0])
            packed[1, 0, j, i] = float(v[1])
    xr = rng.integers(-8, 9, n)
    xi = rng.integers(-8, 9, n)
    return A, np.array(ipiv, np.int32), packed, xr, xi


def known_factor_case_real(n: int, L: int, seed: int):
    """The real counterpart of ``known_factor_case``: A = P^T L U exactly with
    L unit lower, real dyadic multipliers |l_ij| <= 1/2, U upper with dyadic
    entries and diagonal entries +-2^t (1/u_kk dyadic).  Exact partial pivoting
    on |a| picks at step k the unique candidate whose multiplier is 1.
    Returns A [L, n, n], ipiv, the packed factors [L, n, n] and a dyadic
    integer x."""
    rng = np.random.default_rng(seed)
    Lm = [[Fraction(0)] * n for _ in range(n)]
    Um = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        Lm[i][i] = Fraction(1)
        for j in range(i):
            Lm[i][j] = Fraction(int(rng.integers(-4, 5)), 8)        # |l| <= 1/2
        t = int(rng.integers(-2, 3))
        Um[i][i] = Fraction(int(rng.choice([-1, 1]))) * Fraction(2) ** t
        for j in range(i + 1, n):
            Um[i][j] = Fraction(int(rng.integers(-16, 17)), 4)
    sigma = rng.permutation(n)                   # row t of L U goes to row sigma[t] of A
    A = np.zeros((L, n, n))
    for t in range(n):
        for j in range(n):
            v = sum((Lm[t][k] * Um[k][j] for k in range(min(t, j) + 1)), Fraction(0))
            assert float(v) == v
            A[0, j, sigma[t]] = float(v)
    cur = list(range(n))
    ipiv = []
    for k in range(n):
        p = cur.index(int(sigma[k]), k)
        ipiv.append(p + 1)
        cur[k], cur[p] = cur[p], cur[k]
    packed = np.zeros((L, n, n))
    for i in range(n):
        for j in range(n):
            packed[0, j, i] = float(Lm[i][j] if i > j else Um[i][j])
    x = rng.integers(-8, 9, n)
    return A, np.array(ipiv, np.int32), packed, x
