"""Exact rational reference for tiny problems (TEST INFRASTRUCTURE ONLY).

Every stored binary64 limb is a dyadic rational, so the exact value of an
element is the Fraction sum of its limbs.  On that exact input this module runs
Gaussian elimination with partial pivoting (Sec. 3) in exact complex rational
arithmetic with the same pivot key as the library, cabs1(z) = |Re z| + |Im z|,
ties broken towards the lowest row index; it also solves A x = b and
A^H y = c exactly.  Used to pin the pivots, factors and solutions of the
binary64-based oracle for n <= 8.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def fr(x: float) -> Fraction:
    return Fraction(float(x))


def element(A: np.ndarray, i: int, j: int) -> tuple[Fraction, Fraction]:
    """Exact value of element (i, j) of a planes array [2, L, cols, ld]."""
    L = A.shape[1]
    re = sum((fr(A[0, l, j, i]) for l in range(L)), Fraction(0))
    im = sum((fr(A[1, l, j, i]) for l in range(L)), Fraction(0))
    return re, im


def matrix(A: np.ndarray, rows: int | None = None) -> list[list[tuple[Fraction, Fraction]]]:
    cols = A.shape[2]
    rows = A.shape[3] if rows is None else rows
    return [[element(A, i, j) for j in range(cols)] for i in range(rows)]


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def csub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def cdiv(a, b):
    d = b[0] * b[0] + b[1] * b[1]
    return ((a[0] * b[0] + a[1] * b[1]) / d, (a[1] * b[0] - a[0] * b[1]) / d)


def conj(a):
    return (a[0], -a[1])


def cabs1(a) -> Fraction:
    return abs(a[0]) + abs(a[1])


def gepp(M):
    """Exact GEPP.  M: list of rows of complex Fractions (copied).

    Returns (LU, ipiv 1-based, info, gaps) with LU packed like LAPACK; gaps[k]
    is the exact relative gap (k1 - k2)/k1 between the two largest keys.
    """
    A = [row[:] for row in M]
    n = len(A)
    ipiv, info, gaps = [], 0, []
    for k in range(n):
        keys = [cabs1(A[i][k]) for i in range(k, n)]
        p = k + max(range(len(keys)), key=lambda t: (keys[t], -t))
        srt = sorted(keys, reverse=True)
        gaps.append((srt[0] - srt[1]) / srt[0] if len(srt) > 1 and srt[0] > 0 else Fraction(1))
        ipiv.append(p + 1)
        if keys[p - k] == 0:
            info = info or k + 1
            continue
        A[k], A[p] = A[p], A[k]
        for i in range(k + 1, n):
            A[i][k] = cdiv(A[i][k], A[k][k])
            for j in range(k + 1, n):
                A[i][j] = csub(A[i][j], cmul(A[i][k], A[k][j]))
    return A, ipiv, info, gaps


def solve(M, b):
    """Exact solution of M x = b (b: list of complex Fractions)."""
    LU, ipiv, info, _ = gepp(M)
    assert info == 0
    n = len(M)
    x = list(b)
    for k in range(n):
        p = ipiv[k] - 1
        x[k], x[p] = x[p], x[k]
    for k in range(n):
        for i in range(k + 1, n):
            x[i] = csub(x[i], cmul(LU[i][k], x[k]))
    for k in range(n - 1, -1, -1):
        x[k] = cdiv(x[k], LU[k][k])
        for i in range(k):
            x[i] = csub(x[i], cmul(LU[i][k], x[k]))
    return x


def solve_adjoint(M, c):
    """Exact solution of M^H y = c."""
    n = len(M)
    MH = [[conj(M[j][i]) for j in range(n)] for i in range(n)]
    return solve(MH, c)


def to_float(z: Fraction) -> float:
    return float(z)


def rel_err(approx: Fraction, exact: Fraction, scale: Fraction) -> float:
    if scale == 0:
        return 0.0 if approx == exact else float("inf")
    return float(abs(approx - exact) / scale)
