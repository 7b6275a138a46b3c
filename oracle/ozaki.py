"""Oracle for the Ozaki-scheme split (TEST INFRASTRUCTURE ONLY).

Plain Python integers, written from the definition (Sec. 2.3 of the paper,
Ozaki scheme: split operands into slices whose products are exact):

* scale: for a row of A (or a column of B) E = max_j floor(log2 |x_j,0|) + 2
  over the leading limbs of the real and imaginary parts, so |x| < 2^(E-1);
* fixed point: T = sum_l trunc(x_l 2^(beta S - E)) (each limb truncated toward
  zero), so |T| < 2^(beta S - 1);
* digits: T = sum_{p=0}^{S-1} a_p 2^(beta (S-1-p)) with balanced digits
  a_p in [-2^(beta-1), 2^(beta-1) - 1] for p >= 1 and |a_0| <= 2^(beta-1).

The Ozaki product of the sliced operands keeps the pairs p + q <= S - 1.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

CFG = {2: (7, 16), 3: (7, 24), 4: (7, 32)}   # L -> (beta, S)


def leading_exponent(x: float) -> int | None:
    if x == 0.0:
        return None
    return math.frexp(x)[1] - 1          # floor(log2 |x|)


def scale(values) -> int:
    """E for a set of elements given by their leading limbs."""
    es = [leading_exponent(float(v)) for v in values]
    es = [e for e in es if e is not None]
    return max(es) + 2 if es else 0


def trunc_scaled(x: float, shift: int) -> int:
    """trunc(x 2^shift) as an exact integer."""
    if x == 0.0:
        return 0
    num, den = float(x).as_integer_ratio()
    v = Fraction(num, den) * (Fraction(2) ** shift)
    return math.trunc(v)


def fixed_point(limbs, E: int, beta: int, S: int) -> int:
    return sum(trunc_scaled(float(x), beta * S - E) for x in limbs)


def digits(T: int, beta: int, S: int) -> list[int]:
    """Balanced base-2^beta digits, most significant first."""
    out = [0] * S
    half, base = 1 << (beta - 1), 1 << beta
    for p in range(S - 1, 0, -1):
        b = T & (base - 1)
        d = b - base if b >= half else b
        out[p] = d
        T = (T - d) >> beta
    out[0] = T
    return out


def split_rows(X: np.ndarray, rows: int, cols: int, L: int):
    """Row-scaled split of a [2, L, cols, ld] block: returns (E[rows], D[S, rows, cols, 2])."""
    beta, S = CFG[L]
    E = np.zeros(rows, np.int64)
    D = np.zeros((S, rows, cols, 2), np.int64)
    for i in range(rows):
        E[i] = scale([X[c, 0, j, i] for c in range(2) for j in range(cols)])
        for j in range(cols):
            for c in range(2):
                T = fixed_point(X[c, :, j, i], int(E[i]), beta, S)
                D[:, i, j, c] = digits(T, beta, S)
    return E, D


def split_cols(X: np.ndarray, rows: int, cols: int, L: int):
    """Column-scaled split: returns (E[cols], D[S, rows, cols, 2])."""
    beta, S = CFG[L]
    E = np.zeros(cols, np.int64)
    D = np.zeros((S, rows, cols, 2), np.int64)
    for j in range(cols):
        E[j] = scale([X[c, 0, j, i] for c in range(2) for i in range(rows)])
        for i in range(rows):
            for c in range(2):
                T = fixed_point(X[c, :, j, i], int(E[j]), beta, S)
                D[:, i, j, c] = digits(T, beta, S)
    return E, D
