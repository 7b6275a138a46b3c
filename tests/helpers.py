"""Shared helpers for the tests: random canonical multi-component values and
exact (Fraction) evaluation.  No multi-component arithmetic lives here."""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from paper_2403_16013_gb300 import inputs

U_EXP = {2: 104, 3: 157, 4: 209}      # u = 2^-104 / 2^-157 / 2^-209 for DD / TD / QD


def u_of(L: int) -> float:
    return 2.0 ** -U_EXP[L]


def rand_limbs(L: int, count: int, rng, emin: int = -30, emax: int = 30) -> np.ndarray:
    """Random canonical L-limb reals, limb-major [L, count]."""
    lead = np.ldexp(rng.uniform(-1, 1, count), rng.integers(emin, emax + 1, count))
    rest = inputs._lower_limbs(lead, L, rng)
    return np.stack([lead] + rest)


def frac_col(x: np.ndarray, j: int) -> Fraction:
    return sum((Fraction(float(v)) for v in x[:, j]), Fraction(0))


def frac_vec(x: np.ndarray) -> list[Fraction]:
    return [frac_col(x, j) for j in range(x.shape[1])]


def is_nonoverlapping(limbs, strict: bool = True) -> bool:
    """|x_{k+1}| <= ulp(x_k)/2 (strict) or <= ulp(x_k) (ulp-nonoverlapping) for every
    adjacent nonzero pair, and zeros only at the end."""
    seen_zero = False
    for a, b in zip(limbs[:-1], limbs[1:]):
        if a == 0:
            seen_zero = True
        if seen_zero and b != 0:
            return False
        if a != 0 and abs(b) > np.spacing(abs(a)) / (2 if strict else 1):
            return False
    return True
