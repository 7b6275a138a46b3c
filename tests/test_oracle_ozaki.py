"""Pins of the oracle's Ozaki split definition (oracle/ozaki.py):
the digits reconstruct the fixed-point integer exactly, stay in their ranges,
and the sliced value is within L units of 2^(E - beta S) of the exact element
(Fraction).  Also the exactness premise of the tensor-core accumulation: for
K = 64 the sum of S diagonal pair products of extreme digits stays <= 2^24,
over the number of K chunks accumulated before each fold as well."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki
from paper_2403_16013_gb300 import inputs


@pytest.mark.parametrize("L", [2, 3, 4])
def test_digits_reconstruct_and_bound(L):
    beta, S = ozaki.CFG[L]
    X = inputs.spread_matrix(6, 9, L, seed=3, spread=20)
    E, D = ozaki.split_rows(X, 6, 9, L)
    for i in range(6):
        for j in range(9):
            for c in range(2):
                d = [int(v) for v in D[:, i, j, c]]
                assert all(-(1 << (beta - 1)) <= v < (1 << (beta - 1)) for v in d[1:])
                assert abs(d[0]) <= 1 << (beta - 1)
                T = ozaki.fixed_point(X[c, :, j, i], int(E[i]), beta, S)
                assert sum(v << (beta * (S - 1 - p)) for p, v in enumerate(d)) == T
                exact = sum(Fraction(float(x)) for x in X[c, :, j, i])
                sliced = Fraction(T) * Fraction(2) ** (int(E[i]) - beta * S)
                assert abs(sliced - exact) <= L * Fraction(2) ** (int(E[i]) - beta * S)
                assert abs(exact) < Fraction(2) ** (int(E[i]) - 1)


def test_zero_and_negative_symmetry():
    beta, S = ozaki.CFG[2]
    assert ozaki.digits(0, beta, S) == [0] * S
    T = (1 << (beta * S - 1)) - 1                 # largest admissible magnitude
    d = ozaki.digits(T, beta, S)
    assert sum(v << (beta * (S - 1 - p)) for p, v in enumerate(d)) == T and abs(d[0]) <= 1 << (beta - 1)
    d = ozaki.digits(-T, beta, S)
    assert sum(v << (beta * (S - 1 - p)) for p, v in enumerate(d)) == -T and abs(d[0]) <= 1 << (beta - 1)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_accumulation_stays_exact_in_fp32(L):
    beta, S = ozaki.CFG[L]
    dmax = 1 << (beta - 1)
    K = 64
    assert S * K * dmax * dmax <= 1 << 24       # worst diagonal of one K = 64 chunk
    # the K chunks accumulated in TMEM before the epilogue folds them
    # (chunks_per_fold in ozaki.cuh): 4 for DD, 2 for TD and QD
    cpf = {2: 4, 3: 2, 4: 2}[L]
    assert cpf * S * K * dmax * dmax <= 1 << 24 < (cpf + 1) * S * K * dmax * dmax
    assert beta * S >= 53 * L + 6               # slices cover the precision with margin
