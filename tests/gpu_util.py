"""Helpers for the GPU parity tests: numpy planes <-> CUDA tensors, norms."""
from __future__ import annotations

import numpy as np

from helpers import U_EXP


def dev(x: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t) -> np.ndarray:
    return t.detach().cpu().numpy()


def backward_error(orc, A, X, Bm) -> float:
    """||b - A x||_inf / (||A||_inf ||x||_inf) with the exact residual (modulus norms)."""
    R = orc.exact_residual(A, X, Bm, Lr=1)
    r = np.hypot(R[0, 0], R[1, 0]).max()
    Ah = np.hypot(A[0].sum(axis=0), A[1].sum(axis=0))
    anorm = Ah.sum(axis=0).max()
    xh = np.hypot(X[0].sum(axis=0), X[1].sum(axis=0))
    return float(r / (anorm * xh.max()))


def bound(n: int, L: int) -> float:
    return 16.0 * n * 2.0 ** -U_EXP[L]


def value(X: np.ndarray) -> np.ndarray:
    """Leading-order complex value of planes [2, L, cols, ld] as complex128 [ld, cols]."""
    return (X[0].sum(axis=0) + 1j * X[1].sum(axis=0)).T


def exact_diff(orc, g: np.ndarray, o: np.ndarray) -> np.ndarray:
    """RN(sum(g limbs) - sum(o limbs)) per element, exactly (superaccumulator).
    g, o: [L, count] limb-major arrays."""
    V = np.concatenate([g, -o], axis=0).T.copy()
    return orc.exact_sum_rows(V, 1)[:, 0]
