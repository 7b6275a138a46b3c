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


def planes_diff(orc, G: np.ndarray, O: np.ndarray) -> np.ndarray:
    """|value(G) - value(O)| per element, the difference of all limbs of both
    taken exactly (superaccumulator) and rounded to binary64.  G, O: planes
    [2, L, cols, ld] or samples [s, 2, L] (limb axis given by the layout).
    Subtracting limb by limb and summing in binary64 is not exact: two valid
    L-limb forms of one value (e.g. 2 - 2^-52 + 0.4 2^-52 against
    2 - 0.6 2^-52) round their limb differences at the 2^-105 level."""
    G = np.asarray(G, np.float64)
    O = np.asarray(O, np.float64)
    if G.ndim == 4:        # [2, L, cols, ld]
        L = G.shape[1]
        g = np.moveaxis(G, 1, -1).reshape(-1, L)
        o = np.moveaxis(O, 1, -1).reshape(-1, O.shape[1])
        out_shape = (G.shape[0], G.shape[2], G.shape[3])
    else:                  # [s, 2, L]
        g = G.reshape(-1, G.shape[2])
        o = O.reshape(-1, O.shape[2])
        out_shape = G.shape[:2]
    V = np.ascontiguousarray(np.concatenate([g, -o], axis=1))
    return np.abs(orc.exact_sum_rows(V, 1)[:, 0]).reshape(out_shape)
