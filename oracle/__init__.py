"""CPU oracle for complex multi-component LU (TEST INFRASTRUCTURE ONLY).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg (``bench.py`` ``cpu_baseline`` and ``--impl reference``) may
import this package.  It shares no code with the CUDA library: the C source
``mclu_oracle.c`` is built on its own by ``oracle/build.py`` and the two never
link or import each other.

Arrays use the library's plane layout: float64 numpy arrays of shape
``[2, L, cols, ld]`` (component, limb, column, row).  See ``mclu_oracle.c`` for
the definition of every operation and the passages of the paper they follow.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build_oracle

_lib = None

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)

OP_ADD, OP_SUB, OP_MUL, OP_DIV = 0, 1, 2, 3
COP_ADD, COP_SUB, COP_MUL4M, COP_MUL3M, COP_DIV, COP_INV, COP_ABS1 = 0, 1, 2, 3, 4, 5, 6


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        i64, i32, ci, dbl = C.c_int64, C.c_int32, C.c_int, C.c_double
        sig = {
            "orc_error_flag": (ci, []),
            "orc_clear_error": (None, []),
            "orc_num_threads": (ci, []),
            "orc_real_op": (ci, [ci, ci, i64, _D, _D, _D]),
            "orc_cplx_op": (ci, [ci, ci, i64, _D, _D, _D]),
            "orc_eft": (None, [i64, _D, _D, _D, _D, _D, _D]),
            "orc_normalize_rows": (None, [i64, ci, _D, _I32]),
            "orc_zgetrf": (ci, [ci, i64, _D, i64, _I32, _I32, _D]),
            "orc_zgetrs": (ci, [ci, C.c_char, i64, i64, _D, i64, _I32, _D, i64]),
            "orc_dgetrf": (ci, [ci, i64, _D, i64, _I32, _I32, _D]),
            "orc_dgetrs": (ci, [ci, C.c_char, i64, i64, _D, i64, _I32, _D, i64]),
            "orc_zgemm": (ci, [ci, ci, ci, i64, i64, i64, _D, i64, _D, i64, _D, i64]),
            "orc_exact_residual": (ci, [ci, ci, ci, ci, i64, i64, _D, i64, _D, i64, _D, i64, _D]),
            "orc_exact_entries": (ci, [ci, ci, ci, i64, i64, i64, _D, i64, _D, i64, _D, i64, ci, ci, i64,
                                       _I64, _I64, _D]),
            "orc_exact_sum_rows": (None, [i64, ci, _D, ci, _D]),
            "orc_adjoint": (ci, [ci, i64, _D, i64, _I32, _D, _D, _D, i64]),
            "orc_make_ill_conditioned": (ci, [ci, i64, ci, _D, _D, dbl, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    if a.dtype == np.float64:
        return a.ctypes.data_as(_D)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_I32)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_I64)
    raise TypeError(a.dtype)


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"{what}: argument {-rc} invalid")
    if rc > 0 or lib().orc_error_flag():
        raise RuntimeError(f"{what}: oracle normalisation did not converge (flag {lib().orc_error_flag()})")


def num_threads() -> int:
    return lib().orc_num_threads()


# ------------------------------------------------------------- scalars --

def real_op(op: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """x, y: [L, count] limb-major arrays; returns [L, count]."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    L, count = x.shape
    z = np.zeros_like(x)
    _check(lib().orc_real_op(op, L, count, _p(x), _p(y), _p(z)), "real_op")
    return z


def cplx_op(op: int, x: np.ndarray, y: np.ndarray | None = None) -> np.ndarray:
    """x, y: [2, L, count] plane arrays; returns [2, L, count]."""
    x = np.ascontiguousarray(x, np.float64)
    _, L, count = x.shape
    z = np.zeros_like(x)
    yp = _p(np.ascontiguousarray(y, np.float64)) if y is not None else None
    if y is not None:
        y = np.ascontiguousarray(y, np.float64)
        yp = _p(y)
    _check(lib().orc_cplx_op(op, L, count, _p(x), yp, _p(z)), "cplx_op")
    return z


def eft(a: np.ndarray, b: np.ndarray):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    s, e, p, f = (np.zeros_like(a) for _ in range(4))
    lib().orc_eft(a.size, _p(a), _p(b), _p(s), _p(e), _p(p), _p(f))
    return s, e, p, f


def normalize_rows(v: np.ndarray):
    v = np.ascontiguousarray(v, np.float64).copy()
    count, m = v.shape
    ln = np.zeros(count, np.int32)
    lib().orc_normalize_rows(count, m, _p(v), _p(ln))
    return v, ln


def exact_sum_rows(v: np.ndarray, L: int) -> np.ndarray:
    v = np.ascontiguousarray(v, np.float64)
    count, m = v.shape
    out = np.zeros((count, L), np.float64)
    lib().orc_exact_sum_rows(count, m, _p(v), L, _p(out))
    return out


# -------------------------------------------------------------- matrix --

def zgetrf(A: np.ndarray):
    """Unblocked GEPP.  A: [2, L, n, lda] (copied).  Returns (LU, ipiv, info, gap)."""
    LU = np.ascontiguousarray(A, np.float64).copy()
    _, L, n, lda = LU.shape
    ipiv = np.zeros(max(n, 1), np.int32)
    info = np.zeros(1, np.int32)
    gap = np.zeros(max(n, 1), np.float64)
    _check(lib().orc_zgetrf(L, n, _p(LU), lda, _p(ipiv), _p(info), _p(gap)), "zgetrf")
    return LU, ipiv[:n], int(info[0]), gap[:n]


def zgetrs(LU: np.ndarray, ipiv: np.ndarray, B: np.ndarray, trans: str = "N") -> np.ndarray:
    """B: [2, L, nrhs, ldb] (copied); returns X."""
    LU = np.ascontiguousarray(LU, np.float64)
    X = np.ascontiguousarray(B, np.float64).copy()
    _, L, n, lda = LU.shape
    _, _, nrhs, ldb = X.shape
    ip = np.ascontiguousarray(ipiv, np.int32)
    _check(lib().orc_zgetrs(L, trans.encode(), n, nrhs, _p(LU), lda, _p(ip), _p(X), ldb), "zgetrs")
    return X


def dgetrf(A: np.ndarray):
    """Real unblocked GEPP (one plane per limb).  A: [L, n, lda] (copied).
    Returns (LU, ipiv, info, gap)."""
    LU = np.ascontiguousarray(A, np.float64).copy()
    L, n, lda = LU.shape
    ipiv = np.zeros(max(n, 1), np.int32)
    info = np.zeros(1, np.int32)
    gap = np.zeros(max(n, 1), np.float64)
    _check(lib().orc_dgetrf(L, n, _p(LU), lda, _p(ipiv), _p(info), _p(gap)), "dgetrf")
    return LU, ipiv[:n], int(info[0]), gap[:n]


def dgetrs(LU: np.ndarray, ipiv: np.ndarray, B: np.ndarray, trans: str = "N") -> np.ndarray:
    """Real solve with the factors of dgetrf.  B: [L, nrhs, ldb] (copied); trans 'N' or 'T'."""
    LU = np.ascontiguousarray(LU, np.float64)
    X = np.ascontiguousarray(B, np.float64).copy()
    L, n, lda = LU.shape
    _, nrhs, ldb = X.shape
    ip = np.ascontiguousarray(ipiv, np.int32)
    _check(lib().orc_dgetrs(L, trans.encode(), n, nrhs, _p(LU), lda, _p(ip), _p(X), ldb), "dgetrs")
    return X


def zgemm(A: np.ndarray, B: np.ndarray, C: np.ndarray | None = None, method: str = "4m") -> np.ndarray:
    """C = A B (C is None) or C - A B.  A: [2, L, k, lda], B: [2, L, n, ldb]."""
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    _, L, k, lda = A.shape
    _, _, n, ldb = B.shape
    m = lda
    beta = 0 if C is None else 1
    Cout = np.zeros((2, L, n, m), np.float64) if C is None else np.ascontiguousarray(C, np.float64).copy()
    ldc = Cout.shape[3]
    meth = {"4m": 0, "3m": 1}[method]
    _check(lib().orc_zgemm(L, meth, beta, m, n, k, _p(A), lda, _p(B), ldb, _p(Cout), ldc), "zgemm")
    return Cout


def exact_residual(A: np.ndarray, X: np.ndarray, B: np.ndarray, Lr: int = 1) -> np.ndarray:
    """R = B - A X exactly, rounded greedily to Lr limbs: [2, Lr, nrhs, n]."""
    A = np.ascontiguousarray(A, np.float64)
    X = np.ascontiguousarray(X, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    _, L, n, lda = A.shape
    _, Lx, nrhs, ldx = X.shape
    _, Lb, _, ldb = B.shape
    R = np.zeros((2, Lr, nrhs, n), np.float64)
    _check(lib().orc_exact_residual(L, Lx, Lb, Lr, n, nrhs, _p(A), lda, _p(X), ldx, _p(B), ldb, _p(R)),
           "exact_residual")
    return R


def exact_entries(A: np.ndarray, B: np.ndarray, rows, cols, C: np.ndarray | None = None, sign: int = 1,
                  lu: bool = False) -> np.ndarray:
    """Exact (C if given) + sign * (A B) at sampled (row, col), rounded to 4 limbs.

    With ``lu=True``, A and B are the same packed LU array and the product is
    L U with L unit lower and U upper.  Returns [nsamp, 2, 4].
    """
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    _, La, k, lda = A.shape
    _, Lb, n, ldb = B.shape
    m = lda
    rows = np.ascontiguousarray(rows, np.int64)
    cols = np.ascontiguousarray(cols, np.int64)
    out = np.zeros((rows.size, 2, 4), np.float64)
    if C is not None:
        C = np.ascontiguousarray(C, np.float64)
        Lc, ldc, cp = C.shape[1], C.shape[3], _p(C)
    else:
        Lc, ldc, cp = 0, 1, None
    _check(lib().orc_exact_entries(La, Lb, Lc, m, n, k, _p(A), lda, _p(B), ldb, cp, ldc, sign, int(lu),
                                   rows.size, _p(rows), _p(cols), _p(out)), "exact_entries")
    return out


def adjoint(LU: np.ndarray, ipiv: np.ndarray, x: np.ndarray, xbar: np.ndarray):
    """Returns (lambda = A^{-H} xbar (= bbar), Abar = -lambda x^H)."""
    LU = np.ascontiguousarray(LU, np.float64)
    _, L, n, lda = LU.shape
    lam = np.ascontiguousarray(xbar, np.float64).copy()
    x = np.ascontiguousarray(x, np.float64)
    Abar = np.zeros((2, L, n, n), np.float64)
    ip = np.ascontiguousarray(ipiv, np.int32)
    _check(lib().orc_adjoint(L, n, _p(LU), lda, _p(ip), _p(x), _p(lam), _p(Abar), n), "adjoint")
    return lam, Abar


def make_ill_conditioned(L: int, n: int, V1: np.ndarray, V2: np.ndarray, r: float) -> np.ndarray:
    """A = Q1 diag(r^i) Q2^H formed in L-limb arithmetic; V*: [h, 2, n] binary64."""
    V1 = np.ascontiguousarray(V1, np.float64)
    V2 = np.ascontiguousarray(V2, np.float64)
    h = V1.shape[0]
    A = np.zeros((2, L, n, n), np.float64)
    _check(lib().orc_make_ill_conditioned(L, n, h, _p(V1), _p(V2), float(r), _p(A)), "make_ill_conditioned")
    return A


# ------------------------------------------------------------- helpers --

def limbs_exact(x) -> "Fraction":
    from fractions import Fraction
    return sum((Fraction(float(v)) for v in np.atleast_1d(x)), Fraction(0))
