"""Torch-level API over the C ABI: plane tensors in, plane tensors out.

A complex L-limb matrix is a float64 CUDA tensor of shape [2, L, cols, ld]
(component, limb, column, row): each [c, l] plane is column-major.  These
functions allocate outputs with torch, pass raw device pointers and the
current stream to libmclu.so, and check the returned status.  All arithmetic
runs in the CUDA kernels; nothing is computed here.
"""
from __future__ import annotations

import torch

from . import binding as B

LIMBS = B.LIMBS
METHODS = {"4m": B.METHOD_4M, "3m": B.METHOD_3M, "unblocked": B.METHOD_UNBLOCKED, "ozaki": B.METHOD_OZAKI,
           "strassen": B.METHOD_STRASSEN}


def _prec(T: torch.Tensor) -> str:
    L = T.shape[1]
    return {2: "dd", 3: "td", 4: "qd"}[L]


def _check_planes(T: torch.Tensor, name: str):
    if not isinstance(T, torch.Tensor) or not T.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if T.dtype != torch.float64 or T.dim() != 4 or T.shape[0] != 2 or T.shape[1] not in (2, 3, 4):
        raise ValueError(f"{name} must be float64 planes of shape [2, L, cols, ld], L in 2..4; got "
                         f"{tuple(T.shape)} {T.dtype}")
    if not T.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def lu_factor(A: torch.Tensor, method: str = "4m", nb: int = 0, ozaki_slices: int = 0, out: torch.Tensor | None = None,
              sub_nb: int = 0):
    """P A = L U.  Returns (LU planes, ipiv int32 1-based, info int32[1] device).
    ozaki_slices, sub_nb: the Ozaki method's slices per operand and sub-panel width (0: defaults)."""
    _check_planes(A, "A")
    n, lda = A.shape[2], A.shape[3]
    LU = A.clone() if out is None else out.copy_(A)
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = B.zgetrf_ex(_prec(A), n, LU.data_ptr(), lda, ipiv.data_ptr(), info.data_ptr(), nb, METHODS[method],
                     ozaki_slices, _stream(), sub_nb=sub_nb)
    B.check(rc, "zgetrf")
    return LU, ipiv[:n], info


def lu_factor_(A: torch.Tensor, ipiv: torch.Tensor, info: torch.Tensor | None = None, method: str = "4m",
               nb: int = 0, ozaki_slices: int = 0, sub_nb: int = 0):
    """In-place factorisation into caller-owned buffers (no allocation besides the library's workspace)."""
    n, lda = A.shape[2], A.shape[3]
    rc = B.zgetrf_ex(_prec(A), n, A.data_ptr(), lda, ipiv.data_ptr(), 0 if info is None else info.data_ptr(), nb,
                     METHODS[method], ozaki_slices, _stream(), sub_nb=sub_nb)
    B.check(rc, "zgetrf")


def lu_solve(LU: torch.Tensor, ipiv: torch.Tensor, Bm: torch.Tensor, trans: str = "N", inplace: bool = False):
    """Solve A X = B ('N') or A^H X = B ('C') with the factors of lu_factor."""
    _check_planes(LU, "LU")
    _check_planes(Bm, "B")
    X = Bm if inplace else Bm.clone()
    n, lda = LU.shape[2], LU.shape[3]
    nrhs, ldb = X.shape[2], X.shape[3]
    rc = B.zgetrs(_prec(LU), trans, n, nrhs, LU.data_ptr(), lda, ipiv.data_ptr(), X.data_ptr(), ldb, _stream())
    B.check(rc, "zgetrs")
    return X


def _check_real_planes(T: torch.Tensor, name: str):
    if not isinstance(T, torch.Tensor) or not T.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if T.dtype != torch.float64 or T.dim() != 3 or T.shape[0] not in (2, 3, 4) or not T.is_contiguous():
        raise ValueError(f"{name} must be contiguous float64 limb planes of shape [L, cols, ld], L in 2..4; "
                         f"got {tuple(T.shape)} {T.dtype}")


def dlu_factor(A: torch.Tensor, method: str = "4m", nb: int = 0, ozaki_slices: int = 0, sub_nb: int = 0):
    """Real P A = L U.  A: limb planes [L, n, lda].  Returns (LU, ipiv, info)."""
    _check_real_planes(A, "A")
    n, lda = A.shape[1], A.shape[2]
    LU = A.clone()
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = B.dgetrf_ex({2: "dd", 3: "td", 4: "qd"}[A.shape[0]], n, LU.data_ptr(), lda, ipiv.data_ptr(),
                     info.data_ptr(), nb, METHODS[method], ozaki_slices, _stream(), sub_nb=sub_nb)
    B.check(rc, "dgetrf")
    return LU, ipiv[:n], info


def dlu_solve(LU: torch.Tensor, ipiv: torch.Tensor, Bm: torch.Tensor, trans: str = "N"):
    """Solve A X = B ('N') or A^T X = B ('T') with the factors of dlu_factor; B: [L, nrhs, ldb]."""
    _check_real_planes(LU, "LU")
    _check_real_planes(Bm, "B")
    X = Bm.clone()
    n, lda = LU.shape[1], LU.shape[2]
    rc = B.dgetrs({2: "dd", 3: "td", 4: "qd"}[LU.shape[0]], trans, n, X.shape[1], LU.data_ptr(), lda,
                  ipiv.data_ptr(), X.data_ptr(), X.shape[2], _stream())
    B.check(rc, "dgetrs")
    return X


def zgemm(A: torch.Tensor, Bm: torch.Tensor, C: torch.Tensor | None = None, method: str = "4m",
          ozaki_slices: int = 0):
    """C = A B (C is None) or C - A B (returns a new tensor).  ozaki_slices:
    slices kept per operand by the Ozaki method (0 = the precision's S)."""
    _check_planes(A, "A")
    _check_planes(Bm, "B")
    k, m = A.shape[2], A.shape[3]
    n, ldb = Bm.shape[2], Bm.shape[3]
    beta = 0 if C is None else 1
    out = torch.zeros((2, A.shape[1], n, m), dtype=torch.float64, device=A.device) if C is None else C.clone()
    rc = B.zgemm_ex(_prec(A), beta, METHODS[method], ozaki_slices, m, n, k, A.data_ptr(), m, Bm.data_ptr(), ldb,
                    out.data_ptr(), out.shape[3], _stream())
    B.check(rc, "zgemm")
    return out


def adjoint_rank1(lam: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """Abar = -lambda x^H for n x 1 plane vectors."""
    n = lam.shape[3]
    Ab = torch.empty((2, lam.shape[1], n, n), dtype=torch.float64, device=lam.device)
    rc = B.zadjoint_rank1(_prec(lam), n, lam.data_ptr(), x.data_ptr(), Ab.data_ptr(), n, _stream())
    B.check(rc, "zadjoint_rank1")
    return Ab


_VEC_OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "cadd": 10, "csub": 11, "cmul": 12, "cmul3m": 13,
            "cdiv": 14, "cinv": 15, "cabs1": 16, "cinv_newton": 17}


def vec_op(op: str, x: torch.Tensor, y: torch.Tensor | None = None, z: torch.Tensor | None = None) -> torch.Tensor:
    """Elementwise MC arithmetic: real ops on [L, count], complex ops on [2, L, count]."""
    code = _VEC_OPS[op]
    L = x.shape[0] if code < 10 else x.shape[1]
    count = x.shape[-1]
    z = torch.empty_like(x)
    rc = B.vec_op(code, L, count, x.data_ptr(), 0 if y is None else y.data_ptr(), z.data_ptr(), _stream())
    B.check(rc, f"vec_op {op}")
    return z


class _Solve(torch.autograd.Function):
    """x = A^{-1} b with the hand-written adjoint: lambda = A^{-H} xbar (zgetrs 'C'
    on the stored factors), bbar = lambda, Abar = -lambda x^H (fused rank-1)."""

    @staticmethod
    def forward(ctx, A, b, method):
        LU, ipiv, info = lu_factor(A.detach().contiguous(), method=method)
        x = lu_solve(LU, ipiv, b.detach().contiguous())
        ctx.save_for_backward(LU, ipiv, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        LU, ipiv, x = ctx.saved_tensors
        lam = lu_solve(LU, ipiv, gx.contiguous(), trans="C")
        if x.shape[2] != 1:
            raise NotImplementedError("the adjoint is implemented for a single right-hand side")
        Abar = adjoint_rank1(lam, x)
        return Abar, lam, None


def solve(A: torch.Tensor, b: torch.Tensor, method: str = "4m") -> torch.Tensor:
    """Differentiable solve.  Gradients are L-limb values: the sum of the limb
    planes of a gradient is the derivative with respect to the represented
    value (use ``mc_value`` to form losses from the value)."""
    return _Solve.apply(A, b, method)


class _Value(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X):
        ctx.L = X.shape[1]
        return X.sum(dim=1)

    @staticmethod
    def backward(ctx, g):
        G = torch.zeros(g.shape[0], ctx.L, *g.shape[1:], dtype=g.dtype, device=g.device)
        G[:, 0] = g
        return G


def mc_value(X: torch.Tensor) -> torch.Tensor:
    """Binary64 value of each element (limbs summed); its gradient goes into limb 0."""
    return _Value.apply(X)
