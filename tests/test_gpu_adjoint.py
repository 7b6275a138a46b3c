"""GPU parity of the hand-written adjoint of x = A^{-1} b (torch.autograd):
for loss = Re(c^H x), bbar = lambda = A^{-H} c and Abar = -lambda x^H.

* n = 96: the autograd gradients equal the oracle's adjoint within 2^12 n u;
* n = 48: the DD gradient matches QD central finite differences (step
  2^-60, real and imaginary perturbations of 32 sampled entries) computed by
  the oracle with Sherman-Morrison on its QD factors: x(A + tE) =
  x - t w x_j / (1 + t w_j), w = A^{-1} e_i;
* n = 2048 (the adjoint workload): lambda solves A^H lambda = c with
  backward error <= 16 n u (exact residual of the conjugate transpose),
  sampled Abar entries equal -lambda_i conj(x_j) (exact products), and
  bbar = lambda.
"""
from fractions import Fraction

import numpy as np
import pytest

from gpu_util import backward_error, bound, dev, host, planes_diff
from helpers import U_EXP
from paper_2403_16013_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_16013_gb300 import api as a
    from paper_2403_16013_gb300 import build
    build.build()
    return a


def _grads(api, A, b, c):
    import torch
    Ad = dev(A).requires_grad_(True)
    bd = dev(b).requires_grad_(True)
    cd = dev(c)
    x = api.solve(Ad, bd)
    v = api.mc_value(x)                          # [2, 1, n]
    cv = cd.sum(dim=1)                           # binary64 value of c
    loss = (cv[0] * v[0] + cv[1] * v[1]).sum()   # Re(c^H x)
    loss.backward()
    torch.cuda.synchronize()
    return host(x.detach()), host(Ad.grad), host(bd.grad)


def test_adjoint_against_oracle(api, orc):
    n, L = 96, 2
    A = inputs.gaussian_matrix(n, L, seed=41)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    c = inputs.complex_gaussian_vector(n, L, seed=4)
    c[:, 1:] = 0.0                                # the loss sees the binary64 value of c
    x, gA, gb = _grads(api, A, b, c)
    LU, ipiv, _, _ = orc.zgetrf(A)
    xo = orc.zgetrs(LU, ipiv, b)
    lam, Abar = orc.adjoint(LU, ipiv, xo, c)
    u = 2.0 ** -U_EXP[L]
    scale_l = np.abs(lam[:, 0]).max()
    assert planes_diff(orc, gb, lam).max() <= 2.0 ** 12 * n * u * scale_l
    scale_a = scale_l * np.abs(xo[:, 0]).max()
    assert planes_diff(orc, gA, Abar).max() <= 2.0 ** 12 * n * u * scale_a


def _qd_value(X):
    return [(sum(Fraction(float(X[0, l, 0, i])) for l in range(X.shape[1])),
             sum(Fraction(float(X[1, l, 0, i])) for l in range(X.shape[1]))) for i in range(X.shape[3])]


def test_adjoint_against_qd_finite_differences(api, orc):
    n = 48
    A4 = inputs.gaussian_matrix(n, 4, seed=42)
    A = inputs.truncate_limbs(A4, 2)
    A4 = np.zeros_like(A4)
    A4[:, :2] = A                                 # the same matrix, as QD
    xr, xi = inputs.ones_x_true(n)
    b4 = inputs.exact_rhs(A, xr, xi, L_out=4)
    b = inputs.truncate_limbs(b4, 2)
    b4 = np.zeros_like(b4)
    b4[:, :2] = b
    c = inputs.complex_gaussian_vector(n, 2, seed=5)
    c[:, 1:] = 0.0
    x, gA, gb = _grads(api, A, b, c)
    LU4, ip4, _, _ = orc.zgetrf(A4)
    x4 = _qd_value(orc.zgetrs(LU4, ip4, b4))
    cf = [(Fraction(float(c[0, 0, 0, i])), Fraction(float(c[1, 0, 0, i]))) for i in range(n)]
    h = Fraction(1, 2 ** 60)
    rng = np.random.default_rng(7)
    worst = 0.0
    gscale = np.abs(gA[:, 0]).max()
    for _ in range(32):
        i, j = int(rng.integers(n)), int(rng.integers(n))
        e = np.zeros((2, 4, 1, n))
        e[0, 0, 0, i] = 1.0
        w = _qd_value(orc.zgetrs(LU4, ip4, e))    # A^{-1} e_i in QD
        for part in (0, 1):                       # perturb Re(A_ij) or Im(A_ij)
            t = (h, Fraction(0)) if part == 0 else (Fraction(0), h)
            vals = []
            for sgn in (1, -1):
                ts = (sgn * t[0], sgn * t[1])
                # x(A + ts e_i e_j^T) = x - ts w x_j / (1 + ts w_j)
                den = (1 + ts[0] * w[j][0] - ts[1] * w[j][1], ts[0] * w[j][1] + ts[1] * w[j][0])
                num = (ts[0] * x4[j][0] - ts[1] * x4[j][1], ts[0] * x4[j][1] + ts[1] * x4[j][0])
                d2 = den[0] ** 2 + den[1] ** 2
                f = ((num[0] * den[0] + num[1] * den[1]) / d2, (num[1] * den[0] - num[0] * den[1]) / d2)
                loss = sum(cf[k][0] * (x4[k][0] - (w[k][0] * f[0] - w[k][1] * f[1])) +
                           cf[k][1] * (x4[k][1] - (w[k][0] * f[1] + w[k][1] * f[0])) for k in range(n))
                vals.append(loss)
            fd = float((vals[0] - vals[1]) / (2 * h))
            g = gA[part, :, j, i].sum()
            worst = max(worst, abs(g - fd) / gscale)
    assert worst <= 2.0 ** -70, worst


def test_adjoint_full_size_properties(api, orc):
    n, L = 2048, 2
    A = inputs.gaussian_matrix(n, L, seed=1)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.complex_gaussian_vector(n, L, seed=3)
    c = inputs.complex_gaussian_vector(n, L, seed=4)
    c[:, 1:] = 0.0
    x, gA, gb = _grads(api, A, b, c)
    # A^H lambda = c: exact residual with the conjugate transpose
    AH = np.ascontiguousarray(np.transpose(A, (0, 1, 3, 2)))
    AH[1] = -AH[1]
    assert backward_error(orc, AH, gb, c) <= bound(n, L)
    # Abar_ij = -lambda_i conj(x_j) on sampled entries, exactly
    rng = np.random.default_rng(8)
    rows, cols = rng.integers(0, n, 64), rng.integers(0, n, 64)
    lam_col = np.ascontiguousarray(gb)                               # n x 1
    xh = np.ascontiguousarray(np.transpose(x, (0, 1, 3, 2)))         # 1 x n row of x
    xh[1] = -xh[1]
    ex = orc.exact_entries(lam_col, xh, rows, cols, C=np.ascontiguousarray(gA), sign=1)   # Abar + lambda x^H
    mag = np.abs(gb[:, 0]).max() * np.abs(x[:, 0]).max()
    assert np.abs(ex[:, :, 0]).max() <= 8 * 2.0 ** -U_EXP[L] * mag


def test_adjoint_qd_finite_differences_n2048(api, orc):
    """The adjoint workload at its size: n = 2048 DD, b = A (1 + i), c complex
    Gaussian (seed 4), loss Re(c^H x); 64 sampled entries (i, j) and both the
    real and the imaginary perturbation of A_ij.  The central difference of
    the loss with step t = 2^-60 is evaluated exactly (rational arithmetic) by
    Sherman-Morrison, x(A + t e_i e_j^T) = x - t w x_j / (1 + t w_j),
    w = A^{-1} e_i, from QD solutions x and w (the library's QD factorisation
    of the same matrix, 64 right-hand sides in one solve, a path checked
    against the oracle on its own) and the exact dot products c^H w (oracle
    superaccumulator).  The DD gradient must agree within 2^-70 of max|Abar|."""
    import torch
    n = 2048
    A = inputs.gaussian_matrix(n, 2, seed=4)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), 2)
    c = inputs.complex_gaussian_vector(n, 2, seed=4)
    c[:, 1:] = 0.0                                # the loss sees the binary64 value of c
    x, gA, gb = _grads(api, A, b, c)
    # the same matrix and right-hand side in QD (zero-padded limbs), factored on the GPU
    A4 = np.zeros((2, 4, n, n))
    A4[:, :2] = A
    b4 = np.zeros((2, 4, 1, n))
    b4[:, :2] = b
    LU4, ip4, info4 = api.lu_factor(dev(A4), method="ozaki")
    x4 = host(api.lu_solve(LU4, ip4, dev(b4)))
    rng = np.random.default_rng(9)
    rows, cols = rng.integers(0, n, 64), rng.integers(0, n, 64)
    E = np.zeros((2, 4, 64, n))
    E[0, 0, np.arange(64), rows] = 1.0
    W = host(api.lu_solve(LU4, ip4, dev(E)))      # w_s = A^{-1} e_{i_s}, QD, [2, 4, 64, n]
    torch.cuda.synchronize()
    assert int(host(info4)[0]) == 0
    # s_k = c^H w_k exactly: the row c^H (conjugated) times the columns of W
    cH = np.zeros((2, 4, n, 1))
    cH[0, 0, :, 0] = c[0, 0, 0]
    cH[1, 0, :, 0] = -c[1, 0, 0]
    sdot = orc.exact_entries(cH, W, np.zeros(64, np.int64), np.arange(64, dtype=np.int64))  # [64, 2, 4]
    fr = lambda v: sum((Fraction(float(t)) for t in v), Fraction(0))
    h = Fraction(1, 2 ** 60)
    gscale = np.abs(gA[:, 0]).max()
    worst = 0.0
    for k, (i, j) in enumerate(zip(rows, cols)):
        s = (fr(sdot[k, 0]), fr(sdot[k, 1]))
        xj = (fr(x4[0, :, 0, j]), fr(x4[1, :, 0, j]))
        wj = (fr(W[0, :, k, j]), fr(W[1, :, k, j]))
        for part in (0, 1):                       # perturb Re(A_ij) or Im(A_ij)
            t = (h, Fraction(0)) if part == 0 else (Fraction(0), h)
            fs = []
            for sgn in (1, -1):
                ts = (sgn * t[0], sgn * t[1])
                den = (1 + ts[0] * wj[0] - ts[1] * wj[1], ts[0] * wj[1] + ts[1] * wj[0])
                num = (ts[0] * xj[0] - ts[1] * xj[1], ts[0] * xj[1] + ts[1] * xj[0])
                d2 = den[0] ** 2 + den[1] ** 2
                fs.append(((num[0] * den[0] + num[1] * den[1]) / d2, (num[1] * den[0] - num[0] * den[1]) / d2))
            # L(t) - L(-t) = -Re(s (f(t) - f(-t))), Re(c^H x) cancels
            df = (fs[0][0] - fs[1][0], fs[0][1] - fs[1][1])
            fd = float(-(s[0] * df[0] - s[1] * df[1]) / (2 * h))
            g = gA[part, :, j, i].sum()
            worst = max(worst, abs(g - fd) / gscale)
    assert worst <= 2.0 ** -70, worst
