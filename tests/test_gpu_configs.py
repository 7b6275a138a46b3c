"""The ill-conditioned and the exponent-spread workloads on the GPU.

Ill-conditioned complex matrix (n = 2048): A = Q1 diag(sigma) Q2^H, Q1 and Q2
products of 8 Householder reflectors from seeded complex Gaussian vectors,
sigma_i = r^i geometric from 1 to 1e-40 (kappa_2(A) = 1e40), formed in QD by
the oracle; x_true = 1 + i, b = A x_true exactly, rounded to QD; DD and TD
runs take the leading 2 / 3 limbs of A and b.  The paper's error study
(Sec. 4: maximum relative error of the solution) measured on it:

* every precision's normwise backward error (exact residual) <= 16 n u
  (backward stability does not depend on kappa);
* QD forward error against x_true <= 16 n kappa u_QD; TD forward error
  against the QD solution <= 16 n kappa u_TD; DD (kappa u_DD >> 1) only the
  backward error.  The forward errors are printed for the record.

Exponent spread (entries N(0,1) 2^e, e uniform in [-20, 20]; seed 3): the
n = 4096 DD LU with the Ozaki update against the plain 4M update (same
pivots, both backward errors <= 16 n u), and the 4096^3 DD and TD ZGEMM with
the Ozaki and plain forms on 64 sampled entries against the exact product.
"""
import numpy as np
import pytest

from gpu_util import backward_error, bound, dev, exact_diff, host
from helpers import U_EXP
from oracle import ozaki
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


@pytest.fixture(scope="module")
def ill(orc):
    n = 2048
    V1 = inputs.householder_vectors(n, 8, seed=3)
    V2 = inputs.householder_vectors(n, 8, seed=4)
    A = orc.make_ill_conditioned(4, n, V1, V2, inputs.geometric_ratio(n, decades=40.0))
    xr, xi = inputs.ones_x_true(n)
    b = inputs.exact_rhs(A, xr, xi, L_out=4)
    return A, b


def _fwd(orc, x, ref):
    """max_i |x_i - ref_i| / max_i |ref_i|, the differences taken exactly
    (superaccumulator over all limbs of both) and rounded to binary64."""
    d = [exact_diff(orc, x[c, :, 0, :], ref[c, :, 0, :]) for c in range(2)]
    rv = np.hypot(ref[0].sum(axis=0), ref[1].sum(axis=0))
    return float(np.hypot(d[0], d[1]).max() / rv.max())


@pytest.mark.parametrize("method", ["ozaki", "4m"])
def test_ill_conditioned_dd_td_qd(api, orc, ill, method):
    import torch
    A4, b4 = ill
    n, kappa = A4.shape[2], 1e40
    xs, rep = {}, {}
    for L in (4, 3, 2):
        A, b = inputs.truncate_limbs(A4, L), inputs.truncate_limbs(b4, L)
        LU, ipiv, info = api.lu_factor(dev(A), method=method)
        x = api.lu_solve(LU, ipiv, dev(b))
        torch.cuda.synchronize()
        assert int(host(info)[0]) == 0
        X = host(x)
        eta = backward_error(orc, A, X, b)
        assert eta <= bound(n, L), (L, eta)
        xs[L] = X
        rep[L] = {"eta": eta}
    xt = inputs.int_vector_planes(*inputs.ones_x_true(n), 4)
    u = {L: 2.0 ** -U_EXP[L] for L in (2, 3, 4)}
    for L in (4, 3, 2):
        rep[L]["fe_true"] = _fwd(orc, xs[L], xt)
        rep[L]["fe_vs_qd"] = _fwd(orc, xs[L], xs[4]) if L < 4 else 0.0
    assert rep[4]["fe_true"] <= 16 * n * kappa * u[4], rep[4]
    assert rep[3]["fe_vs_qd"] <= 16 * n * kappa * u[3], rep[3]
    for L in (2, 3, 4):
        print(f"ill-conditioned n={n} kappa=1e40 {method} L={L}: backward error {rep[L]['eta']:.3e}, "
              f"forward error vs x_true {rep[L]['fe_true']:.3e}, vs QD solution {rep[L]['fe_vs_qd']:.3e}")


def test_spread_lu_n4096_ozaki_vs_plain(api, orc):
    import torch
    n, L = 4096, 2
    A = inputs.spread_matrix(n, n, L, seed=3, spread=20)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.exact_rhs(A, xr, xi, L_out=L)
    res = {}
    for method in ("ozaki", "4m"):
        LU, ipiv, info = api.lu_factor(dev(A), method=method)
        x = api.lu_solve(LU, ipiv, dev(b))
        torch.cuda.synchronize()
        assert int(host(info)[0]) == 0
        res[method] = (host(ipiv), backward_error(orc, A, host(x), b))
        del LU, x
    assert np.array_equal(res["ozaki"][0], res["4m"][0])
    for method, (_, eta) in res.items():
        assert eta <= bound(n, L), (method, eta)
        print(f"spread 2^+-20 n={n} DD {method}: backward error {eta:.3e}")


@pytest.mark.parametrize("L", [2, 3])
def test_spread_zgemm_4096(api, orc, L):
    """m = n = k = 4096, entries with exponents spread over 2^+-20: Ozaki
    within its bound 2^(Ea_i + Eb_j - beta S) 2k (L + S + 2) (row / column
    scales; the spread costs accuracy only relative to the row and column
    maxima), the plain 4M form within 2 L^2 (k + 2) u_L sum|a||b| (the
    bound of the leveled accumulation, test_gpu_zgemm)."""
    beta, S = ozaki.CFG[L]
    m = n = k = 4096
    A = inputs.spread_matrix(m, k, L, seed=3, spread=20)
    B = inputs.spread_matrix(k, n, L, seed=4, spread=20)
    rng = np.random.default_rng(6)
    rows = rng.integers(0, m, 64)
    cols = rng.integers(0, n, 64)
    ex = orc.exact_entries(A, B, rows, cols)
    Ea = np.array([ozaki.scale([A[c, 0, j, i] for c in range(2) for j in range(k)]) for i in rows])
    Eb = np.array([ozaki.scale([B[c, 0, j, i] for c in range(2) for i in range(k)]) for j in cols])
    aR, aI = np.abs(A[0, 0][:, rows]), np.abs(A[1, 0][:, rows])
    bR, bI = np.abs(B[0, 0][cols, :].T), np.abs(B[1, 0][cols, :].T)
    sab = np.stack([(aR * bR + aI * bI).sum(axis=0), (aR * bI + aI * bR).sum(axis=0)], axis=1)
    import torch
    Ad, Bd = dev(A), dev(B)
    ci = torch.as_tensor(cols, device="cuda")
    ri = torch.as_tensor(rows, device="cuda")
    for method in ("ozaki", "4m"):
        C = api.zgemm(Ad, Bd, method=method)
        g = host(C[:, :, ci, ri].permute(2, 0, 1).contiguous())                         # [s, 2, L]
        del C
        V = np.concatenate([g, -ex], axis=2).reshape(-1, L + 4)
        d = np.abs(orc.exact_sum_rows(V, 1)[:, 0].reshape(-1, 2))
        rnd = 2.0 ** (2 - 53 * L) * np.abs(ex[:, :, 0])
        if method == "ozaki":
            tol = (np.ldexp(1.0, (Ea + Eb - beta * S).astype(int)) * 2 * k * (L + S + 2))[:, None] + rnd
        else:
            tol = 2 * L * L * (k + 2) * 2.0 ** (-53 * L) * sab * 1.01 + rnd
        assert np.all(d <= tol), (method, float(np.max(d / tol)))
        rel = float(np.max(d / np.maximum(sab, 1e-300)))
        print(f"spread 2^+-20 ZGEMM 4096^3 L={L} {method}: max |error| / sum|a||b| = {rel:.3e}")
