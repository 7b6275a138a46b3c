"""GPU parity of the plain complex multi-component ZGEMM (FP64 pipe) through
the C ABI: C = A B (beta_mode 0) and C = C - A B (beta_mode 1), 4M (Eq. 1)
and 3M (Eq. 3), DD / TD / QD.

* Against the exact product (the oracle's superaccumulator, every entry of
  ragged small shapes and 64 sampled entries of m = n = k = 1024): the 4M
  result within 2 L^2 (k + 2) u_L sum|a||b| per component plus the rounding
  of the result to L limbs, u_L = 2^-53L; the 3M imaginary part within
  Higham's 3M form 2 (L^2 + 4) (k + 4) u_L (|Re a| + |Im a|)(|Re b| + |Im b|).
  The GPU accumulates every real product in L levels, exactly (TwoSum,
  TwoProd) down to the last level, where L^2 terms of order u^(L-1) |ab| per
  product are added with rounding (4 / 9 / 16 for DD / TD / QD); each such
  rounding costs at most 2^-53 times the last level's magnitude, about u^(L-1)
  sum|ab|, hence the L^2 (k + 2) form (the oracle, which rounds the exact
  result of every operation once, is pinned to the tighter 4 (k + 2)).
* Dyadic operands whose every product and sum is exact in binary64: the GPU
  result equals the exact one bit for bit (catches any index, sign or
  transposition error exactly).
* k = 0: C = 0 (beta_mode 0) or C unchanged (beta_mode 1).
"""
import numpy as np
import pytest

from gpu_util import dev, host
from paper_2403_16013_gb300 import inputs

pytestmark = pytest.mark.gpu
PREC = {2: "dd", 3: "td", 4: "qd"}


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_16013_gb300 import api as a
    from paper_2403_16013_gb300 import build
    build.build()
    return a


def _gemm(api, A, B, C, method):
    """The library's zgemm on [2, L, k, m] x [2, L, n, k] (C: [2, L, n, m] or None)."""
    return host(api.zgemm(dev(A), dev(B), None if C is None else dev(C), method=method))


def _check_against_exact(orc, A, B, C, out, rows, cols, method):
    L, k = A.shape[1], A.shape[2]
    ex = orc.exact_entries(A, B, rows, cols, C=C, sign=-1 if C is not None else 1)      # [s, 2, 4]
    g = np.stack([out[0, :, cols, rows], out[1, :, cols, rows]], axis=1)                 # [s, 2, L]
    V = np.concatenate([g, -ex], axis=2).reshape(-1, L + 4)
    d = np.abs(orc.exact_sum_rows(V, 1)[:, 0].reshape(-1, 2))                            # exact |gpu - exact|
    u = 2.0 ** (-53 * L)
    aR, aI = np.abs(A[0, 0][:, rows]), np.abs(A[1, 0][:, rows])                          # [k, s]
    bR, bI = np.abs(B[0, 0][cols, :].T), np.abs(B[1, 0][cols, :].T)                       # [k, s]
    rr = (aR * bR + aI * bI).sum(axis=0)
    ri = (aR * bI + aI * bR).sum(axis=0)
    s3 = ((aR + aI) * (bR + bI)).sum(axis=0)
    rnd = 2.0 ** (2 - 53 * L) * np.abs(ex[:, :, 0])
    c4, c3 = 2 * L * L, 2 * (L * L + 4)
    tol_re = c4 * (k + 2) * u * rr * 1.01 + rnd[:, 0]
    tol_im = (c3 * (k + 4) * u * s3 if method == "3m" else c4 * (k + 2) * u * ri) * 1.01 + rnd[:, 1]
    if C is not None:   # the subtraction from C adds one rounding of |C| at the last level
        cabs = np.abs(C[:, 0][:, cols, rows])                                            # [2, s]
        tol_re = tol_re + 4 * u * cabs[0]
        tol_im = tol_im + 4 * u * cabs[1]
    assert np.all(d[:, 0] <= tol_re), float(np.max(d[:, 0] / tol_re))
    assert np.all(d[:, 1] <= tol_im), float(np.max(d[:, 1] / tol_im))


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("beta_mode", [0, 1])
@pytest.mark.parametrize("m,n,k", [(45, 37, 29), (1, 70, 33), (70, 1, 17), (16, 16, 1)])
def test_zgemm_plain_against_exact(api, orc, L, method, beta_mode, m, n, k):
    """Every entry of ragged shapes (tiles of 16 with ragged edges in m, n, k)."""
    A = inputs.gaussian_matrix(k, L, seed=41, rows=m)
    B = inputs.gaussian_matrix(n, L, seed=42, rows=k)
    C = inputs.gaussian_matrix(n, L, seed=43, rows=m) if beta_mode else None
    out = _gemm(api, A, B, C, method)
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    _check_against_exact(orc, A, B, C, out, rows.ravel(), cols.ravel(), method)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("method", ["4m", "3m"])
def test_zgemm_plain_1024_sampled(api, orc, L, method):
    """The standalone product of m = n = k = 1024 (Gaussian limbs), 64 sampled
    entries against the exact product, C = A B and C - A B."""
    m = n = k = 1024
    A = inputs.gaussian_matrix(k, L, seed=1, rows=m)
    B = inputs.gaussian_matrix(n, L, seed=2, rows=k)
    rng = np.random.default_rng(5)
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, 62)])
    cols = np.concatenate([[n - 1, 0], rng.integers(0, n, 62)])
    out = _gemm(api, A, B, None, method)
    _check_against_exact(orc, A, B, None, out, rows, cols, method)
    C = inputs.gaussian_matrix(n, L, seed=3, rows=m)
    out = _gemm(api, A, B, C, method)
    _check_against_exact(orc, A, B, C, out, rows, cols, method)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("method", ["4m", "3m"])
def test_zgemm_plain_dyadic_bit_exact(api, orc, L, method):
    """Entries j/8 with |j| <= 16: every product and partial sum is exact in
    the leading limb, so the result is exact and the lower limbs are zero."""
    m, n, k = 35, 29, 40
    rng = np.random.default_rng(44)
    A = np.zeros((2, L, k, m))
    B = np.zeros((2, L, n, k))
    C = np.zeros((2, L, n, m))
    A[:, 0] = rng.integers(-16, 17, (2, k, m)) / 8.0
    B[:, 0] = rng.integers(-16, 17, (2, n, k)) / 8.0
    C[:, 0] = rng.integers(-64, 65, (2, n, m)) / 4.0
    for beta_mode in (0, 1):
        Cin = C if beta_mode else None
        out = _gemm(api, A, B, Cin, method)
        rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
        rows, cols = rows.ravel(), cols.ravel()
        ex = orc.exact_entries(A, B, rows, cols, C=Cin, sign=-1 if beta_mode else 1)
        assert np.all(ex[:, :, 1:] == 0)
        assert np.array_equal(out[0, 0, cols, rows], ex[:, 0, 0]), (method, beta_mode)
        assert np.array_equal(out[1, 0, cols, rows], ex[:, 1, 0]), (method, beta_mode)
        assert np.all(out[:, 1:] == 0)


@pytest.mark.parametrize("method", ["4m", "3m", "ozaki"])
def test_zgemm_k_zero(api, method):
    m, n, L = 20, 9, 2
    A = np.zeros((2, L, 0, m))
    B = np.zeros((2, L, n, 1))        # k = 0 rows (leading dimension 1)
    C = inputs.gaussian_matrix(n, L, seed=45, rows=m)
    assert np.all(_gemm(api, A, B, None, method) == 0)
    assert np.array_equal(_gemm(api, A, B, C, method), C)
