"""GPU parity of the Strassen form (Sec. 2.3: one level of Winograd's variant,
seven 3M block products instead of eight), through the C ABI: standalone
ZGEMM (C = A B and C - A B) and the LU trailing update.

* Dyadic operands (entries j/8, |j| <= 16): every block sum, product and
  combination is exact, so the result equals the exact product bit for bit
  (any wrong block, sign or index shows), including odd m, n and k (the
  peeled last row, column and k index).
* Gaussian limbs against the exact product: Winograd's variant is accurate
  normwise, not componentwise (its block sums mix entries of different
  size); the error stays within 64 L^2 (k + 8) k u_L max|A| max|B|.
* LU with the Strassen update: the oracle's pivots, factors within the
  parity tolerance, backward error <= 16 n u; odd n (ragged blocks).
"""
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


def _gemm(api, A, B, C):
    return host(api.zgemm(dev(A), dev(B), None if C is None else dev(C), method="strassen"))


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("m,n,k", [(64, 64, 64), (45, 37, 29), (1, 70, 33), (70, 1, 17), (33, 34, 1)])
def test_strassen_dyadic_bit_exact(api, orc, L, m, n, k):
    rng = np.random.default_rng(m + 3 * n + 7 * k)
    A = np.zeros((2, L, k, m))
    B = np.zeros((2, L, n, k))
    C = np.zeros((2, L, n, m))
    A[:, 0] = rng.integers(-16, 17, (2, k, m)) / 8.0
    B[:, 0] = rng.integers(-16, 17, (2, n, k)) / 8.0
    C[:, 0] = rng.integers(-64, 65, (2, n, m)) / 4.0
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    for beta_mode in (0, 1):
        Cin = C if beta_mode else None
        out = _gemm(api, A, B, Cin)
        ex = orc.exact_entries(A, B, rows, cols, C=Cin, sign=-1 if beta_mode else 1)
        assert np.all(ex[:, :, 1:] == 0)
        assert np.array_equal(out[0, 0, cols, rows], ex[:, 0, 0]), beta_mode
        assert np.array_equal(out[1, 0, cols, rows], ex[:, 1, 0]), beta_mode
        assert np.all(out[:, 1:] == 0)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("beta_mode", [0, 1])
@pytest.mark.parametrize("m,n,k", [(45, 37, 29), (96, 80, 64)])
def test_strassen_against_exact(api, orc, L, beta_mode, m, n, k):
    A = inputs.gaussian_matrix(k, L, seed=71, rows=m)
    B = inputs.gaussian_matrix(n, L, seed=72, rows=k)
    C = inputs.gaussian_matrix(n, L, seed=73, rows=m) if beta_mode else None
    out = _gemm(api, A, B, C)
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    ex = orc.exact_entries(A, B, rows, cols, C=C, sign=-1 if beta_mode else 1)
    g = np.stack([out[0, :, cols, rows], out[1, :, cols, rows]], axis=1)
    d = planes_diff(orc, g, ex)
    amax, bmax = np.abs(A[:, 0]).max(), np.abs(B[:, 0]).max()
    tol = 64 * L * L * (k + 8) * k * 2.0 ** (-53 * L) * amax * bmax
    if C is not None:
        tol += 4 * 2.0 ** (-53 * L) * np.abs(C[:, 0]).max()
    assert d.max() <= tol, (d.max(), tol)


def test_strassen_k_zero(api):
    m, n, L = 20, 9, 2
    A = np.zeros((2, L, 0, m))
    B = np.zeros((2, L, n, 1))
    C = inputs.gaussian_matrix(n, L, seed=45, rows=m)
    assert np.all(_gemm(api, A, B, None) == 0)
    assert np.array_equal(_gemm(api, A, B, C), C)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_lu_strassen_parity(api, orc, L):
    n = 201 if L < 4 else 151
    A = inputs.gaussian_matrix(n, L, seed=1)
    LU, ipiv, info = api.lu_factor(dev(A), method="strassen", nb=64 if L < 4 else 48)
    assert int(host(info)[0]) == 0
    LUo, ipo, _, gap = orc.zgetrf(A)
    ipg = host(ipiv)
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    diff = planes_diff(orc, host(LU), LUo).max()
    assert diff <= 2.0 ** 12 * n * 2.0 ** -U_EXP[L] * np.abs(A[:, 0]).max() * max(1.0, np.abs(LUo[:, 0]).max())
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L)
