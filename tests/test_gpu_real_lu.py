"""GPU parity of the real (one-plane) DD / TD / QD LU and solve (dgetrf_*,
dgetrs_*) against the CPU oracle's real LU (orc_dgetrf / orc_dgetrs), through
the C ABI.

* Random matrices, every trailing-update method (4M, 3M, Ozaki, unblocked):
  pivots identical to the oracle's (partial pivoting on |a|, ties to the
  lowest row); factors within 2^10 n u max|A| max|LU| of the oracle's
  (exact difference of all limbs); the 'N' and 'T' solutions within
  2^12 n u max|x| of the oracle's; normwise backward error with the exact
  residual <= 16 n u.
* Known factors A = P^T L U with dyadic entries: pivots and factors bit-exact,
  A x = b solved exactly.
* A zero column: info = the first zero pivot, as in the oracle.
"""
import numpy as np
import pytest

from gpu_util import backward_error, bound, dev, host, planes_diff
from helpers import U_EXP
from lu_cases import known_factor_case_real
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


def _embed(R):
    """[L, cols, ld] real planes -> [2, L, cols, ld] complex planes, zero imaginary part."""
    return np.ascontiguousarray(np.stack([R, np.zeros_like(R)]))


def _real(n, L, seed, rows=None):
    return np.ascontiguousarray(inputs.gaussian_matrix(n, L, seed=seed, rows=rows)[0])


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("method", ["4m", "3m", "ozaki", "unblocked"])
def test_real_lu_parity(api, orc, L, method):
    n = 200 if L < 4 else 150
    A = _real(n, L, seed=61)
    LU, ipiv, info = api.dlu_factor(dev(A), method=method)
    LUo, ipo, info_o, gap = orc.dgetrf(A)
    ipg = host(ipiv)
    assert int(host(info)[0]) == info_o == 0
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    LUg = host(LU)
    u = 2.0 ** -U_EXP[L]
    diff = planes_diff(orc, _embed(LUg), _embed(LUo)).max()
    assert diff <= 2.0 ** 10 * n * u * np.abs(A[0]).max() * max(1.0, np.abs(LUo[0]).max()), diff
    # solves 'N' and 'T' against the oracle's, on the oracle's own factors' answers
    Bm = _real(3, L, seed=62, rows=n)                        # [L, 3, n]: three right-hand sides
    for trans in ("N", "T"):
        X = host(api.dlu_solve(LU, ipiv, dev(Bm), trans=trans))
        Xo = orc.dgetrs(LUo, ipo, Bm, trans)
        dx = planes_diff(orc, _embed(X), _embed(Xo)).max()
        assert dx <= 2.0 ** 12 * n * u * np.abs(Xo[0]).max(), (trans, dx)
    # backward error of A x = b with the exact residual (complex embedding, zero imaginary part)
    xr = np.ones(n, np.int64)
    b = inputs.truncate_limbs(inputs.exact_rhs(_embed(A), xr, np.zeros(n, np.int64), L_out=4), L)[0]
    x = host(api.dlu_solve(LU, ipiv, dev(np.ascontiguousarray(b))))
    assert backward_error(orc, _embed(A), _embed(x), _embed(b)) <= bound(n, L)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("method,nb", [("4m", 16), ("3m", 8), ("unblocked", 0), ("ozaki", 0)])
def test_real_known_factor_bit_exact(api, orc, L, method, nb):
    n = 40
    A, ipiv_ref, packed, x = known_factor_case_real(n, L, seed=120)
    LU, ipiv, info = api.dlu_factor(dev(A), method=method, nb=nb)
    assert np.array_equal(host(ipiv), ipiv_ref)
    assert np.array_equal(host(LU), packed), method
    b = inputs.exact_rhs(_embed(A), x, np.zeros(n, np.int64), L_out=L)[0]
    X = host(api.dlu_solve(LU, ipiv, dev(np.ascontiguousarray(b))))
    assert np.array_equal(X[0, 0], x.astype(float)) and np.all(X[1:] == 0)


def test_real_zero_column_info(api, orc):
    n, L = 40, 3
    A = _real(n, L, seed=63)
    A[:, 9, :] = 0.0
    LU, ipiv, info = api.dlu_factor(dev(A), method="ozaki")
    LUo, ipo, info_o, _ = orc.dgetrf(A)
    assert int(host(info)[0]) == info_o == 10
    assert np.array_equal(host(ipiv), ipo)
