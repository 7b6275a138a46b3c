"""GPU parity of the LU factorisation and solve against the CPU oracle.

Pivots must be identical (integers, bit-exact); the normwise backward error
with the exact residual must be below 16 n u (u = 2^-104 / 2^-157 / 2^-209);
the factors agree with the oracle's element by element within
2^10 n u max|A| (both are backward-stable GEPP on the same input with the same
pivots, differing only in rounding order).
"""
import numpy as np
import pytest

from gpu_util import backward_error, bound, dev, host, planes_diff
from helpers import U_EXP
from lu_cases import known_factor_case
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


def _factor_compare(api, orc, A, method, nb=0):
    n, L = A.shape[2], A.shape[1]
    LU, ipiv, info = api.lu_factor(dev(A), method=method, nb=nb)
    LUo, ipo, info_o, gap = orc.zgetrf(A)
    ipg = host(ipiv)
    assert int(host(info)[0]) == info_o
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    LUg = host(LU)
    scale = np.abs(A[:, 0]).max()
    diff = planes_diff(orc, LUg, LUo).max()
    assert diff <= 2.0 ** 10 * n * 2.0 ** -U_EXP[L] * scale * max(1.0, np.abs(LUo[:, 0]).max()), diff
    return LU, ipiv, LUg, ipg


@pytest.mark.parametrize("L", [2, 3, 4])
def test_unblocked_small(api, orc, L):
    n = 128 if L == 2 else 72
    A = inputs.uniform_matrix(n, L, seed=0)
    LU, ipiv, _, _ = _factor_compare(api, orc, A, "unblocked")
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("method", ["4m", "3m"])
def test_blocked_ragged(api, orc, L, method):
    n = 200 if L < 4 else 150
    A = inputs.gaussian_matrix(n, L, seed=1)
    LU, ipiv, LUg, ipg = _factor_compare(api, orc, A, method, nb=64 if L < 4 else 48)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L)
    xo = orc.zgetrs(LUg, ipg, b)
    assert planes_diff(orc, x, xo).max() <= 2.0 ** 12 * n * 2.0 ** -U_EXP[L]


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("n", [1, 17, 40])
def test_known_factor_bit_exact(api, orc, L, n):
    A, ipiv_ref, packed, xr, xi = known_factor_case(n, L, seed=70 + n)
    for method, nb in (("4m", 16), ("3m", 8), ("unblocked", 0)):
        LU, ipiv, info = api.lu_factor(dev(A), method=method, nb=nb)
        assert np.array_equal(host(ipiv), ipiv_ref)
        assert np.array_equal(host(LU), packed), method
        b = inputs.exact_rhs(A, xr, xi, L_out=L)
        x = host(api.lu_solve(LU, ipiv, dev(b)))
        assert np.array_equal(x[0, 0, 0], xr.astype(float)) and np.array_equal(x[1, 0, 0], xi.astype(float))


@pytest.mark.parametrize("L", [2, 3])
def test_solve_conjugate_transpose(api, orc, L):
    n = 96
    A = inputs.gaussian_matrix(n, L, seed=2)
    LU, ipiv, info = api.lu_factor(dev(A), nb=32)
    c = inputs.complex_gaussian_vector(n, L, seed=3)
    y = host(api.lu_solve(LU, ipiv, dev(c), trans="C"))
    yo = orc.zgetrs(host(LU), host(ipiv), c, "C")
    assert planes_diff(orc, y, yo).max() <= 2.0 ** 12 * n * 2.0 ** -U_EXP[L] * np.abs(yo[:, 0]).max()


def test_zero_column_info(api, orc):
    n, L = 40, 2
    A = inputs.gaussian_matrix(n, L, seed=4)
    A[:, :, 7, :] = 0.0
    LU, ipiv, info = api.lu_factor(dev(A), nb=16)
    LUo, ipo, info_o, _ = orc.zgetrf(A)
    assert int(host(info)[0]) == info_o == 8
    assert np.array_equal(host(ipiv), ipo)


def test_multiple_rhs_and_padding(api, orc):
    n, L, nrhs = 70, 2, 5
    A = inputs.gaussian_matrix(n, L, seed=5)
    Ap = np.zeros((2, L, n, n + 3))
    Ap[..., :n] = A
    LU, ipiv, _ = api.lu_factor(dev(Ap), nb=32)
    Bm = inputs.gaussian_matrix(nrhs, L, seed=6, rows=n)
    X = host(api.lu_solve(LU, ipiv, dev(Bm)))
    LUo, ipo, _, _ = orc.zgetrf(A)
    assert np.array_equal(host(ipiv), ipo)
    Xo = orc.zgetrs(LUo, ipo, Bm)
    assert planes_diff(orc, X, Xo).max() <= 2.0 ** 12 * n * 2.0 ** -U_EXP[L] * np.abs(Xo[:, 0]).max()


def test_bounded_wait_runs_out_and_context_survives(api, orc):
    """The panels' inter-CTA wait on a flag that nothing sets runs out within
    its budget and records it in the status word; the context stays usable
    (a factorisation right after it matches the oracle)."""
    from paper_2403_16013_gb300 import binding
    assert binding.selftest_wait_timeout() == 1
    n, L = 40, 2
    A = inputs.gaussian_matrix(n, L, seed=8)
    LU, ipiv, info = api.lu_factor(dev(A), method="ozaki")
    LUo, ipo, info_o, _ = orc.zgetrf(A)
    assert int(host(info)[0]) == info_o == 0
    assert np.array_equal(host(ipiv), ipo)


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("method", ["4m", "ozaki"])
def test_pivot_near_ties(api, orc, L, method):
    """Leading limbs drawn from the integers -3..3 (lower limbs random in their
    canonical range): in the first columns many rows share the leading-limb
    key |Re a_0| + |Im a_0| inside one CTA and across CTAs (n = 200: 25 CTAs
    of 8 rows), so the panels' candidate and exchange steps take their
    full-key path, where only the lower limbs (or the row index, for equal
    values) decide.  Pivots identical to the oracle's exact cabs1 pivoting."""
    import numpy as np
    n = 200
    rng = np.random.default_rng(91 + L)
    re = rng.integers(-3, 4, (n, n)).astype(float)
    im = rng.integers(-3, 4, (n, n)).astype(float)
    A = inputs._assemble(re, im, L, rng, None)
    for r in (7, 11):                         # rows 7 and 11: column 0 exactly 3 + 3i (equal keys,
        A[:, :, 0, r] = 0.0                   # the largest k0; the lower row wins unless another
        A[0, 0, 0, r] = A[1, 0, 0, r] = 3.0   # row's lower limbs make its key larger)
    LU, ipiv, LUg, ipg = _factor_compare(api, orc, A, method, nb=0)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L)
