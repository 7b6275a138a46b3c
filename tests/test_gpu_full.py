"""Full-size checks at n = 4096 in the benchmark's launch configuration
(blocked, nb = 64 with the 4M and 3M updates, nb = 128 with the Ozaki update), by properties that hold at any
size and that the oracle can evaluate one output at a time:

* backward error with the exact residual: ||b - A x|| / (||A|| ||x||) <= 16 n u;
* sampled entries of L U equal those of P A within 2^6 n u max|A|
  (each entry is an exact dot product evaluated by the oracle);
* partial pivoting on cabs1 bounds every multiplier: |l_ik| <= sqrt(2);
* against the oracle's own run on the same matrix (fixtures under
  tests/golden written by make_full_pivots.py from the oracle alone: DD and TD
  at n = 4096, QD at n = 2048): the pivot sequence identical (bit-exact
  integers), 64 sampled entries of the factors within 2^10 n u max|A| max|LU|
  and 64 sampled solution entries within 2^12 n u max|x| of the oracle's.
"""
import os
import sys

import numpy as np
import pytest

from gpu_util import backward_error, bound, dev, host, planes_diff
from helpers import U_EXP
from paper_2403_16013_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402

# (precision, order) of the oracle fixtures
FIXTURES = {("dd", 4096), ("td", 4096), ("qd", 2048)}


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_16013_gb300 import api as a
    from paper_2403_16013_gb300 import build
    build.build()
    return a


def _apply_pivots(A, ipiv):
    P = np.arange(A.shape[3])
    for k, p in enumerate(ipiv - 1):
        P[k], P[p] = P[p], P[k]
    return P


@pytest.mark.parametrize("prec,method,n", [("dd", "4m", 4096), ("dd", "3m", 4096), ("td", "4m", 4096),
                                           ("qd", "4m", 4096), ("dd", "ozaki", 4096), ("td", "ozaki", 4096),
                                           ("qd", "ozaki", 4096), ("qd", "4m", 2048), ("qd", "ozaki", 2048),
                                           # more than 32 panel rows per CTA (152 CTAs) in the first panels
                                           ("dd", "ozaki", 5120), ("td", "ozaki", 5120)])
def test_full_size(api, orc, prec, method, n):
    import torch
    L = {"dd": 2, "td": 3, "qd": 4}[prec]
    A = inputs.gaussian_matrix(n, L, seed=1)
    b = inputs.complex_gaussian_vector(n, L, seed=2)
    Ad = dev(A)
    LU, ipiv, info = api.lu_factor(Ad, method=method, nb=128 if method == "ozaki" else 64)
    x = api.lu_solve(LU, ipiv, dev(b))
    torch.cuda.synchronize()
    assert int(host(info)[0]) == 0
    X, LUh, ip = host(x), host(LU), host(ipiv)
    del Ad, LU, x
    eta = backward_error(orc, A, X, b)
    assert eta <= bound(n, L), eta
    # multipliers bounded by sqrt(2)
    Lval = np.hypot(LUh[0, 0], LUh[1, 0])            # [col, row] magnitudes of the leading limbs
    low = np.tril(np.ones((n, n), bool), -1).T       # (col, row) with row > col
    assert Lval[low].max() <= np.sqrt(2) * (1 + 1e-12)
    # sampled entries of L U against P A
    rng = np.random.default_rng(9)
    rows = rng.integers(0, n, 96)
    cols = rng.integers(0, n, 96)
    P = _apply_pivots(A, ip)
    PA = np.ascontiguousarray(A[:, :, :, P])
    d = orc.exact_entries(LUh, LUh, rows, cols, C=PA, sign=-1, lu=True)   # exact P A - L U, rounded
    amax = np.abs(A[:, 0]).max()
    err = np.abs(d[:, :, 0]).max()
    assert err <= 2.0 ** 6 * n * 2.0 ** -U_EXP[L] * amax, err
    if (prec, n) in FIXTURES:
        g = make_golden.load(os.path.join(GOLDEN, f"full_{prec}_n{n}.txt"))
        assert int(g["n"][0]) == n and int(g["info"][0]) == 0
        mism = np.nonzero(ip != g["ipiv"])[0]
        assert mism.size == 0, ("pivots differ from the oracle", mism[:4], ip[mism[:4]], g["ipiv"][mism[:4]])
        u = 2.0 ** -U_EXP[L]
        lu = LUh[:, :, g["lu_cols"], g["lu_rows"]].transpose(2, 0, 1)          # [s, 2, L]
        dl = planes_diff(orc, lu, g["lu"]).max()
        assert dl <= 2.0 ** 10 * n * u * amax * max(1.0, np.abs(g["lu"][:, :, 0]).max()), dl
        xg = X[:, :, 0, g["x_rows"]].transpose(2, 0, 1)
        dx = planes_diff(orc, xg, g["x"]).max()
        assert dx <= 2.0 ** 12 * n * u * np.abs(g["x"][:, :, 0]).max(), dx
