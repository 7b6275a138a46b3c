"""GPU parity of the Ozaki-scheme path (tcgen05 slice products).

* split: digits and scales bit-exact against the oracle's integer definition
  (oracle/ozaki.py), both operand sides, ragged sizes, several K chunks;
* ZGEMM (C = AB and C - AB): against the exact product (oracle
  superaccumulator) within the Ozaki bound
  2^(Ea_i + Eb_j) 2k 2^(-beta S) (L + S + 2) + 2^(2 - 53L) |result|;
* LU with the Ozaki update: pivots identical to the oracle's (no mismatch
  accepted), backward error
  <= 16 n u; known-factor matrices reproduced bit for bit.
"""
import numpy as np
import pytest

from gpu_util import backward_error, bound, dev, host, planes_diff
from helpers import U_EXP
from lu_cases import known_factor_case
from oracle import ozaki
from paper_2403_16013_gb300 import inputs

pytestmark = pytest.mark.gpu
PREC = {2: "dd", 3: "td", 4: "qd"}
NTILE = {2: 32, 3: 16, 4: 16}


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_16013_gb300 import api as a
    from paper_2403_16013_gb300 import build
    build.build()
    return a


def _gpu_split(side, X, rows, cols, L):
    import torch
    from paper_2403_16013_gb300 import binding
    beta, S = ozaki.CFG[L]
    if side == 0:
        nch, pad = -(-cols // 32), -(-rows // 128) * 128
    else:
        nch, pad = -(-rows // 32), -(-(2 * cols) // NTILE[L]) * NTILE[L]
    sl = torch.zeros((nch, S, pad, 64), dtype=torch.bfloat16, device="cuda")
    E = torch.zeros(rows if side == 0 else cols, dtype=torch.int32, device="cuda")
    Xd = dev(X)
    rc = binding.zozaki_split(PREC[L], side, rows, cols, Xd.data_ptr(), X.shape[3], sl.data_ptr(), E.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == 0, binding.status_string(rc)
    torch.cuda.synchronize()
    return host(sl.float()).astype(np.int64), host(E)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_split_bit_exact(api, L):
    beta, S = ozaki.CFG[L]
    rows, cols = 150, 40
    X = inputs.spread_matrix(rows, cols, L, seed=21, spread=20)
    X[:, :, 3, :] = 0.0                       # a zero column
    X[:, :, :, 7] = 0.0                       # a zero row
    sl, E = _gpu_split(0, X, rows, cols, L)
    Eo, Do = ozaki.split_rows(X, rows, cols, L)
    assert np.array_equal(E, Eo)
    c = np.arange(cols)
    re = sl[c // 32, :, :rows, c % 32]        # [cols, S, rows]
    im = sl[c // 32, :, :rows, 32 + c % 32]
    assert np.array_equal(np.transpose(re, (1, 2, 0)), Do[..., 0])
    assert np.array_equal(np.transpose(im, (1, 2, 0)), Do[..., 1])
    assert np.all(sl[:, :, rows:, :] == 0)    # padded rows are zero
    # B side
    rows, cols = 40, 37
    X = inputs.spread_matrix(rows, cols, L, seed=22, spread=20)
    sl, E = _gpu_split(1, X, rows, cols, L)
    Eo, Do = ozaki.split_cols(X, rows, cols, L)
    assert np.array_equal(E, Eo)
    r = np.arange(rows)
    for j in range(cols):
        a = sl[r // 32, :, 2 * j, r % 32].T             # [S, rows] real digits
        b = sl[r // 32, :, 2 * j + 1, r % 32].T         # imaginary digits
        assert np.array_equal(a, Do[:, :, j, 0]) and np.array_equal(b, Do[:, :, j, 1])
        assert np.array_equal(sl[r // 32, :, 2 * j, 32 + r % 32].T, -Do[:, :, j, 1])
        assert np.array_equal(sl[r // 32, :, 2 * j + 1, 32 + r % 32].T, Do[:, :, j, 0])


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("beta_mode", [0, 1])
def test_zgemm_ozaki_against_exact(api, orc, L, beta_mode):
    beta, S = ozaki.CFG[L]
    m, n, k = 150, 70, 40
    A = inputs.spread_matrix(m, k, L, seed=31, spread=12)
    B = inputs.spread_matrix(k, n, L, seed=32, spread=12)
    C0 = inputs.gaussian_matrix(n, L, seed=33, rows=m)
    out = host(api.zgemm(dev(A), dev(B), dev(C0) if beta_mode else None, method="ozaki"))
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    ex = orc.exact_entries(A, B, rows, cols, C=C0 if beta_mode else None, sign=-1 if beta_mode else 1)
    Ea, _ = ozaki.split_rows(A, m, k, L)
    Eb, _ = ozaki.split_cols(B, k, n, L)
    # exact difference out - ex per entry, via the superaccumulator
    g = np.stack([out[0, :, cols, rows], out[1, :, cols, rows]], axis=1)   # [nsamp, 2, L]
    V = np.concatenate([g, -ex], axis=2).reshape(-1, L + 4)
    d = orc.exact_sum_rows(V, 1)[:, 0].reshape(-1, 2)
    scale = np.ldexp(1.0, (Ea[rows] + Eb[cols] - beta * S).astype(int)) * 2 * k * (L + S + 2)
    mag = np.abs(ex[:, :, 0])
    tol = scale[:, None] + 2.0 ** (2 - 53 * L) * mag
    assert np.all(np.abs(d) <= tol), float(np.max(np.abs(d) / tol))


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("nb", [0, 64, 96])
def test_lu_ozaki_parity(api, orc, L, nb):
    """Default block (128: four 32-column sub-panels with Ozaki updates between
    them), 64 and 96 (ragged last blocks)."""
    n = 200 if L < 4 else 150
    A = inputs.gaussian_matrix(n, L, seed=1)
    LU, ipiv, info = api.lu_factor(dev(A), method="ozaki", nb=nb)
    assert int(host(info)[0]) == 0
    LUo, ipo, _, gap = orc.zgetrf(A)
    ipg = host(ipiv)
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L)
    diff = planes_diff(orc, host(LU), LUo).max()
    assert diff <= 2.0 ** 10 * n * 2.0 ** -U_EXP[L] * np.abs(A[:, 0]).max() * max(1.0, np.abs(LUo[:, 0]).max())


@pytest.mark.parametrize("L", [2, 3])
def test_lu_ozaki_parity_wide_block(api, orc, L):
    """Blocks of 256 columns (eight 32-column sub-panels), the last one
    ragged (n = 300)."""
    n = 300
    A = inputs.gaussian_matrix(n, L, seed=5)
    LU, ipiv, info = api.lu_factor(dev(A), method="ozaki", nb=256)
    assert int(host(info)[0]) == 0
    LUo, ipo, _, gap = orc.zgetrf(A)
    ipg = host(ipiv)
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L)


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("zc", [0, 7, 31, 32, 63, 71])
def test_lu_ozaki_zero_column(api, orc, L, zc):
    """A zero column stays zero through the elimination: its step has no
    pivot (info = zc + 1, no swap, no multipliers) and the factorisation goes
    on.  Columns at the start, inside and at the end of a 32-column
    sub-panel, and the last column (one block of 72: DD runs k_panel_coop,
    TD k_panel_team)."""
    n = 72
    A = inputs.gaussian_matrix(n, L, seed=4)
    A[:, :, zc, :] = 0.0
    LU, ipiv, info = api.lu_factor(dev(A), method="ozaki")
    LUo, ipo, info_o, gap = orc.zgetrf(A)
    assert int(host(info)[0]) == info_o == zc + 1
    ipg = host(ipiv)
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    diff = planes_diff(orc, host(LU), LUo).max()
    assert diff <= 2.0 ** 10 * n * 2.0 ** -U_EXP[L] * np.abs(A[:, 0]).max() * max(1.0, np.abs(LUo[:, 0]).max())


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("nb", [16, 64])
def test_lu_ozaki_known_factor_bit_exact(api, L, nb):
    A, ipiv_ref, packed, xr, xi = known_factor_case(40, L, seed=110)
    LU, ipiv, info = api.lu_factor(dev(A), method="ozaki", nb=nb)
    assert np.array_equal(host(ipiv), ipiv_ref)
    assert np.array_equal(host(LU), packed)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("frac", [0.2, 0.5, 0.6, 1.0])
def test_zgemm_ozaki_fewer_slices(api, orc, L, frac):
    """Se < S slices per operand (the accuracy knob of Sec. 2.3: the number
    of divisions): against the exact product within the Ozaki bound with Se
    in place of S, 2^(Ea_i + Eb_j - beta Se) 2k (L + Se + 2) + 2^(2 - 53L)|result|;
    Se = S - 1 and about S / 5, S / 2 and 3 S / 5."""
    beta, S = ozaki.CFG[L]
    Se = S - 1 if frac == 1.0 else max(1, int(round(S * frac)))
    m, n, k = 150, 45, 70
    A = inputs.spread_matrix(m, k, L, seed=51, spread=12)
    B = inputs.spread_matrix(k, n, L, seed=52, spread=12)
    C0 = inputs.gaussian_matrix(n, L, seed=53, rows=m)
    out = host(api.zgemm(dev(A), dev(B), dev(C0), method="ozaki", ozaki_slices=Se))
    rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    ex = orc.exact_entries(A, B, rows, cols, C=C0, sign=-1)
    Ea, _ = ozaki.split_rows(A, m, k, L)
    Eb, _ = ozaki.split_cols(B, k, n, L)
    g = np.stack([out[0, :, cols, rows], out[1, :, cols, rows]], axis=1)
    V = np.concatenate([g, -ex], axis=2).reshape(-1, L + 4)
    d = np.abs(orc.exact_sum_rows(V, 1)[:, 0].reshape(-1, 2))
    scale = np.ldexp(1.0, (Ea[rows] + Eb[cols] - beta * Se).astype(int)) * 2 * k * (L + Se + 2)
    tol = scale[:, None] + 2.0 ** (2 - 53 * L) * np.abs(ex[:, :, 0])
    assert np.all(d <= tol), float(np.max(d / tol))
    if frac <= 0.6:   # far fewer bits than the precision: the error must show (the knob acts)
        full = host(api.zgemm(dev(A), dev(B), dev(C0), method="ozaki"))
        assert not np.array_equal(full, out)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_lu_ozaki_one_slice_fewer(api, orc, L):
    """The LU with Se = S - 1 (every Ozaki product of the factorisation):
    the oracle's pivots, backward error within 16 n u 2^(beta (S - Se))."""
    beta, S = ozaki.CFG[L]
    n = 200 if L < 4 else 150
    A = inputs.gaussian_matrix(n, L, seed=1)
    LU, ipiv, info = api.lu_factor(dev(A), method="ozaki", ozaki_slices=S - 1)
    assert int(host(info)[0]) == 0
    LUo, ipo, _, gap = orc.zgetrf(A)
    ipg = host(ipiv)
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L) * 2.0 ** beta


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("sub_nb", [8, 16, 24])
def test_lu_ozaki_sub_panel_width(api, orc, L, sub_nb):
    """Blocks of 128 columns factored as sub-panels of 8, 16 or 24 columns
    (24: the last sub-panel of every block ragged), Ozaki updates between
    them: the oracle's pivots, factors within the parity tolerance, backward
    error <= 16 n u."""
    n = 200
    A = inputs.gaussian_matrix(n, L, seed=1)
    LU, ipiv, info = api.lu_factor(dev(A), method="ozaki", sub_nb=sub_nb)
    assert int(host(info)[0]) == 0
    LUo, ipo, _, gap = orc.zgetrf(A)
    ipg = host(ipiv)
    mism = np.nonzero(ipg != ipo)[0]
    assert mism.size == 0, ("pivots differ", mism[:4], ipg[mism[:4]], ipo[mism[:4]], gap[mism[:4]])
    diff = planes_diff(orc, host(LU), LUo).max()
    assert diff <= 2.0 ** 10 * n * 2.0 ** -U_EXP[L] * np.abs(A[:, 0]).max() * max(1.0, np.abs(LUo[:, 0]).max())
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = host(api.lu_solve(LU, ipiv, dev(b)))
    assert backward_error(orc, A, x, b) <= bound(n, L)
