"""Seeded synthetic inputs for complex multi-component (DD/TD/QD) LU.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds only random draws, placement of lower limbs by
exponent, and exact integer summation (for right-hand sides b = A x_true);
none of the multi-component floating-point arithmetic of the method lives here.

Storage convention (the library's plane layout).  A complex L-limb matrix with
``rows`` rows and ``cols`` columns is a float64 array of shape
``[2, L, cols, ld]`` (``ld >= rows``): component ``c`` (0 = real, 1 = imaginary),
limb ``l``, column ``j``, row ``i``.  Each ``[c, l]`` plane is column-major, so
element (i, j) of plane (c, l) sits at flat offset ``((c*L + l)*cols + j)*ld + i``.

Limbs are canonical: limb k+1 is smaller than half an ulp of limb k, so the
value of an element is the exact sum of its limbs and limb 0 is that sum
rounded to binary64 (up to ties of probability ~2^-52).

Workloads (the paper's experiments, Sec. 2.4 and Sec. 4, use synthetic data:
uniform [0,1] entries, x_k = k + k i, b formed in high precision):

* ``uniform_matrix``      - Re/Im leading limbs U[-1,1), lower limbs uniform
                            in their canonical range (the n=128 DD case).
* ``gaussian_matrix``     - leading limbs N(0,1), lower limbs canonical uniform
                            (the n=1024 / n=4096 DD, TD, QD cases).
* ``spread_matrix``       - N(0,1) * 2^e with e uniform in [-20, 20] per entry
                            (the Ozaki-scheme workload with exponent spread).
* ``paper_matrix``        - leading limbs U[0,1) as in Sec. 4, with
                            x_k = k + k i (``paper_x_true``).
* ``householder_vectors`` - seeded complex Gaussian reflector vectors for the
                            ill-conditioned case; the matrix itself is formed
                            by the caller.
"""
from __future__ import annotations

import numpy as np

LIMBS = {"dd": 2, "td": 3, "qd": 4}


def plane_shape(L: int, rows: int, cols: int, ld: int | None = None):
    return (2, L, cols, rows if ld is None else ld)


def _lower_limbs(lead: np.ndarray, L: int, rng: np.random.Generator) -> list[np.ndarray]:
    """Limbs 1..L-1 drawn uniformly in (-1/2 ulp, 1/2 ulp) of the limb above.

    frexp gives limb = m * 2^E with 0.5 <= |m| < 1, so ulp(limb) = 2^(E-53) and
    a value t * 2^(E-54) with |t| < 1 is below half an ulp: the limbs are
    canonical by construction, with no rounding step.
    """
    out = []
    prev = lead
    for _ in range(1, L):
        t = rng.uniform(-1.0, 1.0, size=lead.shape)
        _, e = np.frexp(prev)
        nxt = np.where(prev != 0.0, np.ldexp(t, e - 54), 0.0)
        out.append(nxt)
        prev = nxt
    return out


def _assemble(lead_re: np.ndarray, lead_im: np.ndarray, L: int, rng, ld: int | None) -> np.ndarray:
    rows, cols = lead_re.shape
    ld = rows if ld is None else ld
    A = np.zeros((2, L, cols, ld), dtype=np.float64)
    for c, lead in enumerate((lead_re, lead_im)):
        limbs = [lead] + _lower_limbs(lead, L, rng)
        for l in range(L):
            A[c, l, :, :rows] = limbs[l].T
    return A


def uniform_matrix(n: int, L: int, seed: int, ld: int | None = None, lo: float = -1.0, hi: float = 1.0):
    """Leading limbs U[lo, hi), lower limbs canonical uniform."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(lo, hi, size=(n, n))
    im = rng.uniform(lo, hi, size=(n, n))
    return _assemble(re, im, L, rng, ld)


def gaussian_matrix(n: int, L: int, seed: int, ld: int | None = None, rows: int | None = None):
    """Leading limbs N(0,1), lower limbs canonical uniform.  ``rows`` x ``n``."""
    rng = np.random.default_rng(seed)
    m = n if rows is None else rows
    re = rng.standard_normal(size=(m, n))
    im = rng.standard_normal(size=(m, n))
    return _assemble(re, im, L, rng, ld)


def spread_matrix(rows: int, cols: int, L: int, seed: int, spread: int = 20, ld: int | None = None):
    """Entries N(0,1) * 2^e, e uniform integer in [-spread, spread] per entry."""
    rng = np.random.default_rng(seed)
    e_re = rng.integers(-spread, spread + 1, size=(rows, cols))
    e_im = rng.integers(-spread, spread + 1, size=(rows, cols))
    re = np.ldexp(rng.standard_normal(size=(rows, cols)), e_re)
    im = np.ldexp(rng.standard_normal(size=(rows, cols)), e_im)
    return _assemble(re, im, L, rng, ld)


def paper_matrix(n: int, L: int, seed: int, ld: int | None = None):
    """Sec. 4: entries of A uniform in [0, 1] (leading limbs), lower limbs canonical."""
    return uniform_matrix(n, L, seed, ld, lo=0.0, hi=1.0)


def ones_x_true(n: int):
    """x_true = (1 + 1i) for every entry, as integer Re/Im parts."""
    return np.ones(n, dtype=np.int64), np.ones(n, dtype=np.int64)


def paper_x_true(n: int):
    """Sec. 4: (x)_k = k + k i, k = 1..n, as integer Re/Im parts."""
    k = np.arange(1, n + 1, dtype=np.int64)
    return k.copy(), k.copy()


def int_vector_planes(xr: np.ndarray, xi: np.ndarray, L: int) -> np.ndarray:
    """An integer complex vector as L-limb planes [2, L, 1, n] (exact in limb 0)."""
    n = xr.shape[0]
    X = np.zeros((2, L, 1, n), dtype=np.float64)
    X[0, 0, 0, :] = xr.astype(np.float64)
    X[1, 0, 0, :] = xi.astype(np.float64)
    return X


def complex_gaussian_vector(n: int, L: int, seed: int) -> np.ndarray:
    """Seeded complex Gaussian vector as planes [2, L, 1, n] (canonical lower limbs)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(size=(n, 1))
    im = rng.standard_normal(size=(n, 1))
    return _assemble(re, im, L, rng, None)


def householder_vectors(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` seeded complex Gaussian vectors, shape [count, 2, n] (binary64)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(count, 2, n))


def geometric_ratio(n: int, decades: float = 40.0) -> float:
    """Binary64 ratio r = 10^(-decades/(n-1)); sigma_i = r^i spans 1 .. 10^-decades."""
    return float(10.0 ** (-decades / (n - 1)))


# ----------------------------------------------------------------------------
# Exact right-hand side b = A x for integer x, by integer binning.
# ----------------------------------------------------------------------------

_CHUNK = 14          # mantissa chunk width: 4 chunks cover the 53-bit significand
_POS_MIN = -1074 - 53 - 8
_NPOS = 2400         # covers binary64 exponents with chunk offsets and carries


def _accumulate(bins: np.ndarray, v: np.ndarray, k: np.ndarray):
    """bins[row, pos] += exact chunks of v[row, col] * k[col] (float64, exact).

    v = mi * 2^p with |mi| < 2^53 an integer; mi is cut into 14-bit chunks, each
    times |k| < 2^20 stays below 2^34, and sums of up to 2^18 of them stay below
    2^53, so float64 bincount accumulation is exact.
    """
    rows = v.shape[0]
    m, e = np.frexp(v)
    mi = np.ldexp(m, 53).astype(np.int64)
    sign = np.sign(mi) * np.sign(k)[None, :]
    mag = np.abs(mi)
    kk = np.abs(k).astype(np.int64)[None, :]
    p = (e - 53).astype(np.int64) - _POS_MIN
    row_idx = np.broadcast_to(np.arange(rows, dtype=np.int64)[:, None], v.shape)
    for q in range(4):
        ch = (mag >> (_CHUNK * q)) & ((1 << _CHUNK) - 1)
        w = (sign * ch * kk).astype(np.float64)
        nz = w != 0
        if not nz.any():
            continue
        idx = row_idx[nz] * _NPOS + (p[nz] + _CHUNK * q)
        bins += np.bincount(idx, weights=w[nz], minlength=bins.size).reshape(bins.shape)


def _bins_to_ints(bins: np.ndarray) -> list[int]:
    """Each row of integer-valued bins (weight 2^pos) to one Python int (scale 2^_POS_MIN)."""
    B = bins.astype(np.int64)
    rows, npos = B.shape
    for pos in range(npos - 1):
        c = B[:, pos] >> 1
        B[:, pos] -= c << 1
        B[:, pos + 1] += c
    top = B[:, npos - 1].copy()
    B[:, npos - 1] = 0
    out = []
    for r in range(rows):
        bits = np.packbits(B[r].astype(np.uint8), bitorder="little")
        N = int.from_bytes(bits.tobytes(), "little") + (int(top[r]) << (npos - 1))
        out.append(N)
    return out


def _round_limbs(N: int, L: int) -> list[float]:
    """Greedy rounding of N * 2^_POS_MIN to L binary64 limbs: l_k = RN(v - sum_{i<k} l_i)."""
    den = 1 << (-_POS_MIN)
    out = []
    for _ in range(L):
        if N == 0:
            out.append(0.0)
            continue
        v = N / den                      # int/int true division is correctly rounded
        num, d = v.as_integer_ratio()
        t = (num << (-_POS_MIN))
        assert t % d == 0
        N -= t // d
        out.append(v)
    return out


def exact_rhs(A: np.ndarray, xr: np.ndarray, xi: np.ndarray, L_out: int, rows: int | None = None,
              col_block: int = 256) -> np.ndarray:
    """b = A x exactly for integer x = xr + i xi, rounded greedily to ``L_out`` limbs.

    A: planes [2, L, cols, ld]; returns planes [2, L_out, 1, rows].
    """
    _, L, cols, ld = A.shape
    rows = ld if rows is None else rows
    assert np.all(np.abs(xr) < (1 << 20)) and np.all(np.abs(xi) < (1 << 20))
    b = np.zeros((2, L_out, 1, rows), dtype=np.float64)
    # Re b = sum_j Re(a) xr - Im(a) xi ;  Im b = sum_j Re(a) xi + Im(a) xr
    plan = {0: ((0, xr), (1, -xi)), 1: ((0, xi), (1, xr))}
    for comp, terms in plan.items():
        bins = np.zeros((rows, _NPOS), dtype=np.float64)
        for c, k in terms:
            for l in range(L):
                for j0 in range(0, cols, col_block):
                    j1 = min(cols, j0 + col_block)
                    v = A[c, l, j0:j1, :rows].T          # rows x block
                    _accumulate(bins, np.ascontiguousarray(v), k[j0:j1])
        for r, N in enumerate(_bins_to_ints(bins)):
            b[comp, :, 0, r] = _round_limbs(N, L_out)
    return b


def truncate_limbs(X: np.ndarray, L: int) -> np.ndarray:
    """First L limbs of a planes array (used to feed DD/TD runs from QD data)."""
    return np.ascontiguousarray(X[:, :L])
