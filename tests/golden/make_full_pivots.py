"""Write the full-size pivot fixtures of this directory (run from the
repository root: ``python tests/golden/make_full_pivots.py dd td qd``).

Each fixture holds what the CPU oracle (``oracle/``, unblocked GEPP, Sec. 3
"Normal LU") computes for the benchmark's matrix: the complex Gaussian-limb
matrix of ``inputs.gaussian_matrix(n, L, seed=1)`` and the right-hand side
``inputs.complex_gaussian_vector(n, L, seed=2)``.  Nothing comes from the
CUDA library.  Stored per precision:

* ``ipiv``: the oracle's 1-based pivot sequence (partial pivoting on cabs1,
  ties to the lowest row);
* ``mingap``: the smallest relative gap between the two largest pivot keys
  over all steps, and the step where it occurs (a near-tie would make the
  pivot sequence depend on rounding; a gap far above 2^-(53 L - 16) means it
  does not);
* ``lu_rows``, ``lu_cols``, ``lu``: 64 sampled entries of the packed factors
  L\\U, all limbs ([sample][re/im][limb]);
* ``x_rows``, ``x``: 64 sampled entries of the solution of A x = b (Sec. 4).

Sizes: n = 4096 for DD and TD (the benchmark's order); n = 2048 for QD,
whose unblocked oracle at n = 4096 needs several hours on a CPU.  The oracle
at these sizes runs for minutes to hours; each precision is written to its
own file as soon as it is done.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from make_golden import write  # noqa: E402
from paper_2403_16013_gb300 import inputs  # noqa: E402

CASES = {"dd": (2, 4096), "td": (3, 4096), "qd": (4, 2048)}
NSAMP = 64


def path_of(prec: str) -> str:
    L, n = CASES[prec]
    return os.path.join(HERE, f"full_{prec}_n{n}.txt")


def samples(n: int):
    """Sampled (row, col) positions of the factors and rows of the solution
    (seeded; the first and last rows and columns always included)."""
    rng = np.random.default_rng(2024)
    r = np.concatenate([[0, n - 1, n - 1, 0], rng.integers(0, n, NSAMP - 4)]).astype(np.int64)
    c = np.concatenate([[0, n - 1, 0, n - 1], rng.integers(0, n, NSAMP - 4)]).astype(np.int64)
    xr = np.concatenate([[0, n - 1], rng.integers(0, n, NSAMP - 2)]).astype(np.int64)
    return r, c, xr


def case(prec: str) -> dict:
    L, n = CASES[prec]
    A = inputs.gaussian_matrix(n, L, seed=1)
    b = inputs.complex_gaussian_vector(n, L, seed=2)
    LU, ipiv, info, gap = oracle.zgetrf(A)
    x = oracle.zgetrs(LU, ipiv, b)
    r, c, xr = samples(n)
    k = int(np.argmin(gap[:-1])) if n > 1 else 0
    return {"n": np.array([n]), "info": np.array([info]), "ipiv": ipiv,
            "mingap": np.array([gap[k]]), "mingap_step": np.array([k]),
            "lu_rows": r, "lu_cols": c, "lu": np.ascontiguousarray(LU[:, :, c, r].transpose(2, 0, 1)),
            "x_rows": xr, "x": np.ascontiguousarray(x[:, :, 0, xr].transpose(2, 0, 1))}


def main(precs):
    for prec in precs:
        t0 = time.time()
        data = case(prec)
        L, n = CASES[prec]
        write(path_of(prec),
              f"# complex {prec.upper()} GEPP (Sec. 3) of inputs.gaussian_matrix(n={n}, L={L}, seed=1) and solve "
              f"(Sec. 4) of b = inputs.complex_gaussian_vector(seed=2): pivots and sampled factors / solution, "
              f"written by make_full_pivots.py from the oracle\n", data)
        print(f"{prec}: n={n} written in {time.time() - t0:.0f} s, min gap {data['mingap'][0]:.3e}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
