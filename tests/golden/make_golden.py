"""Write the golden fixtures of this directory (run from the repository root:
``python tests/golden/make_golden.py``).

Every stored value is computed by the CPU oracle (``oracle/``) on inputs from
the seeded generators (``paper_2403_16013_gb300/inputs.py``); nothing comes
from the CUDA library.  The paper prints no worked numerical example, so these
fixtures pin the oracle against later changes of its own arithmetic and give
the GPU tests fixed expected values:

* ``lu_dd_n6.txt``: a 6 x 6 complex DD matrix (Gaussian leading limbs, seed
  11), its unblocked GEPP factors (Sec. 3, "Normal LU") and pivots, and the
  solution of A x = b for b = A (1 + i, ..., 1 + i) formed exactly (Sec. 4).
* ``cops_qd.txt``: complex QD product (Eq. 1), 3M product (Eq. 2), quotient
  and reciprocal of eight seeded operand pairs, each the exact result rounded
  to four limbs.

Values are written as hexadecimal binary64 (``float.hex``), one plane array
per block, so that they round-trip exactly.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2403_16013_gb300 import inputs  # noqa: E402


def dump(f, name: str, a: np.ndarray):
    a = np.asarray(a)
    f.write(f"{name} {a.dtype.kind} {' '.join(str(d) for d in a.shape)}\n")
    flat = a.ravel()
    if a.dtype.kind == "f":
        f.write(" ".join(float(v).hex() for v in flat) + "\n")
    else:
        f.write(" ".join(str(int(v)) for v in flat) + "\n")


def load(path: str) -> dict:
    out = {}
    with open(path) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    for head, body in zip(lines[0::2], lines[1::2]):
        name, kind, *shape = head.split()
        shape = tuple(int(s) for s in shape)
        if kind == "f":
            vals = [float.fromhex(t) for t in body.split()]
            out[name] = np.array(vals, np.float64).reshape(shape)
        else:
            out[name] = np.array([int(t) for t in body.split()], np.int64).reshape(shape)
    return out


def lu_case():
    n, L = 6, 2
    A = inputs.gaussian_matrix(n, L, seed=11)
    LU, ipiv, info, _ = oracle.zgetrf(A)
    xr, xi = inputs.ones_x_true(n)
    b = inputs.truncate_limbs(inputs.exact_rhs(A, xr, xi, L_out=4), L)
    x = oracle.zgetrs(LU, ipiv, b)
    return {"A": A, "LU": LU, "ipiv": ipiv, "info": np.array([info]), "b": b, "x": x}


def cops_case():
    L, N = 4, 8
    rng = np.random.default_rng(12)
    def rnd():
        lead = np.ldexp(rng.uniform(-1, 1, N), rng.integers(-6, 7, N))
        return np.stack([lead] + inputs._lower_limbs(lead, L, rng))
    x = np.stack([rnd(), rnd()])
    y = np.stack([rnd(), rnd()])
    return {"x": x, "y": y,
            "mul4m": oracle.cplx_op(oracle.COP_MUL4M, x, y),
            "mul3m": oracle.cplx_op(oracle.COP_MUL3M, x, y),
            "div": oracle.cplx_op(oracle.COP_DIV, x, y),
            "inv": oracle.cplx_op(oracle.COP_INV, y)}


def write(path: str, header: str, data: dict):
    with open(path, "w") as f:
        f.write(header)
        for k, v in data.items():
            dump(f, k, v)


def main():
    write(os.path.join(HERE, "lu_dd_n6.txt"),
          "# complex DD LU with partial pivoting (Sec. 3) and solve (Sec. 4), written by make_golden.py from the oracle\n",
          lu_case())
    write(os.path.join(HERE, "cops_qd.txt"),
          "# complex QD operations, Eq. (1), Eq. (2), division and reciprocal, written by make_golden.py from the oracle\n",
          cops_case())


if __name__ == "__main__":
    main()
