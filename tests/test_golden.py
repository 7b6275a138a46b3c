"""Golden fixtures (tests/golden): the oracle reproduces them bit for bit,
and the stored solution meets the backward-error bound with the exact
residual.  The fixtures are written by tests/golden/make_golden.py from the
oracle alone."""
import os
import sys

import numpy as np

from gpu_util import backward_error, bound

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden  # noqa: E402

HERE = os.path.join(os.path.dirname(__file__), "golden")


def test_lu_fixture_reproduced(orc):
    g = make_golden.load(os.path.join(HERE, "lu_dd_n6.txt"))
    r = make_golden.lu_case()
    for k in ("A", "LU", "b", "x"):
        assert np.array_equal(g[k], r[k]), k
    assert np.array_equal(g["ipiv"], r["ipiv"]) and int(g["info"][0]) == 0
    assert backward_error(orc, g["A"], g["x"], g["b"]) <= bound(6, 2)


def test_cops_fixture_reproduced(orc):
    g = make_golden.load(os.path.join(HERE, "cops_qd.txt"))
    r = make_golden.cops_case()
    for k in g:
        assert np.array_equal(g[k], r[k]), k
