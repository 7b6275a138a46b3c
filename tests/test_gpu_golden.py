"""The CUDA path against the golden fixtures of tests/golden (oracle values):
pivots equal, factors and solution within the parity bars, complex QD ops
within their operation bounds."""
import os
import sys

import numpy as np
import pytest

from gpu_util import dev, exact_diff, host, planes_diff

pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden  # noqa: E402

HERE = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_16013_gb300 import api as a
    from paper_2403_16013_gb300 import build
    build.build()
    return a


@pytest.mark.parametrize("method", ["unblocked", "4m", "ozaki"])
def test_lu_golden(api, orc, method):
    g = make_golden.load(os.path.join(HERE, "lu_dd_n6.txt"))
    LU, ipiv, info = api.lu_factor(dev(g["A"]), method=method, nb=4 if method != "unblocked" else 0)
    assert int(host(info)[0]) == 0
    assert np.array_equal(host(ipiv), g["ipiv"])
    n, u = 6, 2.0 ** -104
    scale = np.abs(g["A"][:, 0]).max() * max(1.0, np.abs(g["LU"][:, 0]).max())
    d = planes_diff(orc, host(LU), g["LU"]).max()
    assert d <= 2.0 ** 10 * n * u * scale
    x = host(api.lu_solve(LU, ipiv, dev(g["b"])))
    assert planes_diff(orc, x, g["x"]).max() <= 2.0 ** 12 * n * u * np.abs(g["x"][:, 0]).max()


@pytest.mark.parametrize("op,key,c", [("cmul", "mul4m", 256), ("cmul3m", "mul3m", 256), ("cdiv", "div", 256),
                                      ("cinv", "inv", 256)])
def test_cops_golden(api, orc, op, key, c):
    g = make_golden.load(os.path.join(HERE, "cops_qd.txt"))
    x, y = g["x"], g["y"]
    out = host(api.vec_op(op, dev(y)) if op == "cinv" else api.vec_op(op, dev(x), dev(y)))
    o = g[key]
    err = np.maximum(np.abs(exact_diff(orc, out[0], o[0])), np.abs(exact_diff(orc, out[1], o[1])))
    ax, ay = np.abs(x[:, 0]).sum(axis=0), np.abs(y[:, 0]).sum(axis=0)
    scale = {"mul4m": ax * ay, "mul3m": ax * ay, "div": ax / np.hypot(y[0, 0], y[1, 0]),
             "inv": 1 / np.hypot(y[0, 0], y[1, 0])}[key]
    assert (err / (2.0 ** (-53 * 4) * scale)).max() <= c
