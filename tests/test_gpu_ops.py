"""GPU parity of the elementwise multi-component operations (mc.cuh) against
the oracle's exact-then-rounded operations: |gpu - oracle| within the bound of
each operation, and renormalised (nonoverlapping) limbs."""
import numpy as np
import pytest

from gpu_util import dev, exact_diff, host
from helpers import is_nonoverlapping, rand_limbs

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


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_real_ops(api, orc, L, op):
    rng = np.random.default_rng(500 + L)
    N = 20000
    a = rand_limbs(L, N, rng)
    b = rand_limbs(L, N, rng)
    k = N // 10
    b[:, :k] = -a[:, :k]                                   # exact cancellation
    # cancellation of all but the last limb, b kept canonical
    b[:L - 1, k:2 * k] = -a[:L - 1, k:2 * k]
    _, e = np.frexp(b[L - 2, k:2 * k])
    b[L - 1, k:2 * k] = np.where(b[L - 2, k:2 * k] != 0, np.ldexp(rng.uniform(-1, 1, k), e - 54), 0.0)
    if op == "div":
        b[0, b[0] == 0] = 1.0
    g = host(api.vec_op(op, dev(a), dev(b)))
    code = {"add": orc.OP_ADD, "sub": orc.OP_SUB, "mul": orc.OP_MUL, "div": orc.OP_DIV}[op]
    o = orc.real_op(code, a, b)
    # compare values: the oracle is within 2^(2-53L) of exact; the GPU ops
    # within c 2^(-53L) of exact relative to |a|+|b| (add) or |result| (mul, div)
    scale = (np.abs(a[0]) + np.abs(b[0])) if op in ("add", "sub") else np.abs(o[0])
    c = {"add": 16, "sub": 16, "mul": 16, "div": 64}[op]
    err = np.abs(exact_diff(orc, g, o))
    ratio = err / (2.0 ** (-53 * L) * scale + 1e-300)
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= c, (op, L, worst, ratio[worst], a[:, worst], b[:, worst], g[:, worst], o[:, worst])
    for j in range(0, N, 97):
        assert is_nonoverlapping(list(g[:, j]), strict=False)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("op", ["cmul", "cmul3m", "cdiv", "cinv", "cinv_newton", "cabs1", "cadd"])
def test_complex_ops(api, orc, L, op):
    rng = np.random.default_rng(600 + L)
    N = 8000
    x = np.stack([rand_limbs(L, N, rng, -8, 8), rand_limbs(L, N, rng, -8, 8)])
    y = np.stack([rand_limbs(L, N, rng, -8, 8), rand_limbs(L, N, rng, -8, 8)])
    one_arg = op in ("cinv", "cinv_newton", "cabs1")
    g = host(api.vec_op(op, dev(x), None if one_arg else dev(y)))
    code = {"cmul": orc.COP_MUL4M, "cmul3m": orc.COP_MUL3M, "cdiv": orc.COP_DIV, "cinv": orc.COP_INV,
            "cinv_newton": orc.COP_INV, "cabs1": orc.COP_ABS1, "cadd": orc.COP_ADD}[op]
    o = orc.cplx_op(code, x) if one_arg else orc.cplx_op(code, x, y)
    ax = np.abs(x[:, 0]).sum(axis=0)
    ay = np.abs(y[:, 0]).sum(axis=0)
    scale = {"cmul": ax * ay, "cmul3m": ax * ay, "cdiv": ax / np.hypot(y[0, 0], y[1, 0]),
             "cinv": 1 / np.hypot(x[0, 0], x[1, 0]), "cinv_newton": 1 / np.hypot(x[0, 0], x[1, 0]),
             "cabs1": ax, "cadd": ax + ay}[op]
    err = np.maximum(np.abs(exact_diff(orc, g[0], o[0])), np.abs(exact_diff(orc, g[1], o[1])))
    ratio = err / (2.0 ** (-53 * L) * scale)
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 256, (op, L, worst, ratio[worst])


@pytest.mark.parametrize("L", [2, 3, 4])
def test_inv_newton_edges(api, orc, L):
    """The pivot reciprocal by Newton's method from a binary64 seed (op 17) on
    the cases its exact cancellations rest on: purely real and purely
    imaginary values (one leading product zero), |Re| and |Im| far apart in
    either order, equal or nearly equal (both leading products near 1/2, where
    1 minus either is inexact), and exponents over 2^+-400 -- within the same
    256 u_L of 1/|x| as the multi-component reciprocal, against the oracle."""
    rng = np.random.default_rng(700 + L)
    N = 4000
    x = np.stack([rand_limbs(L, N, rng, -8, 8), rand_limbs(L, N, rng, -8, 8)])
    q = N // 8
    x[1, :, :q] = 0.0                                   # real
    x[0, :, q:2 * q] = 0.0                              # imaginary
    x[1, :, 2 * q:3 * q] *= 2.0 ** -40                  # |Re| >> |Im|
    x[0, :, 3 * q:4 * q] *= 2.0 ** -40                  # |Im| >> |Re|
    x[1, :, 4 * q:5 * q] = x[0, :, 4 * q:5 * q]         # Re = Im
    x[:, :, 5 * q:6 * q] *= 2.0 ** 400
    x[:, :, 6 * q:7 * q] *= 2.0 ** -400
    x[1, 0, 7 * q:] = x[0, 0, 7 * q:] * (1 + 2.0 ** -40)  # Re and Im a few units apart
    x[1, 1:, 7 * q:] = x[0, 1:, 7 * q:]
    g = host(api.vec_op("cinv_newton", dev(x)))
    o = orc.cplx_op(orc.COP_INV, x)
    err = np.maximum(np.abs(exact_diff(orc, g[0], o[0])), np.abs(exact_diff(orc, g[1], o[1])))
    ratio = err / (2.0 ** (-53 * L) / np.hypot(x[0, 0], x[1, 0]))
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 256, (L, worst, ratio[worst], x[:, :, worst])
    for j in range(0, N, 61):
        for c in range(2):
            assert is_nonoverlapping(list(g[c, :, j]), strict=False)
