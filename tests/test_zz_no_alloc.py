"""The allocation-free DD factorisation (zgetrf_dd_noalloc) through the C ABI,
against the allocating one (zgetrf_dd_ex, same 4M / nb = 64 defaults) and
against the CPU oracle.

zgetrf_dd_noalloc exists for callers that cannot allocate device memory
during the call (graph capture, real-time code, fixed memory budgets); it keeps
its scratch in a fixed device array inside the library.  Checked here:

* two calls in a row on different matrices (the second with a zero column)
  give output bit-identical to zgetrf_dd_ex (both run the same kernels, so
  nothing left in the shared array by one call may leak into the next), the
  oracle's pivots and info, and factors within the parity tolerance of the
  oracle's;
* the call allocates nothing: the high-water mark of the device's default
  stream-ordered memory pool (the pool cudaMallocAsync draws from) stays at
  zero across it, while the same mark does rise across a call of the
  allocating entry point (so the check can see an allocation);
* sizes above the fixed capacity are rejected before anything is enqueued.

This file is collected last so that a run stopping at the first failure has
run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import dev, host, planes_diff
from helpers import U_EXP
from paper_2403_16013_gb300 import inputs

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the CUDA driver API
_ATTR_USED_MEM_CURRENT, _ATTR_USED_MEM_HIGH = 7, 8


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_16013_gb300 import binding, build
    build.build()
    return binding


def _factor(binding, A, noalloc):
    import torch
    n, lda = A.shape[2], A.shape[3]
    LU = dev(A)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    if noalloc:
        rc = binding.zgetrf_dd_noalloc(n, LU.data_ptr(), lda, ipiv.data_ptr(), info.data_ptr(), s)
    else:
        rc = binding.zgetrf_ex("dd", n, LU.data_ptr(), lda, ipiv.data_ptr(), info.data_ptr(), 64,
                               binding.METHOD_4M, 0, s)
    assert rc == 0, binding.status_string(rc)
    torch.cuda.synchronize()
    return host(LU), host(ipiv), int(host(info)[0])


class _DefaultPool:
    """The current device's default memory pool, read through the CUDA driver
    API (libcuda): the pool that stream-ordered allocations draw from."""

    def __init__(self):
        import torch
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev_ = ctypes.c_int(0)
        assert self.cu.cuDeviceGet(ctypes.byref(dev_), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev_) == 0

    def get(self, attr: int) -> int:
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return int(v.value)

    def reset_high(self):
        v = ctypes.c_uint64(0)     # the high-water mark may only be reset to zero
        assert self.cu.cuMemPoolSetAttribute(self.pool, _ATTR_USED_MEM_HIGH, ctypes.byref(v)) == 0


def test_noalloc_matches_allocating_path_and_oracle_twice(lib, orc):
    n, L = 300, 2                               # several panels of 64 and a ragged last one
    for seed in (11, 12):                       # two calls in a row on different inputs
        A = inputs.gaussian_matrix(n, L, seed=seed)
        if seed == 12:
            A[:, :, 5, :] = 0.0                 # a zero column: info must be reported afresh
        LUa, ipa, infa = _factor(lib, A, noalloc=False)
        LUn, ipn, infn = _factor(lib, A, noalloc=True)
        assert np.array_equal(LUn, LUa)         # same kernels: bit-identical output
        assert np.array_equal(ipn, ipa)
        assert infn == infa == (6 if seed == 12 else 0)
        LUo, ipo, info_o, _ = orc.zgetrf(A)
        assert np.array_equal(ipn, ipo) and infn == info_o
        diff = planes_diff(orc, LUn, LUo).max()
        assert diff <= 2.0 ** 10 * n * 2.0 ** -U_EXP[L] * np.abs(A[:, 0]).max() * max(1.0, np.abs(LUo[:, 0]).max())


def test_noalloc_allocates_nothing(lib):
    import torch
    if torch.cuda.get_allocator_backend() != "native":
        pytest.skip("torch itself allocates from the default pool (cudaMallocAsync backend)")
    pool = _DefaultPool()
    A = inputs.gaussian_matrix(200, 2, seed=13)
    _factor(lib, A, noalloc=True)               # the first call on the device looks up the array's address
    torch.cuda.synchronize()
    pool.reset_high()
    assert pool.get(_ATTR_USED_MEM_HIGH) == pool.get(_ATTR_USED_MEM_CURRENT) == 0
    _factor(lib, A, noalloc=True)
    assert pool.get(_ATTR_USED_MEM_HIGH) == 0
    _factor(lib, A, noalloc=False)              # control: the allocating path draws from the pool
    assert pool.get(_ATTR_USED_MEM_HIGH) > 0
    pool.reset_high()


def test_noalloc_rejects_oversize(lib):
    nmax = lib.load().zgetrf_dd_noalloc_max_n()
    assert nmax == 8192
    rc = lib.zgetrf_dd_noalloc(nmax + 1, 0, nmax + 1, 0, 0, None)   # rejected before touching anything
    assert rc == 100001                                              # MCLU_ERR_SCRATCH_CAPACITY
    assert "scratch" in lib.status_string(rc)
