"""The allocation-free DD factorisation (zgetrf_dd_noalloc) against the
allocating one (zgetrf_dd_ex, same 4M / nb = 64 defaults), through the C ABI.

zgetrf_dd_noalloc exists for callers that cannot allocate device memory
during the call (graph capture, real-time code, fixed memory budgets); it keeps
its scratch in a fixed device array inside the library.  Two calls in a row on
different matrices check that nothing left in the shared array by one call
leaks into the next.  This file is collected last so that a run stopping at
the first failure has run every other test; it also passes on its own in a
fresh process.
"""
import numpy as np
import pytest

from gpu_util import dev, host
from helpers import U_EXP
from paper_2403_16013_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_allocating_path_twice(lib):
    n = 300                                     # several panels of 64 and a ragged last one
    for seed in (11, 12):                       # two calls in a row on different inputs
        A = inputs.gaussian_matrix(n, 2, seed=seed)
        if seed == 12:
            A[:, :, 5, :] = 0.0                 # a zero column: info must be reported afresh
        LUa, ipa, infa = _factor(lib, A, noalloc=False)
        LUn, ipn, infn = _factor(lib, A, noalloc=True)
        assert np.array_equal(ipn, ipa)
        assert infn == infa == (6 if seed == 12 else 0)
        diff = np.abs((LUn - LUa).sum(axis=1)).max()
        assert diff <= 2.0 ** 10 * n * 2.0 ** -U_EXP[2] * np.abs(LUa[:, 0]).max()


def test_noalloc_rejects_oversize(lib):
    nmax = lib.load().zgetrf_dd_noalloc_max_n()
    assert nmax == 8192
    rc = lib.zgetrf_dd_noalloc(nmax + 1, 0, nmax + 1, 0, 0, None)   # rejected before touching anything
    assert rc == 100001                                              # MCLU_ERR_SCRATCH_CAPACITY
    assert "scratch" in lib.status_string(rc)
