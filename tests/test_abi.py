"""The C-ABI library loads and exports every function include/mclu.h declares;
argument validation answers without touching a GPU (no compute here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mclu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|int64_t|uint64_t|const char \*)\s*\*?\s*(\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_16013_gb300 import binding, build
    build.build()
    return binding.load()


def test_all_declared_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name


def test_argument_validation_without_gpu(lib):
    from paper_2403_16013_gb300 import binding as B
    assert B.zgetrf("dd", -1, 0, 1, 0) == -1
    assert B.zgetrf("td", 4, 0, 4, 0) == -2
    assert B.zgetrf("qd", 4, 8, 3, 8) == -3
    assert B.zgetrf_ex("dd", 4, 8, 4, 8, 0, nb=999) == -6
    assert B.zgetrf_ex("dd", 4, 8, 4, 8, 0, method=7) == -6
    assert B.zgetrs("dd", "X", 4, 1, 8, 4, 8, 8, 4) == -1
    assert B.zgetrs("qd", "N", 4, -1, 8, 4, 8, 8, 4) == -3
    assert B.zgetrs("td", "C", 4, 1, 8, 4, 8, 8, 2) == -8
    assert B.zgemm("dd", 2, 0, 1, 1, 1, 8, 1, 8, 1, 8, 1) == -1
    assert B.zgemm("dd", 0, 9, 1, 1, 1, 8, 1, 8, 1, 8, 1) == -2
    assert B.zgemm_ex("dd", 0, B.METHOD_OZAKI, -1, 1, 1, 1, 8, 1, 8, 1, 8, 1) == -3
    assert B.zgemm_ex("dd", 0, B.METHOD_OZAKI, 17, 1, 1, 1, 8, 1, 8, 1, 8, 1) == B.ERR_UNSUPPORTED
    assert B.zgemm_ex("qd", 0, B.METHOD_OZAKI, 33, 1, 1, 1, 8, 1, 8, 1, 8, 1) == B.ERR_UNSUPPORTED
    assert B.zgemm_ex("td", 0, B.METHOD_4M, 0, -1, 1, 1, 8, 1, 8, 1, 8, 1) == -4     # m, one place further
    assert B.zgemm_ex("td", 0, B.METHOD_4M, 0, 4, 1, 1, 8, 1, 8, 1, 8, 1) == -8      # lda < m
    assert B.zgetrf_ex("dd", 4, 8, 4, 8, 0, method=B.METHOD_OZAKI, ozaki_slices=17) == B.ERR_UNSUPPORTED
    assert B.zgetrf_ex("td", 4, 8, 4, 8, 0, method=B.METHOD_OZAKI, ozaki_slices=-2) == -6
    assert B.dgetrf_ex("td", -1, 8, 1, 8, 0) == -1
    assert B.dgetrf_ex("qd", 4, 8, 3, 8, 0) == -3
    assert B.dgetrs("dd", "C", 4, 1, 8, 4, 8, 8, 4) == -1          # real solves take 'N' or 'T'
    assert B.dgetrs("dd", "T", 4, 1, 8, 4, 8, 8, 2) == -8
    assert B.zadjoint_rank1("dd", 4, 8, 8, 8, 2) == -5
    assert B.vec_op(99, 2, 4, 8, 8, 8) == -1
    assert B.vec_op(0, 5, 4, 8, 8, 8) == -2
    assert B.zgetrf("dd", 0, 0, 1, 0) == 0          # n = 0: nothing to do, no CUDA call
    assert "invalid" in B.status_string(-3)
    assert lib.mclu_version().decode().count(".") == 2
