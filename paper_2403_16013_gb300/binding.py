"""ctypes binding of libmclu.so (the C ABI declared in include/mclu.h).

Argument marshalling only: every function here forwards to the CUDA library
with the same name and arguments (device pointers as integers, the stream as
an integer handle).  There is no fallback: if the library was not built, the
first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmclu.so")

METHOD_4M, METHOD_3M, METHOD_UNBLOCKED, METHOD_OZAKI, METHOD_STRASSEN = 0, 1, 2, 3, 4
ERR_UNSUPPORTED = 100000
LIMBS = {"dd": 2, "td": 3, "qd": 4}


class MCLUOpts(C.Structure):
    _fields_ = [("nb", C.c_int32), ("method", C.c_int32), ("ozaki_slices", C.c_int32), ("sub_nb", C.c_int32)]


_lib = None


def _declare(lib):
    i64, i32, ci, vp, cc = C.c_int64, C.c_int32, C.c_int, C.c_void_p, C.c_char
    for s in ("dd", "td", "qd"):
        f = getattr(lib, f"zgetrf_{s}")
        f.argtypes, f.restype = [i64, vp, i64, vp, vp], ci
        f = getattr(lib, f"zgetrf_{s}_ex")
        f.argtypes, f.restype = [i64, vp, i64, vp, vp, C.POINTER(MCLUOpts), vp], ci
        f = getattr(lib, f"zgetrs_{s}")
        f.argtypes, f.restype = [cc, i64, i64, vp, i64, vp, vp, i64, vp], ci
        f = getattr(lib, f"dgetrf_{s}")
        f.argtypes, f.restype = [i64, vp, i64, vp, vp], ci
        f = getattr(lib, f"dgetrf_{s}_ex")
        f.argtypes, f.restype = [i64, vp, i64, vp, vp, C.POINTER(MCLUOpts), vp], ci
        f = getattr(lib, f"dgetrs_{s}")
        f.argtypes, f.restype = [cc, i64, i64, vp, i64, vp, vp, i64, vp], ci
        f = getattr(lib, f"zgemm_{s}")
        f.argtypes, f.restype = [ci, ci, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp], ci
        f = getattr(lib, f"zgemm_{s}_ex")
        f.argtypes, f.restype = [ci, ci, ci, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp], ci
        f = getattr(lib, f"zadjoint_rank1_{s}")
        f.argtypes, f.restype = [i64, vp, vp, vp, i64, vp], ci
        f = getattr(lib, f"zozaki_split_{s}")
        f.argtypes, f.restype = [ci, i64, i64, vp, i64, vp, vp, vp], ci
    lib.mclu_vec_op.argtypes, lib.mclu_vec_op.restype = [ci, ci, i64, vp, vp, vp, vp], ci
    lib.zgetrf_dd_noalloc.argtypes, lib.zgetrf_dd_noalloc.restype = [i64, vp, i64, vp, vp, vp], ci
    lib.zgetrf_dd_noalloc_max_n.argtypes, lib.zgetrf_dd_noalloc_max_n.restype = [], i64
    lib.mclu_status_string.argtypes, lib.mclu_status_string.restype = [ci], C.c_char_p
    lib.mclu_version.argtypes, lib.mclu_version.restype = [], C.c_char_p
    lib.mclu_selftest_wait_timeout.argtypes, lib.mclu_selftest_wait_timeout.restype = [C.POINTER(C.c_int32)], ci
    lib.mclu_probe_fp64_rate.argtypes, lib.mclu_probe_fp64_rate.restype = [C.POINTER(C.c_double)], ci
    lib.mclu_launch_count.argtypes, lib.mclu_launch_count.restype = [], C.c_uint64
    lib.mclu_profile_begin.argtypes, lib.mclu_profile_begin.restype = [C.c_uint32], ci
    lib.mclu_profile_end.argtypes, lib.mclu_profile_end.restype = [C.POINTER(C.c_double),
                                                                    C.POINTER(C.c_int64), ci], ci


def load(path: str | None = None):
    """Load libmclu.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libmclu.so not found at {p}: build it with paper_2403_16013_gb300/build.py "
                               "(the CUDA library is required; there is no CPU fallback)")
        lib = C.CDLL(p)
        _declare(lib)
        _lib = lib
    return _lib


def launch_count() -> int:
    return int(load().mclu_launch_count())


PROFILE_KINDS = ("panel", "laswp", "trsm", "gemm", "getrs", "other")


def profile_begin(kinds=PROFILE_KINDS) -> None:
    mask = 0
    for k in kinds:
        mask |= 1 << PROFILE_KINDS.index(k)
    check(load().mclu_profile_begin(mask), "mclu_profile_begin")


def profile_end() -> dict:
    n = len(PROFILE_KINDS)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    check(load().mclu_profile_end(ms, cnt, n), "mclu_profile_end")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(PROFILE_KINDS)}


def selftest_wait_timeout() -> int:
    """mclu_selftest_wait_timeout: the status word left by the panels'
    bounded inter-CTA wait on a flag that nothing sets (1 = ran out)."""
    st = C.c_int32(-1)
    check(load().mclu_selftest_wait_timeout(C.byref(st)), "mclu_selftest_wait_timeout")
    return int(st.value)


def probe_fp64_rate() -> float:
    """mclu_probe_fp64_rate: measured FP64 instructions per second of the current device."""
    v = C.c_double(0.0)
    check(load().mclu_probe_fp64_rate(C.byref(v)), "mclu_probe_fp64_rate")
    return float(v.value)


def status_string(rc: int) -> str:
    return load().mclu_status_string(rc).decode()


def check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed: status {rc} ({status_string(rc)})")


def _stream(stream) -> int | None:
    return None if stream in (None, 0) else int(stream)


# Thin mirrors of the C entry points (pointers are integers).

def zgetrf(prec: str, n, A, lda, ipiv, stream=None) -> int:
    return getattr(load(), f"zgetrf_{prec}")(n, A, lda, ipiv, _stream(stream))


def zgetrf_ex(prec: str, n, A, lda, ipiv, info, nb=0, method=METHOD_4M, ozaki_slices=0, stream=None,
              sub_nb=0) -> int:
    o = MCLUOpts(nb, method, ozaki_slices, sub_nb)
    return getattr(load(), f"zgetrf_{prec}_ex")(n, A, lda, ipiv, info, C.byref(o), _stream(stream))


def zgetrf_dd_noalloc(n, A, lda, ipiv, info, stream=None) -> int:
    return load().zgetrf_dd_noalloc(n, A, lda, ipiv, info, _stream(stream))


def dgetrf_ex(prec: str, n, A, lda, ipiv, info, nb=0, method=METHOD_4M, ozaki_slices=0, stream=None,
              sub_nb=0) -> int:
    o = MCLUOpts(nb, method, ozaki_slices, sub_nb)
    return getattr(load(), f"dgetrf_{prec}_ex")(n, A, lda, ipiv, info, C.byref(o), _stream(stream))


def dgetrs(prec: str, trans: str, n, nrhs, A, lda, ipiv, B, ldb, stream=None) -> int:
    return getattr(load(), f"dgetrs_{prec}")(trans.encode(), n, nrhs, A, lda, ipiv, B, ldb, _stream(stream))


def zgetrs(prec: str, trans: str, n, nrhs, A, lda, ipiv, B, ldb, stream=None) -> int:
    return getattr(load(), f"zgetrs_{prec}")(trans.encode(), n, nrhs, A, lda, ipiv, B, ldb, _stream(stream))


def zgemm(prec: str, beta_mode, method, m, n, k, A, lda, B, ldb, Cm, ldc, stream=None) -> int:
    return getattr(load(), f"zgemm_{prec}")(beta_mode, method, m, n, k, A, lda, B, ldb, Cm, ldc, _stream(stream))


def zgemm_ex(prec: str, beta_mode, method, ozaki_slices, m, n, k, A, lda, B, ldb, Cm, ldc, stream=None) -> int:
    return getattr(load(), f"zgemm_{prec}_ex")(beta_mode, method, ozaki_slices, m, n, k, A, lda, B, ldb, Cm, ldc,
                                               _stream(stream))


def zadjoint_rank1(prec: str, n, lam, x, Abar, ldab, stream=None) -> int:
    return getattr(load(), f"zadjoint_rank1_{prec}")(n, lam, x, Abar, ldab, _stream(stream))


def zozaki_split(prec: str, side, rows, cols, X, ld, slices, E, stream=None) -> int:
    return getattr(load(), f"zozaki_split_{prec}")(side, rows, cols, X, ld, slices, E, _stream(stream))


def vec_op(op, L, count, x, y, z, stream=None) -> int:
    return load().mclu_vec_op(op, L, count, x, y, z, _stream(stream))
