"""ctypes binding of the multithreaded CPU permutation (cpu_mt.cpp).  Test and
measurement infrastructure only."""
from __future__ import annotations

import ctypes

import numpy as np

from . import build_cpu

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_cpu.build())
        p = ctypes.c_void_p
        lib.sp_cpu_permute.restype = ctypes.c_int
        lib.sp_cpu_permute.argtypes = [ctypes.c_int64, ctypes.c_int64, p, p, p, p, p, p, p, p]
        lib.sp_cpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return _load().sp_cpu_threads()


def permute(nrows, ncols, rowptr, colidx, values, p, q=None):
    """B = P A Q^T on all host threads; int64 rowptr / p / q, int32 columns, 4-byte values.
    Returns (rowptr, colidx, values) numpy arrays."""
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    vals = np.ascontiguousarray(values).view(np.uint32)
    p = np.ascontiguousarray(p, dtype=np.int64)
    q = None if q is None else np.ascontiguousarray(q, dtype=np.int64)
    orp = np.empty(nrows + 1, np.int64)
    oc = np.empty(colidx.shape[0], np.int32)
    ov = np.empty(colidx.shape[0], np.uint32)
    ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = lib.sp_cpu_permute(nrows, ncols, ptr(rowptr), ptr(colidx), ptr(vals), ptr(p), ptr(q), ptr(orp),
                            ptr(oc), ptr(ov))
    if rc != 0:
        raise ValueError("p or q is not a permutation")
    return orp, oc, ov.view(np.asarray(values).dtype)
