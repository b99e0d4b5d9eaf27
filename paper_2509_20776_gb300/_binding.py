"""ctypes binding of the C ABI in ``include/sp.h`` (argument marshalling only).

Every function here converts torch tensors to device pointers and sizes, calls the
entry point of the same name in ``libspgb.so`` and turns a non-zero status into
``SpError``.  No step of the path runs in Python: if the shared library is missing
the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspgb.so")

SP_I32, SP_I64 = 0, 1
SP_F32, SP_F64 = 0, 1
SP_ASSIGN_REPLACE, SP_ASSIGN_SELECT2ND, SP_ASSIGN_PLUS = 0, 1, 2
SP_OPT_SPIN_LIMIT, SP_OPT_SCAN_HOLD_TILE, SP_OPT_VALIDATE, SP_OPT_TIMING = 0, 1, 2, 3
# kernel shapes (run-time; every value gives the same output)
SP_OPT_TILE_SHAPE, SP_OPT_HEAVY, SP_OPT_COUNT_ROWS, SP_OPT_FILL_ROWS, SP_OPT_BATCH_ROWS = 4, 5, 6, 7, 8
SP_OPT_IDENTIFY = 9
SP_OPT_OVERLAP = 10
SHAPE_OPTIONS = {"tile_shape": SP_OPT_TILE_SHAPE, "heavy": SP_OPT_HEAVY, "count_rows": SP_OPT_COUNT_ROWS,
                 "fill_rows": SP_OPT_FILL_ROWS, "batch_rows": SP_OPT_BATCH_ROWS, "identify": SP_OPT_IDENTIFY}
SHAPE_VALUES = {"tile_shape": (0, 1), "heavy": (128, 256, 512, 1024, 2048, 4096), "count_rows": (1, 2, 3, 4),
                "fill_rows": (1, 2), "batch_rows": (1, 2, 4, 8), "identify": (0, 1)}
OPS = {"permute": 0, "extract": 1, "assign": 2, "batch": 3}
PHASES = ["map", "count", "scan", "partition", "tile", "long", "huge", "gather", "other"]
STATUS = ["SP_OK", "SP_ERR_INVALID_ARG", "SP_ERR_SHAPE", "SP_ERR_INDEX_RANGE",
          "SP_ERR_DUPLICATE_INDEX", "SP_ERR_NOT_PERMUTATION", "SP_ERR_NOT_CANONICAL",
          "SP_ERR_OVERFLOW", "SP_ERR_OOM", "SP_ERR_TIMEOUT", "SP_ERR_CUDA", "SP_ERR_INTERNAL"]


class SpError(RuntimeError):
    def __init__(self, code: int, where: str, detail: int = -1):
        name = STATUS[code] if 0 <= code < len(STATUS) else f"status {code}"
        super().__init__(f"{where}: {name}" + (f" (detail {detail})" if detail != -1 else ""))
        self.code = code
        self.name = name
        self.detail = detail


class sp_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr_type", ctypes.c_int), ("colidx_type", ctypes.c_int),
                ("value_type", ctypes.c_int), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class sp_tune_entry(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("tile_shape", ctypes.c_int32), ("heavy", ctypes.c_int32),
                ("count_rows", ctypes.c_int32), ("fill_rows", ctypes.c_int32), ("batch_rows", ctypes.c_int32),
                ("identify", ctypes.c_int32), ("size_max", ctypes.c_int64)]


def tune_entries(table) -> list:
    """Validated tuning entries from a table (the autotuner's JSON object, or its list of
    entries): dicts with "op" (permute / extract / assign / batch), "size_max" and any of
    the shape names; absent shapes are -1 (keep the context's option).  Entries come out
    ordered by (op, size_max), so the first entry that covers a call is its tightest
    size class."""
    items = table["entries"] if isinstance(table, dict) else table
    out = []
    for e in items:
        if e["op"] not in OPS:
            raise ValueError(f"unknown op {e['op']!r}")
        row = {"op": OPS[e["op"]], "size_max": int(e["size_max"])}
        for k, allowed in SHAPE_VALUES.items():
            v = int(e.get(k, -1))
            if v >= 0 and v not in allowed:
                raise ValueError(f"{k}={v} not in {allowed}")
            row[k] = v
        out.append(row)
    out.sort(key=lambda r: (r["op"], r["size_max"]))
    return out


def tune_array(table):
    """ctypes array of the entries of a table (see ``tune_entries``) and its length."""
    rows = tune_entries(table) if table else []
    arr = (sp_tune_entry * max(1, len(rows)))()
    for i, r in enumerate(rows):
        arr[i] = sp_tune_entry(r["op"], r["tile_shape"], r["heavy"], r["count_rows"], r["fill_rows"],
                               r["batch_rows"], r["identify"], r["size_max"])
    return arr, len(rows)


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class sp_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


class TorchAllocator:
    """Device memory for a context from PyTorch's caching allocator (the sp_allocator hook
    of include/sp.h): ``alloc(nbytes, stream)`` returns a device address or 0, ``free(ptr,
    nbytes, stream)`` returns it.  Subclasses may refuse allocations (failure injection)."""

    def __init__(self, device: int = 0):
        self.device = device

    def alloc(self, nbytes: int, stream: int) -> int:
        return torch.cuda.caching_allocator_alloc(max(1, nbytes), self.device, stream or 0)

    def free(self, ptr: int, nbytes: int, stream: int) -> None:
        torch.cuda.caching_allocator_delete(ptr)


class sp_extract_req(ctypes.Structure):
    _fields_ = [("mat", ctypes.c_int64), ("nI", ctypes.c_int64), ("nJ", ctypes.c_int64),
                ("I", ctypes.c_void_p), ("J", ctypes.c_void_p)]


class sp_permute_req(ctypes.Structure):
    _fields_ = [("mat", ctypes.c_int64), ("p", ctypes.c_void_p), ("q", ctypes.c_void_p)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_PCSR = ctypes.POINTER(sp_csr)
_PREQ = ctypes.POINTER(sp_extract_req)
_PPREQ = ctypes.POINTER(sp_permute_req)
SIGNATURES = {
    "sp_status_str": (ctypes.c_char_p, [_int]),
    "sp_version": (_int, []),
    "sp_ctx_create": (_int, [ctypes.POINTER(_vp), _int, _vp]),
    "sp_ctx_destroy": (_int, [_vp]),
    "sp_ctx_sync": (_int, [_vp, _vp]),
    "sp_ctx_error_detail": (_i64, [_vp]),
    "sp_last_cuda_error": (_int, [ctypes.POINTER(ctypes.c_char_p)]),
    "sp_ctx_set_option": (_int, [_vp, _int, _i64]),
    "sp_ctx_set_tuning": (_int, [_vp, ctypes.POINTER(sp_tune_entry), _int]),
    "sp_tuning_lookup": (_int, [ctypes.POINTER(sp_tune_entry), _int, _int, _i64, ctypes.POINTER(sp_tune_entry)]),
    "sp_permute": (_int, [_vp, _PCSR, _vp, _vp, _int, _PCSR, _vp]),
    "sp_extract_count": (_int, [_vp, _PCSR, _vp, _i64, _vp, _i64, _int, ctypes.POINTER(_vp),
                                ctypes.POINTER(_i64), _vp]),
    "sp_extract_fill": (_int, [_vp, _vp, _PCSR, _vp]),
    "sp_extract": (_int, [_vp, _PCSR, _vp, _i64, _vp, _i64, _int, _PCSR, _vp]),
    "sp_assign_count": (_int, [_vp, _PCSR, _vp, _i64, _vp, _i64, _int, _PCSR, _int,
                               ctypes.POINTER(_vp), ctypes.POINTER(_i64), _vp]),
    "sp_assign_fill": (_int, [_vp, _vp, _PCSR, _vp]),
    "sp_assign": (_int, [_vp, _PCSR, _vp, _i64, _vp, _i64, _int, _PCSR, _int, _PCSR, _vp]),
    "sp_assign_permute_fill": (_int, [_vp, _vp, _vp, _vp, _PCSR, _vp]),
    "sp_assign_permute": (_int, [_vp, _PCSR, _vp, _i64, _vp, _i64, _int, _PCSR, _int, _vp, _vp, _PCSR,
                                 _vp]),
    "sp_extract_batch_count": (_int, [_vp, _PCSR, _i64, _PREQ, _i64, _int, _vp, _vp, _vp]),
    "sp_extract_batch_fill": (_int, [_vp, _vp, _PCSR, _vp]),
    "sp_extract_batch_run": (_int, [_vp, _vp, _PCSR, _vp]),
    "sp_batch_row_offset": (_i64, [_vp, _i64]),
    "sp_batch_destroy": (_int, [_vp, _vp]),
    "sp_permute_batch_plan": (_int, [_vp, _PCSR, _i64, _PPREQ, _i64, _int, _vp, _vp, _vp]),
    "sp_permute_batch_fill": (_int, [_vp, _vp, _PCSR, _vp]),
    "sp_pbatch_row_offset": (_i64, [_vp, _i64]),
    "sp_pbatch_destroy": (_int, [_vp, _vp]),
    "sp_plan_destroy": (_int, [_vp, _vp]),
    "sp_csr_free": (_int, [_vp, _PCSR]),
    "sp_inverse_map": (_int, [_vp, _vp, _i64, _i64, _int, _vp, _int, _vp]),
    "sp_exclusive_scan": (_int, [_vp, _vp, _int, _i64, _vp, _int, _vp]),
    "sp_exclusive_scan_noalloc": (_int, [_vp, _int, _i64, _vp, _int, _vp]),
    "sp_kept_counts": (_int, [_vp, _PCSR, _vp, _i64, _vp, _i64, _int, _vp, _vp]),
    "sp_sort_rows": (_int, [_vp, _PCSR, _vp]),
    "sp_csr_validate": (_int, [_vp, _PCSR, _vp]),
    "sp_ctx_phase_stats": (_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _int]),
    "sp_phase_name": (ctypes.c_char_p, [_int]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libspgb.so (built by ``paper_2509_20776_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run paper_2509_20776_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _itype(dtype: torch.dtype) -> int:
    if dtype == torch.int32:
        return SP_I32
    if dtype == torch.int64:
        return SP_I64
    raise TypeError(f"index tensors must be int32 or int64, got {dtype}")


def _vtype(dtype: torch.dtype) -> int:
    if dtype == torch.float32:
        return SP_F32
    if dtype == torch.float64:
        return SP_F64
    raise TypeError(f"values must be float32 or float64, got {dtype}")


_ITORCH = {SP_I32: torch.int32, SP_I64: torch.int64}
_VTORCH = {SP_F32: torch.float32, SP_F64: torch.float64}


def _ptr(t):
    return None if t is None or t.numel() == 0 else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class CSR:
    """CSR matrix whose arrays are CUDA tensors (rowptr/colidx int32|int64, values f32|f64)."""
    nrows: int
    ncols: int
    rowptr: torch.Tensor
    colidx: torch.Tensor
    values: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    def desc(self) -> sp_csr:
        for t in (self.rowptr, self.colidx, self.values):
            if not t.is_contiguous():
                raise ValueError("CSR arrays must be contiguous")
        return sp_csr(self.nrows, self.ncols, self.nnz, _itype(self.rowptr.dtype),
                      _itype(self.colidx.dtype), _vtype(self.values.dtype),
                      ctypes.c_void_p(self.rowptr.data_ptr()) if self.rowptr.numel() else None,
                      _ptr(self.colidx), _ptr(self.values))


class Context:
    """Owns an ``sp_ctx`` (workspace, device error record) for one CUDA device."""

    def __init__(self, device: int | None = None, allocator=None):
        """``allocator``: an object with ``alloc(nbytes, stream) -> int`` and ``free(ptr,
        nbytes, stream)`` (e.g. ``TorchAllocator``) through which the library takes its
        workspace, plans and library-allocated outputs; None = stream-ordered cudaMallocAsync."""
        self.lib = load_library()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        self._allocator_c = None
        if allocator is not None:
            def _a(user, nbytes, stream):
                try:
                    return allocator.alloc(int(nbytes), int(stream or 0)) or None
                except Exception:  # noqa: BLE001  (a failed allocation is reported as NULL)
                    return None

            def _f(user, ptr, nbytes, stream):
                if ptr:
                    allocator.free(int(ptr), int(nbytes), int(stream or 0))

            self._allocator_c = sp_allocator(_ALLOC_FN(_a), _FREE_FN(_f), None)  # kept alive with the context
        h = ctypes.c_void_p()
        self._check(self.lib.sp_ctx_create(ctypes.byref(h), device,
                                           ctypes.byref(self._allocator_c) if self._allocator_c is not None else None),
                    "sp_ctx_create")
        self.handle = h

    def _check(self, code: int, where: str):
        if code != 0:
            detail = self.lib.sp_ctx_error_detail(self.handle) if getattr(self, "handle", None) else -1
            if code == STATUS.index("SP_ERR_CUDA"):  # name the CUDA error and the library line behind it
                w = ctypes.c_char_p()
                self.lib.sp_last_cuda_error(ctypes.byref(w))
                where = f"{where} [{(w.value or b'').decode()}]"
            raise SpError(code, where, detail)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: int, value: int):
        self._check(self.lib.sp_ctx_set_option(self.handle, key, value), "sp_ctx_set_option")

    def set_shapes(self, **shapes):
        """Context-wide kernel shapes by name (tile_shape, heavy, count_rows, fill_rows,
        batch_rows); -1 restores a default."""
        for k, v in shapes.items():
            self.set_option(SHAPE_OPTIONS[k], int(v))

    def set_tuning(self, table):
        """Installs a tuning table (see ``tune_entries``; a path to the autotuner's JSON
        file also works); None or [] removes it."""
        if isinstance(table, str):
            import json
            with open(table) as f:
                table = json.load(f)
        arr, n = tune_array(table)
        self._check(self.lib.sp_ctx_set_tuning(self.handle, arr, n), "sp_ctx_set_tuning")

    def phase_stats(self, reset: bool = False) -> dict:
        """{phase: (device ms, kernel launches)} accumulated since the last reset."""
        n = len(PHASES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self._check(self.lib.sp_ctx_phase_stats(self.handle, ms, cnt, 1 if reset else 0),
                    "sp_ctx_phase_stats")
        return {PHASES[i]: (ms[i], cnt[i]) for i in range(n)}

    def sync(self, stream=None):
        """Wait for the stream; raise the first device-detected error (if any)."""
        self._check(self.lib.sp_ctx_sync(self.handle, _stream(stream)), "sp_ctx_sync")

    # ---- ops ---------------------------------------------------------------------
    def sp_permute(self, A: CSR, p=None, q=None, rowptr_dtype=None, stream=None,
                   sync: bool = True, out: CSR | None = None) -> CSR:
        """B = P A Q^T, B[i, j] = A[p[i], q[j]] (p/q None = identity; q is p = symmetric).

        ``out``: a preallocated result (same shape and types) to write into."""
        idx_t = _itype((p if p is not None else q).dtype) if (p is not None or q is not None) \
            else SP_I32
        rp_t = _itype(rowptr_dtype or A.rowptr.dtype)
        dev = A.colidx.device
        B = out if out is not None else CSR(
            A.nrows, A.ncols, torch.empty(A.nrows + 1, dtype=_ITORCH[rp_t], device=dev),
            torch.empty(A.nnz, dtype=A.colidx.dtype, device=dev),
            torch.empty(A.nnz, dtype=A.values.dtype, device=dev))
        d = B.desc()
        qp = _ptr(q)  # the same tensor for p and q gives the same pointer: P A P^T
        self._check(self.lib.sp_permute(self.handle, ctypes.byref(A.desc()), _ptr(p), qp, idx_t,
                                         ctypes.byref(d), _stream(stream)), "sp_permute")
        if sync:
            self.sync(stream)
        return B

    def sp_extract(self, A: CSR, I: torch.Tensor, J: torch.Tensor, rowptr_dtype=None,
                   stream=None, sync: bool = True) -> CSR:
        """B = A(I, J): B[i, j] = A[I[i], J[j]] (count, allocate with torch, fill)."""
        idx_t = _itype(I.dtype)
        if J.dtype != I.dtype:
            raise TypeError("I and J must share a dtype")
        plan = ctypes.c_void_p()
        nnz = ctypes.c_int64()
        st = _stream(stream)
        self._check(self.lib.sp_extract_count(self.handle, ctypes.byref(A.desc()), _ptr(I),
                                              I.numel(), _ptr(J), J.numel(), idx_t,
                                              ctypes.byref(plan), ctypes.byref(nnz), st),
                    "sp_extract_count")
        try:
            B = self._alloc(I.numel(), J.numel(), nnz.value, rowptr_dtype or A.rowptr.dtype, A)
            d = B.desc()
            self._check(self.lib.sp_extract_fill(self.handle, plan, ctypes.byref(d), st),
                        "sp_extract_fill")
        finally:
            self.lib.sp_plan_destroy(self.handle, plan)
        if sync:
            self.sync(stream)
        return B

    def sp_assign(self, A: CSR, I: torch.Tensor, J: torch.Tensor, B: CSR,
                  mode: int = SP_ASSIGN_REPLACE, rowptr_dtype=None, stream=None,
                  sync: bool = True) -> CSR:
        """A' = A with A'(I, J) = B (REPLACE), A is left unchanged."""
        idx_t = _itype(I.dtype)
        plan = ctypes.c_void_p()
        nnz = ctypes.c_int64()
        st = _stream(stream)
        self._check(self.lib.sp_assign_count(self.handle, ctypes.byref(A.desc()), _ptr(I),
                                             I.numel(), _ptr(J), J.numel(), idx_t,
                                             ctypes.byref(B.desc()), mode, ctypes.byref(plan),
                                             ctypes.byref(nnz), st), "sp_assign_count")
        try:
            Ap = self._alloc(A.nrows, A.ncols, nnz.value, rowptr_dtype or A.rowptr.dtype, A)
            d = Ap.desc()
            self._check(self.lib.sp_assign_fill(self.handle, plan, ctypes.byref(d), st),
                        "sp_assign_fill")
        finally:
            self.lib.sp_plan_destroy(self.handle, plan)
        if sync:
            self.sync(stream)
        return Ap

    def sp_assign_permute(self, A: CSR, I: torch.Tensor, J: torch.Tensor, B: CSR, p=None, q=None,
                          mode: int = SP_ASSIGN_REPLACE, rowptr_dtype=None, stream=None,
                          sync: bool = True) -> CSR:
        """out = P (A with A(I, J) (+) B) Q^T without forming the assigned matrix
        (p/q None = identity; q is p = symmetric)."""
        idx_t = _itype(I.dtype)
        plan = ctypes.c_void_p()
        nnz = ctypes.c_int64()
        st = _stream(stream)
        self._check(self.lib.sp_assign_count(self.handle, ctypes.byref(A.desc()), _ptr(I),
                                             I.numel(), _ptr(J), J.numel(), idx_t,
                                             ctypes.byref(B.desc()), mode, ctypes.byref(plan),
                                             ctypes.byref(nnz), st), "sp_assign_count")
        try:
            out = self._alloc(A.nrows, A.ncols, nnz.value, rowptr_dtype or A.rowptr.dtype, A)
            d = out.desc()
            self._check(self.lib.sp_assign_permute_fill(self.handle, plan, _ptr(p), _ptr(q),
                                                        ctypes.byref(d), st),
                        "sp_assign_permute_fill")
        finally:
            self.lib.sp_plan_destroy(self.handle, plan)
        if sync:
            self.sync(stream)
        return out

    def extract_batch(self, mats, requests, stream=None) -> "ExtractBatch":
        """Count a batch of extractions B_k = mats[m_k](I_k, J_k); ``requests`` holds
        (m_k, I_k, J_k) with device index tensors of one dtype.  Synchronises once."""
        return ExtractBatch(self, mats, requests, stream)

    def sp_extract_batch(self, mats, requests, rowptr_dtype=torch.int64, stream=None):
        """All results of a batch in one CSR plus the first row of every request."""
        bt = self.extract_batch(mats, requests, stream)
        try:
            out = bt.alloc(rowptr_dtype)
            bt.fill(out, stream)
            self.sync(stream)
            return out, bt.row_offsets()
        finally:
            bt.close()

    def permute_batch(self, mats, requests, stream=None) -> "PermuteBatch":
        """Plan a batch of permutations B_k = P_k mats[m_k] Q_k^T; ``requests`` holds
        (m_k, p_k, q_k) with device index tensors of one dtype (or None for the identity).
        Host only: the output size is the sum of the matrices' nnz."""
        return PermuteBatch(self, mats, requests, stream)

    def sp_permute_batch(self, mats, requests, rowptr_dtype=torch.int64, stream=None):
        """All results of a batch of permutations in one CSR plus the first row of every
        request."""
        bt = self.permute_batch(mats, requests, stream)
        try:
            out = bt.alloc(rowptr_dtype)
            bt.fill(out, stream)
            self.sync(stream)
            return out, bt.row_offsets()
        finally:
            bt.close()

    def _alloc(self, nrows, ncols, nnz, rowptr_dtype, like: CSR) -> CSR:
        dev = like.colidx.device
        return CSR(nrows, ncols, torch.empty(nrows + 1, dtype=rowptr_dtype, device=dev),
                   torch.empty(nnz, dtype=like.colidx.dtype, device=dev),
                   torch.empty(nnz, dtype=like.values.dtype, device=dev))

    # ---- steps ------------------------------------------------------------------------
    def sp_inverse_map(self, idx: torch.Tensor, n: int, require_permutation: bool = False,
                       stream=None, sync: bool = True) -> torch.Tensor:
        inv = torch.empty(n, dtype=idx.dtype, device=idx.device)
        self._check(self.lib.sp_inverse_map(self.handle, _ptr(idx), idx.numel(), n,
                                            _itype(idx.dtype), _ptr(inv),
                                            1 if require_permutation else 0, _stream(stream)),
                    "sp_inverse_map")
        if sync:
            self.sync(stream)
        return inv

    def sp_exclusive_scan(self, x: torch.Tensor, out_dtype=torch.int64, stream=None,
                          sync: bool = True) -> torch.Tensor:
        out = torch.empty(x.numel() + 1, dtype=out_dtype, device=x.device)
        self._check(self.lib.sp_exclusive_scan(self.handle, _ptr(x), _itype(x.dtype), x.numel(),
                                               ctypes.c_void_p(out.data_ptr()), _itype(out_dtype),
                                               _stream(stream)), "sp_exclusive_scan")
        if sync:
            self.sync(stream)
        return out

    def sp_kept_counts(self, A: CSR, I: torch.Tensor, J: torch.Tensor, stream=None) -> torch.Tensor:
        counts = torch.empty(I.numel(), dtype=torch.int64, device=I.device)
        self._check(self.lib.sp_kept_counts(self.handle, ctypes.byref(A.desc()), _ptr(I),
                                            I.numel(), _ptr(J), J.numel(), _itype(I.dtype),
                                            _ptr(counts), _stream(stream)), "sp_kept_counts")
        self.sync(stream)
        return counts

    def sp_sort_rows(self, M: CSR, stream=None, sync: bool = True) -> CSR:
        """Sort each row of M by column in place (columns distinct within a row)."""
        self._check(self.lib.sp_sort_rows(self.handle, ctypes.byref(M.desc()), _stream(stream)),
                    "sp_sort_rows")
        if sync:
            self.sync(stream)
        return M

    def sp_csr_validate(self, A: CSR, stream=None):
        self._check(self.lib.sp_csr_validate(self.handle, ctypes.byref(A.desc()),
                                             _stream(stream)), "sp_csr_validate")


def mat_descs(mats):
    """The descriptor array of a list of matrices, as the batch calls take it (build it
    once for matrices that stay registered)."""
    return (sp_csr * len(mats))(*[m.desc() for m in mats])


class ExtractBatch:
    """A counted batch of extractions (``sp_extract_batch_count``): ``fill`` launches the
    whole batch without synchronising (capturable in a CUDA graph)."""

    def __init__(self, ctx: Context, mats, requests, stream=None, descs=None):
        self.ctx = ctx
        self.mats = list(mats)
        self.requests = list(requests)
        self.handle = None
        if not self.mats:
            raise ValueError("a batch needs at least one matrix")
        dt = self.requests[0][1].dtype if self.requests else torch.int32
        idx_t = _itype(dt)
        # descs: the matrices' descriptor array (mat_descs), reused across batches
        self._descs = descs if descs is not None else mat_descs(self.mats)
        self._reqs = (sp_extract_req * max(1, len(self.requests)))()
        for k, (mi, I, J) in enumerate(self.requests):
            if I.dtype != dt or J.dtype != dt:
                raise TypeError("all index tensors of a batch share one dtype")
            self._reqs[k] = sp_extract_req(int(mi), I.numel(), J.numel(),
                                           I.data_ptr() if I.numel() else None,
                                           J.data_ptr() if J.numel() else None)
        h = ctypes.c_void_p()
        nnz = ctypes.c_int64()
        ctx._check(ctx.lib.sp_extract_batch_count(ctx.handle, self._descs, len(self.mats), self._reqs,
                                                  len(self.requests), idx_t, ctypes.byref(h),
                                                  ctypes.byref(nnz), _stream(stream)),
                   "sp_extract_batch_count")
        self.handle = h
        self.nnz = nnz.value
        self.rows = int(ctx.lib.sp_batch_row_offset(h, len(self.requests)))
        self.ncols = max([J.numel() for _, _, J in self.requests] + [0])

    def row_offsets(self):
        return [int(self.ctx.lib.sp_batch_row_offset(self.handle, k))
                for k in range(len(self.requests) + 1)]

    def alloc(self, rowptr_dtype=torch.int64) -> CSR:
        like = self.mats[0]
        dev = like.colidx.device
        return CSR(self.rows, self.ncols, torch.empty(self.rows + 1, dtype=rowptr_dtype, device=dev),
                   torch.empty(self.nnz, dtype=like.colidx.dtype, device=dev),
                   torch.empty(self.nnz, dtype=like.values.dtype, device=dev))

    def fill(self, out: CSR, stream=None):
        self._out_desc = out.desc()  # kept alive: a captured graph replays with these pointers
        self.ctx._check(self.ctx.lib.sp_extract_batch_fill(self.ctx.handle, self.handle,
                                                           ctypes.byref(self._out_desc), _stream(stream)),
                        "sp_extract_batch_fill")

    def run(self, out: CSR, stream=None):
        """The whole batch again (identify, count, row pointer, fill, sort) into `out`
        (capacity: the counted nnz), without allocating or synchronising: capturable."""
        self._run_desc = out.desc()
        self.ctx._check(self.ctx.lib.sp_extract_batch_run(self.ctx.handle, self.handle,
                                                          ctypes.byref(self._run_desc), _stream(stream)),
                        "sp_extract_batch_run")

    def close(self):
        if self.handle:
            self.ctx.lib.sp_batch_destroy(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PermuteBatch:
    """A planned batch of permutations (``sp_permute_batch_plan``): ``fill`` launches the
    whole batch, its validation included, without synchronising (capturable in a CUDA
    graph)."""

    def __init__(self, ctx: Context, mats, requests, stream=None, descs=None):
        self.ctx = ctx
        self.mats = list(mats)
        self.requests = list(requests)
        self.handle = None
        if not self.mats:
            raise ValueError("a batch needs at least one matrix")
        dts = {t.dtype for _, p, q in self.requests for t in (p, q) if t is not None}
        if len(dts) > 1:
            raise TypeError("all index tensors of a batch share one dtype")
        idx_t = _itype(dts.pop() if dts else torch.int32)
        self._descs = descs if descs is not None else mat_descs(self.mats)
        self._reqs = (sp_permute_req * max(1, len(self.requests)))()
        for k, (mi, p, q) in enumerate(self.requests):
            a = self.mats[int(mi)] if 0 <= int(mi) < len(self.mats) else None
            if a is not None and ((p is not None and p.numel() != a.nrows) or
                                  (q is not None and q.numel() != a.ncols)):
                raise ValueError(f"request {k}: p needs nrows and q ncols entries")
            self._reqs[k] = sp_permute_req(int(mi), p.data_ptr() if p is not None and p.numel() else None,
                                           q.data_ptr() if q is not None and q.numel() else None)
        h = ctypes.c_void_p()
        nnz = ctypes.c_int64()
        ctx._check(ctx.lib.sp_permute_batch_plan(ctx.handle, self._descs, len(self.mats), self._reqs,
                                                 len(self.requests), idx_t, ctypes.byref(h),
                                                 ctypes.byref(nnz), _stream(stream)),
                   "sp_permute_batch_plan")
        self.handle = h
        self.nnz = nnz.value
        self.rows = int(ctx.lib.sp_pbatch_row_offset(h, len(self.requests)))
        self.ncols = max([self.mats[int(mi)].ncols for mi, _, _ in self.requests] + [0])

    def row_offsets(self):
        return [int(self.ctx.lib.sp_pbatch_row_offset(self.handle, k))
                for k in range(len(self.requests) + 1)]

    def alloc(self, rowptr_dtype=torch.int64) -> CSR:
        like = self.mats[0]
        dev = like.colidx.device
        return CSR(self.rows, self.ncols, torch.empty(self.rows + 1, dtype=rowptr_dtype, device=dev),
                   torch.empty(self.nnz, dtype=like.colidx.dtype, device=dev),
                   torch.empty(self.nnz, dtype=like.values.dtype, device=dev))

    def fill(self, out: CSR, stream=None):
        self._out_desc = out.desc()  # kept alive: a captured graph replays with these pointers
        self.ctx._check(self.ctx.lib.sp_permute_batch_fill(self.ctx.handle, self.handle,
                                                           ctypes.byref(self._out_desc), _stream(stream)),
                        "sp_permute_batch_fill")

    def close(self):
        if self.handle:
            self.ctx.lib.sp_pbatch_destroy(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
