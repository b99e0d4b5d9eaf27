"""Shared test helpers: conversions between the synth / oracle / binding matrix types."""
from __future__ import annotations

import numpy as np
import torch

import oracle


def to_oracle(A) -> oracle.CSR:
    """Any CSR with torch tensors (synth.CSRTensors or binding CSR) -> oracle.CSR on host."""
    return oracle.CSR.of(A.nrows, A.ncols, A.rowptr.cpu().numpy().astype(np.int64),
                         A.colidx.cpu().numpy().astype(np.int64), A.values.cpu().numpy())


def to_dev(A, device="cuda", rowptr_dtype=None, colidx_dtype=None):
    from paper_2509_20776_gb300 import CSR
    return CSR(A.nrows, A.ncols, A.rowptr.to(device=device, dtype=rowptr_dtype or A.rowptr.dtype),
               A.colidx.to(device=device, dtype=colidx_dtype or A.colidx.dtype),
               A.values.to(device))


def from_oracle(O: oracle.CSR, rowptr_dtype=torch.int64, colidx_dtype=torch.int32, device="cuda"):
    from paper_2509_20776_gb300 import CSR
    return CSR(O.nrows, O.ncols, torch.from_numpy(O.rowptr).to(device=device, dtype=rowptr_dtype),
               torch.from_numpy(O.colidx).to(device=device, dtype=colidx_dtype),
               torch.from_numpy(np.ascontiguousarray(O.values)).to(device))


def bits(v: np.ndarray) -> np.ndarray:
    return v.view(np.uint64 if v.dtype.itemsize == 8 else np.uint32)


def assert_same(got, want: oracle.CSR, what=""):
    """Bit-exact comparison of a device result with an oracle matrix."""
    assert (got.nrows, got.ncols) == (want.nrows, want.ncols), f"{what}: shape"
    rp = got.rowptr.cpu().numpy().astype(np.int64)
    assert np.array_equal(rp, want.rowptr), f"{what}: rowptr differs at " \
        f"{np.nonzero(rp != want.rowptr)[0][:5]}"
    ci = got.colidx.cpu().numpy().astype(np.int64)
    if not np.array_equal(ci, want.colidx):
        bad = np.nonzero(ci != want.colidx)[0]
        row = np.searchsorted(want.rowptr, bad[0], side="right") - 1
        raise AssertionError(f"{what}: colidx differs at {bad[:5]} (row {row}, "
                             f"{bad.shape[0]} positions)")
    gv = bits(got.values.cpu().numpy())
    assert np.array_equal(gv, bits(np.ascontiguousarray(want.values))), f"{what}: value bits"
