"""Plain, slow, obviously-correct CPU oracle (numpy, no blocking, no fusion).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the bench's CPU
baseline leg; never by the library.  It shares no code with the CUDA path.

Every function follows a definition of arXiv 2509.20776 (HipPerm / HipExtract /
HipAssign), written with 0-based indices (the paper is 1-based):

* permutation, Sec. 2.1: A'[i, j] = A[pvec[i], qvec[j]]  (A' = P A Q^T with
  P[i, pvec[i]] = 1);
* extraction, Sec. 2.2: B[i, j] = A[pvec[i], qvec[j]] for (i, j) in pvec x qvec
  (B = P A Q^T with rectangular P, Q); repeated indices are allowed;
* assignment, Sec. 2.3: A[pvec[i], qvec[j]] = B[i, j] for the stored entries of B
  (A = A (+) P B Q^T with a user-defined add); variants: overwrite (the common one),
  select-second, arithmetic add.

Values are moved, never computed (except the PLUS assignment); they are compared as
bit patterns, so stored zeros, -0.0 and NaN payloads are structure, not absent
entries.  Output matrices are canonical CSR: columns strictly ascending in each row.

The whole-matrix functions take the triplet route named by the definitions: list the
stored (row, col, val) triples of the input, relabel them through the index maps,
sort by (row, col) and rebuild the row pointer.  The ``*_row`` functions compute one
output row straight from the same definitions, so that outputs of very large
matrices can be checked on sampled rows.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

REPLACE, SELECT2ND, PLUS = 0, 1, 2


class OracleError(ValueError):
    """Raised for inputs the definitions reject; ``kind`` names the violated rule."""

    def __init__(self, kind: str, msg: str):
        super().__init__(f"{kind}: {msg}")
        self.kind = kind


@dataclass
class CSR:
    """CSR matrix on the host: int64 rowptr/colidx, values of any numpy dtype."""
    nrows: int
    ncols: int
    rowptr: np.ndarray
    colidx: np.ndarray
    values: np.ndarray

    @staticmethod
    def of(nrows, ncols, rowptr, colidx, values) -> "CSR":
        return CSR(int(nrows), int(ncols), np.asarray(rowptr, dtype=np.int64),
                   np.asarray(colidx, dtype=np.int64), np.asarray(values))

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def row(self, r: int):
        s, e = self.rowptr[r], self.rowptr[r + 1]
        return self.colidx[s:e], self.values[s:e]

    def triplets(self):
        rows = np.repeat(np.arange(self.nrows, dtype=np.int64), np.diff(self.rowptr))
        return rows, self.colidx, self.values


def _bits(values: np.ndarray) -> np.ndarray:
    return values.view(np.uint32 if values.dtype.itemsize == 4 else np.uint64)


def canonical_check(A: CSR) -> None:
    """Raise unless A is canonical CSR (monotone rowptr, in-range strictly sorted columns)."""
    rp = A.rowptr
    if rp.shape[0] != A.nrows + 1 or rp[0] != 0 or rp[-1] != A.nnz:
        raise OracleError("shape", "row pointer does not match nrows/nnz")
    if np.any(np.diff(rp) < 0):
        raise OracleError("not_canonical", "row pointer decreases")
    if A.nnz and (A.colidx.min() < 0 or A.colidx.max() >= A.ncols):
        raise OracleError("index_range", "column index out of range")
    if A.nnz > 1:
        rows = np.repeat(np.arange(A.nrows), np.diff(rp))
        same = rows[1:] == rows[:-1]
        if np.any(same & (A.colidx[1:] <= A.colidx[:-1])):
            raise OracleError("not_canonical", "columns not strictly ascending in a row")


def build_csr(nrows: int, ncols: int, r: np.ndarray, c: np.ndarray, v: np.ndarray) -> CSR:
    """Triplets -> canonical CSR: sort by (row, col), count per row, prefix-sum."""
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    if r.shape[0] > 1 and np.any((r[1:] == r[:-1]) & (c[1:] == c[:-1])):
        raise OracleError("duplicate_entry", "two triplets share one (row, col)")
    counts = np.bincount(r, minlength=nrows) if r.shape[0] else np.zeros(nrows, np.int64)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(nrows, ncols, rowptr, c.astype(np.int64), v)


def inverse_map(idx: np.ndarray, n: int, require_permutation: bool = False) -> np.ndarray:
    """inv[idx[k]] = k, and -1 where no k selects that position.

    This is the index/value swap of the Identify step (pvec[pvec_inv[i]] = i, Sec. 3.1,
    Step 1(a)), extended with -1 for positions absent from a selection vector (the
    sparse-vector form HipExtract builds, Sec. 4).  The entries of ``idx`` must be
    distinct and in [0, n); a permutation must also cover [0, n).
    """
    idx = np.asarray(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise OracleError("index_range", "index outside [0, n)")
    counts = np.bincount(idx, minlength=n) if idx.size else np.zeros(n, np.int64)
    if np.any(counts > 1):
        raise OracleError("not_permutation" if require_permutation else "duplicate_index",
                          "repeated index")
    if require_permutation and idx.shape[0] != n:
        raise OracleError("not_permutation", "length differs from the dimension")
    inv = np.full(n, -1, dtype=np.int64)
    inv[idx] = np.arange(idx.shape[0], dtype=np.int64)
    return inv


def exclusive_scan(x: np.ndarray) -> np.ndarray:
    """out[i] = sum_{k < i} x[k], for i = 0 .. len(x) (len(x)+1 entries, last = total).

    The row-pointer construction of the Build step and the proc_pointer /
    thread_offset prefix sums of Algorithm 2 (Fig. 3(ii)) are exclusive scans.
    """
    x = np.asarray(x, dtype=np.int64)
    out = np.zeros(x.shape[0] + 1, dtype=np.int64)
    np.cumsum(x, out=out[1:])
    return out


def permute(A: CSR, p, q) -> CSR:
    """A'[i, j] = A[p[i], q[j]]  (Sec. 2.1).  ``p``/``q`` None means identity.

    Each stored (r, c, v) lands at (i, j) with p[i] = r and q[j] = c, i.e. at
    (pinv[r], qinv[c]).
    """
    m, n = A.nrows, A.ncols
    p = np.arange(m) if p is None else np.asarray(p, dtype=np.int64)
    q = np.arange(n) if q is None else np.asarray(q, dtype=np.int64)
    pinv = inverse_map(p, m, require_permutation=True)
    qinv = inverse_map(q, n, require_permutation=True)
    r, c, v = A.triplets()
    return build_csr(m, n, pinv[r], qinv[c], v)


def permute_row(A: CSR, p, qinv: np.ndarray | None, i: int):
    """Row i of A' = P A Q^T alone: the entries of row p[i], columns relabelled by qinv,
    in ascending new-column order.  Returns (cols, values)."""
    r = i if p is None else int(p[i])
    c, v = A.row(r)
    newc = c if qinv is None else qinv[c]
    order = np.argsort(newc, kind="stable")
    return newc[order], v[order]


def _multimap(idx: np.ndarray, n: int):
    """For selection vectors with repeats: positions of each value, grouped by value."""
    idx = np.asarray(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise OracleError("index_range", "index outside [0, n)")
    count = np.bincount(idx, minlength=n) if idx.size else np.zeros(n, np.int64)
    start = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(count, out=start[1:])
    positions = np.argsort(idx, kind="stable")
    return count, start, positions


def extract(A: CSR, I, J) -> CSR:
    """B[i, j] = A[I[i], J[j]] for all (i, j) in I x J  (Sec. 2.2).

    Repeated entries of I or J are allowed: every (i, j) pair with I[i] = r and
    J[j] = c receives a copy of the stored A[r, c].
    """
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    cI, sI, pI = _multimap(I, A.nrows)
    cJ, sJ, pJ = _multimap(J, A.ncols)
    r, c, v = A.triplets()
    # one output triplet per (stored entry, i with I[i]=r, j with J[j]=c)
    k = cI[r] * cJ[c]
    ent = np.repeat(np.arange(r.shape[0], dtype=np.int64), k)
    t = np.arange(ent.shape[0], dtype=np.int64) - np.repeat(np.cumsum(k) - k, k)
    nj = cJ[c[ent]]
    ti, tj = t // np.maximum(nj, 1), t % np.maximum(nj, 1)
    new_i = pI[sI[r[ent]] + ti]
    new_j = pJ[sJ[c[ent]] + tj]
    return build_csr(I.shape[0], J.shape[0], new_i, new_j, v[ent])


def kept_counts(A: CSR, I, J) -> np.ndarray:
    """Number of stored entries of row i of A(I, J): #{k in row I[i] : col_k in J},
    counted with multiplicity when J repeats (Alg. 5's first pass counts these)."""
    I = np.asarray(I, dtype=np.int64)
    cJ = np.bincount(np.asarray(J, dtype=np.int64), minlength=A.ncols) if len(J) else \
        np.zeros(A.ncols, np.int64)
    per_entry = cJ[A.colidx]
    csum = np.zeros(A.nnz + 1, dtype=np.int64)
    np.cumsum(per_entry, out=csum[1:])
    return csum[A.rowptr[I + 1]] - csum[A.rowptr[I]]


def extract_row(A: CSR, I, jmap: np.ndarray, i: int):
    """Row i of A(I, J) for distinct J, given jmap[c] = position of c in J or -1."""
    c, v = A.row(int(I[i]))
    newc = jmap[c]
    keep = newc >= 0
    newc, v = newc[keep], v[keep]
    order = np.argsort(newc, kind="stable")
    return newc[order], v[order]


def _check_assign_args(A: CSR, I, J, B: CSR):
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    inverse_map(I, A.nrows)  # distinct, in range (Sec. 2.3: "distinct row and column indices")
    inverse_map(J, A.ncols)
    if B.nrows != I.shape[0] or B.ncols != J.shape[0]:
        raise OracleError("shape", "B must be |I| x |J|")
    return I, J


def assign(A: CSR, I, J, B: CSR, mode: int = REPLACE) -> CSR:
    """A(I, J) = B  (Sec. 2.3), returning the new matrix (A is not modified).

    REPLACE: the region I x J of A is cleared, then every stored B[i, j] is written
    to (I[i], J[j]) -- afterwards A'(I, J) equals B exactly.
    SELECT2ND: A (+) P B Q^T with the select-second add: entries of A inside the region
    that B does not store survive; where both store an entry, B's value wins.
    PLUS: A (+) P B Q^T with arithmetic addition (one IEEE add in the value type).
    """
    I, J = _check_assign_args(A, I, J, B)
    m, n = A.nrows, A.ncols
    ra, ca, va = A.triplets()
    rb, cb, vb = B.triplets()
    rb, cb = I[rb], J[cb]
    if mode == REPLACE:
        inI = np.zeros(m, bool)
        inI[I] = True
        inJ = np.zeros(n, bool)
        inJ[J] = True
        keep = ~(inI[ra] & inJ[ca])
        return build_csr(m, n, np.concatenate([ra[keep], rb]), np.concatenate([ca[keep], cb]),
                         np.concatenate([va[keep], vb]))
    key_a = ra * n + ca
    key_b = rb * n + cb
    both = np.isin(key_a, key_b)
    if mode == SELECT2ND:
        keep = ~both
        return build_csr(m, n, np.concatenate([ra[keep], rb]), np.concatenate([ca[keep], cb]),
                         np.concatenate([va[keep], vb]))
    if mode == PLUS:
        # B's entries that meet an A entry are added onto it; the rest are inserted
        pos_in_b = {int(k): t for t, k in enumerate(key_b)}
        va2 = va.copy()
        hit_b = np.zeros(key_b.shape[0], bool)
        for t in np.nonzero(both)[0]:
            u = pos_in_b[int(key_a[t])]
            va2[t] = va[t] + vb[u]
            hit_b[u] = True
        new = ~hit_b
        return build_csr(m, n, np.concatenate([ra, rb[new]]), np.concatenate([ca, cb[new]]),
                         np.concatenate([va2, vb[new]]))
    raise OracleError("invalid_arg", f"unknown assign mode {mode}")


def assign_row(A: CSR, I, J, B: CSR, rowmap: np.ndarray, jset: np.ndarray, r: int):
    """Row r of A' = (A(I, J) = B) under REPLACE, straight from the definition.

    rowmap[r] = i with I[i] = r or -1; jset is a boolean membership mask of J.
    """
    c, v = A.row(r)
    i = int(rowmap[r])
    if i < 0:
        return c, v
    keep = ~jset[c]
    cb, vb = B.row(i)
    cols = np.concatenate([c[keep], np.asarray(J, dtype=np.int64)[cb]])
    vals = np.concatenate([v[keep], vb])
    order = np.argsort(cols, kind="stable")
    return cols[order], vals[order]


def to_dense(A: CSR):
    """(dense values, presence mask) -- for brute-force checks on tiny matrices."""
    D = np.zeros((A.nrows, A.ncols), dtype=A.values.dtype)
    M = np.zeros((A.nrows, A.ncols), dtype=bool)
    r, c, v = A.triplets()
    D[r, c] = v
    M[r, c] = True
    return D, M


def from_dense(D: np.ndarray, M: np.ndarray) -> CSR:
    r, c = np.nonzero(M)
    return build_csr(D.shape[0], D.shape[1], r.astype(np.int64), c.astype(np.int64), D[r, c])
