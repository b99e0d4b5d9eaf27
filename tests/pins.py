"""Checks that pin the oracle to things other than itself.

Each ``pin_*`` function takes an implementation namespace (the oracle, or a copy of
it with a planted mistake) and raises AssertionError when the implementation
disagrees with:

* dense brute force on tiny matrices -- the paper's definitions evaluated entry by
  entry on dense arrays with a presence mask (Sec. 2.1, 2.2, 2.3);
* exhaustive enumeration of all permutation pairs of a 4 x 4 matrix;
* scipy.sparse fancy indexing (an independent library routine for A[I][:, J]);
* closed forms (exclusive scans of ones and of 0..k-1);
* invariants the paper states or implies: identity, p then p^-1, full extraction,
  permutation as extraction with full index vectors (Sec. 2.2), extract-after-assign,
  the streaming split / re-assign round trip (Sec. 6.3).
"""
from __future__ import annotations

import itertools

import numpy as np


def rand_csr(ns, rng, m, n, density, dtype=np.float64, special=False):
    M = rng.random((m, n)) < density
    D = np.zeros((m, n), dtype=dtype)
    k = int(M.sum())
    vals = (rng.permutation(k) + 1).astype(dtype) * (1 if rng.random() < 0.5 else -0.5)
    if special and k >= 3:
        vals[0] = -0.0
        vals[1] = 0.0
        vals[2] = np.nan
    D[M] = vals
    return ns.from_dense(D, M), D, M


def same_csr(X, Y, what=""):
    assert X.nrows == Y.nrows and X.ncols == Y.ncols, f"{what}: shape"
    assert np.array_equal(X.rowptr, Y.rowptr), f"{what}: rowptr"
    assert np.array_equal(X.colidx, Y.colidx), f"{what}: colidx"
    bx = X.values.view(np.uint64 if X.values.dtype.itemsize == 8 else np.uint32)
    by = Y.values.view(np.uint64 if Y.values.dtype.itemsize == 8 else np.uint32)
    assert np.array_equal(bx, by), f"{what}: value bits"


def dense_eq(X, D, M, what=""):
    assert (X.nrows, X.ncols) == D.shape, f"{what}: shape"
    rows = np.repeat(np.arange(X.nrows), np.diff(X.rowptr))
    # canonical: strictly ascending columns within rows
    if X.nnz > 1:
        same = rows[1:] == rows[:-1]
        assert not np.any(same & (X.colidx[1:] <= X.colidx[:-1])), f"{what}: not canonical"
    XM = np.zeros(D.shape, bool)
    XM[rows, X.colidx] = True
    assert np.array_equal(XM, M), f"{what}: pattern"
    got = X.values.view(np.uint64)
    want = D[rows, X.colidx].view(np.uint64)
    assert np.array_equal(got, want), f"{what}: values"


def pin_permute_dense(ns, seeds=60):
    rng = np.random.default_rng(11)
    for s in range(seeds):
        m, n = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        A, D, M = rand_csr(ns, rng, m, n, 0.35, special=(s % 5 == 0))
        p, q = rng.permutation(m), rng.permutation(n)
        X = ns.permute(A, p, q)
        dense_eq(X, D[p][:, q], M[p][:, q], f"permute seed {s}")
        # symmetric P A P^T on square matrices
        if m == n:
            dense_eq(ns.permute(A, p, p), D[p][:, p], M[p][:, p], f"sym seed {s}")


def pin_permute_exhaustive(ns):
    D = np.arange(1, 17, dtype=np.float64).reshape(4, 4)
    M = np.array([[1, 0, 1, 0], [0, 1, 1, 0], [1, 0, 0, 1], [0, 1, 0, 1]], bool)
    D[~M] = 0
    A = ns.from_dense(D, M)
    for p in itertools.permutations(range(4)):
        for q in itertools.permutations(range(4)):
            p_, q_ = np.array(p), np.array(q)
            dense_eq(ns.permute(A, p_, q_), D[p_][:, q_], M[p_][:, q_], f"perm {p} {q}")


def pin_extract_dense(ns, seeds=60):
    rng = np.random.default_rng(12)
    for s in range(seeds):
        m, n = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        A, D, M = rand_csr(ns, rng, m, n, 0.4, special=(s % 7 == 0))
        kI, kJ = int(rng.integers(0, 2 * m + 1)), int(rng.integers(0, 2 * n + 1))
        if s % 3 == 0:  # distinct, unsorted
            I = rng.permutation(m)[:min(kI, m)]
            J = rng.permutation(n)[:min(kJ, n)]
        else:           # repeats allowed (Sec. 2.2)
            I = rng.integers(0, m, kI)
            J = rng.integers(0, n, kJ)
        X = ns.extract(A, I, J)
        dense_eq(X, D[np.ix_(I, J)], M[np.ix_(I, J)], f"extract seed {s}")
        kc = ns.kept_counts(A, I, J)
        assert np.array_equal(kc, M[np.ix_(I, J)].sum(1)), f"kept counts seed {s}"


def pin_extract_scipy(ns, seeds=20):
    import scipy.sparse as sp
    rng = np.random.default_rng(13)
    for s in range(seeds):
        m, n = int(rng.integers(5, 60)), int(rng.integers(5, 60))
        A, D, M = rand_csr(ns, rng, m, n, 0.2)
        I = rng.integers(0, m, int(rng.integers(1, 2 * m)))
        J = rng.integers(0, n, int(rng.integers(1, 2 * n)))
        S = sp.csr_matrix((A.values, A.colidx, A.rowptr), shape=(m, n))
        T = S[I, :][:, J].tocsr()
        T.sort_indices()
        X = ns.extract(A, I, J)
        assert np.array_equal(X.rowptr, T.indptr), f"scipy rowptr seed {s}"
        assert np.array_equal(X.colidx, T.indices), f"scipy colidx seed {s}"
        assert np.array_equal(X.values, T.data), f"scipy values seed {s}"
        p, q = rng.permutation(m), rng.permutation(n)
        T = S[p, :][:, q].tocsr()
        T.sort_indices()
        X = ns.permute(A, p, q)
        assert np.array_equal(X.colidx, T.indices) and np.array_equal(X.values, T.data), \
            f"scipy permute seed {s}"


def pin_assign_dense(ns, seeds=60):
    rng = np.random.default_rng(14)
    for s in range(seeds):
        m, n = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        A, D, M = rand_csr(ns, rng, m, n, 0.4)
        kI, kJ = int(rng.integers(0, m + 1)), int(rng.integers(0, n + 1))
        I, J = rng.permutation(m)[:kI], rng.permutation(n)[:kJ]
        Bm, BD, BM = rand_csr(ns, rng, kI, kJ, 0.5)
        BD = BD + 100.0 * BM  # distinct from A's values
        Bm = ns.from_dense(BD, BM)
        for mode in (0, 1, 2):
            E, EM = D.copy(), M.copy()
            ix = np.ix_(I, J)
            if mode == 0:      # REPLACE: region cleared, then B written
                E[ix], EM[ix] = BD, BM
            elif mode == 1:    # SELECT2ND: B's stored entries overwrite, others survive
                sub, subm = E[ix], EM[ix]
                sub[BM] = BD[BM]
                subm |= BM
                E[ix], EM[ix] = sub, subm
            else:              # PLUS
                sub, subm = E[ix], EM[ix]
                sub[BM] = sub[BM] + BD[BM]
                subm |= BM
                E[ix], EM[ix] = sub, subm
            E[~EM] = 0
            dense_eq(ns.assign(A, I, J, Bm, mode), E, EM, f"assign seed {s} mode {mode}")


def pin_scan_closed_forms(ns):
    for k in (0, 1, 2, 7, 1000):
        assert np.array_equal(ns.exclusive_scan(np.ones(k, np.int64)), np.arange(k + 1)), \
            "exscan(ones)"
        got = ns.exclusive_scan(np.arange(k, dtype=np.int64))
        want = np.array([i * (i - 1) // 2 for i in range(k + 1)], dtype=np.int64)
        assert np.array_equal(got, want), "exscan(0..k-1) = i(i-1)/2"
    big = np.full(5, 2**40, np.int64)
    assert ns.exclusive_scan(big)[-1] == 5 * 2**40, "64-bit totals"


def pin_inverse_map(ns):
    rng = np.random.default_rng(15)
    for n in (1, 2, 9, 100):
        p = rng.permutation(n)
        inv = ns.inverse_map(p, n, require_permutation=True)
        assert np.array_equal(p[inv], np.arange(n)), "p[pinv[i]] = i"
        assert np.array_equal(inv[p], np.arange(n)), "pinv[p[k]] = k"
        sub = p[: n // 2]
        inv = ns.inverse_map(sub, n)
        assert np.all(inv[np.setdiff1d(np.arange(n), sub)] == -1), "absent -> -1"
        assert np.array_equal(inv[sub], np.arange(sub.shape[0])), "present -> position"


def pin_invariants(ns, seeds=20):
    rng = np.random.default_rng(16)
    for s in range(seeds):
        m, n = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        A, D, M = rand_csr(ns, rng, m, n, 0.25, special=(s % 4 == 0))
        same_csr(ns.permute(A, None, None), A, "identity permutation")
        same_csr(ns.permute(A, np.arange(m), np.arange(n)), A, "explicit identity")
        p, q = rng.permutation(m), rng.permutation(n)
        X = ns.permute(A, p, q)
        assert X.nnz == A.nnz, "nnz conserved"
        assert np.array_equal(np.sort(np.diff(X.rowptr)), np.sort(np.diff(A.rowptr))), \
            "row-length multiset"
        same_csr(ns.permute(X, np.argsort(p), np.argsort(q)), A, "p then p^-1")
        same_csr(ns.extract(A, np.arange(m), np.arange(n)), A, "extract all")
        same_csr(ns.extract(A, p, q), X, "permutation = extraction with full vectors")
        kI, kJ = int(rng.integers(0, m + 1)), int(rng.integers(0, n + 1))
        I, J = rng.permutation(m)[:kI], rng.permutation(n)[:kJ]
        B, _, _ = rand_csr(ns, rng, kI, kJ, 0.3)
        same_csr(ns.extract(ns.assign(A, I, J, B, 0), I, J), B, "extract after assign")


def pin_split_reassign(ns, seeds=10):
    """Streaming update (Sec. 6.3): 80 % base + four 5 % parts re-assigned give A back."""
    rng = np.random.default_rng(17)
    for s in range(seeds):
        m = int(rng.integers(5, 50))
        A, D, M = rand_csr(ns, rng, m, m, 0.3)
        part = rng.choice(5, size=A.nnz, p=[0.8, 0.05, 0.05, 0.05, 0.05])
        r, c, v = A.triplets()
        k0 = part == 0
        cur = ns.build_csr(m, m, r[k0], c[k0], v[k0])
        for k in range(1, 5):
            sel = part == k
            rows, cols = np.unique(r[sel]), np.unique(c[sel])
            Bk = ns.build_csr(rows.shape[0], cols.shape[0], np.searchsorted(rows, r[sel]),
                              np.searchsorted(cols, c[sel]), v[sel])
            cur = ns.assign(cur, rows, cols, Bk, 1)  # select-second union
        same_csr(cur, A, f"split/re-assign seed {s}")


def pin_rows(ns, seeds=10):
    rng = np.random.default_rng(18)
    for s in range(seeds):
        m, n = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        A, D, M = rand_csr(ns, rng, m, n, 0.3)
        p, q = rng.permutation(m), rng.permutation(n)
        X = ns.permute(A, p, q)
        qinv = np.argsort(q)
        for i in range(m):
            c, v = ns.permute_row(A, p, qinv, i)
            assert np.array_equal(c, X.row(i)[0]) and np.array_equal(v, X.row(i)[1]), "perm row"
        J = rng.permutation(n)[: int(rng.integers(0, n + 1))]
        I = rng.integers(0, m, int(rng.integers(0, 2 * m)))
        jmap = np.full(n, -1)
        jmap[J] = np.arange(J.shape[0])
        Y = ns.extract(A, I, J)
        for i in range(I.shape[0]):
            c, v = ns.extract_row(A, I, jmap, i)
            assert np.array_equal(c, Y.row(i)[0]) and np.array_equal(v, Y.row(i)[1]), "ext row"
        kI = int(rng.integers(0, m + 1))
        I = rng.permutation(m)[:kI]
        B, _, _ = rand_csr(ns, rng, kI, J.shape[0], 0.4)
        Z = ns.assign(A, I, J, B, 0)
        rowmap = np.full(m, -1)
        rowmap[I] = np.arange(kI)
        jset = np.zeros(n, bool)
        jset[J] = True
        for r in range(m):
            c, v = ns.assign_row(A, I, J, B, rowmap, jset, r)
            assert np.array_equal(c, Z.row(r)[0]) and np.array_equal(v, Z.row(r)[1]), "asg row"


ALL_PINS = [pin_permute_dense, pin_permute_exhaustive, pin_extract_dense, pin_extract_scipy,
            pin_assign_dense, pin_scan_closed_forms, pin_inverse_map, pin_invariants,
            pin_split_reassign, pin_rows]
