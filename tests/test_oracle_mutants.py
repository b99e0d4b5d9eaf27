"""Planted mistakes in copies of the oracle must each fail at least one pin.

Each mutant is a plausible slip (a dropped inverse, a transposed operand, a wrong
index, an off-by-one, a dropped term); the real oracle passes every pin
(test_oracle_pins.py), so a pin that also passed a mutant would prove nothing.
"""
import types

import numpy as np
import pytest

import oracle
import pins
from oracle import sparse_oracle as so


def ns_with(**over):
    ns = types.SimpleNamespace(**{k: getattr(so, k) for k in dir(so) if not k.startswith("__")})
    for k, v in over.items():
        setattr(ns, k, v)
    return ns


def permute_uses_p_not_pinv(A, p, q):
    m, n = A.nrows, A.ncols
    p = np.arange(m) if p is None else np.asarray(p)
    q = np.arange(n) if q is None else np.asarray(q)
    qinv = so.inverse_map(q, n, True)
    r, c, v = A.triplets()
    return so.build_csr(m, n, p[r], qinv[c], v)


def permute_swaps_p_q(A, p, q):
    return so.permute(A, q if q is None or len(q) == A.nrows else p,
                      p if p is None or len(p) == A.ncols else q) if A.nrows != A.ncols \
        else so.permute(A, q, p)


def permute_columns_untouched(A, p, q):
    return so.permute(A, p, None)


def extract_ignores_repeats(A, I, J):
    I = np.asarray(I)
    J = np.asarray(J)
    jmap = np.full(A.ncols, -1)
    jmap[J] = np.arange(J.shape[0])   # last occurrence wins: drops repeated columns
    rows, cols, vals = [], [], []
    for i, r in enumerate(I):
        c, v = A.row(int(r))
        k = jmap[c] >= 0
        rows.append(np.full(int(k.sum()), i))
        cols.append(jmap[c][k])
        vals.append(v[k])
    if not rows:
        return so.build_csr(0, J.shape[0], np.zeros(0, np.int64), np.zeros(0, np.int64),
                            A.values[:0])
    return so.build_csr(I.shape[0], J.shape[0], np.concatenate(rows), np.concatenate(cols),
                        np.concatenate(vals))


def extract_maps_cols_by_value(A, I, J):
    # uses the column's own index instead of its position in J
    X = so.extract(A, I, np.sort(np.asarray(J)))
    return X


def assign_no_region_clear(A, I, J, B, mode=0):
    return so.assign(A, I, J, B, 1 if mode == 0 else mode)


def assign_transposed_maps(A, I, J, B, mode=0):
    I = np.asarray(I)
    J = np.asarray(J)
    if A.nrows == A.ncols and I.shape[0] == J.shape[0]:
        return so.assign(A, J, I, B, mode)
    return so.assign(A, I, J, B, mode) if I.shape[0] == 0 else so.assign(
        A, I, J, so.build_csr(B.nrows, B.ncols, *B.triplets()[:1],
                              np.zeros(B.nnz, np.int64), B.values) if B.ncols else B, mode)


def assign_plus_as_replace(A, I, J, B, mode=0):
    return so.assign(A, I, J, B, 0 if mode == 2 else mode)


def exclusive_scan_inclusive(x):
    x = np.asarray(x, dtype=np.int64)
    out = np.zeros(x.shape[0] + 1, np.int64)
    out[:-1] = np.cumsum(x)
    out[-1] = out[-2] if x.shape[0] else 0
    return out


def build_csr_unsorted(nrows, ncols, r, c, v):
    order = np.argsort(r, kind="stable")
    r, c, v = r[order], c[order], v[order]
    counts = np.bincount(r, minlength=nrows) if r.shape[0] else np.zeros(nrows, np.int64)
    rowptr = np.zeros(nrows + 1, np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return so.CSR(nrows, ncols, rowptr, c.astype(np.int64), v)


def inverse_map_no_absent(idx, n, require_permutation=False):
    inv = so.inverse_map(idx, n, require_permutation)
    inv[inv < 0] = 0
    return inv


MUTANTS = {
    "permute: p used where pinv belongs": dict(permute=permute_uses_p_not_pinv),
    "permute: row and column vectors swapped": dict(permute=permute_swaps_p_q),
    "permute: columns not relabelled": dict(permute=permute_columns_untouched),
    "extract: repeated columns dropped": dict(extract=extract_ignores_repeats),
    "extract: columns in sorted order, not J's": dict(extract=extract_maps_cols_by_value),
    "assign: region not cleared under REPLACE": dict(assign=assign_no_region_clear),
    "assign: I and J exchanged": dict(assign=assign_transposed_maps),
    "assign: PLUS treated as overwrite": dict(assign=assign_plus_as_replace),
    "scan: inclusive instead of exclusive": dict(exclusive_scan=exclusive_scan_inclusive),
    "build: columns left unsorted": dict(build_csr=build_csr_unsorted),
    "inverse map: absent positions not -1": dict(inverse_map=inverse_map_no_absent),
}


def _rebind(ns):
    """Route the oracle's internal calls through the mutated namespace where it matters."""
    if ns.build_csr is not so.build_csr:
        orig = so.build_csr
        so.build_csr = ns.build_csr
        return lambda: setattr(so, "build_csr", orig)
    return lambda: None


@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_is_caught(name):
    ns = ns_with(**MUTANTS[name])
    undo = _rebind(ns)
    caught = []
    try:
        for pin in pins.ALL_PINS:
            try:
                pin(ns)
            except (AssertionError, so.OracleError, IndexError, ValueError):
                caught.append(pin.__name__)
    finally:
        undo()
    assert caught, f"no pin rejects the mutant '{name}'"


def test_real_oracle_passes_all_pins():
    for pin in pins.ALL_PINS:
        pin(oracle)
