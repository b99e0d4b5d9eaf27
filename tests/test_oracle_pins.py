"""The oracle against its pins (dense brute force, exhaustive cases, scipy, closed forms,
invariants, the paper's worked example).  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    if pin is pins.pin_extract_scipy:
        pytest.importorskip("scipy")
    pin(oracle)


def test_worked_example_fig1b():
    """Fig. 1(b): B[1,1] = 7 lands at A'_new[pvec2[1], qvec2[1]] = A'_new[2,4] (1-based)."""
    g = json.load(open(os.path.join(GOLDEN, "worked_example_assign.json")))
    m, n = 5, 6
    rng = np.random.default_rng(3)
    D = np.zeros((m, n))
    M = rng.random((m, n)) < 0.3
    D[M] = rng.random(int(M.sum())) + 10
    A = oracle.from_dense(D, M)
    # pvec2/qvec2: the given first entries, the rest arbitrary distinct indices
    pvec2 = np.array([g["pvec2_0"], 3, 0])
    qvec2 = np.array([g["qvec2_0"], 0, 5])
    BD = np.zeros((3, 3))
    BM = np.zeros((3, 3), bool)
    BD[g["B_row"], g["B_col"]] = g["B_value"]
    BM[g["B_row"], g["B_col"]] = True
    BD[2, 1], BM[2, 1] = 3.0, True
    B = oracle.from_dense(BD, BM)
    for mode in (0, 1):
        X = oracle.assign(A, pvec2, qvec2, B, mode)
        cols, vals = X.row(g["expected_row"])
        k = np.nonzero(cols == g["expected_col"])[0]
        assert k.shape[0] == 1 and vals[k[0]] == g["B_value"]


@pytest.mark.parametrize("bad,kind", [
    (lambda: oracle.permute(oracle.CSR.of(2, 2, [0, 0, 0], [], np.zeros(0)), [0, 0], None),
     "not_permutation"),
    (lambda: oracle.permute(oracle.CSR.of(2, 2, [0, 0, 0], [], np.zeros(0)), [0, 2], None),
     "index_range"),
    (lambda: oracle.permute(oracle.CSR.of(2, 2, [0, 0, 0], [], np.zeros(0)), [0], None),
     "not_permutation"),
    (lambda: oracle.extract(oracle.CSR.of(2, 2, [0, 0, 0], [], np.zeros(0)), [5], [0]),
     "index_range"),
    (lambda: oracle.assign(oracle.CSR.of(2, 2, [0, 0, 0], [], np.zeros(0)), [1, 1], [0],
                           oracle.CSR.of(2, 1, [0, 0, 0], [], np.zeros(0))),
     "duplicate_index"),
    (lambda: oracle.assign(oracle.CSR.of(2, 2, [0, 0, 0], [], np.zeros(0)), [1], [0],
                           oracle.CSR.of(2, 1, [0, 0, 0], [], np.zeros(0))),
     "shape"),
])
def test_oracle_rejects(bad, kind):
    with pytest.raises(oracle.OracleError) as e:
        bad()
    assert e.value.kind == kind


def test_empty_cases():
    A = oracle.CSR.of(0, 0, [0], [], np.zeros(0))
    assert oracle.permute(A, [], []).nnz == 0
    A = oracle.CSR.of(3, 3, [0, 1, 2, 3], [0, 1, 2], np.array([1.0, 2.0, 3.0]))
    X = oracle.extract(A, [], [0, 1])
    assert X.nrows == 0 and X.ncols == 2 and X.nnz == 0
    X = oracle.extract(A, [0, 1], [])
    assert X.nrows == 2 and X.ncols == 0 and X.nnz == 0 and list(X.rowptr) == [0, 0, 0]
    X = oracle.assign(A, [], [], oracle.CSR.of(0, 0, [0], [], np.zeros(0)))
    pins.same_csr(X, A, "empty assign")


def test_canonical_check():
    oracle.canonical_check(oracle.CSR.of(2, 3, [0, 2, 3], [0, 2, 1], np.ones(3)))
    with pytest.raises(oracle.OracleError):
        oracle.canonical_check(oracle.CSR.of(2, 3, [0, 2, 3], [2, 0, 1], np.ones(3)))
    with pytest.raises(oracle.OracleError):
        oracle.canonical_check(oracle.CSR.of(2, 3, [0, 2, 3], [0, 0, 1], np.ones(3)))
