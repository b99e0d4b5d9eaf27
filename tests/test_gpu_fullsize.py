"""Full-size workloads on the GPU, checked against the oracle on sampled rows plus
properties that hold at any size (row pointer, canonical rows, nnz, round trips), and one
workload of 46 M entries compared whole.

The sampled rows always include the longest output rows (the hub rows that go through
the huge-row kernel), the first and last rows and a seeded random set.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_same, to_oracle

pytestmark = pytest.mark.gpu

NSAMPLE = 1500


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_20776_gb300 import build
    build.build()
    from paper_2509_20776_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def dev_csr(A):
    from paper_2509_20776_gb300 import CSR
    return CSR(A.nrows, A.ncols, A.rowptr, A.colidx, A.values)


def sample_rows(rowptr_dev, n, seed):
    L = (rowptr_dev[1:] - rowptr_dev[:-1])
    top = torch.topk(L, min(64, n)).indices.cpu().numpy()
    rnd = np.random.default_rng(seed).integers(0, n, NSAMPLE)
    return np.unique(np.concatenate([top, rnd, [0, n - 1]]))


def host_row(A, r, rp_host):
    s, e = int(rp_host[r]), int(rp_host[r + 1])
    return A.colidx[s:e].cpu().numpy().astype(np.int64), A.values[s:e].cpu().numpy()


def check_canonical(B):
    """Every row strictly ascending and in range (on the device)."""
    rp = B.rowptr.to(torch.int64)
    c = B.colidx.to(torch.int64)
    if c.numel() < 2:
        return
    rows = torch.repeat_interleave(torch.arange(B.nrows, device=c.device), rp[1:] - rp[:-1])
    same = rows[1:] == rows[:-1]
    assert not bool(torch.any(same & (c[1:] <= c[:-1]))), "row not strictly ascending"
    assert int(c.min()) >= 0 and int(c.max()) < B.ncols


class RowView:
    """oracle.CSR-like access to rows of a device matrix, fetched on demand."""

    def __init__(self, A):
        self.A = A
        self.rp = A.rowptr.cpu().numpy().astype(np.int64)
        self.nrows, self.ncols = A.nrows, A.ncols

    def row(self, r):
        return host_row(self.A, r, self.rp)


def test_cfg2_permute_scale25(ctx):
    A = synth.rmat_csr(25, 16, seed=0, symmetrize=True, value_kind="f32u01", device="cuda")
    n = A.nrows
    p = synth.random_permutation(n, 1, 0, device="cuda")
    pdeg = synth.degree_descending_permutation(A.rowptr)
    q = synth.random_permutation(n, 1, 1, device="cuda")
    Av = RowView(A)
    lens = np.diff(Av.rp)
    for name, pp, qq in (("random", p, p), ("degree", pdeg, pdeg), ("PAQt", p, q)):
        B = ctx.sp_permute(dev_csr(A), pp, qq)
        pn = pp.cpu().numpy()
        # row pointer: exclusive scan of the permuted row lengths
        want_rp = oracle.exclusive_scan(lens[pn])
        assert np.array_equal(B.rowptr.cpu().numpy(), want_rp), name
        check_canonical(B)
        qinv = oracle.inverse_map(qq.cpu().numpy(), n, require_permutation=True)
        Bv = RowView(B)
        for i in sample_rows(B.rowptr, n, 1):
            wc, wv = oracle.permute_row(Av, pn, qinv, int(i))
            gc, gv = Bv.row(int(i))
            assert np.array_equal(gc, wc), f"{name} row {i}"
            assert np.array_equal(gv.view(np.uint32), wv.view(np.uint32)), f"{name} row {i}"
        del B


def test_whole_arrays_rmat20(ctx):
    """Every output array compared whole with the oracle (not sampled rows) at a size whose
    paths are the scale paths: R-MAT scale 20, edge factor 24 (46 M entries), with a hub row
    of 84 K entries (taken first from the back of the key-range split's list), 1351 rows
    longer than 4096 entries (the split, beside the tile sort), runs of both run
    configurations, and the extraction of half the rows and columns."""
    A = synth.rmat_csr(20, 24, seed=3, symmetrize=True, value_kind="f32u01", device="cuda")
    n = A.nrows
    L = A.rowptr[1:] - A.rowptr[:-1]
    assert int(L.max()) >= 65536 and int((L > 4096).sum()) > 1000, "needs hub and split rows"
    Ao = to_oracle(A)
    p = synth.random_permutation(n, 3, 0, device="cuda")
    q = synth.random_permutation(n, 3, 1, device="cuda")
    B = ctx.sp_permute(dev_csr(A), p, q)
    assert_same(B, oracle.permute(Ao, p.cpu().numpy(), q.cpu().numpy()), "P A Q^T, scale 20")
    del B
    I = synth.random_subset(n, n // 2, 3, 2, device="cuda")
    J = synth.random_subset(n, n // 2, 3, 3, device="cuda")
    E = ctx.sp_extract(dev_csr(A), I, J)
    assert_same(E, oracle.extract(Ao, I.cpu().numpy(), J.cpu().numpy()), "A(I, J), scale 20")


def test_cfg3_extract_er_2pow26(ctx):
    n = 1 << 26
    A = synth.er_csr(n, n, 32, seed=0, value_kind="f32u01", device="cuda")
    Av = RowView(A)
    I = synth.random_subset(n, n // 2, 3, 1, device="cuda")
    J = synth.random_subset(n, n // 2, 3, 2, device="cuda")
    B = ctx.sp_extract(dev_csr(A), I, J)
    check_canonical(B)
    In = I.cpu().numpy()
    jmap = oracle.inverse_map(J.cpu().numpy(), n)
    Bv = RowView(B)
    for i in sample_rows(B.rowptr, n // 2, 2):
        wc, wv = oracle.extract_row(Av, In, jmap, int(i))
        gc, gv = Bv.row(int(i))
        assert np.array_equal(gc, wc) and np.array_equal(gv.view(np.uint32), wv.view(np.uint32)), i
    # kept counts of every row against the oracle's definition on the host
    jset = (jmap >= 0)
    kc = ctx.sp_kept_counts(dev_csr(A), I[:200000], J)
    want = np.array([int(jset[Av.row(int(r))[0]].sum()) for r in In[:2000]])
    assert np.array_equal(kc[:2000].cpu().numpy(), want)
    del B
    # contiguous block A(0:n/4, n/4:n/2): a CSR slice with shifted columns
    I2 = torch.arange(0, n // 4, dtype=torch.int32, device="cuda")
    J2 = torch.arange(n // 4, n // 2, dtype=torch.int32, device="cuda")
    B2 = ctx.sp_extract(dev_csr(A), I2, J2)
    check_canonical(B2)
    B2v = RowView(B2)
    rng = np.random.default_rng(4)
    for r in rng.integers(0, n // 4, 500):
        c, v = Av.row(int(r))
        k = (c >= n // 4) & (c < n // 2)
        gc, gv = B2v.row(int(r))
        assert np.array_equal(gc, c[k] - n // 4) and np.array_equal(gv.view(np.uint32),
                                                                    v[k].view(np.uint32))


def test_cfg3_extract_mesh(ctx):
    M = synth.mesh5_csr(4900, 4900, device="cuda")
    assert M.nnz == 120_030_400
    n = M.nrows
    I = synth.random_subset(n, n // 8, 5, 1, device="cuda")
    B = ctx.sp_extract(dev_csr(M), I, I)
    check_canonical(B)
    Mv = RowView(M)
    In = I.cpu().numpy()
    jmap = oracle.inverse_map(In, n)
    Bv = RowView(B)
    for i in sample_rows(B.rowptr, n // 8, 3):
        wc, wv = oracle.extract_row(Mv, In, jmap, int(i))
        gc, gv = Bv.row(int(i))
        assert np.array_equal(gc, wc) and np.array_equal(gv.view(np.uint64), wv.view(np.uint64))


@pytest.mark.parametrize("contiguous", [False, True])
def test_cfg4_assign_scale26(ctx, contiguous):
    A = synth.rmat_csr(26, 24, seed=0, symmetrize=False, value_kind="f32u01", device="cuda")
    n = A.nrows
    k = 1 << 22
    Bm = synth.er_csr(k, k, 8, seed=1, value_kind="f32u01", device="cuda")
    if contiguous:
        I = torch.arange(n // 3, n // 3 + k, dtype=torch.int32, device="cuda")
        J = torch.arange(n // 5, n // 5 + k, dtype=torch.int32, device="cuda")
    else:
        I = synth.random_subset(n, k, 4, 1, device="cuda")
        J = synth.random_subset(n, k, 4, 2, device="cuda")
    Ap = ctx.sp_assign(dev_csr(A), I, J, dev_csr(Bm))
    check_canonical(Ap)
    # extract-after-assign returns B bit-exactly (whole matrix, on the device)
    E = ctx.sp_extract(Ap, I, J)
    assert torch.equal(E.rowptr, Bm.rowptr) and torch.equal(E.colidx, Bm.colidx)
    assert torch.equal(E.values.view(torch.int32), Bm.values.view(torch.int32))
    del E
    In, Jn = I.cpu().numpy(), J.cpu().numpy()
    rowmap = oracle.inverse_map(In, n)
    jset = np.zeros(n, bool)
    jset[Jn] = True
    Av, Bv, Apv = RowView(A), RowView(Bm), RowView(Ap)
    rows = np.unique(np.concatenate([sample_rows(Ap.rowptr, n, 5), In[:300],
                                     np.arange(8)]))  # rows of I and the hub rows
    for r in rows:
        c, v = Av.row(int(r))
        i = int(rowmap[r])
        if i >= 0:
            keep = ~jset[c]
            cb, vb = Bv.row(i)
            cols = np.concatenate([c[keep], Jn[cb]])
            vals = np.concatenate([v[keep], vb])
            o = np.argsort(cols, kind="stable")
            c, v = cols[o], vals[o]
        gc, gv = Apv.row(int(r))
        assert np.array_equal(gc, c) and np.array_equal(gv.view(np.uint32), v.view(np.uint32)), r
