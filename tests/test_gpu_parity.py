"""CUDA path vs the oracle, bit-exact, through the C ABI (small and medium sizes).

Sizes span many tiles, the long-row and huge-row kernels (hub rows beyond the
shared-memory capacities) and ragged tails; values include -0.0 and NaN payloads.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_same, from_oracle, to_dev, to_oracle

pytestmark = pytest.mark.gpu


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


def er(n=4096, draws=8, seed=0, kind="f64um11", rp=torch.int32, ci=torch.int32, m=None):
    return synth.er_csr(m or n, n, draws, seed=seed, value_kind=kind, rowptr_dtype=rp,
                        colidx_dtype=ci)


def special_values(A):
    v = A.values.clone()
    if v.numel() >= 4:
        v[0] = -0.0
        v[1] = float("nan")
        if v.dtype == torch.float64:
            v[2:3] = torch.tensor([0x7FF8DEADBEEF0001], dtype=torch.int64).view(torch.float64)
        else:
            v[2:3] = torch.tensor([0x7FC0BEEF], dtype=torch.int32).view(torch.float32)
        v[3] = 0.0
    return synth.CSRTensors(A.nrows, A.ncols, A.rowptr, A.colidx, v)


# ---- config 1: the tiny workload ----------------------------------------------------
def test_cfg1a_permute(ctx):
    A = special_values(er())
    p = synth.random_permutation(4096, 1, 0)
    q = synth.random_permutation(4096, 1, 1)
    B = ctx.sp_permute(to_dev(A), p.cuda(), q.cuda())
    assert_same(B, oracle.permute(to_oracle(A), p.numpy(), q.numpy()), "cfg1a")


def test_cfg1b_extract(ctx):
    A = er()
    I = synth.random_subset(4096, 1024, 1, 2)
    J = synth.random_subset(4096, 1024, 1, 3)
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, oracle.extract(to_oracle(A), I.numpy(), J.numpy()), "cfg1b")


def test_cfg1c_assign(ctx):
    A = er()
    Bm = synth.er_csr(1024, 1024, 4, seed=5, value_kind="f64um11", rowptr_dtype=torch.int32)
    I = synth.random_subset(4096, 1024, 1, 4)
    J = synth.random_subset(4096, 1024, 1, 5)
    Ap = ctx.sp_assign(to_dev(A), I.cuda(), J.cuda(), to_dev(Bm))
    want = oracle.assign(to_oracle(A), I.numpy(), J.numpy(), to_oracle(Bm))
    assert_same(Ap, want, "cfg1c")
    # extract-after-assign returns B (REPLACE region semantics)
    E = ctx.sp_extract(Ap, I.cuda(), J.cuda())
    assert_same(E, to_oracle(Bm), "extract after assign")


# ---- permutation variants ------------------------------------------------------------
@pytest.mark.parametrize("mode", ["sym", "p_only", "q_only", "identity"])
def test_permute_variants(ctx, mode):
    A = er(2000, 7, seed=3)
    p = synth.random_permutation(2000, 3, 0).cuda()
    q = synth.random_permutation(2000, 3, 1).cuda()
    args = {"sym": (p, p), "p_only": (p, None), "q_only": (None, q), "identity": (None, None)}[mode]
    B = ctx.sp_permute(to_dev(A), *args)
    pa = None if args[0] is None else args[0].cpu().numpy()
    qa = None if args[1] is None else args[1].cpu().numpy()
    assert_same(B, oracle.permute(to_oracle(A), pa, qa), mode)


@pytest.mark.parametrize("rp,ci,ix,kind", [
    (torch.int64, torch.int32, torch.int32, "f32u01"),
    (torch.int64, torch.int64, torch.int64, "f64um11"),
    (torch.int32, torch.int64, torch.int32, "f32u01"),
    (torch.int32, torch.int32, torch.int64, "f64um11"),
])
def test_permute_types(ctx, rp, ci, ix, kind):
    A = er(3000, 9, seed=4, kind=kind, rp=rp, ci=ci)
    p = synth.random_permutation(3000, 4, 0, dtype=ix)
    q = synth.random_permutation(3000, 4, 1, dtype=ix)
    B = ctx.sp_permute(to_dev(A), p.cuda(), q.cuda(), rowptr_dtype=torch.int64)
    assert_same(B, oracle.permute(to_oracle(A), p.numpy(), q.numpy()), str(rp))
    assert B.colidx.dtype == ci


def test_rectangular_permute(ctx):
    A = synth.er_csr(700, 5000, 12, seed=9)
    p = synth.random_permutation(700, 9, 0)
    q = synth.random_permutation(5000, 9, 1)
    B = ctx.sp_permute(to_dev(A), p.cuda(), q.cuda())
    assert_same(B, oracle.permute(to_oracle(A), p.numpy(), q.numpy()), "rect")


def rmat(scale, ef=16, seed=0, kind="f32u01", sym=True):
    return synth.rmat_csr(scale, ef, seed=seed, symmetrize=sym, value_kind=kind)


@pytest.mark.parametrize("order", ["random", "degree"])
def test_rmat_permute_hubs(ctx, order):
    """Power-law rows: tiles, long rows and huge rows (> shared-memory capacity)."""
    A = rmat(16)
    lens = (A.rowptr[1:] - A.rowptr[:-1])
    assert int(lens.max()) > 8192, "needs rows beyond the long-row capacity"
    n = A.nrows
    p = synth.random_permutation(n, 7, 0) if order == "random" else \
        synth.degree_descending_permutation(A.rowptr)
    B = ctx.sp_permute(to_dev(A), p.cuda(), p.cuda())
    assert_same(B, oracle.permute(to_oracle(A), p.numpy(), p.numpy()), order)


def boundary_matrix(lengths, ncols, seed=0, kind="f32u01"):
    """Rows of the given lengths with random distinct columns (rows sorted)."""
    g = torch.Generator().manual_seed(seed)
    cols, counts = [], []
    for L in lengths:
        c = torch.randperm(ncols, generator=g)[:L]
        cols.append(torch.sort(c).values)
        counts.append(L)
    colidx = torch.cat(cols).to(torch.int32) if cols else torch.zeros(0, dtype=torch.int32)
    rowptr = torch.zeros(len(lengths) + 1, dtype=torch.int64)
    rowptr[1:] = torch.cumsum(torch.tensor(counts, dtype=torch.int64), 0)
    vals = synth.draw_values(colidx.numel(), seed, kind, "cpu")
    return synth.CSRTensors(len(lengths), ncols, rowptr, colidx, vals)


def test_row_length_boundaries(ctx):
    Ls = [0, 1, 2, 15, 16, 17, 31, 32, 33, 0, 0, 1023, 1024, 1025, 2047, 2048, 2049, 0, 4095,
          4096, 4097, 8191, 8192, 8193, 16384, 3, 0, 70000, 1, 5, 129, 128, 127, 511, 512, 513]
    A = boundary_matrix(Ls, 200000, seed=2)
    q = synth.random_permutation(200000, 2, 1)
    p = synth.random_permutation(len(Ls), 2, 0)
    B = ctx.sp_permute(to_dev(A), p.cuda(), q.cuda())
    assert_same(B, oracle.permute(to_oracle(A), p.numpy(), q.numpy()), "boundaries")


@pytest.mark.parametrize("overlap", [1, 0])
def test_split_list_both_ends(ctx, overlap):
    """Rows of 4097 .. 65535 entries are queued at the front of the key-range split's list,
    rows of 65536 and more at its back (taken first): several of each, through the
    permutation's partition and through the extraction's fill queue (J keeps every
    column, I repeats the hub rows).  Short rows make tiles, which the permutation sorts
    concurrently with the split (overlap 1) or after it (overlap 0)."""
    from paper_2509_20776_gb300 import SP_OPT_OVERLAP
    Ls = [65536, 5000, 0, 4097, 131072, 70001, 65535, 3, 9000, 65537, 40000, 1, 100000]
    L = boundary_matrix(Ls, 300000, seed=4)
    S = synth.er_csr(3000, 300000, 200, seed=9, value_kind="f32u01", rowptr_dtype=torch.int64)
    A = synth.CSRTensors(L.nrows + S.nrows, 300000, torch.cat([L.rowptr, S.rowptr[1:] + L.nnz]),
                         torch.cat([L.colidx, S.colidx.to(L.colidx.dtype)]), torch.cat([L.values, S.values]))
    q = synth.random_permutation(300000, 4, 1)
    p = synth.random_permutation(A.nrows, 4, 0)
    ctx.set_option(SP_OPT_OVERLAP, overlap)
    try:
        B = ctx.sp_permute(to_dev(A), p.cuda(), q.cuda())
        assert_same(B, oracle.permute(to_oracle(A), p.numpy(), q.numpy()), "split list")
        I = torch.tensor([4, 0, 1, 12, 4, 6, 9, 5, 10, 0, 20, 3000], dtype=torch.int32)
        B = ctx.sp_extract(to_dev(A), I.cuda(), q.cuda())
        assert_same(B, oracle.extract(to_oracle(A), I.numpy(), q.numpy()), "split list extract")
    finally:
        ctx.set_option(SP_OPT_OVERLAP, -1)


@pytest.mark.parametrize("n", [1 << 22, 1 << 24])
def test_skewed_keys_long_row(ctx, n):
    """Keys packed into a narrow range with outliers: heavy buckets in the row sort and,
    at 2^24 columns, a key-range bucket of the split holding more than 4096 entries (the
    second split round, over the bucket's own key range)."""
    L = 6000
    g = torch.Generator().manual_seed(5)
    dense = torch.randperm(5000, generator=g)[:L - 200]
    far = torch.randperm(n - 5000, generator=g)[:200] + 5000
    c = torch.sort(torch.cat([dense, far])).values.to(torch.int32)
    A = synth.CSRTensors(1, n, torch.tensor([0, c.numel()], dtype=torch.int64), c,
                         synth.draw_values(c.numel(), 1, "f32u01", "cpu"))
    q = synth.random_permutation(n, 5, 1)
    # identity-like q on the dense block keeps the skew in the new keys
    q[:5000] = torch.arange(5000, dtype=q.dtype)
    rest = torch.arange(5000, n, dtype=q.dtype)
    q[5000:] = rest[torch.randperm(n - 5000, generator=g)]
    B = ctx.sp_permute(to_dev(A), None, q.cuda())
    assert_same(B, oracle.permute(to_oracle(A), None, q.numpy()), "skew")


# ---- extraction ------------------------------------------------------------------------
def test_extract_repeated_rows_and_full(ctx):
    A = er(3000, 10, seed=6, kind="f32u01", rp=torch.int64)
    g = torch.Generator().manual_seed(1)
    I = torch.randint(0, 3000, (5000,), generator=g, dtype=torch.int32)
    J = synth.random_subset(3000, 1700, 6, 1)
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, oracle.extract(to_oracle(A), I.numpy(), J.numpy()), "repeat I")
    I = torch.arange(3000, dtype=torch.int32)
    J = torch.arange(3000, dtype=torch.int32)
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, to_oracle(A), "extract all")


def test_extract_empty(ctx):
    A = er(500, 5, seed=7)
    e = torch.zeros(0, dtype=torch.int32)
    J = synth.random_subset(500, 100, 7, 1)
    B = ctx.sp_extract(to_dev(A), e.cuda(), J.cuda())
    assert B.nrows == 0 and B.nnz == 0
    I = synth.random_subset(500, 50, 7, 2)
    B = ctx.sp_extract(to_dev(A), I.cuda(), e.cuda())
    assert B.nrows == 50 and B.ncols == 0 and B.nnz == 0
    assert torch.all(B.rowptr == 0)


def test_extract_hubs(ctx):
    A = rmat(15)
    n = A.nrows
    I = synth.random_subset(n, n // 2, 8, 1)
    J = synth.random_subset(n, n // 2, 8, 2)
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, oracle.extract(to_oracle(A), I.numpy(), J.numpy()), "extract rmat")
    kc = ctx.sp_kept_counts(to_dev(A), I.cuda(), J.cuda())
    assert np.array_equal(kc.cpu().numpy(), oracle.kept_counts(to_oracle(A), I.numpy(), J.numpy()))


@pytest.mark.parametrize("jorder", ["general", "ascending"])
def test_extract_lane_rows(ctx, jorder):
    """Rows of 0 .. 12 source entries around the fill's lane path (rows of at most 8
    entries filled and sorted by their own lane), every row selected twice, J keeping
    about half the columns; values include -0.0 and NaN payloads (moved bit for bit)."""
    g = torch.Generator().manual_seed(12)
    Ls = [int(x) for x in torch.randint(0, 13, (5000,), generator=g)]
    A = special_values(boundary_matrix(Ls, 4000, seed=12))
    I = torch.cat([torch.randperm(5000, generator=g), torch.randperm(5000, generator=g)])[:9000].to(torch.int32)
    J = synth.random_subset(4000, 2000, 12, 1)
    if jorder == "ascending":
        J = torch.sort(J).values
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, oracle.extract(to_oracle(A), I.numpy(), J.numpy()), f"lane rows, {jorder} J")


@pytest.mark.parametrize("shape", ["ascending", "consecutive", "consecutive_edge"])
def test_extract_ordered_j(ctx, shape):
    """Ascending J (rows come out of the fill in order, no sort) and consecutive J (binary
    search of each row's kept segment, affine relabel); R-MAT hubs give source rows far
    beyond one warp's share, and I repeats rows."""
    A = special_values(rmat(15))
    n = A.nrows
    g = torch.Generator().manual_seed(31)
    I = torch.randint(0, n, (n // 2,), generator=g).to(torch.int32)
    if shape == "ascending":
        J = torch.sort(synth.random_subset(n, n // 3, 9, 2)).values
    elif shape == "consecutive":
        J = torch.arange(n // 5, n // 5 + n // 3, dtype=torch.int32)
    else:  # the range touches column 0 and the last column
        J = torch.arange(0, n, dtype=torch.int32)
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, oracle.extract(to_oracle(A), I.numpy(), J.numpy()), f"extract {shape}")
    kc = ctx.sp_kept_counts(to_dev(A), I.cuda(), J.cuda())
    assert np.array_equal(kc.cpu().numpy(), oracle.kept_counts(to_oracle(A), I.numpy(), J.numpy()))


@pytest.mark.parametrize("size", ["small", "hubs"])
def test_extract_repeated_j(ctx, size):
    """J with repeats (more positions than columns): every position of a column gets a copy
    (Sec. 2.2 allows repeated indices); I repeats too."""
    A = special_values(er(3000, 8, seed=21) if size == "small" else rmat(14))
    n = A.ncols
    g = torch.Generator().manual_seed(22)
    I = torch.randint(0, A.nrows, (A.nrows // 2,), generator=g).to(torch.int32)
    J = torch.randint(0, n, (n + n // 3,), generator=g).to(torch.int32)
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, oracle.extract(to_oracle(A), I.numpy(), J.numpy()), f"extract repeated J {size}")
    kc = ctx.sp_kept_counts(to_dev(A), I.cuda(), J.cuda())
    assert np.array_equal(kc.cpu().numpy(), oracle.kept_counts(to_oracle(A), I.numpy(), J.numpy()))


def test_extract_consecutive_j_out_of_range(ctx):
    from paper_2509_20776_gb300 import SpError
    A = to_dev(er(100, 4, seed=1))
    J = torch.arange(90, 110, dtype=torch.int32).cuda()
    I = torch.arange(0, 10, dtype=torch.int32).cuda()
    with pytest.raises(SpError):
        ctx.sp_extract(A, I, J)
    ctx.sync()


def test_extract_long_sources_short_outputs(ctx):
    """Hub rows whose sources exceed the tile limit but keep few entries sit between
    ordinary rows of a tile (the tile must leave their output positions alone)."""
    A = rmat(15)
    n = A.nrows
    I = synth.random_permutation(n, 13, 0)
    J = synth.random_subset(n, n // 64, 13, 1)
    B = ctx.sp_extract(to_dev(A), I.cuda(), J.cuda())
    assert_same(B, oracle.extract(to_oracle(A), I.numpy(), J.numpy()), "long src, short out")
    Bm = synth.er_csr(n, n // 64, 2, seed=13)
    Ap = ctx.sp_assign(to_dev(A), I.cuda(), J.cuda(), to_dev(Bm))
    assert_same(Ap, oracle.assign(to_oracle(A), I.numpy(), J.numpy(), to_oracle(Bm)), "assign")
    E = ctx.sp_extract(Ap, I.cuda(), J.cuda())
    assert_same(E, to_oracle(Bm), "extract after assign")


def test_extract_mesh(ctx):
    M = synth.mesh5_csr(60, 70)
    n = M.nrows
    I = synth.random_subset(n, n // 8, 9, 1)
    B = ctx.sp_extract(to_dev(M), I.cuda(), I.cuda())
    assert_same(B, oracle.extract(to_oracle(M), I.numpy(), I.numpy()), "mesh")


# ---- assignment --------------------------------------------------------------------------
def test_assign_hubs_and_roundtrip(ctx):
    A = rmat(15, sym=False)
    n = A.nrows
    Bm = synth.er_csr(4096, 4096, 8, seed=3)
    # the first 8 rows (the R-MAT hubs) plus 4088 random others, in random order
    rest = synth.random_subset(n - 8, 4088, 3, 1) + 8
    I = torch.cat([torch.arange(8, dtype=rest.dtype), rest])
    I = I[torch.randperm(4096, generator=torch.Generator().manual_seed(3))]
    J = synth.random_subset(n, 4096, 3, 2)
    Ap = ctx.sp_assign(to_dev(A), I.cuda(), J.cuda(), to_dev(Bm))
    assert_same(Ap, oracle.assign(to_oracle(A), I.numpy(), J.numpy(), to_oracle(Bm)), "assign")
    E = ctx.sp_extract(Ap, I.cuda(), J.cuda())
    assert_same(E, to_oracle(Bm), "extract after assign")


@pytest.mark.parametrize("longest,overlap", [(32, 1), (32, 0), (33, 1)])
def test_assign_merge_boundaries(ctx, longest, overlap):
    """REPLACE with every row of B at most 32 entries takes the merge fill (A's surviving
    run and B's relabelled row merged in order straight into A', no row sort, while the
    copy of the other rows runs beside it (overlap 1) or before it); one row of 33 takes
    the staged fill and the row sort.  Rows of B of 0, 1, 31 and the longest length, hub
    rows of A on both kernels of the merge (warp and CTA), keys before, between and after
    A's; rows of I next to each other and alone, so copy segments of every length lie
    between the merged rows."""
    from paper_2509_20776_gb300 import SP_OPT_OVERLAP
    A = rmat(14)
    n = A.nrows
    rng = np.random.default_rng(longest)
    rest = synth.random_subset(n - 16, 1500, 5, 1) + 16
    I = torch.cat([torch.arange(16, dtype=rest.dtype), rest])
    I = I[torch.randperm(I.numel(), generator=torch.Generator().manual_seed(5))]
    nJ = 3000
    J = synth.random_subset(n, nJ, 5, 2)
    lens = rng.choice([0, 1, 31, 32], size=I.numel())
    lens[rng.integers(0, I.numel())] = longest
    r = np.repeat(np.arange(I.numel()), lens)
    c = np.concatenate([np.sort(rng.choice(nJ, L, replace=False)) for L in lens]).astype(np.int64)
    v = rng.random(r.shape[0]).astype(np.float32)
    Bo = oracle.build_csr(I.numel(), nJ, r, c, v)
    Bd = from_oracle(Bo)
    ctx.set_option(SP_OPT_OVERLAP, overlap)
    try:
        Ap = ctx.sp_assign(to_dev(A), I.cuda(), J.cuda(), Bd)
    finally:
        ctx.set_option(SP_OPT_OVERLAP, -1)
    assert_same(Ap, oracle.assign(to_oracle(A), I.numpy(), J.numpy(), Bo), f"assign, longest B row {longest}")
    E = ctx.sp_extract(Ap, I.cuda(), J.cuda())
    assert_same(E, Bo, "extract after assign")


def _union_b(A, I, J, seed, kind):
    """B of |I| x |J|: every entry of A(I, J) with a fresh value, plus random others, so
    the union modes meet both B entries that hit A and B entries that do not."""
    E = oracle.extract(to_oracle(A), I.numpy(), J.numpy())
    er_, ec, _ = E.triplets()
    rng = np.random.default_rng(seed)
    nI, nJ = len(I), len(J)
    rr = rng.integers(0, nI, size=nI * 6)
    rc = rng.integers(0, nJ, size=nI * 6)
    rows = np.concatenate([er_, rr])
    cols = np.concatenate([ec, rc])
    key = np.unique(rows * nJ + cols)
    rows, cols = key // nJ, key % nJ
    dt = np.float32 if kind == "f32" else np.float64
    vals = rng.uniform(-1, 1, size=key.size).astype(dt)
    return oracle.build_csr(nI, nJ, rows, cols, vals)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("kind", ["f32", "f64"])
def test_assign_union_modes(ctx, mode, kind):
    """SELECT2ND (1) and PLUS (2): A (+) P B Q^T; hub rows of A give source-long rows."""
    A = rmat(14, sym=False, kind="f32u01" if kind == "f32" else "f64um11")
    n = A.nrows
    I = torch.cat([torch.arange(4, dtype=torch.int32), synth.random_subset(n - 4, 1500, 4, 1) + 4])
    J = synth.random_subset(n, n // 2, 4, 2)
    Bo = _union_b(A, I, J, 5, kind)
    Bd = from_oracle(Bo, rowptr_dtype=torch.int32, colidx_dtype=A.colidx.dtype)
    Ap = ctx.sp_assign(to_dev(A), I.cuda(), J.cuda(), Bd, mode=mode)
    assert_same(Ap, oracle.assign(to_oracle(A), I.numpy(), J.numpy(), Bo, mode), f"assign mode {mode}")


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("perm", ["sym", "pq", "rows_only"])
def test_assign_permute_fused(ctx, mode, perm):
    """out = P (A (+) B') Q^T in one pass equals the oracle's assign followed by permute."""
    A = rmat(14, sym=False)
    n = A.nrows
    I = torch.cat([torch.arange(4, dtype=torch.int32), synth.random_subset(n - 4, 1500, 6, 1) + 4])
    J = synth.random_subset(n, n // 2, 6, 2)
    Bo = _union_b(A, I, J, 7, "f32")
    Bd = from_oracle(Bo, rowptr_dtype=torch.int32, colidx_dtype=A.colidx.dtype)
    p = synth.random_permutation(n, 6, 0)
    q = p if perm == "sym" else (synth.random_permutation(n, 6, 1) if perm == "pq" else None)
    pd = p.cuda()
    qd = pd if perm == "sym" else (q.cuda() if q is not None else None)  # same tensor: P A' P^T
    got = ctx.sp_assign_permute(to_dev(A), I.cuda(), J.cuda(), Bd, pd, qd, mode=mode)
    Ao = oracle.assign(to_oracle(A), I.numpy(), J.numpy(), Bo, mode)
    want = oracle.permute(Ao, p.numpy(), None if q is None else q.numpy())
    assert_same(got, want, f"fused mode {mode} {perm}")


def test_assign_contiguous(ctx):
    A = er(3000, 8, seed=8, kind="f32u01", rp=torch.int64)
    Bm = synth.er_csr(300, 400, 6, seed=9)
    I = torch.arange(1000, 1300, dtype=torch.int32)
    J = torch.arange(2000, 2400, dtype=torch.int32)
    Ap = ctx.sp_assign(to_dev(A), I.cuda(), J.cuda(), to_dev(Bm))
    assert_same(Ap, oracle.assign(to_oracle(A), I.numpy(), J.numpy(), to_oracle(Bm)), "contig")


def test_split_reassign_replace_disjoint(ctx):
    """Streaming update (Sec. 6.3) with disjoint row blocks: parts re-assigned give A."""
    A = er(2000, 6, seed=10, kind="f32u01", rp=torch.int64)
    O = to_oracle(A)
    cur = from_oracle(oracle.assign(O, np.arange(0, 400), np.arange(2000),
                                    oracle.CSR.of(400, 2000, np.zeros(401, np.int64), [],
                                                  np.zeros(0, np.float32))))
    for r0 in range(0, 400, 100):
        I = np.arange(r0, r0 + 100)
        J = np.arange(2000)
        part = oracle.extract(O, I, J)
        cur = ctx.sp_assign(cur, torch.from_numpy(I).int().cuda(), torch.from_numpy(J).int().cuda(),
                            from_oracle(part))
    assert_same(cur, O, "split/re-assign")


# ---- steps on their own -------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 4097, 1 << 20, 3_000_001])
def test_scan(ctx, n):
    g = torch.Generator().manual_seed(n)
    x = torch.randint(0, 50, (n,), generator=g, dtype=torch.int32)
    out = ctx.sp_exclusive_scan(x.cuda())
    assert np.array_equal(out.cpu().numpy(), oracle.exclusive_scan(x.numpy()))


def test_scan_int64_large_values(ctx):
    x = torch.full((100000,), 1 << 40, dtype=torch.int64)
    out = ctx.sp_exclusive_scan(x.cuda())
    assert int(out[-1]) == 100000 << 40


def test_scan_timeout_hook(ctx):
    """A tile that never publishes: successors give up with SP_ERR_TIMEOUT, no hang."""
    from paper_2509_20776_gb300 import SP_OPT_SCAN_HOLD_TILE, SP_OPT_SPIN_LIMIT, SpError
    x = torch.ones(4096 * 8, dtype=torch.int32).cuda()
    ctx.set_option(SP_OPT_SPIN_LIMIT, 2000)
    ctx.set_option(SP_OPT_SCAN_HOLD_TILE, 1)
    try:
        with pytest.raises(SpError) as e:
            ctx.sp_exclusive_scan(x)
        assert e.value.name == "SP_ERR_TIMEOUT"
    finally:
        ctx.set_option(SP_OPT_SCAN_HOLD_TILE, -1)
        ctx.set_option(SP_OPT_SPIN_LIMIT, -1)
    out = ctx.sp_exclusive_scan(x)  # the context still works
    assert np.array_equal(out.cpu().numpy(), np.arange(x.numel() + 1))


def test_inverse_map(ctx):
    p = synth.random_permutation(100000, 11, 0)
    inv = ctx.sp_inverse_map(p.cuda(), 100000, True)
    assert np.array_equal(inv.cpu().numpy(), oracle.inverse_map(p.numpy(), 100000, True))
    sub = synth.random_subset(100000, 777, 11, 1, dtype=torch.int64)
    inv = ctx.sp_inverse_map(sub.cuda(), 100000)
    assert np.array_equal(inv.cpu().numpy(), oracle.inverse_map(sub.numpy(), 100000))


def test_sort_rows(ctx):
    """Rows with shuffled columns (incl. a 2-round huge row: keys need > 27 bits)."""
    Ls = [0, 3, 40, 5000, 9000, 30000, 7, 0, 1]
    n = 1 << 30
    g = torch.Generator().manual_seed(12)
    cols = [torch.unique(torch.randint(0, n, (L * 2 + 8,), generator=g))[:L] for L in Ls]
    cols = [c[torch.randperm(c.numel(), generator=g)] for c in cols]
    counts = [c.numel() for c in cols]
    colidx = torch.cat(cols).to(torch.int32)
    rowptr = torch.zeros(len(Ls) + 1, dtype=torch.int64)
    rowptr[1:] = torch.cumsum(torch.tensor(counts), 0)
    vals = synth.draw_values(colidx.numel(), 12, "f64um11", "cpu")
    M = synth.CSRTensors(len(Ls), n, rowptr, colidx, vals)
    D = to_dev(M)
    ctx.sp_sort_rows(D)
    O = to_oracle(M)
    r, c, v = O.triplets()
    assert_same(D, oracle.build_csr(O.nrows, O.ncols, r, c, v), "sort rows")


# ---- errors -------------------------------------------------------------------------------
def test_errors(ctx):
    from paper_2509_20776_gb300 import SpError
    A = to_dev(er(100, 4, seed=1))
    bad = torch.arange(100, dtype=torch.int32).cuda()
    bad[5] = 7
    with pytest.raises(SpError) as e:
        ctx.sp_permute(A, bad, None)
    assert e.value.name == "SP_ERR_NOT_PERMUTATION"
    with pytest.raises(SpError) as e:  # the same repeat in the column permutation
        ctx.sp_permute(A, None, bad)
    assert e.value.name == "SP_ERR_NOT_PERMUTATION"
    with pytest.raises(SpError) as e:  # and in both (the symmetric form builds one map)
        ctx.sp_permute(A, bad, bad)
    assert e.value.name == "SP_ERR_NOT_PERMUTATION"
    oob = torch.arange(100, dtype=torch.int32).cuda()
    oob[3] = 1000
    with pytest.raises(SpError) as e:
        ctx.sp_permute(A, None, oob)
    assert e.value.name == "SP_ERR_INDEX_RANGE"
    with pytest.raises(SpError) as e:  # assignment needs distinct J (extraction allows repeats)
        ctx.sp_assign(A, torch.tensor([0, 1], dtype=torch.int32).cuda(),
                      torch.tensor([3, 3], dtype=torch.int32).cuda(), to_dev(er(2, 2, seed=1)))
    assert e.value.name == "SP_ERR_DUPLICATE_INDEX"
    with pytest.raises(SpError) as e:  # and distinct I
        ctx.sp_assign(A, torch.tensor([4, 4], dtype=torch.int32).cuda(),
                      torch.tensor([3, 5], dtype=torch.int32).cuda(), to_dev(er(2, 2, seed=1)))
    assert e.value.name == "SP_ERR_DUPLICATE_INDEX"
    with pytest.raises(SpError) as e:  # the fused assignment + permutation checks q the same way
        ctx.sp_assign_permute(A, torch.tensor([0, 1], dtype=torch.int32).cuda(),
                              torch.tensor([3, 5], dtype=torch.int32).cuda(), to_dev(er(2, 2, seed=1)), q=bad)
    assert e.value.name == "SP_ERR_NOT_PERMUTATION"
    with pytest.raises(SpError) as e:
        ctx.sp_extract(A, torch.tensor([0, 100], dtype=torch.int32).cuda(),
                       torch.tensor([3], dtype=torch.int32).cuda())
    assert e.value.name == "SP_ERR_INDEX_RANGE"
    Bm = to_dev(synth.er_csr(3, 3, 2, seed=1))
    with pytest.raises(SpError) as e:
        ctx.sp_assign(A, torch.tensor([0, 1], dtype=torch.int32).cuda(),
                      torch.tensor([0, 1, 2], dtype=torch.int32).cuda(), Bm)
    assert e.value.name == "SP_ERR_SHAPE"
    # the context is still usable
    p = synth.random_permutation(100, 1, 0).cuda()
    B = ctx.sp_permute(A, p, p)
    assert B.nnz == A.nnz


def test_validate(ctx):
    from paper_2509_20776_gb300 import SpError
    A = er(200, 5, seed=2)
    ctx.sp_csr_validate(to_dev(A))
    bad = to_dev(A)
    bad.colidx[3], bad.colidx[4] = bad.colidx[4].clone(), bad.colidx[3].clone()
    with pytest.raises(SpError) as e:
        ctx.sp_csr_validate(bad)
    assert e.value.name == "SP_ERR_NOT_CANONICAL"


def test_deterministic(ctx):
    A = rmat(14)
    p = synth.random_permutation(A.nrows, 1, 0).cuda()
    B1 = ctx.sp_permute(to_dev(A), p, p)
    B2 = ctx.sp_permute(to_dev(A), p, p)
    assert torch.equal(B1.colidx, B2.colidx) and torch.equal(B1.values.view(torch.int32),
                                                             B2.values.view(torch.int32))
