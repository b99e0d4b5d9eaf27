"""Batched permutation (a host-only plan + one fill that runs the whole batch, validation
included, without synchronising) against the oracle, request by request, bit-exact; the
same results alone and in the batch; CUDA graph capture and replay of the whole batch;
host and device errors."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import to_dev, to_oracle

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


def _long_rows(value_dtype=np.float32, seed=5):
    """Rows of 0, 1, 512, 513, 1024, 1025 (either side of the tile limits), 4096, 4097
    (either side of the run limit) and 12000 entries, then short rows."""
    rng = np.random.default_rng(seed)
    n = 20000
    lens = [0, 1, 512, 513, 1024, 1025, 4096, 4097, 12000] + list(rng.integers(0, 40, 200))
    r = np.concatenate([np.full(L, i, np.int64) for i, L in enumerate(lens)])
    c = np.concatenate([np.sort(rng.choice(n, L, replace=False)) for L in lens]).astype(np.int64)
    v = rng.random(r.shape[0]).astype(value_dtype)
    return oracle.build_csr(len(lens), n, r, c, v)


def _mats(vkind="f32u01", cdt=torch.int32):
    ms = [synth.rmat_csr(s, 6, seed=s, symmetrize=True, value_kind=vkind, rowptr_dtype=torch.int64,
                         colidx_dtype=cdt) for s in (9, 11, 13)]
    ms.append(synth.er_csr(3000, 2500, 12, seed=3, value_kind=vkind, rowptr_dtype=torch.int64,
                           colidx_dtype=cdt))
    O = _long_rows(np.float32 if vkind.startswith("f32") else np.float64)
    ms.append(synth.CSRTensors(O.nrows, O.ncols, torch.from_numpy(O.rowptr),
                               torch.from_numpy(O.colidx).to(cdt), torch.from_numpy(O.values)))
    return ms


def _requests(ms, nreq, seed, idt=torch.int32):
    g = torch.Generator().manual_seed(seed)
    reqs = []
    for k in range(nreq):
        mi = k % len(ms) if k < len(ms) else int(torch.randint(0, len(ms), (1,), generator=g))
        m, n = ms[mi].nrows, ms[mi].ncols
        kind = k % 5  # both, rows only, columns only, neither, symmetric (square only)
        p = torch.randperm(m, generator=g).to(idt) if kind in (0, 1, 4) else None
        q = torch.randperm(n, generator=g).to(idt) if kind in (0, 2) else None
        if kind == 4 and m == n:
            q = p
        reqs.append((mi, p, q))
    return reqs


def _dev_reqs(reqs):
    out = []
    for mi, p, q in reqs:
        dp = p.cuda() if p is not None else None
        dq = (dp if q is p else q.cuda()) if q is not None else None
        out.append((mi, dp, dq))
    return out


def _check(out, offs, ms, reqs, what):
    rp = out.rowptr.cpu().numpy().astype(np.int64)
    ci = out.colidx.cpu().numpy()
    vv = out.values.cpu().numpy()
    wide = vv.dtype.itemsize == 8
    assert rp[-1] == sum(ms[mi].nnz for mi, _, _ in reqs), f"{what}: total"
    for k, (mi, p, q) in enumerate(reqs):
        r0, r1 = offs[k], offs[k + 1]
        want = oracle.permute(to_oracle(ms[mi]), None if p is None else p.numpy(),
                              None if q is None else q.numpy())
        assert np.array_equal(rp[r0:r1 + 1] - rp[r0], want.rowptr), f"{what}: request {k} rowptr"
        sl = slice(rp[r0], rp[r1])
        assert np.array_equal(ci[sl].astype(np.int64), want.colidx), f"{what}: request {k} colidx"
        bt = np.uint64 if wide else np.uint32
        assert np.array_equal(vv[sl].view(bt), want.values.view(bt)), f"{what}: request {k} values"


@pytest.mark.parametrize("types", ["i32/f32", "i64/f64"])
def test_pbatch_matches_oracle(ctx, types):
    if types == "i32/f32":
        ms, idt = _mats(), torch.int32
    else:
        ms, idt = _mats("f64um11", torch.int64), torch.int64
    dms = [to_dev(m) for m in ms]
    reqs = _requests(ms, 120, 1, idt)
    out, offs = ctx.sp_permute_batch(dms, _dev_reqs(reqs), rowptr_dtype=torch.int64)
    assert offs[-1] == sum(ms[mi].nrows for mi, _, _ in reqs)
    _check(out, offs, ms, reqs, f"batch {types}")


def test_pbatch_int32_rowptr_and_one_request(ctx):
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    reqs = _requests(ms, 7, 4)
    out, offs = ctx.sp_permute_batch(dms, _dev_reqs(reqs), rowptr_dtype=torch.int32)
    assert out.rowptr.dtype == torch.int32
    _check(out, offs, ms, reqs, "int32 rowptr")
    out, offs = ctx.sp_permute_batch(dms, _dev_reqs(reqs[4:5]))
    _check(out, offs, ms, reqs[4:5], "one request")


def test_pbatch_same_alone_and_in_the_mix(ctx):
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    reqs = _dev_reqs(_requests(ms, 25, 2))
    out, offs = ctx.sp_permute_batch(dms, reqs)
    for k, (mi, p, q) in enumerate(reqs):
        alone = ctx.sp_permute(dms[mi], p, q)
        r0, r1 = offs[k], offs[k + 1]
        base = int(out.rowptr[r0])
        assert torch.equal(alone.rowptr.to(torch.int64), out.rowptr[r0:r1 + 1] - base)
        assert torch.equal(alone.colidx, out.colidx[base:int(out.rowptr[r1])])
        assert torch.equal(alone.values.view(torch.int32), out.values[base:int(out.rowptr[r1])].view(torch.int32))


def test_pbatch_graph_replay(ctx):
    """The whole batch (maps, validation, row table, scan, fill, sort) in one graph; a
    replay after new permutations are copied into the same buffers gives their result."""
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    reqs = _requests(ms, 60, 3)
    dreqs = _dev_reqs(reqs)
    bt = ctx.permute_batch(dms, dreqs)
    out = bt.alloc(torch.int32)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.fill(out, s)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    ctx.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bt.fill(out, torch.cuda.current_stream())
    out.colidx.zero_()
    out.values.zero_()
    g.replay()
    torch.cuda.synchronize()
    ctx.sync()
    _check(out, bt.row_offsets(), ms, reqs, "graph replay")
    # new permutations in the captured buffers
    g2 = torch.Generator().manual_seed(99)
    new = []
    for (mi, p, q), (_, dp, dq) in zip(reqs, dreqs):
        np_ = torch.randperm(p.numel(), generator=g2).to(p.dtype) if p is not None else None
        nq = (np_ if q is p else torch.randperm(q.numel(), generator=g2).to(q.dtype)) if q is not None else None
        if dp is not None:
            dp.copy_(np_)
        if dq is not None and dq is not dp:
            dq.copy_(nq)
        new.append((mi, np_, nq))
    g.replay()
    torch.cuda.synchronize()
    ctx.sync()
    _check(out, bt.row_offsets(), ms, new, "replay with new permutations")
    bt.close()


def test_pbatch_errors(ctx):
    from paper_2509_20776_gb300 import SpError
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    m0, n0 = ms[0].nrows, ms[0].ncols
    good = torch.arange(m0, dtype=torch.int32).cuda()
    rep = good.clone()
    rep[3] = rep[4]  # a repeated row
    with pytest.raises(SpError) as e:
        ctx.sp_permute_batch(dms, [(1, None, None), (0, rep, None)])
    assert e.value.name == "SP_ERR_NOT_PERMUTATION"
    bad_q = torch.arange(n0, dtype=torch.int32).cuda()
    bad_q[7] = n0 + 5  # out of range
    with pytest.raises(SpError) as e:
        ctx.sp_permute_batch(dms, [(0, good, bad_q)])
    assert e.value.name == "SP_ERR_NOT_PERMUTATION"
    with pytest.raises(SpError) as e:
        ctx.sp_permute_batch(dms, [(9, None, None)])
    assert e.value.name == "SP_ERR_INVALID_ARG"
    with pytest.raises(ValueError):
        ctx.sp_permute_batch(dms, [(0, good[:-1], None)])
    # the context is usable after a device error, and an empty batch is fine
    out, offs = ctx.sp_permute_batch(dms, [(0, good, None)])
    _check(out, offs, ms, [(0, good.cpu(), None)], "after errors")
    out, offs = ctx.sp_permute_batch(dms, [])
    assert offs == [0] and out.nnz == 0
