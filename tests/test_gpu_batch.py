"""Batched extraction (one count + one capturable fill for thousands of requests) against
the oracle, request by request, bit-exact, with either identify (per-request rank maps,
or each request's J sorted and searched); the same results alone and in the batch; CUDA
graph capture and replay of the fill."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_same, to_dev, to_oracle

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


def _mats():
    ms = [synth.rmat_csr(s, 6, seed=s, symmetrize=True, value_kind="f32u01", rowptr_dtype=torch.int64,
                         colidx_dtype=torch.int32) for s in (9, 11, 13, 14)]
    ms.append(synth.er_csr(3000, 3000, 12, seed=3, value_kind="f32u01", rowptr_dtype=torch.int64,
                           colidx_dtype=torch.int32))
    return ms


def _requests(ms, nreq, seed):
    g = torch.Generator().manual_seed(seed)
    reqs = []
    for k in range(nreq):
        mi = int(torch.randint(0, len(ms), (1,), generator=g))
        m, n = ms[mi].nrows, ms[mi].ncols
        # sizes log-uniform, with the empty and single-index edge cases and |J| > 4096
        ki = int(min(m, round(2 ** (torch.rand(1, generator=g).item() * 12))))
        kj = int(min(n, round(2 ** (torch.rand(1, generator=g).item() * 13))))
        if k % 50 == 0:
            ki = 0
        if k % 50 == 1:
            kj = 0
        if k % 50 == 2:
            kj = min(n, 6000)
        I = torch.randint(0, m, (ki,), generator=g).to(torch.int32)
        J = torch.randperm(n, generator=g)[:kj].to(torch.int32)
        reqs.append((mi, I, J))
    return reqs


def _check(out, offs, ms, reqs, what):
    rp = out.rowptr.cpu().numpy().astype(np.int64)
    ci = out.colidx.cpu().numpy()
    vv = out.values.cpu().numpy()
    for k, (mi, I, J) in enumerate(reqs):
        r0, r1 = offs[k], offs[k + 1]
        want = oracle.extract(to_oracle(ms[mi]), I.numpy(), J.numpy())
        got_rp = rp[r0:r1 + 1] - rp[r0]
        assert np.array_equal(got_rp, want.rowptr), f"{what}: request {k} rowptr"
        sl = slice(rp[r0], rp[r1])
        assert np.array_equal(ci[sl].astype(np.int64), want.colidx), f"{what}: request {k} colidx"
        assert np.array_equal(vv[sl].view(np.uint32), want.values.view(np.uint32)), f"{what}: request {k} values"


@pytest.mark.parametrize("identify", [0, 1])
def test_batch_matches_oracle(ctx, identify):
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    reqs = _requests(ms, 300, 1)
    dreqs = [(mi, I.cuda(), J.cuda()) for mi, I, J in reqs]
    ctx.set_shapes(identify=identify)
    try:
        out, offs = ctx.sp_extract_batch(dms, dreqs)
    finally:
        ctx.set_shapes(identify=-1)
    _check(out, offs, ms, reqs, f"batch, identify {identify}")


def test_batch_same_alone_and_in_the_mix(ctx):
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    reqs = _requests(ms, 60, 2)
    dreqs = [(mi, I.cuda(), J.cuda()) for mi, I, J in reqs]
    out, offs = ctx.sp_extract_batch(dms, dreqs)
    for k, (mi, I, J) in enumerate(dreqs):
        if I.numel() == 0:
            continue
        alone = ctx.sp_extract(dms[mi], I, J)
        r0, r1 = offs[k], offs[k + 1]
        base = int(out.rowptr[r0])
        assert torch.equal(alone.rowptr.to(torch.int64), out.rowptr[r0:r1 + 1] - base)
        assert torch.equal(alone.colidx, out.colidx[base:int(out.rowptr[r1])])
        assert torch.equal(alone.values.view(torch.int32), out.values[base:int(out.rowptr[r1])].view(torch.int32))


def test_batch_graph_replay(ctx):
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    reqs = _requests(ms, 200, 3)
    dreqs = [(mi, I.cuda(), J.cuda()) for mi, I, J in reqs]
    bt = ctx.extract_batch(dms, dreqs)
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
    bt.close()


@pytest.mark.parametrize("identify", [0, 1])
def test_batch_errors(ctx, identify):
    from paper_2509_20776_gb300 import SpError
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    I = torch.tensor([0, 1], dtype=torch.int32).cuda()
    ctx.set_shapes(identify=identify)
    try:
        with pytest.raises(SpError) as e:
            ctx.sp_extract_batch(dms, [(0, I, torch.tensor([5, 7, 5], dtype=torch.int32).cuda())])
        assert e.value.name == "SP_ERR_DUPLICATE_INDEX"
        with pytest.raises(SpError) as e:
            ctx.sp_extract_batch(dms, [(0, I, torch.tensor([5, 1 << 20], dtype=torch.int32).cuda())])
        assert e.value.name == "SP_ERR_INDEX_RANGE"
        # the same J in two requests is fine (repeats are per request)
        J = torch.tensor([5, 7], dtype=torch.int32).cuda()
        out, offs = ctx.sp_extract_batch(dms, [(0, I, J), (0, I, J)])
        assert offs == [0, 2, 4]
    finally:
        ctx.set_shapes(identify=-1)
    with pytest.raises(SpError) as e:
        ctx.sp_extract_batch(dms, [(9, I, I)])
    assert e.value.name == "SP_ERR_INVALID_ARG"
    out, offs = ctx.sp_extract_batch(dms, [(1, I, torch.tensor([3], dtype=torch.int32).cuda())])
    assert offs == [0, 2]


@pytest.mark.parametrize("identify", [0, 1])
def test_batch_run_whole_graph(ctx, identify):
    """Count once, then the whole batch (identify, count, row pointer, fill, sort) from one
    CUDA graph; replayed after every request's I and J are shuffled in place (the same
    selections, so the same sizes), it gives the new inputs' results."""
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    reqs = _requests(ms, 150, 7)
    dreqs = [(mi, I.cuda(), J.cuda()) for mi, I, J in reqs]
    ctx.set_shapes(identify=identify)
    try:
        bt = ctx.extract_batch(dms, dreqs)
        out = bt.alloc(torch.int64)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            bt.run(out, s)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        ctx.sync()
        _check(out, bt.row_offsets(), ms, reqs, f"run, identify {identify}")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            bt.run(out, torch.cuda.current_stream())
        gen = torch.Generator().manual_seed(17)
        new = []
        for (mi, I, J), (_, dI, dJ) in zip(reqs, dreqs):
            I2 = I[torch.randperm(I.numel(), generator=gen)]
            J2 = J[torch.randperm(J.numel(), generator=gen)]
            dI.copy_(I2)
            dJ.copy_(J2)
            new.append((mi, I2, J2))
        out.colidx.zero_()
        out.values.zero_()
        out.rowptr.zero_()
        g.replay()
        torch.cuda.synchronize()
        ctx.sync()
        _check(out, bt.row_offsets(), ms, new, f"graph replay of the run, identify {identify}")
        bt.close()
    finally:
        ctx.set_shapes(identify=-1)


def test_batch_run_overflow_is_reported(ctx):
    """A run whose inputs now select more entries than the count found reports
    SP_ERR_OVERFLOW at the next sync, writes nothing outside the output, and the
    context stays usable."""
    from paper_2509_20776_gb300 import SpError
    ms = _mats()
    dms = [to_dev(m) for m in ms]
    A = ms[3]  # R-MAT scale 14: rows of very different lengths
    rl = A.rowptr[1:] - A.rowptr[:-1]
    light, heavy = int(torch.argmin(rl + (rl == 0) * 10**9)), int(torch.argmax(rl))
    I = torch.full((8,), light, dtype=torch.int32).cuda()
    J = torch.arange(A.ncols, dtype=torch.int32).cuda()
    bt = ctx.extract_batch(dms, [(3, I, J)])
    cap = bt.nnz
    out = bt.alloc(torch.int64)
    guard = torch.full((1024,), 7, dtype=torch.int32, device="cuda")  # a neighbour to watch
    I.fill_(heavy)
    bt.run(out)
    with pytest.raises(SpError) as e:
        ctx.sync()
    assert e.value.name == "SP_ERR_OVERFLOW"
    assert int(out.rowptr[-1]) == cap
    assert bool((guard == 7).all())
    bt.close()
    I.fill_(light)
    ref, offs = ctx.sp_extract_batch(dms, [(3, I, J)])
    assert ref.nnz == cap and offs == [0, 8]
