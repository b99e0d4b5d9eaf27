"""Run-time kernel shapes and the autotuner: every shape gives the oracle's output bit for
bit (permutation with hub rows and skewed keys, extraction, batched extraction), a
tuning table installs and is applied per call, and the tuner picks valid shapes."""
import json

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
    c.set_tuning(None)
    c.set_shapes(tile_shape=-1, heavy=-1, count_rows=-1, fill_rows=-1, batch_rows=-1, identify=-1)
    c.close()


@pytest.fixture(scope="module")
def rmat():
    # hub rows above 1024 and 4096 entries, and many rows in (512, 1024]: both tile shapes
    # and the run sort see work
    return synth.rmat_csr(16, 16, seed=4, symmetrize=True, value_kind="f32u01", rowptr_dtype=torch.int64,
                          colidx_dtype=torch.int32)


_want = {}


@pytest.mark.parametrize("tile_shape,heavy", [(0, 128), (1, 128), (0, 512), (1, 4096)])
@pytest.mark.parametrize("order", ["random", "degree"])
def test_permute_every_shape(ctx, rmat, tile_shape, heavy, order):
    n = rmat.nrows
    p = synth.random_permutation(n, 7, 0) if order == "random" else synth.degree_descending_permutation(rmat.rowptr)
    if order not in _want:
        _want[order] = oracle.permute(to_oracle(rmat), p.numpy(), p.numpy())
    ctx.set_shapes(tile_shape=tile_shape, heavy=heavy)
    try:
        B = ctx.sp_permute(to_dev(rmat), p.cuda(), p.cuda())
    finally:
        ctx.set_shapes(tile_shape=-1, heavy=-1)
    assert_same(B, _want[order], f"shape {tile_shape}/{heavy} {order}")


@pytest.mark.parametrize("identify", [0, 1])
@pytest.mark.parametrize("jorder", ["random", "ascending"])
def test_extract_every_identify(ctx, rmat, identify, jorder):
    """Both identifies (rank map, sorted-J binary search), with general and ascending J
    (the fill that needs no sort), on a matrix with hub rows (the queued row sorts and
    the CTA-per-row count / fill)."""
    n = rmat.nrows
    g = torch.Generator().manual_seed(11)
    I = torch.randint(0, n, (n // 3,), generator=g).to(torch.int32)  # repeats allowed
    J = torch.randperm(n, generator=g)[: n // 2].to(torch.int32)
    if jorder == "ascending":
        J = torch.sort(J).values
    ctx.set_shapes(identify=identify, tile_shape=identify)
    try:
        B = ctx.sp_extract(to_dev(rmat), I.cuda(), J.cuda())
    finally:
        ctx.set_shapes(identify=-1, tile_shape=-1)
    assert_same(B, oracle.extract(to_oracle(rmat), I.numpy(), J.numpy()), f"identify {identify} {jorder}")


@pytest.mark.parametrize("count_rows,fill_rows", [(1, 1), (2, 2), (3, 1), (4, 2)])
def test_assign_every_rows_per_warp(ctx, rmat, count_rows, fill_rows):
    n = rmat.nrows
    g = torch.Generator().manual_seed(12)
    I = torch.randperm(n, generator=g)[: n // 4].to(torch.int32)
    J = torch.randperm(n, generator=g)[: n // 4].to(torch.int32)
    Bm = synth.er_csr(n // 4, n // 4, 6, seed=13, value_kind="f32u01", rowptr_dtype=torch.int64,
                      colidx_dtype=torch.int32)
    ctx.set_shapes(count_rows=count_rows, fill_rows=fill_rows, tile_shape=count_rows % 2)
    try:
        Ap = ctx.sp_assign(to_dev(rmat), I.cuda(), J.cuda(), to_dev(Bm))
    finally:
        ctx.set_shapes(count_rows=-1, fill_rows=-1, tile_shape=-1)
    want = oracle.assign(to_oracle(rmat), I.numpy(), J.numpy(), to_oracle(Bm))
    assert_same(Ap, want, f"rows {count_rows}/{fill_rows}")


def _batch(n_req, seed):
    ms = [synth.rmat_csr(s, 6, seed=s, symmetrize=True, value_kind="f32u01", rowptr_dtype=torch.int64,
                         colidx_dtype=torch.int32) for s in (9, 12, 14)]
    g = torch.Generator().manual_seed(seed)
    reqs = []
    for k in range(n_req):
        mi = int(torch.randint(0, len(ms), (1,), generator=g))
        m = ms[mi].nrows
        ki = int(min(m, round(2 ** (torch.rand(1, generator=g).item() * 11))))
        kj = int(min(m, round(2 ** (torch.rand(1, generator=g).item() * 12))))
        reqs.append((mi, torch.randint(0, m, (ki,), generator=g).to(torch.int32),
                     torch.randperm(m, generator=g)[:kj].to(torch.int32)))
    return ms, reqs


@pytest.mark.parametrize("batch_rows", [1, 2, 4, 8])
def test_batch_every_rows_per_warp(ctx, batch_rows):
    ms, reqs = _batch(120, 5)
    dms = [to_dev(m) for m in ms]
    dreqs = [(mi, I.cuda(), J.cuda()) for mi, I, J in reqs]
    ctx.set_shapes(batch_rows=batch_rows)
    try:
        out, offs = ctx.sp_extract_batch(dms, dreqs)
    finally:
        ctx.set_shapes(batch_rows=-1)
    rp = out.rowptr.cpu().numpy().astype(np.int64)
    ci = out.colidx.cpu().numpy()
    vv = out.values.cpu().numpy()
    for k, (mi, I, J) in enumerate(reqs):
        want = oracle.extract(to_oracle(ms[mi]), I.numpy(), J.numpy())
        r0, r1 = offs[k], offs[k + 1]
        assert np.array_equal(rp[r0:r1 + 1] - rp[r0], want.rowptr), f"rows/warp {batch_rows}: request {k}"
        sl = slice(rp[r0], rp[r1])
        assert np.array_equal(ci[sl].astype(np.int64), want.colidx), f"rows/warp {batch_rows}: request {k}"
        assert np.array_equal(vv[sl].view(np.uint32), want.values.view(np.uint32))


def test_tuning_table_per_call(ctx, rmat):
    """A table with different shapes per size class: small and large calls each take
    their entry, results stay exact; invalid tables are refused."""
    from paper_2509_20776_gb300 import SpError
    table = {"format": "sp-tuning-1", "entries": [
        {"op": "permute", "size_max": 10_000, "tile_shape": 1, "heavy": 256},
        {"op": "permute", "size_max": 1 << 62, "tile_shape": 0, "heavy": 512},
        {"op": "extract", "size_max": 10_000, "identify": 1},
        {"op": "extract", "size_max": 1 << 62, "identify": 0, "tile_shape": 1},
        {"op": "batch", "size_max": 1 << 62, "batch_rows": 4}]}
    ctx.set_tuning(table)
    try:
        small = synth.er_csr(300, 300, 8, seed=2, value_kind="f64um11", rowptr_dtype=torch.int32)
        for A, seed in ((small, 1), (rmat, 2)):
            p = synth.random_permutation(A.nrows, seed, 0)
            B = ctx.sp_permute(to_dev(A), p.cuda(), p.cuda())
            assert_same(B, oracle.permute(to_oracle(A), p.numpy(), p.numpy()), "tuned permute")
        I = torch.arange(0, rmat.nrows, 3, dtype=torch.int32)
        B = ctx.sp_extract(to_dev(rmat), I.cuda(), I.cuda())
        assert_same(B, oracle.extract(to_oracle(rmat), I.numpy(), I.numpy()), "tuned extract")
        Is = torch.randperm(300, generator=torch.Generator().manual_seed(4))[:100].to(torch.int32)
        B = ctx.sp_extract(to_dev(small), Is.cuda(), Is.flip(0).contiguous().cuda())
        assert_same(B, oracle.extract(to_oracle(small), Is.numpy(), Is.flip(0).numpy()), "tuned small extract")
    finally:
        ctx.set_tuning(None)
    with pytest.raises(ValueError):
        ctx.set_tuning([{"op": "permute", "size_max": 1, "batch_rows": 3}])
    with pytest.raises(SpError) as e:
        ctx.set_option(5, 64)  # heavy threshold below the smallest allowed
    assert e.value.name == "SP_ERR_INVALID_ARG"


def test_autotune_small(ctx, rmat, tmp_path):
    from paper_2509_20776_gb300 import autotune
    from paper_2509_20776_gb300._binding import CSR
    A = to_dev(rmat)
    p = synth.random_permutation(rmat.nrows, 3, 0).cuda()
    ms, reqs = _batch(60, 9)
    dms = [to_dev(m) for m in ms]
    dreqs = [(mi, I.cuda(), J.cuda()) for mi, I, J in reqs]

    def run_batch():
        out, _ = ctx.sp_extract_batch(dms, dreqs)
        return out

    table = autotune.autotune(ctx, [("permute", 1 << 62, lambda: ctx.sp_permute(A, p, p)),
                                    ("batch", 1 << 62, run_batch)], reps=1)
    path = str(tmp_path / "t.json")
    autotune.save(table, path)
    loaded = autotune.load(path)
    assert loaded["entries"] == json.loads(json.dumps(table["entries"]))
    assert {e["op"] for e in loaded["entries"]} == {"permute", "batch"}
    ctx.set_tuning(path)
    try:
        B = ctx.sp_permute(A, p, p)
        pn = p.cpu().numpy()
        assert_same(B, oracle.permute(to_oracle(rmat), pn, pn), "after autotune")
    finally:
        ctx.set_tuning(None)
