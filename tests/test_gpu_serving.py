"""The request server: every result of a mixed permute / extract / assign stream, served
with continuous batching on several streams, equals the plain one-call-per-request
result bit-exactly (each result is the same alone and in the mix)."""
import pytest
import torch

import synth
from helpers import to_dev

pytestmark = pytest.mark.gpu


def _stream(mats, n, seed, rate):
    from paper_2509_20776_gb300.serving import Request
    g = torch.Generator().manual_seed(seed)
    t = 0.0
    reqs = []
    for k in range(n):
        t += float(torch.empty(1).exponential_(rate, generator=g))
        mi = int(torch.randint(0, len(mats), (1,), generator=g))
        m = mats[mi].nrows
        u = float(torch.rand(1, generator=g))
        if u < 0.6:
            p = synth.random_permutation(m, seed * 1000 + k, 0).cuda()
            reqs.append(Request("permute", mi, t, p=p))
        elif u < 0.9:
            ki = int(min(m, 16 + int(torch.randint(0, 500, (1,), generator=g))))
            kj = int(min(m, 16 + int(torch.randint(0, 800, (1,), generator=g))))
            I = torch.randint(0, m, (ki,), generator=g).to(torch.int32).cuda()
            J = torch.randperm(m, generator=g)[:kj].to(torch.int32).cuda()
            reqs.append(Request("extract", mi, t, I=I, J=J))
        else:
            k2 = int(min(m, 64))
            I = torch.randperm(m, generator=g)[:k2].to(torch.int32).cuda()
            J = torch.randperm(m, generator=g)[:k2].to(torch.int32).cuda()
            Bm = synth.er_csr(k2, k2, 4, seed=k, value_kind="f32u01", rowptr_dtype=torch.int64,
                              colidx_dtype=torch.int32)
            reqs.append(Request("assign", mi, t, I=I, J=J, B=to_dev(Bm)))
    return reqs


def test_served_equals_plain():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_20776_gb300 import build
    build.build()
    from paper_2509_20776_gb300 import Context
    from paper_2509_20776_gb300.serving import Server, latency_stats, run_plain
    mats = [to_dev(synth.rmat_csr(s, 6, seed=s, symmetrize=True, value_kind="f32u01",
                                  rowptr_dtype=torch.int64, colidx_dtype=torch.int32)) for s in (9, 11, 12)]
    reqs_a = _stream(mats, 240, 3, 4000.0)
    reqs_b = _stream(mats, 240, 3, 4000.0)
    srv = Server(mats, slots=3, keep_results=True)
    srv.run(reqs_a)
    ctx = Context(0)
    run_plain(ctx, mats, reqs_b, keep_results=True)
    for a, b in zip(reqs_a, reqs_b):
        assert a.done >= a.arrival and b.done >= b.arrival
        want = b.result
        if a.kind == "extract":
            out, r0, r1 = a.result
            base, end = int(out.rowptr[r0]), int(out.rowptr[r1])
            assert torch.equal(out.rowptr[r0:r1 + 1] - base, want.rowptr.to(out.rowptr.dtype))
            assert torch.equal(out.colidx[base:end], want.colidx)
            assert torch.equal(out.values[base:end].view(torch.int32), want.values.view(torch.int32))
            assert a.nnz_out == want.nnz
        else:
            got = a.result
            assert torch.equal(got.rowptr, want.rowptr) and torch.equal(got.colidx, want.colidx)
            assert torch.equal(got.values.view(torch.int32), want.values.view(torch.int32))
    st = latency_stats(reqs_a)
    assert st["p99_ms"] >= st["p50_ms"] >= 0
    srv.close()
    ctx.close()
