"""The request server: every result of a mixed permute / extract / assign stream, served
with continuous batching on several streams, equals the oracle's result for that request
bit-exactly, and equals the plain one-call-per-request result (each result is the same
alone and in the mix)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_same, bits, to_dev, to_oracle

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


def _check_part(result, ref, what):
    """A result that is a slice of a batch's CSR: (out, first row, end row)."""
    out, r0, r1 = result
    base, end = int(out.rowptr[r0]), int(out.rowptr[r1])
    rp = (out.rowptr[r0:r1 + 1] - base).cpu().numpy().astype(np.int64)
    assert np.array_equal(rp, ref.rowptr), f"{what} rowptr"
    assert np.array_equal(out.colidx[base:end].cpu().numpy().astype(np.int64), ref.colidx), f"{what} colidx"
    assert np.array_equal(bits(out.values[base:end].cpu().numpy()), bits(ref.values)), f"{what} values"


def _check_result(result, ref, what):
    if isinstance(result, tuple):
        _check_part(result, ref, what)
    else:
        assert_same(result, ref, what)


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
    hosts = [to_oracle(m) for m in mats]
    for k, (a, b) in enumerate(zip(reqs_a, reqs_b)):
        assert a.done >= a.arrival and b.done >= b.arrival
        want = b.result
        A = hosts[a.mat]
        # the oracle decides: the definition of each operation on the request's inputs
        if a.kind == "permute":
            ref = oracle.permute(A, a.p.cpu().numpy(), a.p.cpu().numpy())
        elif a.kind == "extract":
            ref = oracle.extract(A, a.I.cpu().numpy(), a.J.cpu().numpy())
        else:
            ref = oracle.assign(A, a.I.cpu().numpy(), a.J.cpu().numpy(), to_oracle(a.B))
        _check_result(a.result, ref, f"request {k}: served {a.kind}")
        assert a.nnz_out == ref.nnz
        assert_same(want, ref, f"request {k}: plain {a.kind}")
    st = latency_stats(reqs_a)
    assert st["p99_ms"] >= st["p50_ms"] >= 0
    srv.close()
    ctx.close()


def test_extractions_held_by_memory():
    """A budget smaller than any output: every counted extraction batch waits, counted but
    not filled, until the work in flight retires; every result still equals the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_20776_gb300 import build
    build.build()
    from paper_2509_20776_gb300.serving import Server
    mats = [to_dev(synth.rmat_csr(s, 6, seed=s + 1, symmetrize=True, value_kind="f32u01",
                                  rowptr_dtype=torch.int64, colidx_dtype=torch.int32)) for s in (9, 11)]
    reqs = _stream(mats, 80, 5, 1e9)  # everything arrives at once
    srv = Server(mats, slots=2, mem_budget=1, keep_results=True)
    srv.run(reqs)
    assert srv.stats["held_rounds"] > 0 and srv.stats["batches"] > 0
    hosts = [to_oracle(m) for m in mats]
    for k, r in enumerate(reqs):
        A = hosts[r.mat]
        if r.kind == "permute":
            ref = oracle.permute(A, r.p.cpu().numpy(), r.p.cpu().numpy())
        elif r.kind == "assign":
            ref = oracle.assign(A, r.I.cpu().numpy(), r.J.cpu().numpy(), to_oracle(r.B))
        else:
            ref = oracle.extract(A, r.I.cpu().numpy(), r.J.cpu().numpy())
        _check_result(r.result, ref, f"request {k}")
    srv.close()


def test_permutations_batched_per_round():
    """Everything arrives at once under a large budget: the first round's permutations of
    the small matrices run as one batch, the largest matrix's alone, and every result
    (a slice of the batch's CSR, or a CSR of its own) equals the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_20776_gb300 import build
    build.build()
    from paper_2509_20776_gb300.serving import Server
    mats = [to_dev(synth.rmat_csr(s, 6, seed=s + 2, symmetrize=True, value_kind="f32u01",
                                  rowptr_dtype=torch.int64, colidx_dtype=torch.int32)) for s in (8, 10, 12)]
    reqs = _stream(mats, 90, 7, 1e9)
    srv = Server(mats, slots=2, keep_results=True, perm_batch_nnz=mats[1].nnz)
    srv.run(reqs)
    assert srv.stats["perm_batches"] >= 1
    hosts = [to_oracle(m) for m in mats]
    batched = alone = 0
    for k, r in enumerate(reqs):
        A = hosts[r.mat]
        if r.kind == "permute":
            ref = oracle.permute(A, r.p.cpu().numpy(), r.p.cpu().numpy())
            batched += isinstance(r.result, tuple)
            alone += r.mat == 2 and not isinstance(r.result, tuple)
        elif r.kind == "assign":
            ref = oracle.assign(A, r.I.cpu().numpy(), r.J.cpu().numpy(), to_oracle(r.B))
        else:
            ref = oracle.extract(A, r.I.cpu().numpy(), r.J.cpu().numpy())
        _check_result(r.result, ref, f"request {k}: {r.kind}")
        assert r.nnz_out == ref.nnz
    assert batched > 1 and alone > 0
    srv.close()
