"""The allocator hook (sp_allocator): a context can take all of its device memory from
PyTorch's caching allocator, and when the k-th allocation fails the call returns
SP_ERR_OOM, a library-allocated output comes back freed with zeroed pointers, nothing
leaks, and the context stays usable (its next call gives the oracle's result)."""
import ctypes

import pytest
import torch

import oracle
import synth
from helpers import assert_same, to_dev, to_oracle

pytestmark = pytest.mark.gpu

SP_I32, SP_I64, SP_ERR_OOM = 0, 1, 8


class FailAt:
    """Caching-allocator memory; allocation number `fail_at` (1-based) returns NULL."""

    def __init__(self, fail_at=0):
        from paper_2509_20776_gb300 import TorchAllocator
        self.inner = TorchAllocator(0)
        self.fail_at, self.n, self.live = fail_at, 0, {}

    def alloc(self, nbytes, stream):
        self.n += 1
        if self.n == self.fail_at:
            return 0
        ptr = self.inner.alloc(nbytes, stream)
        self.live[ptr] = nbytes
        return ptr

    def free(self, ptr, nbytes, stream):
        self.live.pop(ptr)
        self.inner.free(ptr, nbytes, stream)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_20776_gb300 import build, load_library
    build.build()
    return load_library()


def _permute_lib_alloc(lib, ctx, A, p):
    """sp_permute with a library-allocated output; returns (status, descriptor)."""
    from paper_2509_20776_gb300 import sp_csr
    B = sp_csr(0, 0, 0, SP_I64, 0, 0, None, None, None)
    st = lib.sp_permute(ctx.handle, ctypes.byref(A.desc()), ctypes.c_void_p(p.data_ptr()),
                        ctypes.c_void_p(p.data_ptr()), SP_I32, ctypes.byref(B),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, B


def test_every_failed_allocation_is_clean(lib):
    from paper_2509_20776_gb300 import Context
    Ah = synth.rmat_csr(12, 8, seed=3, symmetrize=True, value_kind="f32u01", rowptr_dtype=torch.int64,
                        colidx_dtype=torch.int32)
    A = to_dev(Ah)
    p = synth.random_permutation(Ah.nrows, 2, 0).cuda()
    want = oracle.permute(to_oracle(Ah), p.cpu().numpy(), p.cpu().numpy())
    # how many allocations a successful call makes (outputs + workspace)
    probe = FailAt()
    ctx = Context(0, allocator=probe)
    st, B = _permute_lib_alloc(lib, ctx, A, p)
    assert st == 0 and B.rowptr and B.colidx and B.values
    ctx.sync()
    lib.sp_csr_free(ctx.handle, ctypes.byref(B))
    assert not B.rowptr and not B.colidx and not B.values
    n_ok = probe.n
    ctx.close()
    assert n_ok >= 4 and not probe.live  # three output arrays and the workspace, all returned
    for k in range(1, n_ok + 1):
        fa = FailAt(k)
        ctx = Context(0, allocator=fa)
        st, B = _permute_lib_alloc(lib, ctx, A, p)
        assert st == SP_ERR_OOM, f"allocation {k}: status {st}"
        assert not B.rowptr and not B.colidx and not B.values, f"allocation {k}: output not released"
        ctx.sync()
        # the context still works (the failing allocation has passed)
        assert_same(ctx.sp_permute(A, p, p), want, f"after failing allocation {k}")
        ext = ctx.sp_extract(A, p[:100].contiguous(), p[50:300].contiguous())
        assert_same(ext, oracle.extract(to_oracle(Ah), p[:100].cpu().numpy(), p[50:300].cpu().numpy()),
                    f"extract after failing allocation {k}")
        ctx.close()
        assert not fa.live, f"allocation {k}: {len(fa.live)} blocks leaked"


def test_extract_plan_allocation_fails_cleanly(lib):
    """The first allocation of an extraction is its plan: SP_ERR_OOM, nothing leaks."""
    from paper_2509_20776_gb300 import Context, SpError
    Ah = synth.er_csr(500, 400, 6, seed=1, value_kind="f64um11", rowptr_dtype=torch.int32)
    A = to_dev(Ah)
    I = torch.arange(0, 500, 2, dtype=torch.int32, device="cuda")
    J = torch.arange(399, 0, -3, dtype=torch.int32, device="cuda")
    fa = FailAt(1)
    ctx = Context(0, allocator=fa)
    with pytest.raises(SpError) as e:
        ctx.sp_extract(A, I, J)
    assert e.value.name == "SP_ERR_OOM"
    assert_same(ctx.sp_extract(A, I, J), oracle.extract(to_oracle(Ah), I.cpu().numpy(), J.cpu().numpy()),
                "extract after the failed plan")
    ctx.close()
    assert not fa.live
