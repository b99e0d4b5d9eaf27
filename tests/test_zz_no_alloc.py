"""The scan entry point that allocates nothing, against the oracle and the ordinary scan.

sp_exclusive_scan_noalloc serves callers that cannot allocate device memory when they
need a prefix sum (an allocator's own bookkeeping, a service with all memory reserved
up front, a loop that must not synchronise on an allocation).  It keeps its scratch in
a fixed device array inside the library, so this test checks that two calls in a row
-- the second reusing the array the first left behind -- both equal the oracle's
exclusive scan and sp_exclusive_scan exactly, and that an input beyond the array's
limit is refused before any launch.
The file name sorts last so a run that stops at its first failure has run the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

SP_I32, SP_I64 = 0, 1
SP_ERR_SHAPE = 2
MAX_LEN = 1 << 28


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_20776_gb300 import build
    build.build()
    from paper_2509_20776_gb300 import Context, load_library
    lib = load_library()
    ctx = Context(0)
    yield lib, ctx
    ctx.close()


def noalloc_scan(lib, x: torch.Tensor, out_dtype) -> torch.Tensor:
    out = torch.full((x.numel() + 1,), -7, dtype=out_dtype, device=x.device)
    st = torch.cuda.current_stream().cuda_stream
    code = lib.sp_exclusive_scan_noalloc(
        ctypes.c_void_p(x.data_ptr()) if x.numel() else None,
        SP_I32 if x.dtype == torch.int32 else SP_I64, x.numel(),
        ctypes.c_void_p(out.data_ptr()), SP_I32 if out_dtype == torch.int32 else SP_I64,
        ctypes.c_void_p(st))
    assert code == 0, f"sp_exclusive_scan_noalloc returned {code}"
    return out


def test_noalloc_scan_matches_scan_twice(env):
    lib, ctx = env
    g = torch.Generator().manual_seed(2024)
    # first call: many tiles, int64 output; second call: fewer tiles, int32 in/out, so
    # stale status words from the first call sit beyond the second call's tiles
    x1 = torch.randint(0, 1000, (3_000_001,), generator=g, dtype=torch.int64).cuda()
    x2 = torch.randint(0, 50, (123_457,), generator=g, dtype=torch.int32).cuda()
    got1 = noalloc_scan(lib, x1, torch.int64)
    got2 = noalloc_scan(lib, x2, torch.int32)
    # the oracle's scan (plain numpy cumulative sum) decides
    ref1 = oracle.exclusive_scan(x1.cpu().numpy())
    ref2 = oracle.exclusive_scan(x2.cpu().numpy())
    assert np.array_equal(got1.cpu().numpy().astype(np.int64), ref1)
    assert np.array_equal(got2.cpu().numpy().astype(np.int64), ref2)
    want1 = ctx.sp_exclusive_scan(x1, out_dtype=torch.int64)
    want2 = ctx.sp_exclusive_scan(x2, out_dtype=torch.int32)
    assert torch.equal(got1, want1)
    assert torch.equal(got2, want2)
    # and once more with the first input, after the array held the second call's state
    got3 = noalloc_scan(lib, x1, torch.int64)
    assert np.array_equal(got3.cpu().numpy(), ref1)


def test_noalloc_scan_empty_and_limit(env):
    lib, ctx = env
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    got = noalloc_scan(lib, e, torch.int64)
    assert got.cpu().numpy().tolist() == [0]
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    code = lib.sp_exclusive_scan_noalloc(ctypes.c_void_p(dummy.data_ptr()), SP_I32, MAX_LEN + 1,
                                         ctypes.c_void_p(dummy.data_ptr()), SP_I64, None)
    assert code == SP_ERR_SHAPE
    assert np.array_equal(dummy.cpu().numpy(), np.zeros(4, np.int32))
