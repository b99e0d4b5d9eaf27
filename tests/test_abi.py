"""The C ABI library builds, loads without a GPU, and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sp.h")


def declared():
    names = re.findall(r"^SP_API [^(]*?\b(sp_[a-z0-9_]+)\(", open(HEADER).read(), re.M)
    assert names
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2509_20776_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2509_20776_gb300 import SIGNATURES
    assert set(declared()) == set(SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.sp_status_str.restype = ctypes.c_char_p
    assert lib.sp_status_str(0) == b"SP_OK"
    assert lib.sp_status_str(9) == b"SP_ERR_TIMEOUT"
    assert lib.sp_version() == 100


def test_null_arguments_rejected_on_host(lib):
    # host-side argument checks return before touching the device
    assert lib.sp_ctx_create(None, 0, None) == 1
    assert lib.sp_permute(None, None, None, None, 0, None, None) == 1
    assert lib.sp_ctx_set_option(None, 0, 0) == 1


def test_last_cuda_error_starts_clear(lib):
    """No call has failed with SP_ERR_CUDA yet: code 0 and an empty location."""
    lib.sp_last_cuda_error.restype = ctypes.c_int
    lib.sp_last_cuda_error.argtypes = [ctypes.POINTER(ctypes.c_char_p)]
    where = ctypes.c_char_p()
    assert lib.sp_last_cuda_error(ctypes.byref(where)) == 0
    assert (where.value or b"") == b""
    assert lib.sp_last_cuda_error(None) == 0


def _enum(name):
    """name -> value of the C enum typedef'd as `name` in the header."""
    text = open(HEADER).read()
    m = re.search(r"typedef enum " + name + r"\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(SP_[A-Z0-9_]+)\s*=\s*(\d+)", body)}


def test_binding_option_constants_match_header():
    """The binding's option keys are the header's enum values (a drift would set the
    wrong knob without any error)."""
    import paper_2509_20776_gb300._binding as b
    opts = _enum("sp_option")
    assert "SP_OPT_OVERLAP" in opts
    for name, value in opts.items():
        assert getattr(b, name) == value, name


def test_binding_assign_modes_match_header():
    import paper_2509_20776_gb300._binding as b
    for name, value in _enum("sp_assign_mode").items():
        assert getattr(b, name) == value, name
