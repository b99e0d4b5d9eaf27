"""Host side of the tuning table: entry validation and ordering, and the option / op
numbers of the binding against the ones include/sp.h declares."""
import os
import re

import pytest

from paper_2509_20776_gb300 import _binding as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_entries_validated_and_ordered():
    rows = b.tune_entries({"entries": [
        {"op": "batch", "size_max": 5, "batch_rows": 8},
        {"op": "permute", "size_max": 100, "tile_shape": 1},
        {"op": "permute", "size_max": 10, "heavy": 256}]})
    assert [(r["op"], r["size_max"]) for r in rows] == [(0, 10), (0, 100), (3, 5)]
    assert rows[0]["heavy"] == 256 and rows[0]["tile_shape"] == -1
    assert rows[2]["batch_rows"] == 8 and rows[2]["count_rows"] == -1
    for bad in ({"op": "sort", "size_max": 1}, {"op": "permute", "size_max": 1, "heavy": 100},
                {"op": "extract", "size_max": 1, "fill_rows": 3}, {"op": "batch", "size_max": 1, "batch_rows": 16},
                {"op": "extract", "size_max": 1, "identify": 2}):
        with pytest.raises(ValueError):
            b.tune_entries([bad])


def test_numbers_match_header():
    h = open(os.path.join(ROOT, "include", "sp.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"(SP_OPT_[A-Z_]+) = (\d+)", h))
    for name, key in b.SHAPE_OPTIONS.items():
        assert enum["SP_OPT_" + name.upper()] == key
    ops = dict((k, int(v)) for k, v in re.findall(r"SP_OP_([A-Z]+) = (\d+)", h))
    assert {k.lower(): v for k, v in ops.items()} == b.OPS
    # the ctypes entry mirrors the C struct's field order and widths
    assert [f for f, _ in b.sp_tune_entry._fields_] == ["op", "tile_shape", "heavy", "count_rows", "fill_rows",
                                                        "batch_rows", "identify", "size_max"]
    assert b.sp_tune_entry.size_max.offset == 32


def test_autotune_compare_and_files(tmp_path):
    """The tuner's bit-identity check and its table file, on CPU tensors."""
    import json
    import torch
    from paper_2509_20776_gb300 import autotune as at

    class M:  # a CSR-like result
        def __init__(self, v):
            self.rowptr = torch.tensor([0, 2, 3])
            self.colidx = torch.tensor([1, 4, 0], dtype=torch.int32)
            self.values = torch.tensor(v, dtype=torch.float32)

    assert at._same(M([1.0, 2.0, 3.0]), M([1.0, 2.0, 3.0]))
    assert not at._same(M([1.0, 2.0, 3.0]), M([1.0, 2.0, 4.0]))
    assert not at._same(M([0.0, 2.0, 3.0]), M([-0.0, 2.0, 3.0]))  # bit patterns, not values
    assert at._same((M([1.0, 2.0, 3.0]), torch.tensor([5])), (M([1.0, 2.0, 3.0]), torch.tensor([5])))
    assert not at._same((M([1.0, 2.0, 3.0]),), (M([1.0, 2.0, 3.0]), torch.tensor([5])))
    table = {"format": "sp-tuning-1", "entries": [{"op": "batch", "size_max": 1 << 62, "batch_rows": 2,
                                                   "tile_shape": 0, "heavy": 128}]}
    path = tmp_path / "t.json"
    at.save(table, str(path))
    assert at.load(str(path)) == table
    b.tune_entries(at.load(str(path)))  # the binding accepts what the tuner writes
    (tmp_path / "bad.json").write_text(json.dumps({"entries": []}))
    with pytest.raises(ValueError):
        at.load(str(tmp_path / "bad.json"))
    # every knob the tuner searches is a shape the binding and the header know
    assert set(at.SEARCH) == set(b.SHAPE_OPTIONS) and set(at.KNOBS) == set(b.OPS)


def test_library_lookup_takes_the_tightest_class():
    """The C library's per-call lookup (host only): first entry of the op whose size_max
    covers the call, with the binding's ordering making that the tightest class."""
    import ctypes
    lib = b.load_library()
    arr, n = b.tune_array({"entries": [
        {"op": "permute", "size_max": 1 << 40, "tile_shape": 0, "heavy": 512},
        {"op": "permute", "size_max": 1000, "tile_shape": 1},
        {"op": "extract", "size_max": 1 << 40, "count_rows": 2}]})
    out = b.sp_tune_entry()
    assert lib.sp_tuning_lookup(arr, n, b.OPS["permute"], 999, ctypes.byref(out)) == 1
    assert (out.tile_shape, out.heavy, out.size_max) == (1, -1, 1000)
    assert lib.sp_tuning_lookup(arr, n, b.OPS["permute"], 1001, ctypes.byref(out)) == 1
    assert (out.tile_shape, out.heavy) == (0, 512)
    assert lib.sp_tuning_lookup(arr, n, b.OPS["extract"], 5, ctypes.byref(out)) == 1 and out.count_rows == 2
    assert lib.sp_tuning_lookup(arr, n, b.OPS["batch"], 5, ctypes.byref(out)) == 0
    assert lib.sp_tuning_lookup(arr, n, b.OPS["permute"], (1 << 40) + 1, ctypes.byref(out)) == 0
    assert lib.sp_tuning_lookup(None, 2, 0, 5, ctypes.byref(out)) == -1
    assert lib.sp_tuning_lookup(arr, -1, 0, 5, ctypes.byref(out)) == -1
