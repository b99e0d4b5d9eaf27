"""Host-side helpers of the bench line (no GPU): the roofline of the dominant phase,
the row classes of the row sort, the workload name, and the serving latency summary."""
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_row_classes():
    L = torch.tensor([0, 1, 512, 513, 4096, 4097, 100000])
    rp = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(L, 0)])
    cl = bench.row_classes(rp)
    assert cl["tile"] == (0 + 1 + 512, 2)          # empty rows count no entries and no row
    assert cl["long"] == (513 + 4096, 2)
    assert cl["huge"] == (4097 + 100000, 2)


def test_roofline_of_dominant_phase():
    classes = {"tile": (400, 10), "long": (300, 2), "huge": (300, 1)}
    m, n = 100, 100
    stats = {"gather": (6.0, 6), "tile": (3.0, 6), "long": (5.0, 24), "scan": (0.5, 12), "other": (9.0, 3)}
    lk = {"g_per_s": 100.0, "table_bytes": 400, "probe": "x"}
    r = bench.roofline_permute(stats, classes, m, n, ops_per_step=3, steps=2, peak_gbs=1000.0, lookup_peak=lk)
    assert r["phase"] == "gather" and r["kernel"] == "k_gather_chunks"  # "other" has no byte model
    alg = 16 * 1000 + 16 * m  # the scope's 16 B per entry, plus the per-row pointers
    assert r["alg_bytes_per_launch"] == alg
    assert abs(r["achieved"] - alg * 6 / 6e-3 / 1e9) < 0.1
    assert r["frac"] == round(r["achieved"] / 1000.0, 4)
    # the relabel lookup (4 B per entry) only in the separately named fraction
    assert abs(r["frac_incl_lookup"] - (alg + 4 * 1000) * 6 / 6e-3 / 1e9 / 1000.0) < 1e-3
    assert r["avg_launch_ms"] == 1.0
    # lookups: one per entry of each of the 6 launches in 6 ms
    assert r["lookup_roofline"]["achieved"] == round(1000 * 6 / 6e-3 / 1e9, 2)
    assert abs(r["lookup_roofline"]["frac"] - 1000 * 6 / 6e-3 / 1e9 / 100.0) < 1e-4


def test_concurrent_phase_never_dominant():
    """A phase timed on the side stream (the split beside the tile sort) is listed but not
    chosen, however long its events bracket."""
    classes = {"tile": (400, 10), "long": (300, 2), "huge": (300, 1)}
    stats = {"gather": (6.0, 6), "tile": (3.0, 6), "huge": (9.0, 6)}
    r = bench.roofline_permute(stats, classes, 100, 100, 3, 2, 1000.0, None)
    assert r["phase"] == "huge"
    r = bench.roofline_permute(stats, classes, 100, 100, 3, 2, 1000.0, None, concurrent=("huge",))
    assert r["phase"] == "gather" and r["phase_ms_concurrent"] == ["huge"]
    assert r["phase_ms"]["huge"] == 9.0


def test_traffic_only_from_captures():
    classes = {"tile": (10, 5), "long": (0, 0), "huge": (0, 0)}
    r = bench.roofline_permute({"gather": (1.0, 3)}, classes, 5, 5, 3, 1, 100.0, None)
    if bench.GATHER_DRAM_BYTES_PER_ENTRY is None:
        assert r["traffic"] is None
    else:  # a per-entry figure from a capture, scaled by the entries one launch moves
        assert r["traffic"] == int(bench.GATHER_DRAM_BYTES_PER_ENTRY * 10)
    assert "lookup_roofline" not in r
    r = bench.roofline_permute({"tile": (1.0, 3)}, classes, 5, 5, 3, 1, 100.0, None)
    assert r["traffic"] is None and "frac_incl_lookup" not in r


def test_workload_name_follows_scale():
    assert "scale 22" in bench.WORKLOAD.format(scale=22)
    assert "{" not in bench.WORKLOAD.format(scale=25)


def test_latency_stats():
    from paper_2509_20776_gb300.serving import Request, latency_stats
    reqs = [Request("permute", 0, arrival=0.01 * k) for k in range(100)]
    for k, r in enumerate(reqs):
        r.done = r.arrival + 0.001 * (k + 1)
    s = latency_stats(reqs)
    assert abs(s["p50_ms"] - 50.5) < 1e-6 and abs(s["mean_ms"] - 50.5) < 1e-6
    assert 99.0 <= s["p99_ms"] <= 100.0
    assert abs(s["span_s"] - (0.99 + 0.1)) < 1e-9
