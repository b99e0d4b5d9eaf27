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
    r = bench.roofline_permute(stats, classes, m, n, ops_per_step=3, steps=2, peak_gbs=1000.0, scale=7)
    assert r["phase"] == "gather" and r["kernel"] == "k_gather_chunks"  # "other" has no byte model
    alg = 20 * 1000 + 16 * m
    assert r["alg_bytes_per_launch"] == alg
    assert abs(r["achieved"] - alg * 6 / 6e-3 / 1e9) < 0.1
    assert r["frac"] == round(r["achieved"] / 1000.0, 4)
    assert r["traffic"] is None  # no capture at this scale
    assert r["avg_launch_ms"] == 1.0


def test_traffic_only_from_captures():
    for (scale, phase), v in bench.NCU_TRAFFIC.items():
        assert scale == 25 and phase in ("gather", "tile", "huge", "long") and v > 0
    classes = {"tile": (10, 5), "long": (0, 0), "huge": (0, 0)}
    r = bench.roofline_permute({"gather": (1.0, 3)}, classes, 5, 5, 3, 1, 100.0, 25)
    assert r["traffic"] == bench.NCU_TRAFFIC[(25, "gather")]


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
