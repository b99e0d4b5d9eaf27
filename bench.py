#!/usr/bin/env python3
"""Throughput of the GB300 sparse permutation / extraction / assignment path.

Headline workload (printed as `value`): permutation at scale -- R-MAT (a,b,c,d) =
(0.57, 0.19, 0.19, 0.05), scale 25 (33,554,432 rows), edge factor 16, symmetrised,
duplicates merged, int64 row pointer, int32 columns, fp32 values.  One step applies the
three permutations of that workload: P A P^T with a random p, P A P^T with the
degree-descending p, and P A Q^T with independent random p, q.  Metric: output
entries per second (whole job), inputs resident in HBM (each far larger than L2).

Extra measured operations (key "ops"): extraction at scale (Erdos-Renyi n = 2^26,
32 draws/row; A(I, J) with random distinct |I| = |J| = n/2) and assignment at scale
(R-MAT scale 26, edge factor 24; A(I, J) = B with B an ER 2^22 x 2^22 matrix, 8/row,
random distinct I, J of 2^22).

`--impl reference` times the CPU oracle (the reference arm of this build) on a bounded
sample of the same workload.  Under torchrun every rank runs an independent replica
(the path has no exchange step on one GPU), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "output nnz/s & %HBM peak for permute/extract/assign; served p50/p99 vs plain"
UNIT = "output nnz/s"
WORKLOAD = ("R-MAT scale {scale} (a,b,c,d)=(0.57,0.19,0.19,0.05), edge factor 16, symmetrised; "
            "P A P^T random p + P A P^T degree-descending p + P A Q^T random p,q")

# DRAM bytes (read + write) per output entry of one k_gather_chunks launch on the
# first P A P^T (random p), from a one-kernel ncu capture of only
# dram__bytes_read.sum + dram__bytes_write.sum on the rows-limited instance of the same
# workload (bench.py --rows-limit 2097152: 2^21 random rows, all 2^25 columns, so the
# relabel map keeps its full-size L2 pressure); scaled to a full launch by the entries
# it moves (profiles/gather_dram_rmat25_rows2m.md).  Only valid for the kernel
# as captured: retake the capture when it changes.
GATHER_DRAM_BYTES_PER_ENTRY = 25.07  # 1 655 663 104 B over 66 045 976 entries

_T0 = time.time()


def log(msg):
    print(f"[bench {time.time() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=25, help="R-MAT scale of the headline workload")
    ap.add_argument("--no-extra", action="store_true", help="skip the extraction/assignment ops")
    ap.add_argument("--ops", default="extract,assign,batch,pbatch,serve",
                    help="comma list of the extra sections to run (extract, assign, batch, pbatch, serve)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--lookup-sweep", action="store_true",
                    help="print the measured rate of uniform random 4-byte lookups per table size and exit")
    ap.add_argument("--profile-case", default="", choices=["", "assign-rmat24", "extract-er23"],
                    help="one small operation for a one-kernel ncu capture (no bench line): the "
                         "assignment on R-MAT scale 24 ef 24 with |I| = |J| = 2^20, or the extraction "
                         "of half the rows and columns of ER 2^23 x 32")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="1 (default): the row sort's key-range split runs on the context's side "
                         "stream, concurrent with the tile sort; 0: all on one stream")
    ap.add_argument("--rows-limit", type=int, default=0,
                    help="profiling case: R random rows of the headline matrix (all columns), "
                         "one permutation with independent random p, q; prints its line and exits")
    return ap.parse_args()


def peak_gbs():
    """The HBM denominator: the measured copy bandwidth, else the fallback figure."""
    pk = peaks()
    return pk["hbm_gbs"] if pk else 6800.0


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler for SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples: SP_BENCH_CLOCKS_DIR when set, else the system's temporary folder
        import tempfile
        d = os.environ.get("SP_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"sp_bench_clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("SP_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------------------
def permute_workload(scale: int, device):
    import torch
    import synth
    A = synth.rmat_csr(scale, 16, (0.57, 0.19, 0.19, 0.05), seed=0, symmetrize=True,
                       value_kind="f32u01", rowptr_dtype=torch.int64, colidx_dtype=torch.int32,
                       device=device)
    n = A.nrows
    p = synth.random_permutation(n, 1, 0, device=device)
    pdeg = synth.degree_descending_permutation(A.rowptr)
    q = synth.random_permutation(n, 1, 1, device=device)
    return A, [("PAPt_random", p, p), ("PAPt_degree", pdeg, pdeg), ("PAQt_random", p, q)]


TILE_CP, LONG_CAP = 512, 4096  # row-length limits of the tile and long-row kernels


def row_classes(rowptr):
    """Entries / non-empty rows of the row sort's three classes: tiles (rows of at most
    TILE_CP entries), rows sorted alone (at most LONG_CAP) and rows split by key range
    first (longer); row lengths move with the rows under a permutation."""
    import torch
    L = (rowptr[1:] - rowptr[:-1]).to(torch.int64)
    small = L <= TILE_CP
    huge = L > LONG_CAP
    long_ = (~small) & (~huge)
    out = {}
    for name, m in (("tile", small), ("long", long_), ("huge", huge)):
        out[name] = (int(L[m].sum()), int(((L > 0) & m).sum()))
    return out


def roofline_permute(stats, classes, m, n, ops_per_step, steps, peak_gbs, lookup_peak, concurrent=()):
    """Roofline of the phase that takes the most device time: its algorithmic bytes per
    launch over its average CUDA-event duration (int32 columns, fp32 values).  The gather
    moves 16 B per entry (read and write column + value, the scope's per-entry bytes) plus
    16 B per row (output row pointer, source start); its 4-byte relabel lookup per entry is
    counted separately (frac_incl_lookup) and against the measured random-lookup rate.
    Phases in `concurrent` run on a second stream beside another phase: their event times
    include the time they share the SMs, so they are reported but never taken as the
    dominant kernel."""
    e_tile, r_tile = classes["tile"]
    e_long, _ = classes["long"]
    e_huge, _ = classes["huge"]
    nnz = e_tile + e_long + e_huge
    per_op = {
        # gather: read col + val, write col + val; vp pair and source start per row
        "gather": 16 * nnz + 16 * m,
        # in-place sort of tile rows: read and write col + val; row pointer per row
        "tile": 16 * e_tile + 8 * m,
        # rows sorted alone and key-range runs of long rows: read and write col + val
        "long": 16 * (e_long + e_huge),
        # key-range split of long rows: keys, then keys + values, written to the buffer
        "huge": 20 * e_huge,
        # lengths: p, rowptr pair; writes vp and the source start
        "scan": 36 * m,
        "map": 12 * n,
        "partition": 8 * m,
    }
    launches_total = ops_per_step * steps
    best = None
    for ph, (ms, cnt) in stats.items():
        if cnt == 0 or ms <= 0 or ph not in per_op or ph in concurrent:
            continue
        if best is None or ms > best[1]:
            best = (ph, ms, cnt)
    ph, ms, cnt = best
    kernel = {"gather": "k_gather_chunks", "tile": "k_seg_sort<SsTile>", "long": "k_seg_sort<SsRun>",
              "huge": "k_split", "scan": "k_scan", "map": "k_inverse_map", "partition": "k_scan"}[ph]
    byts = per_op[ph] * launches_total
    sec = ms * 1e-3
    achieved = byts / sec / 1e9
    out = {"bound": "hbm", "kernel": kernel, "phase": ph, "achieved": round(achieved, 1),
           "peak": peak_gbs, "unit": "GB/s", "frac": round(achieved / peak_gbs, 4),
           "traffic": None, "alg_bytes_per_launch": per_op[ph], "launches": cnt,
           "frac_of_nominal_7900gbs": round(achieved / 7900.0, 4),
           "avg_launch_ms": round(ms / cnt, 4),
           "phase_ms": {k: round(v[0], 3) for k, v in stats.items() if v[1]}}
    if concurrent:
        out["phase_ms_concurrent"] = sorted(concurrent)
    if ph == "gather":
        with_lookup = (per_op[ph] + 4 * nnz) * launches_total / sec / 1e9
        out["frac_incl_lookup"] = round(with_lookup / peak_gbs, 4)
        if GATHER_DRAM_BYTES_PER_ENTRY is not None:
            out["traffic"] = int(GATHER_DRAM_BYTES_PER_ENTRY * nnz)
        if lookup_peak:
            rate = nnz * launches_total / sec
            out["lookup_roofline"] = {"achieved": round(rate / 1e9, 2), "peak": lookup_peak["g_per_s"],
                                      "unit": "G lookups/s", "frac": round(rate / 1e9 / lookup_peak["g_per_s"], 4),
                                      "table_bytes": lookup_peak["table_bytes"], "probe": lookup_peak["probe"]}
    return out


def lookup_probe(table_elems, cols, device):
    """Measured rate of the relabel lookups alone: PyTorch's gather of an int32 map of
    `table_elems` entries at the workload's own column indices `cols` (the same lookups,
    in the same order, that the gather makes; the index stream is read and the result
    written as well), best of 3 after a warm-up.  The gather cannot relabel faster than
    this, so its lookup rate over this one is its fraction of the lookup ceiling."""
    import torch
    t = torch.arange(table_elems, dtype=torch.int32, device=device)
    out = torch.empty(cols.numel(), dtype=torch.int32, device=device)
    torch.index_select(t, 0, cols, out=out)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        torch.index_select(t, 0, cols, out=out)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    del t, out
    torch.cuda.empty_cache()
    return {"g_per_s": round(cols.numel() / (best * 1e-3) / 1e9, 2), "table_bytes": table_elems * 4,
            "probe": f"torch.index_select of an int32 map of {table_elems} entries at the workload's "
                     f"{cols.numel()} column indices (index read and result write included), best of 3"}


def time_steps(fn, steps, warmup, ws):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(s)
    for _ in range(steps):
        fn()
    ev[1].record(s)
    torch.cuda.synchronize()
    barrier(ws)
    return ev[0].elapsed_time(ev[1])


def run_rows_limited(args, ctx, holder, dev):
    """Profiling case (--rows-limit R): R random rows of the headline matrix (seeded, so
    the row-length mix is the workload's) with all its columns, and
    B = P A Q^T with independent random p (R) and q (all columns): the kernels see the
    full-size column map (the relabel's L2 pressure) at a few GB on the device.  The full
    matrix is released before the measured operation."""
    import torch
    import synth
    from paper_2509_20776_gb300 import CSR
    A0 = holder.pop()
    A = CSR(A0.nrows, A0.ncols, A0.rowptr, A0.colidx, A0.values)
    del A0
    step = max(1, A.nrows // max(1, args.rows_limit))
    # a random subset (evenly spaced rows would favour R-MAT's heavy low-numbered rows)
    I = synth.random_subset(A.nrows, A.nrows // step, 9, 0, device=dev)
    Jall = torch.arange(0, A.ncols, dtype=torch.int32, device=dev)
    Ar = ctx.sp_extract(A, I, Jall)  # consecutive J: rows copied as they are
    del A, I, Jall
    torch.cuda.empty_cache()
    R = Ar.nrows
    p = synth.random_permutation(R, 1, 0, device=dev)
    q = synth.random_permutation(Ar.ncols, 1, 1, device=dev)
    B = ctx.sp_permute(Ar, p, q)
    ms = time_steps(lambda: ctx.sp_permute(Ar, p, q, sync=False, out=B), max(1, args.steps), args.warmup, 1)
    ctx.sync()
    return {"rows_limit": R, "ncols": Ar.ncols, "nnz": Ar.nnz, "ms_per_op": round(ms / max(1, args.steps), 4),
            "workload": "R random rows of the headline matrix, all columns; P A Q^T with random p, q"}


def profile_case(args):
    """--profile-case: the named operation, twice (the second for the capture), at a size
    whose device footprint stays at a few GB; prints its phase times."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2509_20776_gb300 import CSR, Context, SP_OPT_TIMING
    dev = torch.device("cuda", 0)
    ctx = Context(0)
    if args.profile_case == "assign-rmat24":
        A = synth.rmat_csr(24, 24, (0.57, 0.19, 0.19, 0.05), seed=0, symmetrize=False, value_kind="f32u01",
                           rowptr_dtype=torch.int64, colidx_dtype=torch.int32, device=dev)
        k = 1 << 20
        Bm = synth.er_csr(k, k, 8, seed=1, value_kind="f32u01", rowptr_dtype=torch.int64,
                          colidx_dtype=torch.int32, device=dev)
        I = synth.random_subset(A.nrows, k, 4, 1, device=dev)
        J = synth.random_subset(A.ncols, k, 4, 2, device=dev)
        Ad = CSR(A.nrows, A.ncols, A.rowptr, A.colidx, A.values)
        Bd = CSR(Bm.nrows, Bm.ncols, Bm.rowptr, Bm.colidx, Bm.values)
        run = lambda: ctx.sp_assign(Ad, I, J, Bd)  # noqa: E731
    else:
        n = 1 << 23
        A = synth.er_csr(n, n, 32, seed=0, value_kind="f32u01", rowptr_dtype=torch.int64,
                         colidx_dtype=torch.int32, device=dev)
        I = synth.random_subset(n, n // 2, 3, 1, device=dev)
        J = synth.random_subset(n, n // 2, 3, 2, device=dev)
        Ad = CSR(A.nrows, A.ncols, A.rowptr, A.colidx, A.values)
        run = lambda: ctx.sp_extract(Ad, I, J)  # noqa: E731
    for _ in range(2):
        ctx.set_option(SP_OPT_TIMING, 1)
        ctx.phase_stats(reset=True)
        out = run()
        ctx.sync()
        st = ctx.phase_stats(reset=True)
        log(f"{args.profile_case}: {out.nnz} entries, phases (ms) " +
            str({k: round(v[0], 3) for k, v in st.items() if v[1]}))
        del out


def log_summary(res):
    """One short line per measured operation on stderr (the driver keeps the tail)."""
    def line(name, d, ms_key="ms_per_op"):
        if not isinstance(d, dict) or "value" not in d:
            return
        log(f"SUMMARY {name}: {d.get('workload', '')[:70]} | {d.get(ms_key, '?')} ms | "
            f"{d['value'] / 1e9:.2f} G entries/s | op frac {d.get('op_roofline_frac', '-')} | "
            f"alg bytes {d.get('alg_bytes_per_op', '-')}")
    r = res.get("roofline", {})
    log(f"SUMMARY permute: {res['config']['workload'][:70]} | {res['ms_per_step'] / res['config']['ops_per_step']:.3f} "
        f"ms/op | {res['value'] / 1e9:.2f} G entries/s | op frac {res['op_roofline']['frac']} | "
        f"alg bytes {res['op_roofline']['bytes_per_op']} | top kernel {r.get('kernel')} frac {r.get('frac')} "
        f"lookup frac {r.get('lookup_roofline', {}).get('frac')}")
    if "e2e" in res:
        log(f"SUMMARY permute e2e: {res['e2e']['ms_per_step']} ms/step | {res['e2e']['value'] / 1e9:.2f} G entries/s")
    ops = res.get("ops", {})
    ex = ops.get("extract", {})
    line("extract", ex)
    line("extract contiguous", ex.get("contiguous_block"))
    line("extract mesh", ex.get("mesh"))
    asg = ops.get("assign", {})
    line("assign", asg)
    line("assign contiguous", asg.get("contiguous"))
    line("assign+permute fused", asg.get("assign_permute"))
    bt = ops.get("batch_extract", {})
    if "batched_ms" in bt:
        log(f"SUMMARY batch: {bt['batched_ms']} ms batched vs {bt['plain_ms']} ms plain | graph fill "
            f"{bt['graph_fill_ms']} ms | whole batch from one graph {bt.get('graph_run_ms')} ms, frac "
            f"{bt.get('graph_run_roofline', {}).get('frac')} | {bt['batched_value'] / 1e9:.2f} G entries/s")
    pb = ops.get("batch_permute", {})
    if "batched_ms" in pb:
        log(f"SUMMARY batch permute: {pb['batched_ms']} ms batched vs {pb['plain_ms']} ms plain | graph "
            f"{pb['graph_ms']} ms | {pb['graph_value'] / 1e9:.2f} G entries/s")
    sv = ops.get("serve", {})
    for k, v in sv.items():
        if k.startswith("load_"):
            log(f"SUMMARY serve {k}: served p50/p99 {v['served']['p50_ms']}/{v['served']['p99_ms']} ms "
                f"{v['served']['value'] / 1e9:.2f} G/s | plain {v['plain']['p50_ms']}/{v['plain']['p99_ms']} ms "
                f"{v['plain']['value'] / 1e9:.2f} G/s")


def run_ours(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20776_gb300 import CSR, Context, SP_OPT_TIMING, SP_OPT_OVERLAP
    dev = torch.device("cuda", local)
    ctx = Context(local)
    ctx.set_option(SP_OPT_OVERLAP, args.overlap)
    pk = peaks()
    hbm = pk["hbm_gbs"] if pk else 6800.0
    log("generating the permutation workload")
    A, ops = permute_workload(args.scale, dev)
    log(f"generated: {A.nrows} rows, {A.nnz} entries")
    if args.rows_limit:
        del ops
        holder = [A]
        del A
        return run_rows_limited(args, ctx, holder, dev)
    Ad = CSR(A.nrows, A.ncols, A.rowptr, A.colidx, A.values)
    nnz, m = A.nnz, A.nrows
    outs = [ctx.sp_permute(Ad, p, q, sync=True) for _, p, q in ops]  # also validates

    def step():
        for (_, p, q), B in zip(ops, outs):
            ctx.sp_permute(Ad, p, q, sync=False, out=B)

    log("validated the three permutations")
    classes = row_classes(A.rowptr)
    # timed region: device-resident inputs, outputs preallocated
    ctx.phase_stats(reset=True)
    ctx.set_option(SP_OPT_TIMING, 1)
    with Clocks(local) as clk:
        ms = time_steps(step, args.steps, args.warmup, ws)
    ctx.sync()
    ctx.set_option(SP_OPT_TIMING, 0)
    stats = ctx.phase_stats(reset=True)
    # the phase timers include the warm-up steps: scale launches to timed steps only
    total_steps = args.steps + args.warmup
    stats_timed = {k: (v[0] * args.steps / total_steps, v[1] * args.steps // total_steps)
                   for k, v in stats.items()}
    launches_per_step = sum(v[1] for v in stats.values()) / total_steps
    ms = max_over_ranks(ms, ws)
    out_per_step = nnz * len(ops)
    value = out_per_step * args.steps * ws / (ms * 1e-3)
    lk = lookup_probe(A.ncols, A.colidx, dev)
    roof = roofline_permute(stats_timed, classes, m, A.ncols, len(ops), args.steps, hbm, lk,
                            concurrent=("huge",) if args.overlap else ())
    # whole op: read and write col + val per entry, p and rowptr pair per row, q and qinv
    alg_bytes_op = 16 * nnz + 28 * m + 12 * A.ncols
    op_frac = alg_bytes_op * len(ops) * args.steps / (ms * 1e-3) / 1e9 / hbm
    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64 rowptr / int32 col / fp32 values (moved as 32-bit words)",
        "data": "synthetic (seeded R-MAT; the paper's SuiteSparse graphs are not available)",
        "config": {"workload": WORKLOAD.format(scale=args.scale), "rows": m, "nnz": nnz, "ops_per_step": len(ops),
                   "l2": "inputs larger than L2 (no flush needed)",
                   "parallelism": f"replicas x{ws}"},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "roofline": roof,
        "op_roofline": {"bytes_per_op": alg_bytes_op, "frac": round(op_frac, 4),
                        "peak": hbm, "unit": "GB/s", "note": "whole op, algorithmic bytes"},
        "row_classes": {k: {"entries": v[0], "rows": v[1]} for k, v in classes.items()},
        "clocks": clk.summary(),
        "peak_source": "measured (MEASURED_PEAKS.json)" if pk else "fallback",
    }
    log(f"timed permutations: {ms / args.steps:.3f} ms/step")
    # ---- end to end through the public API with host buffers -----------------------
    if not args.no_e2e:
        result["e2e"] = e2e_permute(ctx, A, ops, args, ws)
        log("e2e done")
    # ---- extra operations -------------------------------------------------------------
    del outs
    if not args.no_extra:
        ops_res = {}
        want = set(args.ops.split(","))
        sections = (("extract", "extract", lambda: bench_extract(ctx, args, dev, hbm, ws)),
                    ("assign", "assign", lambda: bench_assign(ctx, args, dev, hbm, ws)),
                    ("batch", "batch_extract", lambda: bench_batch(ctx, args, dev, ws)),
                    ("pbatch", "batch_permute", lambda: bench_pbatch(ctx, args, dev, ws)),
                    ("serve", "serve", lambda: bench_serve(ctx, args, dev)))
        for name, key, fn in sections:
            if name not in want:
                continue
            try:
                ops_res[key] = fn()
                log(f"{name} done")
            except Exception as e:  # noqa: BLE001
                ops_res[key] = {"error": repr(e)[:300]}
            torch.cuda.empty_cache()
        result["ops"] = ops_res
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args)
        log("cpu baseline done")
        result["cpu_baseline_mt"] = cpu_baseline_mt(A, ops[0][1])
        log("multithreaded cpu baseline done")
    ctx.close()
    if rank == 0:
        log_summary(result)
    return result


def e2e_permute(ctx, A, ops, args, ws):
    """Host-resident inputs: H2D of A and p/q, the three ops, D2H of every result."""
    import torch
    from paper_2509_20776_gb300 import CSR
    hA = [t.cpu().pin_memory() for t in (A.rowptr, A.colidx, A.values)]
    hperm = [(p.cpu().pin_memory(), q.cpu().pin_memory() if q is not p else None)
             for _, p, q in ops]
    out_rp = torch.empty_like(hA[0], pin_memory=True)
    out_ci = torch.empty_like(hA[1], pin_memory=True)
    out_v = torch.empty_like(hA[2], pin_memory=True)
    dev = A.rowptr.device
    dA = [torch.empty_like(t, device=dev) for t in hA]
    dperm = [(torch.empty_like(p, device=dev), torch.empty_like(q, device=dev) if q is not None
              else None) for p, q in hperm]
    h2d = sum(t.numel() * t.element_size() for t in hA) + sum(
        p.numel() * p.element_size() + (q.numel() * q.element_size() if q is not None else 0)
        for p, q in hperm)
    d2h = len(ops) * (out_rp.numel() * 8 + out_ci.numel() * 4 + out_v.numel() * 4)

    # Copies of large arrays are cut into NCOPY pieces on NCOPY streams per direction.
    # Steps overlap: the result copies of step k (device -> host) run while step k+1
    # copies its inputs in (host -> device, the link carries both directions at once) and
    # permutes; step k+1 overwrites the device copy of A only after step k's last
    # permutation has read it, and the copy streams keep every result copy in issue
    # order.  The timed region ends after the last result copy of the last step.
    NCOPY = 4
    cps_in = [torch.cuda.Stream(device=dev) for _ in range(NCOPY)]   # host -> device
    cps = [torch.cuda.Stream(device=dev) for _ in range(NCOPY)]      # device -> host

    def pieces(dst, src, streams):
        n = dst.numel()
        for k, st in enumerate(streams):
            a, b = n * k // len(streams), n * (k + 1) // len(streams)
            with torch.cuda.stream(st):
                dst[a:b].copy_(src[a:b], non_blocking=True)

    done = [torch.cuda.Event()]  # the previous step's last permutation (no longer reads dA)
    # results go to a ring of preallocated outputs, RING steps deep: a slot is written again
    # only after its previous result copies have finished (bounded device memory however
    # far the copies lag behind the permutations)
    RING = 3
    ring = [[CSR(A.nrows, A.ncols, torch.empty_like(dA[0]), torch.empty_like(dA[1]), torch.empty_like(dA[2]))
             for _ in ops] for _ in range(RING)]
    copied = [[None for _ in ops] for _ in range(RING)]  # events: the slot's copies are done
    turn = [0]

    def step():
        main = torch.cuda.current_stream()
        slot = turn[0] % RING
        turn[0] += 1
        for st in cps_in:
            st.wait_event(done[0])
        for d, h in zip(dA, hA):
            pieces(d, h, cps_in)
        for st in cps_in:
            main.wait_stream(st)
        Ad = CSR(A.nrows, A.ncols, dA[0], dA[1], dA[2])
        for j, ((dp, dq), (hp, hq)) in enumerate(zip(dperm, hperm)):
            dp.copy_(hp, non_blocking=True)
            if dq is not None:
                dq.copy_(hq, non_blocking=True)
            for ev in copied[slot][j] or []:
                main.wait_event(ev)
            B = ctx.sp_permute(Ad, dp, dq if dq is not None else dp, sync=False, out=ring[slot][j])
            for st in cps:
                st.wait_stream(main)
            for h, t in ((out_rp, B.rowptr), (out_ci, B.colidx), (out_v, B.values)):
                pieces(h, t, cps)
            evs = []
            for st in cps:
                ev = torch.cuda.Event()
                ev.record(st)
                evs.append(ev)
            copied[slot][j] = evs
        done[0] = torch.cuda.Event()
        done[0].record(main)

    def drain():
        main = torch.cuda.current_stream()
        for st in cps:
            main.wait_stream(st)

    steps = max(1, args.steps)
    step()  # warm-up
    drain()
    torch.cuda.synchronize()
    barrier(ws)
    main = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(main)
    for _ in range(steps):
        step()
    drain()
    ev[1].record(main)
    torch.cuda.synchronize()
    barrier(ws)
    ms = ev[0].elapsed_time(ev[1])
    ctx.sync()
    ms = max_over_ranks(ms, ws)
    value = A.nnz * len(ops) * steps * ws / (ms * 1e-3)
    return {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps, "ms_per_step": round(ms / steps, 3),
            "schedule": "steps overlap: result copies of a step run with the next step's input copy and "
                        "permutations (results in a ring of preallocated outputs three steps deep); the "
                        "timed region ends after the last result copy"}


def bench_extract(ctx, args, dev, hbm, ws):
    import torch
    import synth
    from paper_2509_20776_gb300 import CSR
    n = 1 << 26
    A = synth.er_csr(n, n, 32, seed=0, value_kind="f32u01", rowptr_dtype=torch.int64,
                     colidx_dtype=torch.int32, device=dev)
    I = synth.random_subset(n, n // 2, 3, 1, device=dev)
    J = synth.random_subset(n, n // 2, 3, 2, device=dev)
    Ad = CSR(A.nrows, A.ncols, A.rowptr, A.colidx, A.values)
    B = ctx.sp_extract(Ad, I, J)
    nnz_out = B.nnz
    del B
    from paper_2509_20776_gb300 import SP_OPT_TIMING

    def step():
        ctx.sp_extract(Ad, I, J, sync=False)

    steps = max(1, args.steps // 2)
    ctx.phase_stats(reset=True)
    ctx.set_option(SP_OPT_TIMING, 1)
    ms = time_steps(step, steps, 1, ws)
    ctx.sync()
    ctx.set_option(SP_OPT_TIMING, 0)
    phases = {k: round(v[0] / (steps + 1), 3) for k, v in ctx.phase_stats(reset=True).items() if v[1]}
    ms = max_over_ranks(ms, ws)
    # read the columns of the selected rows, read the kept values, write col + val;
    # I, rowptr pairs and J per selected index, the column maps and the output row pointer
    L = (A.rowptr[1:] - A.rowptr[:-1])
    nnz_sel = int(L[I.long()].sum())
    ab = nnz_sel * 4 + nnz_out * 12 + (n // 2) * (4 + 16) + (n // 2) * 4 + n * 4 + (n // 2) * 4 + (n // 2) * 8
    frac = ab * steps / (ms * 1e-3) / 1e9 / hbm
    value = nnz_out * steps * ws / (ms * 1e-3)
    res = {"workload": "ER n=2^26, 32 draws/row; A(I,J), random distinct |I|=|J|=2^25",
           "nnz_in": A.nnz, "nnz_out": nnz_out, "value": round(value, 1), "unit": UNIT,
           "ms_per_op": round(ms / steps, 3), "op_roofline_frac": round(frac, 4),
           "alg_bytes_per_op": ab, "phase_ms_per_op": phases}
    # the contiguous block A(0:n/4, n/4:n/2): each row's kept entries are one segment
    Ic = torch.arange(0, n // 4, dtype=torch.int32, device=dev)
    Jc = torch.arange(n // 4, n // 2, dtype=torch.int32, device=dev)
    B = ctx.sp_extract(Ad, Ic, Jc)
    nnz_c = B.nnz
    del B

    def step_c():
        ctx.sp_extract(Ad, Ic, Jc, sync=False)

    ms_c = max_over_ranks(time_steps(step_c, steps, 1, ws), ws)
    # kept segment read (col + val) and written, I and the rowptr pairs, output row pointer
    ab_c = nnz_c * 16 + (n // 4) * (4 + 16 + 8)
    res["contiguous_block"] = {
        "workload": "same A; A(0:n/4, n/4:n/2)", "nnz_out": nnz_c,
        "value": round(nnz_c * steps * ws / (ms_c * 1e-3), 1), "unit": UNIT,
        "ms_per_op": round(ms_c / steps, 3),
        "op_roofline_frac": round(ab_c * steps / (ms_c * 1e-3) / 1e9 / hbm, 4),
        "alg_bytes_per_op": ab_c}
    del Ad, A, I, J, Ic, Jc
    torch.cuda.empty_cache()
    # road-network stand-in: 5-point mesh with diagonal, 4900 x 4900 grid, fp64 values;
    # I = J = a random eighth of the vertices (short rows, latency-dominated)
    M = synth.mesh5_csr(4900, 4900, device=dev)
    nm = M.nrows
    Im = synth.random_subset(nm, nm // 8, 5, 1, device=dev)
    Md = CSR(M.nrows, M.ncols, M.rowptr, M.colidx, M.values)
    B = ctx.sp_extract(Md, Im, Im)
    nnz_m = B.nnz
    del B

    def step_m():
        ctx.sp_extract(Md, Im, Im, sync=False)

    ms_m = max_over_ranks(time_steps(step_m, steps, 1, ws), ws)
    Lm = (M.rowptr[1:] - M.rowptr[:-1])
    sel_m = int(Lm[Im.long()].sum())
    vb = M.values.element_size()
    ab_m = sel_m * 4 + nnz_m * (vb + 4 + vb) + (nm // 8) * (4 + 16 + 4 + 4 + 8) + nm * 4
    res["mesh"] = {
        "workload": f"5-point mesh 4900x4900 ({M.nnz} entries, fp64); A(I,I), random I of n/8",
        "nnz_out": nnz_m, "value": round(nnz_m * steps * ws / (ms_m * 1e-3), 1), "unit": UNIT,
        "ms_per_op": round(ms_m / steps, 3),
        "op_roofline_frac": round(ab_m * steps / (ms_m * 1e-3) / 1e9 / hbm, 4), "alg_bytes_per_op": ab_m}
    return res


def bench_assign(ctx, args, dev, hbm, ws):
    import torch
    import synth
    from paper_2509_20776_gb300 import CSR
    A = synth.rmat_csr(26, 24, (0.57, 0.19, 0.19, 0.05), seed=0, symmetrize=False,
                       value_kind="f32u01", rowptr_dtype=torch.int64, colidx_dtype=torch.int32,
                       device=dev)
    k = 1 << 22
    Bm = synth.er_csr(k, k, 8, seed=1, value_kind="f32u01", rowptr_dtype=torch.int64,
                      colidx_dtype=torch.int32, device=dev)
    I = synth.random_subset(A.nrows, k, 4, 1, device=dev)
    J = synth.random_subset(A.ncols, k, 4, 2, device=dev)
    Ad = CSR(A.nrows, A.ncols, A.rowptr, A.colidx, A.values)
    Bd = CSR(Bm.nrows, Bm.ncols, Bm.rowptr, Bm.colidx, Bm.values)
    Ap = ctx.sp_assign(Ad, I, J, Bd)
    nnz_out = Ap.nnz
    # extract-after-assign returns B bit-exactly
    E = ctx.sp_extract(CSR(Ap.nrows, Ap.ncols, Ap.rowptr, Ap.colidx, Ap.values), I, J)
    roundtrip = bool(torch.equal(E.rowptr, Bd.rowptr) and torch.equal(E.colidx, Bd.colidx) and
                     torch.equal(E.values.view(torch.int32), Bd.values.view(torch.int32)))
    del Ap, E
    from paper_2509_20776_gb300 import SP_OPT_TIMING

    def step():
        ctx.sp_assign(Ad, I, J, Bd, sync=False)

    steps = max(1, args.steps // 2)
    ctx.phase_stats(reset=True)
    ctx.set_option(SP_OPT_TIMING, 1)
    ms = time_steps(step, steps, 1, ws)
    ctx.sync()
    ctx.set_option(SP_OPT_TIMING, 0)
    phases = {k: round(v[0] / (steps + 1), 3) for k, v in ctx.phase_stats(reset=True).items() if v[1]}
    ms = max_over_ranks(ms, ws)
    m = A.nrows
    ab = A.nnz * 8 + nnz_out * 8 + 2 * (m + 1) * 8 + Bm.nnz * 8 + (k + 1) * 8 + k * 4 + k * 4 + m * 4 + A.ncols // 8
    frac = ab * steps / (ms * 1e-3) / 1e9 / hbm
    value = nnz_out * steps * ws / (ms * 1e-3)
    res = {"workload": "R-MAT scale 26 ef 24; A(I,J)=B, B ER 2^22 x 2^22 8/row, random I,J",
           "nnz_in": A.nnz, "nnz_B": Bm.nnz, "nnz_out": nnz_out, "value": round(value, 1),
           "unit": UNIT, "ms_per_op": round(ms / steps, 3), "op_roofline_frac": round(frac, 4),
           "alg_bytes_per_op": ab, "extract_after_assign_equals_B": roundtrip,
           "phase_ms_per_op": phases}
    # the incremental-update use: the assigned matrix under a random symmetric
    # permutation, fused (one pass) against assign followed by permute
    p = synth.random_permutation(m, 4, 3, device=dev)
    out = ctx.sp_assign_permute(Ad, I, J, Bd, p, p)
    ok = out.nnz == nnz_out
    del out

    def step_fused():
        ctx.sp_assign_permute(Ad, I, J, Bd, p, p, sync=False)

    def step_separate():
        Ap2 = ctx.sp_assign(Ad, I, J, Bd, sync=False)
        ctx.sp_permute(Ap2, p, p, sync=False)

    ms_f = max_over_ranks(time_steps(step_fused, steps, 1, ws), ws)
    ms_s = max_over_ranks(time_steps(step_separate, steps, 1, ws), ws)
    res["assign_permute"] = {
        "workload": "same A, I, J, B; out = P (A(I,J)=B) P^T, random p", "nnz_out": nnz_out,
        "value": round(nnz_out * steps * ws / (ms_f * 1e-3), 1), "unit": UNIT,
        "ms_per_op": round(ms_f / steps, 3), "ms_per_op_assign_then_permute": round(ms_s / steps, 3),
        "nnz_matches_assign": ok}
    # contiguous I, J (a 2^22 x 2^22 block of A replaced by B)
    Ic = torch.arange(A.nrows // 4, A.nrows // 4 + k, dtype=torch.int32, device=dev)
    Jc = torch.arange(A.ncols // 2, A.ncols // 2 + k, dtype=torch.int32, device=dev)
    Apc = ctx.sp_assign(Ad, Ic, Jc, Bd)
    nnz_c = Apc.nnz
    Ec = ctx.sp_extract(CSR(Apc.nrows, Apc.ncols, Apc.rowptr, Apc.colidx, Apc.values), Ic, Jc)
    roundtrip_c = bool(torch.equal(Ec.rowptr, Bd.rowptr) and torch.equal(Ec.colidx, Bd.colidx) and
                       torch.equal(Ec.values.view(torch.int32), Bd.values.view(torch.int32)))
    del Apc, Ec

    def step_c():
        ctx.sp_assign(Ad, Ic, Jc, Bd, sync=False)

    ms_c = max_over_ranks(time_steps(step_c, steps, 1, ws), ws)
    ab_c = A.nnz * 8 + nnz_c * 8 + 2 * (m + 1) * 8 + Bm.nnz * 8 + (k + 1) * 8 + k * 4 + k * 4 + m * 4 + A.ncols // 8
    res["contiguous"] = {
        "workload": "same A and B; I = [m/4, m/4 + 2^22), J = [n/2, n/2 + 2^22)", "nnz_out": nnz_c,
        "value": round(nnz_c * steps * ws / (ms_c * 1e-3), 1), "unit": UNIT, "ms_per_op": round(ms_c / steps, 3),
        "op_roofline_frac": round(ab_c * steps / (ms_c * 1e-3) / 1e9 / hbm, 4), "alg_bytes_per_op": ab_c,
        "extract_after_assign_equals_B": roundtrip_c}
    return res


def batch_workload(dev, nmats=64, nreq=10000, seed=5):
    """64 device-resident power-law matrices (R-MAT, rows 2^10..2^22 log-uniform, edge
    factor 6 symmetrised: ~12 entries per row, fp32) and extraction requests with |I|, |J|
    log-uniform in [16, 65536] (capped at the matrix), I random, J distinct and unsorted."""
    import torch
    import synth
    g = torch.Generator().manual_seed(seed)
    scales = [10 + int(torch.randint(0, 13, (1,), generator=g)) for _ in range(nmats)]
    mats = [synth.rmat_csr(s, 6, seed=200 + t, symmetrize=True, value_kind="f32u01",
                           rowptr_dtype=torch.int64, colidx_dtype=torch.int32, device=dev)
            for t, s in enumerate(scales)]
    gd = torch.Generator(device=dev).manual_seed(seed)
    reqs = []
    for _ in range(nreq):
        mi = int(torch.randint(0, nmats, (1,), generator=g))
        n = mats[mi].nrows
        ki = int(min(n, round(16 * 4096 ** torch.rand(1, generator=g).item())))
        kj = int(min(n, round(16 * 4096 ** torch.rand(1, generator=g).item())))
        I = torch.randint(0, n, (ki,), generator=gd, device=dev, dtype=torch.int32)
        J = torch.unique(torch.randint(0, n, (2 * kj + 8,), generator=gd, device=dev))[:kj]
        J = J[torch.randperm(J.numel(), generator=gd, device=dev)].to(torch.int32)
        reqs.append((mi, I, J))
    return mats, reqs


def bench_batch(ctx, args, dev, ws):
    import time
    import torch
    from paper_2509_20776_gb300 import CSR
    mats, reqs = batch_workload(dev)
    dms = [CSR(m.nrows, m.ncols, m.rowptr, m.colidx, m.values) for m in mats]
    # batched: one count (synchronises once), then the fill replayed from a CUDA graph
    bt = ctx.extract_batch(dms, reqs)
    out = bt.alloc(torch.int64)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.fill(out, s)
    torch.cuda.current_stream().wait_stream(s)
    ctx.sync()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bt.fill(out, torch.cuda.current_stream())
    nnz = bt.nnz
    steps = max(3, args.steps)
    ms_fill = time_steps(graph.replay, steps, 2, ws) / steps
    # the whole batch (identify, count, row pointer, fill, sort) from one graph
    out_r = bt.alloc(torch.int64)
    with torch.cuda.stream(s):
        bt.run(out_r, s)
    torch.cuda.current_stream().wait_stream(s)
    ctx.sync()
    same_run = bool(torch.equal(out_r.rowptr, out.rowptr) and torch.equal(out_r.colidx, out.colidx))
    graph_run = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_run):
        bt.run(out_r, torch.cuda.current_stream())
    ms_run = time_steps(graph_run.replay, steps, 2, ws) / steps
    ctx.sync()
    # algorithmic bytes of the batch: per output row I[i] and the row-pointer pair (read),
    # the output row pointer (write); every selected source column (read); per kept entry
    # its value (read) and column + value (write); J (read)
    sel = 0
    for mi, I, _ in reqs:
        rp, il = mats[mi].rowptr, I.long()
        sel += int((rp[il + 1] - rp[il]).sum())
    nI = sum(I.numel() for _, I, _ in reqs)
    nJ = sum(J.numel() for _, _, J in reqs)
    alg = 28 * nI + 4 * sel + 12 * nnz + 4 * nJ
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        b2 = ctx.extract_batch(dms, reqs)
        o2 = b2.alloc(torch.int64)
        b2.fill(o2)
        ctx.sync()
        b2.close()
    ms_batch = (time.perf_counter() - t0) * 1e3 / 3
    # plain: one count + fill call per request
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_nnz = 0
    for mi, I, J in reqs:
        plain_nnz += ctx.sp_extract(dms[mi], I, J).nnz
    torch.cuda.synchronize()
    ms_plain = (time.perf_counter() - t0) * 1e3
    bt.close()
    res = {"workload": f"{len(mats)} R-MAT matrices (rows 2^10..2^22, ~12/row, {sum(m.nnz for m in mats)} "
                       f"entries); {len(reqs)} extractions, |I|,|J| log-uniform in [16, 65536]",
           "nnz_out": nnz, "same_nnz_as_plain": plain_nnz == nnz,
           "batched_ms": round(ms_batch, 3), "batched_value": round(nnz / (ms_batch * 1e-3), 1),
           "graph_fill_ms": round(ms_fill, 3), "graph_fill_value": round(nnz / (ms_fill * 1e-3), 1),
           "graph_run_ms": round(ms_run, 3), "graph_run_value": round(nnz / (ms_run * 1e-3), 1),
           "graph_run_same_as_fill": same_run,
           "alg_bytes": alg, "selected_source_entries": sel,
           "graph_run_roofline": {"achieved": round(alg / (ms_run * 1e-3) / 1e9, 1), "peak": peak_gbs(),
                                  "unit": "GB/s", "frac": round(alg / (ms_run * 1e-3) / 1e9 / peak_gbs(), 4)},
           "plain_ms": round(ms_plain, 3), "plain_value": round(nnz / (ms_plain * 1e-3), 1),
           "unit": UNIT, "speedup_batched_vs_plain": round(ms_plain / ms_batch, 2)}
    res["autotuned"] = bench_batch_tuned(ctx, dms, reqs, nnz, steps, ws)
    return res


def bench_batch_tuned(ctx, dms, reqs, nnz, steps, ws):
    """The autotuner on the batch itself (rows per warp, tile shape, heavy threshold;
    every candidate's output compared with the default shapes' output), then the batch
    and its graph-replayed fill again with the tuning table installed."""
    import time
    import torch
    from paper_2509_20776_gb300 import autotune

    def run():
        b = ctx.extract_batch(dms, reqs)
        o = b.alloc(torch.int64)
        b.fill(o)
        b.close()
        return o

    t0 = time.perf_counter()
    table = autotune.autotune(ctx, [("batch", 1 << 62, run)], reps=3)
    tune_s = time.perf_counter() - t0
    ctx.set_tuning(table)
    try:
        bt = ctx.extract_batch(dms, reqs)
        out = bt.alloc(torch.int64)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            bt.fill(out, s)
        torch.cuda.current_stream().wait_stream(s)
        ctx.sync()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            bt.fill(out, torch.cuda.current_stream())
        ms_fill = time_steps(graph.replay, steps, 2, ws) / steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            run()
            ctx.sync()
        ms_batch = (time.perf_counter() - t0) * 1e3 / 3
        same = bt.nnz == nnz
        bt.close()
    finally:
        ctx.set_tuning(None)
    e = table["entries"][0]
    return {"shapes": {k: e[k] for k in autotune.KNOBS["batch"]}, "tune_s": round(tune_s, 2),
            "tuner_ms_default": e["default_ms"], "tuner_ms_best": e["ms"], "same_nnz": same,
            "batched_ms": round(ms_batch, 3), "batched_value": round(nnz / (ms_batch * 1e-3), 1),
            "graph_fill_ms": round(ms_fill, 3), "graph_fill_value": round(nnz / (ms_fill * 1e-3), 1)}


def bench_pbatch(ctx, args, dev, ws, nreq=2000, max_rows=1 << 16, seed=6):
    """Batched permutations: `nreq` symmetric reorderings P A P^T over the batching
    workload's matrices of at most `max_rows` rows (the latency-bound end of the serving
    mix), one host-only plan and one fill for the batch, against one call per request.
    A sample of the requests' slices of the batch is compared with their own calls."""
    import time
    import torch
    import synth
    from paper_2509_20776_gb300 import CSR
    mats, _ = batch_workload(dev, nreq=0)
    small = [t for t, m in enumerate(mats) if m.nrows <= max_rows]
    dms = [CSR(m.nrows, m.ncols, m.rowptr, m.colidx, m.values) for m in mats]
    perms = {t: synth.random_permutation(mats[t].nrows, 9, t, device=dev) for t in small}
    g = torch.Generator().manual_seed(seed)
    reqs = []
    for _ in range(nreq):
        t = small[int(torch.randint(0, len(small), (1,), generator=g))]
        reqs.append((t, perms[t], perms[t]))
    bt = ctx.permute_batch(dms, reqs)
    out = bt.alloc(torch.int64)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.fill(out, s)
    torch.cuda.current_stream().wait_stream(s)
    ctx.sync()
    offs = bt.row_offsets()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bt.fill(out, torch.cuda.current_stream())
    nnz = bt.nnz
    steps = max(3, args.steps)
    ms_graph = time_steps(graph.replay, steps, 2, ws) / steps
    ctx.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        b2 = ctx.permute_batch(dms, reqs)
        o2 = b2.alloc(torch.int64)
        b2.fill(o2)
        ctx.sync()
        b2.close()
    ms_batch = (time.perf_counter() - t0) * 1e3 / 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t, p, q in reqs:
        ctx.sp_permute(dms[t], p, q, sync=False)
    ctx.sync()
    torch.cuda.synchronize()
    ms_plain = (time.perf_counter() - t0) * 1e3
    same = True
    for k in range(0, nreq, max(1, nreq // 50)):
        t, p, q = reqs[k]
        alone = ctx.sp_permute(dms[t], p, q)
        a, b = int(out.rowptr[offs[k]]), int(out.rowptr[offs[k + 1]])
        same &= bool(torch.equal(alone.colidx, out.colidx[a:b]) and
                     torch.equal(alone.values.view(torch.int32), out.values[a:b].view(torch.int32)) and
                     torch.equal(alone.rowptr.to(torch.int64), out.rowptr[offs[k]:offs[k + 1] + 1] - a))
    bt.close()
    return {"workload": f"{nreq} P A P^T over the {len(small)} batching-workload matrices of at most "
                        f"{max_rows} rows ({nnz} entries in all)",
            "nnz_out": nnz, "same_as_plain_sampled": same,
            "batched_ms": round(ms_batch, 3), "batched_value": round(nnz / (ms_batch * 1e-3), 1),
            "graph_ms": round(ms_graph, 3), "graph_value": round(nnz / (ms_graph * 1e-3), 1),
            "plain_ms": round(ms_plain, 3), "plain_value": round(nnz / (ms_plain * 1e-3), 1),
            "unit": UNIT, "speedup_batched_vs_plain": round(ms_plain / ms_batch, 2),
            "speedup_graph_vs_plain": round(ms_plain / ms_graph, 2)}


def bench_serve(ctx, args, dev, nreq=100000, nreq_overload=10000):
    """Poisson stream of mixed requests (60 % P A P^T, 30 % extraction, 10 % assignment)
    over the batching workload's 64 matrices: `nreq` requests at 0.8 x the plain path's
    measured capacity and the first `nreq_overload` at 2 x; continuous batching against
    one synchronous call per request."""
    import torch
    import synth
    from paper_2509_20776_gb300 import CSR
    from paper_2509_20776_gb300.serving import Request, Server, latency_stats, run_plain
    mats, ex = batch_workload(dev, nreq=nreq)
    dms = [CSR(m.nrows, m.ncols, m.rowptr, m.colidx, m.values) for m in mats]
    perms = [synth.random_permutation(m.nrows, 7, t, device=dev) for t, m in enumerate(mats)]
    k2 = 256
    Bm = synth.er_csr(k2, k2, 4, seed=9, value_kind="f32u01", rowptr_dtype=torch.int64,
                      colidx_dtype=torch.int32, device=dev)
    Bd = CSR(Bm.nrows, Bm.ncols, Bm.rowptr, Bm.colidx, Bm.values)
    g = torch.Generator().manual_seed(11)
    kinds = torch.rand(nreq, generator=g)

    def make(arrivals):
        reqs = []
        for k in range(nreq):
            mi, I, J = ex[k]
            if kinds[k] < 0.6:
                reqs.append(Request("permute", mi, arrivals[k], p=perms[mi]))
            elif kinds[k] < 0.9:
                reqs.append(Request("extract", mi, arrivals[k], I=I, J=J))
            else:
                m = mats[mi].nrows
                sel = perms[mi][:2 * k2]
                reqs.append(Request("assign", mi, arrivals[k], I=sel[:k2], J=sel[k2:2 * k2] if m >= 2 * k2 else sel[:k2],
                                    B=Bd))
        return reqs

    # capacity of the plain path: a sample served back to back
    ns = min(500, nreq)
    sample = make([0.0] * nreq)[:ns]
    run_plain(ctx, dms, sample)
    cap = ns / max(max(r.done for r in sample), 1e-9)
    res = {"workload": f"{nreq} requests at 0.8x, {nreq_overload} at 2x (60/30/10 % permute/extract/assign) "
                       f"on the batching workload's {len(mats)} matrices, Poisson arrivals",
           "plain_capacity_per_s": round(cap, 1), "unit": UNIT}
    srv = Server(dms, slots=4)
    for load, nr in ((0.8, nreq), (2.0, nreq_overload)):  # below and above the plain path's capacity
        rate = load * cap
        gaps = torch.empty(nreq, dtype=torch.float64).exponential_(rate, generator=g)
        arrivals = torch.cumsum(gaps, 0).tolist()
        plain = run_plain(ctx, dms, make(arrivals)[:nr])
        srv.stats = {k: 0 for k in srv.stats}
        served = srv.run(make(arrivals)[:nr])
        nnz_p = sum(r.nnz_out for r in plain)
        nnz_s = sum(r.nnz_out for r in served)
        sp, ss = latency_stats(plain), latency_stats(served)
        res[f"load_{load}x"] = {"rate_per_s": round(rate, 1), "requests": nr,
                                "plain": {**sp, "value": round(nnz_p / sp["span_s"], 1)},
                                "served": {**ss, "value": round(nnz_s / ss["span_s"], 1)},
                                "same_nnz": nnz_p == nnz_s, "server_stats": dict(srv.stats)}
    srv.close()
    return res


# ---------------------------------------------------------------------------------------
CPU_SCALE = 20


def _cpu_sample(scale, seed_perm, device):
    """The headline generator at a smaller scale, copied to host numpy for the oracle."""
    import numpy as np
    import torch
    import oracle
    import synth
    A = synth.rmat_csr(scale, 16, (0.57, 0.19, 0.19, 0.05), seed=0, symmetrize=True,
                       value_kind="f32u01", device=device)
    O = oracle.CSR.of(A.nrows, A.ncols, A.rowptr.cpu().numpy(), A.colidx.cpu().numpy(),
                      A.values.cpu().numpy())
    p = synth.random_permutation(A.nrows, seed_perm, 0, device=device).cpu().numpy()
    pd = synth.degree_descending_permutation(A.rowptr).cpu().numpy()
    q = synth.random_permutation(A.nrows, seed_perm, 1, device=device).cpu().numpy()
    del np, torch
    return O, [(p, p), (pd, pd), (p, q)]


def cpu_baseline(args):
    """The oracle (numpy, as it stands) on host cores, one P A P^T on a scale-20 sample."""
    import oracle
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    O, perms = _cpu_sample(CPU_SCALE, 1, dev)
    p, q = perms[0]
    t = time.perf_counter()
    B = oracle.permute(O, p, q)
    dt = time.perf_counter() - t
    return {"value": round(B.nnz / dt, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"R-MAT scale {CPU_SCALE} (same a,b,c,d, edge factor 16, symmetrised, "
                      f"{O.nnz} nnz), one P A P^T with a random p, {dt:.1f} s"}


def _mem_available() -> int:
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:  # noqa: BLE001
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_mt(A, p):
    """The multithreaded CPU restatement of Algorithm 2 (oracle/cpu_mt.cpp: count, scan,
    fill, per-row sort; OpenMP on every host thread) on the headline matrix itself, one
    P A P^T with the workload's random p.  Skipped when the host lacks the memory."""
    import numpy as np
    from oracle import cpu_mt
    need = A.nnz * 8 * 2 + A.nrows * 8 * 3 + A.ncols * 4
    avail = _mem_available()
    if avail < 1.5 * need:
        return {"skipped": f"host memory: {avail >> 30} GiB available, {int(1.5 * need) >> 30} GiB wanted"}
    rp, ci, vv = A.rowptr.cpu().numpy(), A.colidx.cpu().numpy(), A.values.cpu().numpy()
    pn = p.cpu().numpy().astype(np.int64)
    t = time.perf_counter()
    cpu_mt.permute(A.nrows, A.ncols, rp, ci, vv, pn)
    dt = time.perf_counter() - t
    return {"value": round(A.nnz / dt, 1), "unit": UNIT, "cores": cpu_mt.threads(), "nproc": os.cpu_count(),
            "cpu_model": _cpu_model(), "kind": "openmp restatement of Algorithm 2 (count, scan, fill, per-row sort)",
            "sample": f"the headline matrix ({A.nnz} entries), one P A P^T with the random p, {dt:.2f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle on a bounded sample per step (scale-18 R-MAT)."""
    import oracle
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    scale = 18
    O, perms = _cpu_sample(scale, 1, dev)

    def step():
        for p, q in perms:
            oracle.permute(O, p, q)

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t
    value = O.nnz * len(perms) * args.steps / dt
    sample = (f"R-MAT scale {scale} (same a,b,c,d, edge factor 16, symmetrised, {O.nnz} nnz); "
              "each step the three permutations of the workload")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64 indices / fp32 values",
            "data": "synthetic (seeded R-MAT)",
            "config": {"workload": WORKLOAD.format(scale=args.scale), "sample": sample},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def lookup_sweep():
    """Rate of uniform random 4-byte lookups (torch.index_select, 2^28 lookups, index read
    and result write included) into int32 tables of 8 MB to 1 GB: where a relabel map stops
    being L2-resident."""
    import torch
    dev = torch.device("cuda", 0)
    rows = []
    for mb in (8, 16, 32, 64, 96, 112, 128, 160, 256, 1024):
        n = mb * (1 << 20) // 4
        t = torch.arange(n, dtype=torch.int32, device=dev)
        g = torch.Generator(device=dev).manual_seed(mb)
        idx = torch.randint(0, n, (1 << 28,), generator=g, device=dev, dtype=torch.int32)
        out = torch.empty(1 << 28, dtype=torch.int32, device=dev)
        torch.index_select(t, 0, idx, out=out)
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            torch.index_select(t, 0, idx, out=out)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        rows.append({"table_mb": mb, "ms": round(best, 3), "g_lookups_per_s": round((1 << 28) / best / 1e6, 1)})
        del t, idx, out
        torch.cuda.empty_cache()
    return {"lookup_sweep": rows}


def main():
    args = parse()
    if args.lookup_sweep:
        print(json.dumps(lookup_sweep()), flush=True)
        return
    if args.profile_case:
        profile_case(args)
        return
    ws, rank, local = dist_init()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    res = run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
