"""Autotuner for the library's run-time kernel shapes.

The shapes (``SP_OPT_TILE_SHAPE``, ``SP_OPT_HEAVY``, ``SP_OPT_COUNT_ROWS``,
``SP_OPT_FILL_ROWS``, ``SP_OPT_BATCH_ROWS``, ``SP_OPT_IDENTIFY`` in ``include/sp.h``)
change how the kernels split the work or identify kept columns, never the output.  For each (op, size class) the tuner times candidate
shapes on a representative workload through the library's own calls, checks that every
candidate's output is bit-identical to the one of the default shapes, and writes a table
that ``Context.set_tuning`` installs: afterwards every call of that op whose size falls in
the class runs with the chosen shapes (the C library looks the entry up per call).

Search: coordinate descent, one knob at a time over its candidate values with the other
knobs held at the best so far; each candidate is the median of ``reps`` CUDA-event
timings after one warm-up run, and replaces the best only when it is faster by more than
``margin`` (so noise does not move the table away from the defaults).

Command line (seeded synthetic workloads of the library's own classes, on cuda:0):
    python -m paper_2509_20776_gb300.autotune --out tuning.json [--quick]
"""
from __future__ import annotations

import json

import torch

from ._binding import SHAPE_VALUES, Context

# knobs each op's kernels read, in the order they are tuned
KNOBS = {
    "permute": ("tile_shape", "heavy"),
    "extract": ("identify", "tile_shape", "heavy"),
    "assign": ("count_rows", "fill_rows", "tile_shape", "heavy"),
    "batch": ("identify", "batch_rows", "tile_shape", "heavy"),
}
SEARCH = {"tile_shape": (0, 1), "heavy": (128, 256, 512), "count_rows": (1, 2, 4), "fill_rows": (1, 2),
          "batch_rows": (1, 2, 4, 8), "identify": (0, 1)}
DEFAULT = {"tile_shape": 0, "heavy": 128, "count_rows": 4, "fill_rows": 2, "batch_rows": 1, "identify": 0}
assert all(set(v) <= set(SHAPE_VALUES[k]) for k, v in SEARCH.items())


def _flatten(out) -> list:
    """The tensors of an op's result (a CSR-like object or nested tuples / lists)."""
    if isinstance(out, torch.Tensor):
        return [out]
    if hasattr(out, "rowptr"):
        return [out.rowptr, out.colidx, out.values]
    if isinstance(out, (tuple, list)):
        return [t for o in out for t in _flatten(o)]
    return []


_BITS = {torch.float32: torch.int32, torch.float64: torch.int64, torch.float16: torch.int16,
         torch.bfloat16: torch.int16}


def _bits(t: torch.Tensor) -> torch.Tensor:
    """Floating tensors as their bit patterns (so -0.0 differs from 0.0, NaN payloads count)."""
    return t.view(_BITS[t.dtype]) if t.dtype in _BITS else t


def _same(a, b) -> bool:
    """Bit-for-bit equality of two results."""
    ta, tb = _flatten(a), _flatten(b)
    return len(ta) == len(tb) and all(x.dtype == y.dtype and x.shape == y.shape and
                                      torch.equal(_bits(x), _bits(y)) for x, y in zip(ta, tb))


def _time(run, reps: int):
    out = run()  # warm-up; its result is the one compared
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sorted(ts)[len(ts) // 2], out


def tune_case(ctx: Context, op: str, run, reps: int = 3, margin: float = 0.02) -> dict:
    """Best shapes for one workload.  ``run()`` issues the op through ``ctx`` (the shapes
    set on the context apply to it) and returns its result; the context's shapes are
    restored to the defaults afterwards."""
    best = dict(DEFAULT)
    try:
        ctx.set_shapes(**best)
        base_ms, ref = _time(run, reps)
        best_ms = base_ms
        for knob in KNOBS[op]:
            for v in SEARCH[knob]:
                if v == best[knob]:
                    continue
                trial = dict(best, **{knob: v})
                ctx.set_shapes(**trial)
                ms, out = _time(run, reps)
                if not _same(out, ref):
                    raise RuntimeError(f"autotune {op}: shapes {trial} changed the output")
                del out
                if ms < best_ms * (1.0 - margin):
                    best, best_ms = trial, ms
    finally:
        ctx.set_shapes(**{k: -1 for k in DEFAULT})
    return {"op": op, **{k: best[k] for k in KNOBS[op]}, "ms": round(best_ms, 4), "default_ms": round(base_ms, 4)}


def autotune(ctx: Context, cases, reps: int = 3, margin: float = 0.02) -> dict:
    """``cases``: (op, size_max, run) triples, one representative workload per size
    class (size: nnz(A), or the total selected rows of a batch).  Returns the table."""
    entries = []
    for op, size_max, run in cases:
        e = tune_case(ctx, op, run, reps, margin)
        e["size_max"] = int(size_max)
        entries.append(e)
    props = torch.cuda.get_device_properties(ctx.device)
    return {"format": "sp-tuning-1", "device": props.name, "sm_count": props.multi_processor_count,
            "entries": entries}


def save(table: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        table = json.load(f)
    if table.get("format") != "sp-tuning-1":
        raise ValueError(f"{path}: not a tuning table")
    return table


def _default_cases(ctx: Context, quick: bool):
    """Seeded synthetic workloads: R-MAT permutations and extractions per size class,
    and a batch of small extractions."""
    import synth  # seeded generators (repository-level module)
    from ._binding import CSR, ExtractBatch

    dev = torch.device("cuda", ctx.device)
    scales = (16, 20) if quick else (16, 20, 23)
    cases = []
    for sc in scales:
        A = synth.rmat_csr(sc, 16, (0.57, 0.19, 0.19, 0.05), seed=0, symmetrize=True, value_kind="f32u01",
                           rowptr_dtype=torch.int64, colidx_dtype=torch.int32, device=dev)
        Ad = CSR(A.nrows, A.ncols, A.rowptr, A.colidx, A.values)
        p = synth.random_permutation(A.nrows, 1, 0, device=dev)
        size_max = (1 << 62) if sc == scales[-1] else A.nnz * 8
        cases.append(("permute", size_max, lambda Ad=Ad, p=p: ctx.sp_permute(Ad, p, p)))
        n2 = A.nrows // 2
        I = synth.random_permutation(A.nrows, 2, 0, device=dev)[:n2].contiguous()
        J = synth.random_permutation(A.ncols, 2, 1, device=dev)[:n2].contiguous()
        cases.append(("extract", size_max, lambda Ad=Ad, I=I, J=J: ctx.sp_extract(Ad, I, J)))
    # a batch of small extractions over a few matrices
    g = torch.Generator().manual_seed(3)
    mats = []
    for k, sc in enumerate((12, 14, 16, 18)):
        M = synth.rmat_csr(sc, 6, (0.57, 0.19, 0.19, 0.05), seed=10 + k, symmetrize=True, value_kind="f32u01",
                           rowptr_dtype=torch.int64, colidx_dtype=torch.int32, device=dev)
        mats.append(CSR(M.nrows, M.ncols, M.rowptr, M.colidx, M.values))
    reqs = []
    for r in range(500 if quick else 2000):
        m = int(torch.randint(len(mats), (1,), generator=g))
        nr = mats[m].nrows
        ni = int(min(nr, 2 ** float(torch.empty(1).uniform_(4, 12, generator=g))))
        nj = int(min(nr, 2 ** float(torch.empty(1).uniform_(4, 12, generator=g))))
        I = torch.randperm(nr, generator=g)[:ni].to(dev)
        J = torch.randperm(nr, generator=g)[:nj].to(dev)
        reqs.append((m, I, J))

    def run_batch():
        bt = ExtractBatch(ctx, mats, reqs)
        out = bt.alloc()
        bt.fill(out)
        bt.close()
        return out

    cases.append(("batch", 1 << 62, run_batch))  # one class: batches mix every size
    return cases


def main(argv=None) -> int:
    import argparse

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default="tuning.json")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--quick", action="store_true", help="smaller workloads")
    args = ap.parse_args(argv)
    ctx = Context(0)
    table = autotune(ctx, _default_cases(ctx, args.quick), reps=args.reps)
    save(table, args.out)
    for e in table["entries"]:
        print(json.dumps(e))
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
