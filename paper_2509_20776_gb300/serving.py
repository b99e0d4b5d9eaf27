"""Continuous-batching request server over device-resident matrices.

Requests (permute / extract / assign on one of the registered matrices) arrive over
time.  Every scheduling round the server
  * retires the requests whose work has finished on the device (latency = completion
    time seen by the host - arrival time);
  * admits the requests that have arrived, in arrival order, while their output bound
    fits the device-memory budget (permutation: nnz(A); assignment: nnz(A) + nnz(B));
  * counts the round's extractions as one batch (``ExtractBatch``: one count for the
    whole round) and admits the batch by the exact output bytes that count returns: a
    batch that does not fit is held, counted but not filled, until retiring work frees
    enough memory (later extractions wait behind it, in order);
  * runs the round's permutations of small matrices (at most ``perm_batch_nnz``
    entries) as one batch (``PermuteBatch``: a host-only plan and one fill for all of
    them); larger ones, whose launches are amortised already, and a lone small one are
    plain calls, so a small request never waits for a large one in its batch;
  * fills admitted batches and issues the permutation batches, permutations and
    assignments round-robin on several stream slots, each with its own library
    context, so their work overlaps.
Requests that arrive while others are on the GPU join the next round: slots and memory
free up as earlier work retires.  ``run_plain`` serves the same stream one synchronous
call per request, for comparison.  Every kernel is the library's; this module only
schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import torch

from ._binding import CSR, Context, ExtractBatch, PermuteBatch, mat_descs


@dataclass
class Request:
    kind: str            # "permute" | "extract" | "assign"
    mat: int             # index of the matrix handle
    arrival: float       # seconds from the start of the stream
    p: torch.Tensor | None = None   # permute: row / column permutation (P A P^T)
    I: torch.Tensor | None = None   # extract / assign
    J: torch.Tensor | None = None
    B: CSR | None = None            # assign
    done: float = -1.0
    nnz_out: int = 0
    result: CSR | tuple | None = None


def _bytes(m: CSR) -> int:
    return m.nnz * (m.colidx.element_size() + m.values.element_size()) + (m.nrows + 1) * 8


@dataclass
class Server:
    mats: list[CSR]
    slots: int = 4
    mem_budget: int = 16 << 30      # bytes of outputs in flight
    max_batch: int = 4096           # extractions per round
    perm_batch_nnz: int = 1 << 20   # permutations of matrices up to this size are batched
    keep_results: bool = False
    device: int = 0
    _ctx: list = field(default_factory=list)
    _streams: list = field(default_factory=list)
    _last: list = field(default_factory=list)  # per slot: event of its latest work
    stats: dict = field(default_factory=dict)

    def __post_init__(self):
        self._ctx = [Context(self.device) for _ in range(self.slots)]
        self._streams = [torch.cuda.Stream(self.device) for _ in range(self.slots)]
        self._last = [None] * self.slots
        self._descs = mat_descs(self.mats)  # built once: the batch calls reuse it
        self.stats = {"rounds": 0, "batches": 0, "perm_batches": 0, "held_rounds": 0, "peak_used": 0}

    def close(self):
        for c in self._ctx:
            c.close()

    def _bound(self, r: Request) -> int:
        a = self.mats[r.mat]
        if r.kind == "permute":
            return _bytes(a)
        if r.kind == "assign":
            return _bytes(a) + _bytes(r.B)
        return 0  # extractions are admitted by their batch's exact count (below)

    @staticmethod
    def _batch_bytes(bt: ExtractBatch) -> int:
        like = bt.mats[0]
        return bt.nnz * (like.colidx.element_size() + like.values.element_size()) + (bt.rows + 1) * 8

    def _slot(self, turn: int) -> int:
        """An idle slot if there is one (a call that synchronises, such as an extraction
        count, then waits for nothing else), else the next in turn."""
        for j in range(self.slots):
            k = (turn + j) % self.slots
            if self._last[k] is None or self._last[k].query():
                return k
        return turn % self.slots

    def run(self, reqs: list[Request]) -> list[Request]:
        """Serve ``reqs`` (sorted by arrival); fills ``done`` / ``nnz_out`` of each."""
        t0 = time.perf_counter()
        i, n = 0, len(reqs)
        inflight: list[tuple[list[Request], torch.cuda.Event, int, object]] = []
        held = None  # (requests, counted batch, slot, bytes): waiting for memory
        used = 0
        turn = 0
        while i < n or inflight or held:
            now = time.perf_counter() - t0
            # retire finished work (in issue order is not required)
            still = []
            for group, ev, nbytes, keep in inflight:
                if ev.query():
                    tdone = time.perf_counter() - t0
                    for r in group:
                        r.done = tdone
                    if isinstance(keep, tuple):  # an extraction batch: per-request sizes
                        _, out, offs = keep
                        rp = out.rowptr.cpu()
                        for j, r in enumerate(group):
                            r.nnz_out = int(rp[offs[j + 1]] - rp[offs[j]])
                    used -= nbytes
                else:
                    still.append((group, ev, nbytes, keep))
            inflight = still
            # admit what has arrived
            ex, other = [], []
            while i < n and reqs[i].arrival <= now:
                r = reqs[i]
                if r.kind == "extract":
                    if held is not None or len(ex) >= self.max_batch:
                        break  # extractions stay in order behind a held batch
                    ex.append(r)
                    i += 1
                    continue
                b = self._bound(r)
                if used + b > self.mem_budget and (inflight or ex or other or held):
                    break  # wait for memory to free up
                other.append(r)
                used += b
                i += 1
            small = [r for r in other if r.kind == "permute" and self.mats[r.mat].nnz <= self.perm_batch_nnz]
            if len(small) > 1:  # the round's small permutations as one batch
                k = self._slot(turn)
                turn = k + 1
                ctx, st = self._ctx[k], self._streams[k]
                with torch.cuda.stream(st):
                    pb = PermuteBatch(ctx, self.mats, [(r.mat, r.p, r.p) for r in small], stream=st,
                                      descs=self._descs)
                    out = pb.alloc()
                    pb.fill(out, st)
                    offs = pb.row_offsets()
                    pb.close()  # stream-ordered after the fill
                    for j, r in enumerate(small):
                        r.nnz_out = self.mats[r.mat].nnz
                        if self.keep_results:
                            r.result = (out, offs[j], offs[j + 1])
                    ev = torch.cuda.Event()
                    ev.record(st)
                    self._last[k] = ev
                inflight.append((small, ev, sum(self._bound(r) for r in small), out))
                self.stats["perm_batches"] += 1
                batched = set(map(id, small))
                other = [r for r in other if id(r) not in batched]
            for r in other:
                k = self._slot(turn)
                turn = k + 1
                ctx, st = self._ctx[k], self._streams[k]
                a = self.mats[r.mat]
                with torch.cuda.stream(st):
                    if r.kind == "permute":
                        out = ctx.sp_permute(a, r.p, r.p, stream=st, sync=False)
                    else:
                        out = ctx.sp_assign(a, r.I, r.J, r.B, stream=st, sync=False)
                    r.nnz_out = out.nnz
                    if self.keep_results:
                        r.result = out
                    ev = torch.cuda.Event()
                    ev.record(st)
                    self._last[k] = ev
                inflight.append(([r], ev, self._bound(r), out))
            if ex:  # count the round's extractions as one batch
                k = self._slot(turn)
                turn = k + 1
                ctx, st = self._ctx[k], self._streams[k]
                with torch.cuda.stream(st):
                    bt = ExtractBatch(ctx, self.mats, [(r.mat, r.I, r.J) for r in ex], stream=st,
                                      descs=self._descs)
                held = (ex, bt, k, self._batch_bytes(bt))
                self.stats["batches"] += 1
            if held is not None:
                ex_h, bt, k, nbytes = held
                if used + nbytes <= self.mem_budget or not inflight:
                    ctx, st = self._ctx[k], self._streams[k]
                    with torch.cuda.stream(st):
                        out = bt.alloc()
                        bt.fill(out, st)
                        offs = bt.row_offsets()
                        if self.keep_results:
                            for j, r in enumerate(ex_h):
                                r.result = (out, offs[j], offs[j + 1])
                        ev = torch.cuda.Event()
                        ev.record(st)
                        self._last[k] = ev
                    used += nbytes
                    inflight.append((ex_h, ev, nbytes, (bt, out, offs)))
                    held = None
                else:
                    self.stats["held_rounds"] += 1
            self.stats["peak_used"] = max(self.stats["peak_used"], used)
            self.stats["rounds"] += 1
            if not other and not ex and held is None and not inflight and i < n:
                while time.perf_counter() - t0 < reqs[i].arrival:  # idle until the next arrival
                    pass
        torch.cuda.synchronize()
        for c in self._ctx:
            c.sync()
        return reqs


def run_plain(ctx: Context, mats: list[CSR], reqs: list[Request], keep_results=False) -> list[Request]:
    """One synchronous library call per request, in arrival order (the baseline)."""
    t0 = time.perf_counter()
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival:
            pass
        a = mats[r.mat]
        if r.kind == "permute":
            out = ctx.sp_permute(a, r.p, r.p)
        elif r.kind == "extract":
            out = ctx.sp_extract(a, r.I, r.J)
        else:
            out = ctx.sp_assign(a, r.I, r.J, r.B)
        r.nnz_out = out.nnz
        r.done = time.perf_counter() - t0
        if keep_results:
            r.result = out
    return reqs


def latency_stats(reqs: list[Request]) -> dict:
    lat = torch.tensor([r.done - r.arrival for r in reqs], dtype=torch.float64)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    by_kind = {}
    for kind in sorted({r.kind for r in reqs}):
        lk = torch.tensor([r.done - r.arrival for r in reqs if r.kind == kind], dtype=torch.float64)
        by_kind[kind] = {"n": int(lk.numel()), "p50_ms": round(float(lk.quantile(0.5)) * 1e3, 3),
                         "p99_ms": round(float(lk.quantile(0.99)) * 1e3, 3)}
    return {"p50_ms": round(float(lat.quantile(0.5)) * 1e3, 3),
            "p99_ms": round(float(lat.quantile(0.99)) * 1e3, 3),
            "mean_ms": round(float(lat.mean()) * 1e3, 3), "span_s": round(span, 3), "by_kind": by_kind}
