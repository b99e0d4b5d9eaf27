"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This module holds no arithmetic of the sparse primitives themselves: it only draws
matrices and index vectors.  Every random number comes from a counter-based hash
(MurmurHash3's 32-bit finaliser ``fmix32``, applied to a (seed, stream, counter)
triple), evaluated with exact 64-bit integer tensor operations.  The same call
therefore yields the same tensors on the CPU and on a GPU, and any element can be
regenerated on its own.

Matrix families (the paper's SuiteSparse inputs are not available; these stand in
for its graph classes):

* Erdos-Renyi (``er_csr``): each row draws ``draws`` columns uniformly, duplicates
  merged -- stands in for GAP-urand.
* R-MAT (``rmat_csr``): recursive quadrant choice with probabilities (a, b, c, d) and no
  noise, optional symmetrisation, duplicates merged -- stands in for the power-law
  social and web graphs (twitter7, GAP-web, uk-2002).
* 2-D 5-point mesh with the diagonal (``mesh5_csr``) -- stands in for GAP-road /
  europe_osm.

Values are drawn after canonicalisation from the global position of the stored entry:
fp32 U(0,1) from 24 random bits, fp64 U(-1,1) from 53 random bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

MASK32 = 0xFFFFFFFF

# stream identifiers (the "stream" part of the hash key); fixed so inputs are stable
S_ER_COL = 1
S_VALUE = 2
S_VALUE_LO = 3
S_PERM = 4
S_SUBSET = 5
S_RMAT = 100  # + level


def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2**32 for int64 tensors holding values in [0, 2**32), without overflow."""
    lo, hi = c & 0xFFFF, c >> 16
    return (x * lo + (((x * hi) & 0xFFFF) << 16)) & MASK32


def fmix32(x: torch.Tensor) -> torch.Tensor:
    """MurmurHash3 32-bit finaliser (Appleby), on int64 tensors holding 32-bit values."""
    x = x ^ (x >> 16)
    x = _mul32(x, 0x85EBCA6B)
    x = x ^ (x >> 13)
    x = _mul32(x, 0xC2B2AE35)
    x = x ^ (x >> 16)
    return x


def _fmix32_int(x: int) -> int:
    x &= MASK32
    x ^= x >> 16
    x = (x * 0x85EBCA6B) & MASK32
    x ^= x >> 13
    x = (x * 0xC2B2AE35) & MASK32
    x ^= x >> 16
    return x


def hash32(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """32 random bits for each counter in ``idx`` (int64, >= 0) under key (seed, stream)."""
    k1 = _fmix32_int(seed * 0x9E3779B1 + stream * 0x85EBCA77 + 0x27D4EB2F)
    k2 = _fmix32_int(k1 ^ 0x165667B1 ^ (stream << 7))
    idx = idx.to(torch.int64)
    x = fmix32((idx & MASK32) ^ k1)
    x = fmix32(x ^ ((idx >> 32) & MASK32) ^ k2)
    return x


def uniform_below(h: torch.Tensor, n: int) -> torch.Tensor:
    """Map 32-bit hashes to [0, n) by multiply-shift (n <= 2**31)."""
    assert 0 < n <= (1 << 31)
    return (h * n) >> 32


@dataclass
class CSRTensors:
    """A CSR matrix as four tensors (any device)."""
    nrows: int
    ncols: int
    rowptr: torch.Tensor
    colidx: torch.Tensor
    values: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    def to(self, device) -> "CSRTensors":
        return CSRTensors(self.nrows, self.ncols, self.rowptr.to(device),
                          self.colidx.to(device), self.values.to(device))

    def astype(self, rowptr_dtype=None, colidx_dtype=None) -> "CSRTensors":
        return CSRTensors(self.nrows, self.ncols,
                          self.rowptr.to(rowptr_dtype or self.rowptr.dtype),
                          self.colidx.to(colidx_dtype or self.colidx.dtype), self.values)


def draw_values(nnz: int, seed: int, kind: str, device, start: int = 0,
                chunk: int = 1 << 26) -> torch.Tensor:
    """Values for stored entries ``start .. start+nnz`` (global positions).

    kind 'f32u01': fp32 U(0,1) from 24 bits; 'f64um11': fp64 U(-1,1) from 53 bits.
    """
    if nnz > chunk:
        dt = torch.float32 if kind == "f32u01" else torch.float64
        out = torch.empty(nnz, dtype=dt, device=device)
        for s0 in range(0, nnz, chunk):
            s1 = min(nnz, s0 + chunk)
            out[s0:s1] = draw_values(s1 - s0, seed, kind, device, start + s0, chunk)
        return out
    pos = torch.arange(start, start + nnz, dtype=torch.int64, device=device)
    if kind == "f32u01":
        h = hash32(seed, S_VALUE, pos)
        return (h >> 8).to(torch.float32) * (2.0 ** -24)
    if kind == "f64um11":
        h1 = hash32(seed, S_VALUE, pos)
        h2 = hash32(seed, S_VALUE_LO, pos)
        u = ((h1 << 21) | (h2 >> 11)).to(torch.float64) * (2.0 ** -53)
        return 2.0 * u - 1.0
    raise ValueError(kind)


def _finish(nrows, ncols, counts, colidx, seed, value_kind, rowptr_dtype, colidx_dtype, device):
    rowptr = torch.zeros(nrows + 1, dtype=torch.int64, device=device)
    if nrows:
        torch.cumsum(counts, 0, out=rowptr[1:])
    nnz = int(colidx.numel())
    values = draw_values(nnz, seed, value_kind, device)
    if rowptr_dtype == torch.int32:
        assert nnz <= 2**31 - 1, "nnz does not fit an int32 row pointer"
    return CSRTensors(nrows, ncols, rowptr.to(rowptr_dtype), colidx.to(colidx_dtype), values)


def er_csr(nrows: int, ncols: int, draws: int, seed: int = 0, value_kind: str = "f32u01",
           rowptr_dtype=torch.int64, colidx_dtype=torch.int32, device="cpu",
           chunk_rows: int = 1 << 20) -> CSRTensors:
    """Erdos-Renyi CSR: each row draws ``draws`` uniform columns; duplicates merged."""
    device = torch.device(device)
    counts = torch.zeros(nrows, dtype=torch.int64, device=device)
    out = torch.empty(nrows * draws, dtype=colidx_dtype, device=device)
    fill = 0
    for r0 in range(0, nrows, chunk_rows):
        r1 = min(nrows, r0 + chunk_rows)
        idx = torch.arange(r0 * draws, r1 * draws, dtype=torch.int64, device=device)
        c = uniform_below(hash32(seed, S_ER_COL, idx), ncols).view(r1 - r0, draws)
        c = torch.sort(c, dim=1).values
        keep = torch.ones_like(c, dtype=torch.bool)
        keep[:, 1:] = c[:, 1:] != c[:, :-1]
        counts[r0:r1] = keep.sum(1)
        sel = c[keep]
        out[fill:fill + sel.numel()] = sel.to(colidx_dtype)
        fill += sel.numel()
        del idx, c, keep, sel
    return _finish(nrows, ncols, counts, out[:fill].clone() if fill < out.numel() else out,
                   seed, value_kind, rowptr_dtype, colidx_dtype, device)


def rmat_keys(scale: int, nedges: int, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 0,
              symmetrize: bool = False, device="cpu", chunk: int = 1 << 25) -> torch.Tensor:
    """Sorted, de-duplicated edge keys ``src << scale | dst`` of an R-MAT graph."""
    device = torch.device(device)
    a, b, c, _ = abcd
    ta = int(math.floor(a * 2**32))
    tab = int(math.floor((a + b) * 2**32))
    tabc = int(math.floor((a + b + c) * 2**32))
    parts = []
    for e0 in range(0, nedges, chunk):
        e1 = min(nedges, e0 + chunk)
        idx = torch.arange(e0, e1, dtype=torch.int64, device=device)
        src = torch.zeros_like(idx)
        dst = torch.zeros_like(idx)
        for lvl in range(scale):
            u = hash32(seed, S_RMAT + lvl, idx)
            sbit = (u >= tab).to(torch.int64)
            dbit = (((u >= ta) & (u < tab)) | (u >= tabc)).to(torch.int64)
            src = src * 2 + sbit
            dst = dst * 2 + dbit
            del u, sbit, dbit
        parts.append((src << scale) | dst)
        if symmetrize:
            parts.append((dst << scale) | src)
        del idx, src, dst
    keys = torch.cat(parts) if len(parts) > 1 else parts[0]
    del parts
    keys = torch.sort(keys).values
    if keys.numel() > 1:
        keep = torch.ones_like(keys, dtype=torch.bool)
        keep[1:] = keys[1:] != keys[:-1]
        keys = keys[keep]
    return keys


def rmat_csr(scale: int, edge_factor: int, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 0,
             symmetrize: bool = False, value_kind: str = "f32u01", rowptr_dtype=torch.int64,
             colidx_dtype=torch.int32, device="cpu", nrows: int | None = None) -> CSRTensors:
    """R-MAT CSR of ``2**scale`` vertices and ``edge_factor * 2**scale`` drawn edges.

    With ``nrows`` < 2**scale the graph is cut to its leading nrows x nrows block.
    """
    n = 1 << scale
    keys = rmat_keys(scale, edge_factor * n, abcd, seed, symmetrize, device)
    rows = keys >> scale
    cols = keys & (n - 1)
    del keys
    m = n if nrows is None else nrows
    if m < n:
        keep = (rows < m) & (cols < m)
        rows, cols = rows[keep], cols[keep]
    counts = torch.bincount(rows, minlength=m)
    del rows
    return _finish(m, m, counts, cols.to(colidx_dtype), seed, value_kind, rowptr_dtype,
                   colidx_dtype, device)


def mesh5_csr(nx: int, ny: int, seed: int = 0, value_kind: str = "f64um11",
              rowptr_dtype=torch.int64, colidx_dtype=torch.int32, device="cpu") -> CSRTensors:
    """5-point stencil (with the diagonal) on an nx-by-ny grid, row-major numbering."""
    device = torch.device(device)
    n = nx * ny
    v = torch.arange(n, dtype=torch.int64, device=device)
    r, c = v // ny, v % ny
    cand = torch.stack([v - ny, v - 1, v, v + 1, v + ny], dim=1)
    ok = torch.stack([r > 0, c > 0, torch.ones_like(r, dtype=torch.bool), c < ny - 1,
                      r < nx - 1], dim=1)
    counts = ok.sum(1)
    cols = cand[ok]
    return _finish(n, n, counts, cols.to(colidx_dtype), seed, value_kind, rowptr_dtype,
                   colidx_dtype, device)


def random_permutation(n: int, seed: int, stream: int = 0, dtype=torch.int32,
                       device="cpu") -> torch.Tensor:
    """A uniformly shuffled permutation of [0, n) (sort by 31 hash bits, ties by index)."""
    assert n < 2**32
    i = torch.arange(n, dtype=torch.int64, device=device)
    key = ((hash32(seed, S_PERM + 16 * stream, i) & 0x7FFFFFFF) << 32) | i
    return (torch.sort(key).values & MASK32).to(dtype)


def random_subset(n: int, k: int, seed: int, stream: int = 0, dtype=torch.int32,
                  device="cpu") -> torch.Tensor:
    """k distinct indices of [0, n) in random (unsorted) order."""
    assert 0 <= k <= n
    return random_permutation(n, seed, 1000 + stream, dtype, device)[:k].clone()


def degree_descending_permutation(rowptr: torch.Tensor, dtype=torch.int32) -> torch.Tensor:
    """p[i] = the vertex with the i-th largest row length; ties by ascending vertex id."""
    deg = (rowptr[1:] - rowptr[:-1]).to(torch.int64)
    n = deg.numel()
    i = torch.arange(n, dtype=torch.int64, device=rowptr.device)
    maxdeg = int(deg.max().item()) if n else 0
    key = ((maxdeg - deg) << 32) | i
    return (torch.sort(key).values & MASK32).to(dtype)


def loguniform_int(lo: int, hi: int, count: int, seed: int, stream: int, device="cpu"):
    """Integers log-uniform in [lo, hi] (used for the uneven batch sizes)."""
    i = torch.arange(count, dtype=torch.int64, device=device)
    u = (hash32(seed, 7000 + stream, i) >> 8).to(torch.float64) * (2.0 ** -24)
    v = torch.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))
    return torch.clamp(v.floor().to(torch.int64), lo, hi)
