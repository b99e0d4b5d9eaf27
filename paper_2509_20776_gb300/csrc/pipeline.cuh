// Host-side sequencing shared by the ops: the single-pass exclusive scan that turns
// per-row counts into the output row pointer, the tile partition of the output, and
// the launch of the tile / long-row / huge-row kernels of segsort.cuh.
#pragma once

#include "internal.h"
#include "segsort.cuh"

namespace sp {

// ------------------------------------------------------------------------------
// Decoupled look-back exclusive scan (Merrill & Garland, 2016).
// Each CTA takes a tile id from an atomic ticket, so a tile only ever waits for tiles
// that already started; every wait is bounded by ScanCtl::spin_limit polls and gives
// up with SP_ERR_TIMEOUT instead of hanging.  Status words pack a 2-bit flag with a
// 62-bit value so one relaxed 64-bit store publishes both.
// ------------------------------------------------------------------------------
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62,
                             kValMask = (1ull << 62) - 1;
constexpr int SCAN_BLOCK = 256, SCAN_ITEMS = 16, SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

struct ScanCtl {
  unsigned long long* status;  // one word per tile, zeroed before the launch
  unsigned* ticket;            // zeroed before the launch
  DevStatus* st;
  long long spin_limit;
  long long hold_tile;  // test hook: this tile never publishes (-1: off)
  long long n;
};

template <class Load, class Store>
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan(Load load, Store store, ScanCtl c) {
  constexpr int B = SCAN_BLOCK, IT = SCAN_ITEMS, TILE = SCAN_TILE;
  __shared__ long long buf[TILE + TILE / 16];
  __shared__ long long tmp[B / 32 + 1];
  __shared__ unsigned s_tile;
  __shared__ long long s_excl;
  const int t = threadIdx.x;
  if (t == 0) s_tile = atomicAdd(c.ticket, 1u);
  __syncthreads();
  const long long tile = s_tile;
  const long long base = tile * TILE;
#pragma unroll
  for (int j = 0; j < IT; ++j) {
    const int x = j * B + t;
    const long long i = base + x;
    buf[x + (x >> 4)] = i < c.n ? (long long)load(i) : 0;
  }
  __syncthreads();
  long long v[IT];
  long long sum = 0;
#pragma unroll
  for (int j = 0; j < IT; ++j) {
    const int x = t * IT + j;
    v[j] = buf[x + (x >> 4)];
    sum += v[j];
  }
  long long agg;
  const long long pre = block_excl_sum<B>(sum, tmp, &agg);
  if (tile == 0) {
    if (t == 0) {
      if (c.hold_tile != 0) st_relaxed_u64(&c.status[0], kFlagInc | (unsigned long long)agg);
      s_excl = 0;
    }
  } else {
    if (t == 0 && tile != c.hold_tile) st_relaxed_u64(&c.status[tile], kFlagAgg | (unsigned long long)agg);
    if (t < 32) {
      long long run = 0, pred = tile - 1;
      bool timeout = false;
      for (;;) {
        const long long idx = pred - t;
        unsigned long long w = kFlagInc;
        if (idx >= 0) {
          w = ld_relaxed_u64(&c.status[idx]);
          long long it = 0;
          while ((w >> 62) == 0) {
            if (++it > c.spin_limit) {
              timeout = true;
              w = kFlagInc;
              break;
            }
            __nanosleep(100);
            w = ld_relaxed_u64(&c.status[idx]);
          }
        }
        const unsigned incm = __ballot_sync(0xffffffffu, (w >> 62) == 2);
        const long long val = (long long)(w & kValMask);
        if (incm) {
          const int f = __ffs(incm) - 1;
          run += warp_sum(t <= f ? val : 0ll);
          break;
        }
        run += warp_sum(val);
        pred -= 32;
      }
      if (__any_sync(0xffffffffu, timeout) && t == 0) dev_fail(c.st, SP_ERR_TIMEOUT, tile);
      if (t == 0) {
        s_excl = run;
        if (tile != c.hold_tile) st_relaxed_u64(&c.status[tile], kFlagInc | (unsigned long long)(run + agg));
      }
    }
  }
  __syncthreads();
  long long run = s_excl + pre;
#pragma unroll
  for (int j = 0; j < IT; ++j) {
    const int x = t * IT + j;
    buf[x + (x >> 4)] = run;
    run += v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < IT; ++j) {
    const int x = j * B + t;
    const long long i = base + x;
    if (i < c.n) store(i, buf[x + (x >> 4)]);
  }
  if (base + TILE >= c.n && t == 0) store(c.n, s_excl + agg);
}

// load functors
template <class T>
struct LoadArray {
  const T* a;
  __device__ long long operator()(long long i) const { return (long long)a[i]; }
};
// stores: the int64 row pointer, optionally mirrored into a typed output array
template <class T>
struct StoreTyped {
  T* out;
  DevStatus* st;
  __device__ void operator()(long long i, long long v) const {
    if (sizeof(T) == 4 && v > 0x7fffffffll) dev_fail(st, SP_ERR_OVERFLOW, i);
    out[i] = T(v);
  }
};
template <class T>
struct StoreDual {
  long long* vp;
  T* out;  // may be null
  DevStatus* st;
  __device__ void operator()(long long i, long long v) const {
    vp[i] = v;
    if (out) {
      if (sizeof(T) == 4 && v > 0x7fffffffll) dev_fail(st, SP_ERR_OVERFLOW, i);
      out[i] = T(v);
    }
  }
};

inline size_t scan_ws_bytes(long long n) {
  long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  return align_up(size_t(tiles + 1) * 8) + kAlign;
}

// Exclusive scan of n values into n+1 outputs; `ws` must hold scan_ws_bytes(n).
template <class Load, class Store>
sp_status launch_scan(sp_ctx* ctx, cudaStream_t s, Load load, Store store, long long n, char* ws,
                      int phase = SP_PHASE_SCAN) {
  long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 0) tiles = 1;
  ScanCtl c;
  c.status = reinterpret_cast<unsigned long long*>(ws);
  c.ticket = reinterpret_cast<unsigned*>(ws + align_up(size_t(tiles + 1) * 8));
  c.st = ctx->dstatus;
  c.spin_limit = ctx->spin_limit;
  c.hold_tile = ctx->hold_tile;
  c.n = n;
  SP_CUDA(cudaMemsetAsync(ws, 0, scan_ws_bytes(n), s));
  if (tiles > 0x7fffffffll) return SP_ERR_OVERFLOW;
  {
    SP_PHASE(phase);
    k_scan<Load, Store><<<unsigned(tiles), SCAN_BLOCK, 0, s>>>(load, store, c);
  }
  SP_CUDA(cudaGetLastError());
  return SP_OK;
}

// ------------------------------------------------------------------------------
// Tile partition, computed by one more scan over the listed rows.  Row r weighs
// TILE_ROW_W plus its output length when the tile kernel sorts it (output length at
// most TILE_CP), so that rows left to k_long / k_huge take no room; c(r) is the
// exclusive prefix of the weights and tile t holds the rows with c(r) in
// [t*TILE_CP, (t+1)*TILE_CP): at most 2*TILE_CP entries and TILE_CP/TILE_ROW_W rows.
// The store of the scan writes tile_first[] directly; with `classify` (source length =
// output length, e.g. permutation) it also lists the rows left to k_long / k_huge.
// The number of tiles is written to *ntiles (tile_first[*ntiles] = nrows).
// ------------------------------------------------------------------------------
__device__ __forceinline__ long long tile_weight(const long long* vp, long long r) {
  const long long L = vp[r + 1] - vp[r];
  return TILE_ROW_W + (L <= TILE_CP ? L : 0);
}

struct TileWeight {
  const long long* vp;
  __device__ long long operator()(long long r) const { return tile_weight(vp, r); }
};

struct PartitionStore {
  const long long* vp;
  long long nrows;
  long long ntiles_cap;  // tile_first holds ntiles_cap + 1 entries
  long long* tile_first;
  long long* ntiles;
  int classify;
  long long* long_rows;
  unsigned* n_long;
  long long long_cap;
  long long* huge_rows;
  unsigned* n_huge;
  long long huge_cap;
  DevStatus* st;
  __device__ void operator()(long long r, long long c) const {
    if (r == nrows) {  // c = total weight
      long long nt = c / TILE_CP + 1;
      if (nt > ntiles_cap) {
        dev_fail(st, SP_ERR_INTERNAL, -14);
        nt = ntiles_cap;
      }
      *ntiles = nt;
      tile_first[nt] = nrows;
      return;
    }
    if (r == 0) tile_first[0] = 0;
    const long long e = c + tile_weight(vp, r);
    long long t_lo = c / TILE_CP + 1, t_hi = e / TILE_CP;
    if (t_hi > ntiles_cap - 1) t_hi = ntiles_cap - 1;
    for (long long t = t_lo; t <= t_hi; ++t) tile_first[t] = r + 1;
    if (classify) {
      const long long L = vp[r + 1] - vp[r];
      if (L > TILE_CP) {
        if (L <= LONG_CAP) {
          const unsigned q = atomicAdd(n_long, 1u);
          if (q < long_cap) long_rows[q] = r;
          else dev_fail(st, SP_ERR_INTERNAL, -10);
        } else {
          const unsigned q = atomicAdd(n_huge, 1u);
          if (q < huge_cap) huge_rows[q] = r;
          else dev_fail(st, SP_ERR_INTERNAL, -11);
        }
      }
    }
  }
};

struct PipeLists {
  long long* long_rows = nullptr;  // rows for k_long in source mode
  unsigned* n_long = nullptr;
  long long long_cap = 0;
  long long* huge_rows = nullptr;  // rows for k_huge round 0
  unsigned* n_huge = nullptr;
  long long huge_cap = 0;
};

// Workspace of the sort pipeline after the counts (lists may already be filled).
struct PipeWs {
  long long* tile_first = nullptr;
  long long ntiles = 0;
  unsigned* counters = nullptr;  // [0..3] tickets, [4] n_final, [5] n_next
  long long* ntiles_dev = nullptr;  // number of tiles, written by the partition
  char* scan_ws = nullptr;          // workspace of the partition scan
  FinalEntry* fin = nullptr;
  long long fin_cap = 0;
  HugeEntry* nxt = nullptr;
  long long nxt_cap = 0;
  uint32_t* tkey = nullptr;
  void* tval = nullptr;
};

inline long long pipe_ntiles(long long nrows, long long nnz_out) {
  return (nnz_out + TILE_ROW_W * nrows) / TILE_CP + 1;
}

constexpr int kPipeSlots = 8;  // workspace slots reserved by pipe_reserve

inline void pipe_reserve(Carver& cv, long long nrows, long long nnz_out, size_t vbytes, size_t* off) {
  const long long ntiles = pipe_ntiles(nrows, nnz_out);
  off[0] = cv.reserve(size_t(ntiles + 1) * 8);
  off[1] = cv.reserve(16 * 4);
  const long long fin_cap = 2 * (3 * (nnz_out / GROUP_CAP) + nnz_out / LONG_CAP + 16);
  off[2] = cv.reserve(size_t(fin_cap) * sizeof(FinalEntry));
  const long long nxt_cap = nnz_out / LONG_CAP + 1;
  off[3] = cv.reserve(size_t(nxt_cap) * sizeof(HugeEntry));
  const bool need_temp = nnz_out > LONG_CAP;
  off[4] = cv.reserve(need_temp ? size_t(nnz_out) * 4 : 0);
  off[5] = cv.reserve(need_temp ? size_t(nnz_out) * vbytes : 0);
  off[6] = cv.reserve(scan_ws_bytes(nrows));
  off[7] = cv.reserve(8);
}

inline PipeWs pipe_bind(const Carver& cv, long long nrows, long long nnz_out, const size_t* off) {
  PipeWs w;
  w.ntiles = pipe_ntiles(nrows, nnz_out);
  w.tile_first = cv.at<long long>(off[0]);
  w.counters = cv.at<unsigned>(off[1]);
  w.fin_cap = 2 * (3 * (nnz_out / GROUP_CAP) + nnz_out / LONG_CAP + 16);
  w.fin = cv.at<FinalEntry>(off[2]);
  w.nxt_cap = nnz_out / LONG_CAP + 1;
  w.nxt = cv.at<HugeEntry>(off[3]);
  w.tkey = cv.at<uint32_t>(off[4]);
  w.tval = cv.at<void>(off[5]);
  w.scan_ws = cv.at<char>(off[6]);
  w.ntiles_dev = cv.at<long long>(off[7]);
  return w;
}

template <class K>
inline void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

// Run partition + tile + long + huge kernels for `nrows` listed output rows with row
// pointer `vp` (nnz_out entries).  With `classify`, long/huge rows are found here from
// the output lengths; otherwise `lists` were filled by the count kernels.
template <class Ld>
sp_status run_pipeline(sp_ctx* ctx, cudaStream_t s, const Ld& ld, const long long* vp,
                       long long nrows, long long nnz_out, int key_bits, bool classify,
                       const PipeLists& lists, const PipeWs& w, typename Ld::CI* out_col,
                       typename Ld::VT* out_val) {
  using VT = typename Ld::VT;
  if (nrows == 0 || nnz_out == 0) return SP_OK;
  SP_CUDA(cudaMemsetAsync(w.counters, 0, 16 * 4, s));
  const int nsm = ctx->num_sms;
  SP_TRY(launch_scan(ctx, s, TileWeight{vp},
                     PartitionStore{vp, nrows, w.ntiles, w.tile_first, w.ntiles_dev, classify ? 1 : 0,
                                    lists.long_rows, lists.n_long, lists.long_cap, lists.huge_rows,
                                    lists.n_huge, lists.huge_cap, ctx->dstatus},
                     nrows, w.scan_ws, SP_PHASE_PARTITION));
  {
    constexpr size_t sm = tile_smem_bytes<Ld>();
    static bool once = (set_smem(k_tile<Ld>, sm), true);
    (void)once;
    // persistent: TILE_PER_SM resident CTAs per SM walk the tiles
    const long long g = w.ntiles < (long long)nsm * TILE_PER_SM ? w.ntiles : (long long)nsm * TILE_PER_SM;
    {
      SP_PHASE(SP_PHASE_TILE);
      k_tile<Ld><<<unsigned(g), TILE_BLOCK, sm, s>>>(ld, vp, w.tile_first, w.ntiles_dev, out_col,
                                                      out_val, key_bits, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
  }
  constexpr size_t lsm = long_smem_bytes<VT>();
  static bool once_l = (set_smem(k_long<Ld>, lsm), true);
  (void)once_l;
  {
    SP_PHASE(SP_PHASE_LONG);
    k_long<Ld><<<2 * nsm, LONG_BLOCK, lsm, s>>>(ld, vp, lists.long_rows, lists.n_long, nullptr,
                                             nullptr, lists.long_cap, w.counters + 0, nullptr, nullptr, out_col,
                                             out_val, key_bits, ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  if (nnz_out > LONG_CAP) {
    constexpr size_t hsm = huge_smem_bytes();
    static bool once_h = (set_smem(k_huge<Ld>, hsm), true);
    (void)once_h;
    VT* tval = static_cast<VT*>(w.tval);
    {
      SP_PHASE(SP_PHASE_HUGE);
      k_huge<Ld><<<nsm, HUGE_BLOCK, hsm, s>>>(
          ld, vp, lists.huge_rows, lists.n_huge, nullptr, nullptr, lists.huge_cap, w.counters + 1, key_bits,
          w.tkey, tval, out_col, out_val, w.fin, w.counters + 4, w.fin_cap, w.nxt,
          w.counters + 5, w.nxt_cap, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    if (key_bits > HUGE_NB_LOG + 13) {  // second round only when buckets can exceed LONG_CAP
      {
        SP_PHASE(SP_PHASE_HUGE);
        k_huge<Ld><<<nsm, HUGE_BLOCK, hsm, s>>>(
            ld, vp, nullptr, nullptr, w.nxt, w.counters + 5, w.nxt_cap, w.counters + 2, key_bits, w.tkey,
            tval, out_col, out_val, w.fin, w.counters + 4, w.fin_cap, w.nxt + 0,
            w.counters + 6, 0, ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
    }
    {
      SP_PHASE(SP_PHASE_LONG);
      k_long<Ld><<<2 * nsm, LONG_BLOCK, lsm, s>>>(ld, vp, nullptr, nullptr, w.fin, w.counters + 4,
                                               w.fin_cap, w.counters + 3, w.tkey, tval, out_col, out_val,
                                               key_bits, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
  }
  return SP_OK;
}

}  // namespace sp
