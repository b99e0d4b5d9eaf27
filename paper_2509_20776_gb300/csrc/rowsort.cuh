// Two-phase Build step (Sec. 3.1, Algorithm 2's fill pass and the per-row sort):
//   phase 1, k_gather_chunks: every output row gets its source entries, relabelled,
//     at its final row position but in source order (a load-balanced gather over
//     fixed chunks of output positions: no shared-memory sort, all loads independent);
//   phase 2, the rows of the output are sorted in place:
//     * rows of at most CP entries (512, or 1024 with the run-time tile shape 1) in
//       tiles of consecutive rows, at most 2 * CP entries each, k_seg_sort<SsTile> or
//       k_seg_sort<SsTileL>;
//     * rows of CP < L <= SS_RUN_MAX entries alone, k_seg_sort<SsRunT<VT>>;
//     * longer rows are first cut by key range (k_split: a coarse, then a fine split) into runs of at
//       most SS_RUN_MAX entries, which k_seg_sort<SsRunT<VT>> then sorts.
//   Buckets of more keys than the (run-time) heavy threshold are queued as runs for up
//   to SS_PASSES later passes.
// One scan over the output rows (RowsPartition) cuts the tiles and the gather chunks
// and lists the rows that do not fit a tile.
#pragma once

#include <type_traits>

#include "scan.cuh"

namespace sp {

constexpr int SS_ROW_W = 4;                    // partition weight of a row
constexpr int SS_HEAVY = 128;                  // default (and smallest) heavy-bucket threshold
constexpr int SS_PASSES = 3;                   // passes over queued heavy buckets

// A sort configuration: BLOCK threads sort items of at most CAP entries, MINB CTAs per
// SM; a tile holds the rows whose partition coordinate starts in a window of
// CP = CAP / 2, so at most ROWS = CP / SS_ROW_W rows (one thread each) of at most CP
// entries.  A single run of L entries uses at most ss_nb(L) <= CAP / 2 bucket counters.
template <int BLOCK_, int CAP_, bool TILES_, int MINB_, bool BACK_ = false>
struct SsCfg {
  static constexpr int B = BLOCK_, CAP = CAP_, CP = CAP_ / 2, ROWS = CP / SS_ROW_W, MINB = MINB_;
  static constexpr int WORDS = CAP_ / 32;  // row-start bitmap words
  static constexpr bool kTiles = TILES_;   // items are tiles (else: single runs)
  static constexpr bool kBack = BACK_;     // runs: taken from the back of the run list
  static constexpr int CNT = TILES_ ? CAP_ : CAP_ / 2;  // bucket counters
  static_assert(!TILES_ || ROWS <= B, "one thread per row of a tile");
  static_assert(WORDS % 32 == 0, "one warp scans the bitmap");
  static_assert(B % 32 == 0 && B * MINB <= 2048, "whole warps, resident CTAs");
};
using SsTile = SsCfg<128, 1024, true, 9>;   // tiles of rows of at most 512 entries
using SsTileL = SsCfg<256, 2048, true, 4>;  // tile shape 1: rows of at most 1024 entries
// single runs of at most 4096 entries: with 4-byte values three CTAs of 384 threads fit
// an SM (72 KB of shared memory each), with 8-byte values two of 512 (88 KB)
template <class VT>
using SsRunT = std::conditional_t<sizeof(VT) == 4, SsCfg<384, 4096, false, 3>, SsCfg<512, 4096, false, 2>>;
// runs of at most 1024 entries (the back of the run list): 128 threads, 8 CTAs per SM
using SsRunS = SsCfg<128, 1024, false, 8, true>;
constexpr int SS_SMALL_RUN = SsRunS::CAP;
constexpr int SS_TILE_MAX = SsTile::CP;  // longest row a tile accepts (the smaller tile shape)
constexpr int SS_RUN_MAX = 4096;         // longest row sorted alone
static_assert(SsRunT<uint32_t>::CAP == SS_RUN_MAX && SsRunT<unsigned long long>::CAP == SS_RUN_MAX,
              "one run capacity");

// Runs handed from one kernel to the next: in the output arrays or in the temporary
// arrays (keys as uint32, values) at the same offsets.
enum BufId : int { BUF_TEMP = 0, BUF_OUT = 1 };

struct FinalEntry {  // a run of at most SS_RUN_MAX entries left to sort in place
  long long off;
  long long len;
  int buf;
  int pad;
};
// The run list is filled from both ends: n[0] counts the runs at its front, n[1] the runs
// of at most SS_SMALL_RUN entries at its back (k_seg_sort<SsRunS>, small CTAs, sorts those;
// k_seg_sort<SsRunT> the front).  cap bounds all the runs a pass queues, so the two ends
// never meet.
__device__ __forceinline__ void queue_run(FinalEntry* list, unsigned* n, long long cap, const FinalEntry& e,
                                          DevStatus* st, long long err) {
  const bool small = e.len <= SS_SMALL_RUN;
  const unsigned q = atomicAdd(n + (small ? 1 : 0), 1u);
  if (q < cap) list[small ? cap - 1 - q : q] = e;
  else dev_fail(st, SP_ERR_INTERNAL, err);
}
struct HugeEntry {  // a run longer than SS_RUN_MAX; coarse split: keys in [lo, lo + 2^wb)
  long long off;
  long long len;
  unsigned lo;
  int wb;
  int buf;
  int pad;
};

// The rows queued for the key-range split.  n[0] counts the rows queued at the front of
// the list, n[1] the rows of at least SPLIT_HUB entries queued from its back; the split
// hands out the back first, so that a hub row (one CTA for up to milliseconds) starts at
// once instead of wherever the queueing order put it.  cap >= nnz / SS_RUN_MAX + 1 bounds
// the number of rows longer than SS_RUN_MAX, so the two ends never meet.
constexpr long long SPLIT_HUB = 1ll << 16;
__device__ __forceinline__ void queue_huge(HugeEntry* list, unsigned* n, long long cap, const HugeEntry& e,
                                           DevStatus* st, long long err) {
  const bool hub = e.len >= SPLIT_HUB;
  const unsigned q = atomicAdd(n + (hub ? 1 : 0), 1u);
  if (q < cap) list[hub ? cap - 1 - q : q] = e;
  else dev_fail(st, SP_ERR_INTERNAL, err);
}

constexpr int GC_BLOCK = 256;                  // gather: threads per CTA
constexpr int GC_CH = 4096;                    // gather: output positions per CTA
constexpr int GC_ITEMS = GC_CH / GC_BLOCK;
constexpr int GC_MINB = 5;                     // gather: resident CTAs per SM (persistent grid)
constexpr int GC_H = 4;                        // gather: positions a thread loads before it stores

// ---- partition ----------------------------------------------------------------------
// Row r weighs SS_ROW_W plus its length when a tile sorts it (length <= tmax, the tile
// shape's CP).  With c(r) the exclusive prefix of the weights, tile t holds the rows with
// c(r) in [t*tmax, (t+1)*tmax): at most tmax / SS_ROW_W rows and 2*tmax entries.  Gather
// chunk k starts at the row holding output position k*GC_CH.
__device__ __forceinline__ long long rows_weight(const long long* vp, long long r, long long tmax) {
  const long long L = vp[r + 1] - vp[r];
  return SS_ROW_W + (L <= tmax ? L : 0);
}

struct RowsWeight {
  const long long* vp;
  long long tmax;
  __device__ long long operator()(long long r) const { return rows_weight(vp, r, tmax); }
};

struct RowsPartition {
  const long long* vp;
  long long nrows;
  long long ntiles_cap;  // tile_first holds ntiles_cap + 1 entries
  long long* tile_first;
  long long* ntiles;
  long long nchunks;
  long long* chunk_first;
  FinalEntry* fin;  // rows sorted alone
  unsigned* fin_n;
  long long fin_cap;
  HugeEntry* huge;  // rows for k_split
  unsigned* huge_n;  // two counts (queue_huge)
  long long huge_cap;
  int key_bits;
  int classify;  // list the rows that do not fit a tile (only when the rows are sorted)
  long long tmax;  // longest row a tile accepts
  DevStatus* st;
  __device__ void operator()(long long r, long long c) const {
    if (r == nrows) {  // c = total weight
      long long nt = c / tmax + 1;
      if (nt > ntiles_cap) {
        dev_fail(st, SP_ERR_INTERNAL, -14);
        nt = ntiles_cap;
      }
      *ntiles = nt;
      tile_first[nt] = nrows;
      return;
    }
    if (r == 0) tile_first[0] = 0;
    const long long o0 = vp[r], o1 = vp[r + 1], L = o1 - o0;
    const long long e = c + SS_ROW_W + (L <= tmax ? L : 0);
    long long t_lo = c / tmax + 1, t_hi = e / tmax;
    if (t_hi > ntiles_cap - 1) t_hi = ntiles_cap - 1;
    for (long long t = t_lo; t <= t_hi; ++t) tile_first[t] = r + 1;
    if (L <= 0) return;
    long long k_hi = (o1 - 1) / GC_CH;
    if (k_hi > nchunks - 1) k_hi = nchunks - 1;
    for (long long k = (o0 + GC_CH - 1) / GC_CH; k <= k_hi; ++k) chunk_first[k] = r;
    if (classify && L > tmax) {
      if (L <= SS_RUN_MAX) {
        queue_run(fin, fin_n, fin_cap, FinalEntry{o0, L, BUF_OUT, 0}, st, -15);
      } else {
        queue_huge(huge, huge_n, huge_cap, HugeEntry{o0, L, 0u, key_bits, BUF_OUT, 0}, st, -16);
      }
    }
  }
};

// ---- conflict-free block scans over shared arrays ------------------------------------------
// Each warp owns a contiguous segment of n / (B / 32) entries and walks it 32 entries at a
// time (lane l reads word base + l: no bank conflicts), carrying its running value; the
// warps' segment totals are combined by one warp.  n must be a multiple of B.
template <int B>
__device__ uint32_t smem_excl_sum_w(uint32_t* a, int n, uint32_t* tmp) {
  constexpr int NW = B / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, seg = n / NW;
  uint32_t* s = a + w * seg;
  uint32_t tot = 0;
  for (int x = lane; x < seg; x += 32) tot += s[x];
  tot = warp_sum(tot);
  if (lane == 0) tmp[w] = tot;
  __syncthreads();
  if (w == 0) {
    const uint32_t v = lane < NW ? tmp[lane] : 0u;
    const uint32_t inc = warp_incl_sum(v);
    if (lane < NW) tmp[lane] = inc - v;
    if (lane == NW - 1) tmp[NW] = inc;
  }
  __syncthreads();
  uint32_t carry = tmp[w];
  for (int x = lane; x < seg; x += 32) {
    const uint32_t v = s[x];
    const uint32_t inc = warp_incl_sum(v);
    s[x] = carry + inc - v;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  const uint32_t total = tmp[NW];
  __syncthreads();
  return total;
}

template <int B>
__device__ void smem_incl_max_w(uint32_t* a, int n, uint32_t* tmp) {
  constexpr int NW = B / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, seg = n / NW;
  uint32_t* s = a + w * seg;
  uint32_t mx = 0;
  for (int x = lane; x < seg; x += 32) mx = s[x] > mx ? s[x] : mx;
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) tmp[w] = mx;
  __syncthreads();
  if (w == 0) {
    const uint32_t v = lane < NW ? tmp[lane] : 0u;
    uint32_t inc = warp_incl_max(v);
    uint32_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) ex = 0u;
    if (lane < NW) tmp[lane] = ex;
  }
  __syncthreads();
  uint32_t carry = tmp[w];
  for (int x = lane; x < seg; x += 32) {
    const uint32_t inc = warp_incl_max(s[x]);
    const uint32_t r = inc > carry ? inc : carry;
    s[x] = r;
    carry = __shfl_sync(0xffffffffu, r, 31);
  }
  __syncthreads();
}

// ---- phase 1: gather ----------------------------------------------------------------
// Chunk k is GC_CH consecutive output positions, starting inside row chunk_first[k].
// Gs: using CI, VT;
//     __device__ long long src(long long r) const;     // source start of output row r
//     __device__ typename Gs::CI col(long long pos) const;  // source column
//     __device__ typename Gs::CI map(long long pos, typename Gs::CI c) const;  // new column
//     __device__ typename Gs::VT val(long long pos) const;
template <class Gs>
__global__ void __launch_bounds__(GC_BLOCK, GC_MINB) k_gather_chunks(Gs gs, const long long* __restrict__ vp,
                                                            long long nrows, long long total,
                                                            const long long* __restrict__ chunk_first,
                                                            long long nchunks,
                                                            typename Gs::CI* __restrict__ out_col,
                                                            typename Gs::VT* __restrict__ out_val) {
  using CI = typename Gs::CI;
  using VT = typename Gs::VT;
  constexpr int B = GC_BLOCK, ITEMS = GC_ITEMS;
  __shared__ uint32_t owner[GC_CH];
  __shared__ long long r_off[B];
  __shared__ long long r_o0[B];
  __shared__ long long r_o1[B];
  __shared__ uint32_t tmp32[B / 32 + 1];
  __shared__ long long s_last;  // output end of the batch's last row
  __shared__ int s_single;      // the batch's first row covers the whole chunk
  const int t = threadIdx.x;
  // row r's output range [o0, o1) and source start
  auto setup = [&](long long r, long long& a, long long& b, long long& s) {
    a = total;
    b = total;
    s = 0;
    if (r < nrows) {
      a = vp[r];
      b = vp[r + 1];
      s = gs.src(r);
    }
  };
  // persistent: chunks blockIdx.x, + gridDim.x, ...; a batch is B consecutive rows.  The
  // next batch's row setup is loaded while this batch's entries are in flight.
  long long c = blockIdx.x;
  if (c >= nchunks) return;
  long long rb = chunk_first[c];
  long long o0, o1, so;
  setup(rb + t, o0, o1, so);
  for (;;) {
    const long long c0 = c * (long long)GC_CH, c1 = c0 + GC_CH < total ? c0 + GC_CH : total;
    const long long cn = c + gridDim.x;
    const long long rb_next_chunk = cn < nchunks ? chunk_first[cn] : 0;
    const bool active = rb + t < nrows && o1 > o0 && o1 > c0 && o0 < c1;
    if (active) {
      r_off[t] = so;
      r_o0[t] = o0;
      r_o1[t] = o1;
    }
    if (t == B - 1) s_last = o1;
    if (t == 0) s_single = active && o0 <= c0 && o1 >= c1;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) owner[t + j * B] = 0;
    __syncthreads();
    // a chunk inside one long row (most of a long row's chunks) needs no owner search
    const bool single = s_single;
    if (!single) {
      if (active) owner[(o0 > c0 ? o0 : c0) - c0] = uint32_t(t + 1);
      __syncthreads();
      smem_incl_max_w<B>(owner, GC_CH, tmp32);
    }
    // the chunk ends with this batch once its last row reaches the end of the chunk
    const bool last_batch = rb + B - 1 >= nrows - 1 || s_last >= c1;
    const bool more = !last_batch || cn < nchunks;
    const long long rb_next = last_batch ? rb_next_chunk : rb + B;
    long long n0 = 0, n1 = 0, ns = 0;
    if (more) setup(rb_next + t, n0, n1, ns);
    // all loads, then all stores (the compiler cannot move stores above later loads)
    constexpr int H = GC_H;
#pragma unroll
    for (int h = 0; h < ITEMS; h += H) {
      CI cv[H];
      VT v[H];
      long long pos[H];
      bool ok[H];
#pragma unroll
      for (int u = 0; u < H; ++u) {
        const int x = t + (h + u) * B;
        const long long g = c0 + x;
        const int ow = single ? 1 : int(owner[x]);
        ok[u] = false;
        pos[u] = 0;
        if (g < c1 && ow > 0) {
          const int k = ow - 1;
          const long long o = r_o0[k];
          // positions past this batch of rows belong to the next batch
          if (g >= o && g < r_o1[k]) {
            ok[u] = true;
            pos[u] = r_off[k] + (g - o);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < H; ++u) cv[u] = ok[u] ? gs.col(pos[u]) : CI(0);
#pragma unroll
      for (int u = 0; u < H; ++u)
        if (ok[u]) v[u] = gs.val(pos[u]);
#pragma unroll
      for (int u = 0; u < H; ++u)
        if (ok[u]) cv[u] = gs.map(pos[u], cv[u]);
#pragma unroll
      for (int u = 0; u < H; ++u) {
        if (!ok[u]) continue;
        const long long g = c0 + t + (h + u) * B;
        st_stream(out_col + g, cv[u]);
        st_stream(out_val + g, v[u]);
      }
    }
    __syncthreads();
    if (!more) break;
    if (last_batch) c = cn;
    rb = rb_next;
    o0 = n0;
    o1 = n1;
    so = ns;
  }
}

// ---- approximate square-root bucketing of the row sort -----------------------------------
// Bucket of key k in a row of L entries: nb = 2^(ceil(log2 L) - 1) buckets spaced evenly
// in an approximate square root of k over the row's key range [0, kmax].  The root is
// the exponent-halving bit trick on the float of k (exact at even powers of two, up to
// 6% high in between): monotone in k (every step is), so buckets stay in key order; the
// scale nb / root(kmax) maps [0, kmax] onto the nb buckets.  The square root keeps
// buckets balanced both for uniformly relabelled columns and for labels crowded at the
// low end (degree-descending orderings).
__device__ __forceinline__ uint32_t ss_nb(uint32_t L) { return L <= 2 ? 1u : 1u << (31 - __clz(L - 1)); }
__device__ __forceinline__ float ss_root(uint32_t k) {
  return __uint_as_float((__float_as_uint(__uint2float_rn(k)) >> 1) + 0x1FC00000u);
}
// 1 / root(kmax): the scale of a range [0, kmax] is nb * ss_inv_root(kmax)
__device__ __forceinline__ float ss_inv_root(uint32_t kmax) { return kmax ? 1.0f / ss_root(kmax) : 0.0f; }
// bucket of `key` given the row's scale and last bucket nb - 1
__device__ __forceinline__ uint32_t ss_bucket(uint32_t key, float scale, uint32_t last) {
  const uint32_t b = __float2uint_rz(ss_root(key) * scale);
  return b < last ? b : last;
}

// ---- key-range split of long runs ------------------------------------------------------
// A run of more than SS_RUN_MAX entries with keys in [lo, lo + 2^wb) is cut into nb = 2^nbl
// buckets of 2^(wb - nbl) consecutive keys: pass 1 counts the bucket sizes, one scan gives
// their offsets, pass 2 moves the run bucket by bucket into the other buffer (output <->
// temporary) at the same offsets.  Consecutive small buckets whose starts fall in one
// GROUP_CAP window form one run for k_seg_sort; a bucket of more than GROUP_CAP entries is
// a run of its own, or (more than SS_RUN_MAX entries) a run for the fine split.
//   Coarse split (SplitCoarse): nb = 2^10 buckets evenly spaced over [lo, lo + 2^wb).  A run
//     is sorted as a whole afterwards, so pass 2 only has to bring every entry into its
//     group's range, not its bucket's: it stages each chunk of B * U entries in shared
//     memory by group and writes every group's share of the chunk as one contiguous piece
//     (groups hold hundreds to thousands of entries, so the writes are coalesced whatever
//     the key distribution).
//   Fine split (SplitFine, the buckets of the coarse split that hold more than SS_RUN_MAX entries,
//     e.g. hub rows under a degree-descending relabelling): 2^13 buckets evenly spaced over
//     the bucket's own [min, max] keys (found by a first pass), scattered directly.  A
//     coarse bucket spans 2^(wb - 10) <= 2^22 keys, so a fine bucket spans at most
//     2^9 < SS_RUN_MAX keys: with keys unique within a row it holds fewer than SS_RUN_MAX
//     entries and no third split is needed.
struct SplitCoarse {
  static constexpr int NBL = 10, B = 256, MINB = 4, U = 8;
  static constexpr bool kStaged = true;
};
struct SplitFine {
  static constexpr int NBL = 13, B = 512, MINB = 2, U = 4;
  static constexpr bool kStaged = false;
};
constexpr int SS_RUN_LOG = 12;             // SS_RUN_MAX = 2^SS_RUN_LOG
static_assert((1 << SS_RUN_LOG) == SS_RUN_MAX, "run capacity is a power of two");
constexpr int GROUP_CAP = SS_RUN_MAX / 2;  // small buckets grouped up to this start window
template <class S, class VT>
constexpr size_t split_smem_bytes() {
  // counts / starts / cursors, previous non-empty bucket, next group boundary; staged:
  // the group of each bucket, the chunk's counts / starts per group, the chunk's base in
  // each group, the chunk's keys and values
  return size_t(1 << S::NBL) * 4 * 3 +
         (S::kStaged ? size_t(1 << S::NBL) * 4 * 3 + size_t(S::B * S::U) * (4 + sizeof(VT)) : 0);
}

template <class S, class CI, class VT>
__global__ void __launch_bounds__(S::B, S::MINB)
    k_split(const HugeEntry* __restrict__ runs, const unsigned* __restrict__ nruns_p, long long runs_cap,
            unsigned* ticket, uint32_t* __restrict__ tkey, VT* __restrict__ tval, CI* __restrict__ out_col,
            VT* __restrict__ out_val, FinalEntry* __restrict__ fin, unsigned* fin_n, long long fin_cap,
            HugeEntry* __restrict__ nxt, unsigned* nxt_n, long long nxt_cap, DevStatus* st) {
  constexpr int B = S::B, U = S::U, NBM = 1 << S::NBL;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem);  // bucket sizes, then starts, then cursors
  uint32_t* prv = hist + NBM;   // 1 + last non-empty bucket at or before x (0: none)
  uint32_t* nxb = prv + NBM;    // reversed: L - start of the first group boundary >= x
  uint32_t* hd = nxb + NBM;     // staged: 1 + first bucket of each bucket's group
  uint32_t* lh = hd + NBM;      // staged: the chunk's count, then start, in each group
  uint32_t* gb = lh + NBM;      // staged: the chunk's offset in each group
  uint32_t* sk = gb + NBM;      // staged: the chunk's keys by group
  VT* sv = reinterpret_cast<VT*>(sk + B * U);  // and values
  __shared__ uint32_t tmp32[B / 32 + 1];
  __shared__ unsigned s_item;
  const int t = threadIdx.x;
  // the list's back (rows of >= SPLIT_HUB entries) first, then its front
  long long nb_ = nruns_p[1], nf_ = nruns_p[0];
  if (nb_ > runs_cap) nb_ = runs_cap;
  if (nf_ > runs_cap - nb_) nf_ = runs_cap - nb_;
  const long long count = nb_ + nf_;
  for (;;) {
    if (t == 0) s_item = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long item = s_item;
    if (item >= count) break;
    const HugeEntry he = runs[item < nb_ ? runs_cap - 1 - item : item - nb_];
    const long long g0 = he.off, L = he.len;
    const int sbuf = he.buf;
    const int dbuf = sbuf == BUF_TEMP ? BUF_OUT : BUF_TEMP;
    const uint32_t* skp = tkey + g0;
    const CI* sop = out_col + g0;
    auto key_at = [&](long long e) -> uint32_t {
      return sbuf == BUF_TEMP ? ld_stream(skp + e) : uint32_t(ld_stream(sop + e));
    };
    uint32_t lo;
    int wb, nbl;
    if constexpr (S::kStaged) {
      lo = he.lo;
      wb = he.wb;
      nbl = wb < S::NBL ? wb : S::NBL;
      static_assert(32 - S::NBL - SplitFine::NBL <= SS_RUN_LOG, "fine-split buckets fit a run");
    } else {
      // the bucket's own key range
      uint32_t mn = 0xFFFFFFFFu, mx = 0u;
      for (long long e0 = t; e0 < L; e0 += (long long)B * U) {
        uint32_t k[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + (long long)u * B < L) k[u] = key_at(e0 + (long long)u * B);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + (long long)u * B < L) {
            mn = k[u] < mn ? k[u] : mn;
            mx = k[u] > mx ? k[u] : mx;
          }
      }
      mn = __reduce_min_sync(0xFFFFFFFFu, mn);
      mx = __reduce_max_sync(0xFFFFFFFFu, mx);
      if ((t & 31) == 0) {
        tmp32[t >> 5] = mn;
        hist[t >> 5] = mx;  // hist is cleared below
      }
      __syncthreads();
      mn = 0xFFFFFFFFu;
      mx = 0u;
      for (int w = 0; w < B / 32; ++w) {
        mn = tmp32[w] < mn ? tmp32[w] : mn;
        mx = hist[w] > mx ? hist[w] : mx;
      }
      __syncthreads();
      lo = mn;
      const uint32_t span = mx >= mn ? mx - mn : 0u;  // keys in [lo, lo + span]
      wb = span ? 32 - __clz(span) : 0;                // 2^wb > span
      nbl = wb < S::NBL ? wb : S::NBL;
    }
    const int nb = 1 << nbl;
    const int sh = wb - nbl;
    const uint32_t rmax = wb >= 32 ? 0xFFFFFFFFu : (1u << wb) - 1u;  // largest offset from lo
    // bucket of key k, or 0xFFFFFFFF for a key outside the run's range (a column outside
    // [0, ncols): reported by pass 1)
    auto bucket = [&](uint32_t k) -> uint32_t {
      if (k < lo || k - lo > rmax) return 0xFFFFFFFFu;
      return (k - lo) >> sh;
    };
    for (int x = t; x < NBM; x += B) hist[x] = 0;
    __syncthreads();
    // pass 1: bucket sizes
    for (long long e0 = t; e0 < L; e0 += (long long)B * U) {
      uint32_t k[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long e = e0 + (long long)u * B;
        if (e < L) k[u] = key_at(e);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long e = e0 + (long long)u * B;
        if (e >= L) continue;
        const uint32_t bk = bucket(k[u]);
        if (bk != 0xFFFFFFFFu) atomicAdd(&hist[bk], 1u);
        else dev_fail(st, SP_ERR_INDEX_RANGE, g0 + e);  // a column outside [0, ncols)
      }
    }
    __syncthreads();
    const uint32_t total = smem_excl_sum_w<B>(hist, NBM, tmp32);
    if (total != uint32_t(L)) {
      if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -5);
      continue;
    }
    // bucket x holds [hist[x], end(x)); bucket order is key order
    auto bend = [&](int x) { return x + 1 < nb ? hist[x + 1] : uint32_t(L); };
    // previous non-empty bucket (inclusive max-scan of x+1 over non-empty buckets)
    for (int x = t; x < NBM; x += B) prv[x] = (x < nb && bend(x) > hist[x]) ? uint32_t(x + 1) : 0u;
    __syncthreads();
    smem_incl_max_w<B>(prv, NBM, tmp32);
    // Groups: a bucket of more than GROUP_CAP entries ("big") stands alone; a small
    // non-empty bucket starts a new group ("head") unless the previous non-empty
    // bucket is small and starts in the same GROUP_CAP window.
    auto kind = [&](int x, bool& big, bool& head) {
      const uint32_t sb = hist[x], cc = x < nb ? bend(x) - sb : 0u;
      big = cc > uint32_t(GROUP_CAP);
      head = false;
      if (cc > 0 && !big) {
        const uint32_t pv = x > 0 ? prv[x - 1] : 0u;
        if (pv == 0) {
          head = true;
        } else {
          const int y = int(pv) - 1;
          head = bend(y) - hist[y] > uint32_t(GROUP_CAP) || (hist[y] / GROUP_CAP) != (sb / GROUP_CAP);
        }
      }
    };
    // next group boundary after each bucket: suffix min of boundary starts, as a prefix
    // max over the reversed array of (L - start)
    for (int x = t; x < NBM; x += B) {
      bool big, head;
      kind(x, big, head);
      nxb[NBM - 1 - x] = (big || head) ? uint32_t(L) - hist[x] : 0u;
      if constexpr (S::kStaged) hd[x] = (big || head) ? uint32_t(x + 1) : 0u;
    }
    __syncthreads();
    smem_incl_max_w<B>(nxb, NBM, tmp32);
    if constexpr (S::kStaged) smem_incl_max_w<B>(hd, NBM, tmp32);  // group of each bucket
    for (int x = t; x < nb; x += B) {
      bool big, head;
      kind(x, big, head);
      const uint32_t sb = hist[x], cc = bend(x) - sb;
      if (big) {
        if (cc <= uint32_t(SS_RUN_MAX)) {
          queue_run(fin, fin_n, fin_cap, FinalEntry{g0 + sb, cc, dbuf, 0}, st, -6);
        } else {
          const unsigned q = atomicAdd(nxt_n, 1u);  // the fine split finds its key range itself
          if (q < nxt_cap) nxt[q] = HugeEntry{g0 + sb, cc, 0u, 0, dbuf, 0};
          else dev_fail(st, SP_ERR_INTERNAL, -7);
        }
      } else if (head) {
        // reversed index of x+1 holds max over buckets >= x+1 of (L - start) -> min start
        const uint32_t nx = (x + 1 < NBM) ? nxb[NBM - 1 - (x + 1)] : 0u;
        const uint32_t end = nx ? uint32_t(L) - nx : uint32_t(L);
        queue_run(fin, fin_n, fin_cap, FinalEntry{g0 + sb, (long long)(end - sb), dbuf, 0}, st, -6);
      }
    }
    __syncthreads();
    // pass 2 (hist now serves as the bucket cursors)
    const VT* svp = sbuf == BUF_TEMP ? tval + g0 : out_val + g0;
    if constexpr (S::kStaged) {
      // chunk by chunk: rank every entry within its group's share of the chunk, stage the
      // chunk by group, then write each share to the group's next free range
      constexpr int CH = B * U;
      for (long long c0 = 0; c0 < L; c0 += CH) {
        const int n = L - c0 < CH ? int(L - c0) : CH;
        for (int x = t; x < NBM; x += B) lh[x] = 0;
        __syncthreads();
        uint32_t k[U], pk[U];  // key; group << 16 | rank in the group's share (CH <= 2^16)
        VT v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = t + u * B;
          if (e < n) k[u] = key_at(c0 + e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = t + u * B;
          if (e < n) v[u] = ld_stream(svp + c0 + e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = t + u * B;
          pk[u] = 0xFFFFFFFFu;
          if (e >= n) continue;
          const uint32_t bk = bucket(k[u]);
          if (bk == 0xFFFFFFFFu) continue;
          const uint32_t g = hd[bk] - 1u;  // every non-empty bucket lies in a group
          pk[u] = (g << 16) | atomicAdd(&lh[g], 1u);
        }
        __syncthreads();
        for (int x = t; x < nb; x += B) {
          gb[x] = hist[x];
          hist[x] += lh[x];
        }
        const uint32_t nst = smem_excl_sum_w<B>(lh, NBM, tmp32);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (pk[u] == 0xFFFFFFFFu) continue;
          const uint32_t q = lh[pk[u] >> 16] + (pk[u] & 0xFFFFu);
          sk[q] = k[u];
          sv[q] = v[u];
        }
        __syncthreads();
        for (int i = t; i < int(nst); i += B) {
          const uint32_t key = sk[i], g = hd[bucket(key)] - 1u;
          const uint32_t q = gb[g] + (uint32_t(i) - lh[g]);
          if (q >= uint32_t(L)) continue;
          if (dbuf == BUF_TEMP) {
            st_stream(tkey + g0 + q, key);
            st_stream(tval + g0 + q, sv[i]);
          } else {
            st_stream(out_col + g0 + q, CI(key));
            st_stream(out_val + g0 + q, sv[i]);
          }
        }
        __syncthreads();
      }
    } else {
      // scatter entry by entry
      for (long long e0 = t; e0 < L; e0 += (long long)B * U) {
        uint32_t k[U];
        VT v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long e = e0 + (long long)u * B;
          if (e < L) k[u] = key_at(e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long e = e0 + (long long)u * B;
          if (e < L) v[u] = ld_stream(svp + e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long e = e0 + (long long)u * B;
          if (e >= L) continue;
          const uint32_t bk = bucket(k[u]);
          if (bk == 0xFFFFFFFFu) continue;
          const uint32_t q = atomicAdd(&hist[bk], 1u);
          if (q >= uint32_t(L)) continue;
          if (dbuf == BUF_TEMP) {
            st_stream(tkey + g0 + q, k[u]);
            st_stream(tval + g0 + q, v[u]);
          } else {
            st_stream(out_col + g0 + q, CI(k[u]));
            st_stream(out_val + g0 + q, v[u]);
          }
        }
      }
      __syncthreads();
    }
  }
}

// ---- phase 2: in-place sort of output rows ---------------------------------------------

template <class Cfg, class VT>
__host__ __device__ constexpr size_t ss_smem_bytes() {
  // values, keys in packed and bucket order, counters, bucket and source of each entry;
  // tiles add the per-row tables and the row-start bitmap (an entry's row is its rank
  // among the row starts, recomputed where needed: no per-entry row array, which keeps
  // a tile CTA small enough for 9 per SM)
  return size_t(Cfg::CAP) * (sizeof(VT) + 4 * 2 + 2 * 2) + size_t(Cfg::CNT) * 4 +
         (Cfg::kTiles ? size_t(Cfg::ROWS) * (4 * 2 + 2 * 2) + size_t(Cfg::WORDS) * 4 * 2 : 0);
}

// In-place exclusive sum of a[0, n); thread t owns the ceil(n / B) consecutive entries
// starting at t * ceil(n / B) (few per thread for the item sizes here, so the blocked
// layout's bank conflicts cost less than a second pass would).
template <int B>
__device__ __forceinline__ void ss_excl_sum(uint32_t* a, int n, uint32_t* tmp) {
  const int t = threadIdx.x;
  const int per = (n + B - 1) / B;
  const int x0 = t * per, x1 = x0 + per < n ? x0 + per : n;
  uint32_t s = 0;
  for (int x = x0; x < x1; ++x) s += a[x];
  uint32_t total;
  uint32_t run = block_excl_sum<B>(s, tmp, &total);
  for (int x = x0; x < x1; ++x) {
    const uint32_t v = a[x];
    a[x] = run;
    run += v;
  }
  __syncthreads();
}

// Work items: tiles [0, *ntiles) of the partition, or runs fin[0, *fin_n) (from the
// back of the list, fin[cap - 1 - k], with Cfg::kBack): rows of SS_TILE_MAX < L <=
// SS_RUN_MAX entries, in the output arrays, and k_split's runs, in the output or in the
// temporary arrays.  Every item's entries are loaded into shared memory
// before any of them is written back, so a run is sorted in place.  A bucket of more
// than SS_HEAVY keys (skewed keys) is written in bucket order and queued in hv[] as a
// run for a later pass, which buckets it over its own key range; without hv (the last
// pass) every bucket is ranked directly.
template <class Cfg, class CI, class VT>
__global__ void __launch_bounds__(Cfg::B, Cfg::MINB)
    k_seg_sort(const long long* __restrict__ vp, const long long* __restrict__ tile_first,
               const long long* __restrict__ ntiles_p, const FinalEntry* __restrict__ fin,
               const unsigned* __restrict__ fin_n, long long fin_cap, const uint32_t* __restrict__ tkey_g,
               const VT* __restrict__ tval_g, CI* __restrict__ out_col, VT* __restrict__ out_val,
               FinalEntry* __restrict__ hv, unsigned* hv_n, long long hv_cap, int key_bits, int heavy,
               DevStatus* st) {
  constexpr int B = Cfg::B, CAP = Cfg::CAP, ROWS = Cfg::ROWS, WORDS = Cfg::WORDS;
  extern __shared__ __align__(16) unsigned char smem[];
  VT* sval = reinterpret_cast<VT*>(smem);
  uint32_t* skey = reinterpret_cast<uint32_t*>(smem + size_t(CAP) * sizeof(VT));  // packed order
  uint32_t* tkey = skey + CAP;        // bucket order
  uint32_t* cnt = tkey + CAP;         // bucket counters
  uint16_t* slot = reinterpret_cast<uint16_t*>(cnt + Cfg::CNT);  // bucket of packed entry
  uint16_t* tidx = slot + CAP;        // packed entry of each bucket-order position
  // tiles only (runs allocate none of these)
  uint32_t* rdel = reinterpret_cast<uint32_t*>(tidx + CAP);  // per row: output offset from base - packed start
  float* rsc = reinterpret_cast<float*>(rdel + ROWS);        // per row: bucket scale
  uint32_t* bits = rdel + 2 * ROWS;   // row starts
  uint32_t* wpre = bits + WORDS;      // row starts in earlier words
  uint16_t* rps = reinterpret_cast<uint16_t*>(wpre + WORDS);  // per row: packed start
  uint16_t* rnm = rps + ROWS;         // per row: last bucket
  __shared__ uint32_t tmp32[B / 32 + 1];
  __shared__ uint32_t s_min, s_max;
  // tiles: row pointers vp[r0 .. r1] of the next tile, copied in while this one is sorted
  __shared__ long long pre_o[Cfg::kTiles ? ROWS + 1 : 1];
  const int t = threadIdx.x;
  const uint32_t kmax = key_bits >= 32 ? 0xFFFFFFFFu : (1u << key_bits) - 1u;
  const float isr = ss_inv_root(kmax);
  long long nitems;
  if constexpr (Cfg::kTiles) {
    nitems = *ntiles_p;
  } else {
    nitems = *fin_n;
    if (nitems > fin_cap) nitems = fin_cap;  // overflow was reported by the producer
  }

  // the next item's descriptor is loaded one item ahead, so its latency hides behind
  // the current item's sort
  long long pf0 = 0, pf1 = 0;  // tiles: row range
  FinalEntry pfe{0, 0, 0, 0};  // runs
  // tiles: start copying the row pointers of the tile whose range is in (pf0, pf1)
  auto prefetch_rows = [&](bool any) {
    if (any) {
      long long n = pf1 - pf0;
      n = n < 0 ? 0 : (n < ROWS ? n : ROWS);
      for (int x = t; x <= n; x += B) cp_async8(pre_o + x, vp + pf0 + x);
    }
    cp_async_commit();
  };
  if (blockIdx.x < nitems) {
    if constexpr (Cfg::kTiles) {
      pf0 = tile_first[blockIdx.x];
      pf1 = tile_first[blockIdx.x + 1];
      prefetch_rows(true);
    } else {
      pfe = fin[Cfg::kBack ? fin_cap - 1 - (long long)blockIdx.x : (long long)blockIdx.x];
    }
  }
  for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
    const long long nx = item + gridDim.x;
    if constexpr (Cfg::kTiles) {
      for (int w = t; w < WORDS; w += B) bits[w] = 0;
    } else if (t == 0) {
      s_min = 0xFFFFFFFFu;
      s_max = 0u;
    }
    long long base;
    int buf = BUF_OUT;
    int E;
    if constexpr (Cfg::kTiles) {
      uint32_t myL = 0;
      long long o0 = 0;
      const long long r0 = pf0;
      long long r1 = pf1;
      if (nx < nitems) {
        pf0 = tile_first[nx];
        pf1 = tile_first[nx + 1];
      }
      cp_async_wait_all();  // this tile's row pointers
      __syncthreads();
      base = pre_o[0];
      if (r1 - r0 > ROWS) {  // cannot happen: see RowsPartition
        if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -17);
        r1 = r0;
      }
      if (t < r1 - r0) {
        o0 = pre_o[t];
        const long long L = pre_o[t + 1] - o0;
        if (L > 0 && L <= Cfg::CP) {
          if (o0 - base > 0xFFFFFFFFll - CAP) dev_fail(st, SP_ERR_OVERFLOW, r0 + t);
          else myL = uint32_t(L);
        }
      }
      // packed start (high half) and rank among the item's rows (low half)
      uint32_t tot;
      const uint32_t pre = block_excl_sum<B>(myL ? ((myL << 16) | 1u) : 0u, tmp32, &tot);
      E = int(tot >> 16);  // <= 2 * Cfg::CP by the partition
      if (E > CAP) {       // cannot happen: see RowsPartition
        if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -19);
        prefetch_rows(nx < nitems);  // every thread has read pre_o (barriers above)
        __syncthreads();
        continue;
      }
      if (myL) {
        const uint32_t k = pre & 0xFFFFu, ps = pre >> 16;
        const uint32_t nb = ss_nb(myL);
        rps[k] = uint16_t(ps);
        rnm[k] = uint16_t(nb - 1);
        rsc[k] = float(nb) * isr;
        rdel[k] = uint32_t(o0 - base) - ps;
        atomicOr(&bits[ps >> 5], 1u << (ps & 31));
      }
      for (int x = t; x < E; x += B) cnt[x] = 0;
      __syncthreads();
      if (t < 32) {
        constexpr int WL = WORDS / 32;  // words per lane
        uint32_t c[WL], s = 0;
#pragma unroll
        for (int j = 0; j < WL; ++j) {
          c[j] = __popc(bits[t * WL + j]);
          s += c[j];
        }
        uint32_t run = warp_incl_sum(s) - s;
#pragma unroll
        for (int j = 0; j < WL; ++j) {
          wpre[t * WL + j] = run;
          run += c[j];
        }
      }
      __syncthreads();
      prefetch_rows(nx < nitems);  // the next tile's row pointers arrive during this sort
    } else {
      const FinalEntry fe = pfe;
      if (nx < nitems) pfe = fin[Cfg::kBack ? fin_cap - 1 - nx : nx];
      base = fe.off;
      buf = fe.buf;
      E = int(fe.len);
      if (fe.len < 0 || fe.len > CAP) {
        if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -18);
        E = 0;
      }
      for (int x = t; x < int(ss_nb(uint32_t(E))); x += B) cnt[x] = 0;
      __syncthreads();
    }
    // load: key and value of every packed entry, bucket histogram
    constexpr int LU = 4;
    if constexpr (Cfg::kTiles) {
      for (int x0 = t; x0 < E; x0 += B * LU) {
        uint32_t kk[LU], kr[LU], oo[LU];  // key, row, offset from base
        VT vv[LU];
#pragma unroll
        for (int u = 0; u < LU; ++u) {
          const int x = x0 + u * B;
          kr[u] = 0;
          oo[u] = 0;
          if (x < E) {
            const int w = x >> 5;
            kr[u] = wpre[w] + __popc(bits[w] & (0xFFFFFFFFu >> (31 - (x & 31)))) - 1u;
            oo[u] = rdel[kr[u]] + uint32_t(x);
          }
        }
        {  // tiles live in the output arrays
          const CI* kp = out_col + base;
          const VT* vq = out_val + base;
#pragma unroll
          for (int u = 0; u < LU; ++u)
            if (x0 + u * B < E) kk[u] = uint32_t(ld_stream(kp + oo[u]));
#pragma unroll
          for (int u = 0; u < LU; ++u)
            if (x0 + u * B < E) vv[u] = ld_stream(vq + oo[u]);
        }
#pragma unroll
        for (int u = 0; u < LU; ++u) {
          const int x = x0 + u * B;
          if (x >= E) continue;
          uint32_t key = kk[u];
          if (key > kmax) {  // a column outside [0, ncols)
            dev_fail(st, SP_ERR_INDEX_RANGE, base + oo[u]);
            key = kmax;
          }
          const uint32_t sl = rps[kr[u]] + ss_bucket(key, rsc[kr[u]], rnm[kr[u]]);
          skey[x] = key;
          sval[x] = vv[u];
          slot[x] = uint16_t(sl);
          atomicAdd(&cnt[sl], 1u);
        }
      }
    } else {
      // a single run (a row sorted alone or a key-range group of a long row): its
      // buckets span the run's own key range [min, max], found while loading
      uint32_t mn = 0xFFFFFFFFu, mx = 0u;
      const CI* kp = out_col + base;
      const VT* vq = out_val + base;
      for (int x0 = t; x0 < E; x0 += B * LU) {
        uint32_t kk[LU];
        VT vv[LU];
        if (buf == BUF_TEMP) {
#pragma unroll
          for (int u = 0; u < LU; ++u)
            if (x0 + u * B < E) kk[u] = ld_stream(tkey_g + base + x0 + u * B);
#pragma unroll
          for (int u = 0; u < LU; ++u)
            if (x0 + u * B < E) vv[u] = ld_stream(tval_g + base + x0 + u * B);
        } else {
#pragma unroll
          for (int u = 0; u < LU; ++u)
            if (x0 + u * B < E) kk[u] = uint32_t(ld_stream(kp + x0 + u * B));
#pragma unroll
          for (int u = 0; u < LU; ++u)
            if (x0 + u * B < E) vv[u] = ld_stream(vq + x0 + u * B);
        }
#pragma unroll
        for (int u = 0; u < LU; ++u) {
          const int x = x0 + u * B;
          if (x >= E) continue;
          uint32_t key = kk[u];
          if (key > kmax) {
            dev_fail(st, SP_ERR_INDEX_RANGE, base + x);
            key = kmax;
          }
          skey[x] = key;
          sval[x] = vv[u];
          mn = key < mn ? key : mn;
          mx = key > mx ? key : mx;
        }
      }
      mn = __reduce_min_sync(0xFFFFFFFFu, mn);
      mx = __reduce_max_sync(0xFFFFFFFFu, mx);
      if ((t & 31) == 0) {
        atomicMin(&s_min, mn);
        atomicMax(&s_max, mx);
      }
      __syncthreads();
      const uint32_t lo = s_min, w = s_max > s_min ? s_max - s_min : 0u;
      const uint32_t nb = ss_nb(uint32_t(E)), last = nb - 1;
      const float sc = float(nb) * ss_inv_root(w);
      for (int x = t; x < E; x += B) {
        const uint32_t sl = ss_bucket(skey[x] - lo, sc, last);
        slot[x] = uint16_t(sl);
        atomicAdd(&cnt[sl], 1u);
      }
    }
    __syncthreads();
    // counters in use: a tile's rows' buckets lie in [0, E), a run's in [0, ss_nb(E))
    ss_excl_sum<B>(cnt, Cfg::kTiles ? E : int(ss_nb(uint32_t(E))), tmp32);
    // scatter to bucket order; afterwards cnt[s] = end of bucket s, cnt[s-1] its start
    for (int x = t; x < E; x += B) {
      const uint32_t p = atomicAdd(&cnt[slot[x]], 1u);
      tkey[p] = skey[x];
      tidx[p] = uint16_t(x);
    }
    __syncthreads();
    // rank inside the bucket and write (heavy buckets: in bucket order, queued)
    CI* const oc = out_col + base;
    VT* const ov = out_val + base;
    for (int p = t; p < E; p += B) {
      const uint32_t x = tidx[p], k = tkey[p];
      const uint32_t s = slot[x];
      const uint32_t end = cnt[s], start = s ? cnt[s - 1] : 0u;
      uint32_t rd = 0u;
      if constexpr (Cfg::kTiles) {  // the entry's row: the row starts at or before x
        const int w = int(x >> 5);
        rd = rdel[wpre[w] + __popc(bits[w] & (0xFFFFFFFFu >> (31 - (x & 31)))) - 1u];
      }
      if (hv && end - start > uint32_t(heavy)) {
        st_stream(oc + rd + p, CI(k));
        st_stream(ov + rd + p, sval[x]);
        if (uint32_t(p) == start) {
          const unsigned q = atomicAdd(hv_n, 1u);
          if (q < hv_cap) hv[q] = FinalEntry{base + rd + start, (long long)(end - start), BUF_OUT, 0};
          else dev_fail(st, SP_ERR_INTERNAL, -22);
        }
        continue;
      }
      uint32_t rank = 0;
      for (uint32_t q = start; q < end; ++q) rank += tkey[q] < k;
      const uint32_t g = rd + start + rank;
      st_stream(oc + g, CI(k));
      st_stream(ov + g, sval[x]);
    }
    __syncthreads();
  }
}

// ---- host side --------------------------------------------------------------------------
struct RowsWs {
  long long ntiles_cap = 0, nchunks = 0, fin_cap = 0, huge_cap = 0, nxt_cap = 0, hv_cap = 0;
  long long* tile_first = nullptr;
  long long* chunk_first = nullptr;
  long long* ntiles = nullptr;
  unsigned* counters = nullptr;  // [0..1] run list counts (front, back) [2] spare [3..4] tickets [5] spare
                                 // [6..7] heavy-run counts [8..9] zero (no tiles)
                                 // [10..11] huge list counts [12..13] nxt list counts
  FinalEntry* fin = nullptr;
  HugeEntry* huge = nullptr;
  HugeEntry* nxt = nullptr;
  FinalEntry* hv[2] = {nullptr, nullptr};  // heavy buckets queued for the next pass
  uint32_t* tkey = nullptr;
  void* tval = nullptr;
  char* scan_ws = nullptr;
  unsigned* huge_n() const { return counters + 10; }
  unsigned* nxt_n() const { return counters + 12; }
};

constexpr int kRowsSlots = 12;

// extra_fin: runs a caller queues itself (beyond the partition's and the split's)
inline void rows_caps(long long nrows, long long nnz, RowsWs* w, long long extra_fin = 0) {
  w->ntiles_cap = (nnz + SS_ROW_W * nrows) / SS_TILE_MAX + 1;
  w->nchunks = (nnz + GC_CH - 1) / GC_CH;
  w->fin_cap = 2 * (3 * (nnz / GROUP_CAP) + nnz / SS_RUN_MAX + 16) + nnz / SS_TILE_MAX + 1 + extra_fin;
  w->huge_cap = nnz / SS_RUN_MAX + 1;
  w->nxt_cap = nnz / SS_RUN_MAX + 1;
  w->hv_cap = nnz / (SS_HEAVY + 1) + 1;  // heavy buckets are disjoint runs of > SS_HEAVY
}

// Workspace of run_rows; `sort` = false reserves only what the gather needs.
inline void rows_reserve(Carver& cv, long long nrows, long long nnz, size_t vbytes, size_t* off,
                         bool sort = true, long long extra_fin = 0) {
  RowsWs w;
  rows_caps(nrows, nnz, &w, extra_fin);
  if (!sort) w.fin_cap = w.huge_cap = w.nxt_cap = w.hv_cap = 0;
  const bool need_temp = sort && nnz > SS_RUN_MAX;
  off[0] = cv.reserve(size_t(w.ntiles_cap + 1) * 8);
  off[1] = cv.reserve(size_t(w.nchunks + 1) * 8);
  off[2] = cv.reserve(8);
  off[3] = cv.reserve(16 * 4);
  off[4] = cv.reserve(size_t(w.fin_cap) * sizeof(FinalEntry));
  off[5] = cv.reserve(size_t(w.huge_cap) * sizeof(HugeEntry));
  off[6] = cv.reserve(size_t(w.nxt_cap) * sizeof(HugeEntry));
  off[7] = cv.reserve(need_temp ? size_t(nnz) * 4 : 0);
  off[8] = cv.reserve(need_temp ? size_t(nnz) * vbytes : 0);
  off[9] = cv.reserve(scan_ws_bytes(nrows));
  off[10] = cv.reserve(size_t(w.hv_cap) * sizeof(FinalEntry));
  off[11] = cv.reserve(size_t(w.hv_cap) * sizeof(FinalEntry));
}

inline RowsWs rows_bind(const Carver& cv, long long nrows, long long nnz, const size_t* off,
                        bool sort = true, long long extra_fin = 0) {
  RowsWs w;
  rows_caps(nrows, nnz, &w, extra_fin);
  if (!sort) w.fin_cap = w.huge_cap = w.nxt_cap = w.hv_cap = 0;
  w.tile_first = cv.at<long long>(off[0]);
  w.chunk_first = cv.at<long long>(off[1]);
  w.ntiles = cv.at<long long>(off[2]);
  w.counters = cv.at<unsigned>(off[3]);
  w.fin = cv.at<FinalEntry>(off[4]);
  w.huge = cv.at<HugeEntry>(off[5]);
  w.nxt = cv.at<HugeEntry>(off[6]);
  w.tkey = cv.at<uint32_t>(off[7]);
  w.tval = cv.at<void>(off[8]);
  w.scan_ws = cv.at<char>(off[9]);
  w.hv[0] = cv.at<FinalEntry>(off[10]);
  w.hv[1] = cv.at<FinalEntry>(off[11]);
  return w;
}

// Phase-1 functor for callers that only sort (the rows are in place already).
template <class CIt, class VTt>
struct NoGather {
  using CI = CIt;
  using VT = VTt;
  __device__ long long src(long long) const { return 0; }
  __device__ CI col(long long) const { return CI(0); }
  __device__ CI map(long long, CI c) const { return c; }
  __device__ VT val(long long) const { return VT(0); }
};

// Key-range split of the rows queued in w.huge (counts w.huge_n()) into runs queued in w.fin.
template <class CI, class VT>
sp_status split_queued(sp_ctx* ctx, cudaStream_t s, const RowsWs& w, CI* out_col, VT* out_val) {
  const int nsm = ctx->num_sms;
  VT* tval = static_cast<VT*>(w.tval);
  constexpr size_t csm = split_smem_bytes<SplitCoarse, VT>(), fsm = split_smem_bytes<SplitFine, VT>();
  SP_CUDA(set_smem(k_split<SplitCoarse, CI, VT>, csm));
  SP_CUDA(set_smem(k_split<SplitFine, CI, VT>, fsm));
  {
    SP_PHASE(SP_PHASE_HUGE);
    k_split<SplitCoarse, CI, VT><<<SplitCoarse::MINB * nsm, SplitCoarse::B, csm, s>>>(
        w.huge, w.huge_n(), w.huge_cap, w.counters + 3, w.tkey, tval, out_col, out_val, w.fin, w.counters + 0,
        w.fin_cap, w.nxt, w.nxt_n(), w.nxt_cap, ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  // the fine split: the coarse buckets that hold more than SS_RUN_MAX entries (skewed keys
  // or very long rows); an empty list costs one short launch
  {
    SP_PHASE(SP_PHASE_HUGE);
    k_split<SplitFine, CI, VT><<<SplitFine::MINB * nsm, SplitFine::B, fsm, s>>>(
        w.nxt, w.nxt_n(), w.nxt_cap, w.counters + 4, w.tkey, tval, out_col, out_val, w.fin, w.counters + 0,
        w.fin_cap, w.nxt, w.counters + 5, 0, ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  return SP_OK;
}

// Sorts the runs queued in w.fin (counters 0 and 1: its two ends), then the heavy buckets
// queued by any sort pass (counters 6, 7), in place.
template <class CI, class VT>
sp_status sort_runs(sp_ctx* ctx, cudaStream_t s, const RowsWs& w, int key_bits, CI* out_col, VT* out_val) {
  const int nsm = ctx->num_sms;
  const int heavy = ctx->cur.heavy;
  VT* tval = static_cast<VT*>(w.tval);
  const long long* no_tiles = reinterpret_cast<const long long*>(w.counters + 8);
  using SsRun = SsRunT<VT>;
  constexpr size_t rsm = ss_smem_bytes<SsRun, VT>(), ssm = ss_smem_bytes<SsRunS, VT>();
  // the runs of at most SS_SMALL_RUN entries (the back of the list), then the others
  SP_CUDA(set_smem(k_seg_sort<SsRunS, CI, VT>, ssm));
  {
    SP_PHASE(SP_PHASE_LONG);
    k_seg_sort<SsRunS, CI, VT><<<SsRunS::MINB * nsm, SsRunS::B, ssm, s>>>(
        nullptr, nullptr, no_tiles, w.fin, w.counters + 1, w.fin_cap, w.tkey, tval, out_col, out_val, w.hv[0],
        w.counters + 6, w.hv_cap, key_bits, heavy, ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  SP_CUDA(set_smem(k_seg_sort<SsRun, CI, VT>, rsm));
  {
    SP_PHASE(SP_PHASE_LONG);
    k_seg_sort<SsRun, CI, VT><<<SsRun::MINB * nsm, SsRun::B, rsm, s>>>(
        nullptr, nullptr, no_tiles, w.fin, w.counters + 0, w.fin_cap, w.tkey, tval, out_col, out_val, w.hv[0],
        w.counters + 6, w.hv_cap, key_bits, heavy, ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  // heavy buckets: runs over their own key range; the last pass ranks every bucket
  for (int pass = 0; pass < SS_PASSES; ++pass) {
    const int a = pass & 1, b = a ^ 1;
    const bool last = pass == SS_PASSES - 1;
    SP_CUDA(cudaMemsetAsync(w.counters + 6 + b, 0, 4, s));
    {
      SP_PHASE(SP_PHASE_LONG);
      k_seg_sort<SsRun, CI, VT><<<SsRun::MINB * nsm, SsRun::B, rsm, s>>>(
          nullptr, nullptr, no_tiles, w.hv[a], w.counters + 6 + a, w.hv_cap, w.tkey, tval, out_col, out_val,
          last ? nullptr : w.hv[b], w.counters + 6 + b, w.hv_cap, key_bits, heavy, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
  }
  return SP_OK;
}

// Sorts in place the rows a caller queued itself in w.fin / w.huge (counters 0, 1 and
// w.huge_n(), zeroed with the rest of w.counters before the caller queued them).
template <class CI, class VT>
sp_status sort_queued(sp_ctx* ctx, cudaStream_t s, const RowsWs& w, int key_bits, CI* out_col, VT* out_val) {
  SP_TRY((split_queued<CI, VT>(ctx, s, w, out_col, out_val)));
  return sort_runs<CI, VT>(ctx, s, w, key_bits, out_col, out_val);
}

// Partition the output rows (row pointer vp, nnz entries), gather them with `gs`
// (when given) and sort every row in place (when `sort`).
template <class CI, class VT, class Gs>
sp_status run_rows(sp_ctx* ctx, cudaStream_t s, const long long* vp, long long nrows, long long nnz,
                   int key_bits, const RowsWs& w, const Gs* gs, bool sort, CI* out_col, VT* out_val) {
  if (nrows == 0 || nnz == 0) return SP_OK;
  SP_CUDA(cudaMemsetAsync(w.counters, 0, 16 * 4, s));
  const int nsm = ctx->num_sms;
  unsigned* fin_n = w.counters + 0;
  unsigned* huge_n = w.huge_n();
  // kernel shapes of this call (context options or the tuning table)
  const bool large_tiles = ctx->cur.tile_shape == 1;
  const long long tmax = large_tiles ? SsTileL::CP : SsTile::CP;
  const int heavy = ctx->cur.heavy;
  SP_TRY(launch_scan(ctx, s, RowsWeight{vp, tmax},
                     RowsPartition{vp, nrows, w.ntiles_cap, w.tile_first, w.ntiles, w.nchunks, w.chunk_first,
                                   w.fin, fin_n, w.fin_cap, w.huge, huge_n, w.huge_cap, key_bits,
                                   sort ? 1 : 0, tmax, ctx->dstatus},
                     nrows, w.scan_ws, SP_PHASE_PARTITION));
  if (gs) {
    if (w.nchunks > 0x7fffffffll) return SP_ERR_OVERFLOW;
    {
      SP_PHASE(SP_PHASE_GATHER);
      const long long g = w.nchunks < (long long)GC_MINB * nsm ? w.nchunks : (long long)GC_MINB * nsm;  // persistent
      k_gather_chunks<Gs><<<unsigned(g), GC_BLOCK, 0, s>>>(*gs, vp, nrows, nnz, w.chunk_first, w.nchunks,
                                                           out_col, out_val);
    }
    SP_CUDA(cudaGetLastError());
  }
  if (!sort) return SP_OK;
  // The key-range split (rows longer than SS_RUN_MAX, queued by the partition) and the
  // tile sort (rows of at most tmax) touch disjoint rows.  With the context's overlap on,
  // the split runs on the context's side stream, whose higher priority dispatches its CTAs
  // (a hub row's first) ahead of the tiles', while the tiles run on `s`: the SMs that the
  // split's tail leaves idle take tiles.  The runs, which the split queues, wait for both.
  constexpr size_t tsm = ss_smem_bytes<SsTile, VT>(), lsm = ss_smem_bytes<SsTileL, VT>();
  SP_CUDA(set_smem(large_tiles ? k_seg_sort<SsTileL, CI, VT> : k_seg_sort<SsTile, CI, VT>, large_tiles ? lsm : tsm));
  const bool fork = nnz > SS_RUN_MAX && ctx->overlap && ctx->side;
  if (fork) {
    SP_CUDA(cudaEventRecord(ctx->fork_ev, s));
    SP_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0));
    const sp_status st = split_queued<CI, VT>(ctx, ctx->side, w, out_col, out_val);
    SP_CUDA(cudaEventRecord(ctx->join_ev, ctx->side));
    if (st != SP_OK) {
      SP_CUDA(cudaStreamWaitEvent(s, ctx->join_ev, 0));
      return st;
    }
  } else if (nnz > SS_RUN_MAX) {
    SP_TRY((split_queued<CI, VT>(ctx, s, w, out_col, out_val)));
  }
  // tiles, then the runs, then the heavy buckets queued by either
  const unsigned* no_runs = w.counters + 8;
  VT* tval = static_cast<VT*>(w.tval);
  {
    SP_PHASE(SP_PHASE_TILE);
    if (large_tiles)
      k_seg_sort<SsTileL, CI, VT><<<SsTileL::MINB * nsm, SsTileL::B, lsm, s>>>(
          vp, w.tile_first, w.ntiles, w.fin, no_runs, 0, w.tkey, tval, out_col, out_val, w.hv[0],
          w.counters + 6, w.hv_cap, key_bits, heavy, ctx->dstatus);
    else
      k_seg_sort<SsTile, CI, VT><<<SsTile::MINB * nsm, SsTile::B, tsm, s>>>(
          vp, w.tile_first, w.ntiles, w.fin, no_runs, 0, w.tkey, tval, out_col, out_val, w.hv[0],
          w.counters + 6, w.hv_cap, key_bits, heavy, ctx->dstatus);
  }
  const cudaError_t launched = cudaGetLastError();
  if (fork) SP_CUDA(cudaStreamWaitEvent(s, ctx->join_ev, 0));
  SP_CUDA(launched);
  return sort_runs<CI, VT>(ctx, s, w, key_bits, out_col, out_val);
}

}  // namespace sp
