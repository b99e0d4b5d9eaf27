// Gather -> remap -> per-row sort -> store, the Identify / Build pipeline of the paper
// (Algorithm 2's fill pass and the Build step's sort, Sec. 3.1) restated for one GPU.
//
// Output rows are laid out contiguously by a row-pointer array `vp` (int64, one entry
// per listed row plus one).  Each output row is filled from one or two source runs
// described by a Loader:
//   struct Loader {
//     using CI = ...;  using VT = ...;           // column index / value word types
//     static constexpr bool kAllKept;            // no source entry is ever dropped
//     RowSrc row(int64 r) const;                 // source runs of listed row r
//     const CI* cols(int part) const;            // column / value arrays of run `part`
//     const VT* vals(int part) const;
//     bool map(int part, int64 c, uint32& key) const;
//         // new column of a source entry with column c, or false if it is dropped
//   };
// Source entries are read in batches (struct Batch): every thread first issues the
// column loads of U entries, then their map lookups, then their value loads, so that
// U independent chains of dependent loads are in flight per thread.
// Rows are routed by length:
//   * rows whose source is at most TILE_CP entries go through k_tile: one CTA gathers
//     the rows of a tile (rows starting in one TILE_CP-wide window of the coordinate
//     vp[r] + TILE_ROW_W * r) into shared memory, packed back to back, sorts every row
//     there and writes them to their output positions;
//   * rows with longer sources but at most LONG_CAP output entries: k_long, one CTA per
//     row;
//   * rows with more than LONG_CAP output entries: k_huge partitions the row by key
//     range into 2^14 buckets (two streaming passes, through a global buffer) and hands
//     groups of consecutive buckets of at most LONG_CAP entries to k_long.
// The shared-memory sort ("bucket-rank"): a segment of length len gets
// 2^(ceil(log2 len) - 1) buckets spaced evenly in sqrt(key); the histogram is built
// while loading, one block-wide exclusive scan of the counts gives every bucket's
// output position, keys are scattered to their buckets and ranked inside them.
// Buckets of more than T_RANK keys (rare) are refined by repeated bucketing over their
// own [min, max] until at most T_SMALL keys remain, then ranked.  Keys are unique
// within a row, so every correct sort gives the same canonical order.
#pragma once

#include "common.cuh"

namespace sp {

struct RowSrc {
  long long s0, s1;  // start of run 0 / run 1 in the source arrays
  long long n0, n1;  // lengths (n1 = 0 for single-run sources)
};

// U source entries read together (see the file comment).
template <class Ld, int U>
struct Batch {
  long long pos[U];
  int part[U];
  bool valid[U];
  bool kept[U];
  uint32_t key[U];
  typename Ld::VT v[U];
  __device__ __forceinline__ void run(const Ld& ld) {
    using CI = typename Ld::CI;
    CI c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) c[u] = valid[u] ? ld_stream(ld.cols(part[u]) + pos[u]) : CI(0);
    if constexpr (Ld::kLoadVals && Ld::kAllKept) {
      // nothing is dropped: the value loads need not wait for the map lookups
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (valid[u]) v[u] = ld_stream(ld.vals(part[u]) + pos[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) kept[u] = valid[u] && ld.map(part[u], (long long)c[u], key[u]);
    if constexpr (Ld::kLoadVals && !Ld::kAllKept) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (kept[u]) v[u] = ld_stream(ld.vals(part[u]) + pos[u]);
    }
  }
  // entry e of a row's source runs
  __device__ __forceinline__ void at(int u, const RowSrc& rs, long long e) {
    part[u] = e < rs.n0 ? 0 : 1;
    pos[u] = part[u] ? rs.s1 + (e - rs.n0) : rs.s0 + e;
  }
};

constexpr int LOAD_U = 4;  // entries per thread per batch

// A loader view that never loads values (histogram and counting passes).
template <class Ld>
struct KeyOnly {
  using CI = typename Ld::CI;
  struct Nothing {};
  using VT = Nothing;
  static constexpr bool kLoadVals = false;
  static constexpr bool kAllKept = Ld::kAllKept;
  Ld ld;
  __device__ __forceinline__ const CI* cols(int part) const { return ld.cols(part); }
  __device__ __forceinline__ bool map(int part, long long c, uint32_t& key) const {
    return ld.map(part, c, key);
  }
};

// A loader view for counting passes: membership only (no key, no value loads).
template <class Ld>
struct CountOnly {
  using CI = typename Ld::CI;
  struct Nothing {};
  using VT = Nothing;
  static constexpr bool kLoadVals = false;
  static constexpr bool kAllKept = false;
  Ld ld;
  __device__ __forceinline__ const CI* cols(int part) const { return ld.cols(part); }
  __device__ __forceinline__ bool map(int part, long long c, uint32_t&) const {
    return ld.test(part, c);
  }
};

constexpr int T_SMALL = 16;  // refinement stops at buckets of this many keys
constexpr int T_RANK = 32;   // bucket-rank ranks buckets of up to this many keys
constexpr int TILE_BLOCK = 256;
constexpr int TILE_CAP = 2048;
constexpr int TILE_CP = TILE_CAP / 2;  // longest source row a tile accepts
constexpr int TILE_ROW_W = 4;          // tile partition weight of a row (bounds rows/tile)
constexpr int LONG_BLOCK = 512;
constexpr int LONG_CAP = 4096;
constexpr int HUGE_BLOCK = 1024;
constexpr int HUGE_NB_LOG = 14;
constexpr int HUGE_NB = 1 << HUGE_NB_LOG;
constexpr int GROUP_CAP = LONG_CAP / 2;

enum BufId : int { BUF_TEMP = 0, BUF_OUT = 1 };

struct FinalEntry {  // a run of at most LONG_CAP entries left to sort in place
  long long off;
  long long len;
  int buf;
  int pad;
};
struct HugeEntry {  // a run longer than LONG_CAP, keys in [lo, lo + 2^wb)
  long long off;
  long long len;
  unsigned lo;
  int wb;
  int buf;
  int pad;
};

// Shared-memory views used by the sort.
struct SortView {
  uint32_t* key;   // CAP
  uint32_t* seg;   // CAP: (segment start << 16) | segment length; 0 = unused position
  uint32_t* cnt;   // CAP
  uint32_t* lo;    // CAP/16 (indexed by segment start >> 4)
  uint32_t* hi;
  uint32_t* base;
  uint16_t* idx;   // CAP: position of the element's value in the staging array
};

template <class VT, int CAP>
__host__ __device__ constexpr size_t sort_smem_bytes() {
  return size_t(CAP) * sizeof(VT) + size_t(CAP) * 4 * 3 + size_t(CAP / 16) * 4 * 3 +
         size_t(CAP) * 2;
}

template <class VT, int CAP>
__device__ __forceinline__ SortView carve_sort(unsigned char* raw, VT** sval) {
  SortView v;
  *sval = reinterpret_cast<VT*>(raw);
  v.key = reinterpret_cast<uint32_t*>(raw + size_t(CAP) * sizeof(VT));
  v.seg = v.key + CAP;
  v.cnt = v.seg + CAP;
  v.lo = v.cnt + CAP;
  v.hi = v.lo + CAP / 16;
  v.base = v.hi + CAP / 16;
  v.idx = reinterpret_cast<uint16_t*>(v.base + CAP / 16);
  return v;
}

// Sort every segment of positions [0, E) by key until each segment holds at most
// T_SMALL keys, with keys of a lower segment all smaller than those of a higher one.
// global_first: round 0 buckets over [0, 2^key_bits) (for a first pass over whole
// rows); otherwise every round uses each segment's [min, max] (refining buckets).
template <int BLOCK, int ITEMS>
__device__ void refine_sort(const SortView& b, int E, int key_bits, uint32_t* tmp32,
                            DevStatus* st, bool global_first = true) {
  const int t = threadIdx.x;
  __shared__ int s_more;
  bool more = true;
  for (int round = 0; more; ++round) {
    // per item: key, segment word, (slot << 16 | value index), new position
    uint32_t k[ITEMS], sg[ITEMS], si[ITEMS], ps[ITEMS];
    bool any = false;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t + j * BLOCK;
      sg[j] = 0;
      k[j] = 0;
      si[j] = 0;
      if (x < E) {
        sg[j] = b.seg[x];
        k[j] = b.key[x];
        si[j] = b.idx[x];
        b.cnt[x] = 0;
      }
      any |= (sg[j] & 0xFFFFu) > uint32_t(T_SMALL);
    }
    const bool adaptive = round > 0 || !global_first;
    if (adaptive && !__syncthreads_or(any)) break;
    if (round >= 12) {  // impossible for 32-bit keys (each round removes >= 4 bits)
      if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -2);
      break;
    }
    if (t == 0) s_more = 0;
    // round 0 buckets over the whole key range [0, 2^key_bits) (keys of a random
    // relabelling are uniform there); later rounds use each segment's [min, max]
    if (adaptive) {
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        const int x = t + j * BLOCK;
        const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
        if (len > uint32_t(T_SMALL) && uint32_t(x) == s) {
          b.lo[s >> 4] = 0xFFFFFFFFu;
          b.hi[s >> 4] = 0u;
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
        if (len > uint32_t(T_SMALL)) {
          atomicMin(&b.lo[s >> 4], k[j]);
          atomicMax(&b.hi[s >> 4], k[j]);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
      if (len > uint32_t(T_SMALL)) {
        const int nbl = ceil_log2_u32(len) - 1;  // nb = 2^nbl < len buckets
        uint32_t L = 0;
        int bits = key_bits;
        if (adaptive) {
          L = b.lo[s >> 4];
          const uint32_t range = b.hi[s >> 4] - L;
          bits = range ? 32 - __clz(range) : 0;
        }
        const int sh = bits > nbl ? bits - nbl : 0;
        uint32_t off = (k[j] - L) >> sh;
        if (off >= (1u << nbl)) off = (1u << nbl) - 1;  // keys beyond key_bits (invalid input)
        const uint32_t slot = s + off;
        si[j] = (slot << 16) | (si[j] & 0xFFFFu);
        atomicAdd(&b.cnt[slot], 1u);
      }
    }
    __syncthreads();
    smem_excl_sum<BLOCK, ITEMS>(b.cnt, E, tmp32);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t + j * BLOCK;
      const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
      if (len > uint32_t(T_SMALL) && uint32_t(x) == s) b.base[s >> 4] = b.cnt[s];
    }
    __syncthreads();
    // scatter into bucket order; cnt[slot] runs from the bucket start to its end
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
      ps[j] = 0;
      if (len > uint32_t(T_SMALL)) {
        const uint32_t slot = si[j] >> 16;
        const uint32_t pos = s + atomicAdd(&b.cnt[slot], 1u) - b.base[s >> 4];
        ps[j] = pos;
        b.key[pos] = k[j];
        b.idx[pos] = uint16_t(si[j] & 0xFFFFu);
      }
    }
    __syncthreads();
    // new segment = the element's bucket: [end of previous bucket, end of own bucket)
    bool big = false;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
      if (len > uint32_t(T_SMALL)) {
        const uint32_t slot = si[j] >> 16;
        const uint32_t bse = b.base[s >> 4];
        const uint32_t e = s + b.cnt[slot] - bse;
        const uint32_t a = slot == s ? s : s + b.cnt[slot - 1] - bse;
        b.seg[ps[j]] = (a << 16) | (e - a);
        big |= (e - a) > uint32_t(T_SMALL);
      }
    }
    more = __syncthreads_or(big);
  }
}

// Rank of position x within its final (<= T_SMALL) segment; returns the sorted
// position, or -1 for unused positions.
__device__ __forceinline__ int final_pos(const SortView& b, int x) {
  const uint32_t sg = b.seg[x];
  const uint32_t len = sg & 0xFFFFu;
  if (!len) return -1;
  const uint32_t s = sg >> 16;
  const uint32_t k = b.key[x];
  uint32_t rank = 0;
  for (uint32_t y = s; y < s + len; ++y) rank += b.key[y] < k;
  return int(s + rank);
}

// ------------------------------------------------------------------------------
// Bucket-rank: the common single pass.  Each segment of length len gets
// 2^(ceil(log2 len)-1) buckets over the whole key range [0, 2^key_bits), i.e. about
// one key per bucket for uniformly relabelled columns; one block-wide exclusive scan of
// the bucket counts gives every bucket's output position; keys are scattered to their
// bucket and ranked inside it.  A bucket of more than T_RANK keys (skewed keys) makes
// the whole block fall back to refine_sort.
// ------------------------------------------------------------------------------
struct BRView {
  uint32_t* key;    // CAP: key of entry x (left unchanged)
  uint32_t* seg;    // CAP: (segment start << 16) | segment length of entry x; 0 = unused
  uint32_t* cnt;    // CAP: bucket counters, slot = segment start + bucket
  uint32_t* tkey;   // CAP: keys in bucket order (fallback: lo/hi/base live here)
  uint16_t* tidx;   // CAP: entry of each bucket-ordered key (fallback: value index)
  uint16_t* tslot;  // CAP: bucket slot of each bucket-ordered key
  uint16_t* ord;    // CAP: ord[f] = entry whose sorted position is f
};

template <int CAP>
__host__ __device__ constexpr size_t br_smem_bytes() {
  return size_t(CAP) * (4 * 4 + 2 * 3);
}

template <int CAP>
__device__ __forceinline__ BRView carve_br(unsigned char* raw) {
  BRView v;
  v.key = reinterpret_cast<uint32_t*>(raw);
  v.seg = v.key + CAP;
  v.cnt = v.seg + CAP;
  v.tkey = v.cnt + CAP;
  v.tidx = reinterpret_cast<uint16_t*>(v.tkey + CAP);
  v.tslot = v.tidx + CAP;
  v.ord = v.tslot + CAP;
  return v;
}

// Bucket of key k in its segment: nb = 2^(ceil(log2 len) - 1) buckets spaced evenly in
// sqrt(k) over [0, 2^key_bits).  Any non-decreasing map keeps buckets in key order;
// the square root stays balanced both for uniformly relabelled columns and for
// orderings that crowd keys at the low end (degree-descending relabelling of a
// power-law graph), where evenly spaced buckets in k overflow.  `isr` is
// 2^(-key_bits/2).
__device__ __forceinline__ uint32_t br_slot(uint32_t sg, uint32_t k, float isr) {
  const uint32_t len = sg & 0xFFFFu, s = sg >> 16;
  const int nbl = len > 1 ? ceil_log2_u32(len) - 1 : 0;
  const uint32_t nb = 1u << nbl;
  uint32_t b = uint32_t(sqrtf(float(k)) * (float(nb) * isr));
  if (b >= nb) b = nb - 1;  // keys beyond key_bits only come from invalid input
  return s + b;
}

__device__ __forceinline__ float br_isr(int key_bits) { return exp2f(-0.5f * float(key_bits)); }

// Sorts the segments of entries [0, E); on return ord[0 .. n) holds the entry index for
// every sorted position (n = number of used entries) and key[] is unchanged.
// Views for refining heavy buckets after the bucket pass: keys and entry indices in
// bucket order (tkey, tidx), segment words in seg[] (bucket order; 0 = final already),
// counters in cnt[], and the per-segment min/max/base words in the tslot/ord storage.
template <int CAP>
__device__ __forceinline__ SortView heavy_view(const BRView& v) {
  SortView r;
  r.key = v.tkey;
  r.seg = v.seg;
  r.cnt = v.cnt;
  r.lo = reinterpret_cast<uint32_t*>(v.tslot);
  r.hi = r.lo + CAP / 16;
  r.base = r.hi + CAP / 16;
  r.idx = v.tidx;
  return r;
}

// With hist_done, cnt[0 .. E) already holds the bucket histogram (built while loading).
template <int BLOCK, int CAP>
__device__ int bucket_rank_sort(const BRView& v, int E, int key_bits, uint32_t* tmp32,
                                DevStatus* st, bool hist_done = false) {
  constexpr int ITEMS = CAP / BLOCK;
  const int t = threadIdx.x;
  const float isr = br_isr(key_bits);
  if (!hist_done) {
    for (int x = t; x < E; x += BLOCK) v.cnt[x] = 0;
    __syncthreads();
    for (int x = t; x < E; x += BLOCK) {
      const uint32_t sg = v.seg[x];
      if (sg & 0xFFFFu) atomicAdd(&v.cnt[br_slot(sg, v.key[x], isr)], 1u);
    }
  }
  __syncthreads();
  const int n = int(smem_excl_sum<BLOCK, ITEMS>(v.cnt, E, tmp32));
  for (int x = t; x < E; x += BLOCK) v.ord[x] = 0;
  for (int x = t; x < E; x += BLOCK) {
    const uint32_t sg = v.seg[x];
    if (!(sg & 0xFFFFu)) continue;
    const uint32_t k = v.key[x];
    const uint32_t slot = br_slot(sg, k, isr);
    const uint32_t p = atomicAdd(&v.cnt[slot], 1u);
    if (p < uint32_t(CAP)) {
      v.tkey[p] = k;
      v.tidx[p] = uint16_t(x);
      v.tslot[p] = uint16_t(slot);
    }
  }
  __syncthreads();
  bool heavy = false;
  uint32_t bw[ITEMS];  // per position: (bucket start << 16 | length) of a heavy bucket, else 0
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int p = t + j * BLOCK;
    bw[j] = 0;
    if (p >= n) continue;
    const uint32_t slot = v.tslot[p], k = v.tkey[p];
    const uint32_t x = v.tidx[p];
    const uint32_t s = v.seg[x] >> 16;
    const uint32_t end = v.cnt[slot];
    const uint32_t start = slot == s ? s : v.cnt[slot - 1];
    if (end - start > uint32_t(T_RANK)) {
      heavy = true;
      bw[j] = (start << 16) | (end - start);
      continue;
    }
    uint32_t rank = 0;
    for (uint32_t q = start; q < end; ++q) rank += v.tkey[q] < k;
    if (start + rank < uint32_t(CAP)) v.ord[start + rank] = uint16_t(x);
  }
  if (__syncthreads_or(heavy)) {
    // skewed keys: refine only the heavy buckets, in bucket order, from their own
    // key range; light buckets are final already
    SortView r = heavy_view<CAP>(v);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int p = t + j * BLOCK;
      if (p < n) v.seg[p] = bw[j];
    }
    __syncthreads();
    refine_sort<BLOCK, ITEMS>(r, n, key_bits, tmp32, st, false);
    for (int p = t; p < n; p += BLOCK) {
      const int fp = final_pos(r, p);
      if (fp >= 0) v.ord[fp] = v.tidx[p];
    }
    __syncthreads();
  }
  return n;
}

// The same sort with the histogram already accumulated during the load pass (cnt[]
// holds the bucket counts of entries [0, E)), and the rank pass handing every entry
// straight to `out(f, x, key)` (f = sorted position, x = entry) instead of building
// ord[].  Entries of buckets larger than T_RANK send the block to refine_sort, whose
// results are handed to `out` again (the earlier calls were already correct).
template <int BLOCK, int CAP, class Out>
__device__ void br_finish(const BRView& v, int E, int key_bits, uint32_t* tmp32, DevStatus* st,
                          const Out& out) {
  constexpr int ITEMS = CAP / BLOCK;
  const int t = threadIdx.x;
  const float isr = br_isr(key_bits);
  const int n = int(smem_excl_sum<BLOCK, ITEMS>(v.cnt, E, tmp32));
  for (int x = t; x < E; x += BLOCK) {
    const uint32_t sg = v.seg[x];
    if (!(sg & 0xFFFFu)) continue;
    const uint32_t k = v.key[x];
    const uint32_t slot = br_slot(sg, k, isr);
    const uint32_t p = atomicAdd(&v.cnt[slot], 1u);
    if (p < uint32_t(CAP)) {
      v.tkey[p] = k;
      v.tidx[p] = uint16_t(x);
      v.tslot[p] = uint16_t(slot);
    }
  }
  __syncthreads();
  bool heavy = false;
  uint32_t bw[ITEMS];  // per position: (bucket start << 16 | length) of a heavy bucket, else 0
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int p = t + j * BLOCK;
    bw[j] = 0;
    if (p >= n) continue;
    const uint32_t slot = v.tslot[p], k = v.tkey[p];
    const uint32_t x = v.tidx[p];
    if (x >= uint32_t(E)) continue;  // only after a reported error
    const uint32_t s = v.seg[x] >> 16;
    const uint32_t end = v.cnt[slot];
    const uint32_t start = slot == s ? s : v.cnt[slot - 1];
    if (end - start > uint32_t(T_RANK)) {
      heavy = true;
      bw[j] = (start << 16) | (end - start);
      continue;
    }
    uint32_t rank = 0;
    for (uint32_t q = start; q < end; ++q) rank += v.tkey[q] < k;
    out(start + rank, x, k);
  }
  if (__syncthreads_or(heavy)) {
    SortView r = heavy_view<CAP>(v);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int p = t + j * BLOCK;
      if (p < n) v.seg[p] = bw[j];
    }
    __syncthreads();
    refine_sort<BLOCK, ITEMS>(r, n, key_bits, tmp32, st, false);
    for (int p = t; p < n; p += BLOCK) {
      const int fp = final_pos(r, p);
      if (fp >= 0) out(uint32_t(fp), v.tidx[p], v.tkey[p]);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------
// Tile kernel: rows with short sources, many rows per CTA.
// ------------------------------------------------------------------------------
template <class Ld>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  return size_t(TILE_CAP) * sizeof(typename Ld::VT) + br_smem_bytes<TILE_CAP>() +
         size_t(TILE_CAP) * 4 + 16 + size_t(TILE_BLOCK) * (8 + 8 + 4 * 6);
}

template <class CI, class VT>
struct TileOut {
  CI* out_col;
  VT* out_val;
  const VT* sval;
  const uint16_t* srow;  // row (within the tile) of each packed entry
  const uint32_t* rdel;  // per row: output offset - packed offset
  long long base;
  __device__ __forceinline__ void operator()(uint32_t f, uint32_t x, uint32_t k) const {
    const long long g = base + f + rdel[srow[x]];
    st_stream(out_col + g, CI(k));
    st_stream(out_val + g, sval[x]);
  }
};

// Tile layout: the rows of a tile that the tile handles are packed back to back in
// shared memory (rows whose source is long are skipped and may sit anywhere in the
// tile's output range); srow[x] is the row of packed entry x and rdel[row] = output
// offset - packed offset of that row.  A tile holds at most TILE_BLOCK rows (the
// partition gives every row a weight of TILE_ROW_W in a window of TILE_CP).
constexpr int TILE_PER_SM = 3;

template <class Ld>
__global__ void __launch_bounds__(TILE_BLOCK, TILE_PER_SM)
    k_tile(Ld ld, const long long* __restrict__ vp, const long long* __restrict__ tile_first,
           const long long* __restrict__ ntiles_p, typename Ld::CI* __restrict__ out_col,
           typename Ld::VT* __restrict__ out_val, int key_bits, DevStatus* st) {
  using VT = typename Ld::VT;
  using CI = typename Ld::CI;
  constexpr int BLOCK = TILE_BLOCK, CAP = TILE_CAP, ITEMS = CAP / BLOCK;
  static_assert(TILE_CP / TILE_ROW_W <= BLOCK, "a tile's rows must fit one pass");
  extern __shared__ __align__(16) unsigned char smem[];
  VT* sval = reinterpret_cast<VT*>(smem);
  BRView b = carve_br<CAP>(smem + size_t(CAP) * sizeof(VT));
  uint16_t* srow = reinterpret_cast<uint16_t*>(smem + size_t(CAP) * sizeof(VT) + br_smem_bytes<CAP>());
  uint16_t* owner = srow + CAP;  // row of each source position
  unsigned char* p = smem + ((size_t(CAP) * sizeof(VT) + br_smem_bytes<CAP>() + size_t(CAP) * 4 + 15) &
                             ~size_t(15));
  long long* r_s0 = reinterpret_cast<long long*>(p);
  long long* r_s1 = r_s0 + BLOCK;
  uint32_t* r_n0 = reinterpret_cast<uint32_t*>(r_s1 + BLOCK);
  uint32_t* r_ls = r_n0 + BLOCK;   // packed start
  uint32_t* r_del = r_ls + BLOCK;  // output offset (from the tile base) - packed start
  uint32_t* r_lo = r_del + BLOCK;  // output length
  uint32_t* r_sp = r_lo + BLOCK;   // source prefix within the tile
  uint32_t* r_cur = r_sp + BLOCK;  // kept cursor
  __shared__ unsigned long long tmp64[BLOCK / 32 + 1];
  __shared__ uint32_t tmp32[BLOCK / 32 + 1];
  const int t = threadIdx.x;
  const float isr = br_isr(key_bits);
  const long long ntiles = *ntiles_p;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r0 = tile_first[tile], r1 = tile_first[tile + 1];
    if (r1 - r0 > BLOCK) {  // cannot happen: see the partition
      if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -13);
      continue;
    }
    const long long base = vp[r0];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      b.seg[t + j * BLOCK] = 0;
      b.cnt[t + j * BLOCK] = 0;
    }
    const long long r = r0 + t;
    uint32_t Ls = 0, Lk = 0;
    long long o0 = 0;
    RowSrc rs{0, 0, 0, 0};
    if (r < r1) {
      o0 = vp[r];
      const long long Lo = vp[r + 1] - o0;
      if (Lo > 0) {
        rs = ld.row(r);
        const long long ls = rs.n0 + rs.n1;
        if (ls <= TILE_CP) {  // longer sources are handled by k_long / k_huge
          if (Lo > TILE_CP || o0 - base + Lo > 0xFFFFFFFFll) {
            dev_fail(st, SP_ERR_INTERNAL, r);
          } else {
            Ls = uint32_t(ls);
            Lk = uint32_t(Lo);
          }
        }
      }
    }
    // packed starts (low half) and source prefixes (high half) in one block scan
    unsigned long long tot;
    const unsigned long long pre =
        block_excl_sum<BLOCK>((unsigned long long)Lk | ((unsigned long long)Ls << 32), tmp64, &tot);
    const uint32_t ls_packed = uint32_t(pre & 0xFFFFFFFFull);
    const uint32_t sp = uint32_t(pre >> 32);
    uint32_t S = uint32_t(tot >> 32);
    int E = int(tot & 0xFFFFFFFFull);
    if (E > CAP) {  // cannot happen: see the partition
      if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -12);
      Ls = 0;
      S = 0;
      E = 0;
    }
    if (Ls > 0) {
      r_s0[t] = rs.s0;
      r_s1[t] = rs.s1;
      r_n0[t] = uint32_t(rs.n0);
      r_ls[t] = ls_packed;
      r_del[t] = uint32_t(o0 - base) - ls_packed;
      r_lo[t] = Lk;
      r_cur[t] = 0;
    }
    r_sp[t] = sp;
    __syncthreads();
    for (uint32_t w0 = 0; w0 < S; w0 += CAP) {
      const uint32_t W = S - w0 < uint32_t(CAP) ? S - w0 : uint32_t(CAP);
      for (uint32_t x = t; x < W; x += BLOCK) owner[x] = 0;
      __syncthreads();
      if (Ls > 0) {
        if (sp >= w0 && sp < w0 + W) owner[sp - w0] = uint16_t(t);
        else if (sp < w0 && sp + Ls > w0) owner[0] = uint16_t(t);
      }
      __syncthreads();
      smem_incl_max16<BLOCK, ITEMS>(owner, int(W), tmp32);
      for (uint32_t x0 = t; x0 < W; x0 += BLOCK * LOAD_U) {
        Batch<Ld, LOAD_U> bt;
        uint32_t kr[LOAD_U], off[LOAD_U];
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          const uint32_t x = x0 + u * BLOCK;
          bt.valid[u] = x < W;
          kr[u] = 0;
          off[u] = 0;
          if (bt.valid[u]) {
            kr[u] = owner[x];
            off[u] = w0 + x - r_sp[kr[u]];
            const uint32_t n0 = r_n0[kr[u]];
            bt.part[u] = off[u] < n0 ? 0 : 1;
            bt.pos[u] = bt.part[u] ? r_s1[kr[u]] + (off[u] - n0) : r_s0[kr[u]] + off[u];
          }
        }
        bt.run(ld);
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          if (!bt.kept[u]) continue;
          const uint32_t c = Ld::kAllKept ? off[u] : atomicAdd(&r_cur[kr[u]], 1u);
          if (c < r_lo[kr[u]]) {
            const uint32_t lp = r_ls[kr[u]] + c;
            const uint32_t sg = (r_ls[kr[u]] << 16) | r_lo[kr[u]];
            b.key[lp] = bt.key[u];
            sval[lp] = bt.v[u];
            b.seg[lp] = sg;
            srow[lp] = uint16_t(kr[u]);
            atomicAdd(&b.cnt[br_slot(sg, bt.key[u], isr)], 1u);  // histogram
          } else {
            dev_fail(st, SP_ERR_INTERNAL, -3);
          }
        }
      }
      __syncthreads();
    }
    br_finish<BLOCK, CAP>(b, E, key_bits, tmp32, st, TileOut<CI, VT>{out_col, out_val, sval, srow, r_del, base});
  }
}

// ------------------------------------------------------------------------------
// Long-row kernel: one CTA per row (source mode) or per buffered run (buffer mode).
// Values are not staged: each output value is read from its source when written.
// ------------------------------------------------------------------------------
template <class VT>
__host__ __device__ constexpr size_t long_smem_bytes() {
  return br_smem_bytes<LONG_CAP>() + size_t(LONG_CAP) * 4;
}

template <class Ld>
__global__ void __launch_bounds__(LONG_BLOCK, 2)
    k_long(Ld ld, const long long* __restrict__ vp, const long long* __restrict__ rows,
           const unsigned* __restrict__ nrows_p, const FinalEntry* __restrict__ runs,
           const unsigned* __restrict__ nruns_p, long long list_cap, unsigned* ticket,
           const uint32_t* __restrict__ tkey, const typename Ld::VT* __restrict__ tval,
           typename Ld::CI* __restrict__ out_col, typename Ld::VT* __restrict__ out_val,
           int key_bits, DevStatus* st) {
  using VT = typename Ld::VT;
  using CI = typename Ld::CI;
  constexpr int BLOCK = LONG_BLOCK, CAP = LONG_CAP, ITEMS = CAP / BLOCK;
  extern __shared__ __align__(16) unsigned char smem[];
  BRView b = carve_br<CAP>(smem);
  uint32_t* eoff = reinterpret_cast<uint32_t*>(smem + br_smem_bytes<CAP>());  // source entry
  __shared__ uint32_t tmp32[BLOCK / 32 + 1];
  __shared__ unsigned s_item;
  __shared__ uint32_t s_cur;
  const int t = threadIdx.x;
  const float isr = br_isr(key_bits);
  const bool src_mode = rows != nullptr;
  unsigned count = src_mode ? *nrows_p : *nruns_p;
  if (count > list_cap) count = unsigned(list_cap);  // overflow was reported by the producer
  for (;;) {
    if (t == 0) {
      s_item = atomicAdd(ticket, 1u);
      s_cur = 0;
    }
    __syncthreads();
    const unsigned item = s_item;
    if (item >= count) break;
    long long g0;
    int E;
    RowSrc rs{0, 0, 0, 0};
    int buf = -1;
    if (src_mode) {
      const long long r = rows[item];
      g0 = vp[r];
      const long long Lo = vp[r + 1] - g0;
      if (Lo > CAP || Lo < 0) {
        if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -8);
        __syncthreads();
        continue;
      }
      E = int(Lo);
      for (int x = t; x < E; x += BLOCK) {
        b.key[x] = 0;
        eoff[x] = 0;
        b.cnt[x] = 0;
      }
      __syncthreads();
      rs = ld.row(r);
      const long long Ls = rs.n0 + rs.n1;
      for (long long e0 = 0; e0 < Ls; e0 += (long long)BLOCK * LOAD_U) {
        Batch<KeyOnly<Ld>, LOAD_U> bt;
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          const long long e = e0 + (long long)u * BLOCK + t;
          bt.valid[u] = e < Ls;
          if (bt.valid[u]) bt.at(u, rs, e);
        }
        bt.run(KeyOnly<Ld>{ld});
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          if (!bt.kept[u]) continue;
          const long long e = e0 + (long long)u * BLOCK + t;
          const uint32_t c = Ld::kAllKept ? uint32_t(e) : atomicAdd(&s_cur, 1u);
          if (c < uint32_t(E)) {
            b.key[c] = bt.key[u];
            eoff[c] = uint32_t(e);
            atomicAdd(&b.cnt[br_slot(uint32_t(E), bt.key[u], isr)], 1u);  // histogram
          } else {
            dev_fail(st, SP_ERR_INTERNAL, -4);
          }
        }
      }
    } else {
      const FinalEntry fe = runs[item];
      g0 = fe.off;
      if (fe.len > CAP || fe.len < 0) {
        if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -9);
        __syncthreads();
        continue;
      }
      E = int(fe.len);
      buf = fe.buf;
      for (int x = t; x < E; x += BLOCK) b.cnt[x] = 0;
      __syncthreads();
      for (int x = t; x < E; x += BLOCK) {
        const uint32_t k = buf == BUF_TEMP ? ld_stream(tkey + g0 + x) : uint32_t(out_col[g0 + x]);
        b.key[x] = k;
        eoff[x] = uint32_t(x);
        atomicAdd(&b.cnt[br_slot(uint32_t(E), k, isr)], 1u);  // histogram
      }
    }
    for (int x = t; x < E; x += BLOCK) b.seg[x] = uint32_t(E);  // one segment at 0
    __syncthreads();
    const int n = bucket_rank_sort<BLOCK, CAP>(b, E, key_bits, tmp32, st, true);
    // read every value before writing any (a run may be sorted in place)
    VT vv[ITEMS];
    uint32_t kk[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int f = t + j * BLOCK;
      if (f < n) {
        uint32_t x = b.ord[f];
        if (x >= uint32_t(E)) x = 0;  // only after a reported error
        kk[j] = b.key[x];
        const long long e = eoff[x];
        if (src_mode) {
          const int part = e < rs.n0 ? 0 : 1;
          const long long pos = part ? rs.s1 + (e - rs.n0) : rs.s0 + e;
          vv[j] = ld_stream(ld.vals(part) + pos);
        } else {
          vv[j] = buf == BUF_TEMP ? ld_stream(tval + g0 + e) : out_val[g0 + e];
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int f = t + j * BLOCK;
      if (f < n) {
        st_stream(out_col + g0 + f, CI(kk[j]));
        st_stream(out_val + g0 + f, vv[j]);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------
// Huge-row kernel: partition one long run by key range into HUGE_NB buckets.
// ------------------------------------------------------------------------------
constexpr size_t huge_smem_bytes() { return size_t(HUGE_NB) * 4 * 2; }

template <class Ld>
__global__ void __launch_bounds__(HUGE_BLOCK, 1)
    k_huge(Ld ld, const long long* __restrict__ vp, const long long* __restrict__ rows,
           const unsigned* __restrict__ nrows_p, const HugeEntry* __restrict__ runs,
           const unsigned* __restrict__ nruns_p, long long list_cap, unsigned* ticket, int key_bits,
           uint32_t* __restrict__ tkey, typename Ld::VT* __restrict__ tval,
           typename Ld::CI* __restrict__ out_col, typename Ld::VT* __restrict__ out_val,
           FinalEntry* __restrict__ fin, unsigned* fin_n, long long fin_cap,
           HugeEntry* __restrict__ nxt, unsigned* nxt_n, long long nxt_cap, DevStatus* st) {
  using VT = typename Ld::VT;
  using CI = typename Ld::CI;
  constexpr int BLOCK = HUGE_BLOCK, ITEMS = HUGE_NB / BLOCK;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem);
  uint32_t* aux = hist + HUGE_NB;
  __shared__ uint32_t tmp32[BLOCK / 32 + 1];
  __shared__ unsigned s_item;
  const int t = threadIdx.x;
  const bool src_mode = rows != nullptr;
  unsigned count = src_mode ? *nrows_p : *nruns_p;
  if (count > list_cap) count = unsigned(list_cap);
  for (;;) {
    if (t == 0) s_item = atomicAdd(ticket, 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= count) break;
    long long g0, L;
    unsigned lo;
    int wb, sbuf;
    RowSrc rs{0, 0, 0, 0};
    if (src_mode) {
      const long long r = rows[item];
      g0 = vp[r];
      L = vp[r + 1] - g0;
      lo = 0;
      wb = key_bits;
      sbuf = -1;
      rs = ld.row(r);
    } else {
      const HugeEntry he = runs[item];
      g0 = he.off;
      L = he.len;
      lo = he.lo;
      wb = he.wb;
      sbuf = he.buf;
    }
    const int dbuf = src_mode ? BUF_TEMP : (sbuf == BUF_TEMP ? BUF_OUT : BUF_TEMP);
    const int nbl = wb < HUGE_NB_LOG ? wb : HUGE_NB_LOG;
    const int nb = 1 << nbl;
    const int sh = wb - nbl;
    for (int x = t; x < HUGE_NB; x += BLOCK) hist[x] = 0;
    __syncthreads();
    // pass 1: histogram of bucket sizes
    if (src_mode) {
      const long long Ls = rs.n0 + rs.n1;
      for (long long e0 = 0; e0 < Ls; e0 += (long long)BLOCK * LOAD_U) {
        Batch<KeyOnly<Ld>, LOAD_U> bt;
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          const long long e = e0 + (long long)u * BLOCK + t;
          bt.valid[u] = e < Ls;
          if (bt.valid[u]) bt.at(u, rs, e);
        }
        bt.run(KeyOnly<Ld>{ld});
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          if (!bt.kept[u]) continue;
          const uint32_t key = bt.key[u];
          const uint32_t bk = (key - lo) >> sh;
          if (key >= lo && bk < uint32_t(nb)) atomicAdd(&hist[bk], 1u);
          else dev_fail(st, SP_ERR_INDEX_RANGE, -20);
        }
      }
    } else {
      for (long long e = t; e < L; e += BLOCK) {
        const uint32_t key = sbuf == BUF_TEMP ? tkey[g0 + e] : uint32_t(out_col[g0 + e]);
        const uint32_t bk = (key - lo) >> sh;
        if (key >= lo && bk < uint32_t(nb)) atomicAdd(&hist[bk], 1u);
        else dev_fail(st, SP_ERR_INDEX_RANGE, g0 + e);
      }
    }
    __syncthreads();
    const uint32_t total = smem_excl_sum<BLOCK, ITEMS>(hist, HUGE_NB, tmp32);
    if (total != uint32_t(L)) {
      if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -5);
      continue;
    }
    // previous non-empty bucket (inclusive max-scan of b+1 over non-empty buckets)
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t * ITEMS + j;
      const uint32_t c = (x + 1 < nb ? hist[x + 1] : uint32_t(L)) - hist[x];
      aux[x] = (x < nb && c > 0) ? uint32_t(x + 1) : 0u;
    }
    __syncthreads();
    smem_incl_max<BLOCK, ITEMS>(aux, HUGE_NB, tmp32);
    // heads of groups: small non-empty buckets that start a new group of consecutive
    // small buckets (group = buckets whose start lies in one GROUP_CAP window, cut at
    // every big bucket); big buckets stand alone.
    bool head[ITEMS], big[ITEMS];
    uint32_t cc[ITEMS], sb[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t * ITEMS + j;
      sb[j] = hist[x];
      cc[j] = x < nb ? (x + 1 < nb ? hist[x + 1] : uint32_t(L)) - sb[j] : 0u;
      big[j] = cc[j] > uint32_t(GROUP_CAP);
      head[j] = false;
      if (cc[j] > 0 && !big[j]) {
        const uint32_t pv = x > 0 ? aux[x - 1] : 0u;  // previous non-empty bucket + 1
        if (pv == 0) {
          head[j] = true;
        } else {
          const int y = int(pv) - 1;
          const uint32_t cy = (y + 1 < nb ? hist[y + 1] : uint32_t(L)) - hist[y];
          head[j] = cy > uint32_t(GROUP_CAP) || (hist[y] / GROUP_CAP) != (sb[j] / GROUP_CAP);
        }
      }
    }
    __syncthreads();
    // next boundary start after each bucket: suffix min over boundary starts, computed
    // as a prefix max over the reversed array of (L - start)
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t * ITEMS + j;
      const bool bnd = head[j] || big[j];
      aux[HUGE_NB - 1 - x] = bnd ? uint32_t(L) - sb[j] : 0u;
    }
    __syncthreads();
    smem_incl_max<BLOCK, ITEMS>(aux, HUGE_NB, tmp32);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t * ITEMS + j;
      if (x >= nb || cc[j] == 0) continue;
      if (big[j]) {
        if (cc[j] <= uint32_t(LONG_CAP)) {
          const unsigned q = atomicAdd(fin_n, 1u);
          if (q < fin_cap) fin[q] = FinalEntry{g0 + sb[j], cc[j], dbuf, 0};
          else dev_fail(st, SP_ERR_INTERNAL, -6);
        } else {
          const unsigned q = atomicAdd(nxt_n, 1u);
          if (q < nxt_cap) nxt[q] = HugeEntry{g0 + sb[j], cc[j], lo + (uint32_t(x) << sh), sh, dbuf, 0};
          else dev_fail(st, SP_ERR_INTERNAL, -7);
        }
      } else if (head[j]) {
        // reversed index of x+1 holds max over buckets >= x+1 of (L - start) -> min start
        const uint32_t nx = (x + 1 < HUGE_NB) ? aux[HUGE_NB - 1 - (x + 1)] : 0u;
        const uint32_t end = nx ? uint32_t(L) - nx : uint32_t(L);
        const unsigned q = atomicAdd(fin_n, 1u);
        if (q < fin_cap) fin[q] = FinalEntry{g0 + sb[j], (long long)(end - sb[j]), dbuf, 0};
        else dev_fail(st, SP_ERR_INTERNAL, -6);
      }
    }
    __syncthreads();
    // pass 2: scatter by bucket (hist now serves as the bucket cursors)
    if (src_mode) {
      const long long Ls = rs.n0 + rs.n1;
      for (long long e0 = 0; e0 < Ls; e0 += (long long)BLOCK * LOAD_U) {
        Batch<Ld, LOAD_U> bt;
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          const long long e = e0 + (long long)u * BLOCK + t;
          bt.valid[u] = e < Ls;
          if (bt.valid[u]) bt.at(u, rs, e);
        }
        bt.run(ld);
#pragma unroll
        for (int u = 0; u < LOAD_U; ++u) {
          if (!bt.kept[u]) continue;
          const uint32_t key = bt.key[u];
          const uint32_t bk = (key - lo) >> sh;
          if (key < lo || bk >= uint32_t(nb)) continue;
          const uint32_t q = atomicAdd(&hist[bk], 1u);
          if (q < uint32_t(L)) {
            tkey[g0 + q] = key;
            tval[g0 + q] = bt.v[u];
          }
        }
      }
    } else {
      for (long long e = t; e < L; e += BLOCK) {
        uint32_t key;
        VT v;
        if (sbuf == BUF_TEMP) {
          key = tkey[g0 + e];
          v = tval[g0 + e];
        } else {
          key = uint32_t(out_col[g0 + e]);
          v = out_val[g0 + e];
        }
        const uint32_t bk = (key - lo) >> sh;
        if (key < lo || bk >= uint32_t(nb)) continue;
        const uint32_t q = atomicAdd(&hist[bk], 1u);
        if (q >= uint32_t(L)) continue;
        if (dbuf == BUF_TEMP) {
          tkey[g0 + q] = key;
          tval[g0 + q] = v;
        } else {
          out_col[g0 + q] = CI(key);
          out_val[g0 + q] = v;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace sp
