// Gather -> remap -> per-row sort -> store, the Identify / Build pipeline of the paper
// (Algorithm 2's fill pass and the Build step's sort, Sec. 3.1) restated for one GPU.
//
// Output rows are laid out contiguously by a row-pointer array `vp` (int64, one entry
// per listed row plus one).  Each output row is filled from one or two source runs
// described by a Loader:
//   struct Loader {
//     using CI = ...;  using VT = ...;           // column index / value word types
//     RowSrc row(int64 r) const;                 // source runs of listed row r
//     bool elem(int part, int64 pos, uint32& key, VT& val) const;
//         // reads source element `pos` of run `part`; returns false if it is dropped,
//         // otherwise its new column (`key`) and its value bits
//   };
// Rows are routed by length:
//   * rows whose source is at most CP = TILE_CAP/2 entries go through k_tile: one CTA
//     gathers all rows of a tile of output positions into shared memory, sorts every
//     row there and writes the tile back with the positions of a canonical CSR;
//   * rows with longer sources but at most LONG_CAP output entries: k_long, one CTA per
//     row with a larger shared-memory capacity;
//   * rows with more than LONG_CAP output entries: k_huge partitions the row by key
//     range into 2^14 buckets (two streaming passes, through a global buffer) and hands
//     groups of consecutive buckets of at most LONG_CAP entries to k_long.
// The shared-memory sort ("bucket refine") splits each segment into ~len/2 buckets by
// the high bits of its key range, scatters, and repeats on buckets larger than
// T_SMALL; buckets of at most T_SMALL keys are finished by ranking (keys are unique
// within a row, so every sort gives the same canonical order).
#pragma once

#include "common.cuh"

namespace sp {

struct RowSrc {
  long long s0, s1;  // start of run 0 / run 1 in the source arrays
  long long n0, n1;  // lengths (n1 = 0 for single-run sources)
};

constexpr int T_SMALL = 16;
constexpr int TILE_BLOCK = 512;
constexpr int TILE_CAP = 4096;
constexpr int TILE_CP = TILE_CAP / 2;  // longest source row a tile accepts
constexpr int LONG_BLOCK = 1024;
constexpr int LONG_CAP = 8192;
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
template <int BLOCK, int ITEMS>
__device__ void refine_sort(const SortView& b, int E, uint32_t* tmp32, DevStatus* st) {
  const int t = threadIdx.x;
  for (int round = 0;; ++round) {
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
      }
      any |= (sg[j] & 0xFFFFu) > uint32_t(T_SMALL);
    }
    if (!__syncthreads_or(any)) break;
    if (round >= 12) {  // impossible for 32-bit keys (each round removes >= 4 bits)
      if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -2);
      break;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t + j * BLOCK;
      if (x < E) {
        b.cnt[x] = 0;
        const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
        if (len > uint32_t(T_SMALL) && uint32_t(x) == s) {
          b.lo[s >> 4] = 0xFFFFFFFFu;
          b.hi[s >> 4] = 0u;
        }
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
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
      if (len > uint32_t(T_SMALL)) {
        const int nbl = ceil_log2_u32(len) - 1;  // nb = 2^nbl < len buckets
        const uint32_t L = b.lo[s >> 4], H = b.hi[s >> 4];
        const uint32_t range = H - L;
        const int bits = range ? 32 - __clz(range) : 0;
        const int sh = bits > nbl ? bits - nbl : 0;
        const uint32_t slot = s + ((k[j] - L) >> sh);
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
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t len = sg[j] & 0xFFFFu, s = sg[j] >> 16;
      if (len > uint32_t(T_SMALL)) {
        const uint32_t slot = si[j] >> 16;
        const uint32_t bse = b.base[s >> 4];
        const uint32_t e = s + b.cnt[slot] - bse;
        const uint32_t a = slot == s ? s : s + b.cnt[slot - 1] - bse;
        b.seg[ps[j]] = (a << 16) | (e - a);
      }
    }
    __syncthreads();
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
// Tile kernel: rows with short sources, many rows per CTA.
// ------------------------------------------------------------------------------
template <class Ld>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  return sort_smem_bytes<typename Ld::VT, TILE_CAP>() + 16 +
         size_t(TILE_BLOCK) * (8 + 8 + 4 * 5);
}

template <class Ld>
__global__ void __launch_bounds__(TILE_BLOCK, 2)
    k_tile(Ld ld, const long long* __restrict__ vp, const long long* __restrict__ tile_first,
           long long ntiles, typename Ld::CI* __restrict__ out_col,
           typename Ld::VT* __restrict__ out_val, DevStatus* st) {
  using VT = typename Ld::VT;
  using CI = typename Ld::CI;
  constexpr int BLOCK = TILE_BLOCK, CAP = TILE_CAP, ITEMS = CAP / BLOCK;
  extern __shared__ __align__(16) unsigned char smem[];
  VT* sval;
  SortView b = carve_sort<VT, CAP>(smem, &sval);
  unsigned char* p = smem + ((sort_smem_bytes<VT, CAP>() + 15) & ~size_t(15));
  long long* r_s0 = reinterpret_cast<long long*>(p);
  long long* r_s1 = r_s0 + BLOCK;
  uint32_t* r_n0 = reinterpret_cast<uint32_t*>(r_s1 + BLOCK);
  uint32_t* r_ls = r_n0 + BLOCK;
  uint32_t* r_lo = r_ls + BLOCK;
  uint32_t* r_sp = r_lo + BLOCK;
  uint32_t* r_cur = r_sp + BLOCK;
  __shared__ uint32_t tmp32[BLOCK / 32 + 1];
  __shared__ uint32_t sE;
  const int t = threadIdx.x;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r0 = tile_first[tile], r1 = tile_first[tile + 1];
    const long long base = vp[r0];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      b.seg[t + j * BLOCK] = 0;
      b.idx[t + j * BLOCK] = 0;
    }
    if (t == 0) sE = 0;
    __syncthreads();
    for (long long rc = r0; rc < r1; rc += BLOCK) {
      const long long r = rc + t;
      uint32_t Ls = 0;
      if (r < r1) {
        const long long o0 = vp[r];
        const long long Lo = vp[r + 1] - o0;
        if (Lo > 0) {
          const RowSrc rs = ld.row(r);
          const long long ls = rs.n0 + rs.n1;
          if (ls <= TILE_CP) {  // longer sources are handled by k_long / k_huge
            if (o0 - base + Lo > CAP || Lo > TILE_CP) {
              dev_fail(st, SP_ERR_INTERNAL, r);
            } else {
              Ls = uint32_t(ls);
              r_s0[t] = rs.s0;
              r_s1[t] = rs.s1;
              r_n0[t] = uint32_t(rs.n0);
              r_ls[t] = uint32_t(o0 - base);
              r_lo[t] = uint32_t(Lo);
              r_cur[t] = 0;
              atomicMax(&sE, uint32_t(o0 - base + Lo));
            }
          }
        }
      }
      uint32_t S;
      const uint32_t sp = block_excl_sum<BLOCK>(Ls, tmp32, &S);
      r_sp[t] = sp;
      __syncthreads();
      for (uint32_t w0 = 0; w0 < S; w0 += CAP) {
        const uint32_t W = S - w0 < uint32_t(CAP) ? S - w0 : uint32_t(CAP);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
          const uint32_t x = t + j * BLOCK;
          if (x < W) b.cnt[x] = 0;
        }
        __syncthreads();
        if (Ls > 0) {
          if (sp >= w0 && sp < w0 + W) b.cnt[sp - w0] = t;
          else if (sp < w0 && sp + Ls > w0) b.cnt[0] = t;
        }
        __syncthreads();
        smem_incl_max<BLOCK, ITEMS>(b.cnt, int(W), tmp32);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
          const uint32_t x = t + j * BLOCK;
          if (x < W) {
            const uint32_t kr = b.cnt[x];
            const uint32_t off = w0 + x - r_sp[kr];
            const uint32_t n0 = r_n0[kr];
            const int part = off < n0 ? 0 : 1;
            const long long pos = part ? r_s1[kr] + (off - n0) : r_s0[kr] + off;
            uint32_t key;
            VT v;
            if (ld.elem(part, pos, key, v)) {
              const uint32_t c = atomicAdd(&r_cur[kr], 1u);
              if (c < r_lo[kr]) {
                const uint32_t lp = r_ls[kr] + c;
                b.key[lp] = key;
                sval[lp] = v;
                b.idx[lp] = uint16_t(lp);
                b.seg[lp] = (r_ls[kr] << 16) | r_lo[kr];
              } else {
                dev_fail(st, SP_ERR_INTERNAL, -3);
              }
            }
          }
        }
        __syncthreads();
      }
    }
    const int E = int(sE);
    refine_sort<BLOCK, ITEMS>(b, E, tmp32, st);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t + j * BLOCK;
      if (x < E) {
        const int fp = final_pos(b, x);
        if (fp >= 0) {
          const long long g = base + fp;
          out_col[g] = CI(b.key[x]);
          out_val[g] = sval[b.idx[x]];
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------
// Long-row kernel: one CTA per row (source mode) or per buffered run (buffer mode).
// ------------------------------------------------------------------------------
template <class VT>
__host__ __device__ constexpr size_t long_smem_bytes() {
  return sort_smem_bytes<VT, LONG_CAP>();
}

template <class Ld>
__global__ void __launch_bounds__(LONG_BLOCK, 1)
    k_long(Ld ld, const long long* __restrict__ vp, const long long* __restrict__ rows,
           const unsigned* __restrict__ nrows_p, const FinalEntry* __restrict__ runs,
           const unsigned* __restrict__ nruns_p, long long list_cap, unsigned* ticket,
           const uint32_t* __restrict__ tkey, const typename Ld::VT* __restrict__ tval,
           typename Ld::CI* __restrict__ out_col, typename Ld::VT* __restrict__ out_val,
           DevStatus* st) {
  using VT = typename Ld::VT;
  using CI = typename Ld::CI;
  constexpr int BLOCK = LONG_BLOCK, CAP = LONG_CAP, ITEMS = CAP / BLOCK;
  extern __shared__ __align__(16) unsigned char smem[];
  VT* sval;
  SortView b = carve_sort<VT, CAP>(smem, &sval);
  __shared__ uint32_t tmp32[BLOCK / 32 + 1];
  __shared__ unsigned s_item;
  __shared__ uint32_t s_cur;
  const int t = threadIdx.x;
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
        b.idx[x] = 0;
      }
      __syncthreads();
      const RowSrc rs = ld.row(r);
      const long long Ls = rs.n0 + rs.n1;
      for (long long e = t; e < Ls; e += BLOCK) {
        const int part = e < rs.n0 ? 0 : 1;
        const long long pos = part ? rs.s1 + (e - rs.n0) : rs.s0 + e;
        uint32_t key;
        VT v;
        if (ld.elem(part, pos, key, v)) {
          const uint32_t c = atomicAdd(&s_cur, 1u);
          if (c < uint32_t(E)) {
            b.key[c] = key;
            sval[c] = v;
            b.idx[c] = uint16_t(c);
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
      for (int x = t; x < E; x += BLOCK) {
        if (fe.buf == BUF_TEMP) {
          b.key[x] = ld_stream(tkey + g0 + x);
          sval[x] = ld_stream(tval + g0 + x);
        } else {
          b.key[x] = uint32_t(out_col[g0 + x]);
          sval[x] = out_val[g0 + x];
        }
        b.idx[x] = uint16_t(x);
      }
    }
    for (int x = t; x < E; x += BLOCK) b.seg[x] = uint32_t(E);  // one segment at 0
    __syncthreads();
    refine_sort<BLOCK, ITEMS>(b, E, tmp32, st);
    for (int x = t; x < E; x += BLOCK) {
      const int fp = final_pos(b, x);
      if (fp >= 0) {
        out_col[g0 + fp] = CI(b.key[x]);
        out_val[g0 + fp] = sval[b.idx[x]];
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
      for (long long e = t; e < Ls; e += BLOCK) {
        const int part = e < rs.n0 ? 0 : 1;
        const long long pos = part ? rs.s1 + (e - rs.n0) : rs.s0 + e;
        uint32_t key;
        VT v;
        if (ld.elem(part, pos, key, v)) {
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
        else dev_fail(st, SP_ERR_INTERNAL, -21);
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
      for (long long e = t; e < Ls; e += BLOCK) {
        const int part = e < rs.n0 ? 0 : 1;
        const long long pos = part ? rs.s1 + (e - rs.n0) : rs.s0 + e;
        uint32_t key;
        VT v;
        if (ld.elem(part, pos, key, v)) {
          const uint32_t bk = (key - lo) >> sh;
          if (key < lo || bk >= uint32_t(nb)) continue;
          const uint32_t q = atomicAdd(&hist[bk], 1u);
          if (q < uint32_t(L)) {
            tkey[g0 + q] = key;
            tval[g0 + q] = v;
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
