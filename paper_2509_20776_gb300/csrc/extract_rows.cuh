// Extraction by rows (Sec. 2.2; HipExtract, Algorithm 5's two passes over the selected
// rows), written for one GPU:
//
//   Identify.  The columns of J become either
//     * a rank map (JRank): one 64-bit word per 32 columns holding the membership bits
//       of J and the number of members in the words before it, plus jpos[r] = the
//       position in J of the r-th smallest member.  A column c is kept when its bit is
//       set; its new column is jpos[rank(c)].  The tables take n/4 + 4|J| bytes (16 MB +
//       128 MB for n = 2^26, |J| = 2^25) instead of the 4n of a dense inverse map, and
//       need no O(n) clearing beyond the n/4 bytes of words;
//     * or J sorted once with its positions (JSorted), searched by binary search per
//       stored entry: Algorithm 5's search, for small |J|.
//   Count (k_xcount).  A warp takes 32 selected rows ("a block"): lane l resolves row
//     i0 + l (I[i], range check, the row-pointer pair), so 32 index chains are in flight,
//     and records the row's source start and length for the fill.  A row of at most
//     XC_LANE entries is then counted by its own lane (all its columns loaded at once,
//     every lane's row in flight together); the warp takes the longer rows XC_ROWS at a
//     time (two columns per lane), tests each column against J's bitmap and counts the
//     members (ballot + popc).
//   Fill (k_xfill).  A warp again takes 32 rows.  A row of at most XF_LANE source
//     entries is filled by its own lane: its columns and values loaded at once, the kept
//     ones relabelled and sorted by a network in registers, written once.  For longer
//     rows the warp loads XF_ROWS rows at once, relabels the kept entries (rank word +
//     position), compacts them (ballot slots) into a per-warp shared buffer and ranks
//     each among its row's new columns, so a row of at most XFAST source entries is
//     written once, sorted, at its final place.  Longer rows are written in source order
//     and queued for the row sort.
//   Random lookups, not HBM bytes, bound both passes: one 4-byte lookup per SM cycle
//   while its table is L2-resident (~300 G/s on GB300), fewer for tables above ~100 MB.
#pragma once

#include <type_traits>

#include "kernels.cuh"
#include "rowsort.cuh"

namespace sp {

constexpr unsigned kFull = 0xffffffffu;
constexpr int XFAST = 64;     // rows of at most this many source entries: masks, warp sort
constexpr int XC_ROWS = 6;    // rows whose columns a counting warp loads together
template <class CI>
constexpr int xc_lane() { return sizeof(CI) == 4 ? 16 : 8; }  // rows a lane counts alone
constexpr int XF_ROWS = 2;    // rows whose kept entries a filling warp loads together
constexpr int XF_LANE = 8;    // rows of at most this many source entries: filled by their own lane

// Sorting network on XF_LANE (key, value) pairs held in registers: 19 comparators in 6
// layers (a test checks the table on all 256 0/1 inputs, which by the 0-1 principle
// proves it sorts every input).
template <class VT>
__device__ __forceinline__ void sort8(uint32_t (&k)[8], VT (&v)[8]) {
  constexpr int P[19][2] = {{0, 2}, {1, 3}, {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}, {0, 1}, {2, 3},
                            {4, 5}, {6, 7}, {2, 4}, {3, 5}, {1, 4}, {3, 6}, {1, 2}, {3, 4}, {5, 6}};
#pragma unroll
  for (int c = 0; c < 19; ++c) {
    const int a = P[c][0], b = P[c][1];
    const bool sw = k[b] < k[a];
    const uint32_t ka = k[a], kb = k[b];
    const VT va = v[a], vb = v[b];
    k[a] = sw ? kb : ka;
    k[b] = sw ? ka : kb;
    v[a] = sw ? vb : va;
    v[b] = sw ? va : vb;
  }
}
constexpr int XB = 256;       // threads per CTA of the count / fill
constexpr unsigned kDropped = 0xFFFFFFFFu;  // padding key: never below a key

// ---- identify ------------------------------------------------------------------------
// Membership only (the count): the bitmap of J.
struct JBits {
  const uint32_t* bits;
  long long n;
  __device__ __forceinline__ bool test(long long c) const {
    return c >= 0 && c < n && ((ld_map(bits + (c >> 5)) >> (c & 31)) & 1u);
  }
};

// Rank map: word w = bits of columns [32w, 32w + 32) (low half) | members before 32w (high).
template <class IX>
struct JRank {
  const unsigned long long* meta;
  const IX* jpos;
  long long n;
  __device__ __forceinline__ bool test(long long c) const {
    if (c < 0 || c >= n) return false;
    const unsigned long long w = (unsigned long long)ld_map(reinterpret_cast<const long long*>(meta) + (c >> 5));
    return (uint32_t(w) >> (c & 31)) & 1u;
  }
  __device__ __forceinline__ bool map(long long c, uint32_t& key) const {
    if (c < 0 || c >= n) return false;
    const unsigned long long w = (unsigned long long)ld_map(reinterpret_cast<const long long*>(meta) + (c >> 5));
    const uint32_t bits = uint32_t(w), b = 1u << (c & 31);
    if (!(bits & b)) return false;
    const uint32_t r = uint32_t(w >> 32) + __popc(bits & (b - 1u));
    key = uint32_t((long long)ld_plain(jpos + r));  // |J| words: larger than L2 at scale
    return true;
  }
};

// Sorted J: jk ascending (the values of J), jp[r] = position in J of jk[r].
struct JSorted {
  const uint32_t* jk;
  const uint32_t* jp;
  long long nJ;
  __device__ __forceinline__ long long find(long long c) const {
    if (c < 0 || c > 0xFFFFFFFFll) return -1;
    long long lo = 0, hi = nJ;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if ((long long)ld_map(jk + mid) < c) lo = mid + 1;
      else hi = mid;
    }
    return lo < nJ && (long long)ld_map(jk + lo) == c ? lo : -1;
  }
  __device__ __forceinline__ bool test(long long c) const { return find(c) >= 0; }
  __device__ __forceinline__ bool map(long long c, uint32_t& key) const {
    const long long r = find(c);
    if (r < 0) return false;
    key = ld_map(jp + r);
    return true;
  }
};

// Scan input / output of the rank words: popcount of each bitmap word, and the word
// written with its exclusive prefix.
struct LoadPopc {
  const uint32_t* bits;
  __device__ long long operator()(long long w) const { return __popc(bits[w]); }
};
struct StoreRank {
  const uint32_t* bits;
  unsigned long long* meta;
  long long nw;
  __device__ void operator()(long long w, long long v) const {
    if (w < nw) meta[w] = (unsigned long long)bits[w] | ((unsigned long long)v << 32);
  }
};

// jpos[rank(J[k])] = k
template <class IX>
__global__ void k_jrank_pos(const IX* __restrict__ J, long long nJ, long long n,
                            const unsigned long long* __restrict__ meta, IX* __restrict__ jpos) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nJ;
       k += (long long)gridDim.x * blockDim.x) {
    const long long c = (long long)J[k];
    if (c < 0 || c >= n) continue;  // reported by the bitmap pass
    const unsigned long long w = meta[c >> 5];
    const uint32_t b = 1u << (c & 31);
    jpos[uint32_t(w >> 32) + __popc(uint32_t(w) & (b - 1u))] = IX(k);
  }
}

// the sorted identify's input: J's values as 32-bit keys, positions as values
template <class IX>
__global__ void k_jsorted_init(const IX* __restrict__ J, long long nJ, uint32_t* __restrict__ jk,
                               uint32_t* __restrict__ jp) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nJ;
       k += (long long)gridDim.x * blockDim.x) {
    jk[k] = uint32_t((long long)J[k]);  // in range (checked by the bitmap pass)
    jp[k] = uint32_t(k);
  }
}

// ---- row sources ---------------------------------------------------------------------
// Where listed row i's entries are and how a stored column is tested / relabelled:
//   using CI, VT;  using H = ...;            per-row handle (the arrays of the row's matrix)
//   H handle(long long i) const;             the handle of listed row i (lane-per-row)
//   static H shfl(const H& h, int lane);     another lane's handle
//   const CI* cols(const H&); const VT* vals(const H&);
//   bool test(const H&, long long c);  bool map(const H&, long long c, uint32_t& key);
//   kLongCta: rows of more than SRC_LONG entries go to the CTA-per-row kernels
// One matrix and one identify for every row:
template <class CIt, class VTt, class Rel>
struct XOne {
  using CI = CIt;
  using VT = VTt;
  static constexpr bool kLongCta = true;
  struct H {};
  const CI* col;
  const VT* val;
  Rel rel;
  __device__ __forceinline__ H handle(long long) const { return H{}; }
  __device__ static __forceinline__ H shfl(const H& h, int) { return h; }
  __device__ __forceinline__ const CI* cols(const H&) const { return col; }
  __device__ __forceinline__ const VT* vals(const H&) const { return val; }
  __device__ __forceinline__ bool test(const H&, long long c) const { return rel.test(c); }
  __device__ __forceinline__ bool map(const H&, long long c, uint32_t& key) const { return rel.map(c, key); }
};

// Row resolvers of the count: listed row i -> (source start, length).
struct XSpan {
  long long s, L;
};
// From the index vector and the row pointer (range-checked; the pair is recorded):
template <class RP, class IX>
struct XResolveI {
  const RP* rowptr;
  const IX* I;
  long long m, nnz;
  long long* rs0;
  long long* rsn;
  DevStatus* st;
  __device__ __forceinline__ XSpan operator()(long long i) const {
    XSpan sp{0, 0};
    const long long r = (long long)I[i];
    if (r < 0 || r >= m) {
      dev_fail(st, SP_ERR_INDEX_RANGE, i);
    } else {
      const long long a = (long long)rowptr[r], b = (long long)rowptr[r + 1];
      if (a >= 0 && b >= a && b <= nnz) sp = XSpan{a, b - a};
    }
    rs0[i] = sp.s;
    rsn[i] = sp.L;
    return sp;
  }
};
// From a table recorded earlier:
struct XResolveRecorded {
  const long long* rs0;
  const long long* rsn;
  __device__ __forceinline__ XSpan operator()(long long i) const { return XSpan{rs0[i], rsn[i]}; }
};

// ---- count ---------------------------------------------------------------------------
// cnt[i] = kept entries of listed row i (with Src::kLongCta, rows of more than SRC_LONG
// source entries are listed for k_count_long instead); *n_slow += rows of more than XFAST
// source entries (the fill queues their sort).
template <class Src, class Res>
__global__ void __launch_bounds__(XB, 4) k_xcount(Src src, Res res, long long nI, long long* __restrict__ cnt,
                                                 long long* __restrict__ cl_rows, unsigned* n_cl, long long cl_cap,
                                                 unsigned* n_slow, DevStatus* st) {
  using CI = typename Src::CI;
  using H = typename Src::H;
  constexpr int R = XC_ROWS, XL = xc_lane<CI>();
  constexpr long long kLong = Src::kLongCta ? SRC_LONG : (1ll << 62);
  __shared__ unsigned char s_lane[XB / 32][32];  // the lanes of the warp's longer rows, in order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i0 = w0 * 32; i0 < nI; i0 += nw * 32) {
    const long long i = i0 + lane;
    long long s = 0, L = 0;
    H h{};
    if (i < nI) {
      const XSpan sp = res(i);
      s = sp.s;
      L = sp.L;
      h = src.handle(i);
    }
    const unsigned slow = __ballot_sync(kFull, L > XFAST);
    if (lane == 0 && slow) atomicAdd(n_slow, unsigned(__popc(slow)));
    if (L > kLong) push_row(cl_rows, n_cl, cl_cap, i, st);
    long long mine = 0;
    // short rows: the lane's own row, all its columns in flight at once
    if (L <= XL) {
      const CI* cp = src.cols(h);
      CI cc[XL];
#pragma unroll
      for (int e = 0; e < XL; ++e) cc[e] = e < L ? ld_stream(cp + s + e) : CI(0);
#pragma unroll
      for (int e = 0; e < XL; ++e) mine += (e < L && src.test(h, (long long)cc[e])) ? 1 : 0;
    }
    // longer rows (up to kLong): the warp, XC_ROWS rows at a time
    const unsigned lm = __ballot_sync(kFull, L > XL && L <= kLong);
    if ((lm >> lane) & 1u) s_lane[wid][__popc(lm & lt)] = (unsigned char)lane;
    __syncwarp();
    const int nr = __popc(lm);
    for (int g = 0; g < nr; g += R) {
      long long ss[R];
      int LL[R];  // the row's length, capped (the loop over a longer row re-reads it)
      int ln[R];  // its lane
      CI c0[R], c1[R];
#pragma unroll
      for (int u = 0; u < R; ++u) ln[u] = g + u < nr ? int(s_lane[wid][g + u]) : 0;
      // the handle of row u of the group (nothing for a single matrix; one shuffle for a batch)
      auto hof = [&](int u) { return Src::shfl(h, ln[u]); };
#pragma unroll
      for (int u = 0; u < R; ++u) {
        ss[u] = __shfl_sync(kFull, s, ln[u]);
        const long long l = __shfl_sync(kFull, L, ln[u]);
        if constexpr (Src::kLongCta) LL[u] = g + u < nr ? int(l) : 0;
        else LL[u] = g + u < nr ? int(l < (1 << 30) ? l : (1 << 30)) : 0;
      }
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const CI* cp = src.cols(hof(u));
        c0[u] = lane < LL[u] ? ld_stream(cp + ss[u] + lane) : CI(0);
        c1[u] = lane + 32 < LL[u] ? ld_stream(cp + ss[u] + 32 + lane) : CI(0);
      }
      bool k0[R], k1[R];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const H hu = hof(u);
        k0[u] = lane < LL[u] && src.test(hu, (long long)c0[u]);
        k1[u] = lane + 32 < LL[u] && src.test(hu, (long long)c1[u]);
      }
#pragma unroll
      for (int u = 0; u < R; ++u) {
        long long c = __popc(__ballot_sync(kFull, k0[u])) + __popc(__ballot_sync(kFull, k1[u]));
        // rows of more than XFAST entries: the rest in batches of LOAD_U x 32
        const H hu = hof(u);
        const CI* cp = src.cols(hu);
        // (single matrix: LL is the length itself; batched rows re-read a capped length)
        using LT = std::conditional_t<Src::kLongCta, int, long long>;
        LT Lu = LT(LL[u]);
        if constexpr (!Src::kLongCta) {
          if (LL[u] > 64) Lu = __shfl_sync(kFull, L, ln[u]);
        }
        for (LT e0 = 64; e0 < Lu; e0 += 32 * LOAD_U) {
          CI cc[LOAD_U];
#pragma unroll
          for (int v = 0; v < LOAD_U; ++v) {
            const LT e = e0 + v * 32 + lane;
            cc[v] = e < Lu ? ld_stream(cp + ss[u] + e) : CI(0);
          }
#pragma unroll
          for (int v = 0; v < LOAD_U; ++v) {
            const LT e = e0 + v * 32 + lane;
            c += __popc(__ballot_sync(kFull, e < Lu && src.test(hu, (long long)cc[v])));
          }
        }
        if (g + u < nr && lane == ln[u]) mine = c;
      }
    }
    __syncwarp();  // s_lane is rewritten by the next block of rows
    if (i < nI && L <= kLong) cnt[i] = mine;
  }
}

// ---- fill ----------------------------------------------------------------------------
template <class CI, class VT>
__device__ __forceinline__ void x_put(CI* out_col, VT* out_val, long long pos, long long end, uint32_t key,
                                      const VT& v, DevStatus* st) {
  if (pos < end) {
    st_stream(out_col + pos, CI(key));
    st_stream(out_val + pos, v);
  } else {
    dev_fail(st, SP_ERR_INTERNAL, -26);
  }
}

// Sort job of a row the warp path did not sort (k kept entries at output offset o).
__device__ __forceinline__ void x_queue(long long o, long long k, int key_bits, FinalEntry* fin, unsigned* fin_n,
                                        long long fin_cap, HugeEntry* huge, unsigned* huge_n, long long huge_cap,
                                        DevStatus* st) {
  if (k <= 1) return;
  if (k <= SS_RUN_MAX) {
    queue_run(fin, fin_n, fin_cap, FinalEntry{o, k, BUF_OUT, 0}, st, -27);
  } else {
    queue_huge(huge, huge_n, huge_cap, HugeEntry{o, k, 0u, key_bits, BUF_OUT, 0}, st, -28);
  }
}

// kSorted: the relabelling keeps the source order (ascending J), so slots are ranks and
// no row is queued.
template <class Src, bool kSorted>
__global__ void __launch_bounds__(XB, 4) k_xfill(Src src, long long nI, const long long* __restrict__ rs0,
                                                const long long* __restrict__ rsn, const long long* __restrict__ vp,
                                                typename Src::CI* __restrict__ out_col,
                                                typename Src::VT* __restrict__ out_val, FinalEntry* fin,
                                                unsigned* fin_n, long long fin_cap, HugeEntry* huge, unsigned* huge_n,
                                                long long huge_cap, int key_bits, int lane_rows, DevStatus* st) {
  // lane_rows: XF_LANE when every key is below kDropped (the lane path pads with it), else
  // 0; the lane path is compiled for 4-byte columns and values (its registers)
  using CI = typename Src::CI;
  using VT = typename Src::VT;
  using H = typename Src::H;
  constexpr bool kLane = sizeof(CI) == 4 && sizeof(VT) == 4;
  constexpr int R = XF_ROWS, NWB = XB / 32, KW = XFAST + 4;
  constexpr long long kLong = Src::kLongCta ? SRC_LONG : (1ll << 62);
  __shared__ __align__(16) uint32_t s_key[NWB][KW];  // a row's kept keys (+ padding for 4-wide loads)
  __shared__ VT s_val[NWB][XFAST];
  __shared__ unsigned char s_lane[NWB][32];  // the lanes of the warp's rows for the warp path, in order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t* wk = s_key[wid];
  VT* wv = s_val[wid];
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i0 = w0 * 32; i0 < nI; i0 += nw * 32) {
    const long long i = i0 + lane;
    long long s = 0, L = 0, o = 0, oe = 0;
    H h{};
    if (i < nI) {
      s = rs0[i];
      L = rsn[i];
      o = vp[i];
      oe = vp[i + 1];
      h = src.handle(i);
    }
    if (!kSorted && L > XFAST) x_queue(o, oe - o, key_bits, fin, fin_n, fin_cap, huge, huge_n, huge_cap, st);
    // rows of at most lane_rows entries: the lane's own row, all its loads and relabels in
    // flight together, the kept entries sorted in registers and written once
    const bool by_lane = L <= (kLane ? lane_rows : 0);
    if constexpr (kLane) if (by_lane && L > 0) {
      const CI* cp = src.cols(h);
      const VT* vq = src.vals(h);
      CI cc[XF_LANE];
      VT vv[XF_LANE];
      uint32_t kk[XF_LANE];
#pragma unroll
      for (int e = 0; e < XF_LANE; ++e) cc[e] = e < L ? ld_stream(cp + s + e) : CI(0);
#pragma unroll
      for (int e = 0; e < XF_LANE; ++e) vv[e] = e < L ? ld_stream(vq + s + e) : VT(0);
      int nk = 0;
#pragma unroll
      for (int e = 0; e < XF_LANE; ++e) {
        uint32_t key = kDropped;
        const bool p = e < L && src.map(h, (long long)cc[e], key);
        kk[e] = p ? key : kDropped;
        nk += p ? 1 : 0;
      }
      if (nk != oe - o) {  // the count disagrees with the fill (a library bug)
        dev_fail(st, SP_ERR_INTERNAL, -29);
      } else {
        sort8(kk, vv);
#pragma unroll
        for (int e = 0; e < XF_LANE; ++e)
          if (e < nk) x_put(out_col, out_val, o + e, oe, kk[e], vv[e], st);
      }
    }
    // rows of lane_rows < L <= XFAST entries: the warp, XF_ROWS rows at a time
    const unsigned lm = __ballot_sync(kFull, !by_lane && L <= XFAST);
    if ((lm >> lane) & 1u) s_lane[wid][__popc(lm & lt)] = (unsigned char)lane;
    __syncwarp();
    const int nr = __popc(lm);
    for (int g = 0; g < nr; g += R) {
      long long ss[R];
      int LL[R];
      int ln[R];
      H hh[R];
      CI c0[R], c1[R];
      VT v0[R], v1[R];
#pragma unroll
      for (int u = 0; u < R; ++u) ln[u] = g + u < nr ? int(s_lane[wid][g + u]) : 0;
#pragma unroll
      for (int u = 0; u < R; ++u) {
        ss[u] = __shfl_sync(kFull, s, ln[u]);
        const long long l = __shfl_sync(kFull, L, ln[u]);
        LL[u] = g + u < nr ? int(l) : 0;
        hh[u] = Src::shfl(h, ln[u]);
      }
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const CI* cp = src.cols(hh[u]);
        c0[u] = lane < LL[u] ? ld_stream(cp + ss[u] + lane) : CI(0);
        c1[u] = lane + 32 < LL[u] ? ld_stream(cp + ss[u] + 32 + lane) : CI(0);
      }
      // values of dropped entries are loaded too: they share sectors with kept ones
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const VT* vq = src.vals(hh[u]);
        if (lane < LL[u]) v0[u] = ld_stream(vq + ss[u] + lane);
        if (lane + 32 < LL[u]) v1[u] = ld_stream(vq + ss[u] + 32 + lane);
      }
      uint32_t k0[R], k1[R];
      bool p0[R], p1[R];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        p0[u] = lane < LL[u] && src.map(hh[u], (long long)c0[u], k0[u]);
        p1[u] = lane + 32 < LL[u] && src.map(hh[u], (long long)c1[u], k1[u]);
      }
#pragma unroll
      for (int u = 0; u < R; ++u) {
        if (LL[u] == 0) continue;  // warp-uniform: empty, long or beyond the block
        const long long ou = __shfl_sync(kFull, o, ln[u]);
        const long long eu = __shfl_sync(kFull, oe, ln[u]);
        const unsigned b0 = __ballot_sync(kFull, p0[u]), b1 = __ballot_sync(kFull, p1[u]);
        const int n0 = __popc(b0), nk = n0 + __popc(b1);
        if (nk != eu - ou) {  // the count disagrees with the fill (a library bug)
          if (lane == 0) dev_fail(st, SP_ERR_INTERNAL, -29);
          continue;
        }
        if (kSorted) {
          if (p0[u]) x_put(out_col, out_val, ou + __popc(b0 & lt), eu, k0[u], v0[u], st);
          if (p1[u]) x_put(out_col, out_val, ou + n0 + __popc(b1 & lt), eu, k1[u], v1[u], st);
          continue;
        }
        // compact the kept entries into the warp's buffer, then rank each among the row
        if (p0[u]) {
          wk[__popc(b0 & lt)] = k0[u];
          wv[__popc(b0 & lt)] = v0[u];
        }
        if (p1[u]) {
          wk[n0 + __popc(b1 & lt)] = k1[u];
          wv[n0 + __popc(b1 & lt)] = v1[u];
        }
        if (lane < 4) wk[nk + lane] = kDropped;  // padding: never below a key
        __syncwarp();
        const uint4* w4 = reinterpret_cast<const uint4*>(wk);
        const int nq = (nk + 3) >> 2;
        const uint32_t a = lane < nk ? wk[lane] : kDropped;
        int ra = 0;
        if (nk <= 32) {
          for (int q = 0; q < nq; ++q) {
            const uint4 x = w4[q];
            ra += int(x.x < a) + int(x.y < a) + int(x.z < a) + int(x.w < a);
          }
          VT va;
          if (lane < nk) va = wv[lane];
          __syncwarp();
          if (lane < nk) x_put(out_col, out_val, ou + ra, eu, a, va, st);
        } else {
          const uint32_t b = lane + 32 < nk ? wk[lane + 32] : kDropped;
          int rb = 0;
          for (int q = 0; q < nq; ++q) {
            const uint4 x = w4[q];
            ra += int(x.x < a) + int(x.y < a) + int(x.z < a) + int(x.w < a);
            rb += int(x.x < b) + int(x.y < b) + int(x.z < b) + int(x.w < b);
          }
          const VT va = wv[lane];
          VT vb;
          if (lane + 32 < nk) vb = wv[lane + 32];
          __syncwarp();
          x_put(out_col, out_val, ou + ra, eu, a, va, st);
          if (lane + 32 < nk) x_put(out_col, out_val, ou + rb, eu, b, vb, st);
        }
      }
    }
    __syncwarp();  // s_lane is rewritten by the next block of rows
    // rows of more than XFAST source entries (up to SRC_LONG with Src::kLongCta): kept
    // entries in source order (ballot slots); their sort was queued above
    unsigned mid = __ballot_sync(kFull, L > XFAST && L <= kLong);
    while (mid) {
      const int k = __ffs(mid) - 1;
      mid &= mid - 1;
      const long long sk = __shfl_sync(kFull, s, k), Lk = __shfl_sync(kFull, L, k);
      const H hk = Src::shfl(h, k);
      const CI* cp = src.cols(hk);
      const VT* vq = src.vals(hk);
      long long ok = __shfl_sync(kFull, o, k);
      const long long ek = __shfl_sync(kFull, oe, k);
      for (long long e0 = 0; e0 < Lk; e0 += 32 * LOAD_U) {
        CI cc[LOAD_U];
        VT vv[LOAD_U];
        uint32_t kk[LOAD_U];
        bool pp[LOAD_U];
#pragma unroll
        for (int v = 0; v < LOAD_U; ++v) {
          const long long e = e0 + v * 32 + lane;
          cc[v] = e < Lk ? ld_stream(cp + sk + e) : CI(0);
          if (e < Lk) vv[v] = ld_stream(vq + sk + e);
        }
#pragma unroll
        for (int v = 0; v < LOAD_U; ++v) {
          const long long e = e0 + v * 32 + lane;
          pp[v] = e < Lk && src.map(hk, (long long)cc[v], kk[v]);
        }
#pragma unroll
        for (int v = 0; v < LOAD_U; ++v) {
          const unsigned b = __ballot_sync(kFull, pp[v]);
          if (pp[v]) x_put(out_col, out_val, ok + __popc(b & lt), ek, kk[v], vv[v], st);
          ok += __popc(b);
        }
      }
    }
  }
}

// Loader view (loaders.cuh) of the recorded rows for the CTA-per-row count and fill of
// rows longer than SRC_LONG.
template <class CIt, class VTt, class Rel>
struct XLongRows {
  using CI = CIt;
  using VT = VTt;
  static constexpr bool kAllKept = false;
  static constexpr bool kLoadVals = true;
  static constexpr bool kEagerVals = true;
  static constexpr bool kRowCtx = false;
  const CI* col;
  const VT* val;
  Rel rel;
  const long long* rs0;
  const long long* rsn;
  __device__ RowSrc row(long long i) const { return RowSrc{rs0[i], 0, rsn[i], 0}; }
  __device__ const CI* cols(int) const { return col; }
  __device__ const VT* vals(int) const { return val; }
  __device__ bool test(int, long long c) const { return rel.test(c); }
  // instantiated only by the fill (the count calls test alone)
  __device__ bool map(int, long long c, uint32_t& key) const { return rel.map(c, key); }
};

}  // namespace sp
