// sp_assign: A' = A with A'(I, J) = B  (Sec. 2.3; HipAssign, Algorithm 4).
//
// HipAssign builds B' = P B Q^T (B's entry (i, j) moved to (I[i], J[j])) and adds it
// into A with a user-chosen operator.  Here, with the overwrite (REPLACE) operator:
//   * rows of A outside I are copied unchanged;
//   * row I[i] becomes (A's row without the columns of J) merged with B's row i
//     relabelled through J; both parts have distinct columns, so sorting their union
//     gives the merged canonical row.
// Identify: rowmap (row -> position in I, -1 elsewhere) and a bitmap of J; counting:
// per row of I, len_A - |A[I[i],:] ∩ J| + len_B(i); two exclusive scans give the row
// pointer of the rebuilt rows and of A'.  Fill: the rebuilt rows are gathered into a
// staging buffer (kept entries of both parts, relabelled) and sorted there in place;
// one load-balanced gather then assembles A' from A's untouched rows and the staged
// rows.
#include "dispatch.h"
#include "extract_rows.cuh"
#include "kernels.cuh"
#include "plan.h"
#include "rowsort.cuh"
#include "segcopy.cuh"

namespace sp {

template <class RP, class CIt, class VTt, class IX>
struct AssignLoader {
  using CI = CIt;
  using VT = VTt;
  // rows go to the CTA kernels by A's run alone, as the REPLACE count lists them
  static constexpr bool kLongFirst = true;
  const RP* rpA;
  const CI* colA;
  const VT* valA;
  const long long* rpB;
  const CI* colB;
  const VT* valB;
  const IX* I;
  const IX* J;
  const uint32_t* jbits;
  long long m, n, nnzA, nJ, nnzB;
  __device__ RowSrc row(long long i) const {
    const long long r = (long long)I[i];
    RowSrc rs{0, 0, 0, 0};
    if (r >= 0 && r < m) {
      const long long s = (long long)rpA[r], e = (long long)rpA[r + 1];
      if (s >= 0 && e >= s && e <= nnzA) {
        rs.s0 = s;
        rs.n0 = e - s;
      }
    }
    const long long s = rpB[i], e = rpB[i + 1];
    if (s >= 0 && e >= s && e <= nnzB) {
      rs.s1 = s;
      rs.n1 = e - s;
    }
    return rs;
  }
  static constexpr bool kAllKept = false;
  static constexpr bool kLoadVals = true;
  static constexpr bool kEagerVals = false;
  static constexpr bool kRowCtx = false;
  __device__ bool in_j(long long c) const { return (ld_map(jbits + (c >> 5)) >> (c & 31)) & 1u; }
  __device__ const CI* cols(int part) const { return part ? colB : colA; }
  __device__ const VT* vals(int part) const { return part ? valB : valA; }
  __device__ bool test(int part, long long c) const {
    return part == 0 ? (c >= 0 && c < n && !in_j(c)) : (c >= 0 && c < nJ);
  }
  __device__ bool map(int part, long long c, uint32_t& key) const {
    if (part == 0) {  // A's entry survives unless its column is assigned
      if (c < 0 || c >= n || in_j(c)) return false;
      key = uint32_t(c);
      return true;
    }
    if (c < 0 || c >= nJ) return false;  // B's column b lands in column J[b]
    key = uint32_t(ld_map(J + c));
    return true;
  }
};

// Rebuilt row I[i] under the union modes (A (+) P B Q^T, Algorithm 4 with a chosen add):
//   SELECT2ND: A's entries survive unless B's row i stores the same column (B wins);
//   PLUS: A's entries all survive, those that meet a B entry carry a + b (one IEEE add),
//   and B's entries survive unless they met an A entry.
// "Meets" is decided by a binary search in the other matrix's sorted row: for A's entry
// at column c in J, B's row i is searched for jinv[c]; for B's entry at column b, A's
// row I[i] is searched for J[b].  Keys stay unique, so the row sort applies unchanged.
template <class RP, class CIt, class VTt, class IX>
struct AssignMergeLoader {
  using CI = CIt;
  using VT = VTt;
  const RP* rpA;
  const CI* colA;
  const VT* valA;
  const long long* rpB;
  const CI* colB;
  const VT* valB;
  const IX* I;
  const IX* J;
  const IX* jinv;  // column of A -> position in J, -1 elsewhere
  const uint32_t* jbits;
  long long m, n, nnzA, nJ, nnzB;
  int plus;  // 0: SELECT2ND, 1: PLUS
  static constexpr bool kAllKept = false;
  static constexpr bool kLoadVals = true;
  static constexpr bool kEagerVals = false;
  static constexpr bool kRowCtx = true;
  __device__ RowSrc row(long long i) const {
    const long long r = (long long)I[i];
    RowSrc rs{0, 0, 0, 0};
    if (r >= 0 && r < m) {
      const long long s = (long long)rpA[r], e = (long long)rpA[r + 1];
      if (s >= 0 && e >= s && e <= nnzA) {
        rs.s0 = s;
        rs.n0 = e - s;
      }
    }
    const long long s = rpB[i], e = rpB[i + 1];
    if (s >= 0 && e >= s && e <= nnzB) {
      rs.s1 = s;
      rs.n1 = e - s;
    }
    return rs;
  }
  __device__ const CI* cols(int part) const { return part ? colB : colA; }
  __device__ const VT* vals(int part) const { return part ? valB : valA; }
  __device__ bool in_j(long long c) const { return (ld_map(jbits + (c >> 5)) >> (c & 31)) & 1u; }
  // position of column b in B's row i, or -1
  __device__ long long find_b(long long i, long long b) const {
    const long long s = rpB[i], e = rpB[i + 1];
    if (s < 0 || e < s || e > nnzB) return -1;
    const long long q = lower_bound_col(colB, s, e, b);
    return (q < e && (long long)colB[q] == b) ? q : -1;
  }
  // does A's row I[i] store column c
  __device__ bool in_a(long long i, long long c) const {
    const long long r = (long long)I[i];
    if (r < 0 || r >= m) return false;
    const long long s = (long long)rpA[r], e = (long long)rpA[r + 1];
    if (s < 0 || e < s || e > nnzA) return false;
    const long long q = lower_bound_col(colA, s, e, c);
    return q < e && (long long)colA[q] == c;
  }
  __device__ bool map_ctx(int part, long long c, uint32_t& key, long long i, long long& aux) const {
    aux = -1;
    if (part == 0) {
      if (c < 0 || c >= n) return false;
      key = uint32_t(c);
      if (!in_j(c)) return true;
      const long long q = find_b(i, (long long)ld_map(jinv + c));
      if (plus) {
        aux = q;  // the B entry added onto this one
        return true;
      }
      return q < 0;
    }
    if (c < 0 || c >= nJ) return false;
    const long long col = (long long)ld_map(J + c);
    key = uint32_t(col);
    return !plus || !in_a(i, col);
  }
  __device__ bool test_ctx(int part, long long c, long long i) const {
    uint32_t key;
    long long aux;
    return map_ctx(part, c, key, i, aux);
  }
  // values are moved as 4- or 8-byte words; PLUS adds them as the IEEE floats they hold
  // (round to nearest, no contraction)
  __device__ VT value_ctx(int part, long long pos, long long aux) const {
    const VT v = ld_stream(vals(part) + pos);
    if (aux < 0) return v;
    const VT w = ld_stream(valB + aux);
    if constexpr (sizeof(VT) == 4) {
      return VT(__float_as_uint(__fadd_rn(__uint_as_float(uint32_t(v)), __uint_as_float(uint32_t(w)))));
    } else {
      return VT(__double_as_longlong(__dadd_rn(__longlong_as_double((long long)v), __longlong_as_double((long long)w))));
    }
  }
};

// length of row r of A': len_A plus a correction that is non-zero only on rows of I
// (rebuilt length - len_A, scattered by k_assign_delta), so the scan reads two dense
// arrays and no map
template <class RP>
__device__ __forceinline__ long long len_a(const RP* rpA, long long r, long long nnzA) {
  const long long s = (long long)rpA[r], e = (long long)rpA[r + 1];
  return (s >= 0 && e >= s && e <= nnzA) ? e - s : 0;
}
template <class RP>
struct AssignLen {
  const RP* rpA;
  const int* delta;
  long long nnzA;
  __device__ long long operator()(long long r) const { return len_a(rpA, r, nnzA) + (long long)delta[r]; }
};
template <class RP, class IX>
__global__ void k_assign_delta(const IX* __restrict__ I, long long nI, const RP* __restrict__ rpA, long long m,
                               long long nnzA, const long long* __restrict__ vt, int* __restrict__ delta,
                               DevStatus* st) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nI;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = (long long)I[i];
    if (r < 0 || r >= m) continue;  // reported by the row map
    const long long d = (vt[i + 1] - vt[i]) - len_a(rpA, r, nnzA);
    if (d > 0x7fffffffll || d < -0x7fffffffll) dev_fail(st, SP_ERR_OVERFLOW, i);
    else delta[r] = int(d);
  }
}

// Assembly of A' as segments (segcopy.cuh): a segment starts at row 0, at every row of I
// and after every row of I; a run of rows outside I is contiguous in A and in A', a row
// of I is its staged rebuilt row.  The scan over the bitmap words of I's rows numbers the
// segment starts (32 rows per element); its store writes each segment (first output
// position, source position) and the count.
__device__ __forceinline__ uint32_t seg_starts(const uint32_t* ibits, long long w, long long m) {
  const uint32_t b = ibits[w], prev = w > 0 ? ibits[w - 1] >> 31 : 1u;  // row 0 starts one
  uint32_t s = b | (b << 1) | prev;
  const long long r0 = w * 32;
  if (m - r0 < 32) s &= (1u << (m - r0)) - 1u;  // rows past the last do not start one
  return s;
}
struct SegWordCount {
  const uint32_t* ibits;
  long long m;
  __device__ long long operator()(long long w) const { return __popc(seg_starts(ibits, w, m)); }
};
template <class RP, class IX>
struct SegWordStore {
  const uint32_t* ibits;
  const IX* rowmap;
  const RP* rpA;
  const long long* vt;  // row pointer of the staged rebuilt rows; null: the merge writes
                        // them in place (their segments are kSegSkip)
  const long long* vp_out;
  CopySeg* segs;
  long long m, nw, cap;
  long long* nseg;
  DevStatus* dst;
  __device__ void operator()(long long w, long long j) const {
    if (w == nw) {  // j = number of segments; the sentinel closes the last one
      if (j > cap) {
        dev_fail(dst, SP_ERR_INTERNAL, -33);
        return;
      }
      *nseg = j;
      segs[j] = CopySeg{vp_out[m], 0};
      return;
    }
    uint32_t sm = seg_starts(ibits, w, m);
    const uint32_t b = ibits[w];
    while (sm) {
      const int k = __ffs(sm) - 1;
      sm &= sm - 1;
      if (j >= cap) {
        dev_fail(dst, SP_ERR_INTERNAL, -36);
        return;
      }
      const long long r = w * 32 + k;
      const bool in_i = (b >> k) & 1u;
      segs[j++] = CopySeg{vp_out[r], !in_i ? (long long)rpA[r] : vt ? (vt[(long long)rowmap[r]] | kSegB) : kSegSkip};
    }
  }
};
// Longest row of B (row pointer rpB, n rows), saturated at 2^32 - 1.
__global__ void k_max_row_len(const long long* __restrict__ rp, long long n, unsigned* out) {
  unsigned mx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long L = rp[i + 1] - rp[i];
    const unsigned l = L <= 0 ? 0u : (L > 0xFFFFFFFFll ? 0xFFFFFFFFu : unsigned(L));
    mx = l > mx ? l : mx;
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// REPLACE count (k_xcount over A's runs): an entry of A survives unless its column is
// assigned; the rebuilt row adds all of B's row, so the row pointer's scan adds it.
struct AssignKeep {
  const uint32_t* jbits;
  long long n;
  __device__ __forceinline__ bool test(long long c) const {
    return c >= 0 && c < n && !((ld_map(jbits + (c >> 5)) >> (c & 31)) & 1u);
  }
  __device__ __forceinline__ bool map(long long c, uint32_t& key) const {
    if (!test(c)) return false;
    key = uint32_t(c);
    return true;
  }
};
struct RebuiltLen {
  const long long* kept;  // kept entries of A's run
  const long long* rpB;
  __device__ long long operator()(long long i) const { return kept[i] + (rpB[i + 1] - rpB[i]); }
};

// ---- rebuilt rows by merging (REPLACE, rows of B of at most 32 entries) ------------------
// Row I[i] of A' is the merge of two sorted runs: A's row without the columns of J
// (ascending already: A is canonical) and B's row i relabelled through J (at most 32
// entries, sorted in registers by a bitonic network).  Every kept A entry lands at its
// kept rank plus the number of B' keys below it (a search over the warp's registers);
// every B' entry at its rank plus the number of kept A entries below it (accumulated
// chunk by chunk).  No row sort follows.
constexpr unsigned kPadKey = 0xFFFFFFFFu;

// lower bound of `key` in the ascending values `v` held by lanes [0, 32) (kPadKey for
// unused lanes): the number of lanes whose value is below `key`.  All lanes call it.
__device__ __forceinline__ int warp_lower_bound(uint32_t v, uint32_t key) {
  int pos = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const uint32_t x = __shfl_sync(0xffffffffu, v, pos + step - 1);
    if (x < key) pos += step;
  }
  const uint32_t x = __shfl_sync(0xffffffffu, v, pos & 31);
  return pos + ((pos < 32 && x < key) ? 1 : 0);
}

// Ascending bitonic sort of (key, value) over the warp's first P lanes (P a power of two,
// the same in every lane; lanes at and above P hold only padding keys).
template <class VT>
__device__ __forceinline__ void warp_sort(uint32_t& k, VT& v, int P) {
  const int lane = threadIdx.x & 31;
  for (int size = 2; size <= P; size <<= 1) {
    for (int j = size >> 1; j > 0; j >>= 1) {
      const uint32_t ok = __shfl_xor_sync(0xffffffffu, k, j);
      const VT ov = __shfl_xor_sync(0xffffffffu, v, j);
      const bool up = (lane & size) == 0, lower = (lane & j) == 0;
      if (lower == up ? ok < k : ok > k) {
        k = ok;
        v = ov;
      }
    }
  }
}

template <class RP, class CI, class VT, class IX>
struct MergeSrc {
  const RP* rpA;
  const CI* colA;
  const VT* valA;
  const long long* rpB;
  const CI* colB;
  const VT* valB;
  const IX* I;
  const IX* J;
  const uint32_t* jbits;
  const long long* rs0;  // A's run of every row of I, recorded by the count
  const long long* rsn;
  long long m, n, nnzA, nJ, nnzB;
  // A's row I[i] (as the count resolved it) and B's row i (range validated)
  __device__ void rows(long long i, long long& sA, long long& LA, long long& sB, long long& LB) const {
    sA = rs0[i];
    LA = rsn[i];
    sB = LB = 0;
    const long long s = rpB[i], e = rpB[i + 1];
    if (s >= 0 && e >= s && e <= nnzB) {
      sB = s;
      LB = e - s;
    }
  }
  // B's row i relabelled through J into this lane's (key, value), sorted across the warp;
  // returns the number of entries (B entries with a column outside [0, nJ) are dropped,
  // as the count drops them)
  __device__ int load_b(long long sB, long long LB, uint32_t& bk, VT& bv) const {
    const int lane = threadIdx.x & 31;
    bk = kPadKey;
    bv = VT(0);
    if (lane < LB) {
      const long long c = (long long)colB[sB + lane];
      if (c >= 0 && c < nJ) {
        bk = uint32_t((long long)ld_map(J + c));
        bv = valB[sB + lane];
      }
    }
    const int P = LB <= 2 ? 2 : 1 << (32 - __clz(int(LB) - 1));
    warp_sort(bk, bv, P);
    return __popc(__ballot_sync(0xffffffffu, bk != kPadKey));
  }
  __device__ bool in_j(long long c) const { return (ld_map(jbits + (c >> 5)) >> (c & 31)) & 1u; }
};

// First output position of rebuilt row i: in A' itself (vdst = A''s row pointer, row I[i])
// or in the staging buffer (vdst null, row pointer vp of the rebuilt rows).
template <class IX>
__device__ __forceinline__ long long merge_out(const long long* vdst, const IX* I, const long long* vp, long long i) {
  return vdst ? vdst[(long long)I[i]] : vp[i];
}

// Rows of at most SRC_LONG source entries (A's and B's together), one warp each.
template <class RP, class CI, class VT, class IX>
__global__ void __launch_bounds__(256) k_assign_merge_warp(MergeSrc<RP, CI, VT, IX> ms, long long nI,
                                                           const long long* __restrict__ vp,
                                                           const long long* __restrict__ vdst, CI* __restrict__ tcol,
                                                           VT* __restrict__ tval, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = w0; i < nI; i += nw) {
    long long sA, LA, sB, LB;
    ms.rows(i, sA, LA, sB, LB);
    if (LA > SRC_LONG) continue;  // k_assign_merge_long (the count listed it)
    const long long o = merge_out(vdst, ms.I, vp, i), oe = o + (vp[i + 1] - vp[i]);
    uint32_t bk;
    VT bv;
    const int nb = ms.load_b(sB, LB, bk, bv);
    long long kbase = 0;
    unsigned cntA = 0;
    for (long long e0 = 0; e0 < LA; e0 += 32) {
      const long long e = e0 + lane;
      const bool valid = e < LA;
      const long long c = valid ? (long long)ld_stream(ms.colA + sA + e) : 0;
      const bool kept = valid && c >= 0 && c < ms.n && !ms.in_j(c);
      VT v;
      if (kept) v = ld_stream(ms.valA + sA + e);
      const unsigned km = __ballot_sync(0xffffffffu, kept);
      const uint32_t ck = valid ? uint32_t(c) : kPadKey;
      const int nless = warp_lower_bound(bk, ck);   // B' keys below this A column
      const int lbc = warp_lower_bound(ck, bk);     // this chunk's A columns below this B' key
      if (kept) {
        const long long pos = o + kbase + __popc(km & lt) + nless;
        if (pos < oe) {
          st_stream(tcol + pos, CI(c));
          st_stream(tval + pos, v);
        } else {
          dev_fail(st, SP_ERR_INTERNAL, -30);
        }
      }
      cntA += __popc(km & (lbc >= 32 ? 0xffffffffu : ((1u << lbc) - 1u)));
      kbase += __popc(km);
    }
    if (lane < nb) {
      const long long pos = o + lane + cntA;
      if (pos < oe) {
        st_stream(tcol + pos, CI(bk));
        st_stream(tval + pos, bv);
      } else {
        dev_fail(st, SP_ERR_INTERNAL, -31);
      }
    }
    if (lane == 0 && o + kbase + nb != oe) dev_fail(st, SP_ERR_INTERNAL, -32);
  }
}

// Rows of more than SRC_LONG source entries (the count's list), one 1024-thread CTA each:
// a step takes LOAD_U x 1024 consecutive entries, warp w of slice u the 32 entries at
// u * 1024 + 32 w; the kept counts of the step's LOAD_U x 32 chunks are scanned once, in
// chunk order, and each warp's counts of kept entries below the B' keys are added up.
template <class RP, class CI, class VT, class IX>
__global__ void __launch_bounds__(1024) k_assign_merge_long(MergeSrc<RP, CI, VT, IX> ms,
                                                            const long long* __restrict__ cl_rows,
                                                            const unsigned* __restrict__ n_cl, long long cl_cap,
                                                            const long long* __restrict__ vp,
                                                            const long long* __restrict__ vdst, unsigned* ticket,
                                                            CI* __restrict__ tcol, VT* __restrict__ tval,
                                                            DevStatus* st) {
  constexpr int NW = 1024 / 32, NCH = NW * LOAD_U;  // chunks of one step
  static_assert(NCH % 32 == 0 && NCH <= 32 * 32, "one warp scans a step's chunks");
  __shared__ unsigned s_item;
  __shared__ unsigned s_wc[NCH], s_tot, s_cnt[32];
  __shared__ long long s_base;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned lt = (1u << lane) - 1u;
  unsigned count = *n_cl;
  if (count > cl_cap) count = unsigned(cl_cap);
  for (;;) {
    if (t == 0) {
      s_item = atomicAdd(ticket, 1u);
      s_base = 0;
    }
    if (t < 32) s_cnt[t] = 0;
    __syncthreads();
    const unsigned item = s_item;
    if (item >= count) break;
    const long long i = cl_rows[item];
    long long sA, LA, sB, LB;
    ms.rows(i, sA, LA, sB, LB);
    const long long o = merge_out(vdst, ms.I, vp, i), oe = o + (vp[i + 1] - vp[i]);
    uint32_t bk;
    VT bv;
    const int nb = ms.load_b(sB, LB, bk, bv);
    unsigned cntA = 0;
    for (long long e0 = 0; e0 < LA; e0 += (long long)blockDim.x * LOAD_U) {
      long long cc[LOAD_U];
      VT vv[LOAD_U];
      unsigned km[LOAD_U];
      int nless[LOAD_U];
#pragma unroll
      for (int u = 0; u < LOAD_U; ++u) {
        const long long e = e0 + (long long)u * blockDim.x + t;
        const bool valid = e < LA;
        cc[u] = valid ? (long long)ld_stream(ms.colA + sA + e) : 0;
        const bool kept = valid && cc[u] >= 0 && cc[u] < ms.n && !ms.in_j(cc[u]);
        if (kept) vv[u] = ld_stream(ms.valA + sA + e);
        km[u] = __ballot_sync(0xffffffffu, kept);
        const uint32_t ck = valid ? uint32_t(cc[u]) : kPadKey;
        nless[u] = warp_lower_bound(bk, ck);
        const int lbc = warp_lower_bound(ck, bk);
        cntA += __popc(km[u] & (lbc >= 32 ? 0xffffffffu : ((1u << lbc) - 1u)));
        if (lane == 0) s_wc[u * NW + w] = __popc(km[u]);
      }
      __syncthreads();
      if (w == 0) {  // exclusive prefix of the step's chunk counts, in chunk order
        constexpr int PER = NCH / 32;
        unsigned x[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          x[q] = s_wc[lane * PER + q];
          sum += x[q];
        }
        const unsigned inc = warp_incl_sum(sum);
        unsigned run = inc - sum;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          s_wc[lane * PER + q] = run;
          run += x[q];
        }
        if (lane == 31) s_tot = inc;
      }
      __syncthreads();
      const long long base = s_base;
#pragma unroll
      for (int u = 0; u < LOAD_U; ++u) {
        if (!((km[u] >> lane) & 1u)) continue;
        const long long pos = o + base + s_wc[u * NW + w] + __popc(km[u] & lt) + nless[u];
        if (pos < oe) {
          st_stream(tcol + pos, CI(cc[u]));
          st_stream(tval + pos, vv[u]);
        } else {
          dev_fail(st, SP_ERR_INTERNAL, -33);
        }
      }
      __syncthreads();  // every thread has read s_base and s_wc
      if (t == 0) s_base += s_tot;
    }
    atomicAdd(&s_cnt[lane], cntA);
    __syncthreads();
    if (w == 0) {
      if (lane < nb) {
        const long long pos = o + lane + s_cnt[lane];
        if (pos < oe) {
          st_stream(tcol + pos, CI(bk));
          st_stream(tval + pos, bv);
        } else {
          dev_fail(st, SP_ERR_INTERNAL, -34);
        }
      }
      if (lane == 0 && o + s_base + nb != oe) dev_fail(st, SP_ERR_INTERNAL, -35);
    }
    __syncthreads();
  }
}

template <class RP, class CI, class IX>
sp_status assign_count_impl(sp_ctx* ctx, sp_plan* pl, cudaStream_t s) {
  const sp_csr& A = pl->A;
  const sp_csr& B = pl->B;
  const long long m = A.nrows, n = A.ncols, nI = pl->nI, nJ = pl->nJ;
  const IX* I = static_cast<const IX*>(pl->I);
  const IX* J = static_cast<const IX*>(pl->J);
  Carver cv;
  const size_t o_rm = cv.reserve(size_t(m) * sizeof(IX));
  const size_t o_jb = cv.reserve(size_t((n + 31) / 32) * 4);
  const size_t o_vt = cv.reserve(size_t(nI + 1) * 8);
  const size_t o_vo = cv.reserve(size_t(m + 1) * 8);
  const size_t o_rb = cv.reserve(size_t(nI + 1) * 8);
  pl->list_cap = nI + 1;
  const size_t o_cl = cv.reserve(size_t(pl->list_cap) * 8);
  const size_t o_cn = cv.reserve(64);
  const size_t o_s1 = cv.reserve(scan_ws_bytes(nI));
  const size_t o_s2 = cv.reserve(scan_ws_bytes(m));
  const bool merge = pl->mode != SP_ASSIGN_REPLACE;
  const size_t o_ji = cv.reserve(merge ? size_t(n) * sizeof(IX) : 0);
  const size_t o_dl = cv.reserve(size_t(m) * 4);                 // row-length corrections on rows of I
  const size_t o_ib = cv.reserve(size_t((m + 31) / 32) * 4);      // bitmap of I's rows
  const size_t o_r0 = cv.reserve(merge ? 0 : size_t(nI) * 8);  // REPLACE: A's run of every row of I
  const size_t o_rn = cv.reserve(merge ? 0 : size_t(nI) * 8);
  SP_TRY(plan_alloc(ctx, pl, cv.total(), s));
  cv.bind(pl->buf);
  IX* rowmap = cv.at<IX>(o_rm);
  uint32_t* jbits = cv.at<uint32_t>(o_jb);
  pl->rowmap = rowmap;
  pl->jmap = jbits;
  pl->vp = cv.at<long long>(o_vt);
  pl->vp_out = cv.at<long long>(o_vo);
  pl->rpB = cv.at<long long>(o_rb);
  pl->cl_rows = cv.at<long long>(o_cl);
  pl->counters = cv.at<unsigned>(o_cn);
  pl->ibits = cv.at<uint32_t>(o_ib);
  int* delta = cv.at<int>(o_dl);
  pl->sstart = merge ? nullptr : cv.at<long long>(o_r0);
  pl->slen = merge ? nullptr : cv.at<long long>(o_rn);
  const int nsm = ctx->num_sms;
  SP_CUDA(cudaMemsetAsync(pl->counters, 0, 64, s));
  SP_CUDA(cudaMemsetAsync(rowmap, 0xFF, size_t(m) * sizeof(IX), s));
  SP_CUDA(cudaMemsetAsync(jbits, 0, size_t((n + 31) / 32) * 4, s));
  SP_CUDA(cudaMemsetAsync(pl->ibits, 0, size_t((m + 31) / 32) * 4, s));
  SP_CUDA(cudaMemsetAsync(delta, 0, size_t(m) * 4, s));
  if (nI > 0) {
    {
      SP_PHASE(SP_PHASE_MAP);
      k_inverse_map_bits<IX><<<grid_for(nI, 256, nsm * 8), 256, 0, s>>>(I, nI, m, rowmap, pl->ibits,
                                                                         ctx->dstatus, SP_ERR_DUPLICATE_INDEX);
    }
    SP_CUDA(cudaGetLastError());
  }
  if (nJ > 0) {
    {
      SP_PHASE(SP_PHASE_MAP);
      k_mark_bits<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, n, jbits, ctx->dstatus,
                                                                  SP_ERR_DUPLICATE_INDEX);
    }
    SP_CUDA(cudaGetLastError());
  }
  IX* jinv = merge ? cv.at<IX>(o_ji) : nullptr;
  pl->jinv = jinv;
  if (merge && nJ > 0) {
    SP_CUDA(cudaMemsetAsync(jinv, 0xFF, size_t(n) * sizeof(IX), s));
    {
      SP_PHASE(SP_PHASE_MAP);
      k_inverse_map<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, n, jinv, ctx->dstatus,
                                                                    SP_ERR_DUPLICATE_INDEX);
    }
    SP_CUDA(cudaGetLastError());
  }
  SP_TRY(widen_rowptr(ctx, s, B.rowptr, B.rowptr_type, nI + 1, pl->rpB));
  if (nI > 0) {
    {
      SP_PHASE(SP_PHASE_COUNT);
      k_max_row_len<<<grid_for(nI, 256, nsm * 8), 256, 0, s>>>(pl->rpB, nI, pl->counters + 6);
    }
    SP_CUDA(cudaGetLastError());
  }
  if (nI > 0) {
    CountLists cl{pl->cl_rows, pl->counters + 0, pl->list_cap};
    auto count = [&](const auto& ct) -> sp_status {
      {
        SP_PHASE(SP_PHASE_COUNT);
        k_count_warp<<<grid_for(nI * 32, 256, nsm * 16), 256, 0, s>>>(ct, nI, pl->vp, cl, ctx->cur.count_rows,
                                                                         ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
      {
        SP_PHASE(SP_PHASE_COUNT);
        k_count_long<<<nsm, 1024, 0, s>>>(ct, pl->vp, cl, pl->counters + 3, ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
      return SP_OK;
    };
    if (merge) {
      SP_TRY(count(AssignMergeLoader<RP, CI, uint32_t, IX>{
          static_cast<const RP*>(A.rowptr), static_cast<const CI*>(A.colidx), nullptr, pl->rpB,
          static_cast<const CI*>(B.colidx), nullptr, I, J, jinv, jbits, m, n, A.nnz, nJ, B.nnz,
          pl->mode == SP_ASSIGN_PLUS ? 1 : 0}));
    } else {
      // REPLACE: the surviving entries of A's runs, lane-per-row (k_xcount; runs of more
      // than SRC_LONG entries listed for one CTA each); B's rows are added by the scan
      const AssignKeep keep{jbits, n};
      const CI* colA = static_cast<const CI*>(A.colidx);
      {
        SP_PHASE(SP_PHASE_COUNT);
        const XOne<CI, uint32_t, AssignKeep> src{colA, nullptr, keep};
        const XResolveI<RP, IX> res{static_cast<const RP*>(A.rowptr), I, m, A.nnz, pl->sstart, pl->slen,
                                    ctx->dstatus};
        k_xcount<<<grid_for((nI + 31) / 32 * 32, XB, nsm * 8), XB, 0, s>>>(
            src, res, nI, pl->vp, pl->cl_rows, pl->counters + 0, pl->list_cap, pl->counters + 4, ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
      {
        SP_PHASE(SP_PHASE_COUNT);
        const XLongRows<CI, uint32_t, AssignKeep> lr{colA, nullptr, keep, pl->sstart, pl->slen};
        k_count_long<<<nsm, 1024, 0, s>>>(lr, pl->vp, cl, pl->counters + 3, ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
    }
  }
  if (merge) {
    SP_TRY(launch_scan(ctx, s, LoadArray<long long>{pl->vp},
                       StoreDual<long long>{pl->vp, nullptr, ctx->dstatus}, nI, cv.at<char>(o_s1)));
  } else {
    SP_TRY(launch_scan(ctx, s, RebuiltLen{pl->vp, pl->rpB}, StoreDual<long long>{pl->vp, nullptr, ctx->dstatus}, nI,
                       cv.at<char>(o_s1)));
  }
  if (nI > 0) {
    SP_PHASE(SP_PHASE_SCAN);
    k_assign_delta<RP, IX><<<grid_for(nI, 256, nsm * 8), 256, 0, s>>>(I, nI, static_cast<const RP*>(A.rowptr), m,
                                                                      A.nnz, pl->vp, delta, ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  AssignLen<RP> len{static_cast<const RP*>(A.rowptr), delta, A.nnz};
  SP_TRY(launch_scan(ctx, s, len, StoreDual<long long>{pl->vp_out, nullptr, ctx->dstatus}, m,
                     cv.at<char>(o_s2)));
  SP_CUDA(cudaMemcpyAsync(pl->h_tail, pl->vp_out + m, 8, cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaMemcpyAsync(pl->h_tail + 1, pl->vp + nI, 8, cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaMemcpyAsync(pl->h_tail + 2, pl->counters + 6, 4, cudaMemcpyDeviceToHost, s));
  SP_TRY(ctx_collect(ctx, s));
  pl->nnz_out = pl->h_tail[0];
  pl->nnz_temp = pl->h_tail[1];
  pl->max_lb = nI > 0 ? (long long)*reinterpret_cast<const unsigned*>(pl->h_tail + 2) : 0;
  return SP_OK;
}

// The rebuilt rows of I (kept entries of both parts, relabelled) into the staging buffer
// at the rebuilt-row pointer pl->vp, in source order.  `ticket` holds 16 bytes.
template <class RP, class CI, class VT, class IX>
sp_status assign_stage(sp_ctx* ctx, sp_plan* pl, CI* tcol, VT* tval, unsigned* ticket, cudaStream_t s) {
  const sp_csr& A = pl->A;
  const sp_csr& B = pl->B;
  const long long nI = pl->nI;
  const int nsm = ctx->num_sms;
  SP_CUDA(cudaMemsetAsync(ticket, 0, 16, s));
  auto fill = [&](const auto& ld) -> sp_status {
    {
      SP_PHASE(SP_PHASE_GATHER);
      k_fill_warp<<<grid_for(nI * 32, 256, nsm * 16), 256, 0, s>>>(ld, nI, pl->vp, tcol, tval, ctx->cur.fill_rows,
                                                                        ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    {
      SP_PHASE(SP_PHASE_GATHER);
      k_fill_long<<<nsm, 1024, 0, s>>>(ld, pl->cl_rows, pl->counters + 0, pl->list_cap, pl->vp, ticket, tcol,
                                       tval, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    return SP_OK;
  };
  if (pl->mode != SP_ASSIGN_REPLACE) {
    return fill(AssignMergeLoader<RP, CI, VT, IX>{
        static_cast<const RP*>(A.rowptr), static_cast<const CI*>(A.colidx), static_cast<const VT*>(A.values),
        pl->rpB, static_cast<const CI*>(B.colidx), static_cast<const VT*>(B.values),
        static_cast<const IX*>(pl->I), static_cast<const IX*>(pl->J), static_cast<const IX*>(pl->jinv),
        static_cast<const uint32_t*>(pl->jmap), A.nrows, A.ncols, A.nnz, pl->nJ, B.nnz,
        pl->mode == SP_ASSIGN_PLUS ? 1 : 0});
  }
  return fill(AssignLoader<RP, CI, VT, IX>{static_cast<const RP*>(A.rowptr), static_cast<const CI*>(A.colidx),
                                           static_cast<const VT*>(A.values), pl->rpB,
                                           static_cast<const CI*>(B.colidx), static_cast<const VT*>(B.values),
                                           static_cast<const IX*>(pl->I), static_cast<const IX*>(pl->J),
                                           static_cast<const uint32_t*>(pl->jmap), A.nrows, A.ncols, A.nnz,
                                           pl->nJ, B.nnz});
}

template <class RP, class CI, class VT, class IX>
sp_status assign_fill_impl(sp_ctx* ctx, sp_plan* pl, sp_csr* Ap, cudaStream_t s) {
  const sp_csr& A = pl->A;
  const long long m = A.nrows, nI = pl->nI, nt = pl->nnz_temp, nnz_out = pl->nnz_out;
  SP_TRY(store_rowptr(ctx, s, pl->vp_out, m + 1, Ap->rowptr_type, Ap->rowptr));
  if (nnz_out == 0) return SP_OK;
  // merge: the rebuilt rows (A's surviving run and B's relabelled row, both in order) are
  // written straight into A'; otherwise they are staged, sorted, and copied with the rest
  const bool merge = nt > 0 && pl->mode == SP_ASSIGN_REPLACE && pl->max_lb <= 32;
  const bool staged = nt > 0 && !merge;
  const long long segcap = m < 2 * nI + 1 ? m : 2 * nI + 1;
  const long long nchunks = (nnz_out + SC_CH - 1) / SC_CH;
  Carver cv;
  const size_t o_tc = cv.reserve(staged ? size_t(nt) * sizeof(CI) : 0);
  const size_t o_tv = cv.reserve(staged ? size_t(nt) * sizeof(VT) : 0);
  const size_t o_tk = cv.reserve(16);
  const size_t o_sg = cv.reserve(size_t(segcap + 1) * sizeof(CopySeg));
  const size_t o_ns = cv.reserve(8);
  const size_t o_cf = cv.reserve(size_t(nchunks) * 8);
  const size_t o_sc = cv.reserve(scan_ws_bytes(m));
  size_t r1[kRowsSlots];
  rows_reserve(cv, staged ? nI : 0, staged ? nt : 0, sizeof(VT), r1);
  char* base;
  SP_TRY(ctx_workspace(ctx, cv.total(), s, &base));
  cv.bind(base);
  CI* tcol = staged ? cv.at<CI>(o_tc) : nullptr;
  VT* tval = staged ? cv.at<VT>(o_tv) : nullptr;
  const int nsm = ctx->num_sms;
  if (staged) {
    // rebuilt rows: A's surviving entries and B's relabelled ones, staged, then sorted
    SP_TRY((assign_stage<RP, CI, VT, IX>(ctx, pl, tcol, tval, cv.at<unsigned>(o_tk), s)));
    const RowsWs w1 = rows_bind(cv, nI, nt, r1);
    const int kb = ceil_log2_u64(uint64_t(A.ncols));
    SP_TRY((run_rows<CI, VT, NoGather<CI, VT>>(ctx, s, pl->vp, nI, nt, kb, w1, nullptr, true, tcol, tval)));
  }
  // assembly: runs of untouched rows from A, rows of I from the staging buffer (or left
  // to the merge)
  const IX* rowmap = static_cast<const IX*>(pl->rowmap);
  CopySeg* segs = cv.at<CopySeg>(o_sg);
  long long* nseg = cv.at<long long>(o_ns);
  long long* chunk_first = cv.at<long long>(o_cf);
  const long long nw = (m + 31) / 32;
  SP_TRY(launch_scan(ctx, s, SegWordCount{pl->ibits, m},
                     SegWordStore<RP, IX>{pl->ibits, rowmap, static_cast<const RP*>(A.rowptr),
                                          staged ? pl->vp : nullptr, pl->vp_out, segs, m, nw, segcap, nseg,
                                          ctx->dstatus},
                     nw, cv.at<char>(o_sc), SP_PHASE_PARTITION));
  SP_CUDA(cudaMemsetAsync(chunk_first, 0xFF, size_t(nchunks) * 8, s));
  {
    SP_PHASE(SP_PHASE_PARTITION);
    k_seg_chunks<<<grid_for(segcap, 256, nsm * 8), 256, 0, s>>>(segs, nseg, nchunks, chunk_first);
  }
  SP_CUDA(cudaGetLastError());
  using CW = std::conditional_t<sizeof(CI) == 4, uint32_t, unsigned long long>;
  using VW = std::conditional_t<sizeof(VT) == 4, uint32_t, unsigned long long>;
  auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int vec = al(A.colidx) && al(A.values) && al(tcol) && al(tval) && al(Ap->colidx) && al(Ap->values);
  // The copy and the merge write disjoint rows of A'.  With the context's overlap on, the
  // copy (bandwidth-bound) runs on the side stream at SC_MINB_OVERLAP CTAs per SM while
  // the merge (latency-bound) takes the rest of each SM on `s`.
  const bool fork = merge && ctx->overlap && ctx->side;
  cudaStream_t cs = fork ? ctx->side : s;
  if (fork) {
    SP_CUDA(cudaEventRecord(ctx->fork_ev, s));
    SP_CUDA(cudaStreamWaitEvent(cs, ctx->fork_ev, 0));
  }
  cudaError_t launched;
  {
    ::sp::PhaseScope ph(ctx, cs, SP_PHASE_GATHER);
    const long long gmax = (long long)(fork ? SC_MINB_OVERLAP : SC_MINB) * nsm;
    const long long g = nchunks < gmax ? nchunks : gmax;
    k_seg_copy<CW, VW><<<unsigned(g), SC_BLOCK, 0, cs>>>(
        segs, nseg, nnz_out, chunk_first, nchunks, static_cast<const CW*>(A.colidx), static_cast<const VW*>(A.values),
        A.nnz, reinterpret_cast<const CW*>(tcol), reinterpret_cast<const VW*>(tval), staged ? nt : 0,
        static_cast<CW*>(Ap->colidx), static_cast<VW*>(Ap->values), vec, ctx->dstatus);
    launched = cudaGetLastError();
  }
  if (fork) SP_CUDA(cudaEventRecord(ctx->join_ev, cs));
  if (launched == cudaSuccess && merge) {
    const sp_csr& B = pl->B;
    const MergeSrc<RP, CI, VT, IX> ms{static_cast<const RP*>(A.rowptr), static_cast<const CI*>(A.colidx),
                                     static_cast<const VT*>(A.values), pl->rpB, static_cast<const CI*>(B.colidx),
                                     static_cast<const VT*>(B.values), static_cast<const IX*>(pl->I),
                                     static_cast<const IX*>(pl->J), static_cast<const uint32_t*>(pl->jmap), pl->sstart,
                                     pl->slen, A.nrows, A.ncols, A.nnz, pl->nJ, B.nnz};
    CI* oc = static_cast<CI*>(Ap->colidx);
    VT* ov = static_cast<VT*>(Ap->values);
    unsigned* ticket = cv.at<unsigned>(o_tk);
    launched = cudaMemsetAsync(ticket, 0, 16, s);
    if (launched == cudaSuccess) {
      SP_PHASE(SP_PHASE_GATHER);
      k_assign_merge_warp<<<grid_for(nI * 32, 256, nsm * 16), 256, 0, s>>>(ms, nI, pl->vp, pl->vp_out, oc, ov,
                                                                            ctx->dstatus);
      launched = cudaGetLastError();
    }
    if (launched == cudaSuccess) {
      SP_PHASE(SP_PHASE_GATHER);
      k_assign_merge_long<<<nsm, 1024, 0, s>>>(ms, pl->cl_rows, pl->counters + 0, pl->list_cap, pl->vp,
                                                pl->vp_out, ticket, oc, ov, ctx->dstatus);
      launched = cudaGetLastError();
    }
  }
  if (fork) SP_CUDA(cudaStreamWaitEvent(s, ctx->join_ev, 0));
  SP_CUDA(launched);
  return SP_OK;
}


// ---- fused assignment + permutation (the paper's incremental-update use, Sec. 6.3) ----
// out = P (A (+) P_I B Q_J^T) Q^T: output row i is row p[i] of A' = A with the
// assignment applied, columns relabelled through qinv, sorted.  Row p[i] of A' is A's
// own row (p[i] outside I) or the staged rebuilt row; one gather reads either, so A' is
// never assembled.
template <class RP, class IX>
struct FusedLen {
  const IX* p;
  const long long* vpa;  // row pointer of A'
  const IX* rowmap;      // row of A -> position in I, -1 elsewhere
  const long long* vt;   // row pointer of the staged rebuilt rows
  const RP* rpA;
  long long m;
  long long* sstart;     // source start of output row i (staged: bit 62 set)
  __device__ long long operator()(long long i) const {
    const long long r = p ? (long long)p[i] : i;
    if (r < 0 || r >= m) {
      sstart[i] = 0;
      return 0;  // reported by the permutation check
    }
    const long long k = (long long)rowmap[r];
    sstart[i] = k >= 0 ? (vt[k] | (1ll << 62)) : (long long)rpA[r];
    return vpa[r + 1] - vpa[r];
  }
};

template <class CIt, class VTt, class IX>
struct FusedGs {
  using CI = CIt;
  using VT = VTt;
  static constexpr long long kStaged = 1ll << 62;
  const CI* colA;
  const VT* valA;
  const CI* tcol;
  const VT* tval;
  const IX* qinv;  // null: identity
  const long long* sstart;
  long long nnzA, ntemp, n;
  __device__ long long src(long long i) const { return sstart[i]; }
  __device__ CI col(long long pos) const {
    if (pos & kStaged) {
      const long long q = pos & ~kStaged;
      return q < ntemp ? ld_stream(tcol + q) : CI(0);
    }
    return (pos >= 0 && pos < nnzA) ? ld_stream(colA + pos) : CI(0);
  }
  __device__ VT val(long long pos) const {
    if (pos & kStaged) {
      const long long q = pos & ~kStaged;
      return q < ntemp ? ld_stream(tval + q) : VT(0);
    }
    return (pos >= 0 && pos < nnzA) ? ld_stream(valA + pos) : VT(0);
  }
  __device__ CI map(long long, CI c) const {
    if (!qinv) return c;
    const long long cl = (long long)c;
    if (cl < 0 || cl >= n) return CI(-1);  // reported as SP_ERR_INDEX_RANGE by the sort
    return CI(ld_map(qinv + cl));
  }
};

template <class RP, class CI, class VT, class IX>
sp_status assign_permute_impl(sp_ctx* ctx, sp_plan* pl, const IX* p, const IX* q, sp_csr* out,
                              cudaStream_t s) {
  const sp_csr& A = pl->A;
  const long long m = A.nrows, n = A.ncols, nt = pl->nnz_temp, nnz_out = pl->nnz_out;
  const bool sym = p && q && (const void*)p == (const void*)q && m == n;
  const bool out64 = out->rowptr_type == SP_I64;
  Carver cv;
  const size_t o_tc = cv.reserve(size_t(nt) * sizeof(CI));
  const size_t o_tv = cv.reserve(size_t(nt) * sizeof(VT));
  const size_t o_tk = cv.reserve(16);
  const size_t o_qinv = cv.reserve(q ? size_t(n) * sizeof(IX) : 0);
  const size_t o_qbits = cv.reserve(q ? size_t((n + 31) / 32) * 4 : 0);
  const size_t o_pbits = cv.reserve((p && !sym) ? size_t((m + 31) / 32) * 4 : 0);
  const size_t o_vp = cv.reserve(out64 ? 0 : size_t(m + 1) * 8);
  const size_t o_ss = cv.reserve(size_t(m) * 8);
  const size_t o_scan = cv.reserve(scan_ws_bytes(m));
  size_t ro[kRowsSlots];
  rows_reserve(cv, m, nnz_out, sizeof(VT), ro);
  char* base;
  SP_TRY(ctx_workspace(ctx, cv.total(), s, &base));
  cv.bind(base);
  const int nsm = ctx->num_sms;
  IX* qinv = q ? cv.at<IX>(o_qinv) : nullptr;
  if (q) {
    uint32_t* qbits = cv.at<uint32_t>(o_qbits);
    SP_CUDA(cudaMemsetAsync(qinv, 0xFF, size_t(n) * sizeof(IX), s));
    SP_CUDA(cudaMemsetAsync(qbits, 0, size_t((n + 31) / 32) * 4, s));
    {
      SP_PHASE(SP_PHASE_MAP);
      k_inverse_map_bits<IX><<<grid_for(n, 256, nsm * 8), 256, 0, s>>>(q, n, n, qinv, qbits, ctx->dstatus,
                                                                        SP_ERR_NOT_PERMUTATION);
    }
    SP_CUDA(cudaGetLastError());
  }
  if (p && !sym) {
    uint32_t* bits = cv.at<uint32_t>(o_pbits);
    SP_CUDA(cudaMemsetAsync(bits, 0, size_t((m + 31) / 32) * 4, s));
    {
      SP_PHASE(SP_PHASE_MAP);
      k_mark_bits<IX><<<grid_for(m, 256, nsm * 8), 256, 0, s>>>(p, m, m, bits, ctx->dstatus,
                                                                SP_ERR_NOT_PERMUTATION);
    }
    SP_CUDA(cudaGetLastError());
  }
  CI* tcol = cv.at<CI>(o_tc);
  VT* tval = cv.at<VT>(o_tv);
  if (nt > 0) SP_TRY((assign_stage<RP, CI, VT, IX>(ctx, pl, tcol, tval, cv.at<unsigned>(o_tk), s)));
  // output row lengths (rows of A' moved by p) and their sources
  long long* vp = out64 ? static_cast<long long*>(out->rowptr) : cv.at<long long>(o_vp);
  long long* sstart = cv.at<long long>(o_ss);
  const FusedLen<RP, IX> len{p, pl->vp_out, static_cast<const IX*>(pl->rowmap), pl->vp,
                             static_cast<const RP*>(A.rowptr), m, sstart};
  if (out64) {
    SP_TRY(launch_scan(ctx, s, len, StoreDual<long long>{vp, nullptr, ctx->dstatus}, m, cv.at<char>(o_scan)));
  } else {
    SP_TRY(launch_scan(ctx, s, len, StoreDual<int32_t>{vp, static_cast<int32_t*>(out->rowptr), ctx->dstatus}, m,
                       cv.at<char>(o_scan)));
  }
  if (nnz_out == 0) return SP_OK;
  const FusedGs<CI, VT, IX> g{static_cast<const CI*>(A.colidx), static_cast<const VT*>(A.values), tcol, tval,
                              qinv, sstart, A.nnz, nt, n};
  const RowsWs w = rows_bind(cv, m, nnz_out, ro);
  const int kb = ceil_log2_u64(uint64_t(n));
  return run_rows(ctx, s, vp, m, nnz_out, kb, w, &g, true, static_cast<CI*>(out->colidx),
                  static_cast<VT*>(out->values));
}

}  // namespace sp

using namespace sp;

extern "C" sp_status sp_assign_count(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                                     const void* J, int64_t nJ, sp_itype idx_type, const sp_csr* B,
                                     sp_assign_mode mode, sp_plan** plan, int64_t* nnz_out,
                                     sp_stream_t stream) {
  if (!ctx || !A || !B || !plan || !nnz_out) return SP_ERR_INVALID_ARG;
  *plan = nullptr;
  SP_TRY(check_csr(A));
  SP_TRY(check_csr(B));
  if (idx_type != SP_I32 && idx_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (mode != SP_ASSIGN_REPLACE && mode != SP_ASSIGN_SELECT2ND && mode != SP_ASSIGN_PLUS)
    return SP_ERR_INVALID_ARG;
  if (nI < 0 || nJ < 0 || nI > A->nrows || nJ > A->ncols) return SP_ERR_SHAPE;
  if ((nI > 0 && !I) || (nJ > 0 && !J)) return SP_ERR_INVALID_ARG;
  if (B->nrows != nI || B->ncols != nJ) return SP_ERR_SHAPE;
  if (B->colidx_type != A->colidx_type || B->value_type != A->value_type) return SP_ERR_INVALID_ARG;
  if (idx_type == SP_I32 && (A->nrows > INT32_MAX || A->ncols > INT32_MAX)) return SP_ERR_OVERFLOW;
  if (A->ncols > J_KEY_LIMIT) return SP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, SP_OP_ASSIGN, A->nnz);
  SP_TRY(validate_if_asked(ctx, A, s));
  SP_TRY(validate_if_asked(ctx, B, s));
  sp_plan* pl = new sp_plan();
  pl->op = 1;
  pl->A = *A;
  pl->B = *B;
  pl->I = I;
  pl->J = J;
  pl->nI = nI;
  pl->nJ = nJ;
  pl->idx_type = idx_type;
  pl->mode = mode;
  pl->stream = s;
  sp_status st = dispatch_i(A->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(A->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_i(idx_type, [&](auto ix) {
        using IX = decltype(ix);
        return assign_count_impl<RP, CI, IX>(ctx, pl, s);
      });
    });
  });
  if (st != SP_OK) {
    plan_release(ctx, pl);
    return st;
  }
  *plan = pl;
  *nnz_out = pl->nnz_out;
  return SP_OK;
}

extern "C" sp_status sp_assign_fill(sp_ctx* ctx, sp_plan* pl, sp_csr* Ap, sp_stream_t stream) {
  if (!ctx || !pl || !Ap || pl->op != 1) return SP_ERR_INVALID_ARG;
  if (Ap->rowptr_type != SP_I32 && Ap->rowptr_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (Ap->rowptr_type == SP_I32 && pl->nnz_out > INT32_MAX) return SP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, SP_OP_ASSIGN, pl->A.nnz);
  pl->stream = s;
  Ap->nrows = pl->A.nrows;
  Ap->ncols = pl->A.ncols;
  Ap->nnz = pl->nnz_out;
  Ap->colidx_type = pl->A.colidx_type;
  Ap->value_type = pl->A.value_type;
  const bool owned = lib_allocates(Ap);
  SP_TRY(alloc_csr(ctx, Ap, s));
  const sp_csr& A = pl->A;
  const sp_status st_ = dispatch_i(A.rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(A.colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(A.value_type, [&](auto vt) {
        using VT = decltype(vt);
        return dispatch_i(pl->idx_type, [&](auto ix) {
          using IX = decltype(ix);
          return assign_fill_impl<RP, CI, VT, IX>(ctx, pl, Ap, s);
        });
      });
    });
  });
  return release_on_error(ctx, Ap, owned, s, st_);
}

extern "C" sp_status sp_assign(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                               const void* J, int64_t nJ, sp_itype idx_type, const sp_csr* B,
                               sp_assign_mode mode, sp_csr* Aprime, sp_stream_t stream) {
  if (!Aprime) return SP_ERR_INVALID_ARG;
  sp_plan* pl = nullptr;
  int64_t nnz = 0;
  SP_TRY(sp_assign_count(ctx, A, I, nI, J, nJ, idx_type, B, mode, &pl, &nnz, stream));
  sp_status st = sp_assign_fill(ctx, pl, Aprime, stream);
  plan_release(ctx, pl);
  return st;
}

extern "C" sp_status sp_assign_permute_fill(sp_ctx* ctx, sp_plan* pl, const void* p, const void* q,
                                            sp_csr* out, sp_stream_t stream) {
  if (!ctx || !pl || !out || pl->op != 1) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type != SP_I32 && out->rowptr_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type == SP_I32 && pl->nnz_out > INT32_MAX) return SP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, SP_OP_ASSIGN, pl->A.nnz);
  pl->stream = s;
  const sp_csr& A = pl->A;
  out->nrows = A.nrows;
  out->ncols = A.ncols;
  out->nnz = pl->nnz_out;
  out->colidx_type = A.colidx_type;
  out->value_type = A.value_type;
  const bool owned = lib_allocates(out);
  SP_TRY(alloc_csr(ctx, out, s));
  const sp_status st_ = dispatch_i(A.rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(A.colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(A.value_type, [&](auto vt) {
        using VT = decltype(vt);
        return dispatch_i(pl->idx_type, [&](auto ix) {
          using IX = decltype(ix);
          return assign_permute_impl<RP, CI, VT, IX>(ctx, pl, static_cast<const IX*>(p),
                                                     static_cast<const IX*>(q), out, s);
        });
      });
    });
  });
  return release_on_error(ctx, out, owned, s, st_);
}

extern "C" sp_status sp_assign_permute(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                                       const void* J, int64_t nJ, sp_itype idx_type, const sp_csr* B,
                                       sp_assign_mode mode, const void* p, const void* q, sp_csr* out,
                                       sp_stream_t stream) {
  if (!out) return SP_ERR_INVALID_ARG;
  sp_plan* pl = nullptr;
  int64_t nnz = 0;
  SP_TRY(sp_assign_count(ctx, A, I, nI, J, nJ, idx_type, B, mode, &pl, &nnz, stream));
  const sp_status st = sp_assign_permute_fill(ctx, pl, p, q, out, stream);
  plan_release(ctx, pl);
  return st;
}
