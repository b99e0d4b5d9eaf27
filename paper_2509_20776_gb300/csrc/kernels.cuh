// Index maps and the per-row count and fill passes.  Every kernel that dereferences an
// index taken from user data checks it first: a bad index is reported through the
// device error record and never read.
#pragma once

#include "loaders.cuh"
#include "scan.cuh"

namespace sp {

// ---- inverse maps (Identify step: pvec[pvec_inv[i]] = i, -1 for absent) ---------
template <class IX>
__global__ void k_inverse_map(const IX* __restrict__ idx, long long len, long long n,
                              IX* __restrict__ inv, DevStatus* st, int dup_code) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x) {
    const long long v = (long long)idx[k];
    if (v < 0 || v >= n) {
      dev_fail(st, SP_ERR_INDEX_RANGE, k);
      continue;
    }
    if (sizeof(IX) == 4) {
      const int old = atomicCAS(reinterpret_cast<int*>(inv) + v, -1, int(k));
      if (old != -1) dev_fail(st, dup_code, k);
    } else {
      const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(inv) + v,
                                               ~0ull, (unsigned long long)k);
      if (old != ~0ull) dev_fail(st, dup_code, k);
    }
  }
}

// The same map with a membership bitmap beside it: a repeated index is found by the
// bitmap's atomicOr (1 bit per value, small enough to stay in L2) and the map takes one
// plain store per index instead of a compare-and-swap on an entry of the n-entry map.
// The first index to set a value's bit writes its position; a later repeat only reports
// dup_code.  inv (-1) and bits (0) are cleared before the launch; afterwards bits is J's,
// I's or q's membership bitmap.
template <class IX>
__global__ void k_inverse_map_bits(const IX* __restrict__ idx, long long len, long long n,
                                   IX* __restrict__ inv, uint32_t* __restrict__ bits, DevStatus* st,
                                   int dup_code) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x) {
    const long long v = (long long)idx[k];
    if (v < 0 || v >= n) {
      dev_fail(st, SP_ERR_INDEX_RANGE, k);
      continue;
    }
    const uint32_t m = 1u << (v & 31);
    if (atomicOr(bits + (v >> 5), m) & m) {
      dev_fail(st, dup_code, k);
      continue;
    }
    inv[v] = IX(k);
  }
}

// membership bitmap (1 bit per index); repeated indices are reported as dup_code, or
// only flagged in *dup_flag when one is given
template <class IX>
__global__ void k_mark_bits(const IX* __restrict__ idx, long long len, long long n,
                            uint32_t* __restrict__ bits, DevStatus* st, int dup_code,
                            int* dup_flag = nullptr) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x) {
    const long long v = (long long)idx[k];
    if (v < 0 || v >= n) {
      dev_fail(st, SP_ERR_INDEX_RANGE, k);
      continue;
    }
    const uint32_t m = 1u << (v & 31);
    const uint32_t old = atomicOr(bits + (v >> 5), m);
    if (old & m) {
      if (dup_flag) *dup_flag = 1;  // repeats are allowed here: only flagged
      else dev_fail(st, dup_code, k);
    }
  }
}

template <class IX>
__global__ void k_range_check(const IX* __restrict__ idx, long long len, long long n, DevStatus* st) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x) {
    const long long v = (long long)idx[k];
    if (v < 0 || v >= n) dev_fail(st, SP_ERR_INDEX_RANGE, k);
  }
}

// Shape of an index vector: flags[0] = 1 unless strictly ascending, flags[1] = 1 unless
// consecutive (idx[k+1] = idx[k] + 1 for all k); the flags are zeroed before the launch.
template <class IX>
__global__ void k_index_shape(const IX* __restrict__ idx, long long len, int* flags) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k + 1 < len;
       k += (long long)gridDim.x * blockDim.x) {
    const long long a = (long long)idx[k], b = (long long)idx[k + 1];
    if (b <= a) flags[0] = 1;
    if (b != a + 1) flags[1] = 1;
  }
}

constexpr long long J_KEY_LIMIT = 1ll << 32;  // new column ids must fit 32-bit sort keys

template <int kDummy = 0>
__global__ void k_diff(const long long* __restrict__ vp, long long n, long long* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = vp[i + 1] - vp[i];
}

template <class T>
__global__ void k_widen(const T* __restrict__ in, long long n, long long* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (long long)in[i];
}
template <class T>
__global__ void k_narrow(const long long* __restrict__ in, long long n, T* __restrict__ out,
                         DevStatus* st) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long v = in[i];
    if (sizeof(T) == 4 && v > 0x7fffffffll) dev_fail(st, SP_ERR_OVERFLOW, i);
    out[i] = T(v);
  }
}

// ---- counting passes (Alg. 5 first pass, restated as a ballot/popc per warp) ------
// A row is "source-long" when its source holds more than SRC_LONG entries: it is
// counted and filled by one CTA (k_count_long, k_fill_long) instead of a warp.
struct CountLists {
  long long* cl_rows;  // source-long rows waiting for k_count_long
  unsigned* n_cl;
  long long cl_cap;
  long long* rs0 = nullptr;  // when given: source start and length of every listed row
  long long* rsn = nullptr;  //   (single-run loaders), for a fill that reads them back
};

__device__ __forceinline__ void push_row(long long* list, unsigned* n, long long cap, long long r,
                                         DevStatus* st) {
  const unsigned q = atomicAdd(n, 1u);
  if (q < cap) list[q] = r;
  else dev_fail(st, SP_ERR_INTERNAL, -12);
}

// Count kernels take a loader (see loaders.cuh) and count the entries its map keeps.
// Short rows: one warp handles COUNT_RB rows per step, reading the first 32 entries of
// all of them in one batch (ballot + popc per row); the rest of longer rows follows
// in batches of LOAD_U x 32.  Source-long rows (> SRC_LONG entries) are listed for
// k_count_long (one CTA per row).
constexpr int COUNT_RB = 4;

// rb (1 to COUNT_RB) rows per warp step: a run-time kernel shape.
template <class Ct>
__global__ void k_count_warp(Ct ct, long long nlisted, long long* __restrict__ counts,
                             CountLists cl, int rb, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const CountOnly<Ct> ko{ct};
  for (long long i0 = w0 * rb; i0 < nlisted; i0 += nw * rb) {
    RowSrc rs[COUNT_RB];
    long long Ls[COUNT_RB], cnt[COUNT_RB];
    bool lng[COUNT_RB];
    Batch<CountOnly<Ct>, COUNT_RB> bt;
#pragma unroll
    for (int u = 0; u < COUNT_RB; ++u) {
      const long long i = i0 + u;
      const bool mine = u < rb && i < nlisted;
      rs[u] = mine ? ct.row(i) : RowSrc{0, 0, 0, 0};
      if (cl.rs0 && lane == 0 && mine) {
        cl.rs0[i] = rs[u].s0;
        cl.rsn[i] = rs[u].n0;
      }
      Ls[u] = rs[u].n0 + rs[u].n1;
      lng[u] = row_is_long<Ct>(rs[u]);
      bt.valid[u] = !lng[u] && lane < Ls[u];
      bt.set_row(u, i);
      if (bt.valid[u]) bt.at(u, rs[u], lane);
    }
    bt.run(ko);
#pragma unroll
    for (int u = 0; u < COUNT_RB; ++u) cnt[u] = __popc(__ballot_sync(0xffffffffu, bt.kept[u]));
#pragma unroll
    for (int u = 0; u < COUNT_RB; ++u) {
      if (lng[u] || Ls[u] <= 32) continue;
      for (long long e0 = 32; e0 < Ls[u]; e0 += 32 * LOAD_U) {
        Batch<CountOnly<Ct>, LOAD_U> b2;
#pragma unroll
        for (int v = 0; v < LOAD_U; ++v) {
          const long long e = e0 + v * 32 + lane;
          b2.valid[v] = e < Ls[u];
          b2.set_row(v, i0 + u);
          if (b2.valid[v]) b2.at(v, rs[u], e);
        }
        b2.run(ko);
#pragma unroll
        for (int v = 0; v < LOAD_U; ++v) cnt[u] += __popc(__ballot_sync(0xffffffffu, b2.kept[v]));
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < COUNT_RB; ++u) {
        const long long i = i0 + u;
        if (u >= rb || i >= nlisted) break;
        if (lng[u]) push_row(cl.cl_rows, cl.n_cl, cl.cl_cap, i, st);
        else counts[i] = cnt[u];
      }
    }
  }
}

template <class Ct>
__global__ void __launch_bounds__(1024) k_count_long(Ct ct, long long* __restrict__ counts, CountLists cl,
                                                     unsigned* ticket, DevStatus* st) {
  __shared__ unsigned s_item;
  __shared__ long long red[33];
  const int t = threadIdx.x;
  const CountOnly<Ct> ko{ct};
  unsigned count = *cl.n_cl;
  if (count > cl.cl_cap) count = unsigned(cl.cl_cap);
  for (;;) {
    if (t == 0) s_item = atomicAdd(ticket, 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= count) break;
    const long long i = cl.cl_rows[item];
    const RowSrc rs = ct.row(i);
    const long long Ls = rs.n0 + rs.n1;
    long long c = 0;
    for (long long e0 = 0; e0 < Ls; e0 += (long long)blockDim.x * LOAD_U) {
      Batch<CountOnly<Ct>, LOAD_U> bt;
#pragma unroll
      for (int u = 0; u < LOAD_U; ++u) {
        const long long e = e0 + (long long)u * blockDim.x + t;
        bt.valid[u] = e < Ls;
        bt.set_row(u, i);
        if (bt.valid[u]) bt.at(u, rs, e);
      }
      bt.run(ko);
#pragma unroll
      for (int u = 0; u < LOAD_U; ++u) c += bt.kept[u];
    }
    c = warp_sum(c);
    if ((t & 31) == 0) red[t >> 5] = c;
    __syncthreads();
    if (t < 32) {
      long long v = t < int(blockDim.x >> 5) ? red[t] : 0;
      v = warp_sum(v);
      if (t == 0) counts[i] = v;
    }
    __syncthreads();
  }
}

// ---- fill passes (Alg. 5 second pass) --------------------------------------------------
// The kept entries of listed row i, relabelled, are written to [vp[i], vp[i+1]) of
// (out_col, out_val) in source order (the row sort then orders them by new column): a warp ballot
// over 32 entries gives each kept entry its slot.  Short rows as in k_count_warp (FILL_RB
// rows per warp step); source-long rows (cl_rows) one CTA each.  Both keep the source
// order within a row, so a monotone relabelling needs no sort afterwards.  A slot past
// the row's end (counts that do not match the fill) is reported
// and not written.
template <class Ld>
__device__ __forceinline__ void fill_put(const Ld&, typename Ld::CI* out_col, typename Ld::VT* out_val,
                                         long long pos, long long end, uint32_t key,
                                         const typename Ld::VT& v, DevStatus* st) {
  if (pos < end) {
    st_stream(out_col + pos, typename Ld::CI(key));
    st_stream(out_val + pos, v);
  } else {
    dev_fail(st, SP_ERR_INTERNAL, -23);
  }
}

constexpr int FILL_RB = 2;  // rows per warp step of the fill (fewer than counting: values)

// rb (1 to FILL_RB) rows per warp step: a run-time kernel shape.
template <class Ld>
__global__ void __launch_bounds__(256, 4) k_fill_warp(Ld ld, long long nlisted, const long long* __restrict__ vp,
                            typename Ld::CI* __restrict__ out_col, typename Ld::VT* __restrict__ out_val,
                            int rb, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i0 = w0 * rb; i0 < nlisted; i0 += nw * rb) {
    RowSrc rs[FILL_RB];
    long long Ls[FILL_RB], o[FILL_RB], oe[FILL_RB];
    bool lng[FILL_RB];
    Batch<Ld, FILL_RB> bt;
#pragma unroll
    for (int u = 0; u < FILL_RB; ++u) {
      const long long i = i0 + u;
      const bool mine = u < rb && i < nlisted;
      rs[u] = mine ? ld.row(i) : RowSrc{0, 0, 0, 0};
      o[u] = mine ? vp[i] : 0;
      oe[u] = mine ? vp[i + 1] : 0;
      Ls[u] = rs[u].n0 + rs[u].n1;
      lng[u] = row_is_long<Ld>(rs[u]);
      bt.valid[u] = !lng[u] && lane < Ls[u];
      bt.set_row(u, i);
      if (bt.valid[u]) bt.at(u, rs[u], lane);
    }
    bt.run(ld);
#pragma unroll
    for (int u = 0; u < FILL_RB; ++u) {
      const unsigned m = __ballot_sync(0xffffffffu, bt.kept[u]);
      if (bt.kept[u]) fill_put(ld, out_col, out_val, o[u] + __popc(m & lt), oe[u], bt.key[u], bt.v[u], st);
      o[u] += __popc(m);
    }
#pragma unroll
    for (int u = 0; u < FILL_RB; ++u) {
      if (lng[u] || Ls[u] <= 32) continue;
      for (long long e0 = 32; e0 < Ls[u]; e0 += 32 * LOAD_U) {
        Batch<Ld, LOAD_U> b2;
#pragma unroll
        for (int v = 0; v < LOAD_U; ++v) {
          const long long e = e0 + v * 32 + lane;
          b2.valid[v] = e < Ls[u];
          b2.set_row(v, i0 + u);
          if (b2.valid[v]) b2.at(v, rs[u], e);
        }
        b2.run(ld);
#pragma unroll
        for (int v = 0; v < LOAD_U; ++v) {
          const unsigned m = __ballot_sync(0xffffffffu, b2.kept[v]);
          if (b2.kept[v]) fill_put(ld, out_col, out_val, o[u] + __popc(m & lt), oe[u], b2.key[v], b2.v[v], st);
          o[u] += __popc(m);
        }
      }
    }
  }
}

template <class Ld>
__global__ void __launch_bounds__(1024) k_fill_long(Ld ld, const long long* __restrict__ cl_rows,
                                                    const unsigned* __restrict__ n_cl, long long cl_cap,
                                                    const long long* __restrict__ vp, unsigned* ticket,
                                                    typename Ld::CI* __restrict__ out_col,
                                                    typename Ld::VT* __restrict__ out_val, DevStatus* st) {
  constexpr int NW = 1024 / 32;
  __shared__ unsigned s_item;
  __shared__ unsigned s_wc[NW], s_wx[NW], s_tot;
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
    __syncthreads();
    const unsigned item = s_item;
    if (item >= count) break;
    const long long i = cl_rows[item];
    const RowSrc rs = ld.row(i);
    const long long Ls = rs.n0 + rs.n1, o = vp[i], oe = vp[i + 1];
    for (long long e0 = 0; e0 < Ls; e0 += (long long)blockDim.x * LOAD_U) {
      Batch<Ld, LOAD_U> bt;
#pragma unroll
      for (int u = 0; u < LOAD_U; ++u) {
        const long long e = e0 + (long long)u * blockDim.x + t;
        bt.valid[u] = e < Ls;
        bt.set_row(u, i);
        if (bt.valid[u]) bt.at(u, rs, e);
      }
      bt.run(ld);
      // slots in source order: warp counts, scanned across the block, slice by slice
#pragma unroll
      for (int u = 0; u < LOAD_U; ++u) {
        const unsigned m = __ballot_sync(0xffffffffu, bt.kept[u]);
        if (lane == 0) s_wc[w] = __popc(m);
        __syncthreads();
        if (w == 0) {
          const unsigned v = s_wc[lane];
          const unsigned inc = warp_incl_sum(v);
          s_wx[lane] = inc - v;
          if (lane == NW - 1) s_tot = inc;
        }
        __syncthreads();
        if (bt.kept[u])
          fill_put(ld, out_col, out_val, o + s_base + s_wx[w] + __popc(m & lt), oe, bt.key[u], bt.v[u], st);
        __syncthreads();
        if (t == 0) s_base += s_tot;
      }
    }
    __syncthreads();
  }
}

}  // namespace sp
