// Index maps, per-row counting passes, the tile partition and the load-balanced row
// gather.  Every kernel that dereferences an index taken from user data checks it
// first: a bad index is reported through the device error record and never read.
#pragma once

#include "pipeline.cuh"

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

// membership bitmap (1 bit per index); repeated indices are reported
template <class IX>
__global__ void k_mark_bits(const IX* __restrict__ idx, long long len, long long n,
                            uint32_t* __restrict__ bits, DevStatus* st, int dup_code) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x) {
    const long long v = (long long)idx[k];
    if (v < 0 || v >= n) {
      dev_fail(st, SP_ERR_INDEX_RANGE, k);
      continue;
    }
    const uint32_t m = 1u << (v & 31);
    const uint32_t old = atomicOr(bits + (v >> 5), m);
    if (old & m) dev_fail(st, dup_code, k);
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
// A row is "source-long" when its source holds more than TILE_CP entries: it is
// counted by k_count_long (one CTA per row) and listed for k_long / k_huge.
struct CountLists {
  long long* cl_rows;  // source-long rows waiting for k_count_long
  unsigned* n_cl;
  long long cl_cap;
  long long* long_rows;
  unsigned* n_long;
  long long long_cap;
  long long* huge_rows;
  unsigned* n_huge;
  long long huge_cap;
};

__device__ __forceinline__ void push_row(long long* list, unsigned* n, long long cap, long long r,
                                         DevStatus* st) {
  const unsigned q = atomicAdd(n, 1u);
  if (q < cap) list[q] = r;
  else dev_fail(st, SP_ERR_INTERNAL, -12);
}

// Count kernels take a loader (see segsort.cuh) and count the entries its map keeps.
// Short rows: one warp handles COUNT_RB rows per step, reading the first 32 entries of
// all of them in one batch (ballot + popc per row); the rest of longer rows follows
// in batches of LOAD_U x 32.  Source-long rows (> TILE_CP entries) are listed for
// k_count_long (one CTA per row) and later handled by k_long / k_huge.
constexpr int COUNT_RB = 4;

template <class Ct>
__global__ void k_count_warp(Ct ct, long long nlisted, long long* __restrict__ counts,
                             CountLists cl, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const CountOnly<Ct> ko{ct};
  for (long long i0 = w0 * COUNT_RB; i0 < nlisted; i0 += nw * COUNT_RB) {
    RowSrc rs[COUNT_RB];
    long long Ls[COUNT_RB], cnt[COUNT_RB];
    bool lng[COUNT_RB];
    Batch<CountOnly<Ct>, COUNT_RB> bt;
#pragma unroll
    for (int u = 0; u < COUNT_RB; ++u) {
      const long long i = i0 + u;
      rs[u] = i < nlisted ? ct.row(i) : RowSrc{0, 0, 0, 0};
      Ls[u] = rs[u].n0 + rs[u].n1;
      lng[u] = Ls[u] > TILE_CP;
      bt.valid[u] = !lng[u] && lane < Ls[u];
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
        if (i >= nlisted) break;
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
      if (t == 0) {
        counts[i] = v;
        if (v <= LONG_CAP) push_row(cl.long_rows, cl.n_long, cl.long_cap, i, st);
        else push_row(cl.huge_rows, cl.n_huge, cl.huge_cap, i, st);
      }
    }
    __syncthreads();
  }
}

// ---- load-balanced row gather -------------------------------------------------------
// out[vp[r] + k] = source element (which, off(r) + k) for k < vp[r+1]-vp[r]; each CTA
// owns GATHER_CH consecutive output positions, so long and short rows cost the same.
// Gs: __device__ void src(long long r, int& which, long long& off) const;
//     __device__ void get(int which, long long pos, CI& c, VT& v) const;
constexpr int GATHER_BLOCK = 512, GATHER_CH = 8192;

template <class Gs>
__global__ void __launch_bounds__(GATHER_BLOCK) k_gather_rows(Gs gs, const long long* __restrict__ vp,
                                                              long long nrows, long long total,
                                                              typename Gs::CI* __restrict__ out_col,
                                                              typename Gs::VT* __restrict__ out_val) {
  using CI = typename Gs::CI;
  using VT = typename Gs::VT;
  constexpr int B = GATHER_BLOCK, ITEMS = GATHER_CH / B;
  __shared__ uint32_t owner[GATHER_CH];
  __shared__ long long r_off[B];
  __shared__ long long r_o0[B];
  __shared__ long long r_o1[B];
  __shared__ int r_which[B];
  __shared__ uint32_t tmp32[B / 32 + 1];
  __shared__ long long s_first;
  const int t = threadIdx.x;
  const long long c0 = blockIdx.x * (long long)GATHER_CH;
  if (c0 >= total) return;
  const long long c1 = c0 + GATHER_CH < total ? c0 + GATHER_CH : total;
  if (t == 0) {  // last row with vp[r] <= c0
    long long lo = 0, hi = nrows;
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (vp[mid] <= c0) lo = mid;
      else hi = mid;
    }
    s_first = lo;
  }
  __syncthreads();
  for (long long rb = s_first;; rb += B) {
    const long long r = rb + t;
    long long o0 = total, o1 = total;
    if (r < nrows) {
      o0 = vp[r];
      o1 = vp[r + 1];
    }
    const bool active = r < nrows && o1 > o0 && o1 > c0 && o0 < c1;
    if (active) {
      int which;
      long long off;
      gs.src(r, which, off);
      r_which[t] = which;
      r_off[t] = off;
      r_o0[t] = o0;
      r_o1[t] = o1;
    }
    for (int j = 0; j < ITEMS; ++j) owner[t + j * B] = 0xFFFFFFFFu;
    __syncthreads();
    if (active) {
      const long long p = o0 > c0 ? o0 : c0;
      owner[p - c0] = uint32_t(t);
    }
    __syncthreads();
    // inclusive max-scan where "unset" (0xFFFFFFFF) is treated as -inf
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int x = t * ITEMS + j;
      if (owner[x] == 0xFFFFFFFFu) owner[x] = 0;
      else owner[x] += 1;
    }
    __syncthreads();
    smem_incl_max<B, ITEMS>(owner, GATHER_CH, tmp32);
    // all loads first, then all stores: the stores may not be moved above later loads
    // (the compiler cannot rule out aliasing), so interleaving would serialise them
    constexpr int H = 8;
#pragma unroll
    for (int h = 0; h < ITEMS; h += H) {
      CI c[H];
      VT v[H];
      bool ok[H];
#pragma unroll
      for (int u = 0; u < H; ++u) {
        const int x = t + (h + u) * B;
        const long long g = c0 + x;
        const uint32_t ow = owner[x];
        ok[u] = false;
        if (g < c1 && ow > 0) {
          const int k = int(ow) - 1;
          const long long o = r_o0[k];
          // positions beyond the chunk's rows belong to the next chunk of rows
          if (g >= o && g < r_o1[k]) {
            ok[u] = true;
            gs.get(r_which[k], r_off[k] + (g - o), c[u], v[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < H; ++u) {
        if (!ok[u]) continue;
        const long long g = c0 + t + (h + u) * B;
        st_stream(out_col + g, c[u]);
        st_stream(out_val + g, v[u]);
      }
    }
    __syncthreads();
    // stop once the chunk's last row reaches the end of this CTA's positions
    const long long rl = rb + B - 1;
    if (rl >= nrows - 1 || vp[rl + 1] >= c1) break;
  }
}

}  // namespace sp
