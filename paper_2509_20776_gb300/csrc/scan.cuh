// The single-pass exclusive scan that turns per-row counts into row pointers (the
// proc_pointer of Algorithm 2), shared by every operation and exposed on its own.
#pragma once

#include "internal.h"

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
__global__ void __launch_bounds__(SCAN_BLOCK, 5) k_scan(Load load, Store store, ScanCtl c) {
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

template <class K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  // set before every launch that needs it: a flag kept in an inline template is shared by
  // every translation unit of the library, but each one launches its own copy of a kernel
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

}  // namespace sp
