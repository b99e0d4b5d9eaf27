// Device-side building blocks shared by every kernel of the library: the device
// error record, integer helpers, warp/block scans and cache-hinted global loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sp.h"

namespace sp {

// First device-detected error wins; `detail` is the offending position (or -1).
struct DevStatus {
  int code;
  int pad;
  long long detail;
};

__device__ __forceinline__ void dev_fail(DevStatus* st, int code, long long detail) {
  if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

__host__ __device__ __forceinline__ int ceil_log2_u64(uint64_t x) {
  // smallest k with 2^k >= x (x >= 1)
#ifdef __CUDA_ARCH__
  return x <= 1 ? 0 : 64 - __clzll((long long)(x - 1));
#else
  int k = 0;
  while ((1ull << k) < x) ++k;
  return k;
#endif
}

__device__ __forceinline__ int ceil_log2_u32(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// ---- cache-hinted loads ------------------------------------------------------
// Streaming data (column indices and values read once) is loaded with an L1
// no-allocate hint so that the L1/L2 capacity stays with the index maps, which are
// read at random and reused.
template <class T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}
// Index-map lookups (random, reused) are tagged L2 evict-last through a cache policy,
// so the write-once output and streamed inputs (evict-first) leave the maps in L2.
__device__ __forceinline__ unsigned long long l2_keep_policy() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int ld_map(const int* p) {
  int v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;"
               : "=r"(v)
               : "l"(p), "l"(l2_keep_policy()));
  return v;
}
__device__ __forceinline__ long long ld_map(const long long* p) {
  long long v;
  asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;"
               : "=l"(v)
               : "l"(p), "l"(l2_keep_policy()));
  return v;
}
__device__ __forceinline__ long ld_map(const long* p) {
  return (long)ld_map(reinterpret_cast<const long long*>(p));
}
__device__ __forceinline__ unsigned ld_map(const unsigned* p) {
  unsigned v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;"
               : "=r"(v)
               : "l"(p), "l"(l2_keep_policy()));
  return v;
}
// Lookups into tables larger than L2 (read at random, rarely reused): plain read-only
// loads, so they do not displace the small tables that carry the evict-last hint.
template <class T>
__device__ __forceinline__ T ld_plain(const T* p) {
  return __ldg(p);
}
// Write-once output: store with the evict-first (streaming) hint.
template <class T>
__device__ __forceinline__ void st_stream(T* p, T v) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte words");
  if constexpr (sizeof(T) == 4) {
    unsigned u;
    memcpy(&u, &v, 4);
    __stcs(reinterpret_cast<unsigned*>(p), u);
  } else {
    unsigned long long u;
    memcpy(&u, &v, 8);
    __stcs(reinterpret_cast<unsigned long long*>(p), u);
  }
}

// Asynchronous global -> shared copy of one 8-byte word; commit closes the thread's
// group of copies, wait_all waits for all of the thread's groups.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
// 16-byte and single-word global -> shared copies (16-byte: both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_word(void* dst, const void* src) {
  static_assert(BYTES == 4 || BYTES == 8, "4- or 8-byte words");
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  if constexpr (BYTES == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---- relaxed 64-bit status words (decoupled look-back) -------------------------
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- warp / block scans ------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_incl_sum(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

template <class T>
__device__ __forceinline__ T warp_incl_max(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v = o > v ? o : v;
  }
  return v;
}

// Exclusive sum of one value per thread over the block; `tmp` holds BLOCK/32+1
// entries of T in shared memory.  Returns the exclusive prefix; *total = block sum.
template <int BLOCK, class T>
__device__ __forceinline__ T block_excl_sum(T v, T* tmp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = BLOCK / 32;
  T inc = warp_incl_sum(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NW ? tmp[lane] : T(0);
    T wi = warp_incl_sum(w);
    if (lane < NW) tmp[lane] = wi - w;
    if (lane == NW - 1) tmp[NW] = wi;
  }
  __syncthreads();
  T res = tmp[warp] + inc - v;
  *total = tmp[NW];
  __syncthreads();
  return res;
}

template <int BLOCK, class T>
__device__ __forceinline__ T block_incl_max(T v, T* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = BLOCK / 32;
  T inc = warp_incl_max(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NW ? tmp[lane] : T(0);
    T wi = warp_incl_max(w);
    // exclusive max of warp totals
    T ex = __shfl_up_sync(0xffffffffu, wi, 1);
    if (lane == 0) ex = T(0);
    if (lane < NW) tmp[lane] = ex;
  }
  __syncthreads();
  T pre = tmp[warp];
  T res = pre > inc ? pre : inc;
  __syncthreads();
  return res;
}

// In-place exclusive sum over a shared array a[0..n), n <= BLOCK*ITEMS.  Each thread
// owns ITEMS consecutive entries.  Returns the total.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ uint32_t smem_excl_sum(uint32_t* a, int n, uint32_t* tmp) {
  const int t = threadIdx.x;
  uint32_t v[ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    int x = t * ITEMS + j;
    v[j] = x < n ? a[x] : 0u;
    s += v[j];
  }
  uint32_t total;
  uint32_t run = block_excl_sum<BLOCK>(s, tmp, &total);
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    int x = t * ITEMS + j;
    if (x < n) a[x] = run;
    run += v[j];
  }
  __syncthreads();
  return total;
}

// In-place inclusive max over a shared array a[0..n), n <= BLOCK*ITEMS.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ void smem_incl_max(uint32_t* a, int n, uint32_t* tmp) {
  const int t = threadIdx.x;
  uint32_t v[ITEMS];
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    int x = t * ITEMS + j;
    v[j] = x < n ? a[x] : 0u;
    m = v[j] > m ? v[j] : m;
  }
  // exclusive max of thread maxima
  uint32_t incl = block_incl_max<BLOCK>(m, tmp);
  uint32_t prev = __shfl_up_sync(0xffffffffu, incl, 1);
  // the exclusive value of lane 0 of each warp comes from the previous warp's total;
  // recompute it through shared memory
  __shared__ uint32_t warp_last[BLOCK / 32];
  if ((t & 31) == 31) warp_last[t >> 5] = incl;
  __syncthreads();
  if ((t & 31) == 0) prev = (t >> 5) ? warp_last[(t >> 5) - 1] : 0u;
  uint32_t run = prev;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    int x = t * ITEMS + j;
    run = v[j] > run ? v[j] : run;
    if (x < n) a[x] = run;
  }
  __syncthreads();
}

// In-place inclusive max over a shared array of 16-bit values a[0..n), n <= BLOCK*ITEMS.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ void smem_incl_max16(uint16_t* a, int n, uint32_t* tmp) {
  const int t = threadIdx.x;
  uint32_t v[ITEMS];
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int x = t * ITEMS + j;
    v[j] = x < n ? a[x] : 0u;
    m = v[j] > m ? v[j] : m;
  }
  const uint32_t incl = block_incl_max<BLOCK>(m, tmp);
  uint32_t prev = __shfl_up_sync(0xffffffffu, incl, 1);
  __shared__ uint32_t warp_last16[BLOCK / 32];
  if ((t & 31) == 31) warp_last16[t >> 5] = incl;
  __syncthreads();
  if ((t & 31) == 0) prev = (t >> 5) ? warp_last16[(t >> 5) - 1] : 0u;
  uint32_t run = prev;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int x = t * ITEMS + j;
    run = v[j] > run ? v[j] : run;
    if (x < n) a[x] = uint16_t(run);
  }
  __syncthreads();
}

}  // namespace sp
