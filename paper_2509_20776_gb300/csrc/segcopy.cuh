// Segment copy: an output assembled from contiguous pieces of one or two source arrays
// (the unchanged-row runs of an assignment, Sec. 2.3 / Algorithm 4's Add step, where rows
// outside I are A's rows verbatim).  Each segment j covers output positions
// [segs[j].dst, segs[j+1].dst) and reads consecutive positions from segs[j].src on (bit 62
// of src selects the second array).  The copy moves 16-byte words: every group of four
// output positions starting at a multiple of four is stored as 16 bytes (two words for
// 8-byte elements); its source is loaded as whole 16-byte words and realigned in
// registers when source and destination differ in alignment.  Groups that cross a
// segment boundary, touch an array's last words, or belong to unaligned arrays are copied
// element by element.  A segment whose src is kSegSkip is left alone: its positions are
// written by another kernel (which may run at the same time, so no 16-byte store of the
// copy ever covers one of them).
#pragma once

#include "common.cuh"

namespace sp {

struct CopySeg {
  long long dst;  // first output position
  long long src;  // first source position; bit 62: the second array
};
constexpr long long kSegB = 1ll << 62;
constexpr long long kSegSkip = 1ll << 61;  // src of a segment another kernel writes: not copied
constexpr int SC_CH = 8192;        // output positions per chunk (a multiple of four)
constexpr int SC_BLOCK = 256;
constexpr int SC_SEGS = SC_BLOCK;  // segment descriptors staged in shared memory at once
constexpr int SC_MINB = 8;          // persistent grid: CTAs per SM
constexpr int SC_MINB_OVERLAP = 4;  // the same while another kernel shares the SMs

// Four consecutive elements of T starting at element s of src (n elements), realigned
// from whole 16-byte words; false when those words would leave [0, n) (caller copies the
// elements one by one).
template <class T>
__device__ __forceinline__ bool load4(const T* __restrict__ src, long long n, long long s, uint4* w);

template <>
__device__ __forceinline__ bool load4<uint32_t>(const uint32_t* __restrict__ src, long long n, long long s, uint4* w) {
  const long long f = s & ~3ll;
  const int k = int(s - f);
  if (k == 0) {
    if (f + 4 > n) return false;
    w[0] = __ldcs(reinterpret_cast<const uint4*>(src + f));
    return true;
  }
  if (f + 8 > n) return false;
  const uint4 a = __ldcs(reinterpret_cast<const uint4*>(src + f));
  const uint4 b = __ldcs(reinterpret_cast<const uint4*>(src + f + 4));
  w[0] = k == 1 ? make_uint4(a.y, a.z, a.w, b.x) : k == 2 ? make_uint4(a.z, a.w, b.x, b.y)
                                                           : make_uint4(a.w, b.x, b.y, b.z);
  return true;
}

template <>
__device__ __forceinline__ bool load4<unsigned long long>(const unsigned long long* __restrict__ src, long long n,
                                                         long long s, uint4* w) {
  const long long f = s & ~1ll;
  if (s == f) {
    if (f + 4 > n) return false;
    w[0] = __ldcs(reinterpret_cast<const uint4*>(src + f));
    w[1] = __ldcs(reinterpret_cast<const uint4*>(src + f + 2));
    return true;
  }
  if (f + 6 > n) return false;
  const uint4 a = __ldcs(reinterpret_cast<const uint4*>(src + f));
  const uint4 b = __ldcs(reinterpret_cast<const uint4*>(src + f + 2));
  const uint4 c = __ldcs(reinterpret_cast<const uint4*>(src + f + 4));
  w[0] = make_uint4(a.z, a.w, b.x, b.y);
  w[1] = make_uint4(b.z, b.w, c.x, c.y);
  return true;
}

template <class T>
__device__ __forceinline__ void store4(T* dst, const uint4* w) {
  __stcs(reinterpret_cast<uint4*>(dst), w[0]);
  if constexpr (sizeof(T) == 8) __stcs(reinterpret_cast<uint4*>(dst) + 1, w[1]);
}

// chunk_first[k] = the segment holding output position k * SC_CH (segments sorted by dst,
// segs[nseg].dst = total; nseg read from the device)
__global__ void k_seg_chunks(const CopySeg* __restrict__ segs, const long long* __restrict__ nseg_p,
                             long long nchunks, long long* __restrict__ chunk_first) {
  const long long nseg = *nseg_p;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nseg;
       j += (long long)gridDim.x * blockDim.x) {
    const long long d = segs[j].dst, dn = segs[j + 1].dst;
    if (dn <= d) continue;
    long long k1 = (dn + SC_CH - 1) / SC_CH;
    if (k1 > nchunks) k1 = nchunks;
    for (long long k = (d + SC_CH - 1) / SC_CH; k < k1; ++k) chunk_first[k] = j;
  }
}

// CI / VT: column / value words (uint32 or unsigned long long views of the arrays).
// vec: every array base is 16-byte aligned (else element by element throughout).
template <class CI, class VT>
__global__ void __launch_bounds__(SC_BLOCK) k_seg_copy(const CopySeg* __restrict__ segs,
                                                       const long long* __restrict__ nseg_p, long long total, const long long* __restrict__ chunk_first,
                                                       long long nchunks, const CI* __restrict__ ca,
                                                       const VT* __restrict__ va, long long na,
                                                       const CI* __restrict__ cb, const VT* __restrict__ vb,
                                                       long long nb, CI* __restrict__ out_col,
                                                       VT* __restrict__ out_val, int vec, DevStatus* st) {
  __shared__ long long s_dst[SC_SEGS + 1];
  __shared__ long long s_src[SC_SEGS];
  __shared__ int s_n;
  const int t = threadIdx.x;
  const long long nseg = *nseg_p;
  for (long long k = blockIdx.x; k < nchunks; k += gridDim.x) {
    const long long c0 = k * SC_CH, c1 = c0 + SC_CH < total ? c0 + SC_CH : total;
    long long j0 = chunk_first[k];
    if (j0 < 0 || j0 >= nseg) {  // cannot happen for a consistent segment list
      if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -34);
      continue;
    }
    long long p0 = c0;  // first position not yet copied
    while (p0 < c1) {
      // stage the next batch of segments: those starting before c1
      __syncthreads();
      if (t == 0) s_n = 0;
      __syncthreads();
      for (int x = t; x < SC_SEGS; x += SC_BLOCK) {
        const long long j = j0 + x;
        if (j < nseg && segs[j].dst < c1) {
          s_dst[x] = segs[j].dst;
          s_src[x] = segs[j].src;
          atomicMax(&s_n, x + 1);
        }
      }
      __syncthreads();
      const int ns = s_n;
      if (ns == 0) {  // cannot happen for a consistent segment list
        if (t == 0) dev_fail(st, SP_ERR_INTERNAL, -31);
        break;
      }
      // end of the staged segments' coverage
      long long p1 = j0 + ns < nseg ? segs[j0 + ns].dst : total;
      if (p1 > c1) p1 = c1;
      if (t == 0) s_dst[ns] = p1;
      __syncthreads();
      // groups of four output positions in [p0, p1)
      const long long g0 = p0 & ~3ll;
      for (long long g = g0 + 4ll * t; g < p1; g += 4ll * SC_BLOCK) {
        // segment of position g (the last staged segment with dst <= g)
        int lo = 0, hi = ns - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_dst[mid] <= g) lo = mid;
          else hi = mid - 1;
        }
        const long long send = s_dst[lo + 1];
        if (s_src[lo] == kSegSkip && g >= p0 && g >= s_dst[lo] && g + 4 <= send) continue;
        const bool whole = vec && g >= p0 && g >= s_dst[lo] && g + 4 <= send;
        if (whole) {
          const long long sp = s_src[lo];
          const bool second = (sp & kSegB) != 0;
          const long long s = (sp & ~kSegB) + (g - s_dst[lo]);
          uint4 wc[2], wv[2];
          const bool ok = second ? (load4<CI>(cb, nb, s, wc) && load4<VT>(vb, nb, s, wv))
                                 : (load4<CI>(ca, na, s, wc) && load4<VT>(va, na, s, wv));
          if (ok) {
            store4<CI>(out_col + g, wc);
            store4<VT>(out_val + g, wv);
            continue;
          }
        }
        // element by element: positions of the group inside [p0, p1)
        int sj = lo;
        for (int e = 0; e < 4; ++e) {
          const long long q = g + e;
          if (q < p0 || q >= p1) continue;
          while (sj + 1 < ns && s_dst[sj + 1] <= q) ++sj;
          const long long sp = s_src[sj];
          if (sp == kSegSkip) continue;
          const long long s = (sp & ~kSegB) + (q - s_dst[sj]);
          if (sp & kSegB) {
            if (s >= 0 && s < nb) {
              out_col[q] = cb[s];
              out_val[q] = vb[s];
            } else {
              dev_fail(st, SP_ERR_INTERNAL, -32);
            }
          } else if (s >= 0 && s < na) {
            out_col[q] = ca[s];
            out_val[q] = va[s];
          } else {
            dev_fail(st, SP_ERR_INTERNAL, -32);
          }
        }
      }
      // a full batch ends where the next segment starts: continue from it
      p0 = p1;
      j0 += ns;
    }
  }
}

}  // namespace sp
