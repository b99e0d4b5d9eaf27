// Batched extraction: B_k = A_{m_k}(I_k, J_k) for thousands of small requests in a fixed
// number of launches over the whole batch (the batching pattern of the serving path).
//
// Identification, per request, by one of (SP_OPT_IDENTIFY):
//   0 (default) a rank map per request: the request's slice of one batch-wide array of
//     64-bit words, one per 32 columns of its matrix (membership bits | members before the
//     word, counted over the whole batch), and the members' positions in J stored in that
//     global rank order; a stored column is tested and relabelled with two lookups.  The
//     slices take ncols/32 words per request; a batch whose slices would exceed
//     kBatchMapBytes falls back to
//   1 each request's J sorted once (positions carried as values), a stored column looked
//     up by binary search in it: the per-(i, j) search of Algorithm 5.
// Every step runs once for the batch: identify (bitmaps, scan, positions; or J gather,
// segmented sort, duplicate check) -> per-row kept counts -> scan -> fill -> segmented
// sort of the output rows.
// The count call synchronises once (the batch's output size); the fill call allocates
// nothing and never synchronises, so it can be captured in a CUDA graph and replayed.
#include <vector>

#include "dispatch.h"
#include "extract_rows.cuh"
#include "kernels.cuh"
#include "rowsort.cuh"

namespace sp {

struct BatchMat {  // a matrix of the batch (device arrays)
  const void* rowptr;
  const void* colidx;
  const void* values;
  long long nrows, ncols, nnz;
};

struct BatchReq {  // a request, with its offsets in the batch's J, output rows and map words
  long long mat, nI, nJ;
  const void* I;
  const void* J;
  long long roff, joff;
  long long moff;  // first word of the request's rank-map slice (identify 0)
};

constexpr long long kBatchMapBytes = 16ll << 30;  // largest rank map a batch builds

// What a batched row needs from its request: the matrix's arrays and the request's
// rank-map slice (built on the host, one per request).
struct ReqView {
  const void* col;
  const void* val;
  const unsigned long long* meta;  // the request's slice of the batch's rank words
  long long ncol;
};


}  // namespace sp

struct sp_batch {
  long long nreq = 0, nmats = 0, rows = 0, jtot = 0, nnz = 0, max_nj = 0;
  sp_itype idx_type = SP_I32, rowptr_type = SP_I64, colidx_type = SP_I32;
  sp_vtype value_type = SP_F32;
  int key_bits = 0;
  std::vector<long long> roff;  // host copy: first output row of every request (+ total)
  char* buf = nullptr;          // device: tables, sorted J, row pointer, scan workspace
  size_t buf_bytes = 0;
  sp::BatchMat* mats = nullptr;
  sp::BatchReq* reqs = nullptr;
  long long* droff = nullptr;   // nreq + 1
  long long* djoff = nullptr;   // nreq + 1
  void* jkey = nullptr;         // jtot entries of idx_type: every J, sorted per request
  uint32_t* jpos = nullptr;     // jtot: position of each sorted J entry in its request
  int identify = 1;             // 0: rank map, 1: sorted J
  long long nwords = 0;         // rank-map words of the whole batch
  uint32_t* jbits = nullptr;    // nwords membership words
  unsigned long long* jmeta = nullptr;  // nwords: bits | members before the word (batch-wide)
  uint32_t* jrp = nullptr;      // jtot: position in its request's J, in batch-wide rank order
  long long* rs0 = nullptr;     // rank map: source start, length and request of every output row
  long long* rsn = nullptr;
  int* rreq = nullptr;
  sp::ReqView* rv = nullptr;    // rank map: every request's arrays and slice
  std::vector<sp::ReqView> hviews;  // host copy (kept: the copy to rv is asynchronous)
  long long n_slow = 0;         // rank map: output rows of more than XFAST source entries
  long long* vp = nullptr;      // rows + 1: counts, then the output row pointer
  unsigned* counters = nullptr; // 16 device counters of the count
  char* scan_ws = nullptr;      // the row pointer scan's workspace
  size_t ws_bytes = 0;          // workspace the fill and the run need (reserved by the count)
  cudaStream_t stream = nullptr;
};

namespace sp {

// request of global output row r: the last k with roff[k] <= r
__device__ __forceinline__ long long batch_req_of(const long long* __restrict__ roff, long long nreq, long long r) {
  long long lo = 0, hi = nreq;
  while (hi - lo > 1) {
    const long long mid = (lo + hi) >> 1;
    if (roff[mid] <= r) lo = mid;
    else hi = mid;
  }
  return lo;
}

// every request's J into one array (positions as values); range-checked
template <class IX>
__global__ void k_batch_gather_j(const BatchReq* __restrict__ reqs, const BatchMat* __restrict__ mats,
                                 long long nreq, IX* __restrict__ jkey, uint32_t* __restrict__ jpos,
                                 DevStatus* st) {
  for (long long k = blockIdx.x; k < nreq; k += gridDim.x) {
    const BatchReq q = reqs[k];
    const long long n = mats[q.mat].ncols;
    const IX* J = static_cast<const IX*>(q.J);
    for (long long b = threadIdx.x; b < q.nJ; b += blockDim.x) {
      const long long c = (long long)J[b];
      if (c < 0 || c >= n) dev_fail(st, SP_ERR_INDEX_RANGE, q.joff + b);
      jkey[q.joff + b] = IX(c < 0 || c >= n ? 0 : c);
      jpos[q.joff + b] = uint32_t(b);
    }
  }
}

// rank map: every request's J marked in its slice of the bitmap (a repeat is an error)
template <class IX>
__global__ void k_batch_mark(const BatchReq* __restrict__ reqs, const BatchMat* __restrict__ mats, long long nreq,
                             uint32_t* __restrict__ bits, DevStatus* st) {
  for (long long k = blockIdx.x; k < nreq; k += gridDim.x) {
    const BatchReq q = reqs[k];
    const long long n = mats[q.mat].ncols;
    const IX* J = static_cast<const IX*>(q.J);
    for (long long b = threadIdx.x; b < q.nJ; b += blockDim.x) {
      const long long c = (long long)J[b];
      if (c < 0 || c >= n) {
        dev_fail(st, SP_ERR_INDEX_RANGE, q.joff + b);
        continue;
      }
      const uint32_t m = 1u << (c & 31);
      if (atomicOr(bits + q.moff + (c >> 5), m) & m) dev_fail(st, SP_ERR_DUPLICATE_INDEX, q.joff + b);
    }
  }
}

// rank map: jrp[rank(J_k[b])] = b, ranks counted over the whole batch
template <class IX>
__global__ void k_batch_jrank(const BatchReq* __restrict__ reqs, const BatchMat* __restrict__ mats, long long nreq,
                              const unsigned long long* __restrict__ meta, uint32_t* __restrict__ jrp) {
  for (long long k = blockIdx.x; k < nreq; k += gridDim.x) {
    const BatchReq q = reqs[k];
    const long long n = mats[q.mat].ncols;
    const IX* J = static_cast<const IX*>(q.J);
    for (long long b = threadIdx.x; b < q.nJ; b += blockDim.x) {
      const long long c = (long long)J[b];
      if (c < 0 || c >= n) continue;  // reported by k_batch_mark
      const unsigned long long w = meta[q.moff + (c >> 5)];
      const uint32_t bit = 1u << (c & 31);
      jrp[uint32_t(w >> 32) + __popc(uint32_t(w) & (bit - 1u))] = uint32_t(b);
    }
  }
}

// rank map: source start, length and request of every output row (one CTA per request
// at a time, its rows in parallel)
template <class RP, class IX>
__global__ void k_batch_rowinfo(const BatchReq* __restrict__ reqs, const BatchMat* __restrict__ mats, long long nreq,
                                long long* __restrict__ rs0, long long* __restrict__ rsn, int* __restrict__ rreq,
                                DevStatus* st) {
  for (long long k = blockIdx.x; k < nreq; k += gridDim.x) {
    const BatchReq q = reqs[k];
    const BatchMat a = mats[q.mat];
    const IX* I = static_cast<const IX*>(q.I);
    const RP* rp = static_cast<const RP*>(a.rowptr);
    for (long long t = threadIdx.x; t < q.nI; t += blockDim.x) {
      const long long r = q.roff + t, src = (long long)I[t];
      long long s = 0, L = 0;
      if (src < 0 || src >= a.nrows) {
        dev_fail(st, SP_ERR_INDEX_RANGE, r);
      } else {
        const long long b = (long long)rp[src], e = (long long)rp[src + 1];
        if (b >= 0 && e >= b && e <= a.nnz) {
          s = b;
          L = e - b;
        }
      }
      rs0[r] = s;
      rsn[r] = L;
      rreq[r] = int(k);
    }
  }
}

// Row source of the batched count and fill (extract_rows.cuh): output row r reads the
// matrix of its request and tests / relabels through the request's rank-map slice.  The
// per-row handle is the request's index; its view is read through the read-only cache.
template <class CIt, class VTt>
struct XBatchSrc {
  using CI = CIt;
  using VT = VTt;
  static constexpr bool kLongCta = false;  // a warp takes every row, however long
  struct H {
    int k;
  };
  const int* rreq;
  const ReqView* rv;
  const uint32_t* jrp;
  __device__ __forceinline__ H handle(long long r) const { return H{rreq[r]}; }
  __device__ static __forceinline__ H shfl(const H& h, int k) { return H{__shfl_sync(kFull, h.k, k)}; }
  __device__ __forceinline__ const CI* cols(const H& h) const { return static_cast<const CI*>(rv[h.k].col); }
  __device__ __forceinline__ const VT* vals(const H& h) const { return static_cast<const VT*>(rv[h.k].val); }
  __device__ __forceinline__ bool test(const H& h, long long c) const {
    const long long n = __ldg(&rv[h.k].ncol);
    if (c < 0 || c >= n) return false;
    const unsigned long long* meta = rv[h.k].meta;
    const unsigned long long w = (unsigned long long)ld_map(reinterpret_cast<const long long*>(meta) + (c >> 5));
    return (uint32_t(w) >> (c & 31)) & 1u;
  }
  __device__ __forceinline__ bool map(const H& h, long long c, uint32_t& key) const {
    const long long n = __ldg(&rv[h.k].ncol);
    if (c < 0 || c >= n) return false;
    const unsigned long long* meta = rv[h.k].meta;
    const unsigned long long w = (unsigned long long)ld_map(reinterpret_cast<const long long*>(meta) + (c >> 5));
    const uint32_t bits = uint32_t(w), b = 1u << (c & 31);
    if (!(bits & b)) return false;
    key = ld_plain(jrp + (uint32_t(w >> 32) + __popc(bits & (b - 1u))));
    return true;
  }
};

// J must be distinct within a request: equal neighbours in the sorted J of one request
template <class IX>
__global__ void k_batch_jdup(const long long* __restrict__ joff, long long nreq, const IX* __restrict__ jkey,
                             long long jtot, DevStatus* st) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e + 1 < jtot;
       e += (long long)gridDim.x * blockDim.x) {
    if (jkey[e] != jkey[e + 1]) continue;
    const long long k = batch_req_of(joff, nreq, e + 1);
    if (joff[k] != e + 1) dev_fail(st, SP_ERR_DUPLICATE_INDEX, e + 1);  // same request
  }
}

// rpw output rows per warp (global index r over the batch; 1, 2, 4 or 8, a run-time
// kernel shape), each served by a group of 32 / rpw lanes: the selected source row, each
// stored column looked up in the request's sorted J.  PASS 0 counts the kept entries
// into vp[r]; PASS 1 writes them (position in J as the column, ballot slots within the
// lane group, source order) at the row pointer vp.
template <int PASS, class RP, class CI, class VT, class IX>
__global__ void k_batch_rows(const BatchReq* __restrict__ reqs, const BatchMat* __restrict__ mats,
                             const long long* __restrict__ roff, long long nreq, long long rows,
                             const IX* __restrict__ jkey, const uint32_t* __restrict__ jpos,
                             long long* __restrict__ vp, CI* __restrict__ out_col, VT* __restrict__ out_val,
                             int rpw, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int G = 32 / rpw, grp = lane / G, gl = lane - grp * G;
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (grp * G);
  const unsigned lt = ((1u << gl) - 1u) << (grp * G);  // lanes of the group below this one
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long rb = w0 * rpw; rb < rows; rb += nw * rpw) {  // warp-uniform
    const long long r = rb + grp;
    long long s = 0, e = 0, nJ = 0, joff = 0;
    const CI* col = nullptr;
    const VT* val = nullptr;
    if (r < rows) {
      const long long k = batch_req_of(roff, nreq, r);
      const BatchReq q = reqs[k];
      const BatchMat a = mats[q.mat];
      const long long src = (long long)static_cast<const IX*>(q.I)[r - q.roff];
      if (src < 0 || src >= a.nrows) {
        if (gl == 0 && PASS == 0) dev_fail(st, SP_ERR_INDEX_RANGE, r);
      } else {
        const RP* rp = static_cast<const RP*>(a.rowptr);
        s = (long long)rp[src];
        e = (long long)rp[src + 1];
        if (s < 0 || e < s || e > a.nnz) s = e = 0;
      }
      col = static_cast<const CI*>(a.colidx);
      val = static_cast<const VT*>(a.values);
      nJ = q.nJ;
      joff = q.joff;
    }
    const IX* jk = jkey + joff;
    long long o = PASS && r < rows ? vp[r] : 0;
    const long long oe = PASS && r < rows ? vp[r + 1] : 0;
    // every lane steps until all groups of the warp are done (the ballots need them all)
    for (long long k0 = s; __any_sync(0xffffffffu, k0 < e); k0 += G) {
      const long long x = k0 + gl;
      bool kept = false;
      long long hit = 0;
      if (x < e) {
        const long long c = (long long)ld_stream(col + x);
        hit = lower_bound_col(jk, 0, nJ, c);
        kept = hit < nJ && (long long)jk[hit] == c;
      }
      const unsigned m = __ballot_sync(0xffffffffu, kept) & gmask;
      if (PASS == 1 && kept) {
        const long long pos = o + __popc(m & lt);
        if (pos < oe) {
          st_stream(out_col + pos, CI(jpos[joff + hit]));
          st_stream(out_val + pos, ld_stream(val + x));
        } else {
          dev_fail(st, SP_ERR_INTERNAL, -25);
        }
      }
      o += __popc(m);
    }
    if (PASS == 0 && gl == 0 && r < rows) vp[r] = o;
  }
}

// Row pointer store of a run: clamped to the counted nnz (the output's capacity).
template <class T>
struct StoreCappedRp {
  long long* vp;
  T* out;
  long long cap;
  DevStatus* st;
  __device__ void operator()(long long i, long long v) const {
    if (v > cap) {
      dev_fail(st, SP_ERR_OVERFLOW, i);
      v = cap;
    }
    vp[i] = v;
    out[i] = T(v);
  }
};

template <class RP, class CI, class VT, class IX>
sp_status batch_device_count(sp_ctx* ctx, sp_batch* b, cudaStream_t s, sp_csr* out);

template <class RP, class CI, class VT, class IX>
sp_status batch_count_impl(sp_ctx* ctx, sp_batch* b, const std::vector<BatchMat>& hm,
                           const std::vector<BatchReq>& hr, cudaStream_t s) {
  const long long nreq = b->nreq, rows = b->rows, jtot = b->jtot, nw = b->nwords;
  // the rank map unless its slices are too large (or the batch's J too long for 32-bit ranks)
  b->identify = (ctx->cur.identify == 0 && nw * 12 <= kBatchMapBytes && jtot < (1ll << 32)) ? 0 : 1;
  const bool rank = b->identify == 0;
  Carver cv;
  const size_t o_m = cv.reserve(hm.size() * sizeof(BatchMat));
  const size_t o_r = cv.reserve(hr.size() * sizeof(BatchReq));
  const size_t o_ro = cv.reserve(size_t(nreq + 1) * 8);
  const size_t o_jo = cv.reserve(size_t(nreq + 1) * 8);
  const size_t o_jk = cv.reserve(rank ? 0 : size_t(jtot) * sizeof(IX));
  const size_t o_jp = cv.reserve(size_t(jtot) * 4);
  const size_t o_jb = cv.reserve(rank ? size_t(nw) * 4 : 0);
  const size_t o_jm = cv.reserve(rank ? size_t(nw) * 8 : 0);
  const size_t o_vp = cv.reserve(size_t(rows + 1) * 8);
  const size_t o_sc = cv.reserve(scan_ws_bytes(rows > nw ? rows : nw));
  const size_t o_rs = cv.reserve(rank ? size_t(rows) * 8 : 0);
  const size_t o_rn = cv.reserve(rank ? size_t(rows) * 8 : 0);
  const size_t o_rq = cv.reserve(rank ? size_t(rows) * 4 : 0);
  const size_t o_rv = cv.reserve(rank ? size_t(nreq) * sizeof(ReqView) : 0);
  const size_t o_ct = cv.reserve(64);
  b->buf = static_cast<char*>(ctx_alloc(ctx, cv.total(), s));
  if (!b->buf) return SP_ERR_OOM;
  b->buf_bytes = cv.total();
  cv.bind(b->buf);
  b->mats = cv.at<BatchMat>(o_m);
  b->reqs = cv.at<BatchReq>(o_r);
  b->droff = cv.at<long long>(o_ro);
  b->djoff = cv.at<long long>(o_jo);
  b->jkey = rank ? nullptr : cv.at<void>(o_jk);
  b->jpos = rank ? nullptr : cv.at<uint32_t>(o_jp);
  b->jrp = rank ? cv.at<uint32_t>(o_jp) : nullptr;
  b->jbits = rank ? cv.at<uint32_t>(o_jb) : nullptr;
  b->jmeta = rank ? cv.at<unsigned long long>(o_jm) : nullptr;
  b->vp = cv.at<long long>(o_vp);
  b->rs0 = rank ? cv.at<long long>(o_rs) : nullptr;
  b->rsn = rank ? cv.at<long long>(o_rn) : nullptr;
  b->rreq = rank ? cv.at<int>(o_rq) : nullptr;
  b->rv = rank ? cv.at<ReqView>(o_rv) : nullptr;
  if (rank && nreq > 0) {
    b->hviews.resize(size_t(nreq));
    for (long long k = 0; k < nreq; ++k) {
      const BatchMat& a = hm[size_t(hr[size_t(k)].mat)];
      b->hviews[size_t(k)] = ReqView{a.colidx, a.values, b->jmeta + hr[size_t(k)].moff, a.ncols};
    }
    SP_CUDA(cudaMemcpyAsync(b->rv, b->hviews.data(), size_t(nreq) * sizeof(ReqView), cudaMemcpyHostToDevice, s));
  }
  std::vector<long long> joff(nreq + 1);
  for (long long k = 0; k <= nreq; ++k) joff[k] = k < nreq ? hr[k].joff : jtot;
  SP_CUDA(cudaMemcpyAsync(b->mats, hm.data(), hm.size() * sizeof(BatchMat), cudaMemcpyHostToDevice, s));
  SP_CUDA(cudaMemcpyAsync(b->reqs, hr.data(), hr.size() * sizeof(BatchReq), cudaMemcpyHostToDevice, s));
  SP_CUDA(cudaMemcpyAsync(b->droff, b->roff.data(), size_t(nreq + 1) * 8, cudaMemcpyHostToDevice, s));
  SP_CUDA(cudaMemcpyAsync(b->djoff, joff.data(), size_t(nreq + 1) * 8, cudaMemcpyHostToDevice, s));
  b->counters = cv.at<unsigned>(o_ct);
  b->scan_ws = cv.at<char>(o_sc);
  SP_TRY((batch_device_count<RP, CI, VT, IX>(ctx, b, s, nullptr)));
  long long* h = ctx->hbuf;  // the context's pinned scratch, read back before returning
  SP_CUDA(cudaMemcpyAsync(h, b->vp + rows, 8, cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaMemcpyAsync(h + 1, b->counters + 1, 4, cudaMemcpyDeviceToHost, s));
  SP_TRY(ctx_collect(ctx, s));
  b->nnz = h[0];
  b->n_slow = rank ? (long long)*reinterpret_cast<const unsigned*>(h + 1) : 0;
  // reserve now the workspace the fill's row sort needs (and a run's: any number of slow
  // rows up to all of them), so neither allocates
  Carver cf, cr;
  size_t rf[kRowsSlots];
  rows_reserve(cf, rows, b->nnz, sizeof(VT), rf, true, b->n_slow);
  rows_reserve(cr, rows, b->nnz, sizeof(VT), rf, true, rank ? rows : 0);
  b->ws_bytes = cf.total() > cr.total() ? cf.total() : cr.total();
  char* base;
  SP_TRY(ctx_workspace(ctx, b->ws_bytes, s, &base));
  return SP_OK;
}

// The device part of the count: identify, per-row kept counts, and their exclusive scan
// into b->vp.  With `out` (a run), the scan is clamped to the counted nnz (an overflow
// is reported as SP_ERR_OVERFLOW) and mirrored into out's row pointer.  Launches only:
// no allocation, no synchronisation.
template <class RP, class CI, class VT, class IX>
sp_status batch_device_count(sp_ctx* ctx, sp_batch* b, cudaStream_t s, sp_csr* out) {
  const long long nreq = b->nreq, rows = b->rows, jtot = b->jtot, nw = b->nwords;
  const bool rank = b->identify == 0;
  unsigned* counters = b->counters;
  const int nsm = ctx->num_sms;
  IX* jkey = static_cast<IX*>(b->jkey);
  if (rank) {
    // every request's slice: bits (repeats reported), batch-wide ranks, positions
    SP_CUDA(cudaMemsetAsync(b->jbits, 0, size_t(nw) * 4, s));
    if (jtot > 0) {
      {
        SP_PHASE(SP_PHASE_MAP);
        k_batch_mark<IX><<<unsigned(nreq < 65535 ? nreq : 65535), 256, 0, s>>>(b->reqs, b->mats, nreq, b->jbits,
                                                                            ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
    }
    SP_TRY(launch_scan(ctx, s, LoadPopc{b->jbits}, StoreRank{b->jbits, b->jmeta, nw}, nw, b->scan_ws,
                       SP_PHASE_MAP));
    if (jtot > 0) {
      {
        SP_PHASE(SP_PHASE_MAP);
        k_batch_jrank<IX><<<unsigned(nreq < 65535 ? nreq : 65535), 256, 0, s>>>(b->reqs, b->mats, nreq, b->jmeta,
                                                                             b->jrp);
      }
      SP_CUDA(cudaGetLastError());
    }
  } else if (jtot > 0) {
    {
      SP_PHASE(SP_PHASE_MAP);
      k_batch_gather_j<IX><<<unsigned(nreq < 65535 ? nreq : 65535), 256, 0, s>>>(b->reqs, b->mats, nreq, jkey,
                                                                                 b->jpos, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    // sort every request's J (a row of the J matrix), positions travel as values
    Carver cw;
    size_t ro[kRowsSlots];
    rows_reserve(cw, nreq, jtot, 4, ro);
    char* base;
    SP_TRY(ctx_workspace(ctx, cw.total(), s, &base));
    cw.bind(base);
    const RowsWs w = rows_bind(cw, nreq, jtot, ro);
    SP_TRY((run_rows<IX, uint32_t, NoGather<IX, uint32_t>>(ctx, s, b->djoff, nreq, jtot, b->key_bits, w,
                                                           nullptr, true, jkey, b->jpos)));
    {
      SP_PHASE(SP_PHASE_MAP);
      k_batch_jdup<IX><<<grid_for(jtot, 256, nsm * 8), 256, 0, s>>>(b->djoff, nreq, jkey, jtot, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
  }
  SP_CUDA(cudaMemsetAsync(counters, 0, 64, s));
  if (rows > 0 && rank) {
    // every output row's source, then the count of k_xcount (lane-per-row, grouped loads)
    {
      SP_PHASE(SP_PHASE_COUNT);
      k_batch_rowinfo<RP, IX><<<unsigned(nreq < 65535 ? nreq : 65535), 256, 0, s>>>(
          b->reqs, b->mats, nreq, b->rs0, b->rsn, b->rreq, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    {
      SP_PHASE(SP_PHASE_COUNT);
      const XBatchSrc<CI, uint32_t> src{b->rreq, b->rv, b->jrp};
      k_xcount<<<grid_for((rows + 31) / 32 * 32, XB, nsm * 8), XB, 0, s>>>(
          src, XResolveRecorded{b->rs0, b->rsn}, rows, b->vp, nullptr, counters, 0, counters + 1, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
  } else if (rows > 0) {
    {
      SP_PHASE(SP_PHASE_COUNT);
      const int rpw = ctx->cur.batch_rows;
      const int g = grid_for((rows + rpw - 1) / rpw * 32, 256, nsm * 16);
      k_batch_rows<0, RP, CI, VT, IX><<<g, 256, 0, s>>>(b->reqs, b->mats, b->droff, nreq, rows, jkey, b->jpos, b->vp,
                                                        nullptr, nullptr, rpw, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
  }
  if (!out) {
    SP_TRY(launch_scan(ctx, s, LoadArray<long long>{b->vp}, StoreDual<long long>{b->vp, nullptr, ctx->dstatus},
                       rows, b->scan_ws));
  } else if (out->rowptr_type == SP_I64) {
    SP_TRY(launch_scan(ctx, s, LoadArray<long long>{b->vp},
                       StoreCappedRp<long long>{b->vp, static_cast<long long*>(out->rowptr), b->nnz, ctx->dstatus},
                       rows, b->scan_ws));
  } else {
    SP_TRY(launch_scan(ctx, s, LoadArray<long long>{b->vp},
                       StoreCappedRp<int32_t>{b->vp, static_cast<int32_t*>(out->rowptr), b->nnz, ctx->dstatus},
                       rows, b->scan_ws));
  }
  return SP_OK;
}

// The fill after the row pointer: kept entries of every output row written at b->vp,
// then the row sort.  nnz: the output's entries (capacity); n_slow: rows the fill may
// queue for the sort.  Its workspace was reserved by the count.
template <class RP, class CI, class VT, class IX>
sp_status batch_fill_body(sp_ctx* ctx, sp_batch* b, sp_csr* out, cudaStream_t s, long long nnz, long long n_slow) {
  const long long rows = b->rows;
  Carver cf;
  size_t rf[kRowsSlots];
  rows_reserve(cf, rows, nnz, sizeof(VT), rf, true, n_slow);
  CI* oc = static_cast<CI*>(out->colidx);
  VT* ov = static_cast<VT*>(out->values);
  const int kb = ceil_log2_u64(uint64_t(b->max_nj > 1 ? b->max_nj : 1));
  if (b->identify == 0) {
    // k_xfill: short rows relabelled, ranked and written once; longer rows in source
    // order, queued for the row sort
    char* base;
    SP_TRY(ctx_workspace(ctx, cf.total(), s, &base));
    cf.bind(base);
    const RowsWs w = rows_bind(cf, rows, nnz, rf, true, n_slow);
    SP_CUDA(cudaMemsetAsync(w.counters, 0, 16 * 4, s));
    {
      SP_PHASE(SP_PHASE_GATHER);
      const XBatchSrc<CI, VT> src{b->rreq, b->rv, b->jrp};
      k_xfill<XBatchSrc<CI, VT>, false><<<grid_for((rows + 31) / 32 * 32, XB, ctx->num_sms * 8), XB, 0, s>>>(
          src, rows, b->rs0, b->rsn, b->vp, oc, ov, w.fin, w.counters + 0, w.fin_cap, w.huge, w.huge_n(),
          w.huge_cap, kb, b->max_nj <= 0xFFFFFFFFll ? XF_LANE : 0, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    return sort_queued<CI, VT>(ctx, s, w, kb, oc, ov);
  }
  {
    SP_PHASE(SP_PHASE_GATHER);
    const int rpw = ctx->cur.batch_rows;
    const int g = grid_for((rows + rpw - 1) / rpw * 32, 256, ctx->num_sms * 16);
    k_batch_rows<1, RP, CI, VT, IX><<<g, 256, 0, s>>>(b->reqs, b->mats, b->droff, b->nreq, rows,
                                                      static_cast<const IX*>(b->jkey), b->jpos, b->vp, oc, ov, rpw,
                                                      ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  char* base;
  SP_TRY(ctx_workspace(ctx, cf.total(), s, &base));
  cf.bind(base);
  const RowsWs w = rows_bind(cf, rows, nnz, rf, true, n_slow);
  return run_rows<CI, VT, NoGather<CI, VT>>(ctx, s, b->vp, rows, nnz, kb, w, nullptr, true, oc, ov);
}

template <class RP, class CI, class VT, class IX>
sp_status batch_fill_impl(sp_ctx* ctx, sp_batch* b, sp_csr* out, cudaStream_t s) {
  const long long rows = b->rows, nnz = b->nnz;
  // the row sort's workspace was reserved by the count: check it before any launch, so
  // a failure leaves the output untouched
  Carver cf;
  size_t rf[kRowsSlots];
  rows_reserve(cf, rows, nnz, sizeof(VT), rf, true, b->n_slow);
  if (nnz > 0 && cf.total() > ctx->ws_cap) return SP_ERR_INTERNAL;
  // the int64 row pointer is the batch's own; an int32 output gets a narrowed copy
  if (out->rowptr_type == SP_I64) {
    SP_CUDA(cudaMemcpyAsync(out->rowptr, b->vp, size_t(rows + 1) * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    SP_PHASE(SP_PHASE_OTHER);
    k_narrow<int32_t><<<grid_for(rows + 1, 256, ctx->num_sms * 8), 256, 0, s>>>(
        b->vp, rows + 1, static_cast<int32_t*>(out->rowptr), ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  if (nnz == 0) return SP_OK;
  return batch_fill_body<RP, CI, VT, IX>(ctx, b, out, s, nnz, b->n_slow);
}

// A run: the count's device part again (clamped to the counted nnz), then the fill.
template <class RP, class CI, class VT, class IX>
sp_status batch_run_impl(sp_ctx* ctx, sp_batch* b, sp_csr* out, cudaStream_t s) {
  const long long rows = b->rows, nnz = b->nnz;
  if (b->ws_bytes > ctx->ws_cap) return SP_ERR_INTERNAL;  // reserved by the count
  SP_TRY((batch_device_count<RP, CI, VT, IX>(ctx, b, s, out)));
  if (nnz == 0) return SP_OK;
  return batch_fill_body<RP, CI, VT, IX>(ctx, b, out, s, nnz, b->identify == 0 ? rows : 0);
}

}  // namespace sp

using namespace sp;

extern "C" sp_status sp_extract_batch_count(sp_ctx* ctx, const sp_csr* mats, int64_t nmats,
                                            const sp_extract_req* reqs, int64_t nreq, sp_itype idx_type,
                                            sp_batch** batch, int64_t* nnz_total, sp_stream_t stream) {
  if (!ctx || !batch || !nnz_total || nmats < 0 || nreq < 0) return SP_ERR_INVALID_ARG;
  if ((nmats > 0 && !mats) || (nreq > 0 && !reqs)) return SP_ERR_INVALID_ARG;
  if (idx_type != SP_I32 && idx_type != SP_I64) return SP_ERR_INVALID_ARG;
  *batch = nullptr;
  if (nmats == 0 && nreq > 0) return SP_ERR_INVALID_ARG;
  for (int64_t t = 0; t < nmats; ++t) {
    SP_TRY(check_csr(&mats[t]));
    if (mats[t].rowptr_type != mats[0].rowptr_type || mats[t].colidx_type != mats[0].colidx_type ||
        mats[t].value_type != mats[0].value_type)
      return SP_ERR_INVALID_ARG;  // one type combination per batch
  }
  sp_batch* b = new sp_batch();
  b->nreq = nreq;
  b->nmats = nmats;
  b->idx_type = idx_type;
  if (nmats > 0) {
    b->rowptr_type = mats[0].rowptr_type;
    b->colidx_type = mats[0].colidx_type;
    b->value_type = mats[0].value_type;
  }
  std::vector<BatchMat> hm(static_cast<size_t>(nmats));
  long long max_cols = 1;
  for (int64_t t = 0; t < nmats; ++t) {
    hm[t] = BatchMat{mats[t].rowptr, mats[t].colidx, mats[t].values, mats[t].nrows, mats[t].ncols, mats[t].nnz};
    if (mats[t].ncols > max_cols) max_cols = mats[t].ncols;
  }
  std::vector<BatchReq> hr(static_cast<size_t>(nreq));
  b->roff.assign(size_t(nreq + 1), 0);
  for (int64_t k = 0; k < nreq; ++k) {
    const sp_extract_req& q = reqs[k];
    if (q.mat < 0 || q.mat >= nmats || q.nI < 0 || q.nJ < 0 || (q.nI > 0 && !q.I) || (q.nJ > 0 && !q.J) ||
        q.nJ > mats[q.mat].ncols || q.nJ > (int64_t(1) << 32)) {
      delete b;
      return q.mat < 0 || q.mat >= nmats || (q.nI > 0 && !q.I) || (q.nJ > 0 && !q.J) ? SP_ERR_INVALID_ARG
                                                                                     : SP_ERR_SHAPE;
    }
    hr[k] = BatchReq{q.mat, q.nI, q.nJ, q.I, q.J, b->rows, b->jtot, b->nwords};
    b->nwords += (mats[q.mat].ncols + 31) / 32;
    b->roff[k] = b->rows;
    b->rows += q.nI;
    b->jtot += q.nJ;
    if (q.nJ > b->max_nj) b->max_nj = q.nJ;
  }
  b->roff[nreq] = b->rows;
  b->key_bits = ceil_log2_u64(uint64_t(max_cols));
  cudaStream_t s = (cudaStream_t)stream;
  b->stream = s;
  sp_status st = cudaSetDevice(ctx->device) == cudaSuccess ? SP_OK : SP_ERR_CUDA;
  ctx_begin_call(ctx, SP_OP_BATCH, b->rows);
  if (st == SP_OK && nmats > 0) {
    st = dispatch_i(b->rowptr_type, [&](auto rp) {
      using RP = decltype(rp);
      return dispatch_i(b->colidx_type, [&](auto ci) {
        using CI = decltype(ci);
        return dispatch_v(b->value_type, [&](auto vt) {
          using VT = decltype(vt);
          return dispatch_i(idx_type, [&](auto ix) {
            using IX = decltype(ix);
            return batch_count_impl<RP, CI, VT, IX>(ctx, b, hm, hr, s);
          });
        });
      });
    });
  }
  if (st != SP_OK) {
    sp_batch_destroy(ctx, b);
    return st;
  }
  *batch = b;
  *nnz_total = b->nnz;
  return SP_OK;
}

extern "C" sp_status sp_extract_batch_fill(sp_ctx* ctx, sp_batch* b, sp_csr* out, sp_stream_t stream) {
  if (!ctx || !b || !out) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type != SP_I32 && out->rowptr_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type == SP_I32 && b->nnz > INT32_MAX) return SP_ERR_OVERFLOW;
  if (!out->rowptr || (b->nnz > 0 && (!out->colidx || !out->values))) return SP_ERR_INVALID_ARG;
  if (out->colidx_type != b->colidx_type || out->value_type != b->value_type) return SP_ERR_INVALID_ARG;
  out->nrows = b->rows;
  out->ncols = b->max_nj;
  out->nnz = b->nnz;
  if (b->nmats == 0) return SP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ctx_begin_call(ctx, SP_OP_BATCH, b->rows);
  return dispatch_i(b->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(b->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(b->value_type, [&](auto vt) {
        using VT = decltype(vt);
        return dispatch_i(b->idx_type, [&](auto ix) {
          using IX = decltype(ix);
          return batch_fill_impl<RP, CI, VT, IX>(ctx, b, out, s);
        });
      });
    });
  });
}

extern "C" sp_status sp_extract_batch_run(sp_ctx* ctx, sp_batch* b, sp_csr* out, sp_stream_t stream) {
  if (!ctx || !b || !out) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type != SP_I32 && out->rowptr_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type == SP_I32 && b->nnz > INT32_MAX) return SP_ERR_OVERFLOW;
  if (!out->rowptr || (b->nnz > 0 && (!out->colidx || !out->values))) return SP_ERR_INVALID_ARG;
  if (out->colidx_type != b->colidx_type || out->value_type != b->value_type) return SP_ERR_INVALID_ARG;
  out->nrows = b->rows;
  out->ncols = b->max_nj;
  out->nnz = b->nnz;
  if (b->nmats == 0) return SP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ctx_begin_call(ctx, SP_OP_BATCH, b->rows);
  return dispatch_i(b->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(b->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(b->value_type, [&](auto vt) {
        using VT = decltype(vt);
        return dispatch_i(b->idx_type, [&](auto ix) {
          using IX = decltype(ix);
          return batch_run_impl<RP, CI, VT, IX>(ctx, b, out, s);
        });
      });
    });
  });
}

extern "C" int64_t sp_batch_row_offset(const sp_batch* b, int64_t k) {
  if (!b || k < 0 || k > b->nreq) return -1;
  return b->roff[size_t(k)];
}

extern "C" sp_status sp_batch_destroy(sp_ctx* ctx, sp_batch* b) {
  if (!b) return SP_OK;
  if (b->buf && ctx) ctx_free(ctx, b->buf, b->buf_bytes, b->stream);
  delete b;
  return SP_OK;
}
