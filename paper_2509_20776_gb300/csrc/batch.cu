// Batched extraction: B_k = A_{m_k}(I_k, J_k) for thousands of small requests in a fixed
// number of launches over the whole batch (the batching pattern of the serving path).
//
// Identification uses each request's J sorted once (positions carried as values): a
// stored column c of a selected row is looked up by binary search in the request's
// sorted J -- the per-(i, j) search of Algorithm 5, which suits small |J| where a dense
// inverse map per request would cost O(ncols).  Every step runs once for the batch:
//   J gather -> segmented sort of the J's -> duplicate check -> per-row kept counts ->
//   scan -> fill -> segmented sort of the output rows.
// The count call synchronises once (the batch's output size); the fill call allocates
// nothing and never synchronises, so it can be captured in a CUDA graph and replayed.
#include <vector>

#include "dispatch.h"
#include "kernels.cuh"
#include "rowsort.cuh"

namespace sp {

struct BatchMat {  // a matrix of the batch (device arrays)
  const void* rowptr;
  const void* colidx;
  const void* values;
  long long nrows, ncols, nnz;
};

struct BatchReq {  // a request, with its offsets in the batch's J and output rows
  long long mat, nI, nJ;
  const void* I;
  const void* J;
  long long roff, joff;
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
  long long* vp = nullptr;      // rows + 1: counts, then the output row pointer
  size_t ws_bytes = 0;          // workspace the fill needs (reserved by the count)
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

template <class RP, class CI, class VT, class IX>
sp_status batch_count_impl(sp_ctx* ctx, sp_batch* b, const std::vector<BatchMat>& hm,
                           const std::vector<BatchReq>& hr, cudaStream_t s) {
  const long long nreq = b->nreq, rows = b->rows, jtot = b->jtot;
  Carver cv;
  const size_t o_m = cv.reserve(hm.size() * sizeof(BatchMat));
  const size_t o_r = cv.reserve(hr.size() * sizeof(BatchReq));
  const size_t o_ro = cv.reserve(size_t(nreq + 1) * 8);
  const size_t o_jo = cv.reserve(size_t(nreq + 1) * 8);
  const size_t o_jk = cv.reserve(size_t(jtot) * sizeof(IX));
  const size_t o_jp = cv.reserve(size_t(jtot) * 4);
  const size_t o_vp = cv.reserve(size_t(rows + 1) * 8);
  const size_t o_sc = cv.reserve(scan_ws_bytes(rows));
  b->buf = static_cast<char*>(ctx_alloc(ctx, cv.total(), s));
  if (!b->buf) return SP_ERR_OOM;
  b->buf_bytes = cv.total();
  cv.bind(b->buf);
  b->mats = cv.at<BatchMat>(o_m);
  b->reqs = cv.at<BatchReq>(o_r);
  b->droff = cv.at<long long>(o_ro);
  b->djoff = cv.at<long long>(o_jo);
  b->jkey = cv.at<void>(o_jk);
  b->jpos = cv.at<uint32_t>(o_jp);
  b->vp = cv.at<long long>(o_vp);
  std::vector<long long> joff(nreq + 1);
  for (long long k = 0; k <= nreq; ++k) joff[k] = k < nreq ? hr[k].joff : jtot;
  SP_CUDA(cudaMemcpyAsync(b->mats, hm.data(), hm.size() * sizeof(BatchMat), cudaMemcpyHostToDevice, s));
  SP_CUDA(cudaMemcpyAsync(b->reqs, hr.data(), hr.size() * sizeof(BatchReq), cudaMemcpyHostToDevice, s));
  SP_CUDA(cudaMemcpyAsync(b->droff, b->roff.data(), size_t(nreq + 1) * 8, cudaMemcpyHostToDevice, s));
  SP_CUDA(cudaMemcpyAsync(b->djoff, joff.data(), size_t(nreq + 1) * 8, cudaMemcpyHostToDevice, s));
  const int nsm = ctx->num_sms;
  IX* jkey = static_cast<IX*>(b->jkey);
  if (jtot > 0) {
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
  if (rows > 0) {
    {
      SP_PHASE(SP_PHASE_COUNT);
      const int rpw = ctx->cur.batch_rows;
      k_batch_rows<0, RP, CI, VT, IX><<<grid_for((rows + rpw - 1) / rpw * 32, 256, nsm * 16), 256, 0, s>>>(
          b->reqs, b->mats, b->droff, nreq, rows, jkey, b->jpos, b->vp, nullptr, nullptr, rpw, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
  }
  SP_TRY(launch_scan(ctx, s, LoadArray<long long>{b->vp}, StoreDual<long long>{b->vp, nullptr, ctx->dstatus},
                     rows, cv.at<char>(o_sc)));
  long long* h = nullptr;
  SP_CUDA(cudaMallocHost(&h, 8));
  cudaMemcpyAsync(h, b->vp + rows, 8, cudaMemcpyDeviceToHost, s);
  const sp_status st = ctx_collect(ctx, s);
  b->nnz = *h;
  cudaFreeHost(h);
  SP_TRY(st);
  // reserve now the workspace the fill's row sort needs, so the fill allocates nothing
  Carver cf;
  size_t rf[kRowsSlots];
  rows_reserve(cf, rows, b->nnz, sizeof(VT), rf);
  b->ws_bytes = cf.total();
  char* base;
  SP_TRY(ctx_workspace(ctx, b->ws_bytes, s, &base));
  return SP_OK;
}

template <class RP, class CI, class VT, class IX>
sp_status batch_fill_impl(sp_ctx* ctx, sp_batch* b, sp_csr* out, cudaStream_t s) {
  const long long rows = b->rows, nnz = b->nnz;
  // the row sort's workspace was reserved by the count: check it before any launch, so
  // a failure leaves the output untouched
  Carver cf;
  size_t rf[kRowsSlots];
  rows_reserve(cf, rows, nnz, sizeof(VT), rf);
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
  CI* oc = static_cast<CI*>(out->colidx);
  VT* ov = static_cast<VT*>(out->values);
  {
    SP_PHASE(SP_PHASE_GATHER);
    const int rpw = ctx->cur.batch_rows;
    k_batch_rows<1, RP, CI, VT, IX><<<grid_for((rows + rpw - 1) / rpw * 32, 256, ctx->num_sms * 16), 256, 0, s>>>(
        b->reqs, b->mats, b->droff, b->nreq, rows, static_cast<const IX*>(b->jkey), b->jpos, b->vp, oc, ov, rpw,
        ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  char* base;
  SP_TRY(ctx_workspace(ctx, cf.total(), s, &base));
  cf.bind(base);
  const RowsWs w = rows_bind(cf, rows, nnz, rf);
  const int kb = ceil_log2_u64(uint64_t(b->max_nj > 1 ? b->max_nj : 1));
  return run_rows<CI, VT, NoGather<CI, VT>>(ctx, s, b->vp, rows, nnz, kb, w, nullptr, true, oc, ov);
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
    hr[k] = BatchReq{q.mat, q.nI, q.nJ, q.I, q.J, b->rows, b->jtot};
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
