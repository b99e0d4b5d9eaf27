// Batched permutation: B_k = P_k A_{m_k} Q_k^T (Sec. 2.1; HipPerm) for many requests over
// device-resident matrices, in a fixed number of launches for the whole batch (the
// batching pattern of the serving path; the paper has no batched form).
//
// The output size of a permutation is the input's, so the plan (host only: request and
// matrix tables, buffer layout) knows every row pointer's extent and the batch's nnz
// without touching the device; the fill then runs everything on one stream with no
// synchronisation and no allocation, so the whole batch can be captured in a CUDA graph:
//   per request: inverse column map qinv_k (validates q_k) and a bitmap of p_k
//   (validates p_k) -> every output row's source (request k and start s packed as
//   k * 2^40 + s) and length -> exclusive scan of the lengths (the row pointer) -> the
//   two-phase path of the single permutation over the whole batch: partition of the
//   output rows, load-balanced chunk gather with the relabelling through each row's
//   request, in-place row sort.
#include <cstring>
#include <vector>

#include "dispatch.h"
#include "kernels.cuh"
#include "rowsort.cuh"

namespace sp {

struct PermReq {  // a request with its offsets in the batch's rows, map words and bitmaps
  long long mat, nrows, ncols;
  const void* p;  // new row -> old row (null: identity)
  const void* q;  // new column -> old column (null: identity)
  long long roff;  // first output row
  long long qoff;  // first entry of the request's qinv
  long long boff;  // first word of the request's row bitmap
};

// what an output row needs from its request (read through the read-only cache)
struct PermView {
  unsigned long long col;   // const CI*
  unsigned long long val;   // const VT*
  unsigned long long qinv;  // const IX*: the request's inverse column map (0: identity)
  long long ncol;
};

constexpr int kReqShift = 40;  // source position = request * 2^40 + entry of its matrix
constexpr long long kEntryMask = (1ll << kReqShift) - 1;
constexpr long long kMaxReqs = 1ll << 23;

// Host tables reach the device as kernel parameters (up to 32 KB per launch, copied at
// launch): a copy from pageable host memory would first wait for the stream's earlier
// work, and the plan must not wait for the device.
constexpr int kUpBytes = 32704;  // payload per launch (parameter space 32764 bytes)
struct UpChunk {
  char* dst;  // 16-byte aligned
  int n;
  alignas(16) unsigned char b[kUpBytes];
};
__global__ void k_upload(const __grid_constant__ UpChunk c) {
  const int nw = c.n >> 4;
  const uint4* src = reinterpret_cast<const uint4*>(c.b);
  uint4* dst = reinterpret_cast<uint4*>(c.dst);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
  for (int i = (nw << 4) + threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = char(c.b[i]);
}

inline sp_status upload(char* dst, const void* src, size_t bytes, cudaStream_t s) {
  static thread_local UpChunk c;
  const char* h = static_cast<const char*>(src);
  for (size_t o = 0; o < bytes; o += kUpBytes) {
    const size_t n = bytes - o < size_t(kUpBytes) ? bytes - o : size_t(kUpBytes);
    c.dst = dst + o;
    c.n = int(n);
    memcpy(c.b, h + o, n);
    k_upload<<<1, 256, 0, s>>>(c);
    SP_CUDA(cudaGetLastError());
  }
  return SP_OK;
}

// per request: qinv[q[j]] = j (a repeat or an index out of range is not a permutation)
// and the bitmap of p
template <class IX>
__global__ void k_pbatch_maps(const PermReq* __restrict__ reqs, long long nreq, IX* __restrict__ qinv,
                              uint32_t* __restrict__ pbits, DevStatus* st) {
  for (long long k = blockIdx.x; k < nreq; k += gridDim.x) {
    const PermReq r = reqs[k];
    const IX* q = static_cast<const IX*>(r.q);
    const IX* p = static_cast<const IX*>(r.p);
    if (q) {
      for (long long j = threadIdx.x; j < r.ncols; j += blockDim.x) {
        const long long c = (long long)q[j];
        if (c < 0 || c >= r.ncols) {
          dev_fail(st, SP_ERR_NOT_PERMUTATION, j);
          continue;
        }
        IX* slot = qinv + r.qoff + c;
        if constexpr (sizeof(IX) == 4) {
          if (atomicCAS(reinterpret_cast<int*>(slot), -1, int(j)) != -1) dev_fail(st, SP_ERR_NOT_PERMUTATION, j);
        } else {
          if (atomicCAS(reinterpret_cast<unsigned long long*>(slot), ~0ull, (unsigned long long)j) != ~0ull)
            dev_fail(st, SP_ERR_NOT_PERMUTATION, j);
        }
      }
    }
    if (p) {
      for (long long i = threadIdx.x; i < r.nrows; i += blockDim.x) {
        const long long v = (long long)p[i];
        if (v < 0 || v >= r.nrows) {
          dev_fail(st, SP_ERR_NOT_PERMUTATION, i);
          continue;
        }
        const uint32_t m = 1u << (v & 31);
        if (atomicOr(pbits + r.boff + (v >> 5), m) & m) dev_fail(st, SP_ERR_NOT_PERMUTATION, i);
      }
    }
  }
}

// every output row's source (request and start, packed) and length
template <class RP, class IX>
__global__ void k_pbatch_rowinfo(const PermReq* __restrict__ reqs, const sp_csr* __restrict__ mats, long long nreq,
                                 long long* __restrict__ rsrc, long long* __restrict__ rsn) {
  for (long long k = blockIdx.x; k < nreq; k += gridDim.x) {
    const PermReq r = reqs[k];
    const sp_csr a = mats[r.mat];
    const IX* p = static_cast<const IX*>(r.p);
    const RP* rp = static_cast<const RP*>(a.rowptr);
    for (long long i = threadIdx.x; i < r.nrows; i += blockDim.x) {
      const long long src = p ? (long long)p[i] : i;
      long long s = 0, L = 0;
      if (src >= 0 && src < r.nrows) {  // else reported by k_pbatch_maps
        const long long b = (long long)rp[src], e = (long long)rp[src + 1];
        if (b >= 0 && e >= b && e <= a.nnz) {
          s = b;
          L = e - b;
        }
      }
      rsrc[r.roff + i] = (k << kReqShift) | s;
      rsn[r.roff + i] = L;
    }
  }
}

// Phase-1 gather (rowsort.cuh) of the batch: output row r reads its request's matrix at
// the packed source position; every column is relabelled through the request's qinv
// (identity without one).  Under a column map a column outside [0, ncols) becomes the
// key 0xFFFFFFFF, which the sort reports as SP_ERR_INDEX_RANGE.
template <class CIt, class VTt, class IX>
struct PermBatchGs {
  using CI = CIt;
  using VT = VTt;
  const PermView* pv;
  const long long* rsrc;
  __device__ long long src(long long r) const { return rsrc[r]; }
  __device__ CI col(long long pos) const {
    const CI* c = reinterpret_cast<const CI*>(__ldg(&pv[pos >> kReqShift].col));
    return ld_stream(c + (pos & kEntryMask));
  }
  __device__ VT val(long long pos) const {
    const VT* v = reinterpret_cast<const VT*>(__ldg(&pv[pos >> kReqShift].val));
    return ld_stream(v + (pos & kEntryMask));
  }
  __device__ CI map(long long pos, CI c) const {
    const PermView* v = pv + (pos >> kReqShift);
    const IX* qinv = reinterpret_cast<const IX*>(__ldg(&v->qinv));
    if (!qinv) return c;
    const long long cl = (long long)c;
    if (cl < 0 || cl >= __ldg(&v->ncol)) return CI(-1);
    return CI(ld_map(qinv + cl));
  }
};

// Scan output of the batch's row pointer, clamped to the output's nnz so that no row
// reaches past the output arrays: the lengths of a valid batch add up to exactly its nnz
// (each source row taken once); a repeated row of p is reported by k_pbatch_maps, a row
// pointer whose lengths do not add up to nnz here (SP_ERR_NOT_CANONICAL).
template <class T>
struct StoreCapped {
  long long* vp;
  T* out;  // may be null
  long long n, cap;
  DevStatus* st;
  __device__ void operator()(long long i, long long v) const {
    if (v > cap || (i == n && v != cap)) {
      dev_fail(st, SP_ERR_NOT_CANONICAL, i);
      if (v > cap) v = cap;
    }
    vp[i] = v;
    if (out) out[i] = T(v);
  }
};

}  // namespace sp

struct sp_pbatch {
  long long nreq = 0, nmats = 0, rows = 0, nnz = 0, qtot = 0, btot = 0, max_cols = 0;
  sp_itype idx_type = SP_I32, rowptr_type = SP_I64, colidx_type = SP_I32;
  sp_vtype value_type = SP_F32;
  std::vector<long long> roff;  // host: first output row of every request (+ total)
  std::vector<sp::PermReq> hreq;
  std::vector<sp::PermView> hview;
  std::vector<sp_csr> hmats;
  char* buf = nullptr;  // device: tables, maps, row table, row pointer, scan and sort workspace
  size_t buf_bytes = 0;
  cudaStream_t stream = nullptr;
  size_t o_req = 0, o_view = 0, o_mat = 0, o_qinv = 0, o_bits = 0, o_rsrc = 0, o_rsn = 0, o_vp = 0,
         o_scan = 0;
  size_t ro[sp::kRowsSlots] = {};
};

namespace sp {

template <class RP, class CI, class VT, class IX>
sp_status pbatch_fill_impl(sp_ctx* ctx, sp_pbatch* b, sp_csr* out, cudaStream_t s) {
  const long long nreq = b->nreq, rows = b->rows, nnz = b->nnz;
  Carver cv;  // the plan's layout, rebuilt to bind the pointers
  cv.bind(b->buf);
  PermReq* reqs = cv.at<PermReq>(b->o_req);
  PermView* views = cv.at<PermView>(b->o_view);
  sp_csr* mats = cv.at<sp_csr>(b->o_mat);
  IX* qinv = cv.at<IX>(b->o_qinv);
  uint32_t* pbits = cv.at<uint32_t>(b->o_bits);
  long long* rsrc = cv.at<long long>(b->o_rsrc);
  long long* rsn = cv.at<long long>(b->o_rsn);
  long long* vp = cv.at<long long>(b->o_vp);
  const unsigned gq = unsigned(nreq < 65535 ? nreq : 65535);
  if (b->qtot > 0) SP_CUDA(cudaMemsetAsync(qinv, 0xFF, size_t(b->qtot) * sizeof(IX), s));
  if (b->btot > 0) SP_CUDA(cudaMemsetAsync(pbits, 0, size_t(b->btot) * 4, s));
  if (nreq > 0) {
    {
      SP_PHASE(SP_PHASE_MAP);
      k_pbatch_maps<IX><<<gq, 256, 0, s>>>(reqs, nreq, qinv, pbits, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    {
      SP_PHASE(SP_PHASE_COUNT);
      k_pbatch_rowinfo<RP, IX><<<gq, 256, 0, s>>>(reqs, mats, nreq, rsrc, rsn);
    }
    SP_CUDA(cudaGetLastError());
  }
  // row pointer of the batch: scan of the row lengths, mirrored into the output's type
  if (out->rowptr_type == SP_I64) {
    SP_TRY(launch_scan(ctx, s, LoadArray<long long>{rsn},
                       StoreCapped<long long>{vp, static_cast<long long*>(out->rowptr), rows, nnz, ctx->dstatus},
                       rows, cv.at<char>(b->o_scan)));
  } else {
    SP_TRY(launch_scan(ctx, s, LoadArray<long long>{rsn},
                       StoreCapped<int32_t>{vp, static_cast<int32_t*>(out->rowptr), rows, nnz, ctx->dstatus},
                       rows, cv.at<char>(b->o_scan)));
  }
  if (nnz == 0 || rows == 0) return SP_OK;
  CI* oc = static_cast<CI*>(out->colidx);
  VT* ov = static_cast<VT*>(out->values);
  // phase 1: gather + relabel over the whole batch; phase 2 (any column map): row sort
  const RowsWs w = rows_bind(cv, rows, nnz, b->ro);
  const int kb = ceil_log2_u64(uint64_t(b->max_cols > 1 ? b->max_cols : 1));
  const PermBatchGs<CI, VT, IX> g{views, rsrc};
  return run_rows(ctx, s, vp, rows, nnz, kb, w, &g, b->qtot > 0, oc, ov);
}

}  // namespace sp

using namespace sp;

extern "C" sp_status sp_permute_batch_plan(sp_ctx* ctx, const sp_csr* mats, int64_t nmats, const sp_permute_req* reqs,
                                           int64_t nreq, sp_itype idx_type, sp_pbatch** plan, int64_t* nnz_total,
                                           sp_stream_t stream) {
  if (!ctx || !plan || !nnz_total || nmats < 0 || nreq < 0) return SP_ERR_INVALID_ARG;
  if ((nmats > 0 && !mats) || (nreq > 0 && !reqs)) return SP_ERR_INVALID_ARG;
  if (idx_type != SP_I32 && idx_type != SP_I64) return SP_ERR_INVALID_ARG;
  *plan = nullptr;
  if (nmats == 0 && nreq > 0) return SP_ERR_INVALID_ARG;
  if (nreq > kMaxReqs) return SP_ERR_OVERFLOW;  // packed source positions
  for (int64_t t = 0; t < nmats; ++t) {
    SP_TRY(check_csr(&mats[t]));
    if (mats[t].rowptr_type != mats[0].rowptr_type || mats[t].colidx_type != mats[0].colidx_type ||
        mats[t].value_type != mats[0].value_type)
      return SP_ERR_INVALID_ARG;  // one type combination per batch
    if (mats[t].ncols > (int64_t(1) << 32)) return SP_ERR_OVERFLOW;  // 32-bit sort keys
    if (mats[t].nnz > kEntryMask) return SP_ERR_OVERFLOW;           // packed source positions
    if (idx_type == SP_I32 && (mats[t].nrows > INT32_MAX || mats[t].ncols > INT32_MAX)) return SP_ERR_OVERFLOW;
  }
  sp_pbatch* b = new sp_pbatch();
  b->nreq = nreq;
  b->nmats = nmats;
  b->idx_type = idx_type;
  if (nmats > 0) {
    b->rowptr_type = mats[0].rowptr_type;
    b->colidx_type = mats[0].colidx_type;
    b->value_type = mats[0].value_type;
  }
  b->hmats.assign(mats, mats + nmats);
  b->hreq.resize(size_t(nreq));
  b->roff.assign(size_t(nreq + 1), 0);
  for (int64_t k = 0; k < nreq; ++k) {
    const sp_permute_req& q = reqs[k];
    if (q.mat < 0 || q.mat >= nmats) {
      delete b;
      return SP_ERR_INVALID_ARG;
    }
    const sp_csr& a = mats[q.mat];
    b->hreq[size_t(k)] = PermReq{q.mat, a.nrows, a.ncols, q.p, q.q, b->rows, q.q ? b->qtot : 0, q.p ? b->btot : 0};
    b->roff[size_t(k)] = b->rows;
    b->rows += a.nrows;
    b->nnz += a.nnz;
    if (q.q) b->qtot += a.ncols;
    if (q.p) b->btot += (a.nrows + 31) / 32;
    if (a.ncols > b->max_cols) b->max_cols = a.ncols;
  }
  b->roff[size_t(nreq)] = b->rows;
  const size_t is = itype_size(idx_type), vs = nmats > 0 ? vtype_size(b->value_type) : 4;
  Carver cv;
  b->o_req = cv.reserve(size_t(nreq) * sizeof(PermReq));
  b->o_view = cv.reserve(size_t(nreq) * sizeof(PermView));
  b->o_mat = cv.reserve(size_t(nmats) * sizeof(sp_csr));
  b->o_qinv = cv.reserve(size_t(b->qtot) * is);
  b->o_bits = cv.reserve(size_t(b->btot) * 4);
  b->o_rsrc = cv.reserve(size_t(b->rows) * 8);
  b->o_rsn = cv.reserve(size_t(b->rows) * 8);
  b->o_vp = cv.reserve(size_t(b->rows + 1) * 8);
  b->o_scan = cv.reserve(scan_ws_bytes(b->rows));
  rows_reserve(cv, b->rows, b->nnz, vs, b->ro);
  cudaStream_t s = (cudaStream_t)stream;
  b->stream = s;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    delete b;
    return SP_ERR_CUDA;
  }
  ctx_begin_call(ctx, SP_OP_BATCH, b->rows);
  b->buf = static_cast<char*>(ctx_alloc(ctx, cv.total(), s));
  if (!b->buf) {
    delete b;
    return SP_ERR_OOM;
  }
  b->buf_bytes = cv.total();
  cv.bind(b->buf);
  b->hview.resize(size_t(nreq));
  {
    char* qbase = cv.at<char>(b->o_qinv);
    for (int64_t k = 0; k < nreq; ++k) {
      const PermReq& r = b->hreq[size_t(k)];
      const sp_csr& a = mats[r.mat];
      b->hview[size_t(k)] = PermView{(unsigned long long)a.colidx, (unsigned long long)a.values,
                                     r.q ? (unsigned long long)(qbase + size_t(r.qoff) * is) : 0ull, a.ncols};
    }
  }
  sp_status st = upload(cv.at<char>(b->o_req), b->hreq.data(), size_t(nreq) * sizeof(PermReq), s);
  if (st == SP_OK) st = upload(cv.at<char>(b->o_view), b->hview.data(), size_t(nreq) * sizeof(PermView), s);
  if (st == SP_OK) st = upload(cv.at<char>(b->o_mat), b->hmats.data(), size_t(nmats) * sizeof(sp_csr), s);
  if (st != SP_OK) {
    sp_pbatch_destroy(ctx, b);
    return st;
  }
  *plan = b;
  *nnz_total = b->nnz;
  return SP_OK;
}

extern "C" sp_status sp_permute_batch_fill(sp_ctx* ctx, sp_pbatch* b, sp_csr* out, sp_stream_t stream) {
  if (!ctx || !b || !out) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type != SP_I32 && out->rowptr_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (out->rowptr_type == SP_I32 && b->nnz > INT32_MAX) return SP_ERR_OVERFLOW;
  if (!out->rowptr || (b->nnz > 0 && (!out->colidx || !out->values))) return SP_ERR_INVALID_ARG;
  if (b->nmats > 0 && (out->colidx_type != b->colidx_type || out->value_type != b->value_type))
    return SP_ERR_INVALID_ARG;
  out->nrows = b->rows;
  out->ncols = b->max_cols;
  out->nnz = b->nnz;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, SP_OP_BATCH, b->rows);
  return dispatch_i(b->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(b->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(b->value_type, [&](auto vt) {
        using VT = decltype(vt);
        return dispatch_i(b->idx_type, [&](auto ix) {
          using IX = decltype(ix);
          return pbatch_fill_impl<RP, CI, VT, IX>(ctx, b, out, s);
        });
      });
    });
  });
}

extern "C" int64_t sp_pbatch_row_offset(const sp_pbatch* b, int64_t k) {
  if (!b || k < 0 || k > b->nreq) return -1;
  return b->roff[size_t(k)];
}

extern "C" sp_status sp_pbatch_destroy(sp_ctx* ctx, sp_pbatch* b) {
  if (!b) return SP_OK;
  if (b->buf && ctx) ctx_free(ctx, b->buf, b->buf_bytes, b->stream);
  delete b;
  return SP_OK;
}
