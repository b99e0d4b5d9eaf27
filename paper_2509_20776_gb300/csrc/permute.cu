// sp_permute: B = P A Q^T, B[i, j] = A[p[i], q[j]]  (Sec. 2.1; HipPerm, Algorithm 1).
//
// One-GPU restatement of Identify-Exchange-Build: the inverse column map qinv is the
// index/value swap of the Identify step; every output row i is the source row p[i]
// (so its length is known without counting), the exclusive scan of those lengths is
// the row pointer of B (the proc_pointer of Algorithm 2), and the gather + column
// relabelling + per-row sort is the fill pass plus the Build step's sort.  There is no
// exchange: all rows live in one address space.
#include "dispatch.h"
#include "kernels.cuh"
#include "rowsort.cuh"

namespace sp {

// Scan input for the permutation: len(A[p[i], :]); records the source start of every
// output row on the way, so the fill kernels need no second lookup through p.
template <class RP, class IX>
struct PermLen {
  const RP* rowptr;
  const IX* p;
  long long m, nnz;
  long long* sstart;
  __device__ long long operator()(long long i) const {
    const long long src = p ? (long long)p[i] : i;
    long long s = 0, e = 0;
    if (src >= 0 && src < m) {
      s = (long long)rowptr[src];
      e = (long long)rowptr[src + 1];
      if (s < 0 || e < s || e > nnz) s = e = 0;
    }
    sstart[i] = s;
    return e - s;
  }
};

// Phase-1 gather of the permutation: output row r is source row p[r] (its start was
// recorded by the length scan), every column relabelled through qinv (identity when
// there is no column permutation).  A column outside [0, n) becomes the key
// 0xFFFFFFFF, which the sort reports as SP_ERR_INDEX_RANGE.
template <class CIt, class VTt, class IX>
struct PermGs {
  using CI = CIt;
  using VT = VTt;
  const CI* c_;
  const VT* v_;
  const IX* qinv;           // old column -> new column (null: identity)
  const long long* sstart;  // source start of output row r
  long long n;
  __device__ long long src(long long r) const { return sstart[r]; }
  __device__ CI col(long long pos) const { return ld_stream(c_ + pos); }
  __device__ VT val(long long pos) const { return ld_stream(v_ + pos); }
  __device__ CI map(long long, CI c) const {
    if (!qinv) return c;
    const long long cl = (long long)c;
    if (cl < 0 || cl >= n) return CI(-1);
    return CI(ld_map(qinv + cl));
  }
};

template <class RP, class CI, class VT, class IX>
sp_status permute_impl(sp_ctx* ctx, const sp_csr* A, const IX* p, const IX* q, sp_csr* B,
                       cudaStream_t s) {
  const long long m = A->nrows, n = A->ncols, nnz = A->nnz;
  const bool sym = p && q && (const void*)p == (const void*)q && m == n;
  const bool out64 = B->rowptr_type == SP_I64;
  Carver cv;
  const size_t o_qinv = cv.reserve(q ? size_t(n) * sizeof(IX) : 0);
  const size_t o_qbits = cv.reserve(q ? size_t((n + 31) / 32) * 4 : 0);
  const size_t o_pbits = cv.reserve((p && !sym) ? size_t((m + 31) / 32) * 4 : 0);
  const size_t o_vp = cv.reserve(out64 ? 0 : size_t(m + 1) * 8);
  const size_t o_scan = cv.reserve(scan_ws_bytes(m));
  const size_t o_ss = cv.reserve(size_t(m) * 8);
  size_t ro[kRowsSlots];
  rows_reserve(cv, m, nnz, sizeof(VT), ro);
  char* base;
  SP_TRY(ctx_workspace(ctx, cv.total(), s, &base));
  cv.bind(base);
  IX* qinv = q ? cv.at<IX>(o_qinv) : nullptr;
  long long* vp = out64 ? static_cast<long long*>(B->rowptr) : cv.at<long long>(o_vp);
  const int nsm = ctx->num_sms;
  // Identify: inverse column map (validates q), row permutation check (validates p)
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
  // row pointer of B: exclusive scan of the permuted row lengths
  long long* sstart = cv.at<long long>(o_ss);
  PermLen<RP, IX> len{static_cast<const RP*>(A->rowptr), p, m, nnz, sstart};
  if (out64) {
    SP_TRY(launch_scan(ctx, s, len, StoreDual<long long>{vp, nullptr, ctx->dstatus}, m,
                       cv.at<char>(o_scan)));
  } else {
    SP_TRY(launch_scan(ctx, s, len,
                       StoreDual<int32_t>{vp, static_cast<int32_t*>(B->rowptr), ctx->dstatus}, m,
                       cv.at<char>(o_scan)));
  }
  if (nnz == 0 || m == 0) return SP_OK;
  CI* out_col = static_cast<CI*>(B->colidx);
  VT* out_val = static_cast<VT*>(B->values);
  // phase 1: gather + relabel; phase 2 (a column permutation only): sort every row
  const PermGs<CI, VT, IX> g{static_cast<const CI*>(A->colidx), static_cast<const VT*>(A->values), qinv,
                             sstart, n};
  const RowsWs w = rows_bind(cv, m, nnz, ro);
  const int kb = ceil_log2_u64(uint64_t(n));
  return run_rows(ctx, s, vp, m, nnz, kb, w, &g, q != nullptr, out_col, out_val);
}

sp_status alloc_csr(sp_ctx* ctx, sp_csr* B, cudaStream_t s) {
  // caller-owned arrays are used as given; none at all means library-allocated
  const bool none = !B->rowptr && !B->colidx && !B->values;
  const bool all = B->rowptr && (B->nnz == 0 || (B->colidx && B->values));
  if (!none && !all) return SP_ERR_INVALID_ARG;
  if (all) return SP_OK;
  const size_t rb = size_t(B->nrows + 1) * itype_size(B->rowptr_type);
  B->rowptr = ctx_alloc(ctx, rb, s);
  B->colidx = ctx_alloc(ctx, size_t(B->nnz) * itype_size(B->colidx_type), s);
  B->values = ctx_alloc(ctx, size_t(B->nnz) * vtype_size(B->value_type), s);
  if (!B->rowptr || !B->colidx || !B->values) {
    ctx_free(ctx, B->rowptr, rb, s);
    ctx_free(ctx, B->colidx, 0, s);
    ctx_free(ctx, B->values, 0, s);
    B->rowptr = B->colidx = B->values = nullptr;
    return SP_ERR_OOM;
  }
  return SP_OK;
}

}  // namespace sp

using namespace sp;

extern "C" sp_status sp_permute(sp_ctx* ctx, const sp_csr* A, const void* p, const void* q,
                                sp_itype idx_type, sp_csr* B, sp_stream_t stream) {
  if (!ctx || !A || !B) return SP_ERR_INVALID_ARG;
  SP_TRY(check_csr(A));
  if (idx_type != SP_I32 && idx_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (B->rowptr_type != SP_I32 && B->rowptr_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (idx_type == SP_I32 && (A->nrows > INT32_MAX || A->ncols > INT32_MAX)) return SP_ERR_OVERFLOW;
  if (B->rowptr_type == SP_I32 && A->nnz > INT32_MAX) return SP_ERR_OVERFLOW;
  if (A->ncols > (int64_t(1) << 32)) return SP_ERR_OVERFLOW;  // 32-bit sort keys
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, SP_OP_PERMUTE, A->nnz);
  SP_TRY(validate_if_asked(ctx, A, s));
  B->nrows = A->nrows;
  B->ncols = A->ncols;
  B->nnz = A->nnz;
  B->colidx_type = A->colidx_type;
  B->value_type = A->value_type;
  const bool owned = lib_allocates(B);
  SP_TRY(alloc_csr(ctx, B, s));
  const sp_status st_ = dispatch_i(A->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(A->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(A->value_type, [&](auto vt) {
        using VT = decltype(vt);
        return dispatch_i(idx_type, [&](auto ix) {
          using IX = decltype(ix);
          return permute_impl<RP, CI, VT, IX>(ctx, A, static_cast<const IX*>(p),
                                              static_cast<const IX*>(q), B, s);
        });
      });
    });
  });
  return release_on_error(ctx, B, owned, s, st_);
}
