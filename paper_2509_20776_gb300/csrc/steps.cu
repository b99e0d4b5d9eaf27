// Steps of the path exposed on their own: inverse map, exclusive scan, per-row sort,
// canonical-form validation, and the release of library-allocated matrices.
#include "dispatch.h"
#include "kernels.cuh"
#include "rowsort.cuh"

namespace sp {

template <class RP>
struct RowLenLoad {
  const RP* rowptr;
  __device__ long long operator()(long long i) const {
    return (long long)rowptr[i + 1] - (long long)rowptr[i];
  }
};

template <class RP, class CI, class VT>
sp_status sort_rows_impl(sp_ctx* ctx, sp_csr* M, cudaStream_t s) {
  const long long m = M->nrows, nnz = M->nnz;
  Carver cv;
  const size_t o_vp = cv.reserve(size_t(m + 1) * 8);
  size_t ro[kRowsSlots];
  rows_reserve(cv, m, nnz, sizeof(VT), ro);
  char* base;
  SP_TRY(ctx_workspace(ctx, cv.total(), s, &base));
  cv.bind(base);
  long long* vp = cv.at<long long>(o_vp);
  const int nsm = ctx->num_sms;
  if (sizeof(RP) == 8) {
    SP_CUDA(cudaMemcpyAsync(vp, M->rowptr, size_t(m + 1) * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    {
      SP_PHASE(SP_PHASE_OTHER);
      k_widen<RP><<<grid_for(m + 1, 256, nsm * 8), 256, 0, s>>>(static_cast<const RP*>(M->rowptr), m + 1, vp);
    }
    SP_CUDA(cudaGetLastError());
  }
  const RowsWs w = rows_bind(cv, m, nnz, ro);
  const int kb = ceil_log2_u64(uint64_t(M->ncols));
  return run_rows<CI, VT, NoGather<CI, VT>>(ctx, s, vp, m, nnz, kb, w, nullptr, true,
                                            static_cast<CI*>(M->colidx), static_cast<VT*>(M->values));
}

// canonical-form check: one warp per row
template <class RP, class CI>
__global__ void k_validate(const RP* __restrict__ rowptr, const CI* __restrict__ col, long long m,
                           long long n, long long nnz, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (w0 == 0 && lane == 0) {
    if ((long long)rowptr[0] != 0 || (long long)rowptr[m] != nnz) dev_fail(st, SP_ERR_NOT_CANONICAL, -1);
  }
  for (long long r = w0; r < m; r += nw) {
    const long long s = (long long)rowptr[r], e = (long long)rowptr[r + 1];
    if (s < 0 || e < s || e > nnz) {
      if (lane == 0) dev_fail(st, SP_ERR_NOT_CANONICAL, r);
      continue;
    }
    bool bad = false;
    for (long long k = s + lane; k < e; k += 32) {
      const long long c = (long long)col[k];
      if (c < 0 || c >= n) bad = true;
      if (k + 1 < e && (long long)col[k + 1] <= c) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) dev_fail(st, SP_ERR_NOT_CANONICAL, r);
  }
}

}  // namespace sp

using namespace sp;

sp_status sp::validate_if_asked(sp_ctx* ctx, const sp_csr* A, cudaStream_t s) {
  if (!ctx->validate) return SP_OK;
  return sp_csr_validate(ctx, A, (sp_stream_t)s);
}

extern "C" sp_status sp_csr_validate(sp_ctx* ctx, const sp_csr* A, sp_stream_t stream) {
  if (!ctx || !A) return SP_ERR_INVALID_ARG;
  SP_TRY(check_csr(A));
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  SP_TRY(ctx_collect(ctx, s));  // report earlier device errors separately
  const long long m = A->nrows;
  sp_status st = dispatch_i(A->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(A->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      {
        SP_PHASE(SP_PHASE_OTHER);
        k_validate<RP, CI><<<grid_for(m * 32 + 32, 256, ctx->num_sms * 16), 256, 0, s>>>(
            static_cast<const RP*>(A->rowptr), static_cast<const CI*>(A->colidx), m, A->ncols,
            A->nnz, ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
      return SP_OK;
    });
  });
  SP_TRY(st);
  return ctx_collect(ctx, s);
}

extern "C" sp_status sp_inverse_map(sp_ctx* ctx, const void* idx, int64_t len, int64_t n,
                                    sp_itype idx_type, void* inv, int require_permutation,
                                    sp_stream_t stream) {
  if (!ctx || len < 0 || n < 0) return SP_ERR_INVALID_ARG;
  if ((len > 0 && !idx) || (n > 0 && !inv)) return SP_ERR_INVALID_ARG;
  if (idx_type != SP_I32 && idx_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (require_permutation && len != n) return SP_ERR_SHAPE;
  if (idx_type == SP_I32 && (n > INT32_MAX || len > INT32_MAX)) return SP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  return dispatch_i(idx_type, [&](auto ix) {
    using IX = decltype(ix);
    if (n > 0) SP_CUDA(cudaMemsetAsync(inv, 0xFF, size_t(n) * sizeof(IX), s));
    if (len > 0) {
      {
        SP_PHASE(SP_PHASE_MAP);
        k_inverse_map<IX><<<grid_for(len, 256, ctx->num_sms * 8), 256, 0, s>>>(
            static_cast<const IX*>(idx), len, n, static_cast<IX*>(inv), ctx->dstatus,
            require_permutation ? SP_ERR_NOT_PERMUTATION : SP_ERR_DUPLICATE_INDEX);
      }
      SP_CUDA(cudaGetLastError());
    }
    return SP_OK;
  });
}

extern "C" sp_status sp_exclusive_scan(sp_ctx* ctx, const void* in, sp_itype in_type, int64_t len,
                                       void* out, sp_itype out_type, sp_stream_t stream) {
  if (!ctx || len < 0 || !out || (len > 0 && !in)) return SP_ERR_INVALID_ARG;
  if ((in_type != SP_I32 && in_type != SP_I64) || (out_type != SP_I32 && out_type != SP_I64))
    return SP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  char* ws;
  SP_TRY(ctx_workspace(ctx, scan_ws_bytes(len), s, &ws));
  return dispatch_i(in_type, [&](auto it) {
    using IT = decltype(it);
    return dispatch_i(out_type, [&](auto ot) {
      using OT = decltype(ot);
      return launch_scan(ctx, s, LoadArray<IT>{static_cast<const IT*>(in)},
                         StoreTyped<OT>{static_cast<OT*>(out), ctx->dstatus}, len, ws);
    });
  });
}

extern "C" sp_status sp_sort_rows(sp_ctx* ctx, sp_csr* M, sp_stream_t stream) {
  if (!ctx || !M) return SP_ERR_INVALID_ARG;
  SP_TRY(check_csr(M));
  if (M->ncols > J_KEY_LIMIT) return SP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, -1, M->nnz);
  if (M->nnz == 0 || M->nrows == 0) return SP_OK;
  return dispatch_i(M->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(M->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(M->value_type, [&](auto vt) {
        using VT = decltype(vt);
        return sort_rows_impl<RP, CI, VT>(ctx, M, s);
      });
    });
  });
}

extern "C" sp_status sp_csr_free(sp_ctx* ctx, sp_csr* M) {
  if (!ctx || !M) return SP_ERR_INVALID_ARG;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_free(ctx, M->rowptr, 0, nullptr);
  ctx_free(ctx, M->colidx, 0, nullptr);
  ctx_free(ctx, M->values, 0, nullptr);
  M->rowptr = M->colidx = M->values = nullptr;
  return SP_OK;
}
