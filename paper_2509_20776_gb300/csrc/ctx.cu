// Context lifecycle, allocator hook, workspace arena and device error reporting.
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <new>

#include "internal.h"

using namespace sp;

namespace sp {

void* ctx_alloc(sp_ctx* ctx, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 1;
  if (!ctx->default_alloc) return ctx->alloc.alloc(ctx->alloc.user, bytes, s);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void ctx_free(sp_ctx* ctx, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (!ctx->default_alloc) {
    ctx->alloc.free(ctx->alloc.user, p, bytes, s);
    return;
  }
  cudaFreeAsync(p, s);
}

sp_status ctx_workspace(sp_ctx* ctx, size_t bytes, cudaStream_t s, char** base) {
  if (bytes <= ctx->ws_cap) {
    *base = ctx->ws;
    return SP_OK;
  }
  size_t cap = bytes + bytes / 4;
  // release the old arena after the work already queued on its stream
  if (ctx->ws) ctx_free(ctx, ctx->ws, ctx->ws_cap, s);
  ctx->ws = static_cast<char*>(ctx_alloc(ctx, cap, s));
  if (!ctx->ws) {
    ctx->ws_cap = 0;
    return SP_ERR_OOM;
  }
  ctx->ws_cap = cap;
  ctx->ws_stream = s;
  *base = ctx->ws;
  return SP_OK;
}

sp_status ctx_collect(sp_ctx* ctx, cudaStream_t s) {
  SP_CUDA(cudaMemcpyAsync(ctx->hstatus, ctx->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaStreamSynchronize(s));
  DevStatus h = *ctx->hstatus;
  if (h.code != 0) {
    ctx->last_detail = h.detail;
    SP_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(DevStatus), s));
    SP_CUDA(cudaStreamSynchronize(s));
    return sp_status(h.code);
  }
  return SP_OK;
}

cudaEvent_t ctx_event(sp_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

sp_status check_csr(const sp_csr* A, bool allow_null_arrays) {
  if (!A) return SP_ERR_INVALID_ARG;
  if (A->nrows < 0 || A->ncols < 0 || A->nnz < 0) return SP_ERR_SHAPE;
  if ((A->rowptr_type != SP_I32 && A->rowptr_type != SP_I64) ||
      (A->colidx_type != SP_I32 && A->colidx_type != SP_I64) ||
      (A->value_type != SP_F32 && A->value_type != SP_F64))
    return SP_ERR_INVALID_ARG;
  if (!allow_null_arrays) {
    if (!A->rowptr) return SP_ERR_INVALID_ARG;
    if (A->nnz > 0 && (!A->colidx || !A->values)) return SP_ERR_INVALID_ARG;
  }
  if (A->rowptr_type == SP_I32 && A->nnz > INT32_MAX) return SP_ERR_OVERFLOW;
  if (A->colidx_type == SP_I32 && A->ncols > (int64_t(1) << 31)) return SP_ERR_OVERFLOW;
  return SP_OK;
}

}  // namespace sp

namespace sp {
namespace {
thread_local int t_cuda_err = 0;
thread_local char t_cuda_where[160] = "";
}  // namespace
void note_cuda_error(cudaError_t e, const char* file, int line) {
  t_cuda_err = int(e);
  const char* base = strrchr(file, '/');
  snprintf(t_cuda_where, sizeof(t_cuda_where), "%s:%d (%s)", base ? base + 1 : file, line, cudaGetErrorName(e));
}
}  // namespace sp

extern "C" {

const char* sp_status_str(sp_status s) {
  switch (s) {
    case SP_OK: return "SP_OK";
    case SP_ERR_INVALID_ARG: return "SP_ERR_INVALID_ARG";
    case SP_ERR_SHAPE: return "SP_ERR_SHAPE";
    case SP_ERR_INDEX_RANGE: return "SP_ERR_INDEX_RANGE";
    case SP_ERR_DUPLICATE_INDEX: return "SP_ERR_DUPLICATE_INDEX";
    case SP_ERR_NOT_PERMUTATION: return "SP_ERR_NOT_PERMUTATION";
    case SP_ERR_NOT_CANONICAL: return "SP_ERR_NOT_CANONICAL";
    case SP_ERR_OVERFLOW: return "SP_ERR_OVERFLOW";
    case SP_ERR_OOM: return "SP_ERR_OOM";
    case SP_ERR_TIMEOUT: return "SP_ERR_TIMEOUT";
    case SP_ERR_CUDA: return "SP_ERR_CUDA";
    case SP_ERR_INTERNAL: return "SP_ERR_INTERNAL";
  }
  return "SP_ERR_UNKNOWN";
}

int sp_version(void) { return 100; }

sp_status sp_ctx_create(sp_ctx** out, int device, const sp_allocator* allocator) {
  if (!out) return SP_ERR_INVALID_ARG;
  *out = nullptr;
  if (allocator && (!allocator->alloc || !allocator->free)) return SP_ERR_INVALID_ARG;
  SP_CUDA(cudaSetDevice(device));
  sp_ctx* ctx = new (std::nothrow) sp_ctx();
  if (!ctx) return SP_ERR_OOM;
  ctx->device = device;
  if (allocator) {
    ctx->alloc = *allocator;
    ctx->default_alloc = false;
  } else {
    // keep freed blocks in this process's stream-ordered pool between calls instead of
    // returning them to the driver at every synchronisation (plans take GBs per call)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      unsigned long long keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&ctx->dstatus, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&ctx->hstatus, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&ctx->hbuf, 16 * sizeof(long long)) != cudaSuccess ||
      cudaMemset(ctx->dstatus, 0, sizeof(DevStatus)) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->dstatus) cudaFree(ctx->dstatus);
    if (ctx->hstatus) cudaFreeHost(ctx->hstatus);
    if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    delete ctx;
    return SP_ERR_CUDA;
  }
  *out = ctx;
  return SP_OK;
}

sp_status sp_ctx_destroy(sp_ctx* ctx) {
  if (!ctx) return SP_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) ctx_free(ctx, ctx->ws, ctx->ws_cap, ctx->ws_stream);
  cudaDeviceSynchronize();
  cudaFree(ctx->dstatus);
  cudaFreeHost(ctx->hstatus);
  cudaFreeHost(ctx->hbuf);
  cudaStreamDestroy(ctx->side);
  cudaEventDestroy(ctx->fork_ev);
  cudaEventDestroy(ctx->join_ev);
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
  return SP_OK;
}

sp_status sp_ctx_sync(sp_ctx* ctx, sp_stream_t stream) {
  if (!ctx) return SP_ERR_INVALID_ARG;
  SP_CUDA(cudaSetDevice(ctx->device));
  return ctx_collect(ctx, (cudaStream_t)stream);
}

int64_t sp_ctx_error_detail(const sp_ctx* ctx) { return ctx ? ctx->last_detail : -1; }


int sp_last_cuda_error(const char** where) {
  if (where) *where = sp::t_cuda_where;
  return sp::t_cuda_err;
}

sp_status sp_ctx_set_option(sp_ctx* ctx, sp_option key, int64_t value) {
  if (!ctx) return SP_ERR_INVALID_ARG;
  switch (key) {
    case SP_OPT_SPIN_LIMIT: ctx->spin_limit = value < 0 ? (int64_t(1) << 22) : value; return SP_OK;
    case SP_OPT_SCAN_HOLD_TILE: ctx->hold_tile = value < 0 ? -1 : value; return SP_OK;
    case SP_OPT_VALIDATE: ctx->validate = value > 0 ? 1 : 0; return SP_OK;
    case SP_OPT_TIMING: ctx->timing = value > 0 ? 1 : 0; return SP_OK;
    case SP_OPT_TILE_SHAPE:
      if (value > 1) return SP_ERR_INVALID_ARG;
      ctx->opt.tile_shape = value < 0 ? 0 : int(value);
      return SP_OK;
    case SP_OPT_HEAVY:
      if (value >= 0 && (value < 128 || value > 4096)) return SP_ERR_INVALID_ARG;
      ctx->opt.heavy = value < 0 ? 128 : int(value);
      return SP_OK;
    case SP_OPT_COUNT_ROWS:
      if (value == 0 || value > 4) return SP_ERR_INVALID_ARG;
      ctx->opt.count_rows = value < 0 ? 4 : int(value);
      return SP_OK;
    case SP_OPT_FILL_ROWS:
      if (value == 0 || value > 2) return SP_ERR_INVALID_ARG;
      ctx->opt.fill_rows = value < 0 ? 2 : int(value);
      return SP_OK;
    case SP_OPT_BATCH_ROWS:
      if (value >= 0 && value != 1 && value != 2 && value != 4 && value != 8) return SP_ERR_INVALID_ARG;
      ctx->opt.batch_rows = value < 0 ? 1 : int(value);
      return SP_OK;
    case SP_OPT_IDENTIFY:
      if (value > 1) return SP_ERR_INVALID_ARG;
      ctx->opt.identify = value < 0 ? 0 : int(value);
      return SP_OK;
    case SP_OPT_OVERLAP:
      if (value > 1) return SP_ERR_INVALID_ARG;
      ctx->overlap = value < 0 ? 1 : int(value);
      return SP_OK;
  }
  return SP_ERR_INVALID_ARG;
}

int sp_tuning_lookup(const sp_tune_entry* table, int n, int op, int64_t size, sp_tune_entry* out) {
  if (n < 0 || (n > 0 && !table) || !out) return -1;
  for (int i = 0; i < n; ++i) {
    if (table[i].op != op || size > table[i].size_max) continue;
    *out = table[i];
    return 1;
  }
  return 0;
}

sp_status sp_ctx_set_tuning(sp_ctx* ctx, const sp_tune_entry* table, int n) {
  if (!ctx || n < 0 || (n > 0 && !table)) return SP_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const sp_tune_entry& e = table[i];
    const bool ok = e.op >= SP_OP_PERMUTE && e.op <= SP_OP_BATCH && e.tile_shape <= 1 &&
                    (e.heavy < 0 || (e.heavy >= 128 && e.heavy <= 4096)) && e.count_rows != 0 &&
                    e.count_rows <= 4 && e.fill_rows != 0 && e.fill_rows <= 2 &&
                    (e.batch_rows < 0 || e.batch_rows == 1 || e.batch_rows == 2 || e.batch_rows == 4 ||
                     e.batch_rows == 8) &&
                    e.identify <= 1;
    if (!ok) return SP_ERR_INVALID_ARG;
  }
  ctx->tuning.assign(table, table + n);
  return SP_OK;
}

sp_status sp_ctx_phase_stats(sp_ctx* ctx, double* ms, int64_t* launches, int reset) {
  if (!ctx) return SP_ERR_INVALID_ARG;
  SP_CUDA(cudaSetDevice(ctx->device));
  static const bool trace = std::getenv("SP_TRACE") != nullptr;
  for (auto& p : ctx->pending) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess)
      ctx->phase_ms[p.phase] += t;
    else
      cudaGetLastError();
    if (trace) std::fprintf(stderr, "[sp trace] %-9s %10.4f ms\n", sp_phase_name(p.phase), t);
    ctx->ev_pool.push_back(p.a);
    ctx->ev_pool.push_back(p.b);
  }
  ctx->pending.clear();
  for (int i = 0; i < SP_NUM_PHASES; ++i) {
    if (ms) ms[i] = ctx->phase_ms[i];
    if (launches) launches[i] = ctx->phase_launches[i];
    if (reset) {
      ctx->phase_ms[i] = 0;
      ctx->phase_launches[i] = 0;
    }
  }
  return SP_OK;
}

const char* sp_phase_name(int phase) {
  static const char* names[SP_NUM_PHASES] = {"map", "count", "scan", "partition", "tile",
                                             "long", "huge", "gather", "other"};
  return (phase >= 0 && phase < SP_NUM_PHASES) ? names[phase] : "?";
}

}  // extern "C"
