// Host-side internals shared by the translation units of the library: the context,
// its workspace arena, status plumbing and the type dispatch used by every op.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "sp.h"

struct sp_ctx {
  int device = 0;
  int num_sms = 0;
  sp_allocator alloc{};
  bool default_alloc = true;
  // grow-only workspace shared by the calls made through this context
  char* ws = nullptr;
  size_t ws_cap = 0;
  cudaStream_t ws_stream = nullptr;
  sp::DevStatus* dstatus = nullptr;  // device error record
  sp::DevStatus* hstatus = nullptr;  // pinned host mirror
  // pinned host scratch for the totals a synchronising call reads back (16 words); one
  // buffer per context, so no call allocates page-locked memory (which would stop kernels
  // on other streams from running concurrently with later work)
  long long* hbuf = nullptr;
  // a second stream of this context (highest priority) and the events that fork work onto
  // it and join it back; overlap = 0 keeps every launch on the caller's stream
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int overlap = 1;
  int64_t spin_limit = int64_t(1) << 22;
  int64_t hold_tile = -1;
  int validate = 0;
  int64_t last_detail = -1;
  // tracing: launches per phase, and (with timing on) event pairs per launch
  int timing = 0;
  struct Pending {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  double phase_ms[SP_NUM_PHASES] = {};
  long long phase_launches[SP_NUM_PHASES] = {};
  // kernel shapes: the context's options, the tuning table, and the values in force for
  // the call being issued (options overridden by the table entry that covers the call)
  struct Shapes {
    int tile_shape = 0, heavy = 128, count_rows = 4, fill_rows = 2, batch_rows = 1, identify = 0;
  };
  Shapes opt, cur;
  std::vector<sp_tune_entry> tuning;
};

namespace sp {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

inline size_t itype_size(sp_itype t) { return t == SP_I64 ? 8 : 4; }
inline size_t vtype_size(sp_vtype t) { return t == SP_F64 ? 8 : 4; }

// The CUDA error behind the calling thread's most recent SP_ERR_CUDA, and where.
void note_cuda_error(cudaError_t e, const char* file, int line);

#define SP_CUDA(call)                                     \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      ::sp::note_cuda_error(e_, __FILE__, __LINE__);      \
      return SP_ERR_CUDA;                                 \
    }                                                     \
  } while (0)

#define SP_TRY(call)                                      \
  do {                                                    \
    sp_status s_ = (call);                                \
    if (s_ != SP_OK) return s_;                           \
  } while (0)

void* ctx_alloc(sp_ctx* ctx, size_t bytes, cudaStream_t s);
void ctx_free(sp_ctx* ctx, void* p, size_t bytes, cudaStream_t s);

// Carves 256-byte aligned slices from one allocation.  Sizes are first declared
// (reserve), then the backing store is obtained once (commit), then slices are taken
// in the same order (take).
class Carver {
 public:
  size_t reserve(size_t bytes) {
    size_t off = total_;
    total_ += align_up(bytes ? bytes : 1);
    return off;
  }
  size_t total() const { return total_; }
  void bind(char* base) { base_ = base; }
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(base_ + off); }

 private:
  size_t total_ = 0;
  char* base_ = nullptr;
};

// Ensure the context workspace holds at least `bytes`; returns its base.
sp_status ctx_workspace(sp_ctx* ctx, size_t bytes, cudaStream_t s, char** base);

// After a synchronising point: read, clear and return the device error record.
sp_status ctx_collect(sp_ctx* ctx, cudaStream_t s);

inline int grid_for(int64_t work, int block, int cap) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return int(g);
}

sp_status check_csr(const sp_csr* A, bool allow_null_arrays = false);

// Scope around one kernel launch: counts it under `phase` and, with timing on, records
// CUDA events before and after it on the launching stream.
cudaEvent_t ctx_event(sp_ctx* ctx);
struct PhaseScope {
  sp_ctx* ctx;
  cudaStream_t s;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseScope(sp_ctx* c, cudaStream_t st, int ph) : ctx(c), s(st), phase(ph) {
    ctx->phase_launches[ph]++;
    if (ctx->timing) {
      a = ctx_event(ctx);
      if (a) cudaEventRecord(a, s);
    }
  }
  ~PhaseScope() {
    if (!a) return;
    cudaEvent_t b = ctx_event(ctx);
    if (!b) return;
    cudaEventRecord(b, s);
    ctx->pending.push_back({phase, a, b});
  }
};
#define SP_PHASE(ph) ::sp::PhaseScope sp_phase_scope_##__LINE__(ctx, s, ph)

// Allocate B's arrays through the context allocator when all three are NULL.
sp_status alloc_csr(sp_ctx* ctx, sp_csr* B, cudaStream_t s);

// A call that allocated its output (`owned`) and then failed releases it (stream-ordered
// after the work already queued on s) and zeroes the pointers; returns st.
inline sp_status release_on_error(sp_ctx* ctx, sp_csr* B, bool owned, cudaStream_t s, sp_status st) {
  if (st == SP_OK || !owned) return st;
  ctx_free(ctx, B->rowptr, 0, s);
  ctx_free(ctx, B->colidx, 0, s);
  ctx_free(ctx, B->values, 0, s);
  B->rowptr = B->colidx = B->values = nullptr;
  return st;
}
inline bool lib_allocates(const sp_csr* B) { return !B->rowptr && !B->colidx && !B->values; }

// With SP_OPT_VALIDATE set, check A is canonical (synchronises); else SP_OK.
sp_status validate_if_asked(sp_ctx* ctx, const sp_csr* A, cudaStream_t s);

// Shapes for the call about to be issued: the context's options, overridden by the
// first tuning-table entry of `op` that covers `size` (op < 0: no table lookup).
inline void ctx_begin_call(sp_ctx* ctx, int op, long long size) {
  ctx->cur = ctx->opt;
  sp_tune_entry e;
  if (op < 0 || sp_tuning_lookup(ctx->tuning.data(), int(ctx->tuning.size()), op, size, &e) != 1) return;
  if (e.tile_shape >= 0) ctx->cur.tile_shape = e.tile_shape;
  if (e.heavy >= 0) ctx->cur.heavy = e.heavy;
  if (e.count_rows >= 0) ctx->cur.count_rows = e.count_rows;
  if (e.fill_rows >= 0) ctx->cur.fill_rows = e.fill_rows;
  if (e.batch_rows >= 0) ctx->cur.batch_rows = e.batch_rows;
  if (e.identify >= 0) ctx->cur.identify = e.identify;
}

}  // namespace sp
