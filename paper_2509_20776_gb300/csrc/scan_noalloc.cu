// Exclusive scan that allocates nothing: the look-back scan of scan.cuh with its
// tile-status words, tile ticket and error record held in a fixed-size file-scope
// device array instead of context workspace.
//
// Who needs this: code that cannot call cudaMalloc / cudaMallocAsync at the moment it
// needs a prefix sum -- a device-memory allocator doing its own bookkeeping (it cannot
// recurse into itself), a service that reserved all device memory up front and may not
// grow, or a latency-critical loop that must not pay for (or implicitly synchronise
// on) an allocation.  Such callers cannot create an sp_ctx either (its error record is
// allocated), so this entry point takes no context.
#include <mutex>

#include "dispatch.h"
#include "scan.cuh"

namespace sp {

constexpr long long kNoAllocMaxLen = 1ll << 28;  // 268,435,456 inputs
constexpr long long kNoAllocMaxTiles = (kNoAllocMaxLen + SCAN_TILE - 1) / SCAN_TILE;
constexpr size_t kNoAllocStatusBytes = size_t(kNoAllocMaxTiles + 1) * 8;
constexpr size_t kNoAllocBytes = kNoAllocStatusBytes + 256;  // + ticket and error record

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_scan_scratch[kNoAllocBytes];

namespace {
std::mutex g_setup_mu;
void* g_scratch_addr[256] = {};  // device address of g_scan_scratch, per device ordinal
}  // namespace

// Device address of the scratch array for the current device (looked up once per
// device; the host-side symbol itself is not a device address).
static sp_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  SP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return SP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SP_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return SP_OK;
}

}  // namespace sp

using namespace sp;

extern "C" sp_status sp_exclusive_scan_noalloc(const void* in, sp_itype in_type, int64_t len,
                                               void* out, sp_itype out_type,
                                               sp_stream_t stream) {
  if (len < 0 || !out || (len > 0 && !in)) return SP_ERR_INVALID_ARG;
  if ((in_type != SP_I32 && in_type != SP_I64) || (out_type != SP_I32 && out_type != SP_I64))
    return SP_ERR_INVALID_ARG;
  if (len > kNoAllocMaxLen) return SP_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* scratch = nullptr;
  SP_TRY(scratch_for_current_device(&scratch));
  long long tiles = (len + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 0) tiles = 1;
  ScanCtl c;
  c.status = reinterpret_cast<unsigned long long*>(scratch);
  c.ticket = reinterpret_cast<unsigned*>(scratch + kNoAllocStatusBytes);
  c.st = reinterpret_cast<DevStatus*>(scratch + kNoAllocStatusBytes + 64);
  c.spin_limit = int64_t(1) << 22;
  c.hold_tile = -1;
  c.n = len;
  // the array keeps the previous call's contents: clear the status words in use, the
  // ticket and the error record
  SP_CUDA(cudaMemsetAsync(scratch, 0, size_t(tiles) * 8, s));
  SP_CUDA(cudaMemsetAsync(scratch + kNoAllocStatusBytes, 0, 256, s));
  sp_status st = dispatch_i(in_type, [&](auto it) {
    using IT = decltype(it);
    return dispatch_i(out_type, [&](auto ot) {
      using OT = decltype(ot);
      k_scan<<<unsigned(tiles), SCAN_BLOCK, 0, s>>>(LoadArray<IT>{static_cast<const IT*>(in)},
                                                   StoreTyped<OT>{static_cast<OT*>(out), c.st}, c);
      SP_CUDA(cudaGetLastError());
      return SP_OK;
    });
  });
  SP_TRY(st);
  DevStatus h{};
  SP_CUDA(cudaMemcpyAsync(&h, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaStreamSynchronize(s));
  return h.code ? sp_status(h.code) : SP_OK;
}
