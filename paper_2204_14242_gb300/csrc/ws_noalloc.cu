// ws_estimate_batch_noalloc: the estimation of ws_estimate_batch for callers that may
// not allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc: a code generator embedded in a
// process whose device memory is owned by another runtime or pool (an inference server
// with a fixed arena, a CUDA-graph-based application that forbids allocations in its
// steady state, a plugin that must not change the host's memory footprint).  For them
// every device buffer of one estimation -- compiled descriptors, counters, sector
// bitmaps, results and ranking -- is carved from the fixed array below, which the CUDA
// runtime reserves when this library's device code is loaded and keeps until the
// process exits.  The call creates no CUDA resource: no cudaMalloc, cudaMallocAsync,
// cudaFree, cudaHostAlloc, stream or event (ws_resource_counts_get shows it).  Its host
// memory is plain heap memory: the descriptor compiler's containers and the pageable
// arrays the descriptors are uploaded from (page-locked blocks are used only when an
// earlier plan left one in the library's cache).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "ws_host.h"

namespace {

// The fixed device scratch.  In host code `g_noalloc_scratch` only names a host-side
// stand-in of the symbol: its device address must be obtained with
// cudaGetSymbolAddress on the device that runs the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[WS_NOALLOC_SCRATCH_BYTES];

struct NoallocDevice {
  std::mutex mu;           // serialises the calls on this device (they share the array)
  bool ready = false;
  ws_ctx ctx;              // wraps the fixed scratch; owns no stream and no allocation
  ws::Arena *arena = nullptr;
};

NoallocDevice g_dev[64];

// Once per device, with that device current: device address of the scratch array and
// the SM count.  Returns WS_OK or WS_ECUDA.  Called with the device's lock held.
int setup(int device) {
  NoallocDevice &d = g_dev[device];
  if (d.ready) return WS_OK;
  void *ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) {
    ws::set_error(std::string("cudaGetSymbolAddress of the no-alloc scratch: ") + cudaGetErrorString(e));
    return WS_ECUDA;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    ws::set_error(std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    return WS_ECUDA;
  }
  d.arena = new ws::Arena((char *)ptr, WS_NOALLOC_SCRATCH_BYTES);
  d.ctx.device = device;
  d.ctx.sm_count = sms;
  d.ctx.owns_arena = false;
  d.ctx.arena = d.arena;
  d.ctx.no_events = true;   // uploads and launches share the caller's stream
  d.ready = true;
  return WS_OK;
}

// Puts the caller's current device back on every return path.
struct CurrentDevice {
  int prev = -1;
  CurrentDevice() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~CurrentDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" int ws_estimate_batch_noalloc(int device, const ws_config *cfgs, int n_cfg, const ws_field *fld,
                                         int n_fld, const ws_access *acc, int n_acc, const ws_hw *hw,
                                         ws_result *out, int32_t *order_out, void *stream) {
  if (device < 0 || device >= 64 || !hw || n_cfg < 0 || (n_cfg > 0 && (!cfgs || !out))) return WS_EINVAL;
  const CurrentDevice keep;
  NoallocDevice &d = g_dev[device];
  std::lock_guard<std::mutex> g(d.mu);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    ws::set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return WS_ECUDA;
  }
  int rc = setup(device);
  if (rc != WS_OK) return rc;
  d.ctx.stream = (cudaStream_t)stream;          // the caller's stream (NULL = legacy default)
  d.ctx.capture_stream = (cudaStream_t)stream;  // unused: this path launches directly
  const ws::NoPinnedScope pageable;             // upload arrays from plain host memory
  ws_plan *p = nullptr;
  // one compile: the plan takes the descriptors from the array, then its bitmaps (in as
  // many passes as needed) and clears them before use, so leftovers of earlier calls
  // (including failed ones) never leak into this one
  rc = ws::plan_create_impl(&d.ctx, cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, nullptr, 0, nullptr, 0, &p, nullptr,
                            -1, 0);
  const std::string too_big = "the batch's descriptors and largest field do not fit the no-alloc entry point's fixed " +
                              std::to_string((size_t)WS_NOALLOC_SCRATCH_BYTES) + " bytes of device scratch";
  if (rc == WS_ENOMEM) {
    ws::set_error(too_big);
    return rc;
  }
  if (rc != WS_OK) return rc;
  // a field whose bitmaps alone exceed what the array has left for scratch: refuse the
  // batch before any kernel runs
  for (int i = 0; i < n_cfg; ++i)
    if (p->up_cfg[(size_t)i].status == WS_ENOMEM) {
      ws_plan_destroy(p);
      ws::set_error(too_big);
      return WS_ENOMEM;
    }
  rc = p->execute(WS_MODE_DIRECT, (cudaStream_t)stream);
  if (rc == WS_OK) rc = ws_plan_results(p, out, order_out, stream);
  ws_plan_destroy(p);
  return rc;
}
