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
// process exits.  No cudaMalloc, cudaMallocAsync, cudaFree, stream creation or
// library allocator is called; the only host allocations are the descriptor
// compiler's temporary host containers.
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
  bool ready = false;
  ws_ctx ctx;              // wraps the fixed scratch; owns no stream and no allocation
  ws::Arena *arena = nullptr;
};

std::mutex g_mu;
NoallocDevice g_dev[64];

// Once per device, with that device current: device address of the scratch array and
// the SM count.  Returns WS_OK or WS_ECUDA.
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
  d.ready = true;
  return WS_OK;
}

}  // namespace

extern "C" int ws_estimate_batch_noalloc(int device, const ws_config *cfgs, int n_cfg, const ws_field *fld,
                                         int n_fld, const ws_access *acc, int n_acc, const ws_hw *hw,
                                         ws_result *out, int32_t *order_out, void *stream) {
  if (device < 0 || device >= 64 || !hw || n_cfg < 0 || (n_cfg > 0 && (!cfgs || !out))) return WS_EINVAL;
  std::lock_guard<std::mutex> g(g_mu);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    ws::set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return WS_ECUDA;
  }
  int rc = setup(device);
  if (rc != WS_OK) return rc;
  // size check before any device work: descriptors, the largest field's bitmaps (the
  // batch runs in as many passes as needed) and the plan's 8 MiB of headroom must fit
  // the fixed scratch
  size_t desc = 0, scratch = 0, max_field = 0;
  ws::plan_requirements(cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, &desc, &scratch, &max_field);
  if (desc + max_field + ((size_t)8 << 20) > (size_t)WS_NOALLOC_SCRATCH_BYTES) {
    ws::set_error("request needs " + std::to_string(desc + max_field) + " bytes of device scratch; the no-alloc "
                  "entry point has a fixed " + std::to_string((size_t)WS_NOALLOC_SCRATCH_BYTES) + " bytes");
    return WS_ENOMEM;
  }
  NoallocDevice &d = g_dev[device];
  d.ctx.stream = (cudaStream_t)stream;          // the caller's stream (NULL = legacy default)
  d.ctx.capture_stream = (cudaStream_t)stream;  // unused: this path launches directly
  ws_plan *p = nullptr;
  // the plan clears its bitmap scratch before use, so leftovers of earlier calls
  // (including failed ones) never leak into this one
  rc = ws::plan_create_impl(&d.ctx, cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, nullptr, 0, nullptr, 0, &p, nullptr,
                            -1, 0);
  if (rc != WS_OK) return rc;
  rc = p->execute(WS_MODE_DIRECT, (cudaStream_t)stream);
  if (rc == WS_OK) rc = ws_plan_results(p, out, order_out, stream);
  ws_plan_destroy(p);
  return rc;
}
