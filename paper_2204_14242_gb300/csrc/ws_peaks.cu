// Microbenchmarks of the device rates that bound the enumeration kernel: 32-bit integer
// add throughput (the address arithmetic) and L2 red.or throughput on distinct words
// (the bitmap inserts).  They give the roofline denominators measured on the device
// the estimator runs on.
#include <cuda_runtime.h>

#include <cstring>

#include "ws_host.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void int_add_kernel(uint32_t *out, int iters, uint32_t seed) {
  uint32_t x[kChains], y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = threadIdx.x * (c + 3) + seed;
    y[c] = blockIdx.x ^ (seed + c);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = x[c] + y[(c + k) % kChains];
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) y[c] ^= x[c];
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c] + y[c];
  if (s == 0x9e3779b9u) out[0] = s;
}

__global__ void l2_red_kernel(uint32_t *buf, uint32_t words_mask, int iters) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t idx = tid * 2654435761u;
  for (int i = 0; i < iters; ++i) {
    atomicOr(buf + (idx & words_mask), 1u << (i & 31));
    idx += 0x9e3779b9u;
  }
}

// The row walk's pattern: every lane sets a run of kRun consecutive 64-bit units (one
// sector range) at its own place, 64-bit red.or per unit; lanes of a warp are far apart.
constexpr int kRun = 3;
__global__ void l2_red64_runs_kernel(unsigned long long *buf, uint32_t units_mask, int iters) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t idx = tid * 2654435761u;
  for (int i = 0; i < iters; ++i) {
    const uint32_t u0 = idx & units_mask & ~7u;
#pragma unroll
    for (int r = 0; r < kRun; ++r) atomicOr(buf + u0 + r, 1ull << ((i + r) & 63));
    idx += 0x9e3779b9u;
  }
}

}  // namespace

extern "C" int ws_measure_peaks(ws_ctx *ctx, double *int_ops_per_s, double *l2_red_per_s) {
  ws_peaks pk;
  const int rc = ws_measure_peaks2(ctx, &pk);
  if (rc == WS_OK) {
    if (int_ops_per_s) *int_ops_per_s = pk.int_ops_per_s;
    if (l2_red_per_s) *l2_red_per_s = pk.l2_red_per_s;
  }
  return rc;
}

extern "C" int ws_measure_peaks2(ws_ctx *ctx, ws_peaks *pk) {
  if (!ctx || !pk) return WS_EINVAL;
  memset(pk, 0, sizeof(*pk));
  double *int_ops_per_s = &pk->int_ops_per_s, *l2_red_per_s = &pk->l2_red_per_s;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return WS_ECUDA;
  const size_t red_words = (size_t)16 << 20;  // 64 MiB: inside L2
  int64_t o_out = ctx->arena->alloc(256), o_buf = ctx->arena->alloc(red_words * 4);
  if (o_out < 0 || o_buf < 0) {
    ctx->arena->release(o_out);
    ctx->arena->release(o_buf);
    return WS_ENOMEM;
  }
  uint32_t *out = (uint32_t *)(ctx->arena->base + o_out);
  uint32_t *buf = (uint32_t *)(ctx->arena->base + o_buf);
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ws::count_resource(ws::RES_EVENT);
  ws::count_resource(ws::RES_EVENT);
  const int blocks = ctx->sm_count * 8, threads = 256;
  float best_int = 1e30f, best_red = 1e30f, best_run = 1e30f;
  const int int_iters = 4096, red_iters = 256, run_iters = 128;
  cudaMemsetAsync(buf, 0, red_words * 4, st);
  for (int r = 0; r < 4; ++r) {
    float ms = 0;
    cudaEventRecord(e0, st);
    int_add_kernel<<<blocks, threads, 0, st>>>(out, int_iters, 12345u + r);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best_int = ms < best_int ? ms : best_int;
    cudaEventRecord(e0, st);
    l2_red_kernel<<<blocks, threads, 0, st>>>(buf, (uint32_t)(red_words - 1), red_iters);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best_red = ms < best_red ? ms : best_red;
    cudaEventRecord(e0, st);
    // units u0 .. u0 + kRun - 1 with u0 a multiple of 8 below red_words / 2 - 8: inside the buffer
    l2_red64_runs_kernel<<<blocks, threads, 0, st>>>((unsigned long long *)buf, (uint32_t)(red_words / 2 - 8),
                                                      run_iters);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best_run = ms < best_run ? ms : best_run;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->arena->release(o_out);
  ctx->arena->release(o_buf);
  if (e != cudaSuccess) {
    ws::set_error(cudaGetErrorString(e));
    return WS_ECUDA;
  }
  const double n_threads = (double)blocks * threads;
  *int_ops_per_s = n_threads * int_iters * (double)(kChains * kUnroll + kChains) / (best_int * 1e-3);
  *l2_red_per_s = n_threads * red_iters / (best_red * 1e-3);
  pk->l2_red64_run_per_s = n_threads * run_iters * kRun / (best_run * 1e-3);
  return WS_OK;
}
