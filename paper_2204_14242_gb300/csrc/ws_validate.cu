// Validation and calibration kernels (see include/warpspeed_validate.h): the streaming
// kernels of Sec. 3 and the two kernel families the estimator is evaluated on in Sec. 5
// (a 3D star stencil with thread folding, a pull lattice-Boltzmann step), written plainly
// so that their memory traffic is what the estimator's address model describes.
#include <cuda_runtime.h>

#include "warpspeed.h"
#include "warpspeed_validate.h"

namespace {

// ---- streaming kernels on a repeated data set (Sec. 3) -----------------------------------
// The values are moved as 8-byte bit patterns with integer operations: GB300's fp64 pipe
// is far slower than its memory system, so an fp64 add or multiply per element would
// measure the fp64 rate instead of the transfer rate.
__global__ void stream_load_kernel(const double *__restrict__ a, double *out, int64_t elems, int iters) {
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t step = T % elems;
  int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) % elems;
  const unsigned long long *p = reinterpret_cast<const unsigned long long *>(a);
  unsigned long long s = 0;
  for (int k = 0; k < iters; ++k) {
    s ^= p[i];
    i += step;
    if (i >= elems) i -= elems;
  }
  if (s == 0x7ff8dead0000beefull) out[0] = __longlong_as_double((long long)s);   // keeps the loads alive
}

__global__ void stream_scale_kernel(const double *__restrict__ a, double *__restrict__ b, int64_t elems, int iters) {
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t step = T % elems;
  int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) % elems;
  const unsigned long long *p = reinterpret_cast<const unsigned long long *>(a);
  unsigned long long *q = reinterpret_cast<unsigned long long *>(b);
  for (int k = 0; k < iters; ++k) {
    q[i] = p[i] ^ 0x8000000000000000ull;   // the sign flip, c = -1
    i += step;
    if (i >= elems) i -= elems;
  }
}

__global__ void fma_kernel(double *out, int iters) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1.0 + 1e-9 * (threadIdx.x + c);
  const double m = 0.999999, a = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 64; ++k) {
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fma(x[c], m, a);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s < 0.0) out[0] = s;
}

struct Geo {
  int32_t N[3], B[3], g[3];
  int64_t sx, sy;   // element strides of y and z (x stride 1)
  int32_t pad;
};

// First folded point of the calling thread (blocks in X-Y-Z order) and its validity.
template <int AXIS, int FOLD>
__device__ __forceinline__ bool thread_point(const Geo &G, int32_t &x, int32_t &y, int32_t &z) {
  const int32_t b = blockIdx.x;
  const int32_t bx = b % G.g[0], by = (b / G.g[0]) % G.g[1], bz = b / (G.g[0] * G.g[1]);
  const int32_t t = threadIdx.x;
  const int32_t tx = t % G.B[0], ty = (t / G.B[0]) % G.B[1], tz = t / (G.B[0] * G.B[1]);
  x = bx * G.B[0] + tx;
  y = (by * G.B[1] + ty) * (AXIS == 1 ? FOLD : 1);
  z = (bz * G.B[2] + tz) * (AXIS == 2 ? FOLD : 1);
  return x < G.N[0] && y < G.N[1] && z < G.N[2];
}

// ---- 3D star stencil, radius R, FOLD consecutive points along AXIS per thread -----------
// The folded points of a thread are unrolled with compile-time offsets, so every distinct
// source address of the thread is loaded once and reused from registers (Sec. 5.4).
template <int R, int AXIS, int FOLD>
__global__ void star_kernel(const double *__restrict__ src, double *__restrict__ dst, Geo G) {
  int32_t x, y0, z0;
  if (!thread_point<AXIS, FOLD>(G, x, y0, z0)) return;
  const double w0 = 0.5, w1 = 0.5 / (6.0 * R);
#pragma unroll
  for (int k = 0; k < FOLD; ++k) {
    const int32_t y = y0 + (AXIS == 1 ? k : 0), z = z0 + (AXIS == 2 ? k : 0);
    if (y >= G.N[1] || z >= G.N[2]) break;
    const int64_t p = (int64_t)(z + G.pad) * G.sy + (int64_t)(y + G.pad) * G.sx + (x + G.pad);
    double s = 0.0;
#pragma unroll
    for (int d = 1; d <= R; ++d)
      s += src[p - d] + src[p + d] + src[p - d * G.sx] + src[p + d * G.sx] + src[p - d * G.sy] + src[p + d * G.sy];
    dst[p] = w0 * src[p] + w1 * s;
  }
}

// ---- pull lattice-Boltzmann step over Q populations --------------------------------------
struct LbmArgs {
  const double *const *src;
  double *const *dst;
  int8_t c[32][3];
  double omega;
};

template <int Q, int AXIS, int FOLD>
__global__ void lbm_kernel(LbmArgs a, Geo G) {
  int32_t x, y0, z0;
  if (!thread_point<AXIS, FOLD>(G, x, y0, z0)) return;
#pragma unroll
  for (int k = 0; k < FOLD; ++k) {
    const int32_t y = y0 + (AXIS == 1 ? k : 0), z = z0 + (AXIS == 2 ? k : 0);
    if (y >= G.N[1] || z >= G.N[2]) break;
    const int64_t p = (int64_t)(z + G.pad) * G.sy + (int64_t)(y + G.pad) * G.sx + (x + G.pad);
    double f[Q], rho = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      f[i] = a.src[i][p - (a.c[i][0] + a.c[i][1] * G.sx + a.c[i][2] * G.sy)];
      rho += f[i];
    }
    const double eq = rho / Q;
#pragma unroll
    for (int i = 0; i < Q; ++i) a.dst[i][p] = f[i] + a.omega * (eq - f[i]);
  }
}

bool geometry(const int32_t N[3], const int32_t B[3], int fold_axis, int fold, int pad, Geo &G) {
  for (int d = 0; d < 3; ++d)
    if (N[d] < 1 || B[d] < 1) return false;
  if ((int64_t)B[0] * B[1] * B[2] > 1024 || fold_axis < 0 || fold_axis > 2 || pad < 0) return false;
  if (!(fold == 1 || fold == 2 || fold == 4) || (fold_axis == 0 && fold != 1)) return false;
  for (int d = 0; d < 3; ++d) {
    G.N[d] = N[d];
    G.B[d] = B[d];
  }
  const int32_t fy = fold_axis == 1 ? fold : 1, fz = fold_axis == 2 ? fold : 1;
  G.g[0] = (N[0] + B[0] - 1) / B[0];
  G.g[1] = (N[1] + B[1] * fy - 1) / (B[1] * fy);
  G.g[2] = (N[2] + B[2] * fz - 1) / (B[2] * fz);
  if ((int64_t)G.g[0] * G.g[1] * G.g[2] >= ((int64_t)1 << 31)) return false;
  G.sx = (int64_t)N[0] + 2 * pad;
  G.sy = G.sx * ((int64_t)N[1] + 2 * pad);
  G.pad = pad;
  return true;
}

template <int R>
cudaError_t launch_star(const double *src, double *dst, const Geo &G, int axis, int fold, cudaStream_t st) {
  const unsigned blocks = (unsigned)((int64_t)G.g[0] * G.g[1] * G.g[2]);
  const int T = G.B[0] * G.B[1] * G.B[2];
  if (axis == 0) star_kernel<R, 0, 1><<<blocks, T, 0, st>>>(src, dst, G);
  else if (axis == 1 && fold == 1) star_kernel<R, 1, 1><<<blocks, T, 0, st>>>(src, dst, G);
  else if (axis == 1 && fold == 2) star_kernel<R, 1, 2><<<blocks, T, 0, st>>>(src, dst, G);
  else if (axis == 1) star_kernel<R, 1, 4><<<blocks, T, 0, st>>>(src, dst, G);
  else if (fold == 1) star_kernel<R, 2, 1><<<blocks, T, 0, st>>>(src, dst, G);
  else if (fold == 2) star_kernel<R, 2, 2><<<blocks, T, 0, st>>>(src, dst, G);
  else star_kernel<R, 2, 4><<<blocks, T, 0, st>>>(src, dst, G);
  return cudaGetLastError();
}

template <int Q>
cudaError_t launch_lbm(const LbmArgs &a, const Geo &G, int axis, int fold, cudaStream_t st) {
  const unsigned blocks = (unsigned)((int64_t)G.g[0] * G.g[1] * G.g[2]);
  const int T = G.B[0] * G.B[1] * G.B[2];
  if (axis == 0) lbm_kernel<Q, 0, 1><<<blocks, T, 0, st>>>(a, G);
  else if (axis == 1 && fold == 1) lbm_kernel<Q, 1, 1><<<blocks, T, 0, st>>>(a, G);
  else if (axis == 1 && fold == 2) lbm_kernel<Q, 1, 2><<<blocks, T, 0, st>>>(a, G);
  else if (axis == 1) lbm_kernel<Q, 1, 4><<<blocks, T, 0, st>>>(a, G);
  else if (fold == 1) lbm_kernel<Q, 2, 1><<<blocks, T, 0, st>>>(a, G);
  else if (fold == 2) lbm_kernel<Q, 2, 2><<<blocks, T, 0, st>>>(a, G);
  else lbm_kernel<Q, 2, 4><<<blocks, T, 0, st>>>(a, G);
  return cudaGetLastError();
}

int status(cudaError_t e) { return e == cudaSuccess ? WS_OK : WS_ECUDA; }

template <class K>
int regs_of(K kernel) {
  cudaFuncAttributes at;
  return cudaFuncGetAttributes(&at, kernel) == cudaSuccess ? at.numRegs : -1;
}

template <int R>
int star_regs(int axis, int fold) {
  if (axis == 0) return regs_of(star_kernel<R, 0, 1>);
  if (axis == 1) return fold == 1 ? regs_of(star_kernel<R, 1, 1>) : fold == 2 ? regs_of(star_kernel<R, 1, 2>)
                                                                             : regs_of(star_kernel<R, 1, 4>);
  return fold == 1 ? regs_of(star_kernel<R, 2, 1>) : fold == 2 ? regs_of(star_kernel<R, 2, 2>)
                                                              : regs_of(star_kernel<R, 2, 4>);
}

template <int Q>
int lbm_regs(int axis, int fold) {
  if (axis == 0) return regs_of(lbm_kernel<Q, 0, 1>);
  if (axis == 1) return fold == 1 ? regs_of(lbm_kernel<Q, 1, 1>) : fold == 2 ? regs_of(lbm_kernel<Q, 1, 2>)
                                                                            : regs_of(lbm_kernel<Q, 1, 4>);
  return fold == 1 ? regs_of(lbm_kernel<Q, 2, 1>) : fold == 2 ? regs_of(lbm_kernel<Q, 2, 2>)
                                                             : regs_of(lbm_kernel<Q, 2, 4>);
}

}  // namespace

extern "C" int ws_val_stream(int kind, const double *a, double *b, double *out, int64_t elems, int blocks, int threads,
                             int iters, void *stream) {
  if (!a || elems < 1 || blocks < 1 || threads < 1 || threads > 1024 || iters < 1) return WS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == 0) {
    if (!out) return WS_EINVAL;
    stream_load_kernel<<<blocks, threads, 0, st>>>(a, out, elems, iters);
  } else if (kind == 1) {
    if (!b) return WS_EINVAL;
    stream_scale_kernel<<<blocks, threads, 0, st>>>(a, b, elems, iters);
  } else {
    return WS_EINVAL;
  }
  return status(cudaGetLastError());
}

extern "C" int ws_val_fma(double *out, int blocks, int threads, int iters, void *stream) {
  if (!out || blocks < 1 || threads < 1 || threads > 1024 || iters < 1) return WS_EINVAL;
  fma_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters);
  return status(cudaGetLastError());
}

extern "C" int ws_val_star(const double *src, double *dst, const int32_t N[3], int r, const int32_t B[3],
                           int fold_axis, int fold, int pad, void *stream) {
  Geo G;
  if (!src || !dst || !N || !B || r < 1 || r > 4 || pad < r || !geometry(N, B, fold_axis, fold, pad, G))
    return WS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  switch (r) {
    case 1: return status(launch_star<1>(src, dst, G, fold_axis, fold, st));
    case 2: return status(launch_star<2>(src, dst, G, fold_axis, fold, st));
    case 3: return status(launch_star<3>(src, dst, G, fold_axis, fold, st));
    case 4: return status(launch_star<4>(src, dst, G, fold_axis, fold, st));
    default: return WS_EINVAL;
  }
}

extern "C" int ws_val_lbm(const double *const *src, double *const *dst, int Q, const int32_t *c, const int32_t N[3],
                          const int32_t B[3], int fold_axis, int fold, int pad, double omega, void *stream) {
  Geo G;
  if (!src || !dst || !c || !N || !B || pad < 1 || !geometry(N, B, fold_axis, fold, pad, G)) return WS_EINVAL;
  LbmArgs a;
  a.src = src;
  a.dst = dst;
  a.omega = omega;
  for (int i = 0; i < 32; ++i)
    for (int d = 0; d < 3; ++d) a.c[i][d] = 0;
  for (int i = 0; i < Q && i < 32; ++i)
    for (int d = 0; d < 3; ++d) {
      if (c[3 * i + d] < -1 || c[3 * i + d] > 1) return WS_EINVAL;
      a.c[i][d] = (int8_t)c[3 * i + d];
    }
  cudaStream_t st = (cudaStream_t)stream;
  switch (Q) {
    case 15: return status(launch_lbm<15>(a, G, fold_axis, fold, st));
    case 19: return status(launch_lbm<19>(a, G, fold_axis, fold, st));
    case 27: return status(launch_lbm<27>(a, G, fold_axis, fold, st));
    default: return WS_EINVAL;
  }
}

extern "C" int ws_val_regs(int kind, int param, int fold_axis, int fold) {
  if (fold_axis < 0 || fold_axis > 2 || !(fold == 1 || fold == 2 || fold == 4) || (fold_axis == 0 && fold != 1))
    return -1;
  if (kind == 0) {
    switch (param) {
      case 1: return star_regs<1>(fold_axis, fold);
      case 2: return star_regs<2>(fold_axis, fold);
      case 3: return star_regs<3>(fold_axis, fold);
      case 4: return star_regs<4>(fold_axis, fold);
      default: return -1;
    }
  }
  if (kind == 1) {
    switch (param) {
      case 15: return lbm_regs<15>(fold_axis, fold);
      case 19: return lbm_regs<19>(fold_axis, fold);
      case 27: return lbm_regs<27>(fold_axis, fold);
      default: return -1;
    }
  }
  return -1;
}
