/*
 * Validation and calibration kernels of the metric estimator (GB300, sm_103a).
 *
 * The estimator predicts data volumes of stencil kernels without running them.  These
 * entry points run such kernels, so that the predictions can be compared with the
 * hardware counters the paper uses (L2 sectors requested by the SMs,
 * lts__t_sectors_srcunit_tex_op_read, and DRAM bytes; Sec. 3, 5.5), and measure the
 * rates a GB300 hardware descriptor needs (Sec. 3: the LOAD / SCALE streaming kernels on
 * a repeated data set give the effective L2 size and the L2 / DRAM bandwidths).
 *
 * All pointers are device pointers owned by the caller; `stream` is a cudaStream_t (NULL
 * = the legacy default stream).  Launches are asynchronous.  Returns 0 (WS_OK), -1
 * (WS_EINVAL) for malformed arguments (nothing is launched) or -6 (WS_ECUDA).
 */
#ifndef WARPSPEED_VALIDATE_H
#define WARPSPEED_VALIDATE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Streaming kernels of Sec. 3 on a repeated data set of `elems` doubles: thread g of
 * `blocks` x `threads` (the grid) touches element g mod elems, `iters` times over
 * strided rounds.  kind 0 = LOAD (c = A[i], the values combined so the loads are not
 * eliminated); kind 1 = SCALE (B[i] = c * A[i] with c = -1).  Values move as 8-byte bit
 * patterns through integer operations, so the rate measured is the transfer rate, not
 * the fp64 rate.  a, b: elems doubles; out: one double (written only in a case that
 * does not occur). */
int ws_val_stream(int kind, const double *a, double *b, double *out, int64_t elems, int blocks, int threads,
                  int iters, void *stream);

/* fp64 fused multiply-add throughput: `blocks` x `threads` threads, each running 8
 * independent chains of `iters` x 64 FMAs (2 flops each); the result is reduced into
 * out[0] only when it is negative (never, for the inputs used), so no work is dropped. */
int ws_val_fma(double *out, int blocks, int threads, int iters, void *stream);

/* 3D star stencil of radius r (1..4), fp64, on an array padded by `pad` >= r ghost
 * points on every side: for every point p of the N[0] x N[1] x N[2] domain,
 *   dst[p] = w0 * src[p] + w1 * sum over the 6r neighbours src[p + k e_d], |k| <= r, k != 0,
 * element (x, y, z) at index (z + pad) * Sy * Sx + (y + pad) * Sx + (x + pad) with
 * Sx = N[0] + 2 pad, Sy = N[1] + 2 pad.  Thread block B[3] (B[0] * B[1] * B[2] <= 1024);
 * thread folding along fold_axis (0 none, 1 y, 2 z) by `fold` consecutive points; blocks
 * in X-Y-Z order.  src and dst: Sx * Sy * (N[2] + 2 pad) doubles. */
int ws_val_star(const double *src, double *dst, const int32_t N[3], int r, const int32_t B[3], int fold_axis,
                int fold, int pad, void *stream);

/* Two-grid pull lattice-Boltzmann step over Q populations (Q <= 32), fp64: for every
 * point p, f_i = src_i[p - c_i] for all i, rho = sum f_i, dst_i[p] = f_i + omega * (rho / Q
 * - f_i).  src, dst: device arrays of Q device pointers, each array padded like
 * ws_val_star with `pad` >= 1; c: Q x 3 velocity components in {-1, 0, 1}, host memory
 * (copied).  Same block / folding / order conventions as ws_val_star. */
int ws_val_lbm(const double *const *src, double *const *dst, int Q, const int32_t *c, const int32_t N[3],
               const int32_t B[3], int fold_axis, int fold, int pad, double omega, void *stream);

/* Registers per thread of the kernel ws_val_star (kind 0, param = r) or ws_val_lbm
 * (kind 1, param = Q) launches for this folding, or -1 for an unsupported combination:
 * what the estimator needs to know to model the same resident blocks per SM. */
int ws_val_regs(int kind, int param, int fold_axis, int fold);

#ifdef __cplusplus
}
#endif
#endif
