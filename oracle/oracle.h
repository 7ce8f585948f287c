/*
 * CPU oracle of the metric estimator (test infrastructure only).
 *
 * Plain, slow, obviously correct: every thread's addresses are walked into
 * std::set containers of 32 B sectors and 128 B lines per level (Sec. 4.2-4.4 of
 * the paper), and the capacity and performance model is evaluated in fp64.
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load this library.  It shares no code, header or constant with the CUDA path.
 *
 * Flat input layout (all arrays row-major, one row per item):
 *   cfg_i [n_cfg][ORC_CFG_NI] int64:
 *       Nx Ny Nz Bx By Bz fold_axis(0 none,1 y,2 z) fold n_field field_off
 *       regs_per_thread wave_blocks_override address_mode(0 linear, 1 multi-dimensional)
 *   cfg_d [n_cfg] double: flops per lattice update
 *   fld_i [..][ORC_FLD_NI] int64:
 *       elem_bytes align sx sy sz const_off n_access access_off
 *   acc_i [..][ORC_ACC_NI] int64: dx dy dz is_store dc
 *   hw_d  [ORC_HW_ND] double:
 *       sms max_threads_sm max_blocks_sm regs_sm clock_hz l1_bytes l2_bytes bw_l2
 *       bw_dram fp_peak banks bank_bytes pair_dist_bytes capacity_model
 *       hit[4][3] (a b c for L1, L2-y, L2-z, L2-store)
 * Flat outputs: out_i [n_cfg][ORC_OUT_NI] int64, out_d [n_cfg][ORC_OUT_ND] double,
 * column meaning given by the ORC_I_* / ORC_D_* indices below.
 */
#ifndef WS_ORACLE_H
#define WS_ORACLE_H
#include <stdint.h>

#define ORC_CFG_NI 13
#define ORC_FLD_NI 8
#define ORC_ACC_NI 5
#define ORC_HW_ND 26

enum {
  ORC_I_STATUS, ORC_I_LUPS_BLOCK, ORC_I_LUPS_WAVE, ORC_I_L1_REQ, ORC_I_BANK_CYCLES,
  ORC_I_L1_STORE, ORC_I_BLK_LOAD_SEC, ORC_I_BLK_LOAD_LINES, ORC_I_BLK_STORE_SEC,
  ORC_I_BLK_STORE_LINES, ORC_I_WAVE_LOAD_SEC, ORC_I_WAVE_LOAD_LINES, ORC_I_WAVE_STORE_SEC,
  ORC_I_WAVE_STORE_LINES, ORC_I_WAVE_STORE_REQ, ORC_I_OV_Y, ORC_I_OV_Z, ORC_I_Y_LINES,
  ORC_I_Z_LINES, ORC_I_WAVE_BLOCKS, ORC_I_WAVE_FIRST, ORC_I_Y_DIST, ORC_I_Z_DIST,
  ORC_I_BLOCKS_PER_SM, ORC_I_LIMITER, ORC_OUT_NI
};
enum {
  ORC_D_V_L1, ORC_D_V_L2_LOAD, ORC_D_V_L2_STORE, ORC_D_V_DRAM_LOAD, ORC_D_V_DRAM_STORE,
  ORC_D_O_L1, ORC_D_O_Y, ORC_D_O_Z, ORC_D_O_ST, ORC_D_T_L1, ORC_D_T_L2, ORC_D_T_DRAM,
  ORC_D_T_FP, ORC_D_T_PRED, ORC_D_GLUPS, ORC_OUT_ND
};

#ifdef __cplusplus
extern "C" {
#endif

/* Estimates n_cfg candidates with up to `threads` host threads (parallel over
 * candidates; each candidate is walked single-threaded).  Returns 0, or -1 on a
 * malformed argument.  A malformed candidate gets status -1 and no counts. */
int orc_estimate(int n_cfg, const int64_t *cfg_i, const double *cfg_d, const int64_t *fld_i,
                 const int64_t *acc_i, const double *hw_d, int64_t *out_i, double *out_d,
                 int threads);

/* Stable ranking: ascending t_pred rounded to 40 significant bits, ties by index.
 * order_out[k] = index of the k-th best candidate. */
int orc_rank(int n, const double *t_pred, int32_t *order_out);

/* Rounds t to 40 significant mantissa bits (round half to even). */
double orc_rank_key(double t);

#ifdef __cplusplus
}
#endif
#endif
