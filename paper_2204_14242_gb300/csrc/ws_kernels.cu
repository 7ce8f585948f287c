// Device side of the metric estimator (sm_103a).
//
//   enum_kernel   persistent, work-stealing enumeration of (modelled warp, access) pairs
//                 of the representative block, the wave and the y / z layer sets
//                 (Sec. 3.2-3.4).  Each lane evaluates its address expression; the warp
//                 merges lanes that fall into the same bitmap word (__reduce_or_sync) and
//                 one lane per word issues a red.or into the field's L2-resident sector
//                 bitmap.  The same merge yields the per-instruction unique sector count
//                 (L1 request / write-through volumes).  Block-level warps also compute
//                 half-warp bank-conflict cycles.
//   count_kernel  read-and-clear popcount of the bitmaps: unique sectors, unique 128 B
//                 lines (nibble OR), y / z overlaps by AND / AND-NOT.  Leaves the
//                 bitmaps zeroed for the next step.
//   model_kernel  fp64 capacity model and limiters (Sec. 2, 3.5), one thread per candidate.
//   rank_kernel   stable counting rank per segment (Sec. 5.7).
#include <cuda_runtime.h>

#include "ws_internal.h"
#include "ws_kernels.h"

namespace ws {

#define FULL 0xffffffffu

__device__ __forceinline__ int64_t floordiv_dev(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

// Warp-cooperative insertion of one access instruction into a sector bitmap.
// rel: byte address relative to the bitmap origin.  Lanes whose word falls outside
// [0, nwords) are not inserted and are counted in *bad (the host compiler sizes every
// bitmap to hold all addresses, so this never happens unless a descriptor is wrong).
// Returns the number of distinct sectors the active lanes touched (warp-uniform).
__device__ __forceinline__ uint32_t bitmap_insert(uint32_t *__restrict__ bm, int64_t rel, bool act,
                                                  uint32_t lane, int64_t nwords, uint32_t &bad) {
  const bool inside = (uint64_t)(rel >> 10) < (uint64_t)nwords;
  bad += act && !inside;
  act = act && inside;
  uint32_t word = (uint32_t)(rel >> 10);
  uint32_t bit = 1u << ((uint32_t)(rel >> 5) & 31u);
  uint32_t pending = __ballot_sync(FULL, act);
  uint32_t cnt = 0;
  while (pending) {
    uint32_t leader = __ffs(pending) - 1;
    uint32_t lw = __shfl_sync(FULL, word, leader);
    bool mine = act && word == lw;
    uint32_t orv = __reduce_or_sync(FULL, mine ? bit : 0u);
    if (lane == leader) atomicOr(bm + lw, orv);
    cnt += __popc(orv);
    pending &= ~__ballot_sync(FULL, mine);
  }
  return cnt;
}

// Bank-conflict visitor for both half warps of one instruction (Sec. 3.2): unique
// bank words of each half warp, split greedily (ascending) into groups spanning less
// than the pairing distance, each group costs its most used bank.  The result is the
// sum over both halves, valid in every lane.
__device__ int bank_cycles_warp(int64_t addr, bool act, uint32_t lane, int banks, int bank_bytes,
                                int pair_dist) {
  int64_t word = floordiv_dev(addr, bank_bytes);
  int bank = (int)(((word % banks) + banks) % banks);
  uint32_t actm = __ballot_sync(FULL, act);
  uint32_t halfm = lane < 16 ? 0x0000ffffu : 0xffff0000u;
  uint32_t same = __match_any_sync(FULL, (unsigned long long)word) & actm & halfm;
  bool uniq = act && lane == (uint32_t)(__ffs(same) - 1);
  uint32_t todo = __ballot_sync(FULL, uniq);
  int cycles = 0;
  while (todo) {
    bool mine = (todo >> lane) & 1u;
    long long v = mine ? (long long)word : 0x7fffffffffffffffll;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
      long long o = __shfl_xor_sync(FULL, v, off);
      v = o < v ? o : v;
    }
    bool member = mine && (word - (int64_t)v) * (int64_t)bank_bytes < (int64_t)pair_dist;
    uint32_t mm = __ballot_sync(FULL, member);
    uint32_t sameb = __match_any_sync(FULL, bank) & mm & halfm;
    int c = member ? __popc(sameb) : 0;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) c = max(c, __shfl_xor_sync(FULL, c, off));
    if ((lane & 15u) == 0) cycles += c;
    todo &= ~mm;
  }
  return __reduce_add_sync(FULL, (uint32_t)cycles);
}

__device__ __forceinline__ int find_cf(const DField *__restrict__ fld, int lo, int hi, int64_t item,
                                       bool counting) {
  // last cf in [lo, hi) whose first item is <= item
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    int64_t b = counting ? fld[mid].citem_begin : fld[mid].item_begin;
    if (b <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(1024) enum_kernel(EnumArgs a) {
  __shared__ int64_t s_boff[kMaxFoldedAccesses];
  __shared__ uint8_t s_kmin[kMaxFoldedAccesses];
  __shared__ uint32_t s_tc[1024];
  __shared__ long long s_item;

  const uint32_t lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  int cur_cf = -1, cur_cfg = -1;

  for (;;) {
    if (threadIdx.x == 0) s_item = a.item_lo + (long long)atomicAdd(a.grab, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= a.item_hi) break;
    const int cf = find_cf(a.fld, a.cf_lo, a.cf_hi, item, false);
    const DField &F = a.fld[cf];
    const DCfg &C = a.cfg[F.cfg];
    if (cf != cur_cf) {
      const int na = F.n_load + F.n_store;
      for (int i = threadIdx.x; i < na; i += blockDim.x) {
        DAcc d = a.acc[F.acc_begin + i];
        s_boff[i] = d.boff;
        s_kmin[i] = (uint8_t)d.kmin;
      }
      if (F.cfg != cur_cfg) {
        for (int t = threadIdx.x; t < C.T; t += blockDim.x) {
          uint32_t tx = t % C.B[0], ty = (t / C.B[0]) % C.B[1], tz = t / (C.B[0] * C.B[1]);
          s_tc[t] = tx | (ty << 10) | (tz << 20);
        }
      }
      __syncthreads();
      cur_cf = cf;
      cur_cfg = F.cfg;
    }
    const int64_t mw0 = (item - F.item_begin) * (int64_t)a.chunk;
    const int64_t mw1 = min(mw0 + (int64_t)a.chunk, F.mw_end);
    unsigned long long acc_lb = 0, acc_lw = 0, acc_req = 0, acc_st = 0, acc_bank = 0, acc_sreq = 0,
                       acc_addr = 0, acc_wi = 0;
    uint32_t bad = 0;

    for (int64_t mw = mw0 + warp; mw < mw1; mw += nwarps) {
      int level;
      int64_t b, j;
      if (mw < C.lev_end[0]) {
        level = 0; b = C.rep; j = mw;
      } else if (mw < C.lev_end[1]) {
        level = 1; j = mw - C.lev_end[0]; b = C.s + j / C.wpb;
      } else if (mw < C.lev_end[2]) {
        level = 2; j = mw - C.lev_end[1]; b = C.y_lo + j / C.wpb;
      } else {
        level = 3; j = mw - C.lev_end[2]; b = C.z_lo + j / C.wpb;
      }
      const int w = (int)(j % C.wpb);
      const int32_t bx = (int32_t)(b % C.g[0]);
      const int64_t bt = b / C.g[0];
      const int32_t by = (int32_t)(bt % C.g[1]);
      const int32_t bz = (int32_t)(bt / C.g[1]);
      if (level == 2 && by == C.g[1] - 1) continue;
      if (level == 3 && b >= C.y_lo && b < C.y_hi && by != C.g[1] - 1) continue;

      const int tid = w * 32 + (int)lane;
      const bool exists = tid < C.T;
      const uint32_t tc = exists ? s_tc[tid] : 0u;
      int32_t x = bx * C.B[0] + (int32_t)(tc & 1023u);
      int32_t y = by * C.B[1] + (int32_t)((tc >> 10) & 1023u);
      int32_t z = bz * C.B[2] + (int32_t)(tc >> 20);
      if (C.fold_axis == 1) y *= C.fold;
      if (C.fold_axis == 2) z *= C.fold;
      const bool valid = exists && x < C.N[0] && y < C.N[1] && z < C.N[2];
      int kv = 0;
      if (valid) kv = C.fold_axis == 1 ? min(C.fold, C.N[1] - y) : C.fold_axis == 2 ? min(C.fold, C.N[2] - z) : 1;
      const int lv = level == 0 ? 0 : 1;
      const int64_t rel = F.base + (int64_t)F.esize * (F.stride[0] * x + F.stride[1] * y + F.stride[2] * z) -
                          32 * F.lo[lv];

      if (F.n_load > 0) {
        uint32_t *bm = a.scratch + F.bm[level == 0 ? BM_BL : level == 1 ? BM_W : level == 2 ? BM_Y : BM_Z];
        for (int i = 0; i < F.n_load; ++i) {
          const bool act = valid && (int)s_kmin[i] < kv;
          const int64_t r = rel + s_boff[i];
          const uint32_t cnt = bitmap_insert(bm, r, act, lane, F.words[lv], bad);
          acc_addr += __popc(__ballot_sync(FULL, act));
          acc_wi += 1;
          if (level == 0) {
            acc_req += cnt;
            acc_bank += bank_cycles_warp(r + 32 * F.lo[0], act, lane, a.banks, a.bank_bytes, a.pair_dist);
          }
        }
      }
      if (F.n_store > 0 && level <= 1) {
        uint32_t *bm = a.scratch + F.bm[level == 0 ? BM_BS : BM_WS];
        for (int i = F.n_load; i < F.n_load + F.n_store; ++i) {
          const bool act = valid && (int)s_kmin[i] < kv;
          const int64_t r = rel + s_boff[i];
          const uint32_t cnt = bitmap_insert(bm, r, act, lane, F.words[lv], bad);
          acc_addr += __popc(__ballot_sync(FULL, act));
          acc_wi += 1;
          if (level == 0) {
            acc_st += cnt;
            acc_bank += bank_cycles_warp(r + 32 * F.lo[0], act, lane, a.banks, a.bank_bytes, a.pair_dist);
          } else {
            acc_sreq += cnt;
          }
        }
      }
      if (F.first_of_cfg && level <= 1) {
        const uint32_t l = __reduce_add_sync(FULL, (uint32_t)kv);
        if (level == 0) acc_lb += l;
        else acc_lw += l;
      }
    }
    bad = __reduce_add_sync(FULL, bad);
    if (lane == 0) {
      unsigned long long *c = (unsigned long long *)(a.counters + (int64_t)F.cfg * N_COUNTERS);
      if (bad) atomicAdd(c + C_OVERFLOW, (unsigned long long)bad);
      if (acc_lb) atomicAdd(c + C_LUPS_BLOCK, acc_lb);
      if (acc_lw) atomicAdd(c + C_LUPS_WAVE, acc_lw);
      if (acc_req) atomicAdd(c + C_L1_REQ, acc_req);
      if (acc_st) atomicAdd(c + C_L1_STORE, acc_st);
      if (acc_bank) atomicAdd(c + C_BANK, acc_bank);
      if (acc_sreq) atomicAdd(c + C_W_SREQ, acc_sreq);
      if (acc_addr) atomicAdd(c + C_ADDR, acc_addr);
      if (acc_wi) atomicAdd(c + C_WINSTR, acc_wi);
    }
    __syncthreads();
  }
}

__constant__ int kCountDst[12] = {C_BLK_LS, C_BLK_LL, C_BLK_SS, C_BLK_SL, C_W_LS, C_W_LL,
                                  C_Y_LINES, C_Z_LINES, C_OV_Y, C_OV_Z, C_W_SS, C_W_SL};

__device__ __forceinline__ uint32_t lines_of(uint32_t x) {
  // bit i <-> sector lo + i with lo a multiple of 32: nibbles are 128 B lines
  uint32_t t = x | (x >> 1);
  t |= t >> 2;
  return __popc(t & 0x11111111u);
}

__device__ __forceinline__ uint4 ld_clear(uint32_t *p) {
  uint4 *q = reinterpret_cast<uint4 *>(p);
  uint4 v = *q;
  *q = make_uint4(0u, 0u, 0u, 0u);
  return v;
}

__global__ void __launch_bounds__(256) count_kernel(CountArgs a) {
  __shared__ long long s_item;
  __shared__ uint32_t s_red[8][12];
  const uint32_t lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_item = a.citem_lo + (long long)atomicAdd(a.grab, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= a.citem_hi) break;
    const int cf = find_cf(a.fld, a.cf_lo, a.cf_hi, item, true);
    const DField &F = a.fld[cf];
    const bool has_blk = F.bm[BM_BL] >= 0 || F.bm[BM_BS] >= 0;
    const int64_t nb = has_blk ? F.words[0] : 0;
    const int64_t ntot = nb + F.words[1];
    const int64_t c0 = (item - F.citem_begin) * (int64_t)a.chunk_words;
    const int64_t c1 = min(c0 + (int64_t)a.chunk_words, ntot);
    uint32_t acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // block part: words [c0, min(c1, nb)) -- BL, BS
    for (int64_t i = c0 + 4 * threadIdx.x; i < min(c1, nb); i += 4 * blockDim.x) {
      if (F.bm[BM_BL] >= 0) {
        uint4 v = ld_clear(a.scratch + F.bm[BM_BL] + i);
        acc[0] += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        acc[1] += lines_of(v.x) + lines_of(v.y) + lines_of(v.z) + lines_of(v.w);
      }
      if (F.bm[BM_BS] >= 0) {
        uint4 v = ld_clear(a.scratch + F.bm[BM_BS] + i);
        acc[2] += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        acc[3] += lines_of(v.x) + lines_of(v.y) + lines_of(v.z) + lines_of(v.w);
      }
    }
    // wave part: words [max(c0, nb), c1) - nb -- W, Y, Z, WS
    for (int64_t i = max(c0, nb) + 4 * threadIdx.x; i < c1; i += 4 * blockDim.x) {
      const int64_t k = i - nb;
      if (F.bm[BM_W] >= 0) {
        uint4 w = ld_clear(a.scratch + F.bm[BM_W] + k);
        uint4 y = ld_clear(a.scratch + F.bm[BM_Y] + k);
        uint4 z = ld_clear(a.scratch + F.bm[BM_Z] + k);
        acc[4] += __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
        acc[5] += lines_of(w.x) + lines_of(w.y) + lines_of(w.z) + lines_of(w.w);
        acc[6] += lines_of(y.x) + lines_of(y.y) + lines_of(y.z) + lines_of(y.w);
        acc[7] += lines_of(z.x) + lines_of(z.y) + lines_of(z.z) + lines_of(z.w);
        acc[8] += __popc(w.x & y.x) + __popc(w.y & y.y) + __popc(w.z & y.z) + __popc(w.w & y.w);
        acc[9] += __popc(w.x & z.x & ~y.x) + __popc(w.y & z.y & ~y.y) + __popc(w.z & z.z & ~y.z) +
                  __popc(w.w & z.w & ~y.w);
      }
      if (F.bm[BM_WS] >= 0) {
        uint4 v = ld_clear(a.scratch + F.bm[BM_WS] + k);
        acc[10] += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        acc[11] += lines_of(v.x) + lines_of(v.y) + lines_of(v.z) + lines_of(v.w);
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      uint32_t v = __reduce_add_sync(FULL, acc[k]);
      if (lane == 0) s_red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
      unsigned long long t = 0;
      for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) t += s_red[wi][threadIdx.x];
      if (t) {
        const int d = kCountDst[threadIdx.x];
        atomicAdd((unsigned long long *)(a.counters + (int64_t)F.cfg * N_COUNTERS + d), t);
      }
    }
    __syncthreads();
  }
}

// R(O) = a * exp(-b * exp(-c * O)), Sec. 3.5
__device__ __forceinline__ double rhat_dev(const double h[3], double O) {
  return __dmul_rn(h[0], exp(-__dmul_rn(h[1], exp(-__dmul_rn(h[2], O)))));
}

__device__ double rank_key_dev(double t) {
  if (!(t > 0.0) || isinf(t)) return t;
  int e = 0;
  double m = frexp(t, &e);
  return ldexp(rint(ldexp(m, 40)), e - 40);
}

// The capacity model and the four limiters, one thread per candidate.  Products and
// quotients use explicit round-to-nearest intrinsics so that no multiply-add is fused
// and the evaluation order is the one written here.
__global__ void model_kernel(ModelArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const DCfg &C = a.cfg[i];
  const int64_t *c = a.counters + (int64_t)i * N_COUNTERS;
  ws_result r;
  memset(&r, 0, sizeof(r));
  r.status = C.status;
  if (r.status == WS_OK && c[C_OVERFLOW] != 0) r.status = WS_EOVERFLOW;
  if (r.status != WS_OK) {
    r.t_pred = __longlong_as_double(0x7ff0000000000000ll);
    r.glups = 0.0;
    a.results[i] = r;
    a.keys[i] = r.t_pred;
    return;
  }
  r.lups_block = c[C_LUPS_BLOCK];
  r.lups_wave = c[C_LUPS_WAVE];
  r.l1_req_sectors = c[C_L1_REQ];
  r.l1_bank_cycles = c[C_BANK];
  r.l1_store_sectors = c[C_L1_STORE];
  r.blk_load_sectors = c[C_BLK_LS];
  r.blk_load_lines = c[C_BLK_LL];
  r.blk_store_sectors = c[C_BLK_SS];
  r.blk_store_lines = c[C_BLK_SL];
  r.wave_load_sectors = c[C_W_LS];
  r.wave_load_lines = c[C_W_LL];
  r.wave_store_sectors = c[C_W_SS];
  r.wave_store_lines = c[C_W_SL];
  r.wave_store_req_sectors = c[C_W_SREQ];
  r.ov_y = c[C_OV_Y];
  r.ov_z = c[C_OV_Z];
  r.y_lines = c[C_Y_LINES];
  r.z_lines = c[C_Z_LINES];
  r.wave_blocks = C.weff;
  r.wave_first_block = C.s;
  r.y_dist_blocks = C.y_dist;
  r.z_dist_blocks = C.z_dist;
  r.blocks_per_sm = C.bpsm;

  const DHw &h = a.hw;
  const double lb = (double)r.lups_block, lw = (double)r.lups_wave;
  const bool cap = h.capacity_model != 0;
  // L1 <-> L2: requests per instruction are V_up, the block footprint is V_comp
  r.v_l1 = __ddiv_rn(__dmul_rn(32.0, (double)r.l1_req_sectors), lb);
  const double v_comp = __ddiv_rn(__dmul_rn(32.0, (double)r.blk_load_sectors), lb);
  r.o_l1 = __ddiv_rn(__dmul_rn(__dmul_rn(128.0, (double)r.blk_load_lines), (double)C.bpsm), h.l1_bytes);
  const double r_l1 = cap ? rhat_dev(h.hit[0], r.o_l1) : 1.0;
  r.v_l2_load = __dadd_rn(v_comp, __dmul_rn(__dsub_rn(1.0, r_l1), __dsub_rn(r.v_l1, v_comp)));
  r.v_l2_store = __ddiv_rn(__dmul_rn(32.0, (double)r.l1_store_sectors), lb);
  // DRAM <-> L2: wave footprint minus layer-condition reuse plus partial-store reads
  const double v_dcomp = __ddiv_rn(__dmul_rn(32.0, (double)r.wave_load_sectors), lw);
  const double alloc = __ddiv_rn(__dmul_rn(128.0, (double)r.wave_load_lines), (double)C.weff);
  r.o_y = __ddiv_rn(__dmul_rn((double)C.y_dist, alloc), h.l2_bytes);
  r.o_z = __ddiv_rn(__dmul_rn((double)C.z_dist, alloc), h.l2_bytes);
  const double r_y = cap ? rhat_dev(h.hit[1], r.o_y) : 1.0;
  const double r_z = cap ? rhat_dev(h.hit[2], r.o_z) : 1.0;
  r.o_st = __ddiv_rn(__dmul_rn(128.0, (double)r.wave_store_lines), h.l2_bytes);
  const double r_st = cap ? rhat_dev(h.hit[3], r.o_st) : 1.0;
  const double v_red = __ddiv_rn(__dmul_rn(32.0, (double)(r.wave_store_req_sectors - r.wave_store_sectors)), lw);
  const double hits = __ddiv_rn(__dadd_rn(__dmul_rn(r_y, __dmul_rn(32.0, (double)r.ov_y)),
                                          __dmul_rn(r_z, __dmul_rn(32.0, (double)r.ov_z))), lw);
  r.v_dram_load = __dadd_rn(__dsub_rn(v_dcomp, hits), __dmul_rn(__dsub_rn(1.0, r_st), v_red));
  r.v_dram_store = __ddiv_rn(__dmul_rn(32.0, (double)r.wave_store_sectors), lw);
  // limiters: seconds per LUP for the whole GPU
  r.t_l1 = __ddiv_rn(__ddiv_rn((double)r.l1_bank_cycles, lb), __dmul_rn(h.clock_hz, (double)h.sms));
  r.t_l2 = __ddiv_rn(__dadd_rn(r.v_l2_load, r.v_l2_store), h.bw_l2);
  r.t_dram = __ddiv_rn(__dadd_rn(r.v_dram_load, r.v_dram_store), h.bw_dram);
  r.t_fp = (C.flops > 0.0 && h.fp_peak > 0.0) ? __ddiv_rn(C.flops, h.fp_peak) : 0.0;
  double best = r.t_l1;
  int lim = WS_LIMITER_L1;
  if (r.t_l2 > best) { best = r.t_l2; lim = WS_LIMITER_L2; }
  if (r.t_dram > best) { best = r.t_dram; lim = WS_LIMITER_DRAM; }
  if (r.t_fp > best) { best = r.t_fp; lim = WS_LIMITER_FP; }
  r.t_pred = best;
  r.limiter = lim;
  r.glups = __ddiv_rn(1e-9, best);
  a.results[i] = r;
  a.keys[i] = rank_key_dev(best);
}

// Stable rank within segments: rank(i) = #{j in seg : key_j < key_i or
// (key_j == key_i and j < i)}; NaN counts as +inf.  order[seg_begin + rank(i)] = i.
__global__ void __launch_bounds__(256) rank_kernel(RankArgs a) {
  __shared__ double s_key[1024];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i_first = (int64_t)blockIdx.x * blockDim.x;
  const int64_t i_last = min((int64_t)a.n, i_first + (int64_t)blockDim.x) - 1;
  if (i_first >= a.n) return;
  auto seg_of = [&](int64_t x) {
    int lo = 0, hi = a.n_seg;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (a.seg[mid] <= x) lo = mid;
      else hi = mid;
    }
    return lo;
  };
  const int s_first = seg_of(i_first), s_last = seg_of(i_last);
  const int64_t j_lo = a.seg[s_first], j_hi = a.seg[s_last + 1];
  int my_seg = i < a.n ? seg_of(i) : -1;
  int64_t my_lo = my_seg >= 0 ? a.seg[my_seg] : 0, my_hi = my_seg >= 0 ? a.seg[my_seg + 1] : 0;
  double ki = 0.0;
  if (i < a.n) {
    ki = a.keys[i];
    if (isnan(ki)) ki = __longlong_as_double(0x7ff0000000000000ll);
  }
  int64_t rank = 0;
  for (int64_t t0 = j_lo; t0 < j_hi; t0 += 1024) {
    __syncthreads();
    for (int k = threadIdx.x; k < 1024 && t0 + k < j_hi; k += blockDim.x) {
      double v = a.keys[t0 + k];
      s_key[k] = isnan(v) ? __longlong_as_double(0x7ff0000000000000ll) : v;
    }
    __syncthreads();
    if (i < a.n) {
      const int64_t a0 = max(t0, my_lo), a1 = min(t0 + 1024, my_hi);
      for (int64_t j = a0; j < a1; ++j) {
        double kj = s_key[j - t0];
        rank += (kj < ki) || (kj == ki && j < i);
      }
    }
  }
  if (i < a.n) a.order[my_lo + rank] = (int32_t)i;
}

// Rank keys of given results (used when ranking results that came from the host).
__global__ void keys_kernel(const ws_result *__restrict__ res, int n, double *__restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = rank_key_dev(res[i].t_pred);
}

// ---- launchers ---------------------------------------------------------------------
cudaError_t launch_enum(const EnumArgs &args, int grid, int threads, cudaStream_t st) {
  enum_kernel<<<grid, threads, 0, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_count(const CountArgs &args, int grid, cudaStream_t st) {
  count_kernel<<<grid, 256, 0, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_model(const ModelArgs &args, cudaStream_t st) {
  if (args.n <= 0) return cudaSuccess;
  model_kernel<<<(args.n + 127) / 128, 128, 0, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_rank(const RankArgs &args, cudaStream_t st) {
  if (args.n <= 0) return cudaSuccess;
  rank_kernel<<<(args.n + 255) / 256, 256, 0, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_keys(const ws_result *res, int n, double *keys, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  keys_kernel<<<(n + 255) / 256, 256, 0, st>>>(res, n, keys);
  return cudaGetLastError();
}
cudaError_t enum_occupancy(int threads, int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, enum_kernel, threads, 0);
}
cudaError_t count_occupancy(int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, count_kernel, 256, 0);
}

}  // namespace ws
