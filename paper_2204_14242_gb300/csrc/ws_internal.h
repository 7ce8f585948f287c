// Internal layouts shared by the host descriptor compiler (ws_plan.cpp) and the
// kernels (ws_kernels.cu).  Not part of the public ABI.
#pragma once
#include <stdint.h>

#include "warpspeed.h"

namespace ws {

// Exact integer counters accumulated per candidate by the kernels (int64 atomics).
enum Counter {
  C_LUPS_BLOCK, C_LUPS_WAVE, C_L1_REQ, C_BANK, C_L1_STORE,
  C_BLK_LS, C_BLK_LL, C_BLK_SS, C_BLK_SL,
  C_W_LS, C_W_LL, C_W_SS, C_W_SL, C_W_SREQ,
  C_OV_Y, C_OV_Z, C_Y_LINES, C_Z_LINES,
  C_ADDR,      // valid address evaluations (diagnostic, for the roofline)
  C_WINSTR,    // modelled (warp, access) pairs (diagnostic)
  C_OVERFLOW,  // bitmap indices outside the bitmap (skipped; the candidate fails)
  C_RED,       // 64-bit red.or issued by the row walk (diagnostic)
  C_ADDR0,     // address evaluations of the representative block (diagnostic)
  C_CBYTES,    // bitmap bytes the counting kernel read (flagged pages only for row-walk fields)
  N_COUNTERS
};

// Bitmaps of one field, in order: block loads, block stores, wave loads, y-set loads,
// z-set loads, wave stores.  Bit i of a bitmap stands for sector (lo + i).
enum Bitmap { BM_BL, BM_BS, BM_W, BM_Y, BM_Z, BM_WS, N_BITMAPS };

// Page flags of the row walk: a page is kPageWords bitmap words (8,192 sectors, 256 KiB of
// address space).  The row walk sets a flag byte for every page it writes into; the
// counting kernel reads only flagged pages and clears their flags.  Flag bytes of a field:
// [BL pages | BS pages | W | Y | Z | WS pages], block bitmaps with ceil(words[0] / 256)
// pages each, the others ceil(words[1] / 256).
constexpr int kPageWords = 256;
constexpr int kPageShiftBytes = 18;   // byte offset in a bitmap's address space -> page

__host__ __device__ inline int64_t page_count(int64_t words) { return (words + kPageWords - 1) / kPageWords; }
__host__ __device__ inline int64_t page_flag_off(int b, int64_t words0, int64_t words1) {
  return b < 2 ? b * page_count(words0) : 2 * page_count(words0) + (b - 2) * page_count(words1);
}
// Words the flags take, a multiple of 4 so that the bitmaps after them stay 16-byte
// aligned (the counting kernel moves bitmaps in 16-byte units).
__host__ __device__ inline int64_t page_flag_words(int64_t words0, int64_t words1) {
  return (2 * page_count(words0) + 4 * page_count(words1) + 15) / 16 * 4;
}

// Division by an invariant 32-bit divisor d >= 1 by multiply and shift (Granlund and
// Montgomery 1994): with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> s for every n < 2^31.
struct FastDiv {
  uint32_t d, m, s, pad;
};

// Thread groups of one candidate, flattened into one index space of "modelled warps":
//   level 0: the representative block      [0, lev_end[0])
//   level 1: the representative wave       [lev_end[0], lev_end[1])
//   level 2: y-set candidate blocks        [lev_end[1], lev_end[2])
//   level 3: z-set candidate blocks        [lev_end[2], lev_end[3])
struct DCfg {
  int32_t N[3];
  int32_t B[3];
  int32_t fold_axis, fold;
  int32_t g[3];           // grid in blocks
  int32_t T, wpb;         // threads per block, warps per block
  int32_t n_field, field_begin;
  int32_t bpsm, status;
  int64_t rep;            // representative block id (X-Y-Z order)
  int64_t s, weff;        // wave = [s, s + weff)
  int64_t y_lo, y_hi;     // y-set candidates [y_lo, y_hi): kept iff by != g[1]-1
  int64_t z_lo, z_hi;     // z-set candidates: kept iff not in the y set
  int64_t y_dist, z_dist; // s - first block of the y / z set (0 if empty)
  int64_t lev_end[4];      // all < 2^31 (checked by the descriptor compiler)
  double flops;
  FastDiv fd_gx, fd_gy, fd_wpb;
  // Row walk of levels 1-3 (wave, y set, z set).  A block row R = by + g[1] * bz of a
  // level holds one run of blocks that are consecutive in x; its threads with the same
  // (ty, tz) form one grid row of consecutive x.  Slot = (block row, thread row).
  // Level 3 of the row walk is the representative block itself (its block bitmaps).
  int32_t rows_R_lo[4], rows_R_cnt[4];
  int64_t rows_slot_end[4];    // cumulative slots: wave, y set, z set, block (< 2^31)
  int32_t rows_per_blk;        // B[1] * B[2]
  int32_t full_end;            // blocks in x that lie entirely inside N[0]
  FastDiv fd_rows, fd_b1;
  FastDiv fd_b2, fd_fold;      // for locating the row of a covering run
};

struct DField {
  int64_t base;           // align + elem_bytes * const_off  (bytes)
  int64_t stride[3];      // elements
  int64_t lo[2];          // first sector of the block bitmaps [0] / wave bitmaps [1]
  int64_t words[2];       // 32-bit words per block bitmap [0] / wave bitmap [1]
  int64_t bm[N_BITMAPS];  // word offset of each bitmap in the pass scratch, -1 = absent
  int64_t pg;             // word offset of the page flags (row-walk fields), -1 = count every word
  int64_t item_begin;     // first enumeration work item (global numbering)
  int64_t citem_begin;    // first counting work item
  int64_t mw_end;         // modelled warps this field visits (loads: all levels, stores: block + wave)
  int64_t mw_block;       // modelled warps of the representative block (work item 0 of the field)
  int32_t esize;
  int32_t n_load, n_store;// folded access counts (loads first, then stores)
  int32_t acc_begin;      // index into the DAcc array
  int32_t cfg;            // owning candidate
  int32_t first_of_cfg;   // 1 if this is the candidate's first field (counts LUPs)
  int32_t wide;           // a bitmap spans >= 2^32 bytes: 64-bit address path
  int32_t lpa_log2p;      // log2 of P = lanes per thread-slice group for the load walk (P >= n_load, <= 32)
  int32_t iv;             // interval walk possible: not wide and |elem_bytes * stride_x| <= 32
  int32_t iv_begin;       // first merged load interval (DIv array)
  int32_t n_iv;           // merged load intervals
  int32_t rows_ok;        // stores: the row segments of one warp never share a sector
  int32_t level_mask;     // levels served: 1 the representative block, 2 wave + y / z sets
  int32_t n_iv_unc;       // merged load intervals without a covering run (they come first)
  int32_t n_iv_zc;        // those covered from another z row (they come next; the rest last)
  int16_t cov_dy, cov_dz; // largest |row displacement| from an interval to its covering run
  int16_t cov_dy_y;       // largest |ddy| of the intervals covered within their z row
  int16_t pad16;
  int32_t zshift;         // 1: the z set's sectors are the wave's moved by whole lines (loads)
  int32_t zc_lo, zc_hi;   // zshift: sectors (from the wave origin) bounding the wave's addresses
  int16_t cnt_load[17];   // folded loads issued by a thread with kv valid points
  int16_t cnt_store[17];  // folded stores likewise
};

// One folded access: byte offset from the thread's first point, and the smallest
// folded point index k that needs it (issued iff k < number of valid points).
struct DAcc {
  int64_t boff;
  int32_t kmin;
  int32_t pad;
};

// A merged load interval of a field: folded loads whose sorted byte offsets are at
// most 32 B apart, so that for a row segment of threads whose addresses step by at
// most 32 B the union of all their sectors is the single sector range
// [(lowest thread address + boff) / 32, (highest thread address + boff + ext) / 32].
//
// Covering run: when every offset of the run lies in one grid row (dy, dz, dc) with x
// offsets dx_lo..dx_hi, and an earlier run of the field (in a fixed order) with the same dc
// and x offsets covering dx_lo..dx_hi lies (ddy, ddz) grid rows back, the range of (row r,
// this run) is contained in the range of (row r + (ddy, ddz), that run) whenever that row
// belongs to the same level with an x range covering r's (and all its folded points are
// valid), so the row walk skips it.  Containment is transitive and the order is strict, so
// a skipped range is always covered by one that is set.  ddy == kNoCover: no covering run.
struct DIv {
  int64_t boff;           // smallest byte offset of the run
  uint32_t ext;           // largest minus smallest byte offset
  int16_t ddy, ddz;       // grid rows to the covering run's row (kNoCover: none)
};
constexpr int16_t kNoCover = -32768;

struct DHw {
  double clock_hz, l1_bytes, l2_bytes, bw_l2, bw_dram, fp_peak;
  double hit[4][3];
  int32_t sms, banks, bank_bytes, pair_dist_bytes, capacity_model, pad;
};

// A field group: consecutive fields of one candidate enumerated together, so that a
// modelled warp is decoded once for all of them.  Work items of the enumeration kernel
// are (group, chunk of modelled warps); item 0 of a group is the representative block.
struct DGroup {
  int64_t item_begin;     // first enumeration work item
  int64_t ritem_begin;    // first row-walk work item (row groups; empty range otherwise)
  int64_t mw_end;         // modelled warps visited (max over the group's fields)
  int64_t mw_block;       // modelled warps of the representative block
  int32_t cfg;            // owning candidate
  int32_t f_begin;        // fields [f_begin, f_begin + f_count)
  int32_t f_count;
  int32_t acc_count;      // folded accesses of all its fields (<= kMaxFoldedAccesses)
  int32_t first_of_cfg;   // the candidate's first group counts LUPs
  int32_t uniform;        // all fields share element size and strides (and none is wide)
  int32_t n_loads;        // folded loads of all its fields
  int32_t n_stores;       // folded stores of all its fields
  int32_t iv;             // uniform and every field allows the interval walk
  int32_t n_iv;           // merged load intervals of all its fields
  int32_t rows;           // levels 1-3 take the row walk (work items are chunks of row slots)
  int32_t n0_items;       // enumeration items of the representative block
  int32_t levels;         // level mask of its fields (1 block, 2 wave + y / z, 3 both)
  int32_t first_wave;     // the candidate's first group with wave work counts the wave LUPs
  // Representative-block warps to evaluate and the number of warps each one stands for
  // (warps with the same lane layout whose addresses differ by a multiple of the bank and
  // sector period give the same per-instruction counts); all warps, once each, unless the
  // row walk builds the block bitmaps.
  int32_t n_rep;
  uint8_t rep_warp[32];
  uint8_t rep_mult[32];
  int32_t pad2;
};

// Classes of representative-block warps with identical per-instruction counts (host).
struct WarpClasses {
  int32_t n = 0;
  uint8_t warp[32], mult[32];
};

// One pass = a contiguous range of field groups whose bitmaps fit the scratch
// together.  Passes run one after the other and reuse the same scratch.
struct DPass {
  int64_t item_lo, item_hi;    // enumeration items of the pass
  int64_t ritem_lo, ritem_hi;  // row-walk items of the pass
  int64_t citem_lo, citem_hi;  // counting items of the pass
  int32_t cf_lo, cf_hi;        // (candidate, field) index range
  int32_t grp_lo, grp_hi;      // field-group index range
  int64_t words;               // scratch words [0, words) holding the pass's bitmaps
};

constexpr int kMaxFoldedAccesses = 2048;   // per field group, staged in shared memory
constexpr int kMaxGroupFields = 32;
constexpr int64_t kMaxBitmapWords = (int64_t)1 << 31;

}  // namespace ws
