// CPU oracle of the metric estimator -- TEST INFRASTRUCTURE, not part of the product.
//
// A plain, slow enumerator written to be checked by eye against the paper:
//   * grid iteration (Sec. 4.2, listing "grid iteration"): every thread of a thread
//     group, every address expression of a field;
//   * unique 32 B sectors and 128 B lines per group (Sec. 4.3, CL32 visitor);
//   * bank-conflict cycles per half-warp (Sec. 4.2, bank-conflict visitor, 16 banks
//     x 8 B, 1024 B pairing distance);
//   * one representative block (Sec. 4.3) and one wave of co-resident blocks in the
//     middle of the grid (Sec. 4.4), plus the y and z layer-condition thread sets
//     (Sec. 4.4.2), the wave-level sets in linear addresses or, optionally, in the
//     multi-dimensional address space of Sec. 4.4.1;
//   * capacity misses (Sec. 4.5, Eqs. for V_cap and R_hit(O)) and the four-limiter
//     performance model (Sec. 2).
// Every set is a std::set; every count is the size of a set.  Floating point is fp64
// in one fixed order.  Readings of points the paper leaves open are noted inline.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <thread>
#include <tuple>
#include <vector>

namespace {

typedef std::tuple<int64_t, int64_t, int64_t, int64_t> Off;  // dx dy dz dc

struct OField {
  int64_t esize, align, stride[3], c;
  std::set<Off> loads, stores;              // offsets as written by the generator
  std::vector<Off> fload, fstore;           // folded per-thread instruction lists
};

struct OCfg {
  int64_t N[3], B[3], fold_axis, fold, regs, wave_override, addr_mode;
  double flops;
  std::vector<OField> fields;
};

struct OHw {
  int64_t sms, max_threads_sm, max_blocks_sm, regs_sm, banks, bank_bytes, pair_dist, cap;
  double clock, l1, l2, bw_l2, bw_dram, fp_peak, hit[4][3];
};

// floor division for possibly negative numerators (addresses may precede the base)
int64_t floordiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

int64_t ceildiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Unit vector of the folding axis as an offset.
Off fold_step(const OCfg &c, int64_t k) {
  if (c.fold_axis == 1) return Off(0, k, 0, 0);
  if (c.fold_axis == 2) return Off(0, 0, k, 0);
  return Off(0, 0, 0, 0);
}

Off add(const Off &a, const Off &b) {
  return Off(std::get<0>(a) + std::get<0>(b), std::get<1>(a) + std::get<1>(b),
             std::get<2>(a) + std::get<2>(b), std::get<3>(a) + std::get<3>(b));
}
Off sub(const Off &a, const Off &b) {
  return Off(std::get<0>(a) - std::get<0>(b), std::get<1>(a) - std::get<1>(b),
             std::get<2>(a) - std::get<2>(b), std::get<3>(a) - std::get<3>(b));
}

// Thread folding (Sec. 5.2): a thread updates `fold` consecutive points along the
// folding axis.  Its loads are the union over k of (offset + k * axis); each distinct
// address is loaded once and reused from registers (Sec. 5.4).  Stores likewise.
std::vector<Off> fold_list(const OCfg &c, const std::set<Off> &offs) {
  std::set<Off> u;
  for (const Off &o : offs)
    for (int64_t k = 0; k < c.fold; ++k) u.insert(add(o, fold_step(c, k)));
  return std::vector<Off>(u.begin(), u.end());
}

// Reading: a folded access is issued iff some valid folded point k < kv needs it.
bool access_needed(const OCfg &c, const std::set<Off> &offs, const Off &o, int64_t kv) {
  for (int64_t k = 0; k < kv; ++k)
    if (offs.count(sub(o, fold_step(c, k)))) return true;
  return false;
}

struct Thread {
  bool exists;   // lane maps to a thread of the block
  bool valid;    // its first point is inside the domain
  int64_t p[3];  // first (k = 0) grid point
  int64_t kv;    // number of its folded points inside the domain
};

// Thread `tid` (linear, x fastest) of block `bid` (linear, X-Y-Z order, Sec. 4.4).
Thread make_thread(const OCfg &c, const int64_t g[3], int64_t bid, int64_t tid) {
  Thread t;
  int64_t T = c.B[0] * c.B[1] * c.B[2];
  t.exists = tid < T;
  t.valid = false;
  t.kv = 0;
  t.p[0] = t.p[1] = t.p[2] = 0;
  if (!t.exists) return t;
  int64_t bx = bid % g[0], by = (bid / g[0]) % g[1], bz = bid / (g[0] * g[1]);
  int64_t tx = tid % c.B[0], ty = (tid / c.B[0]) % c.B[1], tz = tid / (c.B[0] * c.B[1]);
  t.p[0] = bx * c.B[0] + tx;
  t.p[1] = by * c.B[1] + ty;
  t.p[2] = bz * c.B[2] + tz;
  if (c.fold_axis == 1) t.p[1] *= c.fold;
  if (c.fold_axis == 2) t.p[2] *= c.fold;
  // domain guard on every folded point (Sec. 4.4.1)
  for (int64_t k = 0; k < c.fold; ++k) {
    int64_t q[3] = {t.p[0], t.p[1], t.p[2]};
    if (c.fold_axis == 1) q[1] += k;
    if (c.fold_axis == 2) q[2] += k;
    bool in = true;
    for (int d = 0; d < 3; ++d) in = in && q[d] >= 0 && q[d] < c.N[d];
    if (in) t.kv += 1;
  }
  t.valid = t.kv > 0;
  return t;
}

// Address expression with the base pointer replaced by the field alignment (Sec. 4.3).
int64_t address(const OField &f, const Thread &t, const Off &o) {
  int64_t e = f.stride[0] * (t.p[0] + std::get<0>(o)) + f.stride[1] * (t.p[1] + std::get<1>(o)) +
              f.stride[2] * (t.p[2] + std::get<2>(o)) + f.c + std::get<3>(o);
  return f.align + f.esize * e;
}

// Bank-conflict visitor for one half-warp instruction (Sec. 4.2).  Unique bank words,
// in ascending order, are split greedily into groups whose span stays below the
// pairing distance; each group costs as many cycles as its most used bank.
int64_t bank_cycles(const OHw &hw, const std::vector<int64_t> &addrs) {
  std::set<int64_t> words;
  for (int64_t a : addrs) words.insert(floordiv(a, hw.bank_bytes));
  int64_t cycles = 0;
  auto it = words.begin();
  while (it != words.end()) {
    int64_t first = *it;
    std::map<int64_t, int64_t> per_bank;
    while (it != words.end() && (*it - first) * hw.bank_bytes < hw.pair_dist) {
      int64_t b = ((*it % hw.banks) + hw.banks) % hw.banks;
      per_bank[b] += 1;
      ++it;
    }
    int64_t m = 0;
    for (auto &kv : per_bank) m = std::max(m, kv.second);
    cycles += m;
  }
  return cycles;
}

// A sector or line of the wave-level sets.  Linear addresses: (address / unit, 0, 0).
// Multi-dimensional address space (Sec. 4.4.1): the innermost coordinate in bytes
// divided by the unit, and the y and z array coordinates; the base alignment is not
// part of it, and two tuples are distinct when any coordinate differs.
typedef std::tuple<int64_t, int64_t, int64_t> Key3;

Key3 wave_key(const OCfg &c, const OField &f, const Thread &t, const Off &o, int64_t unit) {
  if (c.addr_mode == 0) return Key3(floordiv(address(f, t, o), unit), 0, 0);
  // reading: the constant and component offsets are part of the innermost coordinate
  const int64_t xe = f.stride[0] * (t.p[0] + std::get<0>(o)) + f.c + std::get<3>(o);
  return Key3(floordiv(f.esize * xe, unit), t.p[1] + std::get<1>(o), t.p[2] + std::get<2>(o));
}

struct FieldSets {
  std::set<int64_t> blk_ls, blk_ll, blk_ss, blk_sl;            // block: load/store sectors/lines
  std::set<Key3> w_ls, w_ll, w_ss, w_sl;                       // wave
  std::set<Key3> y_ls, y_ll, z_ls, z_ll;                       // layer-condition sets
};

double rhat(const double h[3], double O) { return h[0] * std::exp(-h[1] * std::exp(-h[2] * O)); }

void estimate_one(const OCfg &c, const OHw &hw, int64_t *oi, double *od) {
  for (int i = 0; i < ORC_OUT_NI; ++i) oi[i] = 0;
  for (int i = 0; i < ORC_OUT_ND; ++i) od[i] = 0.0;

  // ---- validity of the candidate --------------------------------------------------
  int64_t T = c.B[0] * c.B[1] * c.B[2];
  bool ok = c.fields.size() > 0 && T >= 1 && T <= 1024 && c.B[2] <= 64 && c.fold >= 1 &&
            c.fold <= 16 && (c.fold_axis != 0 || c.fold == 1) && c.fold_axis >= 0 &&
            c.fold_axis <= 2 && (c.addr_mode == 0 || c.addr_mode == 1);
  for (int d = 0; d < 3; ++d) ok = ok && c.N[d] >= 1 && c.B[d] >= 1;
  for (const OField &f : c.fields) ok = ok && f.esize >= 1 && (f.loads.size() + f.stores.size()) > 0;
  // blocks per SM: thread slots are allocated per warp
  int64_t bpsm = 0;
  if (ok) {
    int64_t warps = ceildiv(T, 32);
    bpsm = std::min(hw.max_blocks_sm, hw.max_threads_sm / (32 * warps));
    if (c.regs > 0) bpsm = std::min(bpsm, hw.regs_sm / (c.regs * 32 * warps));
    ok = bpsm >= 1;
  }
  if (!ok) {
    oi[ORC_I_STATUS] = -1;
    od[ORC_D_T_PRED] = INFINITY;
    return;
  }

  // ---- launch geometry and the thread groups (Sec. 4.3, 4.4) ----------------------
  int64_t fy = c.fold_axis == 1 ? c.fold : 1, fz = c.fold_axis == 2 ? c.fold : 1;
  int64_t g[3] = {ceildiv(c.N[0], c.B[0]), ceildiv(c.N[1], c.B[1] * fy), ceildiv(c.N[2], c.B[2] * fz)};
  int64_t total = g[0] * g[1] * g[2];
  int64_t W = c.wave_override > 0 ? c.wave_override : hw.sms * bpsm;
  int64_t Weff = std::min(W, total);
  // representative block: the middle of the grid
  int64_t rep = (g[0] / 2) + g[0] * ((g[1] / 2) + g[1] * (g[2] / 2));
  // representative wave: the wave (in X-Y-Z scheduling order) that holds it
  int64_t s = W * (rep / W);
  s = std::min(s, total - Weff);
  std::set<int64_t> wave;
  for (int64_t b = s; b < s + Weff; ++b) wave.insert(b);
  // y / z layer-condition sets: the wave shifted back by one block row / slab,
  // blocks outside the grid dropped, minus the wave (and, for z, minus the y set)
  std::set<int64_t> yset, zset;
  for (int64_t b : wave) {
    int64_t by = (b / g[0]) % g[1];
    if (by >= 1 && !wave.count(b - g[0])) yset.insert(b - g[0]);
  }
  for (int64_t b : wave) {
    int64_t bz = b / (g[0] * g[1]);
    int64_t n = b - g[0] * g[1];
    if (bz >= 1 && !wave.count(n) && !yset.count(n)) zset.insert(n);
  }

  std::vector<OField> fields = c.fields;
  for (OField &f : fields) {
    f.fload = fold_list(c, f.loads);
    f.fstore = fold_list(c, f.stores);
  }
  std::vector<FieldSets> fs(fields.size());
  int64_t lups_block = 0, lups_wave = 0, l1_req = 0, l1_store = 0, bank = 0, wave_store_req = 0;

  // ---- representative block: warp / half-warp visitors and block footprint ---------
  int64_t nwarps = ceildiv(T, 32);
  for (int64_t w = 0; w < nwarps; ++w) {
    std::vector<Thread> lanes;
    for (int64_t l = 0; l < 32; ++l) lanes.push_back(make_thread(c, g, rep, 32 * w + l));
    for (const Thread &t : lanes) lups_block += t.valid ? t.kv : 0;
    for (size_t fi = 0; fi < fields.size(); ++fi) {
      const OField &f = fields[fi];
      for (int st = 0; st < 2; ++st) {
        const std::vector<Off> &list = st ? f.fstore : f.fload;
        const std::set<Off> &offs = st ? f.stores : f.loads;
        for (const Off &o : list) {
          std::set<int64_t> warp_sectors;
          std::vector<int64_t> half[2];
          for (int64_t l = 0; l < 32; ++l) {
            const Thread &t = lanes[l];
            if (!t.valid || !access_needed(c, offs, o, t.kv)) continue;
            int64_t a = address(f, t, o);
            warp_sectors.insert(floordiv(a, 32));
            half[l / 16].push_back(a);
            if (st) {
              fs[fi].blk_ss.insert(floordiv(a, 32));
              fs[fi].blk_sl.insert(floordiv(a, 128));
            } else {
              fs[fi].blk_ls.insert(floordiv(a, 32));
              fs[fi].blk_ll.insert(floordiv(a, 128));
            }
          }
          if (st) l1_store += (int64_t)warp_sectors.size();
          else l1_req += (int64_t)warp_sectors.size();
          bank += bank_cycles(hw, half[0]) + bank_cycles(hw, half[1]);
        }
      }
    }
  }

  // ---- wave, y set and z set footprints ----------------------------------------------
  // level 0: wave (loads and stores), 1: y set (loads), 2: z set (loads)
  const std::set<int64_t> *groups[3] = {&wave, &yset, &zset};
  for (int lev = 0; lev < 3; ++lev) {
    for (int64_t b : *groups[lev]) {
      for (int64_t w = 0; w < nwarps; ++w) {
        std::vector<Thread> lanes;
        for (int64_t l = 0; l < 32; ++l) lanes.push_back(make_thread(c, g, b, 32 * w + l));
        if (lev == 0)
          for (const Thread &t : lanes) lups_wave += t.valid ? t.kv : 0;
        for (size_t fi = 0; fi < fields.size(); ++fi) {
          const OField &f = fields[fi];
          for (int st = 0; st < (lev == 0 ? 2 : 1); ++st) {
            const std::vector<Off> &list = st ? f.fstore : f.fload;
            const std::set<Off> &offs = st ? f.stores : f.loads;
            for (const Off &o : list) {
              std::set<Key3> warp_sectors;
              for (int64_t l = 0; l < 32; ++l) {
                const Thread &t = lanes[l];
                if (!t.valid || !access_needed(c, offs, o, t.kv)) continue;
                const Key3 sec = wave_key(c, f, t, o, 32), line = wave_key(c, f, t, o, 128);
                if (lev == 0 && st) {
                  fs[fi].w_ss.insert(sec);
                  fs[fi].w_sl.insert(line);
                  warp_sectors.insert(sec);
                } else if (lev == 0) {
                  fs[fi].w_ls.insert(sec);
                  fs[fi].w_ll.insert(line);
                } else if (lev == 1) {
                  fs[fi].y_ls.insert(sec);
                  fs[fi].y_ll.insert(line);
                } else {
                  fs[fi].z_ls.insert(sec);
                  fs[fi].z_ll.insert(line);
                }
              }
              if (lev == 0 && st) wave_store_req += (int64_t)warp_sectors.size();
            }
          }
        }
      }
    }
  }

  // ---- per-field counts, summed over fields (fields do not alias, Sec. 4.3) ----------
  int64_t bls = 0, bll = 0, bss = 0, bsl = 0, wls = 0, wll = 0, wss = 0, wsl = 0;
  int64_t ovy = 0, ovz = 0, yl = 0, zl = 0;
  for (const FieldSets &f : fs) {
    bls += f.blk_ls.size(); bll += f.blk_ll.size(); bss += f.blk_ss.size(); bsl += f.blk_sl.size();
    wls += f.w_ls.size(); wll += f.w_ll.size(); wss += f.w_ss.size(); wsl += f.w_sl.size();
    yl += f.y_ll.size(); zl += f.z_ll.size();
    for (const Key3 &x : f.w_ls) {
      if (f.y_ls.count(x)) ovy += 1;
      else if (f.z_ls.count(x)) ovz += 1;   // in the z footprint but not the y footprint
    }
  }
  int64_t ydist = yset.empty() ? 0 : s - *yset.begin();
  int64_t zdist = zset.empty() ? 0 : s - *zset.begin();

  oi[ORC_I_LUPS_BLOCK] = lups_block;  oi[ORC_I_LUPS_WAVE] = lups_wave;
  oi[ORC_I_L1_REQ] = l1_req;          oi[ORC_I_BANK_CYCLES] = bank;
  oi[ORC_I_L1_STORE] = l1_store;
  oi[ORC_I_BLK_LOAD_SEC] = bls;       oi[ORC_I_BLK_LOAD_LINES] = bll;
  oi[ORC_I_BLK_STORE_SEC] = bss;      oi[ORC_I_BLK_STORE_LINES] = bsl;
  oi[ORC_I_WAVE_LOAD_SEC] = wls;      oi[ORC_I_WAVE_LOAD_LINES] = wll;
  oi[ORC_I_WAVE_STORE_SEC] = wss;     oi[ORC_I_WAVE_STORE_LINES] = wsl;
  oi[ORC_I_WAVE_STORE_REQ] = wave_store_req;
  oi[ORC_I_OV_Y] = ovy;               oi[ORC_I_OV_Z] = ovz;
  oi[ORC_I_Y_LINES] = yl;             oi[ORC_I_Z_LINES] = zl;
  oi[ORC_I_WAVE_BLOCKS] = Weff;       oi[ORC_I_WAVE_FIRST] = s;
  oi[ORC_I_Y_DIST] = ydist;           oi[ORC_I_Z_DIST] = zdist;
  oi[ORC_I_BLOCKS_PER_SM] = bpsm;

  // ---- volumes per lattice update, capacity misses, limiters (fp64) ----------------
  double lb = (double)lups_block, lw = (double)lups_wave;
  bool cap = hw.cap != 0;
  // L1: V_up = per-instruction sector requests, V_comp = block footprint (Sec. 4.3, 4.5)
  double v_l1 = 32.0 * (double)l1_req / lb;
  double v_l1_comp = 32.0 * (double)bls / lb;
  double o_l1 = 128.0 * (double)bll * (double)bpsm / hw.l1;
  double r_l1 = cap ? rhat(hw.hit[0], o_l1) : 1.0;
  double v_l2_load = v_l1_comp + (1.0 - r_l1) * (v_l1 - v_l1_comp);
  double v_l2_store = 32.0 * (double)l1_store / lb;   // write-through: every store request
  // DRAM: wave footprint minus reuse from the y / z layer sets, plus reads caused by
  // evicted partially written sectors (Sec. 4.4, 5.6)
  double v_dram_comp = 32.0 * (double)wls / lw;
  double alloc_per_block = 128.0 * (double)wll / (double)Weff;
  double o_y = (double)ydist * alloc_per_block / hw.l2;
  double o_z = (double)zdist * alloc_per_block / hw.l2;
  double r_y = cap ? rhat(hw.hit[1], o_y) : 1.0;
  double r_z = cap ? rhat(hw.hit[2], o_z) : 1.0;
  double o_st = 128.0 * (double)wsl / hw.l2;
  double r_st = cap ? rhat(hw.hit[3], o_st) : 1.0;
  double v_red_st = 32.0 * (double)(wave_store_req - wss) / lw;
  double v_dram_load = v_dram_comp - (r_y * (32.0 * (double)ovy) + r_z * (32.0 * (double)ovz)) / lw +
                       (1.0 - r_st) * v_red_st;
  double v_dram_store = 32.0 * (double)wss / lw;
  // limiters, seconds per lattice update for the whole GPU (Sec. 2, 4.2)
  double t_l1 = ((double)bank / lb) / (hw.clock * (double)hw.sms);
  double t_l2 = (v_l2_load + v_l2_store) / hw.bw_l2;
  double t_dram = (v_dram_load + v_dram_store) / hw.bw_dram;
  double t_fp = (c.flops > 0.0 && hw.fp_peak > 0.0) ? c.flops / hw.fp_peak : 0.0;
  double t[4] = {t_l1, t_l2, t_dram, t_fp};
  int lim = 0;
  for (int i = 1; i < 4; ++i)
    if (t[i] > t[lim]) lim = i;
  oi[ORC_I_LIMITER] = lim;

  od[ORC_D_V_L1] = v_l1;             od[ORC_D_V_L2_LOAD] = v_l2_load;
  od[ORC_D_V_L2_STORE] = v_l2_store; od[ORC_D_V_DRAM_LOAD] = v_dram_load;
  od[ORC_D_V_DRAM_STORE] = v_dram_store;
  od[ORC_D_O_L1] = o_l1; od[ORC_D_O_Y] = o_y; od[ORC_D_O_Z] = o_z; od[ORC_D_O_ST] = o_st;
  od[ORC_D_T_L1] = t_l1; od[ORC_D_T_L2] = t_l2; od[ORC_D_T_DRAM] = t_dram; od[ORC_D_T_FP] = t_fp;
  od[ORC_D_T_PRED] = t[lim];
  od[ORC_D_GLUPS] = 1e-9 / t[lim];
}

}  // namespace

extern "C" int orc_estimate(int n_cfg, const int64_t *cfg_i, const double *cfg_d,
                            const int64_t *fld_i, const int64_t *acc_i, const double *hw_d,
                            int64_t *out_i, double *out_d, int threads) {
  if (n_cfg < 0 || (n_cfg > 0 && (!cfg_i || !cfg_d || !fld_i || !acc_i || !hw_d || !out_i || !out_d)))
    return -1;
  OHw hw;
  hw.sms = (int64_t)hw_d[0];
  hw.max_threads_sm = (int64_t)hw_d[1];
  hw.max_blocks_sm = (int64_t)hw_d[2];
  hw.regs_sm = (int64_t)hw_d[3];
  hw.clock = hw_d[4];
  hw.l1 = hw_d[5];
  hw.l2 = hw_d[6];
  hw.bw_l2 = hw_d[7];
  hw.bw_dram = hw_d[8];
  hw.fp_peak = hw_d[9];
  hw.banks = (int64_t)hw_d[10];
  hw.bank_bytes = (int64_t)hw_d[11];
  hw.pair_dist = (int64_t)hw_d[12];
  hw.cap = (int64_t)hw_d[13];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3; ++j) hw.hit[i][j] = hw_d[14 + 3 * i + j];
  if (hw.sms < 1 || hw.banks < 1 || hw.bank_bytes < 1 || hw.max_threads_sm < 1) return -1;

  std::vector<OCfg> cfgs(n_cfg);
  for (int i = 0; i < n_cfg; ++i) {
    const int64_t *ci = cfg_i + (int64_t)i * ORC_CFG_NI;
    OCfg &c = cfgs[i];
    for (int d = 0; d < 3; ++d) {
      c.N[d] = ci[d];
      c.B[d] = ci[3 + d];
    }
    c.fold_axis = ci[6];
    c.fold = ci[7];
    c.regs = ci[10];
    c.wave_override = ci[11];
    c.addr_mode = ci[12];
    c.flops = cfg_d[i];
    for (int64_t fi = 0; fi < ci[8]; ++fi) {
      const int64_t *f = fld_i + (ci[9] + fi) * ORC_FLD_NI;
      OField of;
      of.esize = f[0];
      of.align = f[1];
      of.stride[0] = f[2];
      of.stride[1] = f[3];
      of.stride[2] = f[4];
      of.c = f[5];
      for (int64_t a = 0; a < f[6]; ++a) {
        const int64_t *ac = acc_i + (f[7] + a) * ORC_ACC_NI;
        Off o(ac[0], ac[1], ac[2], ac[4]);
        if (ac[3]) of.stores.insert(o);
        else of.loads.insert(o);
      }
      c.fields.push_back(of);
    }
  }
  if (threads < 1) threads = 1;
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) {
    pool.emplace_back([&, t]() {
      for (int i = t; i < n_cfg; i += threads)
        estimate_one(cfgs[i], hw, out_i + (int64_t)i * ORC_OUT_NI, out_d + (int64_t)i * ORC_OUT_ND);
    });
  }
  for (auto &th : pool) th.join();
  return 0;
}

extern "C" double orc_rank_key(double t) {
  if (!(t > 0.0) || std::isinf(t)) return t;
  int e = 0;
  double m = std::frexp(t, &e);
  return std::ldexp(std::nearbyint(std::ldexp(m, 40)), e - 40);
}

extern "C" int orc_rank(int n, const double *t_pred, int32_t *order_out) {
  if (n < 0 || (n > 0 && (!t_pred || !order_out))) return -1;
  std::vector<std::pair<double, int32_t>> v;
  for (int i = 0; i < n; ++i) {
    double k = t_pred[i];
    if (std::isnan(k)) k = INFINITY;
    v.push_back(std::make_pair(orc_rank_key(k), (int32_t)i));
  }
  std::sort(v.begin(), v.end());   // pairs: key first, index breaks ties
  for (int i = 0; i < n; ++i) order_out[i] = v[i].second;
  return 0;
}
