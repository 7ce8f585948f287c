// Host side of libwarpspeed: context and device arena, descriptor compiler, plans
// (passes, CUDA-graph capture, plain / batched execution), profiling, autotuning,
// ranking.  See warpspeed.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <climits>
#include <condition_variable>
#include <fstream>
#include <functional>
#include <map>
#include <memory>
#include <memory_resource>
#include <unordered_map>
#include <mutex>
#include <new>
#include <set>
#include <sstream>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "ws_host.h"
#include "ws_internal.h"
#include "ws_kernels.h"

static_assert(sizeof(ws_access) == 24, "ws_access layout");
static_assert(sizeof(ws_field) == 56, "ws_field layout");
static_assert(sizeof(ws_config) == 64, "ws_config layout");
static_assert(sizeof(ws_hw) == 176, "ws_hw layout");
static_assert(sizeof(ws_result) == 312, "ws_result layout");
static_assert(sizeof(ws_cfg_info) == 144, "ws_cfg_info layout");
static_assert(sizeof(ws_field_info) == 40, "ws_field_info layout");
static_assert(sizeof(ws_server_stats) == 72, "ws_server_stats layout");

namespace ws {

// ---------------------------------------------------------------------------------
// device arena: first-fit allocator over one device buffer (the memory budget)
// ---------------------------------------------------------------------------------
Arena::Arena(char *b, size_t n) : base(b), size(n) { free_[0] = n; }

int64_t Arena::alloc(size_t bytes) {
  std::lock_guard<std::mutex> g(mu);
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second >= bytes) {
      size_t off = it->first, rem = it->second - bytes;
      free_.erase(it);
      if (rem) free_[off + bytes] = rem;
      used_[off] = bytes;
      in_use += bytes;
      peak = std::max(peak, in_use);
      return (int64_t)off;
    }
  }
  return -1;
}

void Arena::release(int64_t off) {
  if (off < 0) return;
  std::lock_guard<std::mutex> g(mu);
  auto u = used_.find((size_t)off);
  if (u == used_.end()) return;
  size_t o = u->first, n = u->second;
  used_.erase(u);
  in_use -= n;
  auto nx = free_.lower_bound(o);
  if (nx != free_.end() && o + n == nx->first) {
    n += nx->second;
    nx = free_.erase(nx);
  }
  if (nx != free_.begin()) {
    auto pv = std::prev(nx);
    if (pv->first + pv->second == o) {
      pv->second += n;
      return;
    }
  }
  free_[o] = n;
}

size_t Arena::largest_free() {
  std::lock_guard<std::mutex> g(mu);
  size_t m = 0;
  for (auto &kv : free_) m = std::max(m, kv.second);
  return m;
}

size_t Arena::used() {
  std::lock_guard<std::mutex> g(mu);
  return in_use;
}

// ---------------------------------------------------------------------------------
// descriptor compiler
// ---------------------------------------------------------------------------------
// Process-wide cache of large host blocks (sizes rounded up to 2 MiB; a cached block
// serves a request of at least half its size).  Never destroyed: plans may outlive
// static destructors at exit.
namespace {
struct HostBlockCache {
  std::mutex mu;
  std::multimap<size_t, void *> free_;         // cached blocks by size
  std::unordered_map<void *, size_t> size_;    // size of every live or cached block
  size_t cached = 0;
};
HostBlockCache &host_blocks() {
  static HostBlockCache *c = new HostBlockCache;
  return *c;
}
}  // namespace

void *host_block_alloc(size_t bytes) {
  const size_t unit = (size_t)2 << 20, need = (bytes + unit - 1) / unit * unit;
  HostBlockCache &c = host_blocks();
  {
    std::lock_guard<std::mutex> g(c.mu);
    auto it = c.free_.lower_bound(need);
    if (it != c.free_.end() && it->first <= 2 * need) {
      void *p = it->second;
      c.cached -= it->first;
      c.free_.erase(it);
      return p;
    }
  }
  void *p = aligned_alloc(4096, need);
  if (!p) throw std::bad_alloc();
  std::lock_guard<std::mutex> g(c.mu);
  c.size_[p] = need;
  return p;
}

void host_block_free(void *p) {
  if (!p) return;
  HostBlockCache &c = host_blocks();
  std::lock_guard<std::mutex> g(c.mu);
  auto it = c.size_.find(p);
  if (it == c.size_.end()) return;
  if (c.cached + it->second <= ((size_t)1 << 30)) {
    c.free_.emplace(it->second, p);
    c.cached += it->second;
  } else {
    c.size_.erase(it);
    free(p);
  }
}

// Page-locked blocks: their own cache, sizes rounded up to 64 KiB below 2 MiB and to 2 MiB
// above; a cached block serves requests of at least half its size.  cudaHostAlloc is tried
// once per process: without a usable device the blocks are plain memory.
namespace {
struct PinnedBlock {
  size_t size;
  bool locked;     // page-locked (cudaHostAlloc)
  bool cacheable;  // returned to the cache when released (else freed)
};
struct PinnedCache {
  std::mutex mu;
  std::multimap<size_t, void *> free_;
  std::unordered_map<void *, PinnedBlock> size_;
  size_t cached = 0;
  int state = 0;   // 0 untried, 1 cudaHostAlloc works, -1 it does not
};
PinnedCache &pinned_blocks() {
  static PinnedCache *c = new PinnedCache;
  return *c;
}
thread_local bool t_no_pinned = false;
std::atomic<int64_t> g_resources[N_RES];
}  // namespace

void count_resource(ResourceKind k) { g_resources[k].fetch_add(1, std::memory_order_relaxed); }

NoPinnedScope::NoPinnedScope() : prev(t_no_pinned) { t_no_pinned = true; }
NoPinnedScope::~NoPinnedScope() { t_no_pinned = prev; }

void *pinned_block_alloc(size_t bytes) {
  const size_t unit = bytes < ((size_t)2 << 20) ? ((size_t)64 << 10) : ((size_t)2 << 20);
  const size_t need = std::max(unit, (bytes + unit - 1) / unit * unit);
  PinnedCache &c = pinned_blocks();
  std::lock_guard<std::mutex> g(c.mu);
  auto it = c.free_.lower_bound(need);
  if (it != c.free_.end() && it->first <= 2 * need) {
    void *p = it->second;
    c.cached -= it->first;
    c.free_.erase(it);
    return p;
  }
  void *p = nullptr;
  bool locked = false;
  if (c.state >= 0 && !t_no_pinned) {
    if (cudaHostAlloc(&p, need, cudaHostAllocDefault) == cudaSuccess) {
      c.state = 1;
      locked = true;
      count_resource(RES_PINNED_ALLOC);
    } else {
      cudaGetLastError();   // not sticky: leave no error behind for later calls
      p = nullptr;
      c.state = -1;
    }
  }
  if (!p) p = aligned_alloc(4096, need);
  if (!p) throw std::bad_alloc();
  c.size_[p] = PinnedBlock{need, locked, !t_no_pinned};
  return p;
}

void pinned_block_free(void *p) {
  if (!p) return;
  PinnedCache &c = pinned_blocks();
  std::lock_guard<std::mutex> g(c.mu);
  auto it = c.size_.find(p);
  if (it == c.size_.end()) return;
  if (it->second.cacheable && c.cached + it->second.size <= ((size_t)1 << 30)) {
    c.free_.emplace(it->second.size, p);
    c.cached += it->second.size;
  } else {
    if (it->second.locked) cudaFreeHost(p);
    else free(p);
    c.size_.erase(it);
  }
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static int64_t floor_div128(__int128 a, int64_t b) {
  if (b > 0 && (b & (b - 1)) == 0) return (int64_t)(a >> __builtin_ctzll((unsigned long long)b));   // arithmetic shift = floor
  __int128 q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return (int64_t)q;
}

// Inclusive block-coordinate box of the contiguous block-id range [a, b), b > a.
static void block_box(int64_t a, int64_t b, const int64_t g[3], int64_t lo[3], int64_t hi[3]) {
  int64_t last = b - 1;
  int64_t za = a / (g[0] * g[1]), zb = last / (g[0] * g[1]);
  lo[2] = za;
  hi[2] = zb;
  if (za == zb) {
    lo[1] = (a / g[0]) % g[1];
    hi[1] = (last / g[0]) % g[1];
  } else {
    lo[1] = 0;
    hi[1] = g[1] - 1;
  }
  if (a / g[0] == last / g[0]) {
    lo[0] = a % g[0];
    hi[0] = last % g[0];
  } else {
    lo[0] = 0;
    hi[0] = g[0] - 1;
  }
}

static FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.s = 0;
  while (((uint64_t)1 << f.s) < d) ++f.s;
  f.m = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << f.s) - d)) / d + 1);
  f.pad = 0;
  return f;
}

// What one candidate compiles to.  Its arrays come from a memory resource: in plan
// creation, the monotonic arena of the worker that compiled it (no per-candidate heap
// traffic, everything released at once).
struct Compiled {
  explicit Compiled(std::pmr::memory_resource *r = std::pmr::get_default_resource())
      : f(r), acc(r), iv(r), acc_off(r), iv_off(r), fkey(r), need_words(r) {}
  DCfg d{};
  WarpClasses cls;                    // block warp classes for the layout of field 0
  int64_t lvl_blocks[3] = {0, 0, 0};  // blocks of the wave, y set and z set
  bool rows_geom_ok = false;          // row slots fit the kernel's 32-bit decode
  std::pmr::vector<DField> f;
  std::pmr::vector<DAcc> acc;       // access lists of all its fields, field k at [acc_off[k], acc_off[k + 1])
  std::pmr::vector<DIv> iv;         // merged load intervals likewise
  std::pmr::vector<int32_t> acc_off, iv_off;
  std::pmr::vector<uint64_t> fkey;  // (field index, folding): equal keys have equal access lists
  std::pmr::vector<int64_t> need_words;  // bitmap words per field
  size_t dsc_bytes = 0;             // descriptor bytes of its fields, lists and groups
  size_t need_sum = 0, need_max = 0;  // bitmap bytes of all its fields / of its largest
  size_t items_est = 0;             // bound on its work items (owner table entries)
  int64_t n_acc_own = 0, n_iv_own = 0;  // list entries of its fields that no other candidate shares
  bool any_shared = false;          // some field's lists may be shared with other candidates
};

// Upstream of the compile arenas: large blocks from the host block cache.
class BlockResource : public std::pmr::memory_resource {
  void *do_allocate(size_t bytes, size_t align) override {
    if (bytes >= kHostBlockMin && align <= 4096) return host_block_alloc(bytes);
    return std::pmr::new_delete_resource()->allocate(bytes, align);
  }
  void do_deallocate(void *p, size_t bytes, size_t align) override {
    if (bytes >= kHostBlockMin && align <= 4096) host_block_free(p);
    else std::pmr::new_delete_resource()->deallocate(p, bytes, align);
  }
  bool do_is_equal(const std::pmr::memory_resource &o) const noexcept override { return this == &o; }
};

// The candidates of one plan creation: comp[i] lives in the arena of the pool task that
// compiled it; destroying the arenas releases everything (Compiled holds no other
// resources, so its destructor is not needed).
struct CompileArena {
  BlockResource upstream;
  std::vector<std::unique_ptr<std::pmr::monotonic_buffer_resource>> res;
  std::vector<Compiled *> comp;
};

// What a field compiles to for one folding (independent of domain and block shape):
// folded access list with byte offsets and first needed folded point, the raw offset
// range, and per-kv issued-access counts.
struct FieldFold {
  int status = WS_OK;
  std::vector<DAcc> da;
  std::vector<DIv> iv;     // merged load runs: without a covering run, covered from another z row, from their own
  int32_t n_iv_unc = 0;     // runs without a covering run
  int32_t n_iv_zc = 0;      // runs whose covering run lies in another z row (they come next)
  int16_t cov_dy = 0, cov_dz = 0;   // largest |row displacement| to a covering run
  int16_t cov_dy_y = 0;     // largest |ddy| of the runs covered within their z row (they come last)
  int32_t n_load = 0, n_store = 0;
  __int128 omin = 0, omax = 0;
  int16_t cnt_load[17], cnt_store[17];
};
typedef std::map<uint64_t, FieldFold> FieldCache;

// A folded offset (dx, dy, dz, dc) packed so that unsigned order is lexicographic order:
// |dx|, |dy|, |dz| <= 65535 + 15 fit 18 bits after a 2^17 bias, |dc| < 2^40 fits 41 bits
// after a 2^40 bias; the low 4 bits carry the folded point k (< 16).
typedef unsigned __int128 OffKey;
static inline OffKey off_key(int64_t dx, int64_t dy, int64_t dz, int64_t dc, int k) {
  return ((OffKey)(uint64_t)(dx + (1 << 17)) << 81) | ((OffKey)(uint64_t)(dy + (1 << 17)) << 63) |
         ((OffKey)(uint64_t)(dz + (1 << 17)) << 45) | ((OffKey)(uint64_t)(dc + ((int64_t)1 << 40)) << 4) |
         (OffKey)(unsigned)k;
}
static inline void off_unkey(OffKey q, int64_t o[4]) {
  o[0] = (int64_t)(uint64_t)(q >> 81) - (1 << 17);
  o[1] = (int64_t)((uint64_t)(q >> 63) & ((1u << 18) - 1)) - (1 << 17);
  o[2] = (int64_t)((uint64_t)(q >> 45) & ((1u << 18) - 1)) - (1 << 17);
  o[3] = (int64_t)((uint64_t)(q >> 4) & (((uint64_t)1 << 41) - 1)) - ((int64_t)1 << 40);
}

static void compile_field_fold(const ws_field &F, const ws_access *acc, int n_acc, int fold_axis, int fold,
                               FieldFold &out) {
  out.status = WS_OK;
  if (F.elem_bytes < 1 || F.elem_bytes > 64 || F.n_access < 1 || F.access_off < 0 ||
      F.access_off + F.n_access > n_acc) {
    out.status = WS_EINVAL;
    return;
  }
  for (int k = 0; k < 3; ++k)
    if (std::llabs(F.stride[k]) >= ((int64_t)1 << 40)) out.status = WS_EINVAL;
  if (std::llabs(F.align_bytes) >= ((int64_t)1 << 50) || std::llabs(F.const_off) >= ((int64_t)1 << 40))
    out.status = WS_EINVAL;
  if (out.status != WS_OK) return;
  auto off_elems = [&](int64_t dx, int64_t dy, int64_t dz, int64_t dc) -> __int128 {
    return (__int128)F.stride[0] * dx + (__int128)F.stride[1] * dy + (__int128)F.stride[2] * dz + dc;
  };
  // thread folding (Sec. 5.2): union over k of offset + k * axis, each with the first
  // folded point k that needs it (ascending offsets); loads and stores separately.  An
  // issued folded access o' of a thread whose first point is p0 touches the same address
  // as the raw offset o = o' - kmin * e from the valid point p0 + kmin * e, so valid
  // points x raw offsets bound every address of the field.
  static thread_local std::vector<OffKey> lk, sk;
  lk.clear();
  sk.clear();
  bool first = true;
  for (int a = 0; a < F.n_access; ++a) {
    const ws_access &A = acc[F.access_off + a];
    if (std::abs(A.dx) > 65535 || std::abs(A.dy) > 65535 || std::abs(A.dz) > 65535 ||
        std::llabs(A.dc) >= ((int64_t)1 << 40) || (A.is_store != 0 && A.is_store != 1)) {
      out.status = WS_EINVAL;
      return;
    }
    const __int128 e = off_elems(A.dx, A.dy, A.dz, A.dc);
    if (first || e < out.omin) out.omin = e;
    if (first || e > out.omax) out.omax = e;
    first = false;
    std::vector<OffKey> &v = A.is_store ? sk : lk;
    for (int k = 0; k < fold; ++k)
      v.push_back(off_key(A.dx, A.dy + (fold_axis == 1 ? k : 0), A.dz + (fold_axis == 2 ? k : 0), A.dc, k));
  }
  int hist[2][16] = {{0}};
  for (int ls = 0; ls < 2; ++ls) {
    std::vector<OffKey> &v = ls ? sk : lk;
    std::sort(v.begin(), v.end());
    size_t m = 0;
    for (size_t i = 0; i < v.size(); ++i)
      if (i == 0 || (v[i] >> 4) != (v[m - 1] >> 4)) v[m++] = v[i];
    v.resize(m);
  }
  if ((int64_t)(lk.size() + sk.size()) > kMaxFoldedAccesses) {
    out.status = WS_EINVAL;
    return;
  }
  out.da.resize(lk.size() + sk.size());
  size_t n = 0;
  for (int ls = 0; ls < 2; ++ls)
    for (OffKey q : ls ? sk : lk) {
      int64_t o[4];
      off_unkey(q, o);
      DAcc &x = out.da[n++];
      x.boff = (int64_t)(off_elems(o[0], o[1], o[2], o[3]) * F.elem_bytes);
      x.kmin = (int32_t)(q & 15);
      x.pad = 0;
      hist[ls][x.kmin] += 1;
    }
  out.n_load = (int32_t)lk.size();
  out.n_store = (int32_t)sk.size();
  // merged load intervals: sorted load offsets cut wherever two neighbours are more than
  // 32 B apart (a chain of byte addresses with steps of at most 32 B touches every
  // sector between its ends); for each, the grid row of its offsets and its covering run
  {
    struct Ld {
      int64_t b, o[4];   // byte offset; dx dy dz dc
    };
    static thread_local std::vector<Ld> b;
    b.resize((size_t)out.n_load);
    for (int i = 0; i < out.n_load; ++i) {
      b[(size_t)i].b = out.da[(size_t)i].boff;
      off_unkey(lk[(size_t)i], b[(size_t)i].o);
    }
    std::sort(b.begin(), b.end(), [](const Ld &p, const Ld &q) { return p.b < q.b; });
    struct RunRow {
      bool one_row;
      int64_t dy, dz, dc, dxlo, dxhi;
    };
    static thread_local std::vector<RunRow> rr;
    rr.clear();
    out.iv.clear();
    for (size_t i = 0; i < b.size();) {
      size_t j = i;
      while (j + 1 < b.size() && b[j + 1].b - b[j].b <= 32) ++j;
      DIv v;
      v.boff = b[i].b;
      v.ext = (uint32_t)(b[j].b - b[i].b);
      v.ddy = kNoCover;
      v.ddz = 0;
      out.iv.push_back(v);
      RunRow r{true, b[i].o[1], b[i].o[2], b[i].o[3], b[i].o[0], b[i].o[0]};
      for (size_t q = i; q <= j; ++q) {
        r.one_row = r.one_row && b[q].o[1] == r.dy && b[q].o[2] == r.dz && b[q].o[3] == r.dc;
        r.dxlo = std::min(r.dxlo, b[q].o[0]);
        r.dxhi = std::max(r.dxhi, b[q].o[0]);
      }
      rr.push_back(r);
      i = j + 1;
    }
    // covering runs: order runs by (|dy| + |dz|, dz, dy); a run may be covered by an earlier
    // one of the same dc whose x offsets contain its own, at a row displacement a thread row
    // can make (a multiple of the fold along the folding axis); the nearest one is taken
    const size_t nr = rr.size() <= 512 ? rr.size() : 0;   // bounded host work: no covering beyond 512 runs
    // The covering run of a run e: among the runs of lower rank (|dy| + |dz|, dz, dy, run)
    // with the same dc whose x offsets contain its own, at a row displacement a thread row
    // can make (a multiple of the fold along the folding axis, below 32767 in y and z), the
    // nearest one, the first of the nearest in run order.  Only one-row runs take part.  They
    // are visited in rank order, each scanning those before it; the smallest (displacement,
    // run) score picks the cover.  The rank packs into one integer: |dy|, |dz| <= 65535 + 15
    // fit 18 bits after a 2^17 bias, their sum 18 bits, the run index (< 512) 9 bits.
    static thread_local std::vector<int64_t> rk, ry, rz, rres, rxlo, rxhi, rdc, ridx;
    rk.clear();
    for (size_t e = 0; e < nr; ++e)
      if (rr[e].one_row)
        rk.push_back((int64_t)(((uint64_t)(std::llabs(rr[e].dy) + std::llabs(rr[e].dz)) << 45) |
                               ((uint64_t)(rr[e].dz + (1 << 17)) << 27) | ((uint64_t)(rr[e].dy + (1 << 17)) << 9) |
                               (uint64_t)e));
    std::sort(rk.begin(), rk.end());
    const size_t no = rk.size();
    for (auto *v : {&ry, &rz, &rres, &rxlo, &rxhi, &rdc, &ridx}) v->resize(no);
    const int64_t fm = fold_axis == 0 ? 1 : fold;
    for (size_t i = 0; i < no; ++i) {
      const size_t e = (size_t)(rk[i] & 511);
      const RunRow &r = rr[e];
      ridx[i] = (int64_t)e;
      ry[i] = r.dy;
      rz[i] = r.dz;
      const int64_t ax = fold_axis == 1 ? r.dy : fold_axis == 2 ? r.dz : 0;
      rres[i] = ((ax % fm) + fm) % fm;
      rxlo[i] = r.dxlo;
      rxhi[i] = r.dxhi;
      rdc[i] = r.dc;
    }
    for (size_t i = 1; i < no; ++i) {
      const int64_t ye = ry[i], ze = rz[i], re = rres[i], xlo = rxlo[i], xhi = rxhi[i], dce = rdc[i];
      int64_t best_score = INT64_MAX;
      for (size_t j = 0; j < i; ++j) {
        const int64_t ddy = ye - ry[j], ddz = ze - rz[j];
        const int64_t ay = ddy < 0 ? -ddy : ddy, az = ddz < 0 ? -ddz : ddz;
        const bool ok = (rdc[j] == dce) & (rxlo[j] <= xlo) & (rxhi[j] >= xhi) & (rres[j] == re) & (ay < 32767) &
                        (az < 32767);
        const int64_t score = ok ? (((ay + az) << 9) | ridx[j]) : INT64_MAX;
        best_score = score < best_score ? score : best_score;
      }
      if (best_score != INT64_MAX) {
        const size_t e = (size_t)ridx[i], best = (size_t)(best_score & 511);
        out.iv[e].ddy = (int16_t)(rr[e].dy - rr[best].dy);
        out.iv[e].ddz = (int16_t)(rr[e].dz - rr[best].dz);
      }
    }
    // runs without a covering run first, then those covered from another z row, then those
    // covered within their own z row (ddz == 0): the row walk takes only the first kind at
    // rows whose displaced rows all lie inside the level, the first two kinds at rows whose
    // rows displaced in y alone do, and all runs elsewhere
    auto kind = [](const DIv &v) { return v.ddy == kNoCover ? 0 : v.ddz != 0 ? 1 : 2; };
    {
      static thread_local std::vector<DIv> tmp;
      tmp.clear();
      for (int kd = 0; kd < 3; ++kd)
        for (const DIv &v : out.iv)
          if (kind(v) == kd) tmp.push_back(v);
      out.iv.swap(tmp);
    }
    out.n_iv_unc = out.n_iv_zc = 0;
    out.cov_dy = out.cov_dz = out.cov_dy_y = 0;
    for (const DIv &v : out.iv) {
      const int kd = kind(v);
      if (kd == 0) {
        ++out.n_iv_unc;
        continue;
      }
      if (kd == 1) ++out.n_iv_zc;
      else out.cov_dy_y = std::max<int16_t>(out.cov_dy_y, (int16_t)std::abs(v.ddy));
      out.cov_dy = std::max<int16_t>(out.cov_dy, (int16_t)std::abs(v.ddy));
      out.cov_dz = std::max<int16_t>(out.cov_dz, (int16_t)std::abs(v.ddz));
    }
  }
  // issued accesses of a thread with kv valid folded points: those with kmin < kv
  int nl = 0, ns = 0;
  for (int kv = 0; kv <= 16; ++kv) {
    out.cnt_load[kv] = (int16_t)nl;
    out.cnt_store[kv] = (int16_t)ns;
    if (kv < 16) {
      nl += hist[0][kv];
      ns += hist[1][kv];
    }
  }
}

// Classes of the representative block's warps that give identical per-instruction counts
// (distinct sectors, half-warp bank cycles) for every access of fields with one element
// size and strides: warps whose lanes sit at the same relative points with the same valid
// folded points, and whose lane-0 addresses differ by a multiple of lcm(32, banks * bank
// width) (a translation by such a multiple moves no lane to another sector position or
// bank, and the pairing groups depend on differences only).
static void block_warp_classes(const DCfg &d, int64_t esize, const int64_t stride[3], const ws_hw &hw,
                               WarpClasses &out) {
  auto gcd = [](int64_t a, int64_t b) {
    while (b) {
      const int64_t t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  const int64_t bankp = (int64_t)hw.banks * hw.bank_bytes;
  const int64_t period = 32 / gcd(32, bankp) * bankp;
  const int64_t g0 = d.g[0], g1 = d.g[1];
  const int64_t bx = d.rep % g0, by = (d.rep / g0) % g1, bz = d.rep / (g0 * g1);
  const int64_t fy = d.fold_axis == 1 ? d.fold : 1, fz = d.fold_axis == 2 ? d.fold : 1;
  const int64_t B0 = d.B[0], B1 = d.B[1];
  int64_t ref[32][3];   // lane-0 point of each warp
  int32_t id[32];       // warps with equal ids have equal lane layouts and valid points
  // A block whose points are all inside the domain with whole folds gives every thread
  // the same valid folded points, and a full warp's lane offsets from lane 0 depend only
  // on where its thread index carries into y (first lane c1) and into z (first lane c2).
  // Such warps are keyed by (c1, c2); keys whose layouts coincide share an id.  Other
  // blocks compare the lanes of every warp.
  const bool interior = (bx + 1) * B0 <= d.N[0] && (by + 1) * B1 * fy <= d.N[1] && (bz + 1) * d.B[2] * fz <= d.N[2];
  if (interior) {
    int32_t key[32][2], nk = 0, kid[32];
    int32_t rel[32][32][3];   // lane offsets of each distinct key
    for (int w = 0; w < d.wpb; ++w) {
      const int64_t t0 = 32 * (int64_t)w, tx0 = t0 % B0, ty0 = (t0 / B0) % B1, tz0 = t0 / (B0 * B1);
      ref[w][0] = bx * B0 + tx0;
      ref[w][1] = (by * B1 + ty0) * fy;
      ref[w][2] = (bz * d.B[2] + tz0) * fz;
      if (d.T - t0 < 32) {   // the partial last warp: its missing lanes make it unique
        id[w] = -1 - w;
        continue;
      }
      const int32_t c1 = (int32_t)std::min<int64_t>(B0 - tx0, 32), c2 = (int32_t)std::min<int64_t>((B1 - ty0) * B0 - tx0, 32);
      int k = 0;
      while (k < nk && !(key[k][0] == c1 && key[k][1] == c2)) ++k;
      if (k == nk) {
        key[k][0] = c1;
        key[k][1] = c2;
        int64_t tx = tx0, ty = ty0, tz = 0;
        for (int l = 0; l < 32; ++l) {
          rel[k][l][0] = (int32_t)(tx - tx0);
          rel[k][l][1] = (int32_t)((ty - ty0) * fy);
          rel[k][l][2] = (int32_t)(tz * fz);
          if (++tx == B0) {
            tx = 0;
            if (++ty == B1) {
              ty = 0;
              ++tz;
            }
          }
        }
        kid[k] = k;
        for (int q = 0; q < k; ++q)
          if (kid[q] == q && memcmp(rel[q], rel[k], sizeof(rel[k])) == 0) {
            kid[k] = q;
            break;
          }
        ++nk;
      }
      id[w] = kid[k];
    }
  } else {
    // lane points relative to lane 0 and valid folded points (kv, -1 = no thread); the
    // thread coordinates advance incrementally in x-y-z order
    int32_t rel[32][32][4];
    int64_t tx = 0, ty = 0, tz = 0;
    for (int w = 0; w < d.wpb; ++w) {
      for (int l = 0; l < 32; ++l) {
        const int64_t tid = 32 * w + l;
        int64_t x = 0, y = 0, z = 0, kv = -1;
        if (tid < d.T) {
          x = bx * B0 + tx;
          y = (by * B1 + ty) * fy;
          z = (bz * d.B[2] + tz) * fz;
          const bool valid = x < d.N[0] && y < d.N[1] && z < d.N[2];
          kv = !valid ? 0 : d.fold_axis == 1 ? std::min<int64_t>(d.fold, d.N[1] - y)
                          : d.fold_axis == 2 ? std::min<int64_t>(d.fold, d.N[2] - z) : 1;
          if (++tx == B0) {
            tx = 0;
            if (++ty == B1) {
              ty = 0;
              ++tz;
            }
          }
        }
        if (l == 0) {
          ref[w][0] = x;
          ref[w][1] = y;
          ref[w][2] = z;
        }
        int32_t *r = rel[w][l];
        r[0] = (int32_t)(x - ref[w][0]);
        r[1] = (int32_t)(y - ref[w][1]);
        r[2] = (int32_t)(z - ref[w][2]);
        r[3] = (int32_t)kv;
      }
      id[w] = w;
      for (int q = 0; q < w; ++q)
        if (id[q] == q && memcmp(rel[q], rel[w], sizeof(rel[w])) == 0) {
          id[w] = q;
          break;
        }
    }
  }
  out.n = 0;
  for (int w = 0; w < d.wpb; ++w) {
    int c = 0;
    for (; c < out.n; ++c) {
      const int r = out.warp[c];
      if (id[w] != id[r]) continue;
      const __int128 delta = (__int128)esize * (stride[0] * (ref[w][0] - ref[r][0]) + stride[1] * (ref[w][1] - ref[r][1]) +
                                                stride[2] * (ref[w][2] - ref[r][2]));
      if (delta % period == 0) break;
    }
    if (c < out.n) {
      out.mult[c] += 1;
    } else {
      out.warp[out.n] = (uint8_t)w;
      out.mult[out.n] = 1;
      out.n += 1;
    }
  }
}

// Key of a field's folded access list: equal keys have equal lists.
static uint64_t fold_key(const ws_config &c, int fi) {
  return ((uint64_t)(c.field_off + fi) << 8) | ((uint64_t)c.fold_axis << 5) | (uint64_t)c.fold;
}
static const uint64_t kNoShare = ~(uint64_t)0;   // a list that no other descriptor shares

// Returns WS_OK or a per-candidate error status.  `cache` (may be null) memoizes the
// per-(field, folding) part across candidates that share fields.
static int compile_config(const ws_config &c, const ws_field *fld, int n_fld, const ws_access *acc, int n_acc,
                          const ws_hw &hw, Compiled &out, FieldCache *cache = nullptr,
                          const uint8_t *field_refs = nullptr) {
  DCfg &d = out.d;
  memset(&d, 0, sizeof(d));
  for (int k = 0; k < 3; ++k) {
    if (c.N[k] < 1 || c.N[k] > (1 << 20) || c.B[k] < 1) return WS_EINVAL;
    d.N[k] = c.N[k];
    d.B[k] = c.B[k];
  }
  const int64_t T = (int64_t)c.B[0] * c.B[1] * c.B[2];
  if (T > 1024 || c.B[2] > 64) return WS_EINVAL;
  if (c.fold_axis < 0 || c.fold_axis > 2 || c.fold < 1 || c.fold > 16) return WS_EINVAL;
  if (c.fold_axis == 0 && c.fold != 1) return WS_EINVAL;
  if (c.n_field < 1 || c.field_off < 0 || c.field_off + c.n_field > n_fld) return WS_EINVAL;
  if (c.regs_per_thread < 0 || c.wave_blocks_override < 0) return WS_EINVAL;
  if (c.address_mode != WS_ADDR_LINEAR && c.address_mode != WS_ADDR_MULTIDIM) return WS_EINVAL;
  if (!(c.flops_per_lup >= 0.0) || std::isinf(c.flops_per_lup)) return WS_EINVAL;
  d.fold_axis = c.fold_axis;
  d.fold = c.fold;
  const int64_t fy = c.fold_axis == 1 ? c.fold : 1, fz = c.fold_axis == 2 ? c.fold : 1;
  const int64_t g[3] = {ceil_div(c.N[0], c.B[0]), ceil_div(c.N[1], c.B[1] * fy), ceil_div(c.N[2], c.B[2] * fz)};
  const int64_t total = g[0] * g[1] * g[2];
  if (total >= ((int64_t)1 << 31)) return WS_EINVAL;
  for (int k = 0; k < 3; ++k) d.g[k] = (int32_t)g[k];
  d.T = (int32_t)T;
  d.wpb = (int32_t)ceil_div(T, 32);
  // resident blocks per SM: thread slots are allocated per warp
  int64_t bpsm = std::min<int64_t>(hw.max_blocks_sm, hw.max_threads_sm / (32 * (int64_t)d.wpb));
  if (c.regs_per_thread > 0)
    bpsm = std::min<int64_t>(bpsm, hw.regs_sm / ((int64_t)c.regs_per_thread * 32 * d.wpb));
  if (bpsm < 1) return WS_EINVAL;
  d.bpsm = (int32_t)bpsm;
  d.flops = c.flops_per_lup;

  // representative block (middle of the grid) and wave (X-Y-Z scheduling order)
  const int64_t W = c.wave_blocks_override > 0 ? c.wave_blocks_override : (int64_t)hw.sms * bpsm;
  const int64_t weff = std::min(W, total);
  const int64_t rep = g[0] / 2 + g[0] * (g[1] / 2 + g[1] * (g[2] / 2));
  int64_t s = W * (rep / W);
  s = std::min(s, total - weff);
  d.rep = rep;
  d.s = s;
  d.weff = weff;
  // y set: wave shifted back one block row, minus the wave: [y_lo, y_hi) with by != gy-1
  int64_t y_lo = std::max<int64_t>(0, s - g[0]), y_hi = std::min(s, s + weff - g[0]);
  if (y_hi <= y_lo || g[1] == 1) y_lo = y_hi = 0;
  // z set: wave shifted back one block slab, minus the wave and the y set
  int64_t z_lo = std::max<int64_t>(0, s - g[0] * g[1]), z_hi = std::min(s, s + weff - g[0] * g[1]);
  if (z_hi <= z_lo) z_lo = z_hi = 0;
  d.y_lo = y_lo; d.y_hi = y_hi; d.z_lo = z_lo; d.z_hi = z_hi;
  auto in_y = [&](int64_t b) { return b >= y_lo && b < y_hi && (b / g[0]) % g[1] != g[1] - 1; };
  // first block of the y set
  int64_t y_first = -1;
  if (y_hi > y_lo) {
    if ((y_lo / g[0]) % g[1] != g[1] - 1) y_first = y_lo;
    else if ((y_lo / g[0] + 1) * g[0] < y_hi) y_first = (y_lo / g[0] + 1) * g[0];
  }
  // first block of the z set: z_lo itself, the first block of a row gy-1 at or after
  // z_lo, or the first block after the y range
  int64_t z_first = -1;
  if (z_hi > z_lo) {
    if (!in_y(z_lo)) {
      z_first = z_lo;
    } else {
      int64_t q0 = z_lo / g[0];
      int64_t q = q0 + ((g[1] - 1 - q0 % g[1]) % g[1] + g[1]) % g[1];
      int64_t cand1 = std::max(z_lo, q * g[0]);
      int64_t cand2 = y_hi;
      int64_t best = -1;
      if (cand1 < z_hi) best = cand1;
      if (cand2 < z_hi && (best < 0 || cand2 < best)) best = cand2;
      z_first = best;
    }
  }
  // The z set is the wave moved back by one block slab (every point z - B2 * fz) when it is
  // the whole shifted wave (the wave lies beyond the first slab, spans at most one slab and
  // ends before the y set begins) and every point of the wave lies inside the domain in z:
  // then the same points are valid in both and every thread issues the same accesses, so a
  // field's z-set addresses are its wave addresses less esize * stride_z * B2 * fz bytes.
  const int64_t slab = g[0] * g[1];
  const bool z_is_shifted_wave = s >= slab && weff <= slab && z_lo == s - slab && z_hi == s + weff - slab &&
                                 (y_hi <= y_lo || z_hi <= y_lo) &&
                                 ((s + weff - 1) / slab + 1) * c.B[2] * fz <= c.N[2];
  d.y_dist = y_first >= 0 ? s - y_first : 0;
  d.z_dist = z_first >= 0 ? s - z_first : 0;
  const int64_t wpb = d.wpb;
  d.lev_end[0] = wpb;
  d.lev_end[1] = d.lev_end[0] + weff * wpb;
  d.lev_end[2] = d.lev_end[1] + (y_hi - y_lo) * wpb;
  d.lev_end[3] = d.lev_end[2] + (z_hi - z_lo) * wpb;
  if (d.lev_end[3] >= ((int64_t)1 << 31)) return WS_EINVAL;
  d.fd_gx = make_fastdiv((uint32_t)g[0]);
  d.fd_gy = make_fastdiv((uint32_t)g[1]);
  // row walk geometry: block rows of each level, slots, and the blocks per level left
  // after the y / z set rules (for the modelled-warp statistics)
  {
    d.rows_per_blk = (int32_t)(c.B[1] * c.B[2]);
    d.full_end = (int32_t)(c.N[0] / c.B[0]);
    d.fd_rows = make_fastdiv((uint32_t)d.rows_per_blk);
    d.fd_b1 = make_fastdiv((uint32_t)c.B[1]);
    d.fd_b2 = make_fastdiv((uint32_t)c.B[2]);
    d.fd_fold = make_fastdiv((uint32_t)c.fold);
    const int64_t rng[4][2] = {{s, s + weff}, {y_lo, y_hi}, {z_lo, z_hi}, {rep, rep + 1}};
    int64_t cum = 0;
    for (int lv = 0; lv < 4; ++lv) {
      d.rows_R_lo[lv] = 0;
      d.rows_R_cnt[lv] = 0;
      if (rng[lv][1] > rng[lv][0]) {
        const int64_t R0 = rng[lv][0] / g[0], R1 = (rng[lv][1] - 1) / g[0];
        d.rows_R_lo[lv] = (int32_t)R0;
        d.rows_R_cnt[lv] = (int32_t)(R1 - R0 + 1);
      }
      cum += (int64_t)d.rows_R_cnt[lv] * d.rows_per_blk;
      d.rows_slot_end[lv] = cum;
    }
    out.rows_geom_ok = cum < ((int64_t)1 << 31);
    // blocks b < n of the last block row (by = g[1] - 1)
    auto last_row = [&](int64_t n) {
      const int64_t per = g[0] * g[1];
      int64_t c = (n / per) * g[0];
      const int64_t r = n % per - (g[1] - 1) * g[0];
      return r > 0 ? c + r : c;
    };
    out.lvl_blocks[0] = weff;
    out.lvl_blocks[1] = y_hi > y_lo ? (y_hi - y_lo) - (last_row(y_hi) - last_row(y_lo)) : 0;
    out.lvl_blocks[2] = z_hi - z_lo;
    const int64_t oa = std::max(z_lo, y_lo), ob = std::min(z_hi, y_hi);
    if (z_hi > z_lo && y_hi > y_lo && ob > oa) out.lvl_blocks[2] -= (ob - oa) - (last_row(ob) - last_row(oa));
  }
  d.fd_wpb = make_fastdiv((uint32_t)wpb);

  // point boxes (valid points only) of the block level and of wave + y + z
  int64_t pb_lo[2][3], pb_hi[2][3];
  int64_t pw_lo[3], pw_hi[3];   // the wave's own point box
  {
    int64_t bl2[3], bh2[3];
    block_box(s, s + weff, g, bl2, bh2);
    for (int k = 0; k < 3; ++k) {
      const int64_t f = (k == 1 ? fy : k == 2 ? fz : 1) * c.B[k];
      pw_lo[k] = bl2[k] * f;
      pw_hi[k] = std::min<int64_t>(c.N[k] - 1, (bh2[k] + 1) * f - 1);
    }
  }
  {
    int64_t bl[3] = {rep % g[0], (rep / g[0]) % g[1], rep / (g[0] * g[1])};
    for (int k = 0; k < 3; ++k) {
      int64_t f = (k == 1 ? fy : k == 2 ? fz : 1) * c.B[k];
      pb_lo[0][k] = bl[k] * f;
      pb_hi[0][k] = std::min<int64_t>(c.N[k] - 1, (bl[k] + 1) * f - 1);
    }
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1};
    const int64_t ranges[3][2] = {{s, s + weff}, {y_lo, y_hi}, {z_lo, z_hi}};
    for (auto &r : ranges) {
      if (r[1] <= r[0]) continue;
      int64_t bl2[3], bh2[3];
      block_box(r[0], r[1], g, bl2, bh2);
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], bl2[k]);
        hi[k] = std::max(hi[k], bh2[k]);
      }
    }
    for (int k = 0; k < 3; ++k) {
      int64_t f = (k == 1 ? fy : k == 2 ? fz : 1) * c.B[k];
      pb_lo[1][k] = lo[k] * f;
      pb_hi[1][k] = std::min<int64_t>(c.N[k] - 1, (hi[k] + 1) * f - 1);
    }
  }

  // fields: folded access lists (Sec. 5.2 thread folding), address ranges, bitmaps.
  // `mask`: levels the descriptor serves (1 the representative block, 2 the wave and the
  // y / z sets); `key`: list-sharing key (kNoShare = never shared)
  out.f.clear();
  out.acc.clear();
  out.acc_off.assign(1, 0);
  out.iv_off.assign(1, 0);
  out.iv.clear();
  out.fkey.clear();
  out.need_words.clear();
  {
    const size_t nd = (size_t)c.n_field * (c.address_mode == WS_ADDR_MULTIDIM ? 2 : 1);
    out.f.reserve(nd);
    out.acc_off.reserve(nd + 1);
    out.iv_off.reserve(nd + 1);
    // folded accesses and merged runs: at most fold per raw access (no regrowth in the arena)
    size_t na = 0;
    for (int fi = 0; fi < c.n_field; ++fi) na += (size_t)std::max(0, fld[c.field_off + fi].n_access) * (size_t)c.fold;
    if (na <= (size_t)kMaxFoldedAccesses * (size_t)c.n_field) {
      out.acc.reserve(na * (nd / (size_t)c.n_field));
      out.iv.reserve(na * (nd / (size_t)c.n_field));
    }
    out.fkey.reserve(nd);
    out.need_words.reserve(nd);
  }
  // Pairs of thread rows (t = ty + B1 * tz) ta < tb = ta + j that share a warp.  With
  // jq = j / B1 and jr = j % B1 their (ty, tz) offsets are (jr, jq) when ta % B1 + jr < B1
  // and (jr - B1, jq + 1) otherwise; bit 0 / bit 1 of pair_kind[j] record which occur.
  // The rows of a warp are consecutive, so the residues ta % B1 of its pairs at distance
  // j form one cyclic run starting at t0 % B1.
  uint8_t pair_kind[32] = {0};
  bool pairs_done = false;
  auto row_pairs = [&]() {
    if (pairs_done) return;
    pairs_done = true;
    const int64_t B1 = c.B[1], nrows = (int64_t)c.B[1] * c.B[2];
    for (int64_t w = 0; w < d.wpb; ++w) {
      const int64_t t0 = (32 * w) / c.B[0], t1 = std::min<int64_t>((32 * w + 31) / c.B[0], nrows - 1);
      const int64_t r0 = t0 % B1;
      for (int64_t j = 1; j <= t1 - t0; ++j) {
        const int64_t jr = j % B1, last = r0 + (t1 - j - t0);   // residues r0 .. last (mod B1)
        if (r0 < B1 - jr || last >= B1) pair_kind[j] |= 1;
        if (jr > 0 && last >= B1 - jr) pair_kind[j] |= 2;
      }
    }
  };
  auto emit = [&](const ws_field &F, const FieldFold *ff, int mask, uint64_t key, bool first) -> int {
    DField df;
    memset(&df, 0, sizeof(df));
    df.esize = F.elem_bytes;
    for (int k = 0; k < 3; ++k) df.stride[k] = F.stride[k];
    df.base = F.align_bytes + (int64_t)F.elem_bytes * F.const_off;
    df.n_load = ff->n_load;
    df.n_store = ff->n_store;
    df.level_mask = mask;
    const __int128 omin = ff->omin, omax = ff->omax;
    // address range of each level: valid point box x raw offsets
    for (int lv = 0; lv < 2; ++lv) {
      df.lo[lv] = 0;
      df.words[lv] = 0;
      if (!(mask & (1 << lv))) continue;
      __int128 pmin = 0, pmax = 0;
      for (int k = 0; k < 3; ++k) {
        __int128 a0 = (__int128)F.stride[k] * pb_lo[lv][k], a1 = (__int128)F.stride[k] * pb_hi[lv][k];
        pmin += std::min(a0, a1);
        pmax += std::max(a0, a1);
      }
      __int128 amin = (__int128)df.base + (__int128)F.elem_bytes * (pmin + omin);
      __int128 amax = (__int128)df.base + (__int128)F.elem_bytes * (pmax + omax);
      if (amin < -((__int128)1 << 60) || amax > ((__int128)1 << 60)) return WS_EINVAL;
      int64_t lo = floor_div128(amin, 1024) * 32;
      int64_t hi = floor_div128(amax, 32);
      int64_t words = ceil_div(hi - lo + 1, 32);
      words = (words + 3) & ~(int64_t)3;
      if (words > kMaxBitmapWords) return WS_ENOMEM;
      df.lo[lv] = lo;
      df.words[lv] = words;
    }
    const bool has_l = df.n_load > 0, has_s = df.n_store > 0;
    // z set = wave moved by a multiple of 128 bytes: its sector set is the wave's moved by
    // whole lines, so it has the wave's line count, and only its sectors inside the wave's
    // address range can meet the wave (the row walk clips the z set's ranges to it)
    df.zshift = 0;
    df.zc_lo = 0;
    df.zc_hi = -1;
    if (z_is_shifted_wave && mask == 3 && has_l &&
        ((__int128)F.elem_bytes * F.stride[2] * c.B[2] * fz) % 128 == 0) {
      __int128 pmin = 0, pmax = 0;
      for (int k = 0; k < 3; ++k) {
        const __int128 a0 = (__int128)F.stride[k] * pw_lo[k], a1 = (__int128)F.stride[k] * pw_hi[k];
        pmin += std::min(a0, a1);
        pmax += std::max(a0, a1);
      }
      const __int128 wmin = (__int128)df.base + (__int128)F.elem_bytes * (pmin + omin);
      const __int128 wmax = (__int128)df.base + (__int128)F.elem_bytes * (pmax + omax);
      const __int128 s0 = floor_div128(wmin, 32) - df.lo[1], s1 = floor_div128(wmax, 32) - df.lo[1];
      df.zshift = 1;
      if (s0 >= 0 && s1 < ((__int128)1 << 31) && s0 <= s1) {
        df.zc_lo = (int32_t)s0;
        df.zc_hi = (int32_t)s1;
      } else {
        df.zc_lo = 0;   // no clipping (the row walk does not take such a field)
        df.zc_hi = INT32_MAX;
      }
    }
    df.mw_block = d.lev_end[0];
    df.mw_end = !(mask & 2) ? d.lev_end[0] : has_l ? d.lev_end[3] : d.lev_end[1];
    df.first_of_cfg = first;
    df.wide = (df.words[0] >= ((int64_t)1 << 22) || df.words[1] >= ((int64_t)1 << 22)) ? 1 : 0;
    df.lpa_log2p = 0;
    while ((1 << df.lpa_log2p) < std::min(df.n_load, 32)) ++df.lpa_log2p;
    // row segments of threads step by elem_bytes * stride_x bytes: at most one sector
    // keeps every segment's sectors contiguous; the walk keeps a warp's addresses as
    // 32-bit offsets, so the wave bitmap must span less than 2^31 bytes
    df.iv = (!df.wide && df.words[1] < ((int64_t)1 << 21) && std::llabs(F.stride[0]) * F.elem_bytes <= 32) ? 1 : 0;
    df.iv_begin = 0;
    df.n_iv = (int32_t)ff->iv.size();
    df.n_iv_unc = ff->n_iv_unc;
    df.n_iv_zc = ff->n_iv_zc;
    df.cov_dy = ff->cov_dy;
    df.cov_dz = ff->cov_dz;
    df.cov_dy_y = ff->cov_dy_y;
    // per-instruction store sectors of the row walk add up the row segments of a warp,
    // exact when no two rows of one warp can touch a common sector: their starts lie
    // further apart than a row's byte span plus 31
    df.rows_ok = 1;
    if (ff->n_store > 0) {
      row_pairs();
      const int64_t span = (int64_t)F.elem_bytes * std::llabs(F.stride[0]) * (c.B[0] - 1);
      const int64_t B1 = c.B[1];
      for (int64_t j = 1; j < 32 && df.rows_ok; ++j)
        for (int k = 0; k < 2; ++k) {
          if (!((pair_kind[j] >> k) & 1)) continue;
          const int64_t dyr = k ? j % B1 - B1 : j % B1, dzr = k ? j / B1 + 1 : j / B1;
          __int128 delta = ((__int128)dyr * fy * F.stride[1] + (__int128)dzr * fz * F.stride[2]) * F.elem_bytes;
          if (delta < 0) delta = -delta;
          if (delta <= (__int128)span + 31) {
            df.rows_ok = 0;
            break;
          }
        }
    }
    for (int kv = 0; kv <= 16; ++kv) {
      df.cnt_load[kv] = ff->cnt_load[kv];
      df.cnt_store[kv] = ff->cnt_store[kv];
    }
    for (int k = 0; k < N_BITMAPS; ++k) df.bm[k] = -1;
    int64_t need = 0;
    if (has_l) need += df.words[0] + 3 * df.words[1];
    if (has_s) need += df.words[0] + df.words[1];
    need += page_flag_words(df.words[0], df.words[1]);   // used when the field takes the row walk
    out.f.push_back(df);
    out.acc.insert(out.acc.end(), ff->da.begin(), ff->da.end());
    out.iv.insert(out.iv.end(), ff->iv.begin(), ff->iv.end());
    out.acc_off.push_back((int32_t)out.acc.size());
    out.iv_off.push_back((int32_t)out.iv.size());
    out.fkey.push_back(key);
    out.need_words.push_back(need);
    return WS_OK;
  };
  // the folded lists of field fi: from the cache when other candidates use the field too,
  // else compiled into `local` (then *own = true: the list is this candidate's alone);
  // tl_fold is this thread's reusable one
  static thread_local FieldFold tl_fold;
  auto fold_of = [&](int fi, FieldFold &local, bool *own) -> FieldFold * {
    const ws_field &F = fld[c.field_off + fi];
    *own = !cache || (field_refs && field_refs[c.field_off + fi] < 2);
    if (*own) {
      compile_field_fold(F, acc, n_acc, c.fold_axis, c.fold, local);
      return &local;
    }
    auto it = cache->find(fold_key(c, fi));
    if (it == cache->end()) {
      it = cache->emplace(fold_key(c, fi), FieldFold()).first;
      compile_field_fold(F, acc, n_acc, c.fold_axis, c.fold, it->second);
    }
    return &it->second;
  };
  if (c.address_mode == WS_ADDR_LINEAR) {
    for (int fi = 0; fi < c.n_field; ++fi) {
      bool own;
      FieldFold *ff = fold_of(fi, tl_fold, &own);
      if (ff->status != WS_OK) return ff->status;
      const int rc = emit(fld[c.field_off + fi], ff, 3, own ? kNoShare : fold_key(c, fi), fi == 0);
      if (rc != WS_OK) return rc;
    }
  } else {
    // Multi-dimensional address space (Sec. 4.4.1) for the wave and the y / z sets: a
    // sector is (innermost bytes / 32, y, z), without the base alignment.  Each field
    // becomes a block descriptor (linear addresses, as the per-instruction statistics
    // of the representative block need) and a wave descriptor over a virtual linear
    // layout in which every (y, z) row is its own 128-byte aligned slab of RS bytes:
    // virtual address = Xbias + innermost bytes + RS * (y - y0) + PS * (z - z0), so
    // that virtual sectors and lines are exactly the tuples.  RS and PS are common to
    // the candidate's fields (equal layouts stay one uniform group).
    for (int fi = 0; fi < c.n_field; ++fi) {
      bool own;
      FieldFold *ff = fold_of(fi, tl_fold, &own);
      if (ff->status != WS_OK) return ff->status;
      const int rc = emit(fld[c.field_off + fi], ff, 1, own ? kNoShare : fold_key(c, fi), fi == 0);
      if (rc != WS_OK) return rc;
    }
    __int128 ymin = 0, ymax = 0, zmin = 0, zmax = 0;
    std::vector<__int128> xlo(c.n_field), xhi(c.n_field);
    int64_t L = 128;
    for (int fi = 0; fi < c.n_field; ++fi) {
      const ws_field &F = fld[c.field_off + fi];
      int64_t r[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};   // dx dy dz dc ranges of the raw offsets
      for (int a = 0; a < F.n_access; ++a) {
        const ws_access &A = acc[F.access_off + a];
        const int64_t v[4] = {A.dx, A.dy, A.dz, A.dc};
        for (int q = 0; q < 4; ++q) {
          r[q][0] = a == 0 ? v[q] : std::min(r[q][0], v[q]);
          r[q][1] = a == 0 ? v[q] : std::max(r[q][1], v[q]);
        }
      }
      const __int128 x0 = (__int128)F.stride[0] * (pb_lo[1][0] + r[0][0]), x1 = (__int128)F.stride[0] * (pb_hi[1][0] + r[0][1]);
      xlo[fi] = (__int128)F.elem_bytes * (std::min(x0, x1) + F.const_off + r[3][0]);
      xhi[fi] = (__int128)F.elem_bytes * (std::max(x0, x1) + F.const_off + r[3][1]);
      const __int128 y0 = pb_lo[1][1] + r[1][0], y1 = pb_hi[1][1] + r[1][1];
      const __int128 z0 = pb_lo[1][2] + r[2][0], z1 = pb_hi[1][2] + r[2][1];
      ymin = fi == 0 ? y0 : std::min(ymin, y0);
      ymax = fi == 0 ? y1 : std::max(ymax, y1);
      zmin = fi == 0 ? z0 : std::min(zmin, z0);
      zmax = fi == 0 ? z1 : std::max(zmax, z1);
      L = L / std::__gcd(L, (int64_t)F.elem_bytes) * F.elem_bytes;
    }
    __int128 row = 0;
    std::vector<__int128> xbias(c.n_field);
    for (int fi = 0; fi < c.n_field; ++fi) {
      xbias[fi] = -floor_div128(xlo[fi], 128) * 128;
      row = std::max(row, xhi[fi] + xbias[fi] + 1);
    }
    const __int128 RS = (row + L - 1) / L * L, PS = RS * (ymax - ymin + 1);
    if (PS * (zmax - zmin + 1) >= ((__int128)1 << 50)) return WS_ENOMEM;
    for (int fi = 0; fi < c.n_field; ++fi) {
      const ws_field &F = fld[c.field_off + fi];
      ws_field V = F;
      V.stride[1] = (int64_t)(RS / F.elem_bytes);
      V.stride[2] = (int64_t)(PS / F.elem_bytes);
      V.align_bytes = (int64_t)(xbias[fi] - RS * ymin - PS * zmin);
      compile_field_fold(V, acc, n_acc, c.fold_axis, c.fold, tl_fold);
      if (tl_fold.status != WS_OK) return tl_fold.status;
      const int rc = emit(V, &tl_fold, 2, kNoShare, false);
      if (rc != WS_OK) return rc;
    }
  }
  d.n_field = c.n_field;
  if (!out.f.empty()) block_warp_classes(d, out.f[0].esize, out.f[0].stride, hw, out.cls);
  return WS_OK;
}

// ---------------------------------------------------------------------------------
// last-error text
// ---------------------------------------------------------------------------------
static thread_local std::string g_last_error;
void set_error(const std::string &s) { g_last_error = s; }
const char *last_error() { return g_last_error.c_str(); }

#define CU(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#x) + ": " + cudaGetErrorString(e_));                      \
      return WS_ECUDA;                                                                 \
    }                                                                                  \
  } while (0)

// ---------------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------------
static DHw to_dhw(const ws_hw &h) {
  DHw d;
  memset(&d, 0, sizeof(d));
  d.clock_hz = h.clock_hz;
  d.l1_bytes = h.l1_bytes;
  d.l2_bytes = h.l2_bytes;
  d.bw_l2 = h.bw_l2;
  d.bw_dram = h.bw_dram;
  d.fp_peak = h.fp_peak;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3; ++j) d.hit[i][j] = h.hit[i][j];
  d.sms = h.sms;
  d.banks = h.banks;
  d.bank_bytes = h.bank_bytes;
  d.pair_dist_bytes = h.pair_dist_bytes;
  d.capacity_model = h.capacity_model;
  return d;
}

static bool hw_valid(const ws_hw &h) {
  return h.sms >= 1 && h.max_threads_sm >= 32 && h.max_blocks_sm >= 1 && h.regs_sm >= 1 && h.banks >= 1 &&
         h.bank_bytes >= 1 && h.pair_dist_bytes >= 1 && h.clock_hz > 0 && h.l1_bytes > 0 && h.l2_bytes > 0 &&
         h.bw_l2 > 0 && h.bw_dram > 0 && h.fp_peak >= 0 && std::isfinite(h.clock_hz) && std::isfinite(h.bw_l2) &&
         std::isfinite(h.bw_dram);
}

}  // namespace ws

using namespace ws;

void *ws_plan::dev(int64_t off) const { return ctx->arena->base + off; }

void ws_plan::release_all() {
  for (int64_t o : allocs) ctx->arena->release(o);
  allocs.clear();
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  graph_exec = nullptr;
}

int64_t ws_plan::take(size_t bytes) {
  int64_t o = ctx->arena->alloc(bytes);
  if (o >= 0) allocs.push_back(o);
  return o;
}

static void default_tuning(ws_tuning &t) {
  // defaults measured on the three workloads: 256-thread enumeration CTAs and chunks of 256
  // modelled warps, what the autotuner picks for the mixed set (its step 22.9 -> 22.0 ms
  // against 512 / 1024; the sweeps equal)
  if (t.chunk_warps <= 0) t.chunk_warps = 256;
  if (t.pass_mb == 0) t.pass_mb = -1;
  if (t.enum_threads <= 0) t.enum_threads = 256;
  if (t.count_words <= 0) t.count_words = 16384;   // 64 KiB of words per counting item (fields without page flags)
  t.enum_threads = std::max(64, std::min(512, t.enum_threads / 32 * 32));
  t.count_words = std::min(kCountMaxWords, std::max(kPageWords, t.count_words / kPageWords * kPageWords));
  t.chunk_warps = std::max(1, t.chunk_warps);
  if (t.pass_mb < 0) t.pass_mb = -1;
  if (t.walk != WS_WALK_ADDRESS && t.walk != WS_WALK_SEGMENT) t.walk = WS_WALK_INTERVAL;
}

// Numbers work items and cuts passes for the current tuning.
// Runs fn(lo, hi) over [0, n) in chunks on the host pool (defined with the pool below).
static void parallel_chunks(int64_t n, int64_t chunk, const std::function<void(int64_t, int64_t)> &fn);

// Counting units of field f (chunks of its block bitmaps' words, then of its wave bitmaps'
// words; each chunk a whole number of pages of one part, larger chunks when only flagged
// pages are read): calls unit(u, pages) for each.
template <class F>
static void for_count_units(const DField &f, bool paged, int count_words, F unit) {
  const int64_t cw = paged ? kPagedChunkWords : count_words;
  const int64_t kb = ceil_div(f.words[0], cw), kw = ceil_div(f.words[1], cw);
  for (int64_t u = 0; u < kb + kw; ++u) {
    const int64_t c0 = (u < kb ? u : u - kb) * cw, w = u < kb ? f.words[0] : f.words[1];
    unit(u, ceil_div(std::min(cw, w - c0), (int64_t)kPageWords));
  }
}

void ws_plan::layout() {
  passes.clear();
  const int ng = (int)hgrp.size();
  // per group (in parallel): walk flags, representative warps, bitmap words the pass holds
  // (need_words bound them, with page flags only for the row walk) and the work items of
  // its kernels
  std::vector<int64_t> gneed((size_t)ng, 0), gwords((size_t)ng, 0);
  parallel_chunks(ng, 512, [&](int64_t lo, int64_t hi) {
    for (int64_t g = lo; g < hi; ++g) {
      DGroup &G = hgrp[(size_t)g];
      G.iv = grp_iv_ok[(size_t)g] && tune.walk != WS_WALK_ADDRESS;
      G.rows = grp_rows_ok[(size_t)g] && tune.walk == WS_WALK_INTERVAL;
      // the row walk builds the block bitmaps, so the block path counts one warp per
      // class; otherwise it inserts every warp
      const bool classes = G.rows && (G.levels & 1) && grp_classes[(size_t)g].n > 0;
      const int wpb = (int)G.mw_block;
      G.n_rep = classes ? grp_classes[(size_t)g].n : wpb;
      for (int r = 0; r < G.n_rep; ++r) {
        G.rep_warp[r] = classes ? grp_classes[(size_t)g].warp[r] : (uint8_t)r;
        G.rep_mult[r] = classes ? grp_classes[(size_t)g].mult[r] : (uint8_t)1;
      }
      for (int k = 0; k < G.f_count; ++k) {
        const DField &f = hfld[(size_t)(G.f_begin + k)];
        gneed[(size_t)g] += need_words[(size_t)(G.f_begin + k)];
        if (f.n_load > 0) gwords[(size_t)g] += f.words[0] + 3 * f.words[1];
        if (f.n_store > 0) gwords[(size_t)g] += f.words[0] + f.words[1];
        if (G.rows) gwords[(size_t)g] += page_flag_words(f.words[0], f.words[1]);
      }
    }
  });
  // pass capacity: the tuned pass size, never below the largest field group, never
  // above the scratch the plan holds
  int64_t max_need = 0;
  for (int64_t v : gneed) max_need = std::max(max_need, v);
  int64_t cap = scratch_words;
  if (tune.pass_mb > 0) cap = std::min(cap, std::max(max_need, (int64_t)tune.pass_mb << 18));
  // row slots per row-walk item: 256 (one 32-slot batch for each of a CTA's eight warps),
  // doubled up to 1024 while every resident row-walk CTA (four per SM; a dry run without a
  // device assumes 152 SMs) still gets at least 32 items.  Larger items cost less per slot
  // (the mixed set's row walk 12.8 -> 12.0 ms at 1024), the small sweeps need the finer
  // split to balance (LBM 1.33 -> 1.51 ms at 1024)
  {
    int64_t slots = 0;
    for (int g = 0; g < ng; ++g)
      if (hgrp[(size_t)g].rows) slots += grp_slots[(size_t)g];
    const int64_t ctas = 4 * (int64_t)(ctx ? ctx->sm_count : 152);
    rows_chunk = 256;
    while (!plain_layout && rows_chunk < 1024 && slots / (2 * rows_chunk) >= 32 * ctas) rows_chunk *= 2;
  }
  block_pairs = plain_layout ? kPlainBlockPairs : kBlockPairs;
  count_pack = plain_layout ? 1 : kCountItemUnits;
  // passes (a group starts a new one when its words would overflow the capacity), each
  // group's first scratch word in its pass, and the enumeration and row-walk items: the
  // representative block (exact path) in chunks of (modelled warp, instruction) pairs; then
  // chunks of the remaining modelled warps, or, for the row walk, chunks of row slots
  std::vector<int64_t> gbase((size_t)ng, 0);
  std::vector<int32_t> gpass((size_t)ng, 0);
  int64_t items = 0, ritems = 0;
  {
    DPass cur;
    memset(&cur, 0, sizeof(cur));
    int64_t used = 0;
    for (int g = 0; g < ng; ++g) {
      DGroup &G = hgrp[(size_t)g];
      if (used + gneed[(size_t)g] > cap && g > cur.grp_lo) {
        cur.cf_hi = G.f_begin;
        cur.grp_hi = g;
        cur.item_hi = items;
        cur.ritem_hi = ritems;
        cur.words = used;
        passes.push_back(cur);
        memset(&cur, 0, sizeof(cur));
        cur.item_lo = items;
        cur.ritem_lo = ritems;
        cur.cf_lo = G.f_begin;
        cur.grp_lo = g;
        used = 0;
      }
      gpass[(size_t)g] = (int32_t)passes.size();
      gbase[(size_t)g] = used;
      used += gwords[(size_t)g];
      G.item_begin = items;
      G.ritem_begin = ritems;
      G.n0_items = (G.levels & 1) ? (int32_t)std::max<int64_t>(1, ceil_div((int64_t)G.n_rep * G.acc_count, block_pairs))
                                  : 0;
      items += G.n0_items;
      if (G.rows) ritems += ceil_div(grp_slots[(size_t)g], chunk_rows());
      else if (G.levels & 2) items += ceil_div(G.mw_end - G.mw_block, tune.chunk_warps);
    }
    cur.cf_hi = (int)hfld.size();
    cur.grp_hi = ng;
    cur.item_hi = items;
    cur.ritem_hi = ritems;
    cur.words = used;
    if (ng > 0) passes.push_back(cur);
  }
  // counting: units (field, chunk) packed into items of consecutive units of one candidate
  // and pass (at most kCountMaxPages pages and count_pack units), so that the many small
  // block parts of a large batch do not each pay for a whole item.  Packing never crosses a
  // candidate or a pass, so each such run of groups (a segment) packs on its own: first
  // every segment counts its items and units, then a prefix sum places them, then every
  // segment writes its units, items and its fields' bitmap offsets.
  std::vector<int32_t> seg_start;   // first group of each segment
  for (int g = 0; g < ng; ++g)
    if (g == 0 || gpass[(size_t)g] != gpass[(size_t)g - 1] || hgrp[(size_t)g].cfg != hgrp[(size_t)g - 1].cfg)
      seg_start.push_back(g);
  const int64_t nseg = (int64_t)seg_start.size();
  seg_start.push_back(ng);
  std::vector<int64_t> seg_items((size_t)nseg + 1, 0), seg_units((size_t)nseg + 1, 0);
  std::vector<int32_t> citem_unit_, cunits_;
  auto pack = [&](int64_t sg, bool write, int64_t item0, int64_t unit0) {
    bool open = false;
    int64_t n_items = 0, n_units = 0, pages_in = 0, units_in = 0;
    for (int g = seg_start[(size_t)sg]; g < seg_start[(size_t)sg + 1]; ++g) {
      const DGroup &G = hgrp[(size_t)g];
      int64_t o = gbase[(size_t)g];
      for (int k = 0; k < G.f_count; ++k) {
        const int32_t fi = G.f_begin + k;
        DField &f = hfld[(size_t)fi];
        if (write) {
          const bool has_l = f.n_load > 0, has_s = f.n_store > 0;
          for (int b = 0; b < N_BITMAPS; ++b) f.bm[b] = -1;
          if (has_l) {
            f.bm[BM_BL] = o; o += f.words[0];
            f.bm[BM_W] = o; o += f.words[1];
            f.bm[BM_Y] = o; o += f.words[1];
            f.bm[BM_Z] = o; o += f.words[1];
          }
          if (has_s) {
            f.bm[BM_BS] = o; o += f.words[0];
            f.bm[BM_WS] = o; o += f.words[1];
          }
          // the row walk flags the pages it writes, so the counting reads only those
          f.pg = -1;
          if (G.rows) {
            f.pg = o;
            o += page_flag_words(f.words[0], f.words[1]);
          }
          f.item_begin = G.item_begin;
          f.citem_begin = item0 + n_items - (open ? 1 : 0);
        }
        for_count_units(f, G.rows != 0, tune.count_words, [&](int64_t u, int64_t pages) {
          if (!open || pages_in + pages > kCountMaxPages || units_in == count_pack) {
            if (write) citem_unit_[(size_t)(item0 + n_items)] = (int32_t)(unit0 + n_units);
            ++n_items;
            open = true;
            pages_in = units_in = 0;
          }
          if (write) {
            cunits_[(size_t)(2 * (unit0 + n_units))] = fi;
            cunits_[(size_t)(2 * (unit0 + n_units) + 1)] = (int32_t)u;
          }
          ++n_units;
          pages_in += pages;
          ++units_in;
        });
      }
    }
    seg_items[(size_t)sg] = n_items;
    seg_units[(size_t)sg] = n_units;
  };
  parallel_chunks(nseg, 64, [&](int64_t lo, int64_t hi) {
    for (int64_t sg = lo; sg < hi; ++sg) pack(sg, false, 0, 0);
  });
  std::vector<int64_t> seg_item0((size_t)nseg + 1, 0), seg_unit0((size_t)nseg + 1, 0);
  for (int64_t sg = 0; sg < nseg; ++sg) {
    seg_item0[(size_t)sg + 1] = seg_item0[(size_t)sg] + seg_items[(size_t)sg];
    seg_unit0[(size_t)sg + 1] = seg_unit0[(size_t)sg] + seg_units[(size_t)sg];
  }
  const int64_t citems = seg_item0[(size_t)nseg], units = seg_unit0[(size_t)nseg];
  citem_unit_.assign((size_t)citems, 0);
  cunits_.assign((size_t)(2 * units), 0);
  parallel_chunks(nseg, 64, [&](int64_t lo, int64_t hi) {
    for (int64_t sg = lo; sg < hi; ++sg) pack(sg, true, seg_item0[(size_t)sg], seg_unit0[(size_t)sg]);
  });
  // each pass's counting items: those of its segments
  for (size_t q = 0, sg = 0; q < passes.size(); ++q) {
    while (sg < (size_t)nseg && gpass[(size_t)seg_start[sg]] < (int32_t)q) ++sg;
    passes[q].citem_lo = seg_item0[sg];
    size_t e = sg;
    while (e < (size_t)nseg && gpass[(size_t)seg_start[e]] == (int32_t)q) ++e;
    passes[q].citem_hi = seg_item0[e];
    sg = e;
  }
  item_begin_end = items;
  ritem_begin_end = ritems;
  citem_begin_end = citems;
  // owners of the items: [enumeration | row walk], then the counting items' first units
  // (with an end), then the counting units as (field, chunk) pairs
  own.resize((size_t)(items + ritems + citems + 1) + cunits_.size());
  parallel_chunks(ng, 1024, [&](int64_t lo, int64_t hi) {
    for (int64_t g = lo; g < hi; ++g) {
      const DGroup &G = hgrp[(size_t)g];
      const int64_t e1 = g + 1 < ng ? hgrp[(size_t)g + 1].item_begin : items;
      const int64_t r1 = g + 1 < ng ? hgrp[(size_t)g + 1].ritem_begin : ritems;
      std::fill(own.begin() + G.item_begin, own.begin() + e1, (int32_t)g);
      std::fill(own.begin() + items + G.ritem_begin, own.begin() + items + r1, (int32_t)g);
    }
  });
  std::copy(citem_unit_.begin(), citem_unit_.end(), own.begin() + items + ritems);
  own[(size_t)(items + ritems + citems)] = (int32_t)units;
  std::copy(cunits_.begin(), cunits_.end(), own.begin() + items + ritems + citems + 1);
}

int ws_plan::upload_fields(cudaStream_t st) {
  const size_t ob = std::max<size_t>(own.size() * sizeof(int32_t), 256);
  if (ob > d_own_bytes) {
    // a larger layout (autotuning): the previous array is no longer read once `st` has
    // passed its last launch, which precedes this call on the same stream
    if (d_own >= 0) {
      CU(cudaStreamSynchronize(st));
      ctx->arena->release(d_own);
      allocs.erase(std::find(allocs.begin(), allocs.end(), d_own));
    }
    d_own = take(ob);
    d_own_bytes = d_own >= 0 ? ob : 0;
    if (d_own < 0) {
      set_error("arena exhausted while laying out a plan");
      return WS_ENOMEM;
    }
  }
  if (!own.empty()) CU(cudaMemcpyAsync(dev(d_own), own.data(), own.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (!hfld.empty()) CU(cudaMemcpyAsync(dev(d_fld), hfld.data(), hfld.size() * sizeof(DField), cudaMemcpyHostToDevice, st));
  if (!hgrp.empty()) CU(cudaMemcpyAsync(dev(d_grp), hgrp.data(), hgrp.size() * sizeof(DGroup), cudaMemcpyHostToDevice, st));
  if (graph_exec) {
    cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
  }
  return WS_OK;
}

// log2 of the bank width when banks x width is a power of two dividing 1024 (so that
// bitmap-relative addresses have the absolute banks), else -1.
int ws_plan::bank_shift() const {
  const int64_t b = hw.banks, w = hw.bank_bytes;
  auto pow2 = [](int64_t v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!pow2(b) || !pow2(w) || b * w > 1024 || hw.pair_dist_bytes <= 0) return -1;
  int sh = 0;
  while ((1ll << sh) < w) ++sh;
  return sh;
}

int ws_plan::grid_rows(int64_t items) const {
  int occ = 1;
  rows_occupancy(iv_cap, &occ);
  if (tune.ctas_per_sm > 0) occ = std::min(occ, tune.ctas_per_sm);
  occ = std::max(occ, 1);
  int64_t g = (int64_t)ctx->sm_count * occ;
  g = std::min<int64_t>(g, std::max<int64_t>(items, 1));
  return (int)g;
}

int ws_plan::grid_for(int threads, int64_t items, bool counting) const {
  int occ = 1;
  if (counting) count_occupancy(&occ);
  else enum_occupancy(threads, iv_cap, &occ);
  if (tune.ctas_per_sm > 0) occ = std::min(occ, tune.ctas_per_sm);
  occ = std::max(occ, 1);
  int64_t g = (int64_t)ctx->sm_count * occ;
  g = std::min<int64_t>(g, std::max<int64_t>(items, 1));
  return (int)g;
}

// Enqueues one batched step (all passes, model, rank) on `st`; `ev` (may be null)
// receives events [start, per pass (after enumeration, after row walk, after counting),
// after model, after rank].
int ws_plan::enqueue(cudaStream_t st, std::vector<cudaEvent_t> *ev, ws_profile *prof) {
  auto mark = [&](int k) -> int {
    if (ev) CU(cudaEventRecord((*ev)[k], st));
    return WS_OK;
  };
  int rc;
  if ((rc = mark(0)) != WS_OK) return rc;
  CU(cudaMemsetAsync(dev(d_counters), 0, counters_bytes, st));
  int launches = 0;
  for (size_t p = 0; p < passes.size(); ++p) {
    const DPass &P = passes[p];
    EnumArgs ea;
    ea.cfg = (const DCfg *)dev(d_cfg);
    ea.fld = (const DField *)dev(d_fld);
    ea.grp = (const DGroup *)dev(d_grp);
    ea.acc = (const DAcc *)dev(d_acc);
    ea.iv = (const DIv *)dev(d_iv);
    ea.iv_cap = iv_cap;
    ea.scratch = (uint32_t *)dev(d_scratch);
    ea.counters = (int64_t *)((char *)dev(d_counters) + grab_bytes);
    ea.grab = (unsigned long long *)dev(d_counters) + 3 * p;
    ea.rgrab = ea.grab + 1;
    ea.own_enum = (const int32_t *)dev(d_own);
    ea.own_rows = ea.own_enum + item_begin_end;
    ea.ritem_lo = P.ritem_lo;
    ea.ritem_hi = P.ritem_hi;
    ea.item_lo = P.item_lo;
    ea.item_hi = P.item_hi;
    ea.chunk = tune.chunk_warps;
    ea.chunk_rows = chunk_rows();
    ea.banks = hw.banks;
    ea.bank_bytes = hw.bank_bytes;
    ea.pair_dist = hw.pair_dist_bytes;
    ea.bank_shift = bank_shift();
    ea.block_pairs = block_pairs;
    if (P.item_hi > P.item_lo) {
      CU(launch_enum(ea, grid_for(tune.enum_threads, P.item_hi - P.item_lo, false), tune.enum_threads, st));
      ++launches;
    }
    if ((rc = mark(1 + 3 * (int)p)) != WS_OK) return rc;
    if (P.ritem_hi > P.ritem_lo) {
      CU(launch_rows(ea, grid_rows(P.ritem_hi - P.ritem_lo), st));
      ++launches;
    }
    if ((rc = mark(2 + 3 * (int)p)) != WS_OK) return rc;
    CountArgs ca;
    ca.fld = ea.fld;
    ca.item_unit = ea.own_rows + ritem_begin_end;
    ca.units = ca.item_unit + citem_begin_end + 1;
    ca.scratch = ea.scratch;
    ca.counters = ea.counters;
    ca.grab = ea.grab + 2;
    ca.citem_lo = P.citem_lo;
    ca.citem_hi = P.citem_hi;
    ca.chunk_words = tune.count_words;
    if (P.citem_hi > P.citem_lo) {
      CU(launch_count(ca, grid_for(kCountThreads, P.citem_hi - P.citem_lo, true), st));
      ++launches;
    }
    if ((rc = mark(3 + 3 * (int)p)) != WS_OK) return rc;
  }
  ModelArgs ma;
  ma.cfg = (const DCfg *)dev(d_cfg);
  ma.counters = (const int64_t *)((char *)dev(d_counters) + grab_bytes);
  ma.results = (ws_result *)dev(d_results);
  ma.keys = (double *)dev(d_keys);
  ma.n = n_cfg;
  ma.hw = dhw;
  CU(launch_model(ma, st));
  launches += n_cfg > 0;
  if ((rc = mark(1 + 3 * (int)passes.size())) != WS_OK) return rc;
  RankArgs ra;
  ra.keys = (const double *)dev(d_keys);
  ra.seg = (const int32_t *)dev(d_seg);
  ra.order = (int32_t *)dev(d_order);
  ra.rank = (int32_t *)dev(d_rank);
  ra.n = n_cfg;
  ra.n_seg = n_seg;
  CU(launch_rank(ra, st));
  launches += n_cfg > 0 ? 2 : 0;   // counting rank + scatter
  if ((rc = mark(2 + 3 * (int)passes.size())) != WS_OK) return rc;
  if (prof) prof->launches = launches;
  return WS_OK;
}

// Plain form: for every candidate, its own enumeration / counting / model launches,
// then a synchronisation; the ranking runs once at the end.
int ws_plan::run_plain(cudaStream_t st) {
  // the plain form launches each candidate's kernels by themselves: the finest work items
  // spread one candidate over CTAs (the larger items of a big batch pay off only when the
  // whole batch shares the launches)
  plain_layout = true;
  layout();
  int rc = upload_fields(st);
  if (rc == WS_OK) rc = run_plain_launches(st);
  plain_layout = false;
  layout();
  const int rc2 = upload_fields(st);
  // the uploads read the host arrays, which the next layout rewrites
  const cudaError_t e = cudaStreamSynchronize(st);
  if (rc == WS_OK) rc = rc2;
  if (rc == WS_OK && e != cudaSuccess) {
    set_error(cudaGetErrorString(e));
    rc = WS_ECUDA;
  }
  return rc;
}

int ws_plan::run_plain_launches(cudaStream_t st) {
  CU(cudaMemsetAsync(dev(d_counters), 0, counters_bytes, st));
  int64_t *counters = (int64_t *)((char *)dev(d_counters) + grab_bytes);
  unsigned long long *grab = (unsigned long long *)dev(d_counters);
  const int ng = (int)hgrp.size(), nf = (int)hfld.size();
  for (int i = 0; i < n_cfg; ++i) {
    const int g_a = cfg_grp_begin[i], g_b = cfg_grp_begin[i + 1];
    for (size_t p = 0; p < passes.size() && g_a < g_b; ++p) {
      const DPass &P = passes[p];
      const int glo = std::max(g_a, P.grp_lo), ghi = std::min(g_b, P.grp_hi);
      if (glo >= ghi) continue;
      const int64_t it_lo = hgrp[glo].item_begin, it_hi = ghi < ng ? hgrp[ghi].item_begin : item_begin_end;
      const int cf_lo = hgrp[glo].f_begin, cf_hi = hgrp[ghi - 1].f_begin + hgrp[ghi - 1].f_count;
      const int64_t ct_lo = hfld[cf_lo].citem_begin, ct_hi = cf_hi < nf ? hfld[cf_hi].citem_begin : citem_begin_end;
      const int64_t rt_lo = hgrp[glo].ritem_begin, rt_hi = ghi < ng ? hgrp[ghi].ritem_begin : ritem_begin_end;
      CU(cudaMemsetAsync(grab, 0, 3 * sizeof(unsigned long long), st));
      EnumArgs ea;
      ea.cfg = (const DCfg *)dev(d_cfg);
      ea.fld = (const DField *)dev(d_fld);
      ea.grp = (const DGroup *)dev(d_grp);
      ea.acc = (const DAcc *)dev(d_acc);
      ea.iv = (const DIv *)dev(d_iv);
      ea.iv_cap = iv_cap;
      ea.scratch = (uint32_t *)dev(d_scratch);
      ea.counters = counters;
      ea.grab = grab;
      ea.rgrab = grab + 1;
      ea.own_enum = (const int32_t *)dev(d_own);
      ea.own_rows = ea.own_enum + item_begin_end;
      ea.item_lo = it_lo;
      ea.item_hi = it_hi;
      ea.ritem_lo = rt_lo;
      ea.ritem_hi = rt_hi;
      ea.chunk = tune.chunk_warps;
      ea.chunk_rows = chunk_rows();
      ea.banks = hw.banks;
      ea.bank_bytes = hw.bank_bytes;
      ea.pair_dist = hw.pair_dist_bytes;
      ea.bank_shift = bank_shift();
      ea.block_pairs = block_pairs;
      if (it_hi > it_lo) CU(launch_enum(ea, grid_for(tune.enum_threads, it_hi - it_lo, false), tune.enum_threads, st));
      if (rt_hi > rt_lo) CU(launch_rows(ea, grid_rows(rt_hi - rt_lo), st));
      CountArgs ca;
      ca.fld = ea.fld;
      ca.item_unit = ea.own_rows + ritem_begin_end;
      ca.units = ca.item_unit + citem_begin_end + 1;
      ca.scratch = ea.scratch;
      ca.counters = counters;
      ca.grab = grab + 2;
      ca.citem_lo = ct_lo;
      ca.citem_hi = ct_hi;
      ca.chunk_words = tune.count_words;
      if (ct_hi > ct_lo) CU(launch_count(ca, grid_for(kCountThreads, ct_hi - ct_lo, true), st));
    }
    ModelArgs ma;
    ma.cfg = (const DCfg *)dev(d_cfg) + i;
    ma.counters = counters + (int64_t)i * N_COUNTERS;
    ma.results = (ws_result *)dev(d_results) + i;
    ma.keys = (double *)dev(d_keys) + i;
    ma.n = 1;
    ma.hw = dhw;
    CU(launch_model(ma, st));
    CU(cudaStreamSynchronize(st));
  }
  RankArgs ra;
  ra.keys = (const double *)dev(d_keys);
  ra.seg = (const int32_t *)dev(d_seg);
  ra.order = (int32_t *)dev(d_order);
  ra.rank = (int32_t *)dev(d_rank);
  ra.n = n_cfg;
  ra.n_seg = n_seg;
  CU(launch_rank(ra, st));
  return WS_OK;
}

int ws_plan::wait_ready(cudaStream_t st) {
  if (ready) CU(cudaStreamWaitEvent(st, ready, 0));
  return WS_OK;
}

int ws_plan::execute(int mode, cudaStream_t st) {
  if (mode != WS_MODE_PLAIN && mode != WS_MODE_DIRECT && mode != WS_MODE_BATCHED) {
    set_error("unknown mode");
    return WS_EINVAL;
  }
  if (mode != WS_MODE_BATCHED) {
    const int rc = wait_ready(st);
    if (rc != WS_OK) return rc;
    return mode == WS_MODE_PLAIN ? run_plain(st) : enqueue(st, nullptr, nullptr);
  }
  if (!graph_exec) {
    // the capture cannot wait on an event recorded outside it: wait for the uploads here
    if (ready) CU(cudaEventSynchronize(ready));
    cudaGraph_t graph = nullptr;
    CU(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(ctx->capture_stream, nullptr, nullptr);
    cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (rc != WS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    CU(e);
    e = cudaGraphInstantiate(&graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    CU(e);
  }
  CU(cudaGraphLaunch(graph_exec, st));
  return WS_OK;
}

// ---------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------
extern "C" int ws_version(void) { return WS_VERSION; }

extern "C" const char *ws_status_string(int s) {
  switch (s) {
    case WS_OK: return "ok";
    case WS_EINVAL: return "invalid argument or descriptor";
    case WS_ENOMEM: return "does not fit the device-memory budget";
    case WS_EAGAIN: return "not finished yet";
    case WS_ETIMEDOUT: return "bounded wait ran out";
    case WS_EOVERFLOW: return "counting structure overflow";
    case WS_ECUDA: return "CUDA runtime error";
    case WS_ENOTFOUND: return "unknown request";
    case WS_ECANCELED: return "canceled";
    default: return "unknown status";
  }
}

extern "C" const char *ws_last_error(void) { return last_error(); }

extern "C" void ws_hw_a100(ws_hw *h) {
  if (!h) return;
  memset(h, 0, sizeof(*h));
  h->sms = 108;
  h->max_threads_sm = 2048;
  h->max_blocks_sm = 32;
  h->regs_sm = 65536;
  h->clock_hz = 1.41e9;
  h->l1_bytes = 192.0 * 1024;
  h->l2_bytes = 20.0 * 1024 * 1024;
  h->bw_l2 = 5000e9;
  h->bw_dram = 1400e9;
  h->fp_peak = 4.9e12;
  h->banks = 16;
  h->bank_bytes = 8;
  h->pair_dist_bytes = 1024;
  h->capacity_model = 1;
  const double hit[4][3] = {{1.0, 0.01, -3.07}, {1.0, 0.05, -2.0}, {1.0, 0.01, -3.07}, {1.0, 0.01, -3.07}};
  memcpy(h->hit, hit, sizeof(hit));
}

extern "C" int ws_create(ws_ctx **out, int device, void *arena, size_t arena_bytes) {
  if (!out || arena_bytes < (1 << 20)) return WS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return WS_EINVAL;
  CU(cudaSetDevice(device));
  ws_ctx *c = new ws_ctx();
  c->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete c;
    return WS_ECUDA;
  }
  c->sm_count = prop.multiProcessorCount;
  c->l2_bytes = prop.l2CacheSize;
  char *base = (char *)arena;
  if (!base) {
    if (cudaMalloc((void **)&base, arena_bytes) == cudaSuccess) count_resource(RES_DEVICE_ALLOC);
    else {
      delete c;
      set_error("cudaMalloc of the arena failed");
      return WS_ENOMEM;
    }
    c->owns_arena = true;
  }
  c->arena = new Arena(base, arena_bytes);
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->upload_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->lane_stream, cudaStreamNonBlocking) != cudaSuccess) {
    for (cudaStream_t s : {c->stream, c->capture_stream, c->upload_stream, c->lane_stream})
      if (s) cudaStreamDestroy(s);
    if (c->owns_arena) cudaFree(base);
    delete c->arena;
    delete c;
    return WS_ECUDA;
  }
  for (int k = 0; k < 4; ++k) count_resource(RES_STREAM);
  *out = c;
  return WS_OK;
}

extern "C" int ws_resource_counts_get(ws_resource_counts *out) {
  if (!out) return WS_EINVAL;
  out->device_allocs = g_resources[RES_DEVICE_ALLOC].load();
  out->pinned_host_allocs = g_resources[RES_PINNED_ALLOC].load();
  out->streams = g_resources[RES_STREAM].load();
  out->events = g_resources[RES_EVENT].load();
  return WS_OK;
}

extern "C" int ws_destroy(ws_ctx *c) {
  if (!c) return WS_EINVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  cudaStreamSynchronize(c->upload_stream);
  cudaStreamSynchronize(c->lane_stream);
  cudaStreamDestroy(c->stream);
  cudaStreamDestroy(c->capture_stream);
  cudaStreamDestroy(c->upload_stream);
  cudaStreamDestroy(c->lane_stream);
  if (c->owns_arena) cudaFree(c->arena->base);
  delete c->arena;
  delete c;
  return WS_OK;
}

static cudaStream_t pick_stream(ws_ctx *c, void *s) { return s ? (cudaStream_t)s : c->stream; }

// Compiles every candidate; large batches on several host threads, each with its own
// (field, folding) cache.
// Persistent host worker pool for the descriptor compiler: a call runs fn(t) for
// t = 0..width-1 on the workers and the calling thread.  Workers wait on a condition
// variable between calls; a call that finds the pool busy (another host thread is
// creating a plan) runs on its own thread alone.
class HostPool {
 public:
  static HostPool &get() {
    static HostPool pool;
    return pool;
  }
  int width() const { return (int)workers_.size() + 1; }
  void run(int width, const std::function<void(int)> &fn) {
    std::unique_lock<std::mutex> busy(busy_, std::try_to_lock);
    if (!busy.owns_lock() || width <= 1 || workers_.empty()) {
      for (int t = 0; t < width; ++t) fn(t);
      return;
    }
    {
      std::lock_guard<std::mutex> g(mu_);
      job_ = &fn;
      width_ = width;
      next_ = 0;
      active_ = (int)workers_.size();
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> g(mu_);
    done_.wait(g, [&] { return active_ == 0; });
    job_ = nullptr;
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (auto &t : workers_) t.join();
  }

 private:
  HostPool() {
    const unsigned n = std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    for (unsigned i = 1; i < n; ++i) workers_.emplace_back([this] { loop(); });
  }
  void work() {
    for (;;) {
      int t;
      {
        std::lock_guard<std::mutex> g(mu_);
        t = next_ < width_ ? next_++ : -1;
      }
      if (t < 0) return;
      (*job_)(t);
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_.wait(g, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
      }
      work();
      {
        std::lock_guard<std::mutex> g(mu_);
        --active_;
      }
      done_.notify_all();
    }
  }
  std::vector<std::thread> workers_;
  std::mutex mu_, busy_;
  std::condition_variable cv_, done_;
  const std::function<void(int)> *job_ = nullptr;
  int width_ = 0, next_ = 0, active_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

static void parallel_chunks(int64_t n, int64_t chunk, const std::function<void(int64_t, int64_t)> &fn) {
  const int64_t nch = (n + chunk - 1) / chunk;
  if (nch <= 1) {
    if (n > 0) fn(0, n);
    return;
  }
  std::atomic<int64_t> next(0);
  HostPool::get().run((int)std::min<int64_t>(nch, HostPool::get().width()), [&](int) {
    for (int64_t c = next.fetch_add(1); c < nch; c = next.fetch_add(1)) fn(c * chunk, std::min(n, (c + 1) * chunk));
  });
}

static void compile_all(const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld, const ws_access *acc,
                        int n_acc, const ws_hw &hw, int64_t chunk_warps, CompileArena &ca, std::vector<int> &status) {
  ca.comp.assign(n_cfg, nullptr);
  status.assign(n_cfg, WS_OK);
  // chunks of consecutive candidates handed out dynamically; each thread keeps its fold
  // cache across its chunks (neighbouring candidates often share fields)
  // candidates per field (saturated at 2): only fields that several candidates use go
  // through the fold cache
  std::vector<uint8_t> refs((size_t)n_fld, 0);
  {
    std::vector<int32_t> diff((size_t)n_fld + 1, 0);
    for (int i = 0; i < n_cfg; ++i) {
      const ws_config &c = cfgs[i];
      if (c.n_field < 1 || c.field_off < 0 || c.field_off + c.n_field > n_fld) continue;
      diff[(size_t)c.field_off] += 1;
      diff[(size_t)(c.field_off + c.n_field)] -= 1;
    }
    int32_t run = 0;
    for (int f = 0; f < n_fld; ++f) {
      run += diff[(size_t)f];
      refs[(size_t)f] = (uint8_t)std::min(run, 2);
    }
  }
  const int nth = n_cfg >= 64 ? HostPool::get().width() : 1;
  ca.res.clear();
  for (int t = 0; t < nth; ++t)
    ca.res.emplace_back(new std::pmr::monotonic_buffer_resource(kHostBlockMin, &ca.upstream));
  const int chunk = 32;
  std::atomic<int> next(0);
  HostPool::get().run(nth, [&](int t) {
    FieldCache cache;
    std::pmr::memory_resource *r = ca.res[(size_t)t].get();
    for (int c = next.fetch_add(1); c * chunk < n_cfg; c = next.fetch_add(1))
      for (int i = c * chunk; i < std::min(n_cfg, (c + 1) * chunk); ++i) {
        Compiled &cc = *new (r->allocate(sizeof(Compiled), alignof(Compiled))) Compiled(r);
        ca.comp[(size_t)i] = &cc;
        status[i] = compile_config(cfgs[i], fld, n_fld, acc, n_acc, hw, cc, &cache, refs.data());
        if (status[i] != WS_OK) continue;
        const DCfg &d = cc.d;
        const size_t cr = 256;   // the smallest row-walk item
        for (size_t k = 0; k < cc.f.size(); ++k) {
          const int64_t nacc = cc.acc_off[k + 1] - cc.acc_off[k], niv = cc.iv_off[k + 1] - cc.iv_off[k];
          cc.dsc_bytes += sizeof(DField) + sizeof(DGroup) + (size_t)nacc * sizeof(DAcc) + (size_t)niv * sizeof(DIv);
          cc.need_sum += (size_t)cc.need_words[k] * 4;
          cc.need_max = std::max(cc.need_max, (size_t)cc.need_words[k] * 4);
          // at most one enumeration item per chunk of modelled warps and one row-walk item per
          // chunk of row slots, plus the representative block's items
          const DField &f = cc.f[k];
          cc.items_est += 3 + (size_t)d.lev_end[3] / (size_t)chunk_warps + (size_t)d.rows_slot_end[3] / cr +
                          (size_t)d.wpb * (size_t)(f.n_load + f.n_store) / (size_t)kPlainBlockPairs;
          if (cc.fkey[k] == kNoShare) {
            cc.n_acc_own += nacc;
            cc.n_iv_own += niv;
          } else {
            cc.any_shared = true;
          }
        }
      }
  });
}

// Bytes of device memory a plan of these candidates needs with one pass.
int ws::plan_requirements(const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld, const ws_access *acc,
                          int n_acc, const ws_hw *hw, size_t *desc_bytes, size_t *scratch_bytes,
                          size_t *max_field_bytes) {
  size_t dsc = 0, scr = 0, mf = 0;
  FieldCache cache;
  for (int i = 0; i < n_cfg; ++i) {
    Compiled cc;
    if (compile_config(cfgs[i], fld, n_fld, acc, n_acc, *hw, cc, &cache) != WS_OK) continue;
    for (size_t k = 0; k < cc.f.size(); ++k) {
      dsc += sizeof(DField) + sizeof(DGroup) + (size_t)(cc.acc_off[k + 1] - cc.acc_off[k]) * sizeof(DAcc) +
             (size_t)(cc.iv_off[k + 1] - cc.iv_off[k]) * sizeof(DIv);
      scr += (size_t)cc.need_words[k] * 4;
      mf = std::max(mf, (size_t)cc.need_words[k] * 4);
    }
  }
  *max_field_bytes = mf;
  dsc += (size_t)n_cfg * (sizeof(DCfg) + N_COUNTERS * 8 + sizeof(ws_result) + 8 + 4 + 4) + 64 * 1024;
  *desc_bytes = dsc;
  *scratch_bytes = scr;
  return WS_OK;
}

// Host half of plan creation: compiles the candidates, deduplicates their access lists,
// builds field groups and cuts passes.  avail_fn(descriptor bytes, bitmap bytes of all
// fields) gives the scratch capacity.  Needs no device.
struct HostDesc {
  PinVec<DCfg> hcfg;
  PinVec<DAcc> hacc;
  PinVec<DIv> hiv;
  size_t scratch = 0, desc_bytes = 0;
};

// Field groups of candidate i (fields already in p->hfld): consecutive fields bounded by
// the shared-memory staging (fields, folded accesses) and by what one pass of scratch
// holds; appended to `go` with the per-group walk decisions.
struct GroupOut {
  std::vector<DGroup> g;
  std::vector<char> iv_ok, rows_ok;
  std::vector<int64_t> slots, winstr;
  std::vector<WarpClasses> cls;
  int32_t iv_cap = 0;
};

static void build_groups(const Plan *p, int i, const Compiled &cc, const ws_hw &hw, GroupOut &go) {
  const int a = p->cfg_cf_begin[i], b = p->cfg_cf_begin[i + 1];
  int k = a;
  bool wave_seen = false;
  while (k < b) {
    DGroup G;
    memset(&G, 0, sizeof(G));
    G.cfg = i;
    G.f_begin = k;
    G.first_of_cfg = k == a;
    G.mw_block = p->hfld[k].mw_block;
    G.levels = p->hfld[k].level_mask;
    G.first_wave = (G.levels & 2) && !wave_seen;
    wave_seen = wave_seen || (G.levels & 2);
    int64_t need = 0;
    while (k < b) {
      const DField &f = p->hfld[k];
      const int na = f.n_load + f.n_store;
      if (G.f_count > 0 && (G.f_count >= kMaxGroupFields || G.acc_count + na > kMaxFoldedAccesses ||
                            need + p->need_words[k] > p->scratch_words || f.level_mask != G.levels))
        break;
      G.f_count += 1;
      G.acc_count += na;
      G.n_loads += f.n_load;
      G.n_stores += f.n_store;
      G.mw_end = std::max(G.mw_end, f.mw_end);
      need += p->need_words[k];
      ++k;
    }
    // uniform layout: a field's relative address is the shared thread address plus a
    // per-field constant, so all the group's accesses can be walked as one list
    G.uniform = 1;
    G.iv = 1;
    for (int q = G.f_begin; q < G.f_begin + G.f_count; ++q) {
      const DField &f = p->hfld[q], &f0 = p->hfld[G.f_begin];
      if (f.wide || f.esize != f0.esize || f.stride[0] != f0.stride[0] || f.stride[1] != f0.stride[1] ||
          f.stride[2] != f0.stride[2])
        G.uniform = 0;
      if (!f.iv) G.iv = 0;
      G.n_iv += f.n_iv;
    }
    // interval walk: uniform groups whose row segments have contiguous sectors
    G.iv = G.iv && G.uniform;
    if (G.iv) go.iv_cap = std::max(go.iv_cap, G.n_iv);
    // row walk: interval groups whose store counts add up per row segment
    bool rows = G.iv && cc.rows_geom_ok && (G.levels & 2);
    int64_t instr_w = 0, instr_yz = 0;
    for (int q = G.f_begin; q < G.f_begin + G.f_count; ++q) {
      rows = rows && p->hfld[q].rows_ok;
      instr_w += p->hfld[q].n_load + p->hfld[q].n_store;
      instr_yz += p->hfld[q].n_load;
    }
    const DCfg &dc = cc.d;
    go.iv_ok.push_back((char)G.iv);
    go.rows_ok.push_back((char)rows);
    // with the block level when the group also serves the representative block
    go.slots.push_back(dc.rows_slot_end[(G.levels & 1) ? 3 : 2]);
    {
      const DField &f0 = p->hfld[G.f_begin], &c0 = p->hfld[a];
      WarpClasses wc;
      if (rows && (G.levels & 1)) {
        if (f0.esize == c0.esize && f0.stride[0] == c0.stride[0] && f0.stride[1] == c0.stride[1] &&
            f0.stride[2] == c0.stride[2])
          wc = cc.cls;
        else
          block_warp_classes(dc, f0.esize, f0.stride, hw, wc);
      }
      go.cls.push_back(wc);
    }
    go.winstr.push_back((cc.lvl_blocks[0] * instr_w + (cc.lvl_blocks[1] + cc.lvl_blocks[2]) * instr_yz) * dc.wpb);
    go.g.push_back(G);
  }
}

static void build_host(Plan *p, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                       const ws_access *acc, int n_acc, const ws_hw *hw,
                       const std::function<size_t(size_t, size_t)> &avail_fn, HostDesc &h) {
  PinVec<DCfg> &hcfg = h.hcfg;
  PinVec<DAcc> &hacc = h.hacc;
  PinVec<DIv> &hiv = h.hiv;
  hcfg.resize(n_cfg);
  p->cfg_cf_begin.assign(n_cfg + 1, 0);
  CompileArena ca;
  std::vector<int> status;
  compile_all(cfgs, n_cfg, fld, n_fld, acc, n_acc, *hw, std::max(1, p->tune.chunk_warps), ca, status);
  const std::vector<Compiled *> &comp = ca.comp;
  // scratch capacity: what the arena can give after the descriptors (a field, its access
  // and interval lists, at most one field group each)
  size_t dsc = 64 * 1024, total_need = 0, max_field = 0;
  for (int i = 0; i < n_cfg; ++i) {
    if (status[i] != WS_OK) continue;
    dsc += comp[i]->dsc_bytes;
    total_need += comp[i]->need_sum;
    max_field = std::max(max_field, comp[i]->need_max);
  }
  dsc += (size_t)n_cfg * (sizeof(DCfg) + N_COUNTERS * 8 + sizeof(ws_result) + 8 + 4 + 4 + 4);
  {
    // owner tables of the work items (4 bytes per item): the candidates' enumeration and
    // row-walk items (bounded as they compiled), plus one counting item per chunk of bitmap
    // words per field
    size_t items = total_need / ((size_t)std::max(4, p->tune.count_words) * 4) + 1;
    for (int i = 0; i < n_cfg; ++i)
      if (status[i] == WS_OK) items += comp[i]->items_est;
    // an item or counting unit takes at most three table entries (a counting unit: its
    // (field, chunk) pair and its item's first unit)
    dsc += 4 * 3 * items;
  }
  const size_t avail = avail_fn(dsc, total_need);
  size_t scratch = std::min(total_need, avail);
  scratch = std::max<size_t>(scratch, 16);
  h.scratch = scratch;
  h.desc_bytes = dsc;
  for (int i = 0; i < n_cfg; ++i)
    if (status[i] == WS_OK && comp[i]->need_max > scratch) status[i] = WS_ENOMEM;
  // descriptors: fields in candidate order; candidates that share a field and a folding
  // share its access and interval lists on the device (the first such field owns them)
  std::vector<int64_t> cf_off(n_cfg + 1, 0);
  for (int i = 0; i < n_cfg; ++i) cf_off[i + 1] = cf_off[i] + (status[i] == WS_OK ? (int64_t)comp[i]->f.size() : 0);
  const int64_t nf = cf_off[n_cfg];
  // access / interval list positions: a candidate none of whose fields may be shared takes
  // its lists in one block (the fields' positions inside it are laid out in parallel below);
  // the others go field by field, and a field whose lists an earlier field holds shares them
  std::vector<int32_t> acc_b((size_t)nf), iv_b((size_t)nf);
  std::vector<char> owner((size_t)nf, 0);
  std::vector<int64_t> own_acc_b((size_t)n_cfg, -1), own_iv_b((size_t)n_cfg, -1);
  int64_t na = 0, ni = 0;
  {
    std::unordered_map<uint64_t, int64_t> first;   // shared fold key -> owning field
    for (int i = 0; i < n_cfg; ++i) {
      if (cf_off[i + 1] > cf_off[i] && !comp[i]->any_shared) {
        own_acc_b[(size_t)i] = na;
        own_iv_b[(size_t)i] = ni;
        na += comp[i]->n_acc_own;
        ni += comp[i]->n_iv_own;
        continue;
      }
      for (int64_t j = cf_off[i]; j < cf_off[i + 1]; ++j) {
        const size_t k = (size_t)(j - cf_off[i]);
        const uint64_t key = comp[i]->fkey[k];
        if (key != kNoShare) {
          auto it = first.find(key);
          if (it != first.end()) {
            acc_b[(size_t)j] = acc_b[(size_t)it->second];
            iv_b[(size_t)j] = iv_b[(size_t)it->second];
            continue;
          }
          first.emplace(key, j);
        }
        owner[(size_t)j] = 1;
        acc_b[(size_t)j] = (int32_t)na;
        iv_b[(size_t)j] = (int32_t)ni;
        na += comp[i]->acc_off[k + 1] - comp[i]->acc_off[k];
        ni += comp[i]->iv_off[k + 1] - comp[i]->iv_off[k];
      }
    }
  }
  hacc.resize((size_t)na);
  hiv.resize((size_t)ni);
  p->hfld.resize((size_t)nf);
  p->need_words.resize((size_t)nf);
  for (int i = 0; i <= n_cfg; ++i) p->cfg_cf_begin[i] = (int32_t)cf_off[i];
  p->scratch_words = (int64_t)(scratch / 4);
  // per candidate, in parallel over dynamic chunks: its DCfg, DFields and owned lists,
  // then its field groups (into the chunk's output)
  const int chunk = 64;
  const int n_chunks = (n_cfg + chunk - 1) / chunk;
  std::vector<GroupOut> gout((size_t)n_chunks);
  std::vector<int32_t> grp_count((size_t)n_cfg, 0);
  std::atomic<int> next(0);
  auto fill = [&](int) {
    for (int ch = next.fetch_add(1); ch < n_chunks; ch = next.fetch_add(1)) {
      GroupOut &go = gout[(size_t)ch];
      for (int i = ch * chunk; i < std::min(n_cfg, (ch + 1) * chunk); ++i) {
        DCfg &d = hcfg[i];
        if (status[i] == WS_OK) d = comp[i]->d;
        else memset(&d, 0, sizeof(d));
        d.status = status[i];
        d.field_begin = (int32_t)cf_off[i];
        if (status[i] != WS_OK) {
          d.n_field = 0;
          continue;
        }
        Compiled &cc = *comp[i];
        if (own_acc_b[(size_t)i] >= 0) {
          // the candidate's lists in one block: field k's after those of fields 0 .. k-1
          for (size_t k = 0; k < cc.f.size(); ++k) {
            const size_t j = (size_t)cf_off[i] + k;
            owner[j] = 1;
            acc_b[j] = (int32_t)(own_acc_b[(size_t)i] + cc.acc_off[k]);
            iv_b[j] = (int32_t)(own_iv_b[(size_t)i] + cc.iv_off[k]);
          }
        }
        for (size_t k = 0; k < cc.f.size(); ++k) {
          const size_t j = (size_t)cf_off[i] + k;
          DField f = cc.f[k];
          f.cfg = i;
          f.acc_begin = acc_b[j];
          f.iv_begin = iv_b[j];
          p->hfld[j] = f;
          p->need_words[j] = cc.need_words[k];
          if (owner[j]) {
            std::copy(cc.acc.begin() + cc.acc_off[k], cc.acc.begin() + cc.acc_off[k + 1], hacc.begin() + acc_b[j]);
            std::copy(cc.iv.begin() + cc.iv_off[k], cc.iv.begin() + cc.iv_off[k + 1], hiv.begin() + iv_b[j]);
          }
        }
        const size_t before = go.g.size();
        build_groups(p, i, cc, *hw, go);
        grp_count[(size_t)i] = (int32_t)(go.g.size() - before);
      }
    }
  };
  {
    const int nth = n_cfg >= 256 ? HostPool::get().width() : 1;
    HostPool::get().run(nth, fill);
  }
  p->cfg_cf_begin[n_cfg] = (int32_t)p->hfld.size();
  // concatenate the chunks' groups in candidate order
  p->cfg_grp_begin.assign(n_cfg + 1, 0);
  for (int i = 0; i < n_cfg; ++i) p->cfg_grp_begin[i + 1] = p->cfg_grp_begin[i] + grp_count[(size_t)i];
  const size_t ng = (size_t)p->cfg_grp_begin[n_cfg];
  p->hgrp.clear();
  p->hgrp.reserve(ng);
  p->grp_iv_ok.reserve(ng);
  p->grp_rows_ok.reserve(ng);
  p->grp_slots.reserve(ng);
  p->grp_classes.reserve(ng);
  p->grp_winstr_rows.reserve(ng);
  for (GroupOut &go : gout) {
    p->hgrp.insert(p->hgrp.end(), go.g.begin(), go.g.end());
    p->grp_iv_ok.insert(p->grp_iv_ok.end(), go.iv_ok.begin(), go.iv_ok.end());
    p->grp_rows_ok.insert(p->grp_rows_ok.end(), go.rows_ok.begin(), go.rows_ok.end());
    p->grp_slots.insert(p->grp_slots.end(), go.slots.begin(), go.slots.end());
    p->grp_classes.insert(p->grp_classes.end(), go.cls.begin(), go.cls.end());
    p->grp_winstr_rows.insert(p->grp_winstr_rows.end(), go.winstr.begin(), go.winstr.end());
    p->iv_cap = std::max(p->iv_cap, go.iv_cap);
  }
  p->layout();
}

int ws::plan_create_impl(ws_ctx *ctx, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                         const ws_access *acc, int n_acc, const ws_hw *hw, const int32_t *seg_begin, int n_seg,
                         const ws_tuning *tuning, size_t scratch_cap, ws_plan **out, cudaStream_t upload,
                         int64_t ext_scratch, size_t ext_scratch_bytes) {
  if (!ctx || !out || !hw || n_cfg < 0 || n_fld < 0 || n_acc < 0) return WS_EINVAL;
  if (n_cfg > 0 && (!cfgs || (n_fld > 0 && !fld) || (n_acc > 0 && !acc))) return WS_EINVAL;
  if (!hw_valid(*hw)) return WS_EINVAL;
  *out = nullptr;
  CU(cudaSetDevice(ctx->device));
  std::vector<int32_t> seg;
  if (seg_begin && n_seg > 0) {
    if (seg_begin[0] != 0 || seg_begin[n_seg] != n_cfg) return WS_EINVAL;
    for (int k = 0; k < n_seg; ++k)
      if (seg_begin[k + 1] < seg_begin[k]) return WS_EINVAL;
    seg.assign(seg_begin, seg_begin + n_seg + 1);
  } else {
    seg = {0, n_cfg};
    n_seg = 1;
  }
  Plan *p = new Plan();
  p->ctx = ctx;
  p->n_cfg = n_cfg;
  p->n_seg = n_seg;
  p->hw = *hw;
  p->dhw = to_dhw(*hw);
  memset(&p->tune, 0, sizeof(p->tune));
  if (tuning) p->tune = *tuning;
  else ws::tuning_cache_lookup(ctx, n_cfg, &p->tune);
  default_tuning(p->tune);

  HostDesc h;
  const auto t_begin = std::chrono::steady_clock::now();
  if (ext_scratch == -1) ctx_reclaim(ctx);
  bool ctx_scratch = false;   // the plan runs in the context's kept scratch
  build_host(p, cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, [&](size_t dsc, size_t need) {
    if (ext_scratch == kCtxScratch) {
      // grow the kept scratch to this plan's bitmaps when the arena has the room
      if (ctx->oneshot_bytes < need) {
        if (ctx->oneshot_off >= 0) ctx->arena->release(ctx->oneshot_off);
        ctx->oneshot_off = -1;
        ctx->oneshot_bytes = 0;
        size_t room = ctx->arena->largest_free();
        room = room > dsc + (8 << 20) ? room - dsc - (8 << 20) : 0;
        const size_t want = std::min((need + 255) & ~(size_t)255, room & ~(size_t)255);   // whole bitmaps: one pass
        const int64_t o = want >= 256 ? ctx->arena->alloc(want) : -1;
        if (o >= 0) {
          ctx->oneshot_off = o;
          ctx->oneshot_bytes = want;
          ctx->oneshot_dirty = true;
        }
      }
      if (ctx->oneshot_off >= 0) {
        ctx_scratch = true;
        return ctx->oneshot_bytes;
      }
    }
    size_t avail = ctx->arena->largest_free();
    avail = avail > dsc + (8 << 20) ? avail - dsc - (8 << 20) : 0;
    if (ext_scratch >= 0) avail = ext_scratch_bytes;
    if (scratch_cap) avail = std::min(avail, scratch_cap);
    return avail;
  }, h);
  const auto t_host = std::chrono::steady_clock::now();
  PinVec<DCfg> &hcfg = h.hcfg;
  PinVec<DAcc> &hacc = h.hacc;
  PinVec<DIv> &hiv = h.hiv;
  const size_t scratch = h.scratch;
  {
    // raise the enumeration kernel's shared-memory limit now, outside any capture
    int occ = 0;
    cudaError_t e0 = enum_occupancy(p->tune.enum_threads, p->iv_cap, &occ);
    if (e0 == cudaSuccess) e0 = count_occupancy(&occ);   // the counting kernel's ring limit likewise
    if (e0 != cudaSuccess) {
      set_error(std::string("enumeration kernel setup: ") + cudaGetErrorString(e0));
      delete p;
      return WS_ECUDA;
    }
  }

  // device buffers
  // three work-stealing counters per pass (enumeration, row walk, counting); any tuning
  // makes at most one pass per
  // (candidate, field), so size for that (retuning may change the pass count)
  p->grab_bytes = 24 * (p->hfld.size() + 1);
  p->counters_bytes = p->grab_bytes + (size_t)n_cfg * N_COUNTERS * 8;
  p->d_cfg = p->take(std::max<size_t>(hcfg.size() * sizeof(DCfg), 256));
  p->d_grp = p->take(std::max<size_t>(p->hgrp.size() * sizeof(DGroup), 256));
  p->d_fld = p->take(std::max<size_t>(p->hfld.size() * sizeof(DField), 256));
  p->d_acc = p->take(std::max<size_t>(hacc.size() * sizeof(DAcc), 256));
  p->d_iv = p->take(std::max<size_t>(hiv.size() * sizeof(DIv), 256));
  p->d_seg = p->take((seg.size()) * sizeof(int32_t));
  p->d_counters = p->take(p->counters_bytes);
  p->d_results = p->take(std::max<size_t>((size_t)n_cfg * sizeof(ws_result), 256));
  p->d_keys = p->take(std::max<size_t>((size_t)n_cfg * sizeof(double), 256));
  p->d_order = p->take(std::max<size_t>((size_t)n_cfg * sizeof(int32_t), 256));
  p->d_rank = p->take(std::max<size_t>((size_t)n_cfg * sizeof(int32_t), 256));
  if (ext_scratch >= 0 || ctx_scratch) {
    p->d_scratch = ctx_scratch ? ctx->oneshot_off : ext_scratch;
    p->ext_scratch = true;
  } else {
    p->d_scratch = p->take(scratch);
  }
  for (int64_t o : {p->d_cfg, p->d_grp, p->d_fld, p->d_acc, p->d_iv, p->d_seg, p->d_counters, p->d_results, p->d_keys, p->d_order, p->d_rank,
                    p->d_scratch}) {
    if (o < 0) {
      p->release_all();
      delete p;
      set_error("arena exhausted while creating a plan");
      return WS_ENOMEM;
    }
  }
  cudaStream_t st = upload ? upload : ctx->stream;
  int rc = WS_OK;
  auto fail = [&](cudaError_t e) {
    set_error(std::string("plan upload: ") + cudaGetErrorString(e));
    // copies already issued may still read the plan's device memory: let them finish
    cudaStreamSynchronize(st);
    if (p->ready) cudaEventDestroy(p->ready);
    p->release_all();
    delete p;
    return WS_ECUDA;
  };
  cudaError_t e;
  if (n_cfg && (e = cudaMemcpyAsync(p->dev(p->d_cfg), hcfg.data(), hcfg.size() * sizeof(DCfg), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if (!hacc.empty() && (e = cudaMemcpyAsync(p->dev(p->d_acc), hacc.data(), hacc.size() * sizeof(DAcc), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if (!hiv.empty() && (e = cudaMemcpyAsync(p->dev(p->d_iv), hiv.data(), hiv.size() * sizeof(DIv), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(p->dev(p->d_seg), seg.data(), seg.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((!p->ext_scratch || (ctx_scratch && ctx->oneshot_dirty)) &&
      (e = cudaMemsetAsync(p->dev(p->d_scratch), 0, ctx_scratch ? ctx->oneshot_bytes : scratch, st)) != cudaSuccess)
    return fail(e);
  if (ctx_scratch) ctx->oneshot_dirty = false;
  if ((rc = p->upload_fields(st)) != WS_OK) {
    cudaStreamSynchronize(st);   // the copies issued above must finish before the memory goes back
    p->release_all();
    delete p;
    return rc;
  }
  // launches wait for this event (pageable copies are staged when cudaMemcpyAsync returns,
  // so the host arrays may go now)
  if (!ctx->no_events) {
    if ((e = cudaEventCreateWithFlags(&p->ready, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    count_resource(RES_EVENT);
    if ((e = cudaEventRecord(p->ready, st)) != cudaSuccess) return fail(e);
  }
  p->scratch_bytes = scratch;
  {
    const auto t_end = std::chrono::steady_clock::now();
    p->ms_create_host = std::chrono::duration<float, std::milli>(t_host - t_begin).count();
    p->ms_create_device = std::chrono::duration<float, std::milli>(t_end - t_host).count();
  }
  p->upload_bytes = (int64_t)(hcfg.size() * sizeof(DCfg) + p->hfld.size() * sizeof(DField) +
                              p->hgrp.size() * sizeof(DGroup) + hacc.size() * sizeof(DAcc) +
                              hiv.size() * sizeof(DIv) + seg.size() * sizeof(int32_t) +
                              p->own.size() * sizeof(int32_t));
  // the copies from these page-locked arrays may still be running: the plan keeps them
  p->up_cfg = std::move(hcfg);
  p->up_acc = std::move(hacc);
  p->up_iv = std::move(hiv);
  *out = p;
  return WS_OK;
}

extern "C" int ws_plan_create(ws_ctx *ctx, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                              const ws_access *acc, int n_acc, const ws_hw *hw, const int32_t *seg_begin, int n_seg,
                              const ws_tuning *tuning, ws_plan **plan) {
  return plan_create_impl(ctx, cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, seg_begin, n_seg, tuning, 0, plan, nullptr,
                          -1, 0);
}

extern "C" int ws_plan_execute(ws_plan *p, int mode, void *stream) {
  if (!p) return WS_EINVAL;
  CU(cudaSetDevice(p->ctx->device));
  return p->execute(mode, pick_stream(p->ctx, stream));
}

extern "C" int ws_plan_results(ws_plan *p, ws_result *out, int32_t *order, void *stream) {
  if (!p) return WS_EINVAL;
  CU(cudaSetDevice(p->ctx->device));
  cudaStream_t st = pick_stream(p->ctx, stream);
  if (out && p->n_cfg) CU(cudaMemcpyAsync(out, p->dev(p->d_results), (size_t)p->n_cfg * sizeof(ws_result), cudaMemcpyDeviceToHost, st));
  if (order && p->n_cfg) CU(cudaMemcpyAsync(order, p->dev(p->d_order), (size_t)p->n_cfg * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return WS_OK;
}

extern "C" int ws_plan_device_results(ws_plan *p, ws_result **res, int32_t **order) {
  if (!p) return WS_EINVAL;
  if (res) *res = (ws_result *)p->dev(p->d_results);
  if (order) *order = (int32_t *)p->dev(p->d_order);
  return WS_OK;
}

extern "C" int ws_plan_profile(ws_plan *p, void *stream, ws_profile *out) {
  if (!p || !out) return WS_EINVAL;
  CU(cudaSetDevice(p->ctx->device));
  cudaStream_t st = pick_stream(p->ctx, stream);
  memset(out, 0, sizeof(*out));
  const int nev = 3 + 3 * (int)p->passes.size();
  std::vector<cudaEvent_t> ev(nev);
  for (auto &e : ev) {
    CU(cudaEventCreate(&e));
    count_resource(RES_EVENT);
  }
  int rc = p->wait_ready(st);
  if (rc == WS_OK) rc = p->enqueue(st, &ev, out);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc == WS_OK && e == cudaSuccess) {
    float ms = 0;
    const int np = (int)p->passes.size();
    for (int k = 0; k < np; ++k) {
      cudaEventElapsedTime(&ms, ev[3 * k], ev[1 + 3 * k]);
      out->ms_enum += ms;
      cudaEventElapsedTime(&ms, ev[1 + 3 * k], ev[2 + 3 * k]);
      out->ms_rows += ms;
      cudaEventElapsedTime(&ms, ev[2 + 3 * k], ev[3 + 3 * k]);
      out->ms_count += ms;
    }
    cudaEventElapsedTime(&ms, ev[3 * np], ev[1 + 3 * np]);
    out->ms_model = ms;
    cudaEventElapsedTime(&ms, ev[1 + 3 * np], ev[2 + 3 * np]);
    out->ms_rank = ms;
    cudaEventElapsedTime(&ms, ev[0], ev[2 + 3 * np]);
    out->ms_total = ms;
    out->enum_items = p->item_begin_end + p->ritem_begin_end;
    out->count_items = p->citem_begin_end;
    out->passes = (int64_t)p->passes.size();
    out->upload_bytes = p->upload_bytes;
    out->ms_create_host = p->ms_create_host;
    out->ms_create_device = p->ms_create_device;
    std::vector<int64_t> cnt((size_t)p->n_cfg * N_COUNTERS);
    if (p->n_cfg)
      e = cudaMemcpy(cnt.data(), (char *)p->dev(p->d_counters) + p->grab_bytes, cnt.size() * 8, cudaMemcpyDeviceToHost);
    for (int i = 0; i < p->n_cfg; ++i) {
      out->addresses += cnt[(size_t)i * N_COUNTERS + C_ADDR];
      out->warp_instr += cnt[(size_t)i * N_COUNTERS + C_WINSTR];
      out->row_reds += cnt[(size_t)i * N_COUNTERS + C_RED];
      out->block_addresses += cnt[(size_t)i * N_COUNTERS + C_ADDR0];
      out->count_bytes += cnt[(size_t)i * N_COUNTERS + C_CBYTES];
    }
    // the row walk visits no modelled warps at levels 1-3: their (warp, instruction)
    // pairs are known from the block counts
    for (size_t g = 0; g < p->hgrp.size(); ++g)
      if (p->hgrp[g].rows) out->warp_instr += p->grp_winstr_rows[g];
    int64_t bm = 0;
    for (size_t k = 0; k < p->hfld.size(); ++k) bm += p->need_words[k] * 4;
    out->bitmap_bytes = bm;
  }
  for (auto &x : ev) cudaEventDestroy(x);
  if (rc != WS_OK) return rc;
  CU(e);
  return WS_OK;
}

extern "C" int ws_plan_destroy(ws_plan *p) {
  if (!p) return WS_EINVAL;
  cudaSetDevice(p->ctx->device);
  cudaStreamSynchronize(p->ctx->stream);
  if (p->ready) {
    cudaEventSynchronize(p->ready);
    cudaEventDestroy(p->ready);
  }
  p->release_all();
  delete p;
  return WS_OK;
}

extern "C" int ws_autotune(ws_plan *p, void *stream, ws_tuning *best) {
  if (!p) return WS_EINVAL;
  CU(cudaSetDevice(p->ctx->device));
  cudaStream_t st = pick_stream(p->ctx, stream);
  const ws_tuning orig = p->tune;
  ws_tuning win = orig;
  float win_ms = -1.f;
  const int chunks[] = {64, 256, 1024, 4096};
  const int threads[] = {128, 256, 512};
  const int pass_mbs[] = {96, 1024, 8192, -1};
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  count_resource(RES_EVENT);
  count_resource(RES_EVENT);
  int rc = p->wait_ready(st);
  if (rc != WS_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  }
  for (int ch : chunks) {
    for (int th : threads) {
      for (int pm : pass_mbs) {
      p->tune = orig;
      p->tune.chunk_warps = ch;
      p->tune.enum_threads = th;
      p->tune.pass_mb = pm;
      p->layout();
      if ((rc = p->upload_fields(st)) != WS_OK) break;
      if ((rc = p->enqueue(st, nullptr, nullptr)) != WS_OK) break;  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && rc == WS_OK; ++r) rc = p->enqueue(st, nullptr, nullptr);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = WS_ECUDA;
      if (rc != WS_OK) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (win_ms < 0 || ms < win_ms) {
        win_ms = ms;
        win = p->tune;
      }
      }
      if (rc != WS_OK) break;
    }
    if (rc != WS_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->tune = rc == WS_OK ? win : orig;
  p->layout();
  int rc2 = p->upload_fields(st);
  cudaStreamSynchronize(st);
  if (rc != WS_OK) return rc;
  if (rc2 != WS_OK) return rc2;
  if (best) *best = p->tune;
  ws::tuning_cache_store(p->ctx, p->n_cfg, p->tune);
  return WS_OK;
}

// Pipelined one-shot estimate: the batch is cut into up to kPipeParts contiguous parts,
// each its own plan; part k + 1 compiles on the host and uploads on the context's upload
// stream while part k runs on the caller's stream.  Results are per candidate, so the parts
// give the same results as one plan; the ranking runs once over all results.  Returns
// WS_ENOMEM (the caller then runs one plan) when the parts do not fit the arena together or
// the parts' scratch is too small for a field that the whole arena could hold.  Parts of
// fewer than kPipeMin candidates lose more on the device (launches, tails) than the overlap
// gains (measured on GB300: 755 candidates in 3 parts 2.0 ms against 1.8 ms in one plan;
// 20,000 mixed candidates 99 ms against 107 ms).
// (six parts of the 20,000-candidate mixed set: 35.2 ms per call against 36.5 ms with three)
static constexpr int kPipeMin = 2048, kPipeParts = 6;

static int estimate_pipelined(ws_ctx *ctx, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                              const ws_access *acc, int n_acc, const ws_hw *hw, ws_result *out, int32_t *order_out,
                              cudaStream_t st) {
  // The parts run in two lanes (below), each lane's parts one after another, and the
  // counting kernel leaves the bitmaps zeroed, so a lane's parts share one scratch: half of
  // the context's kept one, allocated (three fifths of the free arena) and zeroed by the
  // first estimate that needs it, reused as it is by the next ones.  When another estimate
  // holds it, each part takes its own share.
  std::unique_lock<std::mutex> kept(ctx->oneshot_mu, std::try_to_lock);
  if (!kept.owns_lock()) ctx_reclaim(ctx);
  const int parts = std::min(kPipeParts, n_cfg / kPipeMin);
  const size_t rb = (size_t)n_cfg * sizeof(ws_result);
  Arena &ar = *ctx->arena;
  const int64_t o_res = ar.alloc(rb), o_keys = ar.alloc((size_t)n_cfg * 8), o_ord = ar.alloc((size_t)n_cfg * 4),
                o_rnk = ar.alloc((size_t)n_cfg * 4), o_seg = ar.alloc(256);
  std::vector<ws_plan *> plans;
  std::vector<cudaEvent_t> evs;
  int rc = WS_OK;
  cudaError_t e = cudaSuccess;
  if (o_res < 0 || o_keys < 0 || o_ord < 0 || o_rnk < 0 || o_seg < 0) rc = WS_ENOMEM;
  char *b = ar.base;
  int64_t shared = -1;
  size_t shared_bytes = 0;
  if (rc == WS_OK && kept.owns_lock()) {
    if (ctx->oneshot_off < 0 || ctx->oneshot_bytes < ((size_t)1 << 30)) {
      if (ctx->oneshot_off >= 0) ar.release(ctx->oneshot_off);
      ctx->oneshot_off = -1;
      ctx->oneshot_bytes = 0;
      const size_t want = (ar.largest_free() / 5 * 3) & ~(size_t)255;
      const int64_t o = want >= ((size_t)64 << 20) ? ar.alloc(want) : -1;
      if (o >= 0) {
        ctx->oneshot_off = o;
        ctx->oneshot_bytes = want;
        ctx->oneshot_dirty = true;
      }
    }
    if (ctx->oneshot_off >= 0) {
      shared = ctx->oneshot_off;
      shared_bytes = ctx->oneshot_bytes;
      if (ctx->oneshot_dirty) {
        e = cudaMemsetAsync(b + shared, 0, shared_bytes, ctx->upload_stream);
        if (e == cudaSuccess) ctx->oneshot_dirty = false;
      }
    }
  }
  // without the shared scratch the parts share what the arena holds
  const size_t cap = rc == WS_OK && shared < 0 ? std::max<size_t>(ar.largest_free() / (size_t)(parts + 1), 16) : 0;
  // Two lanes: even parts run on `st`, odd ones on the context's lane stream, so that one
  // part's kernels fill the SMs its neighbour's tails leave idle.  With the shared scratch
  // each lane takes its own half (a lane's parts run one after another, and the counting
  // leaves their half zeroed); without it every part has its own scratch anyway.
  const size_t half = (shared_bytes / 2) & ~(size_t)255;
  const int lanes = ctx->lane_stream && parts >= 2 && (shared < 0 || half >= ((size_t)512 << 20)) ? 2 : 1;
  auto new_event = [&](cudaEvent_t *ev) {
    cudaError_t r = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (r == cudaSuccess) {
      count_resource(RES_EVENT);
      evs.push_back(*ev);
    }
    return r;
  };
  if (rc == WS_OK && e == cudaSuccess) {
    const int32_t seg[2] = {0, n_cfg};
    e = cudaMemcpyAsync(b + o_seg, seg, sizeof(seg), cudaMemcpyHostToDevice, ctx->upload_stream);
  }
  if (rc == WS_OK && e == cudaSuccess && lanes == 2) {
    // the lane stream starts after the work the caller queued on `st`
    cudaEvent_t fork;
    e = new_event(&fork);
    if (e == cudaSuccess) e = cudaEventRecord(fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->lane_stream, fork, 0);
  }
  for (int k = 0; k < parts && rc == WS_OK && e == cudaSuccess; ++k) {
    const int lo = (int)((int64_t)n_cfg * k / parts), hi = (int)((int64_t)n_cfg * (k + 1) / parts);
    const cudaStream_t sk = lanes == 2 && (k & 1) ? ctx->lane_stream : st;
    const int64_t sh = shared < 0 ? shared : lanes == 2 ? shared + (int64_t)((k & 1) * half) : shared;
    const size_t sh_bytes = shared < 0 ? 0 : lanes == 2 ? half : shared_bytes;
    ws_plan *p = nullptr;
    rc = plan_create_impl(ctx, cfgs + lo, hi - lo, fld, n_fld, acc, n_acc, hw, nullptr, 0, nullptr, cap, &p,
                          ctx->upload_stream, sh, sh_bytes);
    if (rc != WS_OK) break;
    plans.push_back(p);
    cudaEvent_t ev;
    e = new_event(&ev);
    if (e != cudaSuccess) break;
    e = cudaEventRecord(ev, ctx->upload_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sk, ev, 0);
    if (e != cudaSuccess) break;
    rc = p->execute(WS_MODE_DIRECT, sk);
    if (rc != WS_OK) break;
    e = cudaMemcpyAsync(b + o_res + (size_t)lo * sizeof(ws_result), p->dev(p->d_results),
                        (size_t)(hi - lo) * sizeof(ws_result), cudaMemcpyDeviceToDevice, sk);
  }
  if (lanes == 2 && !evs.empty()) {
    // `st` continues (ranking, copies back) once the lane's parts are done; joined even
    // after a failure, so that the synchronisation below covers both lanes
    cudaEvent_t join;
    const cudaError_t ej = new_event(&join);
    const cudaError_t ej2 = ej == cudaSuccess ? cudaEventRecord(join, ctx->lane_stream) : ej;
    const cudaError_t ej3 = ej2 == cudaSuccess ? cudaStreamWaitEvent(st, join, 0) : ej2;
    if (e == cudaSuccess) e = ej3;
  }
  if (rc == WS_OK && e == cudaSuccess) {
    e = launch_keys((const ws_result *)(b + o_res), n_cfg, (double *)(b + o_keys), st);
    if (e == cudaSuccess) {
      RankArgs ra;
      ra.keys = (const double *)(b + o_keys);
      ra.seg = (const int32_t *)(b + o_seg);
      ra.order = (int32_t *)(b + o_ord);
      ra.rank = (int32_t *)(b + o_rnk);
      ra.n = n_cfg;
      ra.n_seg = 1;
      e = launch_rank(ra, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, b + o_res, rb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && order_out)
      e = cudaMemcpyAsync(order_out, b + o_ord, (size_t)n_cfg * 4, cudaMemcpyDeviceToHost, st);
  }
  // everything issued so far must finish before the plans' memory goes back to the arena
  const cudaError_t e1 = cudaStreamSynchronize(st), e2 = cudaStreamSynchronize(ctx->upload_stream);
  const cudaError_t e3 = lanes == 2 ? cudaStreamSynchronize(ctx->lane_stream) : cudaSuccess;
  if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
  if (rc == WS_OK && e != cudaSuccess) {
    set_error(std::string("pipelined estimate: ") + cudaGetErrorString(e));
    rc = WS_ECUDA;
  }
  // a failed step may leave bits set in the shared scratch (its kernels are done: synchronised above)
  if (shared >= 0 && rc != WS_OK) ctx->oneshot_dirty = true;
  std::vector<int> short_of_room;   // candidates a part had too little scratch for
  for (int i = 0; rc == WS_OK && i < n_cfg; ++i)
    if (out[i].status == WS_ENOMEM) short_of_room.push_back(i);
  for (ws_plan *p : plans) ws_plan_destroy(p);
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  for (int64_t o : {o_res, o_keys, o_ord, o_rnk, o_seg})
    if (o >= 0) ar.release(o);
  // a part's share of the arena may be too small for a field that one plan could hold:
  // then the caller runs the batch as one plan instead.  A field too large for the whole
  // arena keeps its WS_ENOMEM (one plan would refuse it as well).
  if (!short_of_room.empty()) {
    // the one plan may use the room the shared scratch takes now
    if (shared >= 0) {
      ar.release(ctx->oneshot_off);
      ctx->oneshot_off = -1;
      ctx->oneshot_bytes = 0;
    }
    const size_t room = ar.largest_free();
    for (int i : short_of_room) {
      size_t dsc = 0, scr = 0, mf = 0;
      plan_requirements(cfgs + i, 1, fld, n_fld, acc, n_acc, hw, &dsc, &scr, &mf);
      if (mf + ((size_t)8 << 20) <= room) return WS_ENOMEM;
    }
  }
  return rc;
}

extern "C" int ws_estimate_batch(ws_ctx *ctx, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                                 const ws_access *acc, int n_acc, const ws_hw *hw, ws_result *out,
                                 int32_t *order_out, int mode, void *stream) {
  if (!ctx || (n_cfg > 0 && !out)) return WS_EINVAL;
  if (mode != WS_MODE_PLAIN && n_cfg >= 2 * kPipeMin && hw && hw_valid(*hw) && cfgs && (n_fld == 0 || fld) &&
      (n_acc == 0 || acc)) {
    CU(cudaSetDevice(ctx->device));
    const int rc = estimate_pipelined(ctx, cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, out, order_out,
                                      pick_stream(ctx, stream));
    if (rc != WS_ENOMEM) return rc;
    // the parts did not fit together: one plan, which may run in several scratch passes
  }
  // one plan; it runs in the context's kept scratch unless another estimate holds it
  std::unique_lock<std::mutex> kept(ctx->oneshot_mu, std::try_to_lock);
  ws_plan *p = nullptr;
  int rc = plan_create_impl(ctx, cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, nullptr, 0, nullptr, 0, &p, nullptr,
                            kept.owns_lock() ? kCtxScratch : -1, 0);
  if (rc != WS_OK) return rc;
  // a one-shot plan would replay its graph once: launch the batched kernels directly
  rc = ws_plan_execute(p, mode == WS_MODE_BATCHED ? WS_MODE_DIRECT : mode, stream);
  if (rc == WS_OK) rc = ws_plan_results(p, out, order_out, stream);
  // a failed step may leave bits set in the kept scratch, and its kernels must be done with
  // it before another estimate takes it
  if (rc != WS_OK && kept.owns_lock()) {
    cudaStreamSynchronize(pick_stream(ctx, stream));
    ctx->oneshot_dirty = true;
  }
  ws_plan_destroy(p);
  return rc;
}

void ws::ctx_reclaim(ws_ctx *ctx) {
  std::unique_lock<std::mutex> kept(ctx->oneshot_mu, std::try_to_lock);
  if (!kept.owns_lock() || ctx->oneshot_off < 0) return;
  ctx->arena->release(ctx->oneshot_off);
  ctx->oneshot_off = -1;
  ctx->oneshot_bytes = 0;
}

extern "C" int ws_describe(const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld, const ws_access *acc,
                           int n_acc, const ws_hw *hw, ws_cfg_info *out) {
  if (n_cfg < 0 || !hw || (n_cfg > 0 && (!cfgs || !out))) return WS_EINVAL;
  if (!hw_valid(*hw)) return WS_EINVAL;
  FieldCache cache;
  for (int i = 0; i < n_cfg; ++i) {
    Compiled cc;
    ws_cfg_info &o = out[i];
    memset(&o, 0, sizeof(o));
    o.status = compile_config(cfgs[i], fld, n_fld, acc, n_acc, *hw, cc, &cache);
    if (o.status != WS_OK) continue;
    const DCfg &d = cc.d;
    for (int k = 0; k < 3; ++k) o.grid[k] = d.g[k];
    o.threads = d.T;
    o.warps_per_block = d.wpb;
    o.blocks_per_sm = d.bpsm;
    o.n_field = d.n_field;
    o.total_blocks = (int64_t)d.g[0] * d.g[1] * d.g[2];
    o.rep_block = d.rep;
    o.wave_first = d.s;
    o.wave_blocks = d.weff;
    o.y_lo = d.y_lo;
    o.y_hi = d.y_hi;
    o.z_lo = d.z_lo;
    o.z_hi = d.z_hi;
    o.y_dist = d.y_dist;
    o.z_dist = d.z_dist;
    o.modelled_warps = d.lev_end[3];
    for (size_t k = 0; k < cc.f.size(); ++k) {
      o.folded_loads += cc.f[k].n_load;
      o.folded_stores += cc.f[k].n_store;
      o.scratch_bytes += cc.need_words[k] * 4;
    }
  }
  return WS_OK;
}

extern "C" int ws_describe_fields(const ws_config *cfg, const ws_field *fld, int n_fld, const ws_access *acc,
                                  int n_acc, const ws_hw *hw, ws_field_info *out) {
  if (!cfg || !hw || !out || !hw_valid(*hw)) return WS_EINVAL;
  Compiled cc;
  int rc = compile_config(*cfg, fld, n_fld, acc, n_acc, *hw, cc);
  if (rc != WS_OK) return rc;
  // multi-dimensional candidates compile to a block and a wave descriptor per field:
  // the block bitmap range comes from the first, the wave range (in the virtual layout)
  // from the second
  const size_t n = (size_t)cfg->n_field, w = cfg->address_mode == WS_ADDR_MULTIDIM ? n : 0;
  for (size_t k = 0; k < n; ++k) {
    ws_field_info &o = out[k];
    memset(&o, 0, sizeof(o));
    o.lo_sector[0] = cc.f[k].lo[0];
    o.words[0] = cc.f[k].words[0];
    o.lo_sector[1] = cc.f[w + k].lo[1];
    o.words[1] = cc.f[w + k].words[1];
    o.n_load = cc.f[k].n_load;
    o.n_store = cc.f[k].n_store;
  }
  return WS_OK;
}

extern "C" int ws_plan_dry_run(const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                               const ws_access *acc, int n_acc, const ws_hw *hw, const ws_tuning *tuning,
                               size_t scratch_bytes, ws_plan_summary *out) {
  if (!hw || !out || n_cfg < 0 || n_fld < 0 || n_acc < 0) return WS_EINVAL;
  if (n_cfg > 0 && (!cfgs || (n_fld > 0 && !fld) || (n_acc > 0 && !acc))) return WS_EINVAL;
  if (!hw_valid(*hw)) return WS_EINVAL;
  memset(out, 0, sizeof(*out));
  Plan p;
  p.n_cfg = n_cfg;
  p.hw = *hw;
  p.dhw = to_dhw(*hw);
  memset(&p.tune, 0, sizeof(p.tune));
  if (tuning) p.tune = *tuning;
  default_tuning(p.tune);
  HostDesc h;
  build_host(&p, cfgs, n_cfg, fld, n_fld, acc, n_acc, hw, [&](size_t, size_t) { return scratch_bytes; }, h);
  for (const DCfg &d : h.hcfg) out->candidates_ok += d.status == WS_OK;
  out->fields = (int64_t)p.hfld.size();
  out->groups = (int64_t)p.hgrp.size();
  out->passes = (int64_t)p.passes.size();
  out->enum_items = p.item_begin_end;
  out->row_items = p.ritem_begin_end;
  out->count_items = p.citem_begin_end;
  out->access_entries = (int64_t)h.hacc.size();
  out->interval_entries = (int64_t)h.hiv.size();
  out->descriptor_bytes = (int64_t)h.desc_bytes;
  out->scratch_bytes = (int64_t)h.scratch;
  for (int64_t w : p.need_words) out->bitmap_bytes += 4 * w;
  return WS_OK;
}

extern "C" double ws_rank_key(double t) {
  if (!(t > 0.0) || std::isinf(t)) return t;
  int e = 0;
  double m = std::frexp(t, &e);
  return std::ldexp(std::nearbyint(std::ldexp(m, 40)), e - 40);
}

extern "C" int ws_rank(ws_ctx *ctx, const ws_result *res, int n, int32_t *order_out, void *stream) {
  if (!ctx || n < 0 || (n > 0 && (!res || !order_out))) return WS_EINVAL;
  if (n == 0) return WS_OK;
  CU(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, stream);
  const size_t rb = (size_t)n * sizeof(ws_result);
  int64_t o_res = ctx->arena->alloc(rb), o_keys = ctx->arena->alloc((size_t)n * 8),
          o_ord = ctx->arena->alloc((size_t)n * 4), o_seg = ctx->arena->alloc(8), o_rnk = ctx->arena->alloc((size_t)n * 4);
  int rc = WS_OK;
  if (o_res < 0 || o_keys < 0 || o_ord < 0 || o_seg < 0 || o_rnk < 0) rc = WS_ENOMEM;
  char *b = ctx->arena->base;
  if (rc == WS_OK) {
    int32_t seg[2] = {0, n};
    cudaError_t e = cudaMemcpyAsync(b + o_res, res, rb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_seg, seg, sizeof(seg), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_keys((const ws_result *)(b + o_res), n, (double *)(b + o_keys), st);
    if (e == cudaSuccess) {
      RankArgs ra;
      ra.keys = (const double *)(b + o_keys);
      ra.seg = (const int32_t *)(b + o_seg);
      ra.order = (int32_t *)(b + o_ord);
      ra.rank = (int32_t *)(b + o_rnk);
      ra.n = n;
      ra.n_seg = 1;
      e = launch_rank(ra, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(order_out, b + o_ord, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("ws_rank: ") + cudaGetErrorString(e));
      rc = WS_ECUDA;
    }
  }
  for (int64_t o : {o_res, o_keys, o_ord, o_seg, o_rnk}) ctx->arena->release(o);
  return rc;
}

// ---------------------------------------------------------------------------------
// autotuner cache: one line per workload class,
// "log2(n_cfg) chunk_warps enum_threads count_words ctas_per_sm pass_mb"
// ---------------------------------------------------------------------------------
static int bucket(int n) {
  int b = 0;
  while (n > 1) {
    n >>= 1;
    ++b;
  }
  return b;
}

void ws::tuning_cache_lookup(ws_ctx *ctx, int n_cfg, ws_tuning *t) {
  const char *path = getenv("WS_TUNE_CACHE");
  if (!path || !*path) return;
  std::ifstream f(path);
  int b, ch, th, cw, cs, pm;
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    if (is >> b >> ch >> th >> cw >> cs >> pm && b == bucket(n_cfg)) {
      t->chunk_warps = ch;
      t->enum_threads = th;
      t->count_words = cw;
      t->ctas_per_sm = cs;
      t->pass_mb = pm;
    }
  }
  (void)ctx;
}

void ws::tuning_cache_store(ws_ctx *ctx, int n_cfg, const ws_tuning &t) {
  const char *path = getenv("WS_TUNE_CACHE");
  if (!path || !*path) return;
  std::ofstream f(path, std::ios::app);
  f << bucket(n_cfg) << " " << t.chunk_warps << " " << t.enum_threads << " " << t.count_words << " "
    << t.ctas_per_sm << " " << t.pass_mb << "\n";
  (void)ctx;
}
