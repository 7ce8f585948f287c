// Device side of the metric estimator (sm_103a).
//
//   enum_kernel   persistent, work-stealing CTAs.  Representative block (Sec. 4.2, 4.3):
//                 every (warp, access instruction) pair exactly -- per-instruction unique
//                 sectors (L1 request / write-through volumes), half-warp bank cycles and
//                 the block bitmaps.  Wave / y / z sets of field groups that cannot take
//                 the row walk: per modelled warp, as sector intervals of row segments
//                 (segment walk) or address by address.
//   rows_kernel   wave, y set and z set as whole grid rows: each merged load run of a
//                 row is one sector range set with 64-bit red.or; per-warp store sectors
//                 by floor sums (Sec. 4.4, closed-form counting instead of implicit sets).
//   count_kernel  popcounts of the bitmaps: unique sectors, unique 128 B lines (nibble
//                 OR), y / z overlaps by AND / AND-NOT, reading only the pages the row
//                 walk flagged, one warp per page.  Leaves the bitmaps and flags zeroed for
//                 the next step (only non-zero positions are written).
//   model_kernel  fp64 capacity model and limiters (Sec. 2, 4.5), one thread per candidate.
//   rank_count_kernel, rank_scatter_kernel   stable counting rank per segment (Sec. 5.8).
// The three persistent kernels take work items from an atomic counter and find each item's
// field group (or field) in an owner table the host lays out with the items.
#include <cuda_runtime.h>

#include <mutex>

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

// Bank-conflict visitor for both half warps of one instruction (Sec. 4.2): unique
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

// The same visitor for power-of-two banks x bank width (their product dividing 1024)
// on 32-bit byte addresses relative to a 1024-byte aligned origin, which have the same
// banks and pairing distances as the absolute ones.
__device__ int bank_cycles_rel32(uint32_t rel, bool act, uint32_t lane, uint32_t bshift, uint32_t bmask,
                                 uint32_t pair_dist) {
  const uint32_t word = rel >> bshift, bank = word & bmask;
  const uint32_t actm = __ballot_sync(FULL, act);
  {
    // every lane active and each half warp's words ascending by 0 or 1 from lane to lane:
    // its unique words are the consecutive words first .. last, which fall in distinct
    // banks round-robin, so a group spanning less than the pairing distance costs
    // ceil(count / banks) cycles
    const uint32_t prev = __shfl_up_sync(FULL, word, 1);
    const bool step = (lane & 15u) == 0u || word - prev <= 1u;
    if (__all_sync(FULL, act && step)) {
      const uint32_t w0 = __shfl_sync(FULL, word, lane & 16u), w1 = __shfl_sync(FULL, word, (lane & 16u) | 15u);
      if (((w1 - w0) << bshift) < pair_dist) {
        const uint32_t nb = bmask + 1u, n = w1 - w0 + 1u;
        const uint32_t c = (n + nb - 1u) / nb;
        return (int)(__shfl_sync(FULL, c, 0) + __shfl_sync(FULL, c, 16));
      }
    }
  }
  const uint32_t halfm = lane < 16 ? 0x0000ffffu : 0xffff0000u;
  const uint32_t same = __match_any_sync(FULL, word) & actm & halfm;
  const bool uniq = act && lane == (uint32_t)(__ffs(same) - 1);
  uint32_t todo = __ballot_sync(FULL, uniq);
  int cycles = 0;
  while (todo) {
    const bool mine = (todo >> lane) & 1u;
    const uint32_t v = __reduce_min_sync(halfm, mine ? word : 0xffffffffu);
    const bool member = mine && ((word - v) << bshift) < pair_dist;
    const uint32_t mm = __ballot_sync(FULL, member);
    const uint32_t sameb = __match_any_sync(FULL, bank) & mm & halfm;
    const uint32_t c = __reduce_max_sync(halfm, member ? (uint32_t)__popc(sameb) : 0u);
    if ((lane & 15u) == 0) cycles += (int)c;
    todo &= ~mm;
  }
  return (int)__reduce_add_sync(FULL, (uint32_t)cycles);
}


__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
  return (__umulhi(n, f.m) + n) >> f.s;
}

// Run-head insertion of one access instruction (32-bit addresses).  Consecutive
// active lanes whose sectors step by 0 or 1 inside one bitmap word form a run; the
// first lane of each run sets the run's bit range [head sector, tail sector] with one
// red.or.  Every sector between head and tail is touched by some lane of the run, so
// the bitmap receives exactly the union of the lanes' sectors whatever the layout
// (a scattered layout just makes more, shorter runs).  r: byte address relative to
// the bitmap origin; lanes with r >= limit are skipped and counted in `bad`.
// With want_count the number of distinct sectors of the instruction is returned
// (warp-uniform): the sum of run lengths when runs increase strictly across the
// warp, else the exact per-word count.
__device__ __forceinline__ uint32_t runs_insert(uint32_t *__restrict__ bm, uint32_t r, bool act, uint32_t limit,
                                                uint32_t lane, uint32_t &bad, bool want_count) {
  const bool inside = r < limit;
  bad += act && !inside;
  act = act && inside;
  const uint32_t sec = r >> 5;
  const uint32_t prev = __shfl_up_sync(FULL, sec, 1);
  const uint32_t actm = __ballot_sync(FULL, act);
  const uint32_t below = actm & ((1u << lane) - 1u);
  const bool prev_act = ((actm << 1) >> lane) & 1u;
  const bool cont = prev_act && (sec - prev) <= 1u && ((sec ^ prev) >> 5) == 0u;
  const bool head = act && !cont;
  const uint32_t heads = __ballot_sync(FULL, head);
  const uint32_t ends = actm & ~((actm & ~heads) >> 1);
  const uint32_t t = __ffs(ends & (0xffffffffu << lane)) - 1u;
  const uint32_t tail = __shfl_sync(FULL, sec, t);
  if (head) {
    const uint32_t hb = sec & 31u, tb = tail & 31u;
    atomicOr(bm + (sec >> 5), (0xffffffffu >> (31u - tb)) & (0xffffffffu << hb));
  }
  if (!want_count) return 0;
  const uint32_t pl = below ? 31u - __clz(below) : 0u;
  const uint32_t psec = __shfl_sync(FULL, sec, pl);
  if (__all_sync(FULL, !head || below == 0u || sec > psec))
    return __reduce_add_sync(FULL, head ? tail - sec + 1u : 0u);
  uint32_t cnt = 0;   // overlapping runs: count distinct sectors word by word
  const uint32_t word = sec >> 5, bit = 1u << (sec & 31u);
  uint32_t pending = actm;
  while (pending) {
    const uint32_t lw = __shfl_sync(FULL, word, __ffs(pending) - 1);
    const bool mine = act && word == lw;
    cnt += __popc(__reduce_or_sync(FULL, mine ? bit : 0u));
    pending &= ~__ballot_sync(FULL, mine);
  }
  return cnt;
}

// Lane-per-access walk of the wave / y / z loads.  With P = the smallest power of two
// >= the field's folded loads (at most 32), the warp's lanes form 32/P groups of P
// lanes; lane (g, a) evaluates access a for the P threads g*P .. g*P+P-1 of the
// modelled warp, merging the sector bits of one bitmap word in a register and
// flushing it with one red.or when the word changes.  tbase: the slice's relative
// thread addresses; slice: which of them are valid.
template <int P, bool CHECK>
__device__ __forceinline__ void lpa_walk(const uint32_t *__restrict__ tbase, uint32_t slice, uint32_t b32,
                                         uint32_t limit, uint32_t *__restrict__ bm, uint32_t &cw, uint32_t &cb,
                                         uint32_t &bad) {
  auto step = [&](uint32_t tb) {
    const uint32_t r = tb + b32;
    if (CHECK && r >= limit) {
      ++bad;
      return;
    }
    const uint32_t w = r >> 10;
    const bool flush = w != cw;
    if (flush && cb) atomicOr(bm + cw, cb);
    cb = (flush ? 0u : cb) | __funnelshift_l(0u, 1u, r >> 5);
    cw = w;
  };
  constexpr uint32_t full = P == 32 ? 0xffffffffu : ((1u << P) - 1u);
  if (P >= 4) {
    const uint4 *t4 = reinterpret_cast<const uint4 *>(tbase);
    if (slice == full) {
#pragma unroll
      for (int q = 0; q < P / 4; ++q) {
        const uint4 v = t4[q];
        step(v.x);
        step(v.y);
        step(v.z);
        step(v.w);
      }
    } else {
#pragma unroll
      for (int q = 0; q < P / 4; ++q) {
        const uint4 v = t4[q];
        const uint32_t m = slice >> (4 * q);
        if (m & 1u) step(v.x);
        if (m & 2u) step(v.y);
        if (m & 4u) step(v.z);
        if (m & 8u) step(v.w);
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < P; ++t)
      if ((slice >> t) & 1u) step(tbase[t]);
  }
}

// The same walk over all 32 threads of a modelled warp, also counting the distinct
// sectors of the lane's access instruction: the number of sector changes along the
// walk, exact when the lane's sectors never decrease (`mono`).
__device__ __forceinline__ void lpa_walk_count(const uint32_t *__restrict__ tbase, uint32_t vmask, uint32_t b32,
                                               uint32_t *__restrict__ bm, uint32_t &cw, uint32_t &cb,
                                               uint32_t &nsec, bool &mono) {
  uint32_t last = 0xffffffffu;
  auto step = [&](uint32_t tb) {
    const uint32_t r = tb + b32;
    const uint32_t sec = r >> 5;
    nsec += sec != last;
    mono = mono && (last == 0xffffffffu || sec >= last);
    last = sec;
    const uint32_t w = r >> 10;
    const bool flush = w != cw;
    if (flush && cb) atomicOr(bm + cw, cb);
    cb = (flush ? 0u : cb) | __funnelshift_l(0u, 1u, sec);
    cw = w;
  };
  const uint4 *t4 = reinterpret_cast<const uint4 *>(tbase);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint4 v = t4[q];
    const uint32_t m = vmask >> (4 * q);
    if (m & 1u) step(v.x);
    if (m & 2u) step(v.y);
    if (m & 4u) step(v.z);
    if (m & 8u) step(v.w);
  }
}

// Exact distinct sectors of one instruction whose lanes hold relative addresses r.
__device__ __forceinline__ uint32_t warp_distinct_sectors(uint32_t r, bool act) {
  {
    // every lane active and sectors not decreasing from lane to lane: equal sectors are
    // neighbours, so the distinct ones are the lanes that start a new sector
    const uint32_t sec = r >> 5, prev = __shfl_up_sync(FULL, sec, 1);
    const uint32_t lane = threadIdx.x & 31u;
    if (__all_sync(FULL, act && (lane == 0u || sec >= prev)))
      return (uint32_t)__popc(__ballot_sync(FULL, lane == 0u || sec != prev));
  }
  const uint32_t word = r >> 10, bit = 1u << ((r >> 5) & 31u);
  uint32_t pending = __ballot_sync(FULL, act), cnt = 0;
  while (pending) {
    const uint32_t lw = __shfl_sync(FULL, word, __ffs(pending) - 1);
    const bool mine = act && word == lw;
    cnt += __popc(__reduce_or_sync(FULL, mine ? bit : 0u));
    pending &= ~__ballot_sync(FULL, mine);
  }
  return cnt;
}


// A uniform field group walks its loads (stores) lane per access when it has at least
// this many; with fewer, most lanes of such a walk would idle.
constexpr int kCombinedWalkMin = 8;

// Sets sectors [s0, s1] of a bitmap viewed as 64-bit units (one red.or per unit).
__device__ __forceinline__ void set_sector_range(unsigned long long *__restrict__ bm, uint32_t s0, uint32_t s1) {
  const uint32_t u0 = s0 >> 6, u1 = s1 >> 6;
  const unsigned long long m0 = ~0ull << (s0 & 63u);
  const unsigned long long m1 = ~0ull >> (63u - (s1 & 63u));
  if (u0 == u1) {
    atomicOr(bm + u0, m0 & m1);
    return;
  }
  atomicOr(bm + u0, m0);
  for (uint32_t u = u0 + 1; u < u1; ++u) atomicOr(bm + u, ~0ull);
  atomicOr(bm + u1, m1);
}

// Adds sectors [s0, s1] to a lane's pending 64-bit unit (cu, cb), flushing it with one
// red.or when the range leaves that unit; units the range covers entirely are written
// directly.  The caller flushes the last pending unit.  Returns the red.or issued.
__device__ __forceinline__ uint32_t put_range(unsigned long long *__restrict__ bm, uint32_t &cu,
                                              unsigned long long &cb, uint32_t s0, uint32_t s1) {
  const uint32_t u0 = s0 >> 6, u1 = s1 >> 6;
  const unsigned long long m0 = ~0ull << (s0 & 63u);
  const unsigned long long m1 = ~0ull >> (63u - (s1 & 63u));
  uint32_t n = 0;
  if (u0 == u1) {
    if (u0 == cu) {
      cb |= m0 & m1;
      return 0;
    }
    if (cb) {
      atomicOr(bm + cu, cb);
      n = 1;
    }
    cu = u0;
    cb = m0 & m1;
    return n;
  }
  if (u0 == cu) {
    atomicOr(bm + u0, cb | m0);
  } else {
    if (cb) {
      atomicOr(bm + cu, cb);
      n = 1;
    }
    atomicOr(bm + u0, m0);
  }
  for (uint32_t u = u0 + 1; u < u1; ++u) atomicOr(bm + u, ~0ull);
  cu = u1;
  cb = m1;
  return n + (u1 - u0);
}

// Flags the pages [p0, p1] of one bitmap as written.  The flag array starts zeroed and only
// ever receives ones until the counting kernel clears it, so plain byte stores suffice (the
// same value from any number of writers; reading a flag first to skip the store was slower).
__device__ __forceinline__ void flag_pages(uint8_t *__restrict__ fl, uint32_t p0, uint32_t p1) {
  for (uint32_t p = p0; p <= p1; ++p) fl[p] = 1;
}

// Byte range [lo, hi] (relative to the bitmap origin) of one row segment of a
// modelled warp under byte offset bo and extent ext.  Thread addresses are kept as
// their low 32 bits; `mn` is the warp's smallest full thread address, and every valid
// thread lies less than 2^32 bytes above it (the bitmap of a non-wide field spans
// less than that), so address - mn is exact in 32 bits.  Returns false when the range
// leaves [0, limit).
__device__ __forceinline__ bool segment_range(uint32_t th, uint32_t tt, int64_t mn, int64_t bo, uint32_t ext,
                                              uint32_t limit, uint32_t &lo, uint32_t &hi) {
  const uint32_t m32 = (uint32_t)mn;
  const uint32_t dh = th - m32, dt = tt - m32;
  const int64_t vlo = mn + (int64_t)min(dh, dt) + bo;
  const int64_t vhi = mn + (int64_t)max(dh, dt) + bo + (int64_t)ext;
  if (vlo < 0 || vhi >= (int64_t)limit) return false;
  lo = (uint32_t)vlo;
  hi = (uint32_t)vhi;
  return true;
}

// Sum_{i=0}^{n-1} floor((a*i + b) / m) for a, b < m <= 32 and n < 2^31, by lattice-point
// counting: with t = floor((a*(n-1) + b) / m) levels the sum equals t*n minus the
// number of (i, k) with k <= t and a*i + b < k*m, which is the same kind of sum with the
// roles of a and m exchanged; the exchanges follow Euclid's algorithm on (m, a), so all
// divisors stay below 33.
__device__ int64_t floor_sum_small(int64_t n, uint32_t m, uint32_t a, uint32_t b) {
  int64_t res = 0, sgn = 1;
  while (n > 0) {
    if (a >= m) {
      res += sgn * (int64_t)(a / m) * (n * (n - 1) / 2);
      a %= m;
    }
    if (b >= m) {
      res += sgn * (int64_t)(b / m) * n;
      b %= m;
    }
    if (a == 0) break;
    const int64_t t = ((int64_t)a * (n - 1) + b) / m;
    if (t == 0) break;
    res += sgn * t * n;
    const uint32_t nb = m - b + a - 1;
    n = t;
    const uint32_t om = m;
    m = a;
    a = om;
    b = nb;
    sgn = -sgn;
  }
  return res;
}

// Sum_{i<n} floor((P*i + c) / 32) where every term's argument is >= 0 (P of any sign).
// The multiple-of-32 part of P and c comes out in closed form; what is left is a sum
// with a, b < 32 (none at all when P is a multiple of 32, as for every fp64 row of four
// or more threads).
__device__ __forceinline__ int64_t sum_floor32(int64_t n, int64_t P, int64_t c) {
  if (n <= 0) return 0;
  if (P < 0) {
    c += P * (n - 1);
    P = -P;
  }
  int64_t res = (P >> 5) * (n * (n - 1) / 2) + (c >> 5) * n;
  const uint32_t a = (uint32_t)(P & 31), b = (uint32_t)(c & 31);
  if (a != 0) res += floor_sum_small(n, 32u, a, b);
  return res;
}

// Distinct sectors of one store instruction summed over the warps of a row walk's grid
// row: the row's threads are split into warp segments (consecutive threads of one warp
// within one block; a warp's other segments lie in other rows and share no sector with
// this one), each counted as floor(last / 32) - floor(first / 32) + 1 bytes-to-sectors.
// Segments repeat from block to block with the address step B0 * step, so each segment
// position contributes two floor sums over the row's whole blocks; the block cut by N0
// is counted directly.  A0 + step * x is the relative address of point x of the row.
__device__ int64_t row_store_sectors(int64_t A0, int64_t step, int32_t B0, int32_t N0, int32_t full_end,
                                     uint32_t t, uint32_t bxa, uint32_t bxb) {
  auto direct = [&](int64_t x0, int64_t x1) -> int64_t {
    const int64_t p = A0 + step * x0, q = A0 + step * x1;
    return (max(p, q) >> 5) - (min(p, q) >> 5) + 1;
  };
  int64_t cnt = 0;
  const int64_t xa = (int64_t)bxa * B0, xb = min((int64_t)bxb * B0, (int64_t)N0);
  if ((B0 & 31) == 0) {
    // warps tile the row in aligned runs of 32 threads
    const int64_t nx = xb - xa, nq = nx >> 5;
    if (nq > 0) {
      const int64_t p0 = A0 + step * xa, p1 = A0 + step * (xa + 31);
      cnt += sum_floor32(nq, 32 * step, max(p0, p1)) - sum_floor32(nq, 32 * step, min(p0, p1)) + nq;
    }
    if (nx & 31) cnt += direct(xa + (nq << 5), xb - 1);
    return cnt;
  }
  const int32_t f1 = (int32_t)((32 - (((int64_t)t * B0) & 31)) & 31);
  const uint32_t bfe = min(bxb, (uint32_t)full_end);
  const int64_t nfull = bfe > bxa ? (int64_t)(bfe - bxa) : 0;
  const int64_t P = (int64_t)B0 * step;
  for (int32_t ta = 0; ta < B0;) {
    const int32_t tb = (ta == 0 && f1 > 0) ? min(f1, B0) : min(ta + 32, B0);
    if (nfull > 0) {
      const int64_t p0 = A0 + step * (xa + ta), p1 = A0 + step * (xa + tb - 1);
      cnt += sum_floor32(nfull, P, max(p0, p1)) - sum_floor32(nfull, P, min(p0, p1)) + nfull;
    }
    if (bxb > bfe) {
      const int64_t xs = (int64_t)full_end * B0 + ta, xe = min((int64_t)full_end * B0 + tb, (int64_t)N0);
      if (xe > xs) cnt += direct(xs, xe - 1);
    }
    ta = tb;
  }
  return cnt;
}

// Shared-memory images of one field group, staged by the enumeration and row kernels.
struct StageSmem {
  DCfg *c;
  DGroup *g;
  DField *fk;
  int32_t *loff, *soff, *ioff;   // first load / store / merged interval of field k
  uint8_t *af;                   // field of each staged access
  int64_t *boff;                 // byte offset of each staged access
  uint32_t *b32;                 // uniform groups: 32-bit offset from the shared thread address (may be null)
  uint8_t *kmin;                 // first folded point that needs each access
  int32_t (*gad)[17];            // issued accesses per thread by valid folded points, [0] levels 0-1, [1] 2-3
  int32_t *gwi;                  // access instructions, [0] levels 0-1, [1] 2-3
  int64_t *ibo;                  // merged load runs: offset relative to the field's bitmap origin
  uint32_t *iext;                //   extent
  uint8_t *iaf;                  //   field
  // row walk only (else null): the runs without a covering run of all fields first, then
  // those covered from another z row, then those covered within their z row; idst[j][k] =
  // first staged slot of field k's runs of kind j; cov = {runs without a covering run,
  // largest |ddy|, largest |ddz| of the covered runs, runs of the first two kinds, largest
  // |ddy| of the last kind}
  int32_t (*idst)[kMaxGroupFields];
  int32_t *cov;
};

// Stages group gi (and its candidate when it differs from cur_cfg); ends with a barrier.
// Returns true when the candidate changed.
__device__ bool stage_group(const EnumArgs &a, int gi, int cur_cfg, const StageSmem &m) {
  if (threadIdx.x == 0) *m.g = a.grp[gi];
  __syncthreads();
  const DGroup &G = *m.g;
  {
    // the group's fields, copied as 8-byte words by all threads
    static_assert(sizeof(DField) % 8 == 0, "DField is copied as 8-byte words");
    const int nw = G.f_count * (int)(sizeof(DField) / 8);
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.fld + G.f_begin);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(m.fk);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
  }
  const bool new_cfg = G.cfg != cur_cfg;
  if (new_cfg && threadIdx.x == 0) *m.c = a.cfg[G.cfg];
  __syncthreads();
  if (threadIdx.x == 0) {
    // all loads of the group first (field by field), then all stores
    int o = 0;
    for (int k = 0; k < G.f_count; ++k) {
      m.loff[k] = o;
      o += m.fk[k].n_load;
    }
    m.loff[G.f_count] = o;
    for (int k = 0; k < G.f_count; ++k) {
      m.soff[k] = o;
      o += m.fk[k].n_store;
    }
    m.soff[G.f_count] = o;
    o = 0;
    for (int k = 0; k < G.f_count; ++k) {
      m.ioff[k] = o;
      o += G.iv ? m.fk[k].n_iv : 0;
    }
    m.ioff[G.f_count] = o;
    if (m.cov) {
      int u = 0, dy = 0, dz = 0, dyy = 0;
      for (int k = 0; k < G.f_count; ++k)
        if (G.iv) {
          m.idst[0][k] = u;
          u += m.fk[k].n_iv_unc;
          if (m.fk[k].n_iv_unc < m.fk[k].n_iv) {
            dy = max(dy, (int)m.fk[k].cov_dy);
            dz = max(dz, (int)m.fk[k].cov_dz);
            dyy = max(dyy, (int)m.fk[k].cov_dy_y);
          }
        }
      int c = u;
      for (int k = 0; k < G.f_count; ++k)
        if (G.iv) {
          m.idst[1][k] = c;
          c += m.fk[k].n_iv_zc;
        }
      const int uz = c;
      for (int k = 0; k < G.f_count; ++k)
        if (G.iv) {
          m.idst[2][k] = c;
          c += m.fk[k].n_iv - m.fk[k].n_iv_unc - m.fk[k].n_iv_zc;
        }
      m.cov[0] = u;
      m.cov[1] = dy;
      m.cov[2] = dz;
      m.cov[3] = uz;
      m.cov[4] = dyy;
    }
  }
  for (int t = threadIdx.x; t < 34; t += blockDim.x) {
    // issued accesses per thread (by valid folded points) and access instructions,
    // summed over the group's fields: [0] block and wave (loads and stores), [1] y / z
    const int lv = t / 17, kv = t % 17;
    int ad = 0, wi = 0;
    for (int k = 0; k < G.f_count; ++k) {
      ad += m.fk[k].cnt_load[kv] + (lv == 0 ? m.fk[k].cnt_store[kv] : 0);
      wi += m.fk[k].n_load + (lv == 0 ? m.fk[k].n_store : 0);
    }
    m.gad[lv][kv] = ad;
    if (kv == 0) m.gwi[lv] = wi;
  }
  __syncthreads();
  // merged load runs, offsets relative to each field's bitmap origin (the enumeration kernel
  // uses them only for groups without the row walk)
  const int n_runs = (m.cov != nullptr || !G.rows) ? m.ioff[G.f_count] : 0;
  for (int j = threadIdx.x; j < n_runs; j += blockDim.x) {
    int k = 0;
    while (m.ioff[k + 1] <= j) ++k;
    const DField &F = m.fk[k];
    const int jj = j - m.ioff[k];
    const DIv v = a.iv[F.iv_begin + jj];
    const int d = !m.cov                          ? j
                  : jj < F.n_iv_unc               ? m.idst[0][k] + jj
                  : jj < F.n_iv_unc + F.n_iv_zc   ? m.idst[1][k] + (jj - F.n_iv_unc)
                                                  : m.idst[2][k] + (jj - F.n_iv_unc - F.n_iv_zc);
    m.ibo[d] = v.boff + F.base - 32 * F.lo[1];
    m.iext[d] = v.ext;
    m.iaf[d] = (uint8_t)k;
  }
  // raw folded accesses; uniform groups fold each field's constant into the 32-bit
  // offsets, so that address = shared thread address + offset for every field
  for (int j = threadIdx.x; j < m.soff[G.f_count]; j += blockDim.x) {
    const bool st = j >= m.loff[G.f_count];
    int k = 0;
    if (!st) {
      while (m.loff[k + 1] <= j) ++k;
    } else {
      while (m.soff[k + 1] <= j) ++k;
    }
    const DField &F = m.fk[k];
    const int i = st ? F.n_load + (j - m.soff[k]) : j - m.loff[k];
    const DAcc d = a.acc[F.acc_begin + i];
    m.boff[j] = d.boff;
    if (m.b32) m.b32[j] = (uint32_t)d.boff + (G.uniform ? (uint32_t)(F.base - 32 * F.lo[1]) : 0u);
    m.kmin[j] = (uint8_t)d.kmin;
    m.af[j] = (uint8_t)k;
  }
  __syncthreads();
  return new_cfg;
}

__global__ void __launch_bounds__(512, 2) enum_kernel(EnumArgs a) {
  __shared__ DCfg s_c;
  __shared__ DGroup s_g;
  __shared__ DField s_fk[kMaxGroupFields];
  __shared__ int32_t s_loff[kMaxGroupFields + 1];   // first load of field k in the staged lists
  __shared__ int32_t s_soff[kMaxGroupFields + 1];   // first store of field k (after all loads)
  __shared__ uint8_t s_af[kMaxFoldedAccesses];      // field of each staged access
  __shared__ int64_t s_boff[kMaxFoldedAccesses];
  __shared__ uint32_t s_b32[kMaxFoldedAccesses];
  __shared__ uint8_t s_kmin[kMaxFoldedAccesses];
  __shared__ uint32_t s_tc[1024];
  __shared__ __align__(16) uint32_t s_tbase[16][32];   // per warp: relative address of each thread's first point
  __shared__ uint8_t s_tkv[16][32];                    // per warp: valid folded points of each thread
  __shared__ uint32_t s_seg[16][32];                   // per warp: row segments (head lane, tail lane, kv)
  __shared__ int32_t s_ioff[kMaxGroupFields + 1];      // first merged interval of field k
  __shared__ uint16_t s_lg[2][32];                     // interval walk lanes: entry | segment phase << 8
  __shared__ uint32_t s_lgG[2];                        //   lanes per entry ([0] merged runs, [1] raw loads)
  __shared__ int32_t s_gad[2][17];                     // group's issued accesses per thread with kv points
  __shared__ int32_t s_gwi[2];                         // group's access instructions ([0] levels 0-1, [1] 2-3)
  __shared__ long long s_item;
  // merged load intervals of an interval-walk group (dynamic): offset, extent, field
  extern __shared__ __align__(16) unsigned char s_dyn[];
  const int iv_cap16 = (a.iv_cap + 15) & ~15;
  int64_t *const s_ibo = reinterpret_cast<int64_t *>(s_dyn);
  uint32_t *const s_iext = reinterpret_cast<uint32_t *>(s_dyn + 8 * iv_cap16);
  uint8_t *const s_iaf = s_dyn + 12 * iv_cap16;
  const StageSmem sm{&s_c, &s_g, s_fk, s_loff, s_soff, s_ioff, s_af, s_boff, s_b32, s_kmin, s_gad, s_gwi,
                     s_ibo, s_iext, s_iaf, nullptr, nullptr};

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t nwarps = blockDim.x >> 5;
  int cur_g = -1, cur_cfg = -1;

  for (;;) {
    if (threadIdx.x == 0) s_item = a.item_lo + (long long)atomicAdd(a.grab, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= a.item_hi) break;
    const int gi = a.own_enum[item];
    if (gi != cur_g) {
      // stage the group, then the interval walk's lane layout and the thread table
      const bool new_cfg = stage_group(a, gi, cur_cfg, sm);
      // with M < 32 entries, G = 32 / M lanes share an entry and take every G-th row segment
      if (threadIdx.x < 64) {
        const int pi = threadIdx.x >> 5, l = threadIdx.x & 31;
        const int M = pi == 0 ? s_ioff[s_g.f_count] : s_loff[s_g.f_count];
        const int G = (M > 0 && M < 32) ? 32 / M : 1;
        const int e = G > 1 ? l % M : l, g = G > 1 ? l / M : 0;
        s_lg[pi][l] = (uint16_t)(e | (g << 8));
        if (l == 0) s_lgG[pi] = (uint32_t)G;
      }
      if (new_cfg) {
        for (int t = threadIdx.x; t < s_c.T; t += blockDim.x) {
          const uint32_t tx = t % s_c.B[0], ty = (t / s_c.B[0]) % s_c.B[1], tz = t / (s_c.B[0] * s_c.B[1]);
          s_tc[t] = tx | (ty << 10) | (tz << 20);
        }
      }
      __syncthreads();
      cur_g = gi;
      cur_cfg = s_g.cfg;
    }
    // the first n0_items items of a group cover the representative block as chunks of
    // (modelled warp, access instruction) pairs; the others chunks of the remaining
    // modelled warps (groups without the row walk)
    const int64_t kk = item - s_g.item_begin;
    const bool blk = kk < s_g.n0_items;
    const uint32_t mw0 = blk ? 0u : (uint32_t)(s_g.mw_block + (kk - s_g.n0_items) * (int64_t)a.chunk);
    const uint32_t mw1 = blk ? 0u : (uint32_t)min(s_g.mw_block + (kk - s_g.n0_items + 1) * (int64_t)a.chunk,
                                                   s_g.mw_end);
    uint32_t acc_lb = 0, acc_lw = 0, acc_req = 0, acc_st = 0, acc_bank = 0, acc_sreq = 0, acc_addr = 0, acc_wi = 0;
    uint32_t bad = 0;

    if (blk) {
      // ---- representative block (Sec. 4.2, 4.3): every (warp, instruction) exactly --
      // distinct sectors per instruction (L1 requests / write-through stores), the block
      // footprint bitmaps, and half-warp bank cycles.  Each warp takes a contiguous run of
      // the item's (class warp, instruction) pairs, instruction fastest, and keeps the class
      // warp's thread coordinates and the field's address base while they stay the same.
      const uint32_t LS = (uint32_t)s_soff[s_g.f_count], L = (uint32_t)s_loff[s_g.f_count];
      const uint32_t np = (uint32_t)s_g.n_rep * LS;
      const uint32_t p0 = (uint32_t)kk * (uint32_t)a.block_pairs, p1 = min(p0 + (uint32_t)a.block_pairs, np);
      const uint32_t per = (p1 - p0 + nwarps - 1) / nwarps;
      const uint32_t q0 = min(p0 + warp * per, p1), q1 = min(q0 + per, p1);
      const bool fast_banks = a.bank_shift >= 0;
      // with the row walk the block bitmaps are built there: count only, one warp per class
      const bool count_only = s_g.rows;
      const uint32_t b = (uint32_t)s_c.rep;
      const uint32_t bt = fdiv(b, s_c.fd_gx);
      const uint32_t bx = b - bt * (uint32_t)s_c.g[0];
      const uint32_t bz = fdiv(bt, s_c.fd_gy);
      const uint32_t by = bt - bz * (uint32_t)s_c.g[1];
      const int32_t faxis = s_c.fold_axis, fold = s_c.fold;
      uint32_t r = q0 / max(LS, 1u), j = q0 - r * LS;
      int cur_r = -1, cur_k = -1;
      uint32_t mult = 0;
      int32_t x = 0, y = 0, z = 0;
      int kv = 0;
      bool valid = false;
      int64_t rbase = 0, rlim = 0;
      for (uint32_t pp = q0; pp < q1; ++pp) {
        if ((int)r != cur_r) {
          cur_r = (int)r;
          cur_k = -1;
          const uint32_t mw = s_g.rep_warp[r];
          mult = s_g.rep_mult[r];
          const uint32_t tid = mw * 32u + lane;
          const bool exists = tid < (uint32_t)s_c.T;
          const uint32_t tc = exists ? s_tc[tid] : 0u;
          x = (int32_t)bx * s_c.B[0] + (int32_t)(tc & 1023u);
          y = (int32_t)by * s_c.B[1] + (int32_t)((tc >> 10) & 1023u);
          z = (int32_t)bz * s_c.B[2] + (int32_t)(tc >> 20);
          if (faxis == 1) y *= fold;
          if (faxis == 2) z *= fold;
          valid = exists && x < s_c.N[0] && y < s_c.N[1] && z < s_c.N[2];
          kv = 0;
          if (valid) kv = faxis == 1 ? min(fold, s_c.N[1] - y) : faxis == 2 ? min(fold, s_c.N[2] - z) : 1;
        }
        if (j == 0u) {
          if (s_g.first_of_cfg) acc_lb += mult * __reduce_add_sync(FULL, (uint32_t)kv);
          acc_addr += mult * __reduce_add_sync(FULL, (uint32_t)s_gad[0][kv]);
          acc_wi += mult * (uint32_t)s_gwi[0];
        }
        const int k = s_af[j];
        if (k != cur_k) {
          cur_k = k;
          const DField &F = s_fk[k];
          const int64_t lin = F.stride[0] * x + F.stride[1] * y + F.stride[2] * z;
          rbase = F.base + (int64_t)F.esize * lin - 32 * F.lo[0];
          rlim = F.words[0] << 10;
        }
        const DField &F = s_fk[k];
        const bool act = valid && (int)s_kmin[j] < kv;
        const int64_t rr = rbase + s_boff[j];
        const bool inside = rr >= 0 && rr < rlim;
        uint32_t nsec;
        if (count_only) nsec = warp_distinct_sectors((uint32_t)rr, act && inside);
        else nsec = bitmap_insert(a.scratch + F.bm[j < L ? BM_BL : BM_BS], rr, act, lane, F.words[0], bad);
        if (j < L) acc_req += mult * nsec;
        else acc_st += mult * nsec;
        if (fast_banks && !F.wide)
          acc_bank += mult * bank_cycles_rel32((uint32_t)rr, act && inside, lane, (uint32_t)a.bank_shift,
                                               (uint32_t)(a.banks - 1), (uint32_t)a.pair_dist);
        else
          acc_bank += mult * bank_cycles_warp(rr + 32 * F.lo[0], act, lane, a.banks, a.bank_bytes, a.pair_dist);
        if (++j == LS) {
          j = 0;
          ++r;
        }
      }
    }
    for (uint32_t mw = mw0 + warp; mw < mw1; mw += nwarps) {
      // ---- decode the modelled warp once for every field of the group
      uint32_t level, b, j;
      const FastDiv fwpb = s_c.fd_wpb;
      if (mw < (uint32_t)s_c.lev_end[0]) {
        level = 0; j = mw; b = (uint32_t)s_c.rep;
      } else if (mw < (uint32_t)s_c.lev_end[1]) {
        level = 1; j = mw - (uint32_t)s_c.lev_end[0]; b = (uint32_t)s_c.s + fdiv(j, fwpb);
      } else if (mw < (uint32_t)s_c.lev_end[2]) {
        level = 2; j = mw - (uint32_t)s_c.lev_end[1]; b = (uint32_t)s_c.y_lo + fdiv(j, fwpb);
      } else {
        level = 3; j = mw - (uint32_t)s_c.lev_end[2]; b = (uint32_t)s_c.z_lo + fdiv(j, fwpb);
      }
      const uint32_t gx = (uint32_t)s_c.g[0], gy = (uint32_t)s_c.g[1];
      const uint32_t w = j - fdiv(j, fwpb) * (uint32_t)s_c.wpb;
      const uint32_t bt = fdiv(b, s_c.fd_gx);
      const uint32_t bx = b - bt * gx;
      const uint32_t bz = fdiv(bt, s_c.fd_gy);
      const uint32_t by = bt - bz * gy;
      if (level == 2 && by == gy - 1) continue;
      if (level == 3 && b >= (uint32_t)s_c.y_lo && b < (uint32_t)s_c.y_hi && by != gy - 1) continue;

      const uint32_t tid = w * 32u + lane;
      const bool exists = tid < (uint32_t)s_c.T;
      const uint32_t tc = exists ? s_tc[tid] : 0u;
      const int32_t x = (int32_t)bx * s_c.B[0] + (int32_t)(tc & 1023u);
      int32_t y = (int32_t)by * s_c.B[1] + (int32_t)((tc >> 10) & 1023u);
      int32_t z = (int32_t)bz * s_c.B[2] + (int32_t)(tc >> 20);
      const int32_t faxis = s_c.fold_axis, fold = s_c.fold;
      if (faxis == 1) y *= fold;
      if (faxis == 2) z *= fold;
      const bool valid = exists && x < s_c.N[0] && y < s_c.N[1] && z < s_c.N[2];
      int kv = 0;
      if (valid) kv = faxis == 1 ? min(fold, s_c.N[1] - y) : faxis == 2 ? min(fold, s_c.N[2] - z) : 1;
      if (s_g.first_wave && level == 1) acc_lw += __reduce_add_sync(FULL, (uint32_t)kv);
      const uint32_t vmask = __ballot_sync(FULL, valid);
      // a thread with fewer valid folded points than the fold skips some accesses; such
      // warps (only at the domain edge) bound-check every address
      const bool partial = __any_sync(FULL, valid && kv < fold);
      uint32_t naddr = 0;

      bool fields_done = false;
      if (level >= 1 && s_g.iv) {
        // ---- interval walk (exact closed-form counting, Sec. 4.4): the warp's valid
        // threads form row segments of consecutive x, and a (segment, merged load run)
        // pair covers one contiguous sector range.  Partial warps (a thread with fewer
        // valid folded points than the fold) take the raw folded loads instead, each
        // checked against the segment's valid points.
        const DField &F0 = s_fk[0];
        const int64_t el = (int64_t)F0.esize * (F0.stride[0] * x + F0.stride[1] * y + F0.stride[2] * z);
        const uint32_t tme = (uint32_t)el;
        s_tbase[warp][lane] = tme;
        const int L = s_loff[s_g.f_count];
        const int S = level == 1 ? s_soff[s_g.f_count] - L : 0;
        if (vmask) {
          // the warp's address range: offsets from its first valid thread fit 32 bits
          // (every bitmap of an interval group spans less than 2^31 bytes); anything
          // else is a descriptor error and the warp is skipped
          const int64_t e0 = (int64_t)__shfl_sync(FULL, (long long)el, __ffs(vmask) - 1);
          const int64_t dd = el - e0;
          const bool fits = !valid || (dd >= -(int64_t)0x7fffffff && dd <= (int64_t)0x7fffffff);
          if (__all_sync(FULL, fits)) {
            const int32_t d = (int32_t)dd;
            const int64_t mn = e0 + __reduce_min_sync(FULL, valid ? d : 0x7fffffff);
            const int64_t mx = e0 + __reduce_max_sync(FULL, valid ? d : -0x7fffffff);
            const uint32_t tx = tc & 1023u;
            const uint32_t heads = __ballot_sync(FULL, valid && (lane == 0u || tx == 0u));
            const uint32_t ends = vmask & ~((vmask & ~heads) >> 1);
            const uint32_t nseg = __popc(heads);
            if ((heads >> lane) & 1u) {
              const uint32_t t = __ffs(ends & (0xffffffffu << lane)) - 1u;
              s_seg[warp][__popc(heads & ((1u << lane) - 1u))] = lane | (t << 8) | ((uint32_t)kv << 16);
            }
            __syncwarp();
            // loads: a lane takes one entry and every G-th segment (G lanes share an
            // entry when there are fewer than 32)
            const int pi = partial ? 1 : 0;
            const int M = partial ? L : s_ioff[s_g.f_count];
            const uint32_t G = s_lgG[pi], lg = s_lg[pi][lane];
            const uint32_t e_l = lg & 255u, g_l = lg >> 8;
            const int bsel = level == 1 ? BM_W : level == 2 ? BM_Y : BM_Z;
            for (int r0 = 0; r0 < M; r0 += 32) {
              const int e = r0 + (int)e_l;
              if (e >= M || g_l >= G) continue;
              int k;
              int64_t bo;
              uint32_t ext;
              if (!partial) {
                k = s_iaf[e];
                bo = s_ibo[e];
                ext = s_iext[e];
              } else {
                k = s_af[e];
                bo = s_boff[e] + s_fk[k].base - 32 * s_fk[k].lo[1];
                ext = 0u;
              }
              const DField &F = s_fk[k];
              const uint32_t limit = (uint32_t)(F.words[1] << 10);
              unsigned long long *const bm = reinterpret_cast<unsigned long long *>(a.scratch + F.bm[bsel]);
              uint32_t cu = 0xffffffffu;
              unsigned long long cb = 0ull;
              if (!partial) {
                // every segment issues the entry: one exact range check for the warp
                if (mn + bo < 0 || mx + bo + (int64_t)ext >= (int64_t)limit) {
                  ++bad;
                  continue;
                }
                const uint32_t b32 = (uint32_t)bo;
                for (uint32_t si = g_l; si < nseg; si += G) {
                  const uint32_t sg = s_seg[warp][si];
                  const uint32_t ra = s_tbase[warp][sg & 255u] + b32, rb = s_tbase[warp][(sg >> 8) & 255u] + b32;
                  put_range(bm, cu, cb, min(ra, rb) >> 5, (max(ra, rb) + ext) >> 5);
                }
              } else {
                const uint32_t kmin = s_kmin[e];
                for (uint32_t si = g_l; si < nseg; si += G) {
                  const uint32_t sg = s_seg[warp][si];
                  if (kmin >= (sg >> 16)) continue;
                  uint32_t lo, hi;
                  if (!segment_range(s_tbase[warp][sg & 255u], s_tbase[warp][(sg >> 8) & 255u], mn, bo, 0u, limit,
                                     lo, hi)) {
                    ++bad;
                    continue;
                  }
                  put_range(bm, cu, cb, lo >> 5, hi >> 5);
                }
              }
              if (cb) atomicOr(bm + cu, cb);
            }
            if (!partial) {
              // stores: lane per store instruction over all segments, counting the
              // instruction's distinct sectors (exact for non-decreasing segments)
              for (int a0 = 0; a0 < S; a0 += 32) {
                const int j = L + a0 + (int)lane;
                uint32_t nsec = 0u, plo = 0u, phi = 0u;
                bool mono = true, ok = false;
                if (j < L + S) {
                  const DField &F = s_fk[s_af[j]];
                  const int64_t bo = s_boff[j] + F.base - 32 * F.lo[1];
                  const uint32_t limit = (uint32_t)(F.words[1] << 10);
                  unsigned long long *const bm = reinterpret_cast<unsigned long long *>(a.scratch + F.bm[BM_WS]);
                  if (mn + bo < 0 || mx + bo >= (int64_t)limit) {
                    ++bad;
                  } else {
                    ok = true;
                    const uint32_t b32 = (uint32_t)bo;
                    uint32_t cu = 0xffffffffu;
                    unsigned long long cb = 0ull;
                    for (uint32_t si = 0; si < nseg; ++si) {
                      const uint32_t sg = s_seg[warp][si];
                      const uint32_t ra = s_tbase[warp][sg & 255u] + b32, rb = s_tbase[warp][(sg >> 8) & 255u] + b32;
                      const uint32_t s0 = min(ra, rb) >> 5, s1 = max(ra, rb) >> 5;
                      put_range(bm, cu, cb, s0, s1);
                      if (si == 0u) {
                        nsec = s1 - s0 + 1u;
                      } else {
                        mono = mono && s0 >= plo && s1 >= phi;
                        const uint32_t from = max(phi + 1u, s0);
                        nsec += s1 >= from ? s1 - from + 1u : 0u;
                      }
                      plo = s0;
                      phi = s1;
                    }
                    if (cb) atomicOr(bm + cu, cb);
                  }
                }
                acc_sreq += __reduce_add_sync(FULL, (ok && mono) ? nsec : 0u);
                uint32_t redo = __ballot_sync(FULL, ok && !mono);
                while (redo) {
                  const int src = __ffs(redo) - 1;
                  redo &= redo - 1;
                  acc_sreq += warp_distinct_sectors(tme + s_b32[L + a0 + src], valid);
                }
              }
            } else {
              for (int j = L; j < L + S; ++j) {
                const DField &F = s_fk[s_af[j]];
                const uint32_t limit = (uint32_t)(F.words[1] << 10);
                const bool act = valid && (int)s_kmin[j] < kv;
                acc_sreq += runs_insert(a.scratch + F.bm[BM_WS], tme + s_b32[j], act, limit, lane, bad, true);
              }
            }
          } else if (lane == 0u) {
            ++bad;
          }
        }
        __syncwarp();
        fields_done = true;
        naddr += (uint32_t)s_gad[level <= 1 ? 0 : 1][kv];
        acc_wi += (uint32_t)s_gwi[level <= 1 ? 0 : 1];
      } else if (level >= 1 && s_g.uniform && !partial) {
        // ---- uniform groups, wave / y / z levels: one walk over all the group's accesses
        const DField &F0 = s_fk[0];
        const int64_t el = (int64_t)F0.esize * (F0.stride[0] * x + F0.stride[1] * y + F0.stride[2] * z);
        s_tbase[warp][lane] = (uint32_t)el;
        int64_t mn = valid ? el : INT64_MAX, mx = valid ? el : INT64_MIN;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          mn = min(mn, (int64_t)__shfl_xor_sync(FULL, (long long)mn, off));
          mx = max(mx, (int64_t)__shfl_xor_sync(FULL, (long long)mx, off));
        }
        __syncwarp();
        const int L = s_loff[s_g.f_count];
        const int S = level == 1 ? s_soff[s_g.f_count] - L : 0;
        const uint32_t tme = s_tbase[warp][lane];
        if (L >= kCombinedWalkMin) {
          // lane per access over all 32 threads of the modelled warp
          for (int a0 = 0; a0 < L && vmask; a0 += 32) {
            const int j = a0 + (int)lane;
            uint32_t cw = 0xffffffffu, cb = 0u;
            uint32_t *bm = nullptr;
            if (j < L) {
              const DField &F = s_fk[s_af[j]];
              const int64_t bo = s_boff[j] + F.base - 32 * F.lo[1];
              const uint32_t limit = (uint32_t)(F.words[1] << 10);
              bm = a.scratch + F.bm[level == 1 ? BM_W : level == 2 ? BM_Y : BM_Z];
              if (mn + bo < 0 || mx + bo >= (int64_t)limit) bad += __popc(vmask);
              else lpa_walk<32, false>(&s_tbase[warp][0], vmask, s_b32[j], limit, bm, cw, cb, bad);
            }
            if (cb) atomicOr(bm + cw, cb);
          }
        } else {
          // few accesses: lane per thread, one run-head insertion per access
          for (int j = 0; j < L; ++j) {
            const DField &F = s_fk[s_af[j]];
            const uint32_t limit = (uint32_t)(F.words[1] << 10);
            uint32_t *const bm = a.scratch + F.bm[level == 1 ? BM_W : level == 2 ? BM_Y : BM_Z];
            runs_insert(bm, tme + s_b32[j], valid, limit, lane, bad, false);
          }
        }
        if (S >= kCombinedWalkMin) {
          for (int a0 = 0; a0 < S && vmask; a0 += 32) {
            const int j = L + a0 + (int)lane;
            uint32_t cw = 0xffffffffu, cb = 0u, nsec = 0u;
            bool mono = true, ok = false;
            uint32_t *bm = nullptr;
            if (j < L + S) {
              const DField &F = s_fk[s_af[j]];
              const int64_t bo = s_boff[j] + F.base - 32 * F.lo[1];
              const uint32_t limit = (uint32_t)(F.words[1] << 10);
              bm = a.scratch + F.bm[BM_WS];
              if (mn + bo < 0 || mx + bo >= (int64_t)limit) {
                bad += __popc(vmask);
              } else {
                lpa_walk_count(&s_tbase[warp][0], vmask, s_b32[j], bm, cw, cb, nsec, mono);
                ok = true;
              }
            }
            if (cb) atomicOr(bm + cw, cb);
            // per-instruction distinct sectors: the lane's count when its sectors never
            // decreased, else an exact recount by the whole warp
            acc_sreq += __reduce_add_sync(FULL, (ok && mono) ? nsec : 0u);
            uint32_t redo = __ballot_sync(FULL, ok && !mono);
            while (redo) {
              const int src = __ffs(redo) - 1;
              redo &= redo - 1;
              acc_sreq += warp_distinct_sectors(tme + s_b32[L + a0 + src], valid);
            }
          }
        } else {
          for (int j = L; j < L + S; ++j) {
            const DField &F = s_fk[s_af[j]];
            const uint32_t limit = (uint32_t)(F.words[1] << 10);
            acc_sreq += runs_insert(a.scratch + F.bm[BM_WS], tme + s_b32[j], valid, limit, lane, bad, true);
          }
        }
        __syncwarp();
        fields_done = true;
        naddr += (uint32_t)s_gad[level <= 1 ? 0 : 1][kv];
        acc_wi += (uint32_t)s_gwi[level <= 1 ? 0 : 1];
      }

      // ---- every field of the group
      for (int k = 0; k < s_g.f_count && !fields_done; ++k) {
        const DField &F = s_fk[k];
        const int n_load = F.n_load;
        const int nst = level <= 1 ? F.n_store : 0;
        if (n_load + (level <= 1 ? nst : 0) == 0 || (level >= 2 && n_load == 0)) continue;
        const int lo_ = s_loff[k], so_ = s_soff[k] - n_load;   // load i at lo_ + i, store i at so_ + i
        naddr += (uint32_t)(F.cnt_load[kv] + (level <= 1 ? F.cnt_store[kv] : 0));
        acc_wi += (uint32_t)(n_load + nst);
        const int64_t lin = F.stride[0] * x + F.stride[1] * y + F.stride[2] * z;

        if (!F.wide) {
          const int64_t rel = F.base + (int64_t)F.esize * lin - 32 * F.lo[1];
          // uniform groups staged the field constant into the 32-bit offsets already
          const uint32_t r0 = s_g.uniform ? (uint32_t)((int64_t)F.esize * lin) : (uint32_t)rel;
          const uint32_t limit = (uint32_t)(F.words[1] << 10);
          uint32_t *const bm = a.scratch + F.bm[level == 1 ? BM_W : level == 2 ? BM_Y : BM_Z];
          if (n_load > 0) {
            // lane per access over slices of P threads (P = 2^lp >= loads, <= 32)
            const int lp = F.lpa_log2p, P = 1 << lp;
            if (P > 1) {
              s_tbase[warp][lane] = r0;
              s_tkv[warp][lane] = (uint8_t)kv;
              __syncwarp();
            }
            // fields with a full warp per access check each lane's range once
            int64_t mn = 0, mx = 0;
            if (P == 32 && !partial) {
              mn = valid ? rel : INT64_MAX;
              mx = valid ? rel : INT64_MIN;
#pragma unroll
              for (int off = 16; off >= 1; off >>= 1) {
                mn = min(mn, (int64_t)__shfl_xor_sync(FULL, (long long)mn, off));
                mx = max(mx, (int64_t)__shfl_xor_sync(FULL, (long long)mx, off));
              }
            }
            const uint32_t al = lane & (uint32_t)(P - 1), g0 = (lane >> lp) << lp;
            const uint32_t slice = (P == 32 ? vmask : (vmask >> g0) & ((1u << P) - 1u));
            const uint32_t *tb = &s_tbase[warp][g0];
            for (int a0 = 0; a0 < n_load && vmask; a0 += P) {
              const int ai = a0 + (int)al;
              uint32_t cw = 0xffffffffu, cb = 0u;
              if (ai < n_load && slice) {
                const uint32_t b32 = s_b32[lo_ + ai];
                if (!partial) {
                  if (P == 32) {
                    const int64_t bo = s_boff[lo_ + ai];
                    if (mn + bo < 0 || mx + bo >= (int64_t)limit) bad += __popc(slice);
                    else lpa_walk<32, false>(tb, slice, b32, limit, bm, cw, cb, bad);
                  } else {
                    switch (lp) {
                      case 0: {  // one thread per lane: its own address, no staging
                        const uint32_t r = r0 + b32;
                        if (r >= limit) {
                          ++bad;
                        } else {
                          cw = r >> 10;
                          cb = __funnelshift_l(0u, 1u, r >> 5);
                        }
                        break;
                      }
                      case 1: lpa_walk<2, true>(tb, slice, b32, limit, bm, cw, cb, bad); break;
                      case 2: lpa_walk<4, true>(tb, slice, b32, limit, bm, cw, cb, bad); break;
                      case 3: lpa_walk<8, true>(tb, slice, b32, limit, bm, cw, cb, bad); break;
                      default: lpa_walk<16, true>(tb, slice, b32, limit, bm, cw, cb, bad); break;
                    }
                  }
                } else {
                  const int km = s_kmin[lo_ + ai];
                  for (int t = 0; t < P; ++t) {
                    if (!((slice >> t) & 1u) || km >= (P > 1 ? (int)s_tkv[warp][g0 + t] : kv)) continue;
                    const uint32_t r = (P > 1 ? tb[t] : r0) + b32;
                    if (r >= limit) {
                      ++bad;
                      continue;
                    }
                    const uint32_t wd = r >> 10;
                    if (wd != cw) {
                      if (cb) atomicOr(bm + cw, cb);
                      cw = wd;
                      cb = 0u;
                    }
                    cb |= 1u << ((r >> 5) & 31u);
                  }
                }
              }
              if (P == 32) {
                if (cb) atomicOr(bm + cw, cb);
              } else {
                // several slices per access: lanes whose last word coincides (other
                // slices, other accesses) merge it into one red.or
                const uint32_t key = cb ? cw : (0x80000000u | lane);
                const uint32_t m = __match_any_sync(FULL, key);
                const uint32_t orcb = __reduce_or_sync(m, cb);
                if (cb && lane == (uint32_t)(__ffs(m) - 1)) atomicOr(bm + cw, orcb);
              }
            }
            if (P > 1) __syncwarp();
          }
          // wave stores: per-instruction unique sectors (partial-store model)
          uint32_t *const ws_ = a.scratch + F.bm[BM_WS];
          for (int i = n_load; i < n_load + nst; ++i) {
            const bool act = valid && (int)s_kmin[so_ + i] < kv;
            acc_sreq += runs_insert(ws_, r0 + s_b32[so_ + i], act, limit, lane, bad, true);
          }
        } else {
          const int64_t rel = F.base + (int64_t)F.esize * lin - 32 * F.lo[1];
          uint32_t *const bm = a.scratch + F.bm[level == 1 ? BM_W : level == 2 ? BM_Y : BM_Z];
          for (int i = 0; i < n_load; ++i) {
            const bool act = valid && (int)s_kmin[lo_ + i] < kv;
            bitmap_insert(bm, rel + s_boff[lo_ + i], act, lane, F.words[1], bad);
          }
          uint32_t *const ws_ = a.scratch + F.bm[BM_WS];
          for (int i = n_load; i < n_load + nst; ++i) {
            const bool act = valid && (int)s_kmin[so_ + i] < kv;
            acc_sreq += bitmap_insert(ws_, rel + s_boff[so_ + i], act, lane, F.words[1], bad);
          }
        }
      }
      acc_addr += __reduce_add_sync(FULL, naddr);
    }
    bad = __reduce_add_sync(FULL, bad);
    if (lane == 0) {
      unsigned long long *c = (unsigned long long *)(a.counters + (int64_t)s_g.cfg * N_COUNTERS);
      typedef unsigned long long u64;
      if (bad) atomicAdd(c + C_OVERFLOW, (u64)bad);
      if (acc_lb) atomicAdd(c + C_LUPS_BLOCK, (u64)acc_lb);
      if (acc_lw) atomicAdd(c + C_LUPS_WAVE, (u64)acc_lw);
      if (acc_req) atomicAdd(c + C_L1_REQ, (u64)acc_req);
      if (acc_st) atomicAdd(c + C_L1_STORE, (u64)acc_st);
      if (acc_bank) atomicAdd(c + C_BANK, (u64)acc_bank);
      if (acc_sreq) atomicAdd(c + C_W_SREQ, (u64)acc_sreq);
      if (acc_addr) atomicAdd(c + C_ADDR, (u64)acc_addr);
      if (acc_addr && blk) atomicAdd(c + C_ADDR0, (u64)acc_addr);
      if (acc_wi) atomicAdd(c + C_WINSTR, (u64)acc_wi);
    }
    __syncthreads();
  }
}


// Row walk of the wave and the y / z layer sets (exact closed-form interval counting,
// Sec. 4.4).  The blocks of a level that share a block row are consecutive in x, so
// the threads of those blocks with one (ty, tz) form one grid row of consecutive x.
// Work item = (field group, chunk of row slots); one grid row per warp.  Each merged
// load run (raw loads when the row has fewer valid folded points than the fold) is one
// sector range of the row; wave stores also add their per-warp sector counts in closed
// form (row_store_sectors).
// Magic numbers of FastDiv for a divisor fixed per work item (once per thread and item).
__device__ __forceinline__ FastDiv make_fastdiv_dev(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.s = d <= 1u ? 0u : 32u - __clz(d - 1u);
  f.m = (uint32_t)((((unsigned long long)1 << 32) * (((unsigned long long)1 << f.s) - d)) / d + 1ull);
  f.pad = 0u;
  return f;
}

// One decoded row slot (a lane's): the byte range of its row (relative to the field
// base; the fields of a row-walk group share element size and strides), the start of the
// row, its thread row, block run, level and valid folded points.
struct RowSlot {
  int64_t lo, hi, el0;
  uint32_t t, bxa, bxb;
  int32_t y, z;           // grid row of the slot's first folded point
  uint8_t lv, kv, pad[2];
};

// True when every grid row displaced from row (y, z) of level lv by at most dy rows in y
// and dz in z (multiples of the fold along the folding axis) is a thread row of the same
// level whose block run contains [bxa, bxb) and whose folded points are all inside the
// domain.  The displaced rows' block rows lie between those of the two extreme corners
// (R = by + gy * bz grows with by and bz), so the level's block interval is checked at
// those two; the z set is checked against its tighter bound (before the y set) throughout.
// Then every run whose covering run lies within that displacement may be skipped at this
// row: the covering run sets a containing range from the displaced row, which the walk
// visits with a containing block run (and if it skips that run there in turn, a run even
// earlier in the covering order covers both).
__device__ __forceinline__ bool row_interior(const DCfg &c, int lv, int32_t y, int32_t z, uint32_t bxa, uint32_t bxb,
                                             int32_t dy, int32_t dz) {
  const int32_t fy = c.fold_axis == 1 ? c.fold : 1, fz = c.fold_axis == 2 ? c.fold : 1;
  if (y < dy || z < dz || y + dy + fy > c.N[1] || z + dz + fz > c.N[2]) return false;
  uint32_t y0 = (uint32_t)(y - dy), y1 = (uint32_t)(y + dy), z0 = (uint32_t)(z - dz), z1 = (uint32_t)(z + dz);
  if (c.fold_axis == 1) {
    y0 = fdiv(y0, c.fd_fold);
    y1 = fdiv(y1, c.fd_fold);
  } else if (c.fold_axis == 2) {
    z0 = fdiv(z0, c.fd_fold);
    z1 = fdiv(z1, c.fd_fold);
  }
  const uint32_t by0 = fdiv(y0, c.fd_b1), by1 = fdiv(y1, c.fd_b1);
  const uint32_t bz0 = fdiv(z0, c.fd_b2), bz1 = fdiv(z1, c.fd_b2);
  if (lv == 3) return by0 == by1 && bz0 == bz1;   // the representative block's own thread rows
  const int64_t gx = c.g[0], gy = c.g[1];
  const int64_t lo = ((int64_t)by0 + gy * (int64_t)bz0) * gx + bxa;
  const int64_t hi = ((int64_t)by1 + gy * (int64_t)bz1) * gx + bxb;
  if (lv == 0) return c.s <= lo && hi <= c.s + c.weff;
  if (lv == 1) return (int64_t)by1 != gy - 1 && c.y_lo <= lo && hi <= c.y_hi;
  const int64_t up = c.y_hi > c.y_lo ? min(c.z_hi, c.y_lo) : c.z_hi;
  return c.z_lo <= lo && hi <= up;
}

__global__ void __launch_bounds__(256, 4) rows_kernel(EnumArgs a) {
  __shared__ DCfg s_c;
  __shared__ DGroup s_g;
  __shared__ DField s_fk[kMaxGroupFields];
  __shared__ int32_t s_loff[kMaxGroupFields + 1];
  __shared__ int32_t s_soff[kMaxGroupFields + 1];
  __shared__ int32_t s_ioff[kMaxGroupFields + 1];
  __shared__ int32_t s_idst[3][kMaxGroupFields];
  __shared__ int32_t s_cov[5];
  __shared__ uint8_t s_af[kMaxFoldedAccesses];
  __shared__ int64_t s_boff[kMaxFoldedAccesses];
  __shared__ uint8_t s_kmin[kMaxFoldedAccesses];
  __shared__ int32_t s_gad[2][17];
  __shared__ int32_t s_gwi[2];
  __shared__ long long s_item;
  __shared__ unsigned long long s_memo_key[kRowsThreads];       // per thread: last store-sector count
  __shared__ uint32_t s_memo_val[kRowsThreads];
  // per field of the staged group: bitmap word offsets, page-flag byte offsets, bitmap byte
  // sizes (block, wave), wave minus block origin and the stores' origin adjustment (block, wave)
  __shared__ int64_t s_fbm[kMaxGroupFields][N_BITMAPS];
  __shared__ int64_t s_fpg[kMaxGroupFields][N_BITMAPS];
  __shared__ int64_t s_flim[kMaxGroupFields][2];
  __shared__ int64_t s_fblk[kMaxGroupFields];
  __shared__ int64_t s_forg[kMaxGroupFields][2];
  __shared__ uint32_t s_fzc[kMaxGroupFields][2];                 // z-set clip window (sectors)
  __shared__ unsigned long long s_acc[kRowsThreads / 32][5];     // per warp: the item's counts
  __shared__ int s_batch;                                         // next batch of 32 slots of the item
  extern __shared__ __align__(16) unsigned char s_dyn[];
  const int iv_cap16 = (a.iv_cap + 15) & ~15;
  int64_t *const s_ibo = reinterpret_cast<int64_t *>(s_dyn);
  uint32_t *const s_iext = reinterpret_cast<uint32_t *>(s_dyn + 8 * iv_cap16);
  uint8_t *const s_iaf = s_dyn + 12 * iv_cap16;
  const StageSmem sm{&s_c, &s_g, s_fk, s_loff, s_soff, s_ioff, s_af, s_boff, nullptr, s_kmin, s_gad, s_gwi,
                     s_ibo, s_iext, s_iaf, s_idst, s_cov};

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  int cur_g = -1, cur_cfg = -1;

  for (;;) {
    if (threadIdx.x == 0) {
      s_item = a.ritem_lo + (long long)atomicAdd(a.rgrab, 1ull);
      s_batch = 0;
    }
    __syncthreads();
    const int64_t item = s_item;
    if (item >= a.ritem_hi) break;
    const int gi = a.own_rows[item];
    if (gi != cur_g) {
      stage_group(a, gi, cur_cfg, sm);
      cur_g = gi;
      cur_cfg = s_g.cfg;
      s_memo_key[threadIdx.x] = ~0ull;   // store-sector counts hold for one candidate's geometry
      for (int i = threadIdx.x; i < s_g.f_count * N_BITMAPS; i += blockDim.x) {
        const int k = i / N_BITMAPS, b = i - k * N_BITMAPS;
        const DField &F = s_fk[k];
        s_fbm[k][b] = F.bm[b];
        s_fpg[k][b] = 4 * F.pg + page_flag_off(b, F.words[0], F.words[1]);
        if (b < 2) {
          s_flim[k][b] = F.words[b] << 10;
          s_forg[k][b] = F.base - 32 * F.lo[b];
        }
        if (b == 0) {
          s_fblk[k] = 32 * (F.lo[1] - F.lo[0]);
          s_fzc[k][0] = F.zshift ? (uint32_t)F.zc_lo : 0u;
          s_fzc[k][1] = F.zshift ? (uint32_t)F.zc_hi : 0xffffffffu;
        }
      }
      __syncthreads();
    }
    const int64_t kk = item - s_g.ritem_begin;
    // ---- row walk of levels 1-3 and the block: every slot is one grid row of a level
    // (block run x thread row); each merged load run (raw loads when the row has fewer
    // valid folded points than the fold) is one sector range of the row, and stores also
    // add their per-warp sector counts in closed form.  A warp takes 32 slots at once, one
    // per lane, and each lane walks the runs and stores of its own row.
    const int64_t q0 = kk * (int64_t)a.chunk_rows;
    const int64_t q1 = min(q0 + (int64_t)a.chunk_rows, s_c.rows_slot_end[(s_g.levels & 1) ? 3 : 2]);
    const int L = s_loff[s_g.f_count];
    const int S = s_soff[s_g.f_count] - L;
    const int Mfull = s_ioff[s_g.f_count];
    // runs [0, Mu) have no covering run; at rows inside their level (row_interior) only those
    // are taken, when they are at most half of all runs (otherwise the test of each row costs
    // more than the runs it saves: all runs are taken everywhere).  Runs [Muz, Mfull) are
    // covered from their own z row: at rows whose rows displaced in y alone lie inside the
    // level (a wave is often thinner in z than the z displacements) [0, Muz) are taken.
    const int Mu = 2 * s_cov[0] <= Mfull ? s_cov[0] : Mfull;
    const int Muz = s_cov[3];
    const DField &F0 = s_fk[0];
    const int64_t es = F0.esize, sxe = es * F0.stride[0];
    const int32_t faxis = s_c.fold_axis, fold = s_c.fold;
    uint32_t bad = 0, nred = 0;
    unsigned long long lups = 0, naddr = 0, sreq = 0;
    // the warps take the item's batches of 32 slots as they finish the previous one
    for (;;) {
      int bi = 0;
      if (lane == 0) bi = atomicAdd(&s_batch, 1);
      const int64_t b0 = q0 + 32 * (int64_t)__shfl_sync(FULL, bi, 0);
      if (b0 >= q1) break;
      // ---- decode: lane l takes slot b0 + l
      const int64_t slot = b0 + lane;
      bool ok = false;
      RowSlot r;
      if (slot < q1) {
        int lv;
        int64_t loc;
        if (slot < s_c.rows_slot_end[0]) {
          lv = 0; loc = slot;
        } else if (slot < s_c.rows_slot_end[1]) {
          lv = 1; loc = slot - s_c.rows_slot_end[0];
        } else if (slot < s_c.rows_slot_end[2]) {
          lv = 2; loc = slot - s_c.rows_slot_end[1];
        } else {
          lv = 3; loc = slot - s_c.rows_slot_end[2];   // the representative block's rows
        }
        const uint32_t pq = fdiv((uint32_t)loc, s_c.fd_rows);
        const uint32_t t = (uint32_t)loc - pq * (uint32_t)s_c.rows_per_blk;
        const uint32_t R = (uint32_t)s_c.rows_R_lo[lv] + pq;
        const uint32_t gx = (uint32_t)s_c.g[0], gy = (uint32_t)s_c.g[1];
        const uint32_t bz = fdiv(R, s_c.fd_gy), by = R - bz * gy;
        const int64_t rb0 = (int64_t)R * gx, rb1 = rb0 + gx;
        int64_t ba, bb;
        bool in = true;
        if (lv == 0) {
          ba = max(s_c.s, rb0);
          bb = min(s_c.s + s_c.weff, rb1);
        } else if (lv == 3) {
          ba = s_c.rep;
          bb = s_c.rep + 1;
        } else if (lv == 1) {
          in = by != gy - 1;
          ba = max(s_c.y_lo, rb0);
          bb = min(s_c.y_hi, rb1);
        } else {
          // z set minus the y set: the y set takes [y_lo, y_hi) outside the last block row,
          // and z_hi <= y_hi (both are the wave shifted back, the z set by a whole slab), so
          // only the blocks before y_lo remain in the other rows
          ba = max(s_c.z_lo, rb0);
          bb = min(s_c.z_hi, rb1);
          if (by != gy - 1 && s_c.y_hi > s_c.y_lo) bb = min(bb, s_c.y_lo);
        }
        const uint32_t tz = fdiv(t, s_c.fd_b1), ty = t - tz * (uint32_t)s_c.B[1];
        int32_t y = (int32_t)(by * (uint32_t)s_c.B[1] + ty), z = (int32_t)(bz * (uint32_t)s_c.B[2] + tz);
        if (faxis == 1) y *= fold;
        if (faxis == 2) z *= fold;
        if (in && ba < bb && y < s_c.N[1] && z < s_c.N[2]) {
          ok = true;
          r.bxa = (uint32_t)(ba - rb0);
          r.bxb = (uint32_t)(bb - rb0);
          const int32_t xa = (int32_t)r.bxa * s_c.B[0], xb = min((int32_t)r.bxb * s_c.B[0], s_c.N[0]);
          const int kv = faxis == 1 ? min(fold, s_c.N[1] - y) : faxis == 2 ? min(fold, s_c.N[2] - z) : 1;
          const int64_t nx = xb - xa;
          // the block level only fills the block bitmaps: its counts come from enum_kernel
          if (lv != 3) {
            if (lv == 0 && s_g.first_wave) lups += (unsigned long long)(nx * kv);
            naddr += (unsigned long long)(nx * s_gad[lv == 0 ? 0 : 1][kv]);
          }
          r.el0 = es * (F0.stride[1] * y + F0.stride[2] * z);
          const int64_t ea = r.el0 + sxe * xa, eb = r.el0 + sxe * (xb - 1);
          r.lo = min(ea, eb);
          r.hi = max(ea, eb);
          r.t = t;
          r.y = y;
          r.z = z;
          r.lv = (uint8_t)lv;
          r.kv = (uint8_t)kv;
        }
      }
      const bool full = ok && r.kv == fold;
      const bool inner = full && Mu < Mfull && row_interior(s_c, r.lv, r.y, r.z, r.bxa, r.bxb, s_cov[1], s_cov[2]);
      const bool inner_y = full && !inner && Muz < Mfull && row_interior(s_c, r.lv, r.y, r.z, r.bxa, r.bxb, s_cov[4], 0);
      const bool blk = r.lv == 3;
      const int bsel = r.lv == 0 ? BM_W : r.lv == 1 ? BM_Y : r.lv == 2 ? BM_Z : BM_BL;
      // ---- loads of a full-fold row: its merged runs, [0, Mu) when it lies inside its level.
      // The lanes walk the same run at the same time (broadcast shared-memory reads); a lane
      // keeps its field's bitmap pointers, merges consecutive runs that end in one 64-bit
      // unit into one red.or, and stores a page flag only when the page range moves.  The
      // z-set ranges of a field whose z set is the wave moved by whole lines are clipped to
      // the wave's address range: the counts take only their sectors that meet the wave.
      if (__any_sync(FULL, full)) {
        const int me = !full ? 0 : inner ? Mu : inner_y ? Muz : Mfull;
        int kc = -1;
        unsigned long long *bm = nullptr;
        uint8_t *fl = nullptr;
        int64_t lim = 0, fb = 0;
        uint32_t cu = 0xffffffffu, pl0 = 1u, pl1 = 0u, zlo = 0u, zhi = 0xffffffffu;
        unsigned long long cb = 0ull;
        for (int e = 0; e < me; ++e) {
          const int k = s_iaf[e];
          if (k != kc) {
            if (cb) {
              atomicOr(bm + cu, cb);
              ++nred;
            }
            cu = 0xffffffffu;
            cb = 0ull;
            kc = k;
            bm = reinterpret_cast<unsigned long long *>(a.scratch + s_fbm[k][bsel]);
            fl = reinterpret_cast<uint8_t *>(a.scratch) + s_fpg[k][bsel];
            lim = s_flim[k][blk ? 0 : 1];
            fb = blk ? s_fblk[k] : 0;   // staged offsets are relative to the wave origin
            pl0 = 1u;
            pl1 = 0u;
            zlo = r.lv == 2 ? s_fzc[k][0] : 0u;
            zhi = r.lv == 2 ? s_fzc[k][1] : 0xffffffffu;
          }
          const int64_t bo = s_ibo[e] + fb;
          const int64_t a0 = r.lo + bo, a1 = r.hi + bo + (int64_t)s_iext[e];
          if (a0 < 0 || a1 >= lim) {
            ++bad;
            continue;
          }
          const uint32_t s0 = max((uint32_t)(a0 >> 5), zlo), s1 = min((uint32_t)(a1 >> 5), zhi);
          if (s0 > s1) continue;
          nred += put_range(bm, cu, cb, s0, s1);
          constexpr int kPageShiftSectors = kPageShiftBytes - 5;
          const uint32_t p0 = s0 >> kPageShiftSectors, p1 = s1 >> kPageShiftSectors;
          if (p0 < pl0 || p1 > pl1) {
            flag_pages(fl, p0, p1);
            pl0 = p0;
            pl1 = p1;
          }
        }
        if (cb) {
          atomicOr(bm + cu, cb);
          ++nred;
        }
      }
      // ---- loads of rows with fewer valid folded points than the fold (domain edge): the
      // raw folded loads, each issued iff a valid point needs it
      if (__any_sync(FULL, ok && !full)) {
        if (ok && !full) {
          for (int e = 0; e < L; ++e) {
            if ((int)s_kmin[e] >= r.kv) continue;
            const int k = s_af[e];
            const int64_t bo = s_boff[e] + s_forg[k][blk ? 0 : 1];
            const int64_t a0 = r.lo + bo, a1 = r.hi + bo;
            if (a0 < 0 || a1 >= s_flim[k][blk ? 0 : 1]) {
              ++bad;
              continue;
            }
            unsigned long long *const bm = reinterpret_cast<unsigned long long *>(a.scratch + s_fbm[k][bsel]);
            uint32_t cu = 0xffffffffu;
            unsigned long long cb = 0ull;
            nred += put_range(bm, cu, cb, (uint32_t)(a0 >> 5), (uint32_t)(a1 >> 5)) + (cb ? 1u : 0u);
            if (cb) atomicOr(bm + cu, cb);
            flag_pages(reinterpret_cast<uint8_t *>(a.scratch) + s_fpg[k][bsel], (uint32_t)(a0 >> kPageShiftBytes),
                       (uint32_t)(a1 >> kPageShiftBytes));
          }
        }
      }
      // ---- stores of wave and block rows; wave rows add their per-warp store sectors
      const bool st = ok && (r.lv == 0 || r.lv == 3) && S > 0;
      if (__any_sync(FULL, st)) {
        if (st) {
          const int sb = blk ? BM_BS : BM_WS;
          for (int j = L; j < L + S; ++j) {
            if ((int)s_kmin[j] >= r.kv) continue;
            const int k = s_af[j];
            const int64_t bo = s_boff[j] + s_forg[k][blk ? 0 : 1];
            const int64_t a0 = r.lo + bo, a1 = r.hi + bo;
            if (a0 < 0 || a1 >= s_flim[k][blk ? 0 : 1]) {
              ++bad;
              continue;
            }
            unsigned long long *const bm = reinterpret_cast<unsigned long long *>(a.scratch + s_fbm[k][sb]);
            uint32_t cu = 0xffffffffu;
            unsigned long long cb = 0ull;
            nred += put_range(bm, cu, cb, (uint32_t)(a0 >> 5), (uint32_t)(a1 >> 5)) + (cb ? 1u : 0u);
            if (cb) atomicOr(bm + cu, cb);
            flag_pages(reinterpret_cast<uint8_t *>(a.scratch) + s_fpg[k][sb], (uint32_t)(a0 >> kPageShiftBytes),
                       (uint32_t)(a1 >> kPageShiftBytes));
            if (!blk) {
              // the count depends on the row start only modulo 32 bytes, on t only through
              // t * B0 modulo 32 (where the row's first warp ends) and on the block run, so
              // rows that agree on those reuse this thread's previous count
              const int64_t A0 = r.el0 + bo;
              const unsigned long long key = (unsigned long long)(A0 & 31) |
                                             ((unsigned long long)((r.t * (uint32_t)s_c.B[0]) & 31u) << 5) |
                                             ((unsigned long long)r.bxa << 10) | ((unsigned long long)r.bxb << 37);
              if (s_memo_key[threadIdx.x] != key) {
                s_memo_val[threadIdx.x] =
                    (uint32_t)row_store_sectors(A0, sxe, s_c.B[0], s_c.N[0], s_c.full_end, r.t, r.bxa, r.bxb);
                s_memo_key[threadIdx.x] = key;
              }
              sreq += s_memo_val[threadIdx.x];
            }
          }
        }
      }
    }

    // the item's counts: per warp, then once per CTA
    bad = __reduce_add_sync(FULL, bad);
    nred = __reduce_add_sync(FULL, nred);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      lups += __shfl_xor_sync(FULL, lups, o);
      naddr += __shfl_xor_sync(FULL, naddr, o);
      sreq += __shfl_xor_sync(FULL, sreq, o);
    }
    if (lane == 0) {
      s_acc[warp][0] = lups;
      s_acc[warp][1] = naddr;
      s_acc[warp][2] = sreq;
      s_acc[warp][3] = bad;
      s_acc[warp][4] = nred;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      const int k = threadIdx.x;
      unsigned long long v = 0;
      for (int w = 0; w < kRowsThreads / 32; ++w) v += s_acc[w][k];
      unsigned long long *const c = (unsigned long long *)(a.counters + (int64_t)s_g.cfg * N_COUNTERS);
      const int dst = k == 0 ? C_LUPS_WAVE : k == 1 ? C_ADDR : k == 2 ? C_W_SREQ : k == 3 ? C_OVERFLOW : C_RED;
      if (v) atomicAdd(c + dst, v);
    }
  }
}

__constant__ int kCountDst[12] = {C_BLK_LS, C_BLK_LL, C_BLK_SS, C_BLK_SL, C_W_LS, C_W_LL,
                                  C_Y_LINES, C_Z_LINES, C_OV_Y, C_OV_Z, C_W_SS, C_W_SL};

// Lines of four consecutive bitmap words: bit i of a word <-> sector lo + i with lo a
// multiple of 32, so each nibble is one 128 B line; a word's nibbles are reduced to one bit
// each (bit 4k) and the four words' bits interleaved into one word for a single popcount.
__device__ __forceinline__ uint32_t line_bits(uint32_t x) {
  uint32_t t = x | (x >> 1);
  t |= t >> 2;
  return t & 0x11111111u;
}
__device__ __forceinline__ uint32_t lines4(const uint4 &v) {
  return __popc(line_bits(v.x) | (line_bits(v.y) << 1) | (line_bits(v.z) << 2) | (line_bits(v.w) << 3));
}

__device__ __forceinline__ bool nz(const uint4 &v) { return (v.x | v.y | v.z | v.w) != 0u; }

__device__ __forceinline__ void tally_sectors_lines(uint32_t &sec, uint32_t &lin, const uint4 &v) {
  sec += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
  lin += lines4(v);
}

// zs: the z set is the wave moved by whole lines (its bitmap holds only the sectors that can
// meet the wave), so its lines are the wave's
__device__ __forceinline__ void tally_wave(uint32_t acc[12], const uint4 &w, const uint4 &y, const uint4 &z, bool zs) {
  tally_sectors_lines(acc[4], acc[5], w);
  acc[6] += lines4(y);
  acc[7] += lines4(zs ? w : z);
  acc[8] += __popc(w.x & y.x) + __popc(w.y & y.y) + __popc(w.z & y.z) + __popc(w.w & y.w);
  acc[9] += __popc(w.x & z.x & ~y.x) + __popc(w.y & z.y & ~y.y) + __popc(w.z & z.z & ~y.z) + __popc(w.w & z.w & ~y.w);
}

// Read-and-clear counting of the bitmaps of one pass.  Counting unit = (field, chunk of the
// words of its block bitmaps or of its wave bitmaps); work item = consecutive units of one
// candidate (at most kCountMaxPages pages, kCountItemUnits units), so that a CTA places the
// many small block parts of a large batch together.  Chunks are cut into pages of
// kPageWords words; for a field the row walk filled, only the pages it flagged are read
// (and their flags cleared), otherwise every page.  One warp takes one page at a time: each
// lane loads two 16-byte positions of every bitmap of the part that has the page flagged
// (all loads in flight together), tallies sectors, lines and overlaps, and clears the
// non-zero positions, so the bitmaps are left zeroed for the next step.
__device__ __forceinline__ uint4 ld_v4(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(kCountThreads, 4) count_kernel(CountArgs a) {
  __shared__ long long s_item[2];   // this item and the next one (fetched while this one is counted)
  __shared__ uint32_t s_red[kCountThreads / 32][13];
  __shared__ uint32_t s_pl[kCountMaxPages];        // pages to read: bitmap mask | unit << 4 | page << 12
  __shared__ int s_npl;
  // the item's units: bitmap positions (16-byte units), their flags, first item page
  __shared__ uint4 *s_ubp[kCountItemUnits][4];
  __shared__ uint8_t *s_ufl[kCountItemUnits][4];
  __shared__ int64_t s_uq0[kCountItemUnits];       // first 16-byte position of the chunk
  __shared__ int64_t s_uq1[kCountItemUnits];       // end position of the chunk
  __shared__ int32_t s_uw[kCountItemUnits];        // words of the chunk
  __shared__ int32_t s_upg[kCountItemUnits + 1];   // first item page of each unit, then the end
  __shared__ uint8_t s_unb[kCountItemUnits];       // bitmaps of the part (2 block, 4 wave)
  __shared__ uint8_t s_uzs[kCountItemUnits];       // the field's z set is its wave moved by whole lines
  __shared__ int s_cfg;
  const uint32_t lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    s_item[0] = a.citem_lo + (long long)atomicAdd(a.grab, 1ull);
    s_npl = 0;
  }
  __syncthreads();
  for (int par = 0;; par ^= 1) {
    const int64_t item = s_item[par];
    if (item >= a.citem_hi) break;
    long long nxt = 0;
    if (threadIdx.x == 0) nxt = a.citem_lo + (long long)atomicAdd(a.grab, 1ull);
    const int u0 = a.item_unit[item], nu = a.item_unit[item + 1] - u0;
    // ---- a thread per unit: where its chunk's bitmaps and flags lie
    if (threadIdx.x < nu) {
      const int t = threadIdx.x;
      const int cf = a.units[2 * (u0 + t)];
      const int64_t k = a.units[2 * (u0 + t) + 1];
      const DField &F = a.fld[cf];
      const bool paged = F.pg >= 0;
      const int64_t cw = paged ? kPagedChunkWords : a.chunk_words;
      const int64_t kb = (F.words[0] + cw - 1) / cw;
      const bool blk = k < kb;
      const int64_t c0 = (blk ? k : k - kb) * cw;
      const int64_t c1 = min(c0 + cw, blk ? F.words[0] : F.words[1]);
      const int NB = blk ? 2 : 4;
      const int b0 = blk ? BM_BL : BM_W;   // BL, BS | W, Y, Z, WS are consecutive bitmap indices
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const bool has = b < NB && F.bm[b0 + b] >= 0;
        s_ubp[t][b] = has ? reinterpret_cast<uint4 *>(a.scratch + F.bm[b0 + b]) : nullptr;
        s_ufl[t][b] = has && paged ? reinterpret_cast<uint8_t *>(a.scratch + F.pg) +
                                         page_flag_off(b0 + b, F.words[0], F.words[1]) + c0 / kPageWords
                                   : nullptr;
      }
      s_uq0[t] = c0 / 4;
      s_uq1[t] = c1 / 4;
      s_uw[t] = (int32_t)(c1 - c0);
      s_upg[t + 1] = (int32_t)((c1 - c0 + kPageWords - 1) / kPageWords);
      s_unb[t] = (uint8_t)NB;
      s_uzs[t] = (uint8_t)(F.zshift != 0);
      if (t == 0) {
        s_cfg = F.cfg;
        s_upg[0] = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int t = 0; t < nu; ++t) s_upg[t + 1] += s_upg[t];
    __syncthreads();
    const int npg = s_upg[nu];
    uint32_t rd = 0;   // bitmap bytes of the pages this thread lists
    // ---- a thread per page: which bitmaps to read (flags cleared in device memory as they
    // are taken); pages with none are dropped
    for (int j = threadIdx.x; j < npg; j += kCountThreads) {
      int lo = 0, hi = nu - 1;   // the unit holding page j: s_upg[u] <= j < s_upg[u + 1]
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_upg[mid] <= j) lo = mid;
        else hi = mid - 1;
      }
      const int u = lo, lp = j - s_upg[u];
      const uint32_t pbytes = 4u * (uint32_t)min(kPageWords, s_uw[u] - lp * kPageWords);
      uint32_t m = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (s_ubp[u][b] == nullptr) continue;
        bool on = true;
        uint8_t *const fl = s_ufl[u][b];
        if (fl != nullptr) {
          const uint8_t v = fl[lp];
          if (v) fl[lp] = 0;
          on = v != 0;
        }
        if (on) {
          m |= 1u << b;
          rd += pbytes;
        }
      }
      if (m) s_pl[atomicAdd(&s_npl, 1)] = m | ((uint32_t)u << 4) | ((uint32_t)lp << 12);
    }
    __syncthreads();
    uint32_t acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int npl = s_npl;
    for (int i = warp; i < npl; i += kCountThreads / 32) {
      const uint32_t ent = s_pl[i];
      const uint32_t m = ent & 15u;
      const int u = (int)((ent >> 4) & 255u), lp = (int)(ent >> 12);
      const bool blk = s_unb[u] == 2, zs = s_uzs[u] != 0;
      uint4 *const *const bp = s_ubp[u];
      const int64_t q0 = s_uq0[u] + (int64_t)lp * (kPageWords / 4);           // first position of the page
      const int np = (int)min((int64_t)(kPageWords / 4), s_uq1[u] - q0);      // its positions (<= 64)
      uint4 v[4][2];
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = (int)lane + 32 * h;
          v[b][h] = ((m >> b) & 1u) && r < np ? ld_v4(bp[b] + q0 + r) : zero;
        }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t q = q0 + (int)lane + 32 * h;
        if (blk) {
          if (nz(v[0][h])) {
            tally_sectors_lines(acc[0], acc[1], v[0][h]);
            bp[0][q] = zero;
          }
          if (nz(v[1][h])) {
            tally_sectors_lines(acc[2], acc[3], v[1][h]);
            bp[1][q] = zero;
          }
        } else {
          if (nz(v[0][h]) | nz(v[1][h]) | nz(v[2][h])) {
            tally_wave(acc, v[0][h], v[1][h], v[2][h], zs);
#pragma unroll
            for (int b = 0; b < 3; ++b)
              if (nz(v[b][h])) bp[b][q] = zero;
          }
          if (nz(v[3][h])) {
            tally_sectors_lines(acc[10], acc[11], v[3][h]);
            bp[3][q] = zero;
          }
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < 12; ++kk) {
      uint32_t v = __reduce_add_sync(FULL, acc[kk]);
      if (lane == 0) s_red[warp][kk] = v;
    }
    {
      const uint32_t v = __reduce_add_sync(FULL, rd);
      if (lane == 0) s_red[warp][12] = v;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
      unsigned long long t = 0;
      for (int wi = 0; wi < kCountThreads / 32; ++wi) t += s_red[wi][threadIdx.x];
      const int dst = threadIdx.x < 12 ? kCountDst[threadIdx.x] : C_CBYTES;
      if (t) atomicAdd((unsigned long long *)(a.counters + (int64_t)s_cfg * N_COUNTERS + dst), t);
    }
    if (threadIdx.x == 0) {
      s_item[par ^ 1] = nxt;
      s_npl = 0;
    }
    __syncthreads();
  }
}

// R(O) = a * exp(-b * exp(-c * O)), Sec. 4.5
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
// Block (x, y) compares its kRankTile candidates with the y-th tile of kRankTile keys of
// their segments and adds the partial counts to rank[i] (zeroed before); the scatter
// kernel then places every candidate.
constexpr int kRankTile = 256;

__device__ __forceinline__ int rank_seg_of(const RankArgs &a, int64_t x) {
  int lo = 0, hi = a.n_seg;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.seg[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The rank keys as integers in the same order as the doubles they stand for (NaN
// counts as +inf, -0 as +0): a sign-magnitude bit pattern maps monotonically to two's
// complement by flipping the magnitude bits of negative values.  Integer compares keep
// the ranking off the fp64 pipe.
__device__ __forceinline__ long long rank_ord_of(double v) {
  long long b = isnan(v) ? 0x7ff0000000000000ll : __double_as_longlong(v);
  if ((b << 1) == 0) b = 0;
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

__global__ void __launch_bounds__(kRankTile) rank_count_kernel(RankArgs a) {
  __shared__ long long s_key[kRankTile];
  const int64_t i_first = (int64_t)blockIdx.x * kRankTile;
  if (i_first >= a.n) return;
  const int64_t i = i_first + threadIdx.x;
  const int64_t i_last = min((int64_t)a.n, i_first + kRankTile) - 1;
  const int64_t j_lo = a.seg[rank_seg_of(a, i_first)], j_hi = a.seg[rank_seg_of(a, i_last) + 1];
  const int64_t t0 = j_lo + (int64_t)blockIdx.y * kRankTile;
  if (t0 >= j_hi) return;
  if (t0 + threadIdx.x < j_hi) s_key[threadIdx.x] = rank_ord_of(a.keys[t0 + threadIdx.x]);
  __syncthreads();
  if (i >= a.n) return;
  const int my_seg = rank_seg_of(a, i);
  const int64_t a0 = max(t0, (int64_t)a.seg[my_seg]), a1 = min(t0 + kRankTile, (int64_t)a.seg[my_seg + 1]);
  const long long ki = rank_ord_of(a.keys[i]);
  int cnt = 0;
  for (int64_t j = a0; j < a1; ++j) {
    const long long kj = s_key[j - t0];
    cnt += (kj < ki) || (kj == ki && j < i);
  }
  if (cnt) atomicAdd(a.rank + i, cnt);
}

__global__ void rank_scatter_kernel(RankArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  a.order[a.seg[rank_seg_of(a, i)] + a.rank[i]] = (int32_t)i;
}

// Rank keys of given results (used when ranking results that came from the host).
__global__ void keys_kernel(const ws_result *__restrict__ res, int n, double *__restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = rank_key_dev(res[i].t_pred);
}

// ---- launchers ---------------------------------------------------------------------
size_t enum_dyn_smem(int iv_cap) { return (size_t)((iv_cap + 15) & ~15) * (8 + 4 + 1); }

// Raises the dynamic shared-memory limit of the enumeration and row kernels (once per
// device and size).
static cudaError_t enum_allow_smem(size_t dyn) {
  static std::mutex mu;
  static size_t allowed[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (dyn <= allowed[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(enum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e == cudaSuccess) allowed[dev] = dyn;
  return e;
}

cudaError_t launch_enum(const EnumArgs &args, int grid, int threads, cudaStream_t st) {
  const size_t dyn = enum_dyn_smem(args.iv_cap);
  cudaError_t e = enum_allow_smem(dyn);
  if (e != cudaSuccess) return e;
  enum_kernel<<<grid, threads, dyn, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_rows(const EnumArgs &args, int grid, cudaStream_t st) {
  const size_t dyn = enum_dyn_smem(args.iv_cap);
  cudaError_t e = enum_allow_smem(dyn);
  if (e != cudaSuccess) return e;
  rows_kernel<<<grid, kRowsThreads, dyn, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_count(const CountArgs &args, int grid, cudaStream_t st) {
  count_kernel<<<grid, kCountThreads, 0, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_model(const ModelArgs &args, cudaStream_t st) {
  if (args.n <= 0) return cudaSuccess;
  // one warp per CTA: the model is fp64 (1/64 of the fp32 rate on this part), so the
  // candidates are spread over as many SMs' fp64 pipes as possible
  model_kernel<<<(args.n + 31) / 32, 32, 0, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_rank(const RankArgs &args, cudaStream_t st) {
  if (args.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(args.rank, 0, (size_t)args.n * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  const unsigned tiles = (unsigned)((args.n + kRankTile - 1) / kRankTile);
  rank_count_kernel<<<dim3(tiles, tiles), kRankTile, 0, st>>>(args);
  rank_scatter_kernel<<<tiles, kRankTile, 0, st>>>(args);
  return cudaGetLastError();
}
cudaError_t launch_keys(const ws_result *res, int n, double *keys, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  keys_kernel<<<(n + 255) / 256, 256, 0, st>>>(res, n, keys);
  return cudaGetLastError();
}
cudaError_t enum_occupancy(int threads, int iv_cap, int *blocks_per_sm) {
  const size_t dyn = enum_dyn_smem(iv_cap);
  cudaError_t e = enum_allow_smem(dyn);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, enum_kernel, threads, dyn);
}
cudaError_t rows_occupancy(int iv_cap, int *blocks_per_sm) {
  const size_t dyn = enum_dyn_smem(iv_cap);
  cudaError_t e = enum_allow_smem(dyn);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, rows_kernel, kRowsThreads, dyn);
}
cudaError_t count_occupancy(int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, count_kernel, kCountThreads, 0);
}

}  // namespace ws
