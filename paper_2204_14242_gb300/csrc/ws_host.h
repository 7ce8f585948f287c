// Host-side objects of libwarpspeed (context, arena, plan), shared by ws_plan.cpp
// and ws_server.cpp.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "warpspeed.h"
#include "ws_internal.h"

namespace ws {

// First-fit allocator over one device buffer; offsets are 256-byte aligned.
struct Arena {
  char *base;
  size_t size;
  size_t in_use = 0, peak = 0;
  std::map<size_t, size_t> free_, used_;
  std::mutex mu;
  Arena(char *b, size_t n);
  int64_t alloc(size_t bytes);  // offset, or -1
  void release(int64_t off);
  size_t largest_free();
  size_t used();
};

// Blocks of at least kHostBlockMin bytes for large host arrays, from a process-wide
// cache (up to 1 GiB of returned blocks is kept), so that creating plan after plan does
// not fault in fresh pages each time.
constexpr size_t kHostBlockMin = (size_t)1 << 20;
void *host_block_alloc(size_t bytes);
void host_block_free(void *p);

// Allocator whose resize() leaves trivially constructible elements uninitialised, so
// that large descriptor arrays are first touched by the threads that fill them; large
// arrays come from the block cache.
template <class T>
struct DefaultInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = DefaultInitAlloc<U>;
  };
  DefaultInitAlloc() = default;
  template <class U>
  DefaultInitAlloc(const DefaultInitAlloc<U> &) {}
  T *allocate(size_t n) {
    if (n * sizeof(T) >= kHostBlockMin) return static_cast<T *>(host_block_alloc(n * sizeof(T)));
    return std::allocator<T>::allocate(n);
  }
  void deallocate(T *p, size_t n) {
    if (n * sizeof(T) >= kHostBlockMin) host_block_free(p);
    else std::allocator<T>::deallocate(p, n);
  }
  template <class U>
  void construct(U *p) {
    ::new ((void *)p) U;
  }
  template <class U, class... Args>
  void construct(U *p, Args &&...args) {
    ::new ((void *)p) U(std::forward<Args>(args)...);
  }
};
template <class T>
using HostVec = std::vector<T, DefaultInitAlloc<T>>;

// Page-locked host blocks for the arrays a plan uploads (when a CUDA device is present;
// plain memory otherwise), from their own process-wide cache.  Copies from them are
// asynchronous: the arrays live in the plan until it is destroyed.
void *pinned_block_alloc(size_t bytes);
void pinned_block_free(void *p);

template <class T>
struct PinnedAlloc : DefaultInitAlloc<T> {
  template <class U>
  struct rebind {
    using other = PinnedAlloc<U>;
  };
  PinnedAlloc() = default;
  template <class U>
  PinnedAlloc(const PinnedAlloc<U> &) {}
  T *allocate(size_t n) { return static_cast<T *>(pinned_block_alloc(n * sizeof(T))); }
  void deallocate(T *p, size_t) { pinned_block_free(p); }
};
template <class T>
using PinVec = std::vector<T, PinnedAlloc<T>>;

void set_error(const std::string &s);
const char *last_error();

// Resources the library creates (for ws_resource_counts_get): device allocations,
// page-locked host allocations, streams and events.
enum ResourceKind { RES_DEVICE_ALLOC, RES_PINNED_ALLOC, RES_STREAM, RES_EVENT, N_RES };
void count_resource(ResourceKind k);

// While alive on a thread, the page-locked block allocator of that thread never calls
// cudaHostAlloc: a request the cache cannot serve gets plain (pageable) memory, which is
// freed, not cached, when released.
struct NoPinnedScope {
  NoPinnedScope();
  ~NoPinnedScope();
  bool prev;
};

}  // namespace ws

struct ws_ctx {
  int device = 0;
  int sm_count = 0;
  int l2_bytes = 0;
  bool owns_arena = false;
  ws::Arena *arena = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  cudaStream_t upload_stream = nullptr;   // descriptor uploads of pipelined one-shot estimates
  cudaStream_t lane_stream = nullptr;     // second lane of a pipelined estimate's parts
  // Scratch kept between one-shot estimates (ws_estimate_batch): the counting kernel leaves
  // it zeroed, so a later estimate needs no memset.  Held while `oneshot_mu` is; given back
  // to the arena when a plan or server of the context needs the room.
  std::mutex oneshot_mu;
  int64_t oneshot_off = -1;
  size_t oneshot_bytes = 0;
  bool oneshot_dirty = false;   // not known to be zero (new, or an execution failed)
  // Plans of this context create no readiness event (their uploads and launches share one
  // stream; used by the entry point that may create no CUDA resources).
  bool no_events = false;
};

struct ws_plan {
  ws_ctx *ctx = nullptr;
  int n_cfg = 0, n_seg = 1;
  ws_hw hw;
  ws::DHw dhw;
  ws_tuning tune;
  ws::PinVec<ws::DField> hfld;
  ws::PinVec<ws::DGroup> hgrp;
  std::vector<char> grp_iv_ok;   // group allows the interval walk (used unless tune.walk asks otherwise)
  std::vector<char> grp_rows_ok; // group allows the row walk of levels 1-3
  std::vector<int64_t> grp_slots;        // row slots of the group's candidate
  std::vector<ws::WarpClasses> grp_classes;  // block warp classes per group (used with the row walk)
  std::vector<int64_t> grp_winstr_rows;  // modelled (warp, instruction) pairs of levels 1-3
  // work-item sizes set by layout(): row slots per row-walk item (256, 512 or 1024),
  // (warp, instruction) pairs per representative-block item, counting units per counting
  // item.  plain_layout selects the finest ones (256, kPlainBlockPairs, 1) for the plain
  // form, whose launches serve one candidate at a time.
  bool plain_layout = false;
  int32_t rows_chunk = 256;
  int32_t block_pairs = 128;
  int32_t count_pack = 1;
  int32_t chunk_rows() const { return rows_chunk; }
  std::vector<int32_t> cfg_grp_begin;
  ws::HostVec<int64_t> need_words;
  std::vector<int32_t> cfg_cf_begin;
  std::vector<ws::DPass> passes;
  int64_t scratch_words = 0;
  size_t scratch_bytes = 0;
  int64_t item_begin_end = 0, ritem_begin_end = 0, citem_begin_end = 0;
  size_t grab_bytes = 0, counters_bytes = 0;
  // uploaded arrays that the plan owns until it is destroyed (their copies are asynchronous)
  ws::PinVec<ws::DCfg> up_cfg;
  ws::PinVec<ws::DAcc> up_acc;
  ws::PinVec<ws::DIv> up_iv;
  int64_t upload_bytes = 0;
  float ms_create_host = 0, ms_create_device = 0;   // wall times of the creation (host part, device part)
  int64_t d_grp = -1;
  int32_t iv_cap = 0;  // most merged load intervals of an interval-walk group (dynamic shared memory)
  // owner of every work item (enumeration and row-walk items: field group; counting
  // items: (candidate, field)), filled by layout(), uploaded with the fields
  ws::PinVec<int32_t> own;              // [enumeration items | row-walk items | counting items]
  int64_t d_own = -1;
  size_t d_own_bytes = 0;
  int64_t d_cfg = -1, d_fld = -1, d_acc = -1, d_iv = -1, d_seg = -1, d_counters = -1, d_results = -1, d_keys = -1,
          d_order = -1, d_rank = -1, d_scratch = -1;
  std::vector<int64_t> allocs;
  bool ext_scratch = false;  // scratch lent by a server pool (kept zeroed by the counting kernel)
  cudaGraphExec_t graph_exec = nullptr;

  void *dev(int64_t off) const;
  int64_t take(size_t bytes);
  void release_all();
  void layout();
  int upload_fields(cudaStream_t st);
  int grid_for(int threads, int64_t items, bool counting) const;
  int grid_rows(int64_t items) const;
  int bank_shift() const;
  int enqueue(cudaStream_t st, std::vector<cudaEvent_t> *ev, ws_profile *prof);
  // Recorded after the descriptor uploads: launches on any stream wait for it (a graph
  // capture waits on the host instead, once).
  cudaEvent_t ready = nullptr;
  int wait_ready(cudaStream_t st);
  int run_plain(cudaStream_t st);
  int run_plain_launches(cudaStream_t st);
  int execute(int mode, cudaStream_t st);
};

namespace ws {
using Plan = ::ws_plan;

int plan_requirements(const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld, const ws_access *acc,
                      int n_acc, const ws_hw *hw, size_t *desc_bytes, size_t *scratch_bytes,
                      size_t *max_field_bytes);
// ext_scratch value of plan_create_impl: use (and grow) the context's kept one-shot scratch;
// the caller holds ctx->oneshot_mu.
constexpr int64_t kCtxScratch = -2;
// Gives the context's kept one-shot scratch back to the arena unless an estimate holds it.
void ctx_reclaim(ws_ctx *ctx);
int plan_create_impl(ws_ctx *ctx, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                     const ws_access *acc, int n_acc, const ws_hw *hw, const int32_t *seg_begin, int n_seg,
                     const ws_tuning *tuning, size_t scratch_cap, ws_plan **out, cudaStream_t upload,
                     int64_t ext_scratch, size_t ext_scratch_bytes);
void tuning_cache_lookup(ws_ctx *ctx, int n_cfg, ws_tuning *t);
void tuning_cache_store(ws_ctx *ctx, int n_cfg, const ws_tuning &t);
}  // namespace ws
