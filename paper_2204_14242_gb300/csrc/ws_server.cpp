// Continuous-batching estimation server.
//
// Requests (one candidate list each) are queued by ws_server_submit.  A worker thread
// admits queued requests into a device step whenever a stream slot and enough scratch
// are free, so requests that arrive while others are running on the GPU start at once
// and overlap with them on the device.  Each step is one batched launch sequence
// (enumeration, counting, model, per-request ranking) over all candidates it admitted;
// its descriptors stay resident in device memory until the step retires.  Scratch
// bitmaps come from a pool that is zeroed once: the counting kernel clears every word
// it reads, so a finished step hands back zeroed scratch and no step needs a memset.
// Completion is signalled by a host callback on the step's stream; ws_server_poll
// waits with a bounded timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ws_host.h"
#include "ws_internal.h"

namespace {

struct Request {
  uint64_t id = 0;
  std::vector<ws_config> cfgs;
  std::vector<ws_field> fld;
  std::vector<ws_access> acc;
  size_t scratch_bytes = 0;    // one-pass scratch of the whole request
  size_t max_field_bytes = 0;  // the least scratch it can run with (several passes)
  int status = WS_EAGAIN;  // WS_EAGAIN until finished
  bool done = false;
  std::vector<ws_result> results;
  std::vector<int32_t> order;
};

struct Slot {
  cudaStream_t stream = nullptr;
  ws_result *h_res = nullptr;  // pinned
  int32_t *h_ord = nullptr;    // pinned
  size_t cap = 0;
  bool busy = false;
};

struct Step {
  ws_plan *plan = nullptr;
  std::vector<Request *> reqs;
  std::vector<int32_t> offsets;  // candidate offset of each request in the step
  int slot = -1;
  int64_t pool_off = -1;
  bool finished = false;          // set by the stream callback
  int status = WS_OK;
};

}  // namespace

struct ws_server {
  ws_ctx *ctx = nullptr;
  ws_hw hw;
  ws_server_opts opts;
  int64_t pool_off = -1;         // pool allocation in the context arena
  ws::Arena *pool = nullptr;     // scratch pool (offsets relative to pool_off)
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::map<uint64_t, Request *> reqs;
  std::vector<Step *> inflight;
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  bool paused = false;     // admit no new steps (ws_server_pause)
  uint64_t next_id = 1;
  ws_server_stats stats;
};

namespace {

void CUDART_CB step_done_cb(void *p) {
  auto *pair = static_cast<std::pair<ws_server *, Step *> *>(p);
  ws_server *s = pair->first;
  {
    std::lock_guard<std::mutex> g(s->mu);
    pair->second->finished = true;
  }
  s->cv_work.notify_all();
  delete pair;
}

bool ensure_slot_capacity(Slot &sl, size_t n) {
  if (sl.cap >= n) return true;
  if (sl.h_res) cudaFreeHost(sl.h_res);
  if (sl.h_ord) cudaFreeHost(sl.h_ord);
  sl.h_res = nullptr;
  sl.h_ord = nullptr;
  size_t c = std::max<size_t>(n, 1024);
  if (cudaHostAlloc((void **)&sl.h_res, c * sizeof(ws_result), cudaHostAllocDefault) != cudaSuccess) return false;
  ws::count_resource(ws::RES_PINNED_ALLOC);
  if (cudaHostAlloc((void **)&sl.h_ord, c * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) return false;
  ws::count_resource(ws::RES_PINNED_ALLOC);
  sl.cap = c;
  return true;
}

// Builds and launches one step from the head of the queue.  Called with the lock held;
// drops it while the plan is compiled and launched (the stream callbacks of other
// steps take the lock).  Returns true if a step was launched.
bool admit(ws_server *s, std::unique_lock<std::mutex> &lk) {
  if (s->queue.empty()) return false;
  int slot = -1;
  for (size_t k = 0; k < s->slots.size(); ++k)
    if (!s->slots[k].busy) {
      slot = (int)k;
      break;
    }
  if (slot < 0) return false;
  // take requests from the head while they fit the pool (one pass each) and the step
  // size; a head request larger than the free scratch runs alone in several passes
  // once enough of the pool is free (or nothing else is running)
  std::vector<Request *> take;
  size_t bytes = 0;
  int ncfg = 0;
  size_t room = s->pool->largest_free() & ~(size_t)255;
  for (Request *r : s->queue) {
    if (!take.empty() && ncfg + (int)r->cfgs.size() > s->opts.max_step_cfgs) break;
    size_t b = (r->scratch_bytes + 255) & ~(size_t)255;
    if (bytes + b > room) {
      if (take.empty() && room >= r->max_field_bytes &&
          (s->inflight.empty() || room >= std::min(b, s->pool->size / 2))) {
        take.push_back(r);
        bytes = room;
        ncfg += (int)r->cfgs.size();
      }
      break;
    }
    take.push_back(r);
    bytes += b;
    ncfg += (int)r->cfgs.size();
  }
  if (take.empty()) return false;
  int64_t off = s->pool->alloc(std::max<size_t>(bytes, 256));
  if (off < 0) return false;
  s->queue.erase(s->queue.begin(), s->queue.begin() + take.size());

  // concatenate the requests into one plan, one ranking segment per request
  std::vector<ws_config> cfgs;
  std::vector<ws_field> fld;
  std::vector<ws_access> acc;
  std::vector<int32_t> seg = {0};
  Step *st = new Step();
  st->reqs = take;
  st->slot = slot;
  st->pool_off = off;
  for (Request *r : take) {
    st->offsets.push_back((int32_t)cfgs.size());
    const int64_t f0 = (int64_t)fld.size(), a0 = (int64_t)acc.size();
    for (ws_field f : r->fld) {
      f.access_off += a0;
      fld.push_back(f);
    }
    acc.insert(acc.end(), r->acc.begin(), r->acc.end());
    for (ws_config c : r->cfgs) {
      c.field_off += f0;
      cfgs.push_back(c);
    }
    seg.push_back((int32_t)cfgs.size());
  }
  Slot &sl = s->slots[slot];
  sl.busy = true;
  lk.unlock();
  int rc = ws::plan_create_impl(s->ctx, cfgs.data(), (int)cfgs.size(), fld.data(), (int)fld.size(), acc.data(),
                                (int)acc.size(), &s->hw, seg.data(), (int)take.size(), nullptr, 0, &st->plan,
                                sl.stream, s->pool_off + off, std::max<size_t>(bytes, 256));
  if (rc == WS_OK && sl.cap < cfgs.size()) rc = WS_ENOMEM;
  if (rc == WS_OK) rc = st->plan->execute(WS_MODE_DIRECT, sl.stream);
  if (rc == WS_OK && !cfgs.empty()) {
    if (cudaMemcpyAsync(sl.h_res, st->plan->dev(st->plan->d_results), cfgs.size() * sizeof(ws_result),
                        cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaMemcpyAsync(sl.h_ord, st->plan->dev(st->plan->d_order), cfgs.size() * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
      rc = WS_ECUDA;
  }
  if (rc == WS_OK) {
    auto *arg = new std::pair<ws_server *, Step *>(s, st);
    if (cudaLaunchHostFunc(sl.stream, step_done_cb, arg) != cudaSuccess) {
      delete arg;
      rc = WS_ECUDA;
    }
  }
  lk.lock();
  st->status = rc;
  if (rc != WS_OK) st->finished = true;  // retired (with the error) by the worker
  s->inflight.push_back(st);
  s->stats.steps += 1;
  return true;
}

// Retires finished steps.  Called with the lock held.  Returns the steps retired.
int retire(ws_server *s) {
  int n_retired = 0;
  for (size_t k = 0; k < s->inflight.size();) {
    Step *st = s->inflight[k];
    if (!st->finished) {
      ++k;
      continue;
    }
    Slot &sl = s->slots[st->slot];
    cudaError_t e = cudaStreamSynchronize(sl.stream);  // already drained; surfaces errors
    int rc = st->status != WS_OK ? st->status : (e == cudaSuccess ? WS_OK : WS_ECUDA);
    for (size_t r = 0; r < st->reqs.size(); ++r) {
      Request *q = st->reqs[r];
      const int32_t o = st->offsets[r], n = (int32_t)q->cfgs.size();
      if (rc == WS_OK) {
        q->results.assign(sl.h_res + o, sl.h_res + o + n);
        q->order.resize(n);
        for (int32_t i = 0; i < n; ++i) q->order[i] = sl.h_ord[o + i] - o;
      }
      q->status = rc;
      q->done = true;
      s->stats.completed += 1;
      s->stats.configs_done += n;
    }
    if (rc != WS_OK && st->plan) {
      // a failed step may leave bits set: clear its scratch before it is reused
      cudaMemsetAsync(s->ctx->arena->base + s->pool_off + st->pool_off, 0, st->plan->scratch_bytes, sl.stream);
      cudaStreamSynchronize(sl.stream);
    }
    if (st->plan) ws_plan_destroy(st->plan);
    s->pool->release(st->pool_off);
    sl.busy = false;
    delete st;
    s->inflight.erase(s->inflight.begin() + k);
    ++n_retired;
  }
  s->stats.bytes_in_use = (int64_t)s->pool->used();
  s->stats.peak_bytes = (int64_t)s->pool->peak;
  return n_retired;
}

void worker_main(ws_server *s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // wake the pollers whenever requests completed, including the last step of a burst
    // (the server then goes idle and nothing else would wake them before their deadline)
    if (retire(s) > 0) s->cv_done.notify_all();
    bool launched = false;
    if (!s->stop && !s->paused)
      while (admit(s, lk)) launched = true;
    if (launched) continue;
    if (s->stop) {
      if (s->inflight.empty()) break;
    }
    s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
  }
  // cancel what never ran
  for (Request *q : s->queue) {
    q->status = WS_ECANCELED;
    q->done = true;
  }
  s->queue.clear();
  s->cv_done.notify_all();
}

}  // namespace

extern "C" int ws_server_create(ws_ctx *ctx, const ws_server_opts *opts, const ws_hw *hw, ws_server **out) {
  if (!ctx || !hw || !out) return WS_EINVAL;
  *out = nullptr;
  ws_server *s = new ws_server();
  s->ctx = ctx;
  s->hw = *hw;
  memset(&s->opts, 0, sizeof(s->opts));
  if (opts) s->opts = *opts;
  if (s->opts.max_inflight <= 0) s->opts.max_inflight = 4;
  s->opts.max_inflight = std::min(s->opts.max_inflight, 8);
  if (s->opts.max_step_cfgs <= 0) s->opts.max_step_cfgs = 4096;
  if (s->opts.max_queue <= 0) s->opts.max_queue = 1 << 20;
  memset(&s->stats, 0, sizeof(s->stats));
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    delete s;
    return WS_ECUDA;
  }
  ws::ctx_reclaim(ctx);
  size_t budget = s->opts.mem_budget ? s->opts.mem_budget : ctx->arena->largest_free() / 4 * 3;
  budget = std::min(budget, ctx->arena->largest_free());
  budget &= ~(size_t)255;
  s->pool_off = ctx->arena->alloc(budget);
  if (s->pool_off < 0 || budget < (1 << 20)) {
    if (s->pool_off >= 0) ctx->arena->release(s->pool_off);
    delete s;
    ws::set_error("server pool does not fit the arena");
    return WS_ENOMEM;
  }
  s->pool = new ws::Arena(ctx->arena->base + s->pool_off, budget);
  if (cudaMemset(ctx->arena->base + s->pool_off, 0, budget) != cudaSuccess) {
    ctx->arena->release(s->pool_off);
    delete s->pool;
    delete s;
    return WS_ECUDA;
  }
  s->slots.resize(s->opts.max_inflight);
  for (Slot &sl : s->slots) {
    const bool made = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess;
    if (made) ws::count_resource(ws::RES_STREAM);
    else sl.stream = nullptr;
    if (!made || !ensure_slot_capacity(sl, (size_t)s->opts.max_step_cfgs)) {
      for (Slot &x : s->slots) {
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.h_res) cudaFreeHost(x.h_res);
        if (x.h_ord) cudaFreeHost(x.h_ord);
      }
      ctx->arena->release(s->pool_off);
      delete s->pool;
      delete s;
      return WS_ECUDA;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return WS_OK;
}

extern "C" int ws_server_submit(ws_server *s, const ws_request *req, uint64_t *req_id) {
  if (!s || !req || !req_id || req->n_cfg < 1 || req->n_fld < 1 || req->n_acc < 1 || !req->cfgs || !req->fld ||
      !req->acc || req->n_cfg > s->opts.max_step_cfgs)
    return WS_EINVAL;
  Request *r = new Request();
  r->cfgs.assign(req->cfgs, req->cfgs + req->n_cfg);
  r->fld.assign(req->fld, req->fld + req->n_fld);
  r->acc.assign(req->acc, req->acc + req->n_acc);
  size_t dsc = 0, scr = 0, mf = 0;
  ws::plan_requirements(r->cfgs.data(), req->n_cfg, r->fld.data(), req->n_fld, r->acc.data(), req->n_acc, &s->hw,
                        &dsc, &scr, &mf);
  r->scratch_bytes = scr;
  r->max_field_bytes = mf;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) {
    delete r;
    return WS_ECANCELED;
  }
  if (((mf + 255) & ~(size_t)255) > s->pool->size) {
    s->stats.rejected += 1;
    delete r;
    return WS_ENOMEM;
  }
  if ((int)s->queue.size() >= s->opts.max_queue) {
    s->stats.rejected += 1;
    delete r;
    return WS_EAGAIN;
  }
  r->id = s->next_id++;
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  s->stats.submitted += 1;
  *req_id = r->id;
  s->cv_work.notify_all();
  return WS_OK;
}

extern "C" int ws_server_poll(ws_server *s, uint64_t id, ws_result *out, int32_t *order, int64_t timeout_us) {
  if (!s) return WS_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return WS_ENOTFOUND;
  Request *r = it->second;
  if (!r->done && timeout_us > 0) {
    auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    s->cv_work.notify_all();
    while (!r->done) {
      if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
    }
  }
  if (!r->done) return WS_EAGAIN;
  int rc = r->status;
  if (rc == WS_OK) {
    if (out) memcpy(out, r->results.data(), r->results.size() * sizeof(ws_result));
    if (order) memcpy(order, r->order.data(), r->order.size() * sizeof(int32_t));
  }
  s->reqs.erase(it);
  delete r;
  return rc;
}

extern "C" int ws_server_pause(ws_server *s, int paused) {
  if (!s) return WS_EINVAL;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->paused = paused != 0;
  }
  s->cv_work.notify_all();
  return WS_OK;
}

extern "C" int ws_server_cancel(ws_server *s, uint64_t id) {
  if (!s) return WS_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return WS_ENOTFOUND;
  Request *r = it->second;
  auto q = std::find(s->queue.begin(), s->queue.end(), r);
  if (q == s->queue.end()) return r->done && r->status == WS_ECANCELED ? WS_OK : WS_EAGAIN;
  s->queue.erase(q);
  r->status = WS_ECANCELED;
  r->done = true;
  s->stats.canceled += 1;
  s->cv_done.notify_all();
  return WS_OK;
}

extern "C" int ws_server_stats_get(ws_server *s, ws_server_stats *out) {
  if (!s || !out) return WS_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->stats;
  out->inflight_steps = (int32_t)s->inflight.size();
  out->queued = (int32_t)s->queue.size();
  out->bytes_in_use = (int64_t)s->pool->used();
  out->peak_bytes = (int64_t)s->pool->peak;
  return WS_OK;
}

extern "C" int ws_server_destroy(ws_server *s) {
  if (!s) return WS_EINVAL;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  for (Slot &sl : s->slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
    if (sl.h_res) cudaFreeHost(sl.h_res);
    if (sl.h_ord) cudaFreeHost(sl.h_ord);
  }
  for (auto &kv : s->reqs) delete kv.second;
  s->ctx->arena->release(s->pool_off);
  delete s->pool;
  delete s;
  return WS_OK;
}
