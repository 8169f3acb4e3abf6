// serve.cu — device-resident request loop over render_batch (the serving half of the batch /
// serve step; the paper renders one image at a time and has no counterpart).
//
// Host-side only.  A worker thread owns all GPU submission:
//   1. admission: pending requests, in arrival order, receive their output image (rgb + alpha)
//      from the caller's device arena as long as it fits, at most one batch ahead of the GPU;
//   2. batching: admitted requests are grouped (up to max_batch_views, at most
//      UT_MAX_BATCH_SCENES distinct scenes) into one render_batch call whose key capacity is a
//      learned per-(scene, resolution) estimate times the headroom, and whose workspace is also
//      carved from the arena;
//   3. overlap: up to max_in_flight batches run concurrently on separate non-blocking streams,
//      so requests arriving while others render start as soon as memory and a stream free up;
//   4. completion: each batch records an event that the worker polls; a batch whose true key
//      count exceeded its capacity is re-run with the observed count before completing.
// With use_graphs, each batch's launch sequence is captured on its stream and replayed as a
// CUDA graph; consecutive batches of the same shape update the instantiated graph in place.
// Nothing here blocks on the device except bounded host-side polls; no kernel waits.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ut3d_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t1) {
  return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

// Allocator over [0, size) with 256-byte granularity: workspaces first-fit from the bottom,
// request outputs (which live until the client releases them) last-fit from the top, so that the
// long-lived outputs do not scatter holes through the space the large workspaces need.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    if (size >= 256) free_[0] = size & ~size_t(255);
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        size_t rest = it->second - bytes;
        size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  bool alloc_high(size_t bytes, size_t *off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.rbegin(); it != free_.rend(); ++it) {
      if (it->second >= bytes) {
        it->second -= bytes;  // the block keeps its start and gives up its top
        *off = it->first + it->second;
        if (it->second == 0) free_.erase(std::next(it).base());
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (auto &kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  std::map<size_t, size_t> free_;
};

enum ReqState { PENDING = 0, ADMITTED = 1, RUNNING = 2, DONE = 3, FAILED = 4 };

struct Request {
  uint64_t id;
  int scene;
  ut_camera cam;
  Clock::time_point t_submit, t_done;
  ReqState state = PENDING;
  ut_status status = UT_OK;
  size_t out_off = 0, out_bytes = 0;
  bool has_out = false;  // output image carved from the arena
  uint64_t key_class = 0;
  int overflows = 0;  // key-capacity overflows of the batches it was in
};

// A request whose batches overflowed this often (the arena cannot hold the workspace its key
// count needs) fails with UT_ERR_CAPACITY instead of being retried for ever.
constexpr int kMaxOverflows = 6;

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool busy = false;
  std::vector<uint64_t> reqs;
  size_t ws_off = 0, ws_bytes = 0;
  int64_t cap = 0;
  std::vector<double> est;  // per request key estimate used for the capacity
};

}  // namespace

struct ut_server {
  ut_server_config cfg;
  std::vector<ut_scene> scenes;
  char *arena_base = nullptr;
  Arena arena;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;    // not yet admitted, arrival order
  std::deque<uint64_t> admitted;   // outputs allocated, waiting for a batch
  std::unordered_map<uint64_t, Request> reqs;
  std::unordered_map<uint64_t, double> keys_per_pixel;  // learned (keys / pixel) per (scene, size)
  std::vector<Slot> slots;
  std::thread worker;
  std::atomic<bool> stop{false};
  uint64_t next_id = 1;
  ut_server_stats stats{};
  ut_status fatal = UT_OK;
};

namespace {

size_t out_bytes(const ut_camera &c) { return (size_t)16 * (size_t)c.width * (size_t)c.height; }

// Largest key capacity of one batch (render_batch needs key_capacity < 2^32).
constexpr double kMaxBatchKeys = 4.0e9;

uint64_t key_class(int scene, const ut_camera &c) {
  return ((uint64_t)scene << 40) ^ ((uint64_t)c.model << 36) ^ ((uint64_t)c.width << 18) ^ (uint64_t)c.height;
}

double key_estimate(ut_server *s, const Request &r) {
  auto it = s->keys_per_pixel.find(r.key_class);
  double kpp = it != s->keys_per_pixel.end() ? it->second : 2.0;  // first guess: 2 keys per pixel
  return kpp * (double)r.cam.width * (double)r.cam.height + 1024.0;
}

ut_view make_view(ut_server *s, const Request &r) {
  ut_view v;
  std::memset(&v, 0, sizeof(v));
  v.scene = r.scene;
  v.camera = r.cam;
  v.rgb = reinterpret_cast<float *>(s->arena_base + r.out_off);
  v.alpha = v.rgb + 3 * (size_t)r.cam.width * r.cam.height;
  return v;
}

// Renders a slot's batch on its stream (directly or through a captured graph).
ut_status launch_slot(ut_server *s, Slot &sl) {
  std::vector<ut_view> views;
  for (uint64_t id : sl.reqs) views.push_back(make_view(s, s->reqs[id]));
  char *ws = s->arena_base + sl.ws_off;
  int64_t *k_out = reinterpret_cast<int64_t *>(ws);
  void *wsb = ws + 256;
  size_t wsb_bytes = sl.ws_bytes - 256;
  ut_stream st = reinterpret_cast<ut_stream>(sl.stream);
  if (!s->cfg.use_graphs) {
    ut_status r = render_batch(s->scenes.data(), (int)s->scenes.size(), views.data(), (int)views.size(), &s->cfg.ut,
                               &s->cfg.options, wsb, wsb_bytes, sl.cap, k_out, st);
    if (r != UT_OK) return r;
  } else {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return UT_ERR_CUDA;
    ut_status r = render_batch(s->scenes.data(), (int)s->scenes.size(), views.data(), (int)views.size(), &s->cfg.ut,
                               &s->cfg.options, wsb, wsb_bytes, sl.cap, k_out, st);
    cudaError_t e = cudaStreamEndCapture(sl.stream, &g);
    if (r != UT_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess || !g) return UT_ERR_CUDA;
    bool ok = false;
    if (sl.exec) {
      cudaGraphExecUpdateResultInfo info;
      ok = cudaGraphExecUpdate(sl.exec, g, &info) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        cudaGraphExecDestroy(sl.exec);
        sl.exec = nullptr;
      }
    }
    if (!ok) {
      if (cudaGraphInstantiate(&sl.exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        sl.exec = nullptr;
        return UT_ERR_CUDA;
      }
      s->stats.graph_instantiations++;
    }
    cudaGraphDestroy(g);
    if (cudaGraphLaunch(sl.exec, sl.stream) != cudaSuccess) return UT_ERR_CUDA;
    s->stats.graph_launches++;
  }
  if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return UT_ERR_CUDA;
  s->stats.batches++;
  return UT_OK;
}

void fail_slot(ut_server *s, Slot &sl, ut_status err) {
  auto now = Clock::now();
  for (uint64_t id : sl.reqs) {
    Request &r = s->reqs[id];
    r.state = FAILED;
    r.status = err;
    r.t_done = now;
    s->stats.failed++;
  }
  if (sl.ws_bytes) s->arena.release(sl.ws_off, sl.ws_bytes);
  sl.ws_bytes = 0;
  sl.reqs.clear();
  sl.busy = false;
  s->cv_done.notify_all();  // waiters of the failed requests
}

// Admission and batching (called with the lock held).  Returns true if it launched something.
bool schedule(ut_server *s) {
  // admit pending requests in arrival order while their outputs fit, at most one batch ahead of
  // the GPU: admitting further ahead gains nothing (the slots are busy) and, under a burst,
  // would fill the arena with waiting outputs and leave no room for any batch's workspace
  while (!s->pending.empty() && s->admitted.size() < (size_t)s->cfg.max_batch_views) {
    Request &r = s->reqs[s->pending.front()];
    size_t off;
    if (!s->arena.alloc_high(r.out_bytes, &off)) break;
    r.out_off = off;
    r.has_out = true;
    r.state = ADMITTED;
    s->admitted.push_back(r.id);
    s->pending.pop_front();
  }
  if (s->admitted.empty()) return false;
  Slot *free_slot = nullptr;
  for (auto &sl : s->slots)
    if (!sl.busy) {
      free_slot = &sl;
      break;
    }
  if (!free_slot) return false;
  Slot &sl = *free_slot;
  // take admitted requests in order, shrinking the batch until its workspace fits
  size_t nmax = std::min<size_t>(s->admitted.size(), (size_t)s->cfg.max_batch_views);
  for (size_t nb = nmax; nb >= 1; --nb) {
    std::vector<ut_view> views;
    std::vector<double> est;
    double cap = 0;
    for (size_t j = 0; j < nb; ++j) {
      Request &r = s->reqs[s->admitted[j]];
      views.push_back(make_view(s, r));
      est.push_back(key_estimate(s, r));
      cap += est.back();
    }
    const double want = cap * (double)s->cfg.key_headroom;
    if (want > kMaxBatchKeys && nb > 1) continue;  // more keys than one batch can sort: fewer views
    int64_t capacity = (int64_t)std::min(want, kMaxBatchKeys);
    size_t need = ut_batch_workspace_size(s->scenes.data(), (int)s->scenes.size(), views.data(), (int)nb,
                                          &s->cfg.options, capacity);
    if (need == 0) {
      // an invalid request: fail the first one alone
      Request &r = s->reqs[s->admitted.front()];
      r.state = FAILED;
      r.status = UT_ERR_INVALID_ARG;
      s->stats.failed++;
      r.t_done = Clock::now();
      s->admitted.pop_front();
      s->cv_done.notify_all();
      return true;
    }
    size_t off;
    if (!s->arena.alloc(need + 256, &off)) {
      if (nb > 1) continue;
      // one view whose estimated keys do not fit while nothing else holds arena memory: run it
      // with the largest capacity the arena can hold (an overflow re-runs it with the observed
      // count; the estimate may be inflated).  With batches in flight, wait for their memory.
      bool any_busy = false;
      for (auto &x : s->slots) any_busy |= x.busy;
      if (any_busy) break;
      const size_t avail = s->arena.largest();
      int64_t lo = 0, hi = capacity;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        const size_t nm = ut_batch_workspace_size(s->scenes.data(), (int)s->scenes.size(), views.data(), 1,
                                                  &s->cfg.options, mid);
        if (nm != 0 && ((nm + 256 + 255) & ~(size_t)255) <= avail) lo = mid;
        else hi = mid - 1;
      }
      if (lo < 1024) break;
      capacity = lo;
      need = ut_batch_workspace_size(s->scenes.data(), (int)s->scenes.size(), views.data(), 1, &s->cfg.options,
                                     capacity);
      if (need == 0 || !s->arena.alloc(need + 256, &off)) break;
    }
    sl.ws_off = off;
    sl.ws_bytes = need + 256;
    sl.cap = capacity;
    sl.est = est;
    sl.reqs.assign(s->admitted.begin(), s->admitted.begin() + nb);
    s->admitted.erase(s->admitted.begin(), s->admitted.begin() + nb);
    for (uint64_t id : sl.reqs) s->reqs[id].state = RUNNING;
    sl.busy = true;
    ut_status r = launch_slot(s, sl);
    if (r != UT_OK) fail_slot(s, sl, r);
    return true;
  }
  // not even one view's workspace fits: if nothing is in flight it never will
  bool any_busy = false;
  for (auto &x : s->slots) any_busy |= x.busy;
  if (!any_busy) {
    Request &r = s->reqs[s->admitted.front()];
    r.state = FAILED;
    r.status = UT_ERR_CAPACITY;
    s->stats.failed++;
    r.t_done = Clock::now();
    s->admitted.pop_front();
    s->cv_done.notify_all();
  }
  return false;
}

// Completion of finished batches (lock held).  Returns true if anything completed.
bool reap(ut_server *s) {
  bool any = false;
  for (auto &sl : s->slots) {
    if (!sl.busy) continue;
    cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    any = true;
    if (q != cudaSuccess) {
      fail_slot(s, sl, UT_ERR_CUDA);
      continue;
    }
    int64_t K = 0;
    if (cudaMemcpyAsync(&K, s->arena_base + sl.ws_off, sizeof(K), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaStreamSynchronize(sl.stream) != cudaSuccess) {
      fail_slot(s, sl, UT_ERR_CUDA);
      continue;
    }
    // learn keys per pixel: scale every class of the batch by observed / estimated
    double est_total = 0;
    for (double e : sl.est) est_total += e;
    double ratio = est_total > 0 ? (double)K / est_total : 1.0;
    for (size_t j = 0; j < sl.reqs.size(); ++j) {
      Request &r = s->reqs[sl.reqs[j]];
      double px = (double)r.cam.width * r.cam.height;
      double kpp = std::max(1e-3, (sl.est[j] - 1024.0) / px * ratio);
      auto it = s->keys_per_pixel.find(r.key_class);
      s->keys_per_pixel[r.key_class] = it == s->keys_per_pixel.end() ? kpp : std::max(0.5 * it->second, kpp);
    }
    if (K > sl.cap) {
      // overflow: re-run the same batch with the observed key count
      s->stats.retries++;
      s->arena.release(sl.ws_off, sl.ws_bytes);
      sl.ws_bytes = 0;
      std::vector<ut_view> views;
      for (uint64_t id : sl.reqs) views.push_back(make_view(s, s->reqs[id]));
      const double want = (double)K * s->cfg.key_headroom + 1024.0;
      int worst = 0;
      for (uint64_t id : sl.reqs) worst = std::max(worst, ++s->reqs[id].overflows);
      if ((want > kMaxBatchKeys || worst > kMaxOverflows) && sl.reqs.size() == 1) {
        // one view with more keys than any batch can sort, or than the arena could ever give it
        fail_slot(s, sl, UT_ERR_CAPACITY);
        continue;
      }
      // (a batch of several views whose keys exceed one batch goes back to the queue; its views'
      // learned key estimates now split it)
      int64_t capacity = (int64_t)std::min(want, kMaxBatchKeys);
      size_t need = want > kMaxBatchKeys ? 0
                                         : ut_batch_workspace_size(s->scenes.data(), (int)s->scenes.size(),
                                                                   views.data(), (int)views.size(), &s->cfg.options,
                                                                   capacity);
      size_t off;
      if (need == 0 || !s->arena.alloc(need + 256, &off)) {
        // put the requests back at the head of the queue, to be re-batched when memory frees up
        s->stats.requeued++;
        sl.ws_bytes = 0;
        for (auto it = sl.reqs.rbegin(); it != sl.reqs.rend(); ++it) {
          s->reqs[*it].state = ADMITTED;
          s->admitted.push_front(*it);
        }
        sl.reqs.clear();
        sl.busy = false;
        continue;
      }
      sl.ws_off = off;
      sl.ws_bytes = need + 256;
      sl.cap = capacity;
      ut_status r = launch_slot(s, sl);
      if (r != UT_OK) fail_slot(s, sl, r);
      continue;
    }
    auto now = Clock::now();
    for (uint64_t id : sl.reqs) {
      Request &r = s->reqs[id];
      r.state = DONE;
      r.t_done = now;
      s->stats.completed++;
    }
    s->arena.release(sl.ws_off, sl.ws_bytes);
    sl.ws_bytes = 0;
    sl.reqs.clear();
    sl.busy = false;
  }
  if (any) s->cv_done.notify_all();
  return any;
}

void worker_main(ut_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool busy = false;
    for (auto &sl : s->slots) busy |= sl.busy;
    if (s->stop.load() && !busy) break;
    bool progress = reap(s);
    if (!s->stop.load()) progress |= schedule(s);
    busy = false;
    for (auto &sl : s->slots) busy |= sl.busy;
    if (progress) continue;
    // nothing to do right now: sleep until a submission, or poll the GPU again shortly
    if (busy) s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    else s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
  }
}

}  // namespace

using namespace ut3d;

extern "C" {

ut_status ut_server_create(const ut_server_config *cfg, const ut_scene *scenes, int32_t n_scenes, void *arena,
                           size_t arena_bytes, ut_server **out) {
  if (!cfg || !scenes || !out || !arena || n_scenes < 1 || n_scenes > UT_MAX_BATCH_SCENES) return UT_ERR_INVALID_ARG;
  if (cfg->max_batch_views < 1 || cfg->max_batch_views > UT_MAX_BATCH_VIEWS || cfg->max_in_flight < 1 ||
      cfg->max_in_flight > 8 || !(cfg->key_headroom >= 1.f) || (reinterpret_cast<uintptr_t>(arena) & 255))
    return UT_ERR_INVALID_ARG;
  for (int k = 0; k < n_scenes; ++k)
    if (scenes[k].sh_degree != scenes[0].sh_degree || scenes[k].n < 0) return UT_ERR_INVALID_ARG;
  ut_server *s = new ut_server();
  s->cfg = *cfg;
  s->scenes.assign(scenes, scenes + n_scenes);
  s->arena_base = static_cast<char *>(arena);
  s->arena.init(arena_bytes);
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return UT_ERR_CUDA;
  }
  s->slots.resize(cfg->max_in_flight);
  for (auto &sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      for (auto &x : s->slots) {
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.done) cudaEventDestroy(x.done);
      }
      delete s;
      return UT_ERR_CUDA;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return UT_OK;
}

ut_status ut_server_submit(ut_server *s, int32_t scene, const ut_camera *cam, uint64_t *id) {
  if (!s || !cam || !id || scene < 0 || scene >= (int)s->scenes.size()) return UT_ERR_INVALID_ARG;
  if (cam->width < 1 || cam->height < 1 || cam->width > 32767 || cam->height > 32767) return UT_ERR_INVALID_ARG;
  Request r;
  r.scene = scene;
  r.cam = *cam;
  r.out_bytes = out_bytes(*cam);
  r.key_class = key_class(scene, *cam);
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r.out_bytes > s->arena.largest() && s->pending.empty() && s->admitted.empty()) {
      bool busy = false;
      for (auto &sl : s->slots) busy |= sl.busy;
      if (!busy) return UT_ERR_CAPACITY;
    }
    r.id = s->next_id++;
    s->reqs[r.id] = r;
    s->pending.push_back(r.id);
    *id = r.id;
  }
  s->cv_work.notify_one();
  return UT_OK;
}

ut_status ut_server_wait(ut_server *s, uint64_t id, int32_t timeout_ms, int32_t *done, const float **rgb,
                         const float **alpha, double *latency_ms) {
  if (!s || !done) return UT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return UT_ERR_INVALID_ARG;
  auto finished = [&] { return it->second.state == DONE || it->second.state == FAILED; };
  if (!finished() && timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
  const Request &r = it->second;
  if (!finished()) {
    *done = 0;
    return timeout_ms > 0 ? UT_ERR_TIMEOUT : UT_OK;
  }
  *done = 1;
  if (r.state == FAILED) return r.status;
  if (rgb) *rgb = reinterpret_cast<const float *>(s->arena_base + r.out_off);
  if (alpha) *alpha = reinterpret_cast<const float *>(s->arena_base + r.out_off) + 3 * (size_t)r.cam.width * r.cam.height;
  if (latency_ms) *latency_ms = ms_since(r.t_submit, r.t_done);
  return UT_OK;
}

ut_status ut_server_release(ut_server *s, uint64_t id) {
  if (!s) return UT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return UT_ERR_INVALID_ARG;
    Request &r = it->second;
    if (r.state != DONE && r.state != FAILED) return UT_ERR_INVALID_ARG;
    if (r.has_out) s->arena.release(r.out_off, r.out_bytes);
    s->reqs.erase(it);
  }
  s->cv_work.notify_one();
  return UT_OK;
}

ut_status ut_server_get_stats(ut_server *s, ut_server_stats *stats) {
  if (!s || !stats) return UT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *stats = s->stats;
  return UT_OK;
}

ut_status ut_server_destroy(ut_server *s) {
  if (!s) return UT_ERR_INVALID_ARG;
  s->stop.store(true);
  s->cv_work.notify_all();
  // the worker drains the batches in flight; give it a bounded time
  auto t0 = Clock::now();
  while (true) {
    bool busy = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto &sl : s->slots) busy |= sl.busy;
    }
    if (!busy || ms_since(t0, Clock::now()) > 30000.0) break;
    std::this_thread::sleep_for(std::chrono::milliseconds(1));
  }
  ut_status st = UT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &sl : s->slots)
      if (sl.busy) st = UT_ERR_TIMEOUT;
  }
  if (st == UT_OK) {
    s->worker.join();
    for (auto &sl : s->slots) {
      if (sl.exec) cudaGraphExecDestroy(sl.exec);
      cudaEventDestroy(sl.done);
      cudaStreamDestroy(sl.stream);
    }
    delete s;
  } else {
    // the GPU did not finish within the bound: leave the worker and its resources alive
    // rather than free memory that kernels may still be using
    s->worker.detach();
  }
  return st;
}

}  // extern "C"
