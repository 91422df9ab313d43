// Serving form (not in the paper): a request loop over resident graphs with
// continuous batching.  Graphs are oriented once on arrival and kept in a
// device pool the caller provides; count, local-clustering and listing
// requests arrive at any time and are admitted as soon as one of the server's
// slots (a CUDA stream each) and enough pool memory are free, so requests that
// arrive while others run join the device immediately and overlap with them.
// Admission is by footprint (workspace plus outputs) against the pool; a
// request that can never fit is rejected.  Completion is signalled from the
// stream by a host function, so the worker thread never polls the GPU.
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

#include "tc_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// First-fit sub-allocator over the caller's device pool (256-byte granules).
class Pool {
 public:
  Pool() = default;
  void init(char* base, size_t bytes) {
    base_ = base;
    cap_ = bytes & ~size_t(255);
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
    used_ = 0;
  }
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, left = it->second - bytes;
        free_.erase(it);
        if (left) free_[off + bytes] = left;
        live_[off] = bytes;
        used_ += bytes;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void release(void* p) {
    if (!p) return;
    const size_t off = static_cast<size_t>(static_cast<char*>(p) - base_);
    auto lv = live_.find(off);
    if (lv == live_.end()) return;
    size_t size = lv->second;
    live_.erase(lv);
    used_ -= size;
    size_t start = off;
    auto next = free_.lower_bound(off);
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        start = prev->first;
        size += prev->second;
        free_.erase(prev);
      }
    }
    next = free_.lower_bound(start + size);
    if (next != free_.end() && next->first == start + size) {
      size += next->second;
      free_.erase(next);
    }
    free_[start] = size;
  }
  size_t used() const { return used_; }
  size_t capacity() const { return cap_; }

 private:
  char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
  std::unordered_map<size_t, size_t> live_;
};

struct GraphRec {
  int32_t n = 0;
  int64_t m = 0;
  int64_t* offsets = nullptr;
  int32_t* cols = nullptr;
  int32_t* deg = nullptr;
  int32_t* dhat = nullptr;
  void* block = nullptr;  // one pool block holds the whole CSR
  int inflight = 0;
  bool removed = false;
};

enum ReqState { REQ_PENDING, REQ_RUNNING, REQ_LIST_WAIT, REQ_DONE };

struct Request {
  int64_t ticket = 0, graph = 0;
  int kind = 0;
  ReqState state = REQ_PENDING;
  tc_status status = TC_OK;
  int slot = -1;
  int phase = 0;            // listing: 0 = counting, 1 = writing
  Clock::time_point t_wait; // listing: when its output buffer was first refused
  void* ws = nullptr;
  void* out = nullptr;      // pool block: total (+ T_v, C_v)
  int32_t* tri = nullptr;   // listing output (pool)
  uint64_t T = 0;
  Clock::time_point t_submit, t_admit, t_done;
};

constexpr int32_t kLargeTileQuota = 4;  // vertex chunks per warp before a block of a large request retires

struct Slot {
  cudaStream_t stream = nullptr;
  bool high = false;            // high-priority stream: small requests only
  tc::Ctx ctx;
  uint64_t* h_total = nullptr;  // pinned
  std::atomic<bool> done{false};
  int64_t ticket = -1;
  void* err_block = nullptr;
};

}  // namespace

struct tc_server {
  int device = 0;
  Pool pool;
  std::mutex admin_mu;  // one graph is added at a time (admin stream and its error word)
  std::mutex mu;
  std::condition_variable cv_done;
  // wake-ups of the worker: completions (from stream host functions) and
  // submissions bump `kicks` under wake_mu, which is never held across a CUDA
  // call, so a host function can always take it
  std::mutex wake_mu;
  std::condition_variable cv_wake;
  uint64_t kicks = 0;
  std::thread worker;
  bool stop = false;
  std::vector<Slot*> slots;
  std::map<int64_t, GraphRec> graphs;
  std::map<int64_t, Request> reqs;
  std::deque<int64_t> pending;
  int64_t next_graph = 1, next_ticket = 1;
  cudaStream_t admin = nullptr;
  tc::Ctx admin_ctx;
  uint64_t* admin_h = nullptr;
  void* admin_err = nullptr;
  int64_t admitted = 0, completed = 0, rejected = 0, edges_done = 0;
  int64_t admit_timeout_ms = 10000;
  int64_t small_edges = int64_t(1) << 21;
  size_t resident_bytes = 0;  // resident graphs and slot blocks: memory no request can reclaim
  char last_error[256] = {0};
};

namespace {

tc_status set_error(tc_server* s, tc_status st, const char* msg) {
  if (s) snprintf(s->last_error, sizeof(s->last_error), "%s", msg);
  return st;
}

void kick(tc_server* s) {
  {
    std::lock_guard<std::mutex> g(s->wake_mu);
    ++s->kicks;
  }
  s->cv_wake.notify_all();
}

void CUDART_CB on_slot_done(void* p) {
  auto* pr = static_cast<std::pair<tc_server*, Slot*>*>(p);
  pr->second->done.store(true, std::memory_order_release);
  kick(pr->first);
  delete pr;
}

size_t count_ws_bytes(int op, int32_t n, int64_t m) {
  size_t b = 0;
  tc_workspace_size(static_cast<tc_op>(op), n, m, &b);
  return b;
}

// Footprint of a request at admission (listing: its first phase).
size_t footprint(const GraphRec& g, int kind) {
  size_t out = 256;
  if (kind == TC_REQ_LOCAL) out += 16 * static_cast<size_t>(g.n) + 512;
  const int op = kind == TC_REQ_LIST ? TC_OP_LIST : TC_OP_COUNT;
  return count_ws_bytes(op, g.n, g.m) + out;
}

// Enqueue the work of request r (current phase) on its slot; caller holds the lock.
cudaError_t launch_request(tc_server* s, Request& r, GraphRec& g) {
  Slot& sl = *s->slots[static_cast<size_t>(r.slot)];
  cudaStream_t st = sl.stream;
  tc::Ctx* ctx = &sl.ctx;
  uint64_t* total = static_cast<uint64_t*>(r.out);
  cudaError_t e = cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), st);
  tc::Carver c(r.ws);
  if (r.kind == TC_REQ_COUNT || r.kind == TC_REQ_LOCAL) {
    tc::CountWs w = tc::carve_count(c, g.n, g.m, false);
    int64_t* tv = r.kind == TC_REQ_LOCAL ? reinterpret_cast<int64_t*>(static_cast<char*>(r.out) + 256) : nullptr;
    double* cc = r.kind == TC_REQ_LOCAL ? reinterpret_cast<double*>(tv + g.n) : nullptr;
    if (e == cudaSuccess) e = cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
    if (e == cudaSuccess && tv) e = cudaMemsetAsync(tv, 0, sizeof(int64_t) * static_cast<size_t>(g.n), st);
    tc::CountArgs a{g.n, g.m, g.offsets, g.cols, reinterpret_cast<unsigned long long*>(total), tv, nullptr, 0};
    if (e == cudaSuccess) e = tc::launch_count(ctx, tv ? tc::MODE_LOCAL : tc::MODE_COUNT, a, w, st);
    if (e == cudaSuccess && cc) e = tc::launch_clustering(ctx, g.n, g.deg, tv, cc, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_total, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  } else {
    tc::CountWs w = tc::carve_count(c, g.n, g.m, true);
    if (r.phase == 0) {
      if (e == cudaSuccess) e = cudaMemsetAsync(w.ecount, 0, sizeof(int32_t) * static_cast<size_t>(g.m), st);
      tc::CountArgs a{g.n, g.m, g.offsets, g.cols, nullptr, nullptr, nullptr, 0};
      if (e == cudaSuccess) e = tc::launch_count(ctx, tc::MODE_LIST_COUNT, a, w, st);
      if (e == cudaSuccess) e = tc::launch_list_offsets(ctx, g.m, w, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_total, w.eoff + g.m, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    } else {
      tc::CountArgs a{g.n, g.m, g.offsets, g.cols, nullptr, nullptr, r.tri, static_cast<int64_t>(r.T)};
      a.reuse_hub = true;  // phase 0 built the hub schedule in this workspace with the same slot settings
      if (e == cudaSuccess) e = tc::launch_count(ctx, tc::MODE_LIST_WRITE, a, w, st);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) {
    sl.done.store(false);
    e = cudaLaunchHostFunc(st, on_slot_done, new std::pair<tc_server*, Slot*>(s, &sl));
  }
  return e;
}

void finish_request(tc_server* s, Request& r, tc_status st) {
  r.status = st;
  r.state = REQ_DONE;
  r.t_done = Clock::now();
  if (r.ws) {
    s->pool.release(r.ws);
    r.ws = nullptr;
  }
  auto git = s->graphs.find(r.graph);
  if (git != s->graphs.end()) {
    git->second.inflight--;
    if (st == TC_OK) s->edges_done += git->second.m;
  }
  if (r.slot >= 0) {
    s->slots[static_cast<size_t>(r.slot)]->ticket = -1;
    r.slot = -1;
  }
  if (st == TC_OK) s->completed++;
  else if (st == TC_ERR_REJECTED) s->rejected++;
  s->cv_done.notify_all();
}

// A launch that failed part way: kernels already queued on the slot's stream may
// still run, and the slot's completion callback may still be queued.  Wait for the
// stream before the workspace and result go back to the pool and the slot is reused.
void fail_launched(tc_server* s, Request& r) {
  if (r.slot >= 0 && static_cast<size_t>(r.slot) < s->slots.size()) {
    Slot& sl = *s->slots[static_cast<size_t>(r.slot)];
    cudaStreamSynchronize(sl.stream);
    sl.done.store(false);
  }
  finish_request(s, r, TC_ERR_CUDA);
}

tc_status status_of(uint32_t bits) {
  if (!bits) return TC_OK;
  if (bits & tc::ERR_CAPACITY) return TC_ERR_CAPACITY;
  if (bits & tc::ERR_TOO_LONG) return TC_ERR_UNSUPPORTED;
  return TC_ERR_INVALID_GRAPH;
}

bool anything_running(tc_server* s) {
  for (Slot* sl : s->slots)
    if (sl->ticket >= 0) return true;
  return false;
}

void worker_loop(tc_server* s) {
  cudaSetDevice(s->device);
  uint64_t seen = 0;
  for (;;) {
    {
      std::lock_guard<std::mutex> g(s->wake_mu);
      seen = s->kicks;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) break;
    bool progressed = false;
    // 1. retire finished slots
    for (size_t i = 0; i < s->slots.size(); ++i) {
      Slot& sl = *s->slots[i];
      if (sl.ticket < 0 || !sl.done.load(std::memory_order_acquire)) continue;
      progressed = true;
      sl.done.store(false);
      Request& r = s->reqs[sl.ticket];
      GraphRec& g = s->graphs[r.graph];
      const tc_status st = status_of(*sl.ctx.h_err);
      if (st != TC_OK) {
        finish_request(s, r, st);
        continue;
      }
      if (r.kind == TC_REQ_LIST && r.phase == 0) {
        r.T = *sl.h_total;
        r.phase = 1;
        r.tri = static_cast<int32_t*>(s->pool.alloc(12 * static_cast<size_t>(r.T > 0 ? r.T : 1)));
        if (!r.tri) {  // hold the slot until memory frees up (bounded by the admission timeout)
          r.state = REQ_LIST_WAIT;
          r.t_wait = Clock::now();
          continue;
        }
        if (launch_request(s, r, g) != cudaSuccess) fail_launched(s, r);
        continue;
      }
      if (r.kind != TC_REQ_LIST) r.T = *sl.h_total;
      finish_request(s, r, TC_OK);
    }
    // listing requests waiting for their output buffer
    for (size_t i = 0; i < s->slots.size(); ++i) {
      Slot& sl = *s->slots[i];
      if (sl.ticket < 0) continue;
      Request& r = s->reqs[sl.ticket];
      if (r.state != REQ_LIST_WAIT) continue;
      r.tri = static_cast<int32_t*>(s->pool.alloc(12 * static_cast<size_t>(r.T > 0 ? r.T : 1)));
      if (r.tri) {
        r.state = REQ_RUNNING;
        progressed = true;
        if (launch_request(s, r, s->graphs[r.graph]) != cudaSuccess) fail_launched(s, r);
      } else {
        const size_t need = 12 * static_cast<size_t>(r.T > 0 ? r.T : 1);
        const bool never = need + s->resident_bytes > s->pool.capacity();
        if (never || ms_between(r.t_wait, Clock::now()) > static_cast<double>(s->admit_timeout_ms)) {
          progressed = true;
          finish_request(s, r, TC_ERR_REJECTED);
        }
      }
    }
    // 2. admit pending requests while slots and memory allow (in arrival order; a
    //    request that does not fit yet lets later, smaller ones go first)
    for (auto it = s->pending.begin(); it != s->pending.end();) {
      Request& r = s->reqs[*it];
      GraphRec& g = s->graphs[r.graph];
      // small requests prefer a high-priority slot and may take any; large ones only low-priority slots
      const bool small = g.m <= s->small_edges;
      int free_slot = -1;
      for (size_t i = 0; i < s->slots.size(); ++i) {
        const Slot& sl = *s->slots[i];
        if (sl.ticket >= 0 || (sl.high && !small)) continue;
        if (free_slot < 0 || (sl.high && !s->slots[static_cast<size_t>(free_slot)]->high)) free_slot = static_cast<int>(i);
      }
      if (free_slot < 0) {
        if (small) break;  // every slot is busy
        ++it;              // no low-priority slot: later small requests may still start
        continue;
      }
      const size_t need = footprint(g, r.kind);
      const size_t ws_b = need - (r.kind == TC_REQ_LOCAL ? 16 * static_cast<size_t>(g.n) + 768 : 256);
      void* ws = s->pool.alloc(ws_b);
      void* out = ws ? s->pool.alloc(need - ws_b) : nullptr;
      if (!ws || !out) {
        s->pool.release(ws);
        // refuse what can never fit, or what has waited past the admission timeout
        const bool never = need + s->resident_bytes > s->pool.capacity();
        if (never || ms_between(r.t_submit, Clock::now()) > static_cast<double>(s->admit_timeout_ms)) {
          progressed = true;
          r.slot = -1;
          finish_request(s, r, TC_ERR_REJECTED);
          it = s->pending.erase(it);
          continue;
        }
        ++it;
        continue;
      }
      progressed = true;
      r.ws = ws;
      r.out = out;
      r.slot = free_slot;
      r.state = REQ_RUNNING;
      r.t_admit = Clock::now();
      s->slots[static_cast<size_t>(free_slot)]->ticket = r.ticket;
      s->admitted++;
      it = s->pending.erase(it);
      if (launch_request(s, r, g) != cudaSuccess) fail_launched(s, r);
    }
    lk.unlock();
    if (!progressed) {  // sleep until a completion or submission (or a timeout check is due)
      std::unique_lock<std::mutex> g(s->wake_mu);
      s->cv_wake.wait_for(g, std::chrono::milliseconds(20), [&] { return s->kicks != seen; });
    }
  }
}

}  // namespace

extern "C" {

tc_status tc_serve_create(int device, const tc_serve_config* cfg, void* pool_dev, size_t pool_bytes,
                          tc_server** out) {
  if (!out || !pool_dev || pool_bytes < (size_t(1) << 16)) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  const int slots = cfg && cfg->slots > 0 ? cfg->slots : 8;
  if (slots > 64) return TC_ERR_INVALID_ARG;
  const int64_t admit_timeout = cfg && cfg->admit_timeout_ms > 0 ? cfg->admit_timeout_ms : 10000;
  const int32_t tile_max = cfg && cfg->tile_max > 0 ? cfg->tile_max : 0;
  const int32_t high = cfg && cfg->high_slots > 0 ? cfg->high_slots : slots / 2;
  if (slots > 1 && high >= slots) return TC_ERR_INVALID_ARG;
  const int32_t n_high = slots > 1 ? high : 0;
  const int32_t grid_div = cfg && cfg->grid_div > 0 ? cfg->grid_div : 2;
  if (grid_div > 64) return TC_ERR_INVALID_ARG;
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (cudaSetDevice(device) != cudaSuccess) return TC_ERR_CUDA;
  tc_server* s = new tc_server();
  s->device = device;
  s->admit_timeout_ms = admit_timeout;
  if (cfg && cfg->small_edges > 0) s->small_edges = cfg->small_edges;
  s->pool.init(static_cast<char*>(pool_dev), pool_bytes);
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  auto fail_create = [&]() {
    tc_serve_destroy(s);
    return TC_ERR_CUDA;
  };
  if (cudaStreamCreateWithFlags(&s->admin, cudaStreamNonBlocking) != cudaSuccess) return fail_create();
  s->admin_err = s->pool.alloc(256);
  if (cudaHostAlloc(reinterpret_cast<void**>(&s->admin_h), 256, cudaHostAllocDefault) != cudaSuccess) return fail_create();
  s->admin_ctx.device = device;
  s->admin_ctx.sm_count = sms;
  s->admin_ctx.async = 1;
  s->admin_ctx.d_err = static_cast<uint32_t*>(s->admin_err);
  s->admin_ctx.h_err = reinterpret_cast<uint32_t*>(s->admin_h);
  for (int i = 0; i < slots; ++i) {
    Slot* sl = new Slot();
    s->slots.push_back(sl);
    sl->high = i < n_high;
    if (cudaStreamCreateWithPriority(&sl->stream, cudaStreamNonBlocking, sl->high ? prio_high : prio_low) !=
        cudaSuccess)
      return fail_create();
    sl->err_block = s->pool.alloc(256);
    if (!sl->err_block) return fail_create();
    if (cudaHostAlloc(reinterpret_cast<void**>(&sl->h_total), 64, cudaHostAllocDefault) != cudaSuccess)
      return fail_create();
    sl->ctx.device = device;
    sl->ctx.sm_count = sms;
    sl->ctx.async = 1;
    sl->ctx.grid_div = sl->high ? 1 : grid_div;  // small requests' grids are sized by their work
    // large requests' tile-kernel blocks retire after a few vertex chunks, so that
    // blocks of high-priority small requests find free SMs within microseconds
    sl->ctx.tile_quota = sl->high ? 0 : kLargeTileQuota;
    sl->ctx.tile_max = tile_max;
    sl->ctx.d_err = static_cast<uint32_t*>(sl->err_block);
    sl->ctx.h_err = reinterpret_cast<uint32_t*>(sl->h_total + 4);
  }
  s->resident_bytes = s->pool.used();
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return TC_OK;
}

void tc_serve_destroy(tc_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  kick(s);
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (Slot* sl : s->slots) {
    if (sl->stream) {
      cudaStreamSynchronize(sl->stream);
      cudaStreamDestroy(sl->stream);
    }
    if (sl->h_total) cudaFreeHost(sl->h_total);
    delete sl;
  }
  if (s->admin) {
    cudaStreamSynchronize(s->admin);
    cudaStreamDestroy(s->admin);
  }
  if (s->admin_h) cudaFreeHost(s->admin_h);
  delete s;
}

const char* tc_serve_last_error(const tc_server* s) { return s ? s->last_error : "no server"; }

tc_status tc_serve_add_graph(tc_server* s, int32_t n, int64_t m, const int32_t* edges_host, int64_t* graph_id) {
  if (!s || !graph_id || n < 0 || m < 0 || (m > 0 && !edges_host)) return TC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> admin(s->admin_mu);
  std::unique_lock<std::mutex> lk(s->mu);
  cudaSetDevice(s->device);
  const size_t nn = static_cast<size_t>(n), mm = static_cast<size_t>(m);
  const size_t csr = 8 * (nn + 1) + 256 + 4 * mm + 256 + 4 * nn + 256 + 4 * nn + 256;
  void* block = s->pool.alloc(csr);
  size_t ows = 0;
  tc_workspace_size(TC_OP_ORIENT, n, m, &ows);
  void* scratch = block ? s->pool.alloc(ows + 8 * mm + 256) : nullptr;
  if (!block || !scratch) {
    s->pool.release(block);
    return set_error(s, TC_ERR_REJECTED, "graph does not fit in the serving pool");
  }
  GraphRec g;
  g.n = n;
  g.m = m;
  g.block = block;
  tc::Carver c(block);
  g.offsets = c.take<int64_t>(nn + 1);
  g.cols = c.take<int32_t>(mm > 0 ? mm : 1);
  g.deg = c.take<int32_t>(nn > 0 ? nn : 1);
  g.dhat = c.take<int32_t>(nn > 0 ? nn : 1);
  tc::Carver sc(scratch);
  int32_t* edges_dev = sc.take<int32_t>(2 * (mm > 0 ? mm : 1));
  void* ws = sc.take<char>(ows);
  tc::Carver wc(ws);
  tc::OrientWs ow = tc::carve_orient(wc, n, m);
  cudaError_t e = cudaMemsetAsync(s->admin_ctx.d_err, 0, sizeof(uint32_t), s->admin);
  if (e == cudaSuccess && m > 0)
    e = cudaMemcpyAsync(edges_dev, edges_host, 8 * mm, cudaMemcpyHostToDevice, s->admin);
  if (e == cudaSuccess) e = tc::launch_orient(&s->admin_ctx, n, m, edges_dev, g.offsets, g.cols, g.deg, g.dhat, ow, s->admin);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->admin_h, s->admin_ctx.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->admin);
  lk.unlock();  // the orientation runs while other requests are served
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->admin);
  lk.lock();
  s->pool.release(scratch);
  if (e != cudaSuccess) {
    s->pool.release(block);
    return set_error(s, TC_ERR_CUDA, cudaGetErrorString(e));
  }
  const uint32_t bits = *reinterpret_cast<uint32_t*>(s->admin_h);
  if (bits) {
    s->pool.release(block);
    return set_error(s, bits & tc::ERR_TOO_LONG ? TC_ERR_UNSUPPORTED : TC_ERR_INVALID_GRAPH,
                     "the edge list is not a simple graph on [0, n)");
  }
  const int64_t id = s->next_graph++;
  s->graphs[id] = g;
  s->resident_bytes += (csr + 255) & ~size_t(255);
  *graph_id = id;
  return TC_OK;
}

tc_status tc_serve_remove_graph(tc_server* s, int64_t graph_id) {
  if (!s) return TC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->graphs.find(graph_id);
  if (it == s->graphs.end() || it->second.removed) return TC_ERR_INVALID_ARG;
  if (it->second.inflight > 0) return set_error(s, TC_ERR_NOT_READY, "requests on this graph are still running");
  s->pool.release(it->second.block);
  const size_t nn = static_cast<size_t>(it->second.n), mm = static_cast<size_t>(it->second.m);
  s->resident_bytes -= (8 * (nn + 1) + 256 + 4 * mm + 256 + 4 * nn + 256 + 4 * nn + 256 + 255) & ~size_t(255);
  it->second.removed = true;
  return TC_OK;
}

tc_status tc_serve_submit(tc_server* s, int64_t graph_id, int kind, int64_t* ticket) {
  if (!s || !ticket || kind < TC_REQ_COUNT || kind > TC_REQ_LIST) return TC_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->graphs.find(graph_id);
    if (it == s->graphs.end() || it->second.removed) return set_error(s, TC_ERR_INVALID_ARG, "unknown graph");
    Request r;
    r.ticket = s->next_ticket++;
    r.graph = graph_id;
    r.kind = kind;
    r.t_submit = Clock::now();
    it->second.inflight++;
    s->reqs[r.ticket] = r;
    s->pending.push_back(r.ticket);
    *ticket = r.ticket;
  }
  kick(s);
  return TC_OK;
}

static void fill_result(tc_server* s, const Request& r, tc_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->status = r.status;
  out->kind = r.kind;
  out->graph_id = r.graph;
  out->triangles = r.T;
  const GraphRec& g = s->graphs[r.graph];
  out->n = g.n;
  if (r.status == TC_OK && r.kind == TC_REQ_LOCAL) {
    out->tv = reinterpret_cast<const int64_t*>(static_cast<char*>(r.out) + 256);
    out->cc = reinterpret_cast<const double*>(out->tv + g.n);
  }
  if (r.status == TC_OK && r.kind == TC_REQ_LIST) out->tri = r.tri;
  out->queue_ms = r.state == REQ_DONE && r.t_admit.time_since_epoch().count() ? ms_between(r.t_submit, r.t_admit) : 0.0;
  out->latency_ms = ms_between(r.t_submit, r.t_done);
}

tc_status tc_serve_poll(tc_server* s, int64_t ticket, tc_result* out) {
  if (!s || !out) return TC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return TC_ERR_INVALID_ARG;
  if (it->second.state != REQ_DONE) return TC_ERR_NOT_READY;
  fill_result(s, it->second, out);
  return it->second.status;
}

tc_status tc_serve_wait(tc_server* s, int64_t ticket, int64_t timeout_ms, tc_result* out) {
  if (!s || !out) return TC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return TC_ERR_INVALID_ARG;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms > 0 ? timeout_ms : 0);
  while (it->second.state != REQ_DONE) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state != REQ_DONE)
      return TC_ERR_TIMEOUT;
  }
  fill_result(s, it->second, out);
  return it->second.status;
}

tc_status tc_serve_release(tc_server* s, int64_t ticket) {
  if (!s) return TC_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TC_ERR_INVALID_ARG;
    if (it->second.state != REQ_DONE) return TC_ERR_NOT_READY;
    s->pool.release(it->second.out);
    s->pool.release(it->second.tri);
    s->reqs.erase(it);
  }
  kick(s);  // freed memory may admit a waiting request
  return TC_OK;
}

tc_status tc_serve_stats(tc_server* s, tc_serve_stats_t* out) {
  if (!s || !out) return TC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->pending = static_cast<int64_t>(s->pending.size());
  int64_t running = 0;
  for (Slot* sl : s->slots) running += sl->ticket >= 0;
  out->running = running;
  out->pool_used = s->pool.used();
  out->pool_capacity = s->pool.capacity();
  out->edges_done = s->edges_done;
  return TC_OK;
}

}  // extern "C"
