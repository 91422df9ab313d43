// The extern "C" entry points of libtc (declared in include/tc.h): argument
// checks on the host, workspace carving, device error-word handling, and the
// stream-ordered launch sequences of the other translation units.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tc_internal.cuh"

using tc::Carver;
using tc::Ctx;

struct tc_ctx : public Ctx {};

namespace {

tc_status fail(tc_ctx* ctx, tc_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->last_error, sizeof(ctx->last_error), fmt, ap);
    va_end(ap);
    // a call that fails inside a capture spoils the recorded sequence
    if (ctx->capturing && st != TC_OK && ctx->capture_status == TC_OK) ctx->capture_status = st;
  }
  return st;
}

tc_status cuda_fail(tc_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, TC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

tc_status status_from_bits(tc_ctx* ctx, uint32_t bits) {
  if (bits == 0) return TC_OK;
  if (bits & tc::ERR_BAD_ID) return fail(ctx, TC_ERR_INVALID_GRAPH, "vertex id outside [0, n)");
  if (bits & tc::ERR_SELF_LOOP) return fail(ctx, TC_ERR_INVALID_GRAPH, "self-loop in the edge list");
  if (bits & tc::ERR_DUPLICATE) return fail(ctx, TC_ERR_INVALID_GRAPH, "repeated edge in the edge list");
  if (bits & tc::ERR_BAD_CSR) return fail(ctx, TC_ERR_INVALID_GRAPH, "offsets not monotone or outside [0, m]");
  if (bits & tc::ERR_TOO_LONG) return fail(ctx, TC_ERR_UNSUPPORTED, "an oriented list exceeds the supported length");
  if (bits & tc::ERR_CAPACITY) return fail(ctx, TC_ERR_CAPACITY, "listing output buffer too small");
  if (bits & tc::ERR_TIMEOUT) return fail(ctx, TC_ERR_TIMEOUT, "a bounded device wait ran out");
  return fail(ctx, TC_ERR_CUDA, "unknown device error bits 0x%x", bits);
}

// Start of a call: in synchronous mode the error word is cleared for this call.
tc_status begin(tc_ctx* ctx, cudaStream_t s) {
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, TC_ERR_CUDA, "cudaSetDevice failed");
  if (!ctx->async) {
    cudaError_t e = cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "clear error word");
  }
  return TC_OK;
}

// End of a call: in synchronous mode wait for the stream and read the error word.
tc_status finish(tc_ctx* ctx, cudaStream_t s, cudaError_t launch) {
  if (launch != cudaSuccess) return cuda_fail(ctx, launch, "launch");
  if (ctx->async) return TC_OK;
  cudaError_t e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  return status_from_bits(ctx, *ctx->h_err);
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

tc_status check_ws(tc_ctx* ctx, tc_op op, int32_t n, int64_t m, void* ws, size_t ws_bytes) {
  size_t need = 0;
  tc_status st = tc_workspace_size(op, n, m, &need);
  if (st != TC_OK) return fail(ctx, st, "bad sizes n=%d m=%lld", n, static_cast<long long>(m));
  if (ws_bytes < need)
    return fail(ctx, TC_ERR_WORKSPACE, "workspace %zu bytes, need %zu", ws_bytes, need);
  if (need > 0 && (!ws || !aligned(ws, 256))) return fail(ctx, TC_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  return TC_OK;
}

tc_status check_graph(tc_ctx* ctx, const tc_graph* g) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (!g) return fail(ctx, TC_ERR_INVALID_ARG, "graph is NULL");
  if (g->n < 0 || g->m < 0) return fail(ctx, TC_ERR_INVALID_ARG, "negative n or m");
  if (!g->offsets) return fail(ctx, TC_ERR_INVALID_ARG, "offsets is NULL");
  if (g->m > 0 && !g->cols) return fail(ctx, TC_ERR_INVALID_ARG, "cols is NULL");
  if (!aligned(g->offsets, 8)) return fail(ctx, TC_ERR_INVALID_ARG, "offsets not 8-byte aligned");
  return TC_OK;
}

cudaEvent_t take_event(Ctx* ctx) {
  auto& pool = ctx->prof.pool;
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void resolve_stages(Ctx* ctx) {
  for (auto& p : ctx->prof.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
      ctx->prof.totals[p.index].ms += ms;
      ctx->prof.totals[p.index].calls += 1;
    }
    ctx->prof.pool.push_back(p.start);
    ctx->prof.pool.push_back(p.stop);
  }
  ctx->prof.pending.clear();
}

}  // namespace

namespace tc {

Stage::Stage(Ctx* ctx, cudaStream_t s, const char* name) : ctx_(ctx), s_(s) {
  if (!ctx->prof.on || ctx->capturing) return;
  auto& t = ctx->prof.totals;
  for (size_t i = 0; i < t.size(); ++i)
    if (t[i].name == name) index_ = static_cast<int>(i);
  if (index_ < 0) {
    t.push_back(StageTotal{name, 0.0, 0});
    index_ = static_cast<int>(t.size()) - 1;
  }
  start_ = take_event(ctx);
  cudaEventRecord(start_, s);
}

Stage::~Stage() {
  if (index_ < 0) return;
  cudaEvent_t stop = take_event(ctx_);
  cudaEventRecord(stop, s_);
  ctx_->prof.pending.push_back(PendingStage{index_, start_, stop});
}

}  // namespace tc

extern "C" {

const char* tc_version(void) { return "libtc 0.1 (sm_103a)"; }

const char* tc_status_string(tc_status s) {
  switch (s) {
    case TC_OK: return "ok";
    case TC_ERR_INVALID_ARG: return "invalid argument";
    case TC_ERR_INVALID_GRAPH: return "invalid graph";
    case TC_ERR_WORKSPACE: return "workspace too small";
    case TC_ERR_CAPACITY: return "output capacity too small";
    case TC_ERR_CUDA: return "CUDA error";
    case TC_ERR_UNSUPPORTED: return "unsupported size";
    case TC_ERR_TIMEOUT: return "timeout";
    case TC_ERR_REJECTED: return "rejected";
    case TC_ERR_NOT_READY: return "not ready";
  }
  return "unknown status";
}

tc_status tc_ctx_create(int device, tc_ctx** out) {
  if (!out) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return TC_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return TC_ERR_CUDA;
  tc_ctx* c = new tc_ctx();
  c->device = device;
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  c->sm_count = v > 0 ? v : 1;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = static_cast<size_t>(v);
  if (cudaMalloc(&c->d_err, sizeof(uint32_t)) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&c->h_err), sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess ||
      cudaMemset(c->d_err, 0, sizeof(uint32_t)) != cudaSuccess) {
    if (c->d_err) cudaFree(c->d_err);
    if (c->h_err) cudaFreeHost(c->h_err);
    delete c;
    return TC_ERR_CUDA;
  }
  *c->h_err = 0;
  *out = c;
  return TC_OK;
}

void tc_ctx_destroy(tc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  resolve_stages(ctx);
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  for (cudaEvent_t e : ctx->copy_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(ctx->d_err);
  cudaFreeHost(ctx->h_err);
  delete ctx;
}

tc_status tc_ctx_set_async(tc_ctx* ctx, int async) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (ctx->capturing) return fail(ctx, TC_ERR_INVALID_ARG, "capture in progress");
  ctx->async = async ? 1 : 0;
  return TC_OK;
}

tc_status tc_ctx_status(tc_ctx* ctx, tc_stream stream) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (ctx->capturing) return fail(ctx, TC_ERR_INVALID_ARG, "cannot synchronize while capturing");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status");
  return status_from_bits(ctx, *ctx->h_err);
}

tc_status tc_ctx_set_hub_min(tc_ctx* ctx, int32_t hub_min) {
  if (!ctx || hub_min < -1) return TC_ERR_INVALID_ARG;
  ctx->hub_min = hub_min;
  return TC_OK;
}

tc_status tc_ctx_set_tuning(tc_ctx* ctx, int32_t tile_max, int32_t grid_div) {
  if (!ctx || tile_max < 0 || tile_max > 512 || grid_div < 0 || grid_div > 64) return TC_ERR_INVALID_ARG;
  ctx->tile_max = tile_max;
  ctx->grid_div = grid_div > 0 ? grid_div : 1;
  return TC_OK;
}

tc_status tc_ctx_set_kernel_shape(tc_ctx* ctx, int32_t tile_ids, int32_t tile_windows, int32_t hash_batch,
                                  int32_t hash_windows) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  int shape = -1;
  if ((tile_ids == 0 && tile_windows == 0) || (tile_ids == 256 && tile_windows == 8)) shape = 0;
  else if (tile_ids == 256 && tile_windows == 4) shape = 1;
  else if (tile_ids == 128 && tile_windows == 8) shape = 2;
  if (shape < 0) return fail(ctx, TC_ERR_INVALID_ARG, "tile shape must be 256x8, 256x4 or 128x8");
  if (hash_batch != 0 && hash_batch != 16 && hash_batch != 32)
    return fail(ctx, TC_ERR_INVALID_ARG, "hash batch must be 16 or 32");
  if (hash_windows != 0 && hash_windows != 4 && hash_windows != 8)
    return fail(ctx, TC_ERR_INVALID_ARG, "hash windows must be 4 or 8");
  ctx->tile_shape = shape;
  ctx->hash_batch = hash_batch ? hash_batch : 32;
  ctx->hash_windows = hash_windows ? hash_windows : 4;
  return TC_OK;
}

tc_status tc_ctx_set_profiling(tc_ctx* ctx, int on) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  ctx->prof.on = on != 0;
  return TC_OK;
}

int tc_ctx_stage_count(tc_ctx* ctx) {
  if (!ctx) return 0;
  resolve_stages(ctx);
  return static_cast<int>(ctx->prof.totals.size());
}

tc_status tc_ctx_stage(tc_ctx* ctx, int i, const char** name, double* ms, int64_t* calls) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  resolve_stages(ctx);
  if (i < 0 || i >= static_cast<int>(ctx->prof.totals.size())) return TC_ERR_INVALID_ARG;
  const tc::StageTotal& t = ctx->prof.totals[static_cast<size_t>(i)];
  if (name) *name = t.name.c_str();
  if (ms) *ms = t.ms;
  if (calls) *calls = t.calls;
  return TC_OK;
}

tc_status tc_ctx_reset_stats(tc_ctx* ctx) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  resolve_stages(ctx);
  ctx->prof.totals.clear();
  ctx->launches = 0;
  return TC_OK;
}

int64_t tc_ctx_launches(const tc_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* tc_last_error(const tc_ctx* ctx) { return ctx ? ctx->last_error : "no context"; }

int tc_ctx_sm_count(const tc_ctx* ctx) { return ctx ? ctx->sm_count : 0; }

tc_status tc_workspace_size(tc_op op, int32_t n, int64_t m, size_t* bytes) {
  if (!bytes || n < 0 || m < 0) return TC_ERR_INVALID_ARG;
  Carver c(nullptr);
  switch (op) {
    case TC_OP_ORIENT: tc::carve_orient(c, n, m); break;
    case TC_OP_COUNT: tc::carve_count(c, n, m, false); break;
    case TC_OP_LIST: tc::carve_count(c, n, m, true); break;
    case TC_OP_SPARSIFY: tc::carve_sparsify(c, n, m); break;
    case TC_OP_BATCH: tc::carve_batch(c, n, m); break;
    case TC_OP_PARTITION: tc::carve_partition(c, n); break;
    default: return TC_ERR_INVALID_ARG;
  }
  *bytes = c.size();
  return TC_OK;
}

tc_status tc_orient(tc_ctx* ctx, int32_t n, int64_t m, const int32_t* edges, int64_t* offsets, int32_t* cols,
                    int32_t* deg, int32_t* dhat, void* ws, size_t ws_bytes, tc_stream stream) {
  return tc_orient_by(ctx, n, m, edges, nullptr, offsets, cols, deg, dhat, ws, ws_bytes, stream);
}

tc_status tc_orient_by(tc_ctx* ctx, int32_t n, int64_t m, const int32_t* edges, const int64_t* keys_dev,
                       int64_t* offsets, int32_t* cols, int32_t* deg, int32_t* dhat, void* ws, size_t ws_bytes,
                       tc_stream stream) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (keys_dev && !aligned(keys_dev, 8)) return fail(ctx, TC_ERR_INVALID_ARG, "keys not 8-byte aligned");
  if (n < 0 || m < 0) return fail(ctx, TC_ERR_INVALID_ARG, "negative n or m");
  if (!offsets || (n > 0 && (!deg || !dhat)) || (m > 0 && (!edges || !cols)))
    return fail(ctx, TC_ERR_INVALID_ARG, "NULL buffer");
  if (m > 0 && !aligned(edges, 8)) return fail(ctx, TC_ERR_INVALID_ARG, "edges not 8-byte aligned");
  if (!aligned(offsets, 8)) return fail(ctx, TC_ERR_INVALID_ARG, "offsets not 8-byte aligned");
  tc_status st = check_ws(ctx, TC_OP_ORIENT, n, m, ws, ws_bytes);
  if (st != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::OrientWs w = tc::carve_orient(c, n, m);
  return finish(ctx, s, tc::launch_orient(ctx, n, m, edges, offsets, cols, deg, dhat, w, s, keys_dev));
}

tc_status tc_orient_host(tc_ctx* ctx, int32_t n, int64_t m, const int32_t* edges_host, int32_t* edges_dev,
                         int64_t* offsets, int32_t* cols, int32_t* deg, int32_t* dhat, void* ws, size_t ws_bytes,
                         tc_stream stream) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (n < 0 || m < 0) return fail(ctx, TC_ERR_INVALID_ARG, "negative n or m");
  if (!offsets || (n > 0 && (!deg || !dhat)) || (m > 0 && (!edges_host || !edges_dev || !cols)))
    return fail(ctx, TC_ERR_INVALID_ARG, "NULL buffer");
  if (m > 0 && !aligned(edges_dev, 8)) return fail(ctx, TC_ERR_INVALID_ARG, "edges_dev not 8-byte aligned");
  if (!aligned(offsets, 8)) return fail(ctx, TC_ERR_INVALID_ARG, "offsets not 8-byte aligned");
  if (m > 0) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, edges_host) != cudaSuccess || at.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return fail(ctx, TC_ERR_INVALID_ARG, "edges_host is not page-locked host memory");
    }
  }
  tc_status st = check_ws(ctx, TC_OP_ORIENT, n, m, ws, ws_bytes);
  if (st != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::OrientWs w = tc::carve_orient(c, n, m);
  return finish(ctx, s, tc::launch_orient(ctx, n, m, edges_dev, offsets, cols, deg, dhat, w, s, nullptr, edges_host));
}

static tc_status count_impl(tc_ctx* ctx, const tc_graph* g, uint64_t* total_dev, int64_t* tv_dev, double* cc_dev,
                            void* ws, size_t ws_bytes, cudaStream_t s) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (!total_dev) return fail(ctx, TC_ERR_INVALID_ARG, "total_dev is NULL");
  const bool local = tv_dev != nullptr;
  if (cc_dev && (!local || (g->n > 0 && !g->deg)))
    return fail(ctx, TC_ERR_INVALID_ARG, "clustering needs tv_dev and g->deg");
  if ((st = check_ws(ctx, TC_OP_COUNT, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::CountWs w = tc::carve_count(c, g->n, g->m, false);
  cudaError_t e = cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s);
  if (e == cudaSuccess && local) e = cudaMemsetAsync(tv_dev, 0, sizeof(int64_t) * static_cast<size_t>(g->n), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clear outputs");
  tc::CountArgs a{g->n, g->m, g->offsets, g->cols, reinterpret_cast<unsigned long long*>(total_dev), tv_dev,
                  nullptr, 0};
  e = tc::launch_count(ctx, local ? tc::MODE_LOCAL : tc::MODE_COUNT, a, w, s);
  if (e == cudaSuccess && cc_dev) e = tc::launch_clustering(ctx, g->n, g->deg, tv_dev, cc_dev, s);
  return finish(ctx, s, e);
}

tc_status tc_count_range(tc_ctx* ctx, const tc_graph* g, int32_t v_begin, int32_t v_end, uint64_t* total_dev,
                         int64_t* tv_dev, void* ws, size_t ws_bytes, tc_stream stream) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (!total_dev) return fail(ctx, TC_ERR_INVALID_ARG, "total_dev is NULL");
  if (v_begin < 0 || v_end < v_begin || v_end > g->n)
    return fail(ctx, TC_ERR_INVALID_ARG, "need 0 <= v_begin <= v_end <= n");
  if ((st = check_ws(ctx, TC_OP_COUNT, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  if (v_begin == v_end) return finish(ctx, s, cudaSuccess);
  Carver c(ws);
  tc::CountWs w = tc::carve_count(c, g->n, g->m, false);
  tc::CountArgs a{g->n, g->m, g->offsets, g->cols, reinterpret_cast<unsigned long long*>(total_dev), tv_dev,
                  nullptr, 0};
  a.v_lo = v_begin;
  a.v_hi = v_end;
  return finish(ctx, s, tc::launch_count(ctx, tv_dev ? tc::MODE_LOCAL : tc::MODE_COUNT, a, w, s));
}

tc_status tc_count_streamed_workspace_size(int32_t n, int64_t m, size_t list_bytes, size_t* bytes) {
  if (!bytes) return TC_ERR_INVALID_ARG;
  *bytes = 0;
  if (n < 0 || m < 0) return TC_ERR_INVALID_ARG;
  Carver c(nullptr);
  tc::carve_stream(c, n, m, list_bytes);
  *bytes = c.size();
  return TC_OK;
}

tc_status tc_count_streamed(tc_ctx* ctx, int32_t n, int64_t m, const int64_t* offsets_host, const int32_t* cols_host,
                            uint64_t* total_dev, int64_t* tv_dev, size_t list_bytes, void* ws, size_t ws_bytes,
                            tc_stream stream) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (ctx->capturing) return fail(ctx, TC_ERR_INVALID_ARG, "tc_count_streamed plans its copies on the host: not inside a capture");
  if (n < 0 || m < 0) return fail(ctx, TC_ERR_INVALID_ARG, "negative n or m");
  if (!offsets_host || (m > 0 && !cols_host)) return fail(ctx, TC_ERR_INVALID_ARG, "offsets_host or cols_host is NULL");
  if (!total_dev) return fail(ctx, TC_ERR_INVALID_ARG, "total_dev is NULL");
  if (!aligned(total_dev, 8) || (tv_dev && !aligned(tv_dev, 8)))
    return fail(ctx, TC_ERR_INVALID_ARG, "total_dev / tv_dev not 8-byte aligned");
  size_t need = 0;
  tc_count_streamed_workspace_size(n, m, list_bytes, &need);
  if (ws_bytes < need) return fail(ctx, TC_ERR_WORKSPACE, "workspace %zu bytes, need %zu", ws_bytes, need);
  if (!ws || !aligned(ws, 256)) return fail(ctx, TC_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tc_status st = begin(ctx, s);
  if (st != TC_OK) return st;
  Carver c(ws);
  tc::StreamWs w = tc::carve_stream(c, n, m, list_bytes);
  const char* why = nullptr;
  const cudaError_t e = tc::launch_count_streamed(ctx, n, m, offsets_host, cols_host, total_dev, tv_dev, w, s, &why);
  if (why) {
    // nothing was copied: the plan was refused on the host
    return fail(ctx, e == cudaErrorMemoryAllocation ? TC_ERR_WORKSPACE : TC_ERR_INVALID_GRAPH, "%s", why);
  }
  return finish(ctx, s, e);
}

tc_status tc_partition(tc_ctx* ctx, const tc_graph* g, int32_t parts, int cost, int64_t* bounds_dev,
                       uint64_t* part_cost_dev, void* ws, size_t ws_bytes, tc_stream stream) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (parts < 1 || parts > 65536) return fail(ctx, TC_ERR_INVALID_ARG, "parts must be in [1, 65536]");
  if (cost < TC_COST_VERTICES || cost > TC_COST_WORK) return fail(ctx, TC_ERR_INVALID_ARG, "unknown cost function");
  if ((cost == TC_COST_DEGREE || cost == TC_COST_DEG_DHAT) && g->n > 0 && !g->deg)
    return fail(ctx, TC_ERR_INVALID_ARG, "this cost function needs g->deg");
  if (!bounds_dev) return fail(ctx, TC_ERR_INVALID_ARG, "bounds_dev is NULL");
  if ((st = check_ws(ctx, TC_OP_PARTITION, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::PartitionWs w = tc::carve_partition(c, g->n);
  return finish(ctx, s, tc::launch_partition(ctx, g->n, g->m, g->offsets, g->cols, g->deg, cost, parts, bounds_dev,
                                             part_cost_dev, w, s));
}

tc_status tc_count(tc_ctx* ctx, const tc_graph* g, uint64_t* total_dev, void* ws, size_t ws_bytes, tc_stream stream) {
  return count_impl(ctx, g, total_dev, nullptr, nullptr, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

tc_status tc_count_local(tc_ctx* ctx, const tc_graph* g, uint64_t* total_dev, int64_t* tv_dev, double* cc_dev,
                         void* ws, size_t ws_bytes, tc_stream stream) {
  if (ctx && !tv_dev) return fail(ctx, TC_ERR_INVALID_ARG, "tv_dev is NULL");
  return count_impl(ctx, g, total_dev, tv_dev, cc_dev, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

tc_status tc_list_count(tc_ctx* ctx, const tc_graph* g, int64_t* total_dev, void* ws, size_t ws_bytes,
                        tc_stream stream) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (!total_dev) return fail(ctx, TC_ERR_INVALID_ARG, "total_dev is NULL");
  if ((st = check_ws(ctx, TC_OP_LIST, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::CountWs w = tc::carve_count(c, g->n, g->m, true);
  cudaError_t e = cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clear outputs");
  tc::CountArgs a{g->n, g->m, g->offsets, g->cols, reinterpret_cast<unsigned long long*>(total_dev), nullptr,
                  nullptr, 0};
  // vertices with fewer than two out-neighbours are not visited: clear their edges' counts
  e = cudaMemsetAsync(w.ecount, 0, sizeof(int32_t) * static_cast<size_t>(g->m), s);
  if (e == cudaSuccess) e = tc::launch_count(ctx, tc::MODE_LIST_COUNT, a, w, s);
  if (e == cudaSuccess) e = tc::launch_list_offsets(ctx, g->m, w, s);
  return finish(ctx, s, e);
}

// The write pass; reuse_hub when the counting pass on the same workspace ran just before (same call).
static tc_status list_write_impl(tc_ctx* ctx, const tc_graph* g, int32_t* tri_dev, int64_t cap, void* ws, size_t ws_bytes,
                          tc_stream stream, bool reuse_hub) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (cap < 0 || (cap > 0 && !tri_dev)) return fail(ctx, TC_ERR_INVALID_ARG, "bad output buffer");
  if ((st = check_ws(ctx, TC_OP_LIST, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::CountWs w = tc::carve_count(c, g->n, g->m, true);
  tc::CountArgs a{g->n, g->m, g->offsets, g->cols, nullptr, nullptr, tri_dev, cap};
  a.reuse_hub = reuse_hub;
  return finish(ctx, s, tc::launch_count(ctx, tc::MODE_LIST_WRITE, a, w, s));
}

tc_status tc_list_write(tc_ctx* ctx, const tc_graph* g, int32_t* tri_dev, int64_t cap, void* ws, size_t ws_bytes,
                        tc_stream stream) {
  return list_write_impl(ctx, g, tri_dev, cap, ws, ws_bytes, stream, false);
}

tc_status tc_list(tc_ctx* ctx, const tc_graph* g, int32_t* tri_dev, int64_t cap, int64_t* count_out, void* ws,
                  size_t ws_bytes, tc_stream stream) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (ctx->capturing) return fail(ctx, TC_ERR_INVALID_ARG, "tc_list synchronizes: not capturable");
  if (!count_out) return fail(ctx, TC_ERR_INVALID_ARG, "count_out is NULL");
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if ((st = check_ws(ctx, TC_OP_LIST, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver c(ws);
  tc::CountWs w = tc::carve_count(c, g->n, g->m, true);
  // the total is the last entry of the edge offsets the count pass scans
  int64_t* total_dev = w.eoff + g->m;
  const int was_async = ctx->async;
  ctx->async = 0;
  st = tc_list_count(ctx, g, w.eoff + g->m, ws, ws_bytes, stream);
  ctx->async = was_async;
  if (st != TC_OK) return st;
  int64_t total = 0;
  cudaError_t e = cudaMemcpyAsync(&total, total_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read listing total");
  *count_out = total;
  if (total > cap) return fail(ctx, TC_ERR_CAPACITY, "listing needs %lld triples, capacity %lld",
                               static_cast<long long>(total), static_cast<long long>(cap));
  return list_write_impl(ctx, g, tri_dev, cap, ws, ws_bytes, stream, true);
}

tc_status tc_analyze(tc_ctx* ctx, const tc_graph* g, uint64_t* total_dev, int64_t* tv_dev, double* cc_dev,
                     int32_t* tri_dev, int64_t cap, int64_t* count_out, void* ws, size_t ws_bytes, tc_stream stream) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (ctx->capturing) return fail(ctx, TC_ERR_INVALID_ARG, "tc_analyze synchronizes: not capturable");
  if (!total_dev || !tv_dev || !count_out) return fail(ctx, TC_ERR_INVALID_ARG, "NULL output");
  if (cc_dev && g->n > 0 && !g->deg) return fail(ctx, TC_ERR_INVALID_ARG, "clustering needs g->deg");
  if (cap < 0 || (cap > 0 && !tri_dev)) return fail(ctx, TC_ERR_INVALID_ARG, "bad output buffer");
  if ((st = check_ws(ctx, TC_OP_LIST, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::CountWs w = tc::carve_count(c, g->n, g->m, true);
  cudaError_t e = cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tv_dev, 0, sizeof(int64_t) * static_cast<size_t>(g->n), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.ecount, 0, sizeof(int32_t) * static_cast<size_t>(g->m), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clear outputs");
  // pass 1: T, T_v and the triangles of each oriented edge (into w.ecount)
  tc::CountArgs a{g->n, g->m, g->offsets, g->cols, reinterpret_cast<unsigned long long*>(total_dev), tv_dev,
                  nullptr, 0};
  e = tc::launch_count(ctx, tc::MODE_LOCAL, a, w, s);
  if (e == cudaSuccess && cc_dev) e = tc::launch_clustering(ctx, g->n, g->deg, tv_dev, cc_dev, s);
  if (e == cudaSuccess) e = tc::launch_list_offsets(ctx, g->m, w, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "launch");
  // the total decides whether the triples fit: wait for it (and for the checks)
  int64_t total = 0;
  e = cudaMemcpyAsync(&total, w.eoff + g->m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read listing total");
  if (!ctx->async && (st = status_from_bits(ctx, *ctx->h_err)) != TC_OK) return st;
  *count_out = total;
  if (total > cap) return fail(ctx, TC_ERR_CAPACITY, "listing needs %lld triples, capacity %lld",
                               static_cast<long long>(total), static_cast<long long>(cap));
  // pass 2: write the triples (the hub schedule of pass 1 is still in the workspace)
  a.total = nullptr;
  a.tv = nullptr;
  a.tri = tri_dev;
  a.cap = cap;
  a.reuse_hub = true;
  return finish(ctx, s, tc::launch_count(ctx, tc::MODE_LIST_WRITE, a, w, s));
}

tc_status tc_batch(tc_ctx* ctx, int32_t G, int32_t N, int64_t E, const int64_t* vbase_dev, const int64_t* ebase_dev,
                   const int32_t* edges_dev, int64_t* offsets, int32_t* cols, int32_t* deg, int32_t* dhat,
                   uint64_t* totals_dev, int64_t* tv_dev, void* ws, size_t ws_bytes, tc_stream stream) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (G <= 0 || N < 0 || E < 0) return fail(ctx, TC_ERR_INVALID_ARG, "need G > 0, N >= 0, E >= 0");
  if (!vbase_dev || !ebase_dev || !offsets || !totals_dev || (N > 0 && (!deg || !dhat)) ||
      (E > 0 && (!edges_dev || !cols)))
    return fail(ctx, TC_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(vbase_dev, 8) || !aligned(ebase_dev, 8) || !aligned(offsets, 8) || (E > 0 && !aligned(edges_dev, 8)))
    return fail(ctx, TC_ERR_INVALID_ARG, "misaligned buffer");
  tc_status st = check_ws(ctx, TC_OP_BATCH, N, E, ws, ws_bytes);
  if (st != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::BatchWs w = tc::carve_batch(c, N, E);
  cudaError_t e = cudaMemsetAsync(totals_dev, 0, sizeof(uint64_t) * static_cast<size_t>(G), s);
  if (e == cudaSuccess && tv_dev) e = cudaMemsetAsync(tv_dev, 0, sizeof(int64_t) * static_cast<size_t>(N), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clear outputs");
  e = tc::launch_batch_prepare(ctx, G, N, E, vbase_dev, ebase_dev, edges_dev, w, s);
  if (e == cudaSuccess) e = tc::launch_orient(ctx, N, E, w.edges, offsets, cols, deg, dhat, w.orient, s);
  if (e == cudaSuccess) {
    tc::CountArgs a{N, E, offsets, cols, nullptr, tv_dev, nullptr, 0};
    a.graph_total = reinterpret_cast<unsigned long long*>(totals_dev);
    a.gid = w.gid;
    e = tc::launch_count(ctx, tv_dev ? tc::MODE_LOCAL : tc::MODE_COUNT, a, w.count, s);
  }
  return finish(ctx, s, e);
}

tc_status tc_sparsify_count_part(tc_ctx* ctx, const tc_graph* g, double q, uint64_t seed, int32_t part,
                                 int32_t v_begin, int32_t v_end, uint64_t* kept_tri_dev, int64_t* kept_edges_dev,
                                 void* ws, size_t ws_bytes, tc_stream stream) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (!(q >= 0.0 && q <= 1.0)) return fail(ctx, TC_ERR_INVALID_ARG, "q must be in [0, 1]");
  if (part < 0) return fail(ctx, TC_ERR_INVALID_ARG, "part must be >= 0");
  if (v_begin < 0 || v_end < v_begin || v_end > g->n)
    return fail(ctx, TC_ERR_INVALID_ARG, "need 0 <= v_begin <= v_end <= n");
  if (!kept_tri_dev || !kept_edges_dev) return fail(ctx, TC_ERR_INVALID_ARG, "NULL output");
  if ((st = check_ws(ctx, TC_OP_SPARSIFY, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::SparsifyWs w = tc::carve_sparsify(c, g->n, g->m);
  const uint64_t t53 = static_cast<uint64_t>(std::ceil(q * 9007199254740992.0));
  cudaError_t e = tc::launch_sparsify(ctx, g->n, g->m, g->offsets, g->cols, t53, seed, static_cast<uint32_t>(part), w,
                                      kept_edges_dev, s);
  if (e == cudaSuccess && v_end > v_begin) {
    tc::CountArgs a{g->n, g->m, w.offsets, w.cols, reinterpret_cast<unsigned long long*>(kept_tri_dev), nullptr,
                    nullptr, 0};
    a.v_lo = v_begin;
    a.v_hi = v_end;
    e = tc::launch_count(ctx, tc::MODE_COUNT, a, w.count, s);
  }
  return finish(ctx, s, e);
}

tc_status tc_sparsify_count(tc_ctx* ctx, const tc_graph* g, double q, uint64_t seed, uint64_t* kept_tri_dev,
                            int64_t* kept_edges_dev, void* ws, size_t ws_bytes, tc_stream stream) {
  tc_status st = check_graph(ctx, g);
  if (st != TC_OK) return st;
  if (!(q >= 0.0 && q <= 1.0)) return fail(ctx, TC_ERR_INVALID_ARG, "q must be in [0, 1]");
  if (!kept_tri_dev || !kept_edges_dev) return fail(ctx, TC_ERR_INVALID_ARG, "NULL output");
  if ((st = check_ws(ctx, TC_OP_SPARSIFY, g->n, g->m, ws, ws_bytes)) != TC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = begin(ctx, s)) != TC_OK) return st;
  Carver c(ws);
  tc::SparsifyWs w = tc::carve_sparsify(c, g->n, g->m);
  // keep iff (w0 >> 11) * 2^-53 < q  <=>  (w0 >> 11) < ceil(q * 2^53); q * 2^53 is exact
  const uint64_t t53 = static_cast<uint64_t>(std::ceil(q * 9007199254740992.0));
  cudaError_t e = cudaMemsetAsync(kept_tri_dev, 0, sizeof(uint64_t), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clear outputs");
  e = tc::launch_sparsify(ctx, g->n, g->m, g->offsets, g->cols, t53, seed, 0, w, kept_edges_dev, s);
  if (e == cudaSuccess) {
    tc::CountArgs a{g->n, g->m, w.offsets, w.cols, reinterpret_cast<unsigned long long*>(kept_tri_dev), nullptr,
                    nullptr, 0};
    e = tc::launch_count(ctx, tc::MODE_COUNT, a, w.count, s);
  }
  return finish(ctx, s, e);
}

// ---- captured launch sequences ----------------------------------------------

struct tc_exec {
  int device = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
};

tc_status tc_capture_begin(tc_ctx* ctx, tc_stream stream) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (!stream) return fail(ctx, TC_ERR_INVALID_ARG, "the legacy default stream cannot be captured");
  if (ctx->capturing) return fail(ctx, TC_ERR_INVALID_ARG, "capture already in progress");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, TC_ERR_CUDA, "cudaSetDevice failed");
  // tc_orient_host forks its copies onto the context's copy stream: create it outside the capture
  cudaError_t e = tc::ensure_copy_stream(ctx);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
  e = cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
  ctx->capturing = 1;
  ctx->capture_status = TC_OK;
  ctx->saved_async = ctx->async;
  ctx->async = 1;
  return TC_OK;
}

tc_status tc_capture_end(tc_ctx* ctx, tc_stream stream, tc_exec** out) {
  if (!ctx) return TC_ERR_INVALID_ARG;
  if (!ctx->capturing) return fail(ctx, TC_ERR_INVALID_ARG, "no capture in progress");
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &graph);
  ctx->capturing = 0;
  ctx->async = ctx->saved_async;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, "end capture");
  }
  if (ctx->capture_status != TC_OK) {  // last_error still holds the failed call's message
    cudaGraphDestroy(graph);
    return static_cast<tc_status>(ctx->capture_status);
  }
  if (!out) {
    cudaGraphDestroy(graph);
    return fail(ctx, TC_ERR_INVALID_ARG, "out is NULL");
  }
  size_t nodes = 0;
  e = cudaGraphGetNodes(graph, nullptr, &nodes);
  std::vector<cudaGraphNode_t> list(nodes);
  if (e == cudaSuccess && nodes) e = cudaGraphGetNodes(graph, list.data(), &nodes);
  int64_t kernels = 0;
  for (size_t i = 0; e == cudaSuccess && i < nodes; ++i) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(list[i], &t);
    if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, "instantiate capture");
  }
  tc_exec* x = new tc_exec;
  x->device = ctx->device;
  x->graph = graph;
  x->exec = exec;
  x->kernels = kernels;
  *out = x;
  return TC_OK;
}

tc_status tc_exec_launch(tc_exec* x, tc_stream stream) {
  if (!x) return TC_ERR_INVALID_ARG;
  if (cudaSetDevice(x->device) != cudaSuccess) return TC_ERR_CUDA;
  return cudaGraphLaunch(x->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

int64_t tc_exec_kernels(const tc_exec* x) { return x ? x->kernels : 0; }

void tc_exec_destroy(tc_exec* x) {
  if (!x) return;
  cudaSetDevice(x->device);
  if (x->exec) cudaGraphExecDestroy(x->exec);
  if (x->graph) cudaGraphDestroy(x->graph);
  delete x;
}

}  // extern "C"
