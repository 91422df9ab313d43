// Orientation by the degree order: the preprocessing of NodeIteratorN
// (Figure 2): for each edge (u, v) store the later endpoint in the list of the
// earlier one, where u precedes v iff d_u < d_v, or d_u = d_v and u < v
// (Eq. (1)); then sort every list N_v ascending.  tc_orient_by replaces the
// degree by a caller's key (any total order: Theorem 1 keeps T; Theorem 3 says
// the degree order minimises sum_v d_v * dhat_v).
//
// GB300 mapping (all HBM/L2 traffic, no tensor cores):
//   k_degree        grid-stride over the edge list, 8-byte pair loads, RED.ADD
//                   into deg[] (4n bytes, L2-resident for n <= 2^25); the edge
//                   stream is read evict-first in all three passes (and cols
//                   written so) to keep deg[] in L2 for the random gathers
//   k_deg8          min(d_v, 255) per vertex (n bytes: L2-resident up to n ~ 2^27)
//   k_orient_count  same pass shape, gathers the saturated degrees of both
//                   endpoints (the full ones only when both are >= 255),
//                   counts dhat[src] and writes one bit per edge: which
//                   endpoint stores it
//   exclusive scan  offsets = scan(dhat)
//   k_scatter       third pass, no gathers: the edge's bit gives src;
//                   cols[offsets[src] + cursor[src]++] = dst
//   k_sort_small    one thread per vertex: lists of <= 32 ids sorted in
//                   registers by a bitonic network sized to the warp's longest
//                   list, the warp's run of lists staged in shared memory;
//                   longer lists are queued
//   k_sort_big      one block per queued list: bitonic sort in shared memory
// Sorted lists are checked for repeated ids (a repeated edge of the input).
#include <algorithm>
#include <climits>

#include "tc_internal.cuh"

namespace tc {

OrientWs carve_orient(Carver& c, int32_t n, int64_t m) {
  OrientWs w;
  w.cursor = c.take<int32_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.deg8 = c.take<uint8_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.fwd = c.take<uint32_t>(static_cast<size_t>(m > 0 ? (m + 31) / 32 : 1));
  w.big_queue = c.take<int32_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.mid_queue = c.take<int32_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.counters = c.take<uint32_t>(4);
  w.scan = carve_scan(c, n);
  return w;
}

namespace {

__device__ __forceinline__ bool precedes(int64_t da, int32_t a, int64_t db, int32_t b) {
  return da < db || (da == db && a < b);
}

__device__ __forceinline__ bool edge_ok(int2 p, int32_t n, uint32_t* err) {
  if (static_cast<uint32_t>(p.x) >= static_cast<uint32_t>(n) ||
      static_cast<uint32_t>(p.y) >= static_cast<uint32_t>(n)) {
    set_err(err, ERR_BAD_ID);
    return false;
  }
  if (p.x == p.y) {
    set_err(err, ERR_SELF_LOOP);
    return false;
  }
  return true;
}

// Runs of equal keys in consecutive lanes (the usual case for an edge list in
// adjacency-list order, where one endpoint repeats) are combined so that one
// lane per run does the atomic.  Returns the run length at the run's first
// lane and 0 elsewhere; *head_lane receives the first lane of this lane's run.
__device__ __forceinline__ int run_length(int32_t key, bool valid, int* head_lane) {
  const int lane = lane_id();
  const int32_t prev = __shfl_up_sync(FULL, key, 1);
  const bool pvalid = __shfl_up_sync(FULL, valid, 1);
  const bool head = lane == 0 || key != prev || valid != pvalid;
  const unsigned heads = __ballot_sync(FULL, head);
  *head_lane = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  if (!head || !valid) return 0;
  const unsigned after = heads & ~(0xffffffffu >> (31 - lane));
  const int end = after ? __ffs(after) - 1 : 32;
  return end - lane;
}

// Warp-strided edge loop: every lane of a warp runs the same iterations.
#define FOR_EDGES(e, m)                                                                            \
  for (int64_t e##0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) & ~int64_t(31); \
       e##0 < (m); e##0 += static_cast<int64_t>(gridDim.x) * blockDim.x)

__global__ void k_degree(const int2* __restrict__ edges, int64_t m, int32_t n, int32_t* __restrict__ deg,
                         uint32_t* err) {
  FOR_EDGES(e, m) {
    const int64_t e = e0 + lane_id();
    int2 p = make_int2(0, 0);
    bool ok = false;
    if (e < m) {
      p = __ldcs(edges + e);  // evict-first: the stream must not push deg[] out of L2
      ok = edge_ok(p, n, err);
    }
    int hl;
    const int cx = run_length(p.x, ok, &hl);
    if (cx) atomicAdd(&deg[p.x], cx);
    const int cy = run_length(p.y, ok, &hl);
    if (cy) atomicAdd(&deg[p.y], cy);
  }
}

__device__ __forceinline__ bool edge_valid(int2 p, int32_t n) {
  return static_cast<uint32_t>(p.x) < static_cast<uint32_t>(n) && static_cast<uint32_t>(p.y) < static_cast<uint32_t>(n) &&
         p.x != p.y;
}

constexpr int32_t kDeg8Max = 255;

// min(d_v, 255) per vertex: one byte per vertex, so the order's random gathers
// touch a quarter of the bytes of deg[] (the whole array stays in L2 for n up
// to about 2^27).
__global__ void k_deg8(int32_t n, const int32_t* __restrict__ deg, uint8_t* __restrict__ deg8) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride)
    deg8[v] = static_cast<uint8_t>(min(deg[v], kDeg8Max));
}

// Eq. (1) from the saturated bytes: they decide the order unless both degrees are
// at least 255, and then the full degrees are gathered.
__device__ __forceinline__ bool precedes_deg8(const uint8_t* deg8, const int32_t* deg, int32_t a, int32_t b) {
  const int32_t sa = __ldg(deg8 + a), sb = __ldg(deg8 + b);
  if (sa != sb) return sa < sb;
  if (sa < kDeg8Max) return a < b;
  return precedes(deg[a], a, deg[b], b);
}

// Counts dhat and records, one bit per edge, which endpoint stores the edge;
// k_scatter reads the bits instead of gathering the order's keys again.
__global__ void k_orient_count(const int2* __restrict__ edges, int64_t m, int32_t n,
                               const int32_t* __restrict__ deg, const uint8_t* __restrict__ deg8,
                               const int64_t* __restrict__ keys, int32_t* __restrict__ dhat,
                               uint32_t* __restrict__ fwd_bits) {
  FOR_EDGES(e, m) {
    const int64_t e = e0 + lane_id();
    int32_t src = 0;
    bool ok = false, fwd = false;
    if (e < m) {
      const int2 p = __ldcs(edges + e);
      ok = edge_valid(p, n);
      if (ok) {
        fwd = keys ? precedes(keys[p.x], p.x, keys[p.y], p.y) : precedes_deg8(deg8, deg, p.x, p.y);
        src = fwd ? p.x : p.y;
      }
    }
    const unsigned bits = __ballot_sync(FULL, fwd);
    if (lane_id() == 0 && e0 < m) fwd_bits[e0 >> 5] = bits;
    int hl;
    const int c = run_length(src, ok, &hl);
    if (c) atomicAdd(&dhat[src], c);
  }
}

__global__ void k_scatter(const int2* __restrict__ edges, int64_t m, int32_t n,
                          const uint32_t* __restrict__ fwd_bits, const int64_t* __restrict__ offsets,
                          int32_t* __restrict__ cursor, int32_t* __restrict__ cols, uint32_t* err) {
  FOR_EDGES(e, m) {
    const int lane = lane_id();
    const int64_t e = e0 + lane;
    int32_t src = 0, dst = 0;
    bool ok = false;
    if (e < m) {
      const int2 p = __ldcs(edges + e);
      ok = edge_valid(p, n);
      if (ok) {
        const bool fwd = (__ldg(fwd_bits + (e0 >> 5)) >> lane) & 1u;
        src = fwd ? p.x : p.y;
        dst = fwd ? p.y : p.x;
      }
    }
    int hl;
    const int c = run_length(src, ok, &hl);
    int64_t base = 0;
    if (c) base = offsets[src] + atomicAdd(&cursor[src], c);
    base = __shfl_sync(FULL, base, hl);
    if (ok) {
      const int64_t pos = base + (lane - hl);
      if (pos < offsets[src + 1]) __stcs(cols + pos, dst);
      else set_err(err, ERR_BAD_CSR);  // unreachable for a consistent count
    }
  }
}

// Bitonic sorting network over N registers (ascending), fully unrolled so the
// array stays in registers.
template <int N>
__device__ __forceinline__ void bitonic_regs(int32_t (&a)[N]) {
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          int32_t x = a[i], y = a[l];
          int32_t lo = min(x, y), hi = max(x, y);
          a[i] = up ? lo : hi;
          a[l] = up ? hi : lo;
        }
      }
    }
  }
}

template <int N>
__device__ __forceinline__ void sort_list_regs(int32_t* __restrict__ p, int len, uint32_t* err) {
  int32_t a[N];
#pragma unroll
  for (int i = 0; i < N; ++i) a[i] = i < len ? p[i] : INT_MAX;
  bitonic_regs<N>(a);
  bool dup = false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i < len) p[i] = a[i];
    if (i > 0 && i < len) dup |= a[i] == a[i - 1];
  }
  if (dup) set_err(err, ERR_DUPLICATE);
}

// One thread per vertex.  The network size is the warp's longest short list
// rounded up to a power of two, so one warp runs one network.  The 32 lists of
// a warp are one contiguous run of cols; when the run fits kSortStage ids the
// warp copies it to shared memory and back with coalesced accesses, so that
// the threads' element-wise loads and stores of their own lists stay on chip
// (otherwise each of those global stores is 32 scattered sector writes).
constexpr int kSortSmallThreads = 256;
constexpr int kSortStage = 1024;  // ids per warp staged in shared memory
__global__ void __launch_bounds__(kSortSmallThreads) k_sort_small(int32_t n, const int64_t* __restrict__ offsets,
                                                                  int32_t* __restrict__ cols,
                                                                  int32_t* __restrict__ big_queue,
                                                                  int32_t* __restrict__ mid_queue,
                                                                  uint32_t* __restrict__ counters, uint32_t* err) {
  __shared__ int32_t s_run[kSortSmallThreads / 32][kSortStage];
  int32_t* run = s_run[threadIdx.x >> 5];
  const int lane = lane_id();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  // whole warps iterate together so the warp-wide reduction below is legal
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n; base += stride) {
    const int64_t v = base + threadIdx.x;
    int len = 0;
    int64_t beg = 0, end = 0;
    if (v < n) {
      beg = offsets[v];
      end = offsets[v + 1];
      const int64_t l = end - beg;
      if (l > kSortWarpCap) {
        big_queue[atomicAdd(&counters[0], 1u)] = static_cast<int32_t>(v);
      } else if (l > 32) {
        mid_queue[atomicAdd(&counters[1], 1u)] = static_cast<int32_t>(v);
      } else {
        len = static_cast<int>(l);
      }
    }
    const int wmax = __reduce_max_sync(FULL, len);
    if (wmax <= 1) continue;
    // the warp's run [first, last): lanes past n hold no list
    const int nv = static_cast<int>(min64(32, n - (v - lane)));
    const int64_t first = __shfl_sync(FULL, beg, 0);
    const int64_t last = __shfl_sync(FULL, end, nv - 1);
    const bool staged = last - first <= kSortStage && first >= 0 && last >= first;
    int32_t* p = cols + beg;
    if (staged) {
      const int span = static_cast<int>(last - first);
      for (int i = lane; i < span; i += 32) run[i] = cols[first + i];
      __syncwarp();
      p = run + (beg - first);
    }
    if (wmax <= 2) sort_list_regs<2>(p, len, err);
    else if (wmax <= 4) sort_list_regs<4>(p, len, err);
    else if (wmax <= 8) sort_list_regs<8>(p, len, err);
    else if (wmax <= 16) sort_list_regs<16>(p, len, err);
    else sort_list_regs<32>(p, len, err);
    if (staged) {
      __syncwarp();
      const int span = static_cast<int>(last - first);
      for (int i = lane; i < span; i += 32) cols[first + i] = run[i];
      __syncwarp();
    }
  }
}

// One warp per queued list of 33 .. kSortWarpCap ids: bitonic sort in shared memory.
constexpr int kSortWarps = 8;
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_warp(const int64_t* __restrict__ offsets,
                                                               int32_t* __restrict__ cols,
                                                               const int32_t* __restrict__ mid_queue,
                                                               const uint32_t* __restrict__ counters, uint32_t* err) {
  __shared__ int32_t sbuf[kSortWarps][kSortWarpCap];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  int32_t* buf = sbuf[wid];
  const uint32_t qn = counters[1];
  for (uint32_t qi = blockIdx.x * kSortWarps + wid; qi < qn; qi += gridDim.x * kSortWarps) {
    const int32_t v = mid_queue[qi];
    const int64_t beg = offsets[v];
    const int len = static_cast<int>(offsets[v + 1] - beg);  // 33 .. kSortWarpCap by construction
    int P = 64;
    while (P < len) P <<= 1;
    for (int i = lane; i < P; i += 32) buf[i] = i < len ? cols[beg + i] : INT_MAX;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int l = i ^ j;
          if (l > i) {
            const bool up = (i & k) == 0;
            const int32_t x = buf[i], y = buf[l];
            if ((x > y) == up) {
              buf[i] = y;
              buf[l] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    bool dup = false;
    for (int i = lane; i < len; i += 32) {
      cols[beg + i] = buf[i];
      if (i > 0) dup |= buf[i] == buf[i - 1];
    }
    if (__any_sync(FULL, dup) && lane == 0) set_err(err, ERR_DUPLICATE);
    __syncwarp();
  }
}

// One block sorts a list longer than its shared memory holds, in place in
// global memory: bitonic sort in the form whose merges start by comparing each
// element with its mirror in the block, so every comparator puts the smaller
// key first and positions past the end act as +infinity without being stored.
__device__ void sort_in_place(int32_t* a, int32_t len, uint32_t* err) {
  int64_t P = 1;
  while (P < len) P <<= 1;
  for (int64_t k = 2; k <= P; k <<= 1) {
    for (int64_t j = k >> 1; j > 0; j >>= 1) {
      const int64_t mask = j == (k >> 1) ? k - 1 : j;  // first step of the merge: the mirror element
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const int64_t l = i ^ mask;
        if (l > i && l < len) {
          const int32_t x = a[i], y = a[l];
          if (x > y) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  bool dup = false;
  for (int64_t i = threadIdx.x + 1; i < len; i += blockDim.x) dup |= a[i] == a[i - 1];
  if (dup) set_err(err, ERR_DUPLICATE);
  __syncthreads();
}

// One block per queued list (kSortWarpCap+1 .. kSortBlockCap ids): bitonic sort in shared memory.
__global__ void __launch_bounds__(1024) k_sort_big(const int64_t* __restrict__ offsets, int32_t* __restrict__ cols,
                                                   const int32_t* __restrict__ big_queue,
                                                   const uint32_t* __restrict__ counters, uint32_t* err) {
  extern __shared__ int32_t sbuf[];
  const uint32_t qn = counters[0];
  for (uint32_t qi = blockIdx.x; qi < qn; qi += gridDim.x) {
    const int32_t v = big_queue[qi];
    const int64_t beg = offsets[v];
    const int64_t len = offsets[v + 1] - beg;
    if (len > kSortBlockCap) {  // longer than shared memory holds (any order): sort in place in global memory
      if (len > kMaxListLen) {
        if (threadIdx.x == 0) set_err(err, ERR_TOO_LONG);
        continue;
      }
      sort_in_place(cols + beg, static_cast<int32_t>(len), err);
      continue;
    }
    int P = 64;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) sbuf[i] = i < len ? cols[beg + i] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) {
            const bool up = (i & k) == 0;
            int32_t x = sbuf[i], y = sbuf[l];
            if ((x > y) == up) {
              sbuf[i] = y;
              sbuf[l] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    bool dup = false;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      cols[beg + i] = sbuf[i];
      if (i > 0) dup |= sbuf[i] == sbuf[i - 1];
    }
    if (dup) set_err(err, ERR_DUPLICATE);
    __syncthreads();
  }
}

bool g_big_attr_set[64] = {false};

}  // namespace

// Host ingest: edges per copy chunk (128 MB; about 0.6 ms on a 200 GB/s host link).
constexpr int64_t kIngestChunk = int64_t(1) << 24;

cudaError_t launch_orient(Ctx* ctx, int32_t n, int64_t m, const int32_t* edges, int64_t* offsets, int32_t* cols,
                          int32_t* deg, int32_t* dhat, OrientWs ws, cudaStream_t s, const int64_t* keys,
                          const int32_t* edges_host) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(deg, 0, sizeof(int32_t) * static_cast<size_t>(n), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(dhat, 0, sizeof(int32_t) * static_cast<size_t>(n), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.cursor, 0, sizeof(int32_t) * static_cast<size_t>(n), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.counters, 0, sizeof(uint32_t) * 4, s)) != cudaSuccess) return e;
  const int2* ep = reinterpret_cast<const int2*>(edges);
  const int threads = 512;
  const int grid_e = static_cast<int>(min64((m + threads - 1) / threads, static_cast<int64_t>(ctx->sm_count) * 8));
  if (m > 0) {
    {
      Stage st(ctx, s, "orient.degree");
      if (edges_host) {
        // chunk i is copied on the copy stream while the degree pass counts chunk i - 1
        if ((e = ensure_copy_stream(ctx)) != cudaSuccess) return e;
        cudaStream_t cs = ctx->copy_stream;
        // the copies start after the work queued before (which may still read `edges`)
        if ((e = cudaEventRecord(ctx->copy_ev[4], s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(cs, ctx->copy_ev[4], 0)) != cudaSuccess) return e;
        for (int64_t lo = 0; lo < m; lo += kIngestChunk) {
          const int64_t len = min64(kIngestChunk, m - lo);
          if ((e = cudaMemcpyAsync(const_cast<int32_t*>(edges) + 2 * lo, edges_host + 2 * lo,
                                   sizeof(int2) * static_cast<size_t>(len), cudaMemcpyHostToDevice, cs)) !=
              cudaSuccess)
            return e;
          if ((e = cudaEventRecord(ctx->copy_ev[0], cs)) != cudaSuccess) return e;
          if ((e = cudaStreamWaitEvent(s, ctx->copy_ev[0], 0)) != cudaSuccess) return e;
          const int grid_c = static_cast<int>(min64((len + threads - 1) / threads, static_cast<int64_t>(ctx->sm_count) * 8));
          k_degree<<<grid_c, threads, 0, s>>>(ep + lo, len, n, deg, ctx->d_err);
          counted(ctx);
        }
      } else {
        k_degree<<<grid_e, threads, 0, s>>>(ep, m, n, deg, ctx->d_err);
        counted(ctx);
      }
    }
    {
      Stage st(ctx, s, "orient.orient_count");
      if (!keys) {
        const int grid_v = static_cast<int>(min64((n + 255) / 256, static_cast<int64_t>(ctx->sm_count) * 16));
        k_deg8<<<grid_v, 256, 0, s>>>(n, deg, ws.deg8);
        counted(ctx);
      }
      k_orient_count<<<grid_e, threads, 0, s>>>(ep, m, n, deg, ws.deg8, keys, dhat, ws.fwd);
    }
    counted(ctx);
  }
  {
    Stage st(ctx, s, "orient.scan");
    if ((e = exclusive_scan_i32(dhat, offsets, n, ws.scan, s)) != cudaSuccess) return e;
    counted(ctx, n > 0 ? 3 : 1);
  }
  if (m > 0) {
    Stage st(ctx, s, "orient.scatter");
    k_scatter<<<grid_e, threads, 0, s>>>(ep, m, n, ws.fwd, offsets, ws.cursor, cols, ctx->d_err);
    counted(ctx);
  }
  if (n > 0) {
    const int grid_v = static_cast<int>(
        min64((n + kSortSmallThreads - 1) / kSortSmallThreads, static_cast<int64_t>(ctx->sm_count) * 16));
    {
      Stage st(ctx, s, "orient.sort_small");
      k_sort_small<<<grid_v, kSortSmallThreads, 0, s>>>(n, offsets, cols, ws.big_queue, ws.mid_queue, ws.counters, ctx->d_err);
    }
    {
      Stage st(ctx, s, "orient.sort_mid");
      const int grid_w = static_cast<int>(min64(static_cast<int64_t>(ctx->sm_count) * 8,
                                                max64(1, n / (33 * kSortWarps) + 1)));
      k_sort_warp<<<grid_w, kSortWarps * 32, 0, s>>>(offsets, cols, ws.mid_queue, ws.counters, ctx->d_err);
    }
    const size_t smem = sizeof(int32_t) * kSortBlockCap;
    if (ctx->device >= 0 && ctx->device < 64 && !g_big_attr_set[ctx->device]) {
      if ((e = cudaFuncSetAttribute(k_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem))) != cudaSuccess)
        return e;
      g_big_attr_set[ctx->device] = true;
    }
    {
      Stage st(ctx, s, "orient.sort_big");
      const int grid_b = static_cast<int>(min64(ctx->sm_count, max64(1, n / (kSortWarpCap + 1) + 1)));
      k_sort_big<<<grid_b, 1024, smem, s>>>(offsets, cols, ws.big_queue, ws.counters, ctx->d_err);
    }
    counted(ctx, 3);
  }
  return cudaGetLastError();
}

}  // namespace tc
