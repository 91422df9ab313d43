// Counting, per-vertex counts, listing: the counting loop of NodeIteratorN
// (Figure 2): for v in V, for u in N_v, T += |N_v intersect N_u|.  Theorem 1:
// each triangle {x1 < x2 < x3} is found exactly once, at v = x1, u = x2, with
// w = x3 in N_v intersect N_u.  Per-vertex counts add one to each of v, u, w
// (Figure "localcount"); listing writes (v, u, w) (Figure "tlisting").
//
// GB300 mapping.  The work of apex vertex v is reading N_v once and N_u for
// every u in N_v (Theorem 2's sum_v d_v * dhat_v reads, of which N_v's share
// is served from shared memory here):
//   k_count_warp   one warp per vertex with |N_v| <= kWarpCap, vertices handed
//                  out in chunks by an atomic cursor (persistent grid).  N_v is
//                  staged in shared memory.  The lists N_u of a batch of up to
//                  32 out-neighbours are laid end to end and walked in 32-wide
//                  windows: lane i reads the i-th id of the window (coalesced),
//                  finds its list by a 5-step search of the batch's prefix
//                  sums, and binary-searches the id in the staged N_v.  Counts
//                  are summed by __reduce_add_sync per vertex and by one
//                  64-bit atomicAdd per block.
//   k_count_block  one block per vertex with |N_v| > kWarpCap (queued by the
//                  warp kernel): N_v staged in chunks of kBlockCap ids, the
//                  block's warps share the out-neighbour batches.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kWarpCap = 256;    // longest N_v the warp kernel stages
constexpr int kCountWarps = 8;   // warps per block, warp kernel
constexpr int kVChunk = 16;      // vertices per cursor grab
constexpr int kBlockCap = 8192;  // ids of N_v staged per pass, block kernel
constexpr int kBlockWarps = 8;   // warps per block, block kernel

struct BatchSmem {
  int64_t beg[32];  // start of N_u minus its offset in the flattened batch
  int32_t exc[32];  // exclusive prefix of |N_u| over the batch
  int32_t u[32];
};

// Intersect the staged sorted list sv[0..dv) with N_u for each u of ulist[0..nb)
// (nb <= 32).  Returns this lane's number of matches.
template <int MODE, bool FILTER, bool SHARED_CURSOR>
__device__ __forceinline__ uint32_t intersect_batch(const int32_t* sv, int dv, int top, int32_t lo, int32_t hi,
                                                    const int32_t* ulist, int nb, int32_t v, const CountArgs& a,
                                                    BatchSmem& bs, uint32_t* err, int64_t& opos,
                                                    unsigned long long* cursor) {
  const int lane = lane_id();
  int32_t u = 0;
  int64_t ubeg = 0;
  int32_t len = 0;
  if (lane < nb) {
    u = ulist[lane];
    if (static_cast<uint32_t>(u) < static_cast<uint32_t>(a.n)) {
      const int64_t b = a.offsets[u], e = a.offsets[u + 1];
      if (b >= 0 && b <= e && e <= a.m) {
        if (e - b <= kMaxListLen) {
          ubeg = b;
          len = static_cast<int32_t>(e - b);
        } else {
          set_err(err, ERR_TOO_LONG);
        }
      } else {
        set_err(err, ERR_BAD_CSR);
      }
    } else {
      set_err(err, ERR_BAD_ID);
    }
  }
  int32_t incl = len;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t t = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += t;
  }
  const int32_t tot = __shfl_sync(FULL, incl, 31);
  const int32_t excl = incl - len;
  __syncwarp();
  bs.beg[lane] = ubeg - excl;
  bs.exc[lane] = excl;
  bs.u[lane] = u;
  __syncwarp();

  uint32_t cnt = 0;
  for (int32_t p0 = 0; p0 < tot; p0 += 32) {
    const int32_t p = p0 + lane;
    bool found = false;
    int32_t w = 0;
    int s = 0;
    if (p < tot) {
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (bs.exc[s + step] <= p) s += step;
      w = a.cols[bs.beg[s] + p];
      if (!FILTER || (w >= lo && w <= hi)) {
        int pos = 0;
        for (int step = top; step > 0; step >>= 1) {
          const int q = pos + step;
          if (q <= dv && sv[q - 1] <= w) pos = q;
        }
        found = pos > 0 && sv[pos - 1] == w;
      }
    }
    cnt += found ? 1u : 0u;
    if (MODE == MODE_LOCAL && found) {
      atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + bs.u[s]), 1ull);
      atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + w), 1ull);
    }
    if (MODE == MODE_LIST_WRITE) {
      const unsigned mask = __ballot_sync(FULL, found);
      if (mask) {
        int64_t base;
        if (SHARED_CURSOR) {
          unsigned long long b0 = 0;
          if (lane == 0) b0 = atomicAdd(cursor, static_cast<unsigned long long>(__popc(mask)));
          base = static_cast<int64_t>(__shfl_sync(FULL, b0, 0));
        } else {
          base = opos;
          opos += __popc(mask);
        }
        if (found) {
          const int64_t idx = base + __popc(mask & ((1u << lane) - 1u));
          if (idx < a.cap) {
            a.tri[3 * idx] = v;
            a.tri[3 * idx + 1] = bs.u[s];
            a.tri[3 * idx + 2] = w;
          } else {
            set_err(err, ERR_CAPACITY);
          }
        }
      }
    }
  }
  return cnt;
}

template <int MODE>
__global__ void __launch_bounds__(kCountWarps * 32) k_count_warp(CountArgs a, CountWs ws, uint32_t* err) {
  __shared__ int32_t s_sv[kCountWarps][kWarpCap];
  __shared__ BatchSmem s_b[kCountWarps];
  __shared__ unsigned long long s_sum[kCountWarps];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  int32_t* sv = s_sv[wid];
  unsigned long long acc = 0;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&ws.counters[1], static_cast<uint32_t>(kVChunk));
    base = __shfl_sync(FULL, base, 0);
    if (base >= static_cast<uint32_t>(a.n)) break;
    const int32_t vend = static_cast<int32_t>(min64(static_cast<int64_t>(base) + kVChunk, a.n));
    for (int32_t v = static_cast<int32_t>(base); v < vend; ++v) {
      const int64_t b = a.offsets[v], e = a.offsets[v + 1];
      if (b < 0 || e < b || e > a.m) {
        if (lane == 0) set_err(err, ERR_BAD_CSR);
        continue;
      }
      const int64_t dv64 = e - b;
      if (dv64 < 2) {
        if (MODE == MODE_LIST_COUNT && lane == 0) ws.vcount[v] = 0;
        continue;
      }
      if (dv64 > kWarpCap) {
        if (lane == 0) ws.big_queue[atomicAdd(&ws.counters[0], 1u)] = v;
        continue;
      }
      const int dv = static_cast<int>(dv64);
      bool bad = false;
      for (int i = lane; i < dv; i += 32) {
        const int32_t x = a.cols[b + i];
        sv[i] = x;
        bad |= static_cast<uint32_t>(x) >= static_cast<uint32_t>(a.n);
      }
      if (__any_sync(FULL, bad)) {
        if (lane == 0) set_err(err, ERR_BAD_ID);
        continue;
      }
      __syncwarp();
      const int top = 1 << (31 - __clz(dv));
      int64_t opos = 0;
      if (MODE == MODE_LIST_WRITE) opos = ws.voff[v];
      uint32_t cnt = 0;
      for (int ub = 0; ub < dv; ub += 32)
        cnt += intersect_batch<MODE, false, false>(sv, dv, top, 0, 0, sv + ub, static_cast<int>(min64(32, dv - ub)), v, a,
                                                   s_b[wid], err, opos, nullptr);
      cnt = __reduce_add_sync(FULL, cnt);
      if (lane == 0) {
        if (MODE == MODE_LOCAL && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + v), cnt);
        if (MODE == MODE_LIST_COUNT) ws.vcount[v] = cnt;
        acc += cnt;
      }
      __syncwarp();
    }
  }
  if (lane == 0) s_sum[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && a.total) {
    unsigned long long t = 0;
    for (int w = 0; w < kCountWarps; ++w) t += s_sum[w];
    if (t) atomicAdd(a.total, t);
  }
}

template <int MODE>
__global__ void __launch_bounds__(kBlockWarps * 32) k_count_block(CountArgs a, CountWs ws, uint32_t* err) {
  extern __shared__ int32_t sv[];
  __shared__ BatchSmem s_b[kBlockWarps];
  __shared__ unsigned long long s_red[kBlockWarps];
  __shared__ unsigned long long s_cursor;
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  unsigned long long acc = 0;
  const uint32_t qn = ws.counters[0];
  for (uint32_t qi = blockIdx.x; qi < qn; qi += gridDim.x) {
    const int32_t v = ws.big_queue[qi];
    const int64_t b = a.offsets[v], e = a.offsets[v + 1];
    const int64_t dv = e - b;
    if (threadIdx.x == 0 && MODE == MODE_LIST_WRITE) s_cursor = static_cast<unsigned long long>(ws.voff[v]);
    unsigned long long cv = 0;
    for (int64_t c0 = 0; c0 < dv; c0 += kBlockCap) {
      const int clen = static_cast<int>(min64(kBlockCap, dv - c0));
      __syncthreads();
      bool bad = false;
      for (int i = threadIdx.x; i < clen; i += blockDim.x) {
        const int32_t x = a.cols[b + c0 + i];
        sv[i] = x;
        bad |= static_cast<uint32_t>(x) >= static_cast<uint32_t>(a.n);
      }
      if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) set_err(err, ERR_BAD_ID);
        break;
      }
      const int32_t lo = sv[0], hi = sv[clen - 1];
      const int top = 1 << (31 - __clz(clen));
      int64_t unused = 0;
      for (int64_t ub = static_cast<int64_t>(wid) * 32; ub < dv; ub += kBlockWarps * 32) {
        const int nb = static_cast<int>(min64(32, dv - ub));
        cv += intersect_batch<MODE, true, true>(sv, clen, top, lo, hi, a.cols + b + ub, nb, v, a, s_b[wid], err,
                                                unused, &s_cursor);
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cv += __shfl_down_sync(FULL, cv, d);
    if (lane == 0) s_red[wid] = cv;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kBlockWarps; ++w) t += s_red[w];
      if (MODE == MODE_LOCAL && t) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + v), t);
      if (MODE == MODE_LIST_COUNT) ws.vcount[v] = static_cast<int64_t>(t);
      acc += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && acc && a.total) atomicAdd(a.total, acc);
}

__global__ void k_clustering(int32_t n, const int32_t* __restrict__ deg, const int64_t* __restrict__ tv,
                             double* __restrict__ cc) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int64_t d = deg[v];
    // C_v = 2 T_v / (d_v (d_v - 1)): both operands exact in double, one IEEE division
    cc[v] = d < 2 ? 0.0 : __ddiv_rn(2.0 * static_cast<double>(tv[v]), static_cast<double>(d * (d - 1)));
  }
}

template <int MODE>
cudaError_t launch_mode(Ctx* ctx, const CountArgs& a, CountWs ws, cudaStream_t s) {
  static const char* kNames[4][2] = {{"count.warp", "count.block"},
                                     {"local.warp", "local.block"},
                                     {"list_count.warp", "list_count.block"},
                                     {"list_write.warp", "list_write.block"}};
  const int wgrid = persistent_blocks(ctx, reinterpret_cast<const void*>(&k_count_warp<MODE>), kCountWarps * 32, 0);
  {
    Stage st(ctx, s, kNames[MODE][0]);
    k_count_warp<MODE><<<wgrid, kCountWarps * 32, 0, s>>>(a, ws, ctx->d_err);
  }
  const size_t smem = sizeof(int32_t) * kBlockCap;
  const int bgrid =
      persistent_blocks(ctx, reinterpret_cast<const void*>(&k_count_block<MODE>), kBlockWarps * 32, smem);
  {
    Stage st(ctx, s, kNames[MODE][1]);
    k_count_block<MODE><<<bgrid, kBlockWarps * 32, smem, s>>>(a, ws, ctx->d_err);
  }
  counted(ctx, 2);
  return cudaGetLastError();
}

}  // namespace

CountWs carve_count(Carver& c, int32_t n, bool listing) {
  CountWs w{};
  w.big_queue = c.take<int32_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.counters = c.take<uint32_t>(4);
  if (listing) {
    w.vcount = c.take<int64_t>(static_cast<size_t>(n) + 1);
    w.voff = c.take<int64_t>(static_cast<size_t>(n) + 1);
    w.scan = carve_scan(c, n);
  }
  return w;
}

int persistent_blocks(Ctx* ctx, const void* kernel, int threads, size_t dyn_smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * ctx->sm_count;
}

cudaError_t launch_count(Ctx* ctx, CountMode mode, const CountArgs& a, CountWs ws, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ws.counters, 0, sizeof(uint32_t) * 4, s);
  if (e != cudaSuccess) return e;
  if (a.n <= 0) return cudaGetLastError();
  switch (mode) {
    case MODE_COUNT: return launch_mode<MODE_COUNT>(ctx, a, ws, s);
    case MODE_LOCAL: return launch_mode<MODE_LOCAL>(ctx, a, ws, s);
    case MODE_LIST_COUNT: return launch_mode<MODE_LIST_COUNT>(ctx, a, ws, s);
    case MODE_LIST_WRITE: return launch_mode<MODE_LIST_WRITE>(ctx, a, ws, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_clustering(Ctx* ctx, int32_t n, const int32_t* deg, const int64_t* tv, double* cc,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = static_cast<int>(min64((n + 255) / 256, 4096));
  Stage st(ctx, s, "local.clustering");
  k_clustering<<<grid, 256, 0, s>>>(n, deg, tv, cc);
  counted(ctx);
  return cudaGetLastError();
}

}  // namespace tc
