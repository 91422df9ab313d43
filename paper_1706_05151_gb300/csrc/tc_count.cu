// Counting, per-vertex counts, listing: the counting loop of NodeIteratorN
// (Figure 2): for v in V, for u in N_v, T += |N_v intersect N_u|.  Theorem 1:
// each triangle {x1 < x2 < x3} is found exactly once, at v = x1, u = x2, with
// w = x3 in N_v intersect N_u.  Per-vertex counts add one to each of v, u, w
// (Figure "localcount"); listing writes (v, u, w) (Figure "tlisting").
//
// GB300 mapping.  The work of apex vertex v is reading N_v and N_u for every
// u in N_v (Theorem 2's sum_v d_v * dhat_v reads); N_v is read once from HBM
// and served from shared memory afterwards.
//
//   k_count_tile   a warp takes 32 consecutive vertices (one coalesced load of
//                  their offsets); their lists, contiguous in cols, are staged
//                  as one shared-memory tile of up to kTile ids (lists longer
//                  than kTile are queued for k_count_block).  The tile's
//                  oriented edges (v, u) are processed 32 at a time: lane i
//                  loads the bounds of N_u for edge i, the 32 lists N_u are laid
//                  end to end and walked in 32-wide windows, kUnroll windows at
//                  once so each lane has kUnroll independent global loads in
//                  flight.  A candidate w of N_u finds its edge by a 5-step
//                  search of the batch's prefix sums and is binary-searched in
//                  N_v's slice of the tile.  Matches are summed per edge and per
//                  vertex in shared memory, per warp by shuffles and per block
//                  by one 64-bit atomicAdd.
//   k_count_block  one block per queued vertex: N_v staged in chunks of
//                  kBlockCap ids; the block's warps share the out-neighbour
//                  batches (a candidate outside the chunk's id range is skipped,
//                  so each is tested against exactly one chunk).
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kTile = 512;       // ids staged per warp; longer lists go to the block kernel
constexpr int kTileWarps = 8;    // warps per block, tile kernel
constexpr int kUnroll = 4;       // candidate windows in flight per lane
constexpr int kBlockCap = 8192;  // ids of N_v staged per pass, block kernel
constexpr int kBlockWarps = 8;   // warps per block, block kernel

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Largest i in [0, 32) with keys[i] <= x, for non-decreasing keys with keys[0] <= x.
template <class T>
__device__ __forceinline__ int search32(const T* keys, T x) {
  int s = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1)
    if (keys[s + step] <= x) s += step;
  return s;
}

// Is w in the sorted run base[0 .. len)?  `top` is a power of two with
// 2 * top > len, shared by the warp, so every lane runs the same steps.
__device__ __forceinline__ bool member(const int32_t* base, int len, int top, int32_t w) {
  int pos = 0;
  for (int step = top; step > 0; step >>= 1) {
    const int q = pos + step;
    if (q <= len && base[q - 1] <= w) pos = q;
  }
  return pos > 0 && base[pos - 1] == w;
}

// Bounds of N_u, checked against n and m: returns |N_u| and its start in *b,
// or 0 with an error bit.
__device__ __forceinline__ int32_t list_bounds(const CountArgs& a, int32_t u, int64_t& b, uint32_t* err) {
  b = 0;
  if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(a.n)) {
    set_err(err, ERR_BAD_ID);
    return 0;
  }
  const int64_t lo = a.offsets[u], hi = a.offsets[u + 1];
  if (lo < 0 || hi < lo || hi > a.m) {
    set_err(err, ERR_BAD_CSR);
    return 0;
  }
  if (hi - lo > kMaxListLen) {
    set_err(err, ERR_TOO_LONG);
    return 0;
  }
  b = lo;
  return static_cast<int32_t>(hi - lo);
}

__device__ __forceinline__ int32_t warp_incl_scan(int32_t x) {
  const int lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t t = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += t;
  }
  return x;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(FULL, x, d);
  return x;
}

// ---------------------------------------------------------------------------
// Tile kernel
// ---------------------------------------------------------------------------

struct EdgeBatch {     // one batch of up to 32 oriented edges (v, u) of a tile
  int64_t beg[32];     // start of N_u minus the edge's offset in the flattened batch
  int32_t exc[32];     // exclusive prefix of |N_u| over the batch
  int32_t u[32];
  int32_t lo[32];      // N_v's slice of the tile: [lo, lo + len)
  int32_t len[32];
  int32_t vl[32];      // chunk lane of v
  uint32_t cnt[32];    // matches of the edge
};

struct TileSmem {
  int32_t tile[kTile];
  int32_t vlo[32];     // tile start of each chunk lane's list (-1 before the group, > S after)
  uint32_t vcnt[32];   // triangles with apex v (chunk lane)
  int32_t vrun[32];    // listing: triples written so far per chunk lane
  EdgeBatch eb;
};

template <int MODE>
__device__ __forceinline__ void tile_edge_batch(TileSmem& sm, int t0, int S, int top, int32_t glen, int32_t vbase,
                                                const CountArgs& a, const CountWs& ws, uint32_t* err) {
  const int lane = lane_id();
  EdgeBatch& eb = sm.eb;
  const int t = t0 + lane;
  const bool act = t < S;
  int vl = 0;
  int32_t u = 0, len = 0;
  int64_t ub = 0;
  if (act) {
    vl = search32(sm.vlo, static_cast<int32_t>(t));
    u = sm.tile[t];
    len = list_bounds(a, u, ub, err);
  }
  const int32_t vlen = __shfl_sync(FULL, glen, vl);
  const int32_t incl = warp_incl_scan(len);
  const int32_t tot = __shfl_sync(FULL, incl, 31);
  const int32_t excl = incl - len;
  __syncwarp();
  eb.beg[lane] = ub - excl;
  eb.exc[lane] = excl;
  eb.u[lane] = u;
  eb.vl[lane] = vl;
  eb.lo[lane] = sm.vlo[vl];
  eb.len[lane] = vlen;
  eb.cnt[lane] = 0;
  __syncwarp();

  for (int32_t p0 = 0; p0 < tot; p0 += 32 * kUnroll) {
    int32_t w[kUnroll];
    int s[kUnroll];
    bool f[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      s[k] = 0;
      w[k] = -1;
      if (p < tot) {
        s[k] = search32(eb.exc, p);
        w[k] = a.cols[eb.beg[s[k]] + p];
      }
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      f[k] = p < tot && member(sm.tile + eb.lo[s[k]], eb.len[s[k]], top, w[k]);
      if (f[k]) {
        atomicAdd(&eb.cnt[s[k]], 1u);
        if (MODE == MODE_LOCAL) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + w[k]), 1ull);
      }
    }
    if (MODE == MODE_LIST_WRITE) {
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const unsigned fm = __ballot_sync(FULL, f[k]);
        if (!fm) continue;
        const int32_t p = p0 + 32 * k + lane;
        const int key = p < tot ? eb.vl[s[k]] : 32 + lane;
        const unsigned same = __match_any_sync(FULL, key);
        if (f[k]) {
          const int vlk = eb.vl[s[k]];
          const int32_t v = vbase + vlk;
          const int64_t idx = ws.voff[v] + sm.vrun[vlk] + __popc(fm & same & lanemask_lt());
          if (idx < a.cap) {
            a.tri[3 * idx] = v;
            a.tri[3 * idx + 1] = eb.u[s[k]];
            a.tri[3 * idx + 2] = w[k];
          } else {
            set_err(err, ERR_CAPACITY);
          }
        }
        __syncwarp();
        if (p < tot && lane == 31 - __clz(same)) sm.vrun[eb.vl[s[k]]] += __popc(fm & same);
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (act) {
    const uint32_t c = eb.cnt[lane];
    if (c) {
      if (MODE == MODE_LOCAL)
        atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + u), static_cast<unsigned long long>(c));
      atomicAdd(&sm.vcnt[vl], c);
    }
  }
  __syncwarp();
}

template <int MODE>
__global__ void __launch_bounds__(kTileWarps * 32) k_count_tile(CountArgs a, CountWs ws, uint32_t* err) {
  __shared__ TileSmem s_t[kTileWarps];
  __shared__ unsigned long long s_sum[kTileWarps];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  TileSmem& sm = s_t[wid];
  unsigned long long acc = 0;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&ws.counters[1], 32u);
    base = __shfl_sync(FULL, base, 0);
    if (base >= static_cast<uint32_t>(a.n)) break;
    const int32_t v = static_cast<int32_t>(base) + lane;
    const bool valid = v < a.n;
    int64_t b = 0, e = 0;
    if (valid) {
      b = a.offsets[v];
      e = a.offsets[v + 1];
      if (b < 0 || e < b || e > a.m) {
        set_err(err, ERR_BAD_CSR);
        b = e = 0;
      }
    }
    const int64_t d = e - b;
    const bool big = valid && d > kTile;
    const unsigned bigmask = __ballot_sync(FULL, big);
    if (bigmask) {
      uint32_t qb = 0;
      if (lane == 0) qb = atomicAdd(&ws.counters[0], static_cast<uint32_t>(__popc(bigmask)));
      qb = __shfl_sync(FULL, qb, 0);
      if (big) ws.big_queue[qb + __popc(bigmask & lanemask_lt())] = v;
    }
    // Groups: maximal runs of consecutive short lists whose ids fit one tile.
    int g0 = 0;
    while (g0 < 32) {
      const int32_t len = (lane >= g0 && valid && !big) ? static_cast<int32_t>(d) : 0;
      const int32_t incl = warp_incl_scan(len);
      const bool stop = lane >= g0 && (!valid || big || incl > kTile);
      const unsigned smask = __ballot_sync(FULL, stop);
      const int g1 = smask ? __ffs(smask) - 1 : 32;
      if (g1 == g0) {  // lane g0 is past the end or a queued long list
        if (!__shfl_sync(FULL, valid, g0)) break;
        ++g0;
        continue;
      }
      const bool in_group = lane >= g0 && lane < g1;
      const int32_t glen = in_group ? len : 0;
      const int32_t S = __shfl_sync(FULL, incl, g1 - 1);
      const int64_t start = __shfl_sync(FULL, b, g0);
      __syncwarp();
      bool bad = false;
      for (int t = lane; t < S; t += 32) {
        const int32_t x = a.cols[start + t];
        sm.tile[t] = x;
        bad |= static_cast<uint32_t>(x) >= static_cast<uint32_t>(a.n);
      }
      sm.vlo[lane] = lane < g0 ? -1 : (lane < g1 ? incl - len : S + 1);
      sm.vcnt[lane] = 0;
      sm.vrun[lane] = 0;
      if (__any_sync(FULL, bad)) {
        if (lane == 0) set_err(err, ERR_BAD_ID);
        g0 = g1;
        continue;
      }
      __syncwarp();
      const int maxlen = __reduce_max_sync(FULL, glen);
      const int top = maxlen > 0 ? 1 << (31 - __clz(maxlen)) : 0;
      for (int t0 = 0; t0 < S; t0 += 32)
        tile_edge_batch<MODE>(sm, t0, S, top, glen, static_cast<int32_t>(base), a, ws, err);
      if (in_group) {
        const uint32_t c = sm.vcnt[lane];
        if (MODE == MODE_LOCAL && c)
          atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + v), static_cast<unsigned long long>(c));
        if ((MODE == MODE_LIST_COUNT || MODE == MODE_LOCAL) && ws.vcount) ws.vcount[v] = c;
        acc += c;
      }
      __syncwarp();
      g0 = g1;
    }
  }
  acc = warp_sum64(acc);
  if (lane == 0) s_sum[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && a.total) {
    unsigned long long t = 0;
    for (int w = 0; w < kTileWarps; ++w) t += s_sum[w];
    if (t) atomicAdd(a.total, t);
  }
}

// ---------------------------------------------------------------------------
// Block kernel (lists longer than kTile)
// ---------------------------------------------------------------------------

struct BatchSmem {
  int64_t beg[32];
  int32_t exc[32];
  int32_t u[32];
};

// Intersect the staged sorted chunk sv[0..dv) (ids in [lo, hi]) with N_u for each
// u of ulist[0..nb) (nb <= 32).  Returns this lane's number of matches.
template <int MODE>
__device__ __forceinline__ uint32_t intersect_batch(const int32_t* sv, int dv, int top, int32_t lo, int32_t hi,
                                                    const int32_t* ulist, int nb, int32_t v, const CountArgs& a,
                                                    BatchSmem& bs, uint32_t* err, unsigned long long* cursor) {
  const int lane = lane_id();
  int32_t u = 0, len = 0;
  int64_t ub = 0;
  if (lane < nb) {
    u = ulist[lane];
    len = list_bounds(a, u, ub, err);
  }
  const int32_t incl = warp_incl_scan(len);
  const int32_t tot = __shfl_sync(FULL, incl, 31);
  const int32_t excl = incl - len;
  __syncwarp();
  bs.beg[lane] = ub - excl;
  bs.exc[lane] = excl;
  bs.u[lane] = u;
  __syncwarp();
  uint32_t cnt = 0;
  for (int32_t p0 = 0; p0 < tot; p0 += 32 * kUnroll) {
    int32_t w[kUnroll];
    int s[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      s[k] = 0;
      w[k] = lo - 1;
      if (p < tot) {
        s[k] = search32(bs.exc, p);
        w[k] = a.cols[bs.beg[s[k]] + p];
      }
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const bool found = w[k] >= lo && w[k] <= hi && member(sv, dv, top, w[k]);
      cnt += found ? 1u : 0u;
      if (MODE == MODE_LOCAL && found) {
        atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + bs.u[s[k]]), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + w[k]), 1ull);
      }
      if (MODE == MODE_LIST_WRITE) {
        const unsigned mask = __ballot_sync(FULL, found);
        if (mask) {
          unsigned long long b0 = 0;
          if (lane == 0) b0 = atomicAdd(cursor, static_cast<unsigned long long>(__popc(mask)));
          const int64_t base = static_cast<int64_t>(__shfl_sync(FULL, b0, 0));
          if (found) {
            const int64_t idx = base + __popc(mask & lanemask_lt());
            if (idx < a.cap) {
              a.tri[3 * idx] = v;
              a.tri[3 * idx + 1] = bs.u[s[k]];
              a.tri[3 * idx + 2] = w[k];
            } else {
              set_err(err, ERR_CAPACITY);
            }
          }
        }
      }
    }
  }
  return cnt;
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
      for (int64_t ub = static_cast<int64_t>(wid) * 32; ub < dv; ub += kBlockWarps * 32) {
        const int nb = static_cast<int>(min64(32, dv - ub));
        cv += intersect_batch<MODE>(sv, clen, top, lo, hi, a.cols + b + ub, nb, v, a, s_b[wid], err, &s_cursor);
      }
    }
    cv = warp_sum64(cv);
    if (lane == 0) s_red[wid] = cv;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kBlockWarps; ++w) t += s_red[w];
      if (MODE == MODE_LOCAL && t) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + v), t);
      if ((MODE == MODE_LIST_COUNT || MODE == MODE_LOCAL) && ws.vcount) ws.vcount[v] = static_cast<int64_t>(t);
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
    const int64_t t = tv[v];
    // C_v = 2 T_v / (d_v (d_v - 1)): both operands exact in double, one IEEE
    // division; T_v = 0 gives +0.0 exactly, so the division is skipped there
    cc[v] = (d < 2 || t == 0) ? 0.0 : __ddiv_rn(2.0 * static_cast<double>(t), static_cast<double>(d * (d - 1)));
  }
}

template <int MODE>
cudaError_t launch_mode(Ctx* ctx, const CountArgs& a, CountWs ws, cudaStream_t s) {
  static const char* kNames[4][2] = {{"count.tile", "count.block"},
                                     {"local.tile", "local.block"},
                                     {"list_count.tile", "list_count.block"},
                                     {"list_write.tile", "list_write.block"}};
  const int tgrid = persistent_blocks(ctx, reinterpret_cast<const void*>(&k_count_tile<MODE>), kTileWarps * 32, 0);
  {
    Stage st(ctx, s, kNames[MODE][0]);
    k_count_tile<MODE><<<tgrid, kTileWarps * 32, 0, s>>>(a, ws, ctx->d_err);
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
  const int grid = static_cast<int>(min64((n + 255) / 256, static_cast<int64_t>(ctx->sm_count) * 16));
  Stage st(ctx, s, "local.clustering");
  k_clustering<<<grid, 256, 0, s>>>(n, deg, tv, cc);
  counted(ctx);
  return cudaGetLastError();
}

}  // namespace tc
