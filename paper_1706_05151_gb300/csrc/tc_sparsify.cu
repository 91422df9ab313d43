// Edge sparsification (Section 9.1, Figure "sparsification"): each edge is
// kept with probability q, independently; the kept graph keeps the order of
// the original degrees (the lists are filtered, not re-oriented), and its
// triangle count T' gives the unbiased estimate T'/q^3.
//
// The coin of undirected edge {a, b} depends only on the edge:
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter
// (min(a,b), max(a,b), 0, 0) and key (seed, 0); keep iff (w0 >> 11) < t53,
// where t53 = ceil(q * 2^53) is computed on the host.  With partition-local
// coins (Section 9.2, tc_sparsify_count_part) the third counter word is the
// part's index, so each part draws its own coin for every edge it holds.
//
// GB300 mapping: a warp takes 32 consecutive vertices, whose lists are one
// contiguous run of cols; lanes walk that run 32 ids at a time (coalesced), and
// find their source vertex by a 5-step search over the 32 list starts.
//   k_mark     coin per oriented edge -> keep[] bytes and kept count per vertex
//   scan       kept counts -> kept CSR offsets
//   k_compact  copy the kept ids, order preserved, into the kept CSR
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

SparsifyWs carve_sparsify(Carver& c, int32_t n, int64_t m) {
  SparsifyWs w{};
  w.keep = c.take<uint8_t>(static_cast<size_t>(m > 0 ? m : 1));
  w.kept_count = c.take<int32_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.offsets = c.take<int64_t>(static_cast<size_t>(n) + 1);
  w.cols = c.take<int32_t>(static_cast<size_t>(m > 0 ? m : 1));
  w.scan = carve_scan(c, n);
  w.count = carve_count(c, n, m, false);
  return w;
}

namespace {

__device__ __forceinline__ uint64_t philox4x64_10_w0(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                     uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  return c0;
}

// Per-warp view of 32 consecutive vertices [vb, vb+32) and their id run.
struct Run {
  int64_t first, last;  // run of cols covered: [first, last)
};

__device__ __forceinline__ Run load_run(int32_t vb, int32_t n, int64_t m, const int64_t* __restrict__ off,
                                        int64_t* s_beg, uint32_t* err, bool& ok) {
  const int lane = lane_id();
  const int64_t v = static_cast<int64_t>(vb) + lane;
  int64_t b = 0, e = 0;
  bool bad = false;
  if (v < n) {
    b = off[v];
    e = off[v + 1];
    bad = b < 0 || e < b || e > m;
  }
  ok = !__any_sync(FULL, bad);
  if (!ok) {
    if (lane == 0) set_err(err, ERR_BAD_CSR);
    return Run{0, 0};
  }
  const int64_t first = __shfl_sync(FULL, b, 0);
  const int nv = static_cast<int>(min64(32, static_cast<int64_t>(n) - vb));
  const int64_t last = __shfl_sync(FULL, e, nv - 1);
  __syncwarp();
  s_beg[lane] = v < n ? b : last;  // lanes past the end never match
  __syncwarp();
  return Run{first, last};
}

__device__ __forceinline__ int owner(const int64_t* s_beg, int64_t idx) {
  int s = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1)
    if (s_beg[s + step] <= idx) s += step;
  return s;
}

constexpr int kSpWarps = 8;

__global__ void __launch_bounds__(kSpWarps * 32) k_mark(int32_t n, int64_t m, const int64_t* __restrict__ off,
                                                        const int32_t* __restrict__ cols, uint64_t t53,
                                                        uint64_t seed, uint64_t part, uint8_t* __restrict__ keep,
                                                        int32_t* __restrict__ kept_count, uint32_t* err) {
  __shared__ int64_t s_beg[kSpWarps][32];
  __shared__ int32_t s_cnt[kSpWarps][32];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t vb = gw * 32; vb < n; vb += nwarps * 32) {
    bool ok;
    const Run r = load_run(static_cast<int32_t>(vb), n, m, off, s_beg[wid], err, ok);
    if (!ok) continue;
    s_cnt[wid][lane] = 0;
    __syncwarp();
    for (int64_t idx = r.first + lane; idx < r.last; idx += 32) {
      const int s = owner(s_beg[wid], idx);
      const uint64_t v = static_cast<uint64_t>(vb + s);
      const uint64_t u = static_cast<uint64_t>(static_cast<uint32_t>(cols[idx]));
      const uint64_t w0 = philox4x64_10_w0(v < u ? v : u, v < u ? u : v, part, 0, seed, 0);
      const bool k = (w0 >> 11) < t53;
      keep[idx] = k ? 1 : 0;
      if (k) atomicAdd(&s_cnt[wid][s], 1);
    }
    __syncwarp();
    if (vb + lane < n) kept_count[vb + lane] = s_cnt[wid][lane];
  }
}

__global__ void __launch_bounds__(kSpWarps * 32) k_compact(int32_t n, int64_t m, const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ cols,
                                                           const uint8_t* __restrict__ keep,
                                                           const int64_t* __restrict__ new_off,
                                                           int32_t* __restrict__ new_cols, uint32_t* err) {
  __shared__ int64_t s_beg[kSpWarps][32];
  __shared__ int64_t s_run[kSpWarps][32];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t vb = gw * 32; vb < n; vb += nwarps * 32) {
    bool ok;
    const Run r = load_run(static_cast<int32_t>(vb), n, m, off, s_beg[wid], err, ok);
    if (!ok) continue;
    s_run[wid][lane] = (vb + lane < n) ? new_off[vb + lane] : 0;
    __syncwarp();
    for (int64_t w0 = r.first; w0 < r.last; w0 += 32) {
      const int64_t idx = w0 + lane;
      const bool act = idx < r.last;
      const int s = act ? owner(s_beg[wid], idx) : 31;
      const bool k = act && keep[idx];
      const unsigned mask = __ballot_sync(FULL, k);
      // lanes of the same list are contiguous in the window; count kept ones before me
      const int64_t seg_start = s_beg[wid][s];
      const int first_lane = static_cast<int>(max64(seg_start - w0, 0));
      const unsigned before = mask & ((1u << lane) - 1u) & ~((1u << first_lane) - 1u);
      const int64_t dst = s_run[wid][s] + __popc(before);
      if (k) new_cols[dst] = cols[idx];
      // the last lane of each list in this window advances that list's cursor
      const int s_next = __shfl_down_sync(FULL, s, 1);
      const bool last_of_seg = act && (lane == 31 || s_next != s || idx + 1 >= r.last);
      __syncwarp();
      if (last_of_seg) {
        const unsigned upto = (lane == 31) ? FULL : ((1u << (lane + 1)) - 1u);
        s_run[wid][s] += __popc(mask & upto & ~((1u << first_lane) - 1u));
      }
      __syncwarp();
    }
  }
}

__global__ void k_copy_last(const int64_t* __restrict__ new_off, int32_t n, int64_t* __restrict__ kept_edges) {
  kept_edges[0] = new_off[n];
}

}  // namespace

cudaError_t launch_sparsify(Ctx* ctx, int32_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                            uint64_t threshold53, uint64_t seed, uint64_t part, SparsifyWs ws, int64_t* kept_edges,
                            cudaStream_t s) {
  cudaError_t e;
  if (n > 0) {
    const int grid = persistent_blocks(ctx, reinterpret_cast<const void*>(&k_mark), kSpWarps * 32, 0);
    Stage st(ctx, s, "sparsify.mark");
    k_mark<<<grid, kSpWarps * 32, 0, s>>>(n, m, offsets, cols, threshold53, seed, part, ws.keep, ws.kept_count,
                                          ctx->d_err);
    counted(ctx);
  }
  {
    Stage st(ctx, s, "sparsify.scan");
    if ((e = exclusive_scan_i32(ws.kept_count, ws.offsets, n, ws.scan, s)) != cudaSuccess) return e;
    counted(ctx, n > 0 ? 3 : 1);
  }
  if (n > 0) {
    const int grid = persistent_blocks(ctx, reinterpret_cast<const void*>(&k_compact), kSpWarps * 32, 0);
    Stage st(ctx, s, "sparsify.compact");
    k_compact<<<grid, kSpWarps * 32, 0, s>>>(n, m, offsets, cols, ws.keep, ws.offsets, ws.cols, ctx->d_err);
    counted(ctx);
  }
  k_copy_last<<<1, 1, 0, s>>>(ws.offsets, n, kept_edges);
  counted(ctx);
  return cudaGetLastError();
}

}  // namespace tc
