// Edge sparsification (Section 9.1, Figure "sparsification"): each edge is
// kept with probability q, independently; the kept graph keeps the order of
// the original degrees (the lists are filtered, not re-oriented), and its
// triangle count T' gives the unbiased estimate T'/q^3.
//
// The coin of undirected edge {a, b} depends only on the edge:
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with 32-bit counter words
// (min(a,b), max(a,b), 0, 0) and key (lo32(seed), hi32(seed)); with r the top
// 53 bits of the output words x0:x1, keep iff r < t53, where
// t53 = ceil(q * 2^53) is computed on the host.  With partition-local coins
// (Section 9.2, tc_sparsify_count_part) the third counter word is the part's
// index, so each part draws its own coin for every edge it holds.  The 32-bit
// variant keeps the coin to two 32x32->64 products per round; the 64-bit one
// spends about four times the integer issue slots on emulated 64-bit products.
//
// GB300 mapping: consecutive vertices' lists are one contiguous run of cols,
// which a warp walks 32 ids at a time (coalesced).
//   k_mark     a warp takes 32 vertices; lanes find the source vertex of their
//              id by a 5-step search over the 32 list starts and write the
//              coin of the oriented edge (keep[] byte) and kept counts per vertex
//   scan       kept counts -> kept CSR offsets
//   k_compact  copy the kept ids, order preserved, into the kept CSR (a
//              stream compaction over runs of 64 vertices' lists)
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

// Top 53 bits of words 0 and 1 of Philox4x32-10 (ten rounds of two 32x32->64
// products, xor of the high halves with the other words and the round key,
// then a Weyl step of the key).
__device__ __forceinline__ uint64_t philox4x32_10_top53(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                        uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(M0) * c0;
    const uint64_t p1 = static_cast<uint64_t>(M1) * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
    c0 = n0;
    c1 = static_cast<uint32_t>(p1);
    c2 = n2;
    c3 = static_cast<uint32_t>(p0);
    k0 += W0;
    k1 += W1;
  }
  return (static_cast<uint64_t>(c0) << 21) | (c1 >> 11);
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
constexpr int kSpUnroll = 4;  // windows of 32 ids whose loads one warp keeps in flight
constexpr int kCompactSpan = 64;  // vertices per warp task, k_compact

__global__ void __launch_bounds__(kSpWarps * 32) k_mark(int32_t n, int64_t m, const int64_t* __restrict__ off,
                                                        const int32_t* __restrict__ cols, uint64_t t53,
                                                        uint64_t seed, uint32_t part, uint8_t* __restrict__ keep,
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
    // kSpUnroll windows of 32 ids per round: their loads are issued together
    for (int64_t base = r.first; base < r.last; base += 32 * kSpUnroll) {
      uint32_t u[kSpUnroll];
#pragma unroll
      for (int j = 0; j < kSpUnroll; ++j) {
        const int64_t idx = base + 32 * j + lane;
        u[j] = idx < r.last ? static_cast<uint32_t>(cols[idx]) : 0u;
      }
#pragma unroll
      for (int j = 0; j < kSpUnroll; ++j) {
        const int64_t idx = base + 32 * j + lane;
        if (idx < r.last) {
          const int s = owner(s_beg[wid], idx);
          const uint32_t v = static_cast<uint32_t>(vb + s);
          const uint64_t r53 = philox4x32_10_top53(v < u[j] ? v : u[j], v < u[j] ? u[j] : v, part, 0,
                                                   static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
          const bool k = r53 < t53;
          keep[idx] = k ? 1 : 0;
          if (k) atomicAdd(&s_cnt[wid][s], 1);
        }
      }
    }
    __syncwarp();
    if (vb + lane < n) kept_count[vb + lane] = s_cnt[wid][lane];
  }
}

// The kept ids of consecutive vertices are contiguous in the kept CSR, in the
// order of cols, so placing them is a stream compaction: the kept ids of
// vertices [vb, ve) go to new_cols[new_off[vb] ...] in order.  A warp takes
// kCompactSpan vertices at a time and advances one running count by the
// ballot of each window; no per-list bookkeeping is needed.
__global__ void __launch_bounds__(kSpWarps * 32) k_compact(int32_t n, int64_t m, const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ cols,
                                                           const uint8_t* __restrict__ keep,
                                                           const int64_t* __restrict__ new_off,
                                                           int32_t* __restrict__ new_cols, uint32_t* err) {
  const int lane = lane_id();
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t vb = gw * kCompactSpan; vb < n; vb += nwarps * kCompactSpan) {
    const int64_t ve = min64(n, vb + kCompactSpan);
    const int64_t first = off[vb], last = off[ve];
    const int64_t base = new_off[vb], base_end = new_off[ve];
    if (first < 0 || last < first || last > m || base < 0 || base_end < base || base_end - base > last - first) {
      if (lane == 0) set_err(err, ERR_BAD_CSR);
      continue;
    }
    const int64_t room = base_end - base;
    int64_t done = 0;  // kept ids of this span placed so far
    for (int64_t p0 = first; p0 < last; p0 += 32 * kSpUnroll) {
      bool kk[kSpUnroll];
      int32_t c[kSpUnroll];
#pragma unroll
      for (int j = 0; j < kSpUnroll; ++j) {
        const int64_t idx = p0 + 32 * j + lane;
        const bool act = idx < last;
        kk[j] = act && keep[idx];
        c[j] = act ? cols[idx] : 0;
      }
#pragma unroll
      for (int j = 0; j < kSpUnroll; ++j) {
        const unsigned mask = __ballot_sync(FULL, kk[j]);
        const int64_t r = done + __popc(mask & ((1u << lane) - 1u));
        if (kk[j]) {
          if (r < room) new_cols[base + r] = c[j];
          else set_err(err, ERR_BAD_CSR);  // keep bytes disagree with the kept counts
        }
        done += __popc(mask);
      }
    }
    if (lane == 0 && done != room) set_err(err, ERR_BAD_CSR);
  }
}

__global__ void k_copy_last(const int64_t* __restrict__ new_off, int32_t n, int64_t* __restrict__ kept_edges) {
  kept_edges[0] = new_off[n];
}

}  // namespace

cudaError_t launch_sparsify(Ctx* ctx, int32_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                            uint64_t threshold53, uint64_t seed, uint32_t part, SparsifyWs ws, int64_t* kept_edges,
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
