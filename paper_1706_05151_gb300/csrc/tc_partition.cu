// Cost-balanced partition of the apex vertices: the paper's load-balancing
// step (Section "load balancing", Table "lbscheme").  Each processor of the
// paper counts the triangles of a contiguous range of core vertices; the
// ranges are chosen so that the sums of a per-vertex cost f(v) are about
// equal: F(t) = f(0) + ... + f(t), alpha = F(n-1) / p, and the boundary node
// of part j is the smallest v with F(v) >= j * alpha.
//
// GB300 mapping: one thread per vertex computes f(v) (TC_COST_WORK walks N_v
// and reads dhat_u from the offsets), the device scan gives F, and one thread
// per part finds its two boundary nodes by binary search over F, comparing
// p * F(v) with j * F(n-1) exactly in 128-bit integers.
#include "tc_internal.cuh"

namespace tc {

PartitionWs carve_partition(Carver& c, int32_t n) {
  PartitionWs w{};
  w.f = c.take<int64_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.F = c.take<int64_t>(static_cast<size_t>(n) + 1);
  w.scan = carve_scan(c, n);
  return w;
}

namespace {

__global__ void k_cost(int32_t n, int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                       const int32_t* __restrict__ deg, int cost, int64_t* __restrict__ f, uint32_t* err) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int64_t b = off[v], e = off[v + 1];
    if (b < 0 || e < b || e > m) {
      set_err(err, ERR_BAD_CSR);
      f[v] = 0;
      continue;
    }
    const int64_t dh = e - b;
    int64_t c = 0;
    switch (cost) {
      case TC_COST_VERTICES: c = 1; break;
      case TC_COST_DEGREE: c = deg[v]; break;
      case TC_COST_DHAT: c = dh; break;
      case TC_COST_DEG_DHAT: c = static_cast<int64_t>(deg[v]) * dh; break;
      case TC_COST_DHAT_SQ: c = dh * dh; break;
      default: {  // TC_COST_WORK: sum over u in N_v of (dhat_v + dhat_u)
        c = dh * dh;
        for (int64_t i = b; i < e; ++i) {
          const int32_t u = cols[i];
          if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(n)) {
            set_err(err, ERR_BAD_ID);
            continue;
          }
          c += off[u + 1] - off[u];
        }
      }
    }
    f[v] = c;
  }
}

// Smallest v in [0, n) with parts * F(v) >= j * F(n-1), F inclusive (= Fx[v + 1]
// of the exclusive scan Fx); n if there is none.
__device__ __forceinline__ int64_t boundary(const int64_t* Fx, int32_t n, int32_t parts, int64_t j) {
  const unsigned __int128 target = static_cast<unsigned __int128>(j) * static_cast<uint64_t>(Fx[n]);
  int64_t lo = 0, hi = n;  // answer in [lo, hi]
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (static_cast<unsigned __int128>(parts) * static_cast<uint64_t>(Fx[mid + 1]) >= target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__global__ void k_bounds(int32_t n, int32_t parts, const int64_t* __restrict__ Fx, int64_t* __restrict__ bounds,
                         uint64_t* __restrict__ part_cost) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j > parts) return;
  const int64_t lo = j == 0 ? 0 : (j == parts ? n : boundary(Fx, n, parts, j));
  bounds[j] = lo;
  if (part_cost && j < parts) {
    const int64_t hi = j + 1 == parts ? n : boundary(Fx, n, parts, j + 1);
    part_cost[j] = static_cast<uint64_t>(Fx[hi] - Fx[lo]);
  }
}

}  // namespace

cudaError_t launch_partition(Ctx* ctx, int32_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                             const int32_t* deg, int cost, int32_t parts, int64_t* bounds, uint64_t* part_cost,
                             PartitionWs ws, cudaStream_t s) {
  Stage st(ctx, s, "partition");
  if (n > 0) {
    const int grid = static_cast<int>(min64((static_cast<int64_t>(n) + 255) / 256,
                                            static_cast<int64_t>(ctx->sm_count) * 16));
    k_cost<<<grid, 256, 0, s>>>(n, m, offsets, cols, deg, cost, ws.f, ctx->d_err);
    counted(ctx);
  }
  cudaError_t e = exclusive_scan_i64(ws.f, ws.F, n, ws.scan, s);
  counted(ctx, n > 0 ? 3 : 1);
  if (e != cudaSuccess) return e;
  k_bounds<<<(parts + 1 + 255) / 256, 256, 0, s>>>(n, parts, ws.F, bounds, part_cost);
  counted(ctx);
  return cudaGetLastError();
}

}  // namespace tc
