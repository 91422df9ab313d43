// Batched form (not in the paper): G independent graphs oriented and counted
// in one launch sequence.  The graphs are laid side by side as one disjoint
// union -- graph g owns the global ids [vbase[g], vbase[g+1]) -- so that
//   * the orientation of the union is exactly every graph's own orientation
//     (degrees and the order of Eq. (1) are per vertex), and
//   * one persistent counting launch walks every vertex of every graph through
//     the device-side vertex cursor and the queue of long lists, adding each
//     apex vertex's count to its graph's total.
//   k_translate   edges with local ids -> global ids, checked against n_g
//   k_graph_ids   graph id of every global vertex
#include "tc_internal.cuh"

namespace tc {

BatchWs carve_batch(Carver& c, int32_t n, int64_t m) {
  BatchWs w{};
  w.edges = c.take<int32_t>(static_cast<size_t>(2 * (m > 0 ? m : 1)));
  w.gid = c.take<int32_t>(static_cast<size_t>(n > 0 ? n : 1));
  w.orient = carve_orient(c, n, m);
  w.count = carve_count(c, n, m, false);
  return w;
}

namespace {

// Largest g in [0, G) with base[g] <= x (base non-decreasing, base[0] = 0).
__device__ __forceinline__ int32_t graph_of(const int64_t* __restrict__ base, int32_t G, int64_t x) {
  int32_t lo = 0, hi = G - 1;
  while (lo < hi) {
    const int32_t mid = lo + (hi - lo + 1) / 2;
    if (base[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_translate(int32_t G, int64_t E, const int64_t* __restrict__ vbase, const int64_t* __restrict__ ebase,
                            const int2* __restrict__ in, int2* __restrict__ out, uint32_t* err) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int32_t g = graph_of(ebase, G, e);
    const int64_t vb = vbase[g];
    const int64_t ng = vbase[g + 1] - vb;
    const int2 p = in[e];
    if (p.x < 0 || p.y < 0 || p.x >= ng || p.y >= ng) {
      set_err(err, ERR_BAD_ID);
      out[e] = make_int2(-1, -1);  // rejected again, without a read, by the orientation
    } else {
      out[e] = make_int2(static_cast<int32_t>(vb + p.x), static_cast<int32_t>(vb + p.y));
    }
  }
}

__global__ void k_graph_ids(int32_t G, int32_t N, const int64_t* __restrict__ vbase, int32_t* __restrict__ gid) {
  for (int32_t g = blockIdx.x; g < G; g += gridDim.x) {
    const int64_t b = max64(vbase[g], 0), e = min64(vbase[g + 1], N);  // clamped: bases are checked separately
    for (int64_t v = b + threadIdx.x; v < e; v += blockDim.x) gid[v] = g;
  }
}

__global__ void k_check_bases(int32_t G, int32_t N, int64_t E, const int64_t* __restrict__ vbase,
                              const int64_t* __restrict__ ebase, uint32_t* err) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x) {
    bool bad = false;
    if (g == 0) bad = vbase[0] != 0 || ebase[0] != 0;
    else bad = vbase[g] < vbase[g - 1] || ebase[g] < ebase[g - 1];
    if (g == G) bad |= vbase[G] != N || ebase[G] != E;
    if (bad) set_err(err, ERR_BAD_CSR);
  }
}

}  // namespace

cudaError_t launch_batch_prepare(Ctx* ctx, int32_t G, int32_t N, int64_t E, const int64_t* vbase,
                                 const int64_t* ebase, const int32_t* edges_local, BatchWs ws, cudaStream_t s) {
  {
    Stage st(ctx, s, "batch.check");
    k_check_bases<<<static_cast<int>(min64((G + 256) / 256, 1024)), 256, 0, s>>>(G, N, E, vbase, ebase, ctx->d_err);
    counted(ctx);
  }
  if (E > 0) {
    Stage st(ctx, s, "batch.translate");
    const int grid = static_cast<int>(min64((E + 255) / 256, static_cast<int64_t>(ctx->sm_count) * 16));
    k_translate<<<grid, 256, 0, s>>>(G, E, vbase, ebase, reinterpret_cast<const int2*>(edges_local),
                                     reinterpret_cast<int2*>(ws.edges), ctx->d_err);
    counted(ctx);
  }
  if (N > 0) {
    Stage st(ctx, s, "batch.graph_ids");
    k_graph_ids<<<static_cast<int>(min64(G, static_cast<int64_t>(ctx->sm_count) * 8)), 256, 0, s>>>(G, N, vbase, ws.gid);
    counted(ctx);
  }
  return cudaGetLastError();
}

}  // namespace tc
