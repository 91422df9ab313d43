// Counting a CSR held in host memory (tc_count_streamed): the single-GPU form
// of the paper's space-efficient algorithm with non-overlapping partitions
// (its surrogate approach).  There, each processor keeps only the lists of its
// own vertices; for an edge (v, u) whose u belongs to another processor, N_v is
// sent to u's owner, which computes N_v intersected with N_u.  Here the device
// plays every processor in turn:
//
//   target ranges  consecutive vertices [u_k, u_k+1) whose lists N_u fill at
//                  most half of the device list buffer; one range at a time is
//                  copied in (one contiguous copy) and stays resident;
//   apex chunks    consecutive vertices [v_c, v_c+1) whose lists fill at most
//                  a quarter of the buffer: they stream past the resident range
//                  on a second stream, double-buffered (chunk c + 1 is copied
//                  while chunk c is counted), the "messages" of the paper;
//   counting       the unchanged apex-side kernels (k_count_tile for short apex
//                  lists, k_count_block for long ones) with the apex lists read
//                  from the chunk's slot, N_u read from the resident range, and
//                  only edges (v, u) with u in that range counted.
//
// A triangle v < u < w (in the order of Eq. (1)) is found at its apex v and
// its middle vertex u, i.e. in exactly one (range, chunk) pair, so the sums of
// T and T_v over all pairs are exact.  Host traffic: 4m bytes per range (the
// apex stream) plus 4m for the ranges, in copies of up to a quarter of the
// buffer each.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

StreamWs carve_stream(Carver& c, int32_t n, int64_t, size_t list_bytes) {
  StreamWs w{};
  const size_t n1 = static_cast<size_t>(n > 0 ? n : 1);
  w.offsets = c.take<int64_t>(n1 + 1);
  w.count.big_queue = c.take<int32_t>(n1);
  w.count.counters = c.take<uint32_t>(kCtrSlots);
  w.count.off32 = c.take<int32_t>(n1 + 1);
  w.list_ids = static_cast<int64_t>(list_bytes / sizeof(int32_t)) & ~int64_t(63);
  w.lists = c.take<int32_t>(static_cast<size_t>(w.list_ids > 0 ? w.list_ids : 1));
  return w;
}

namespace {

// Consecutive vertex ranges [b[i], b[i+1]) whose lists hold at most `cap` ids
// each (greedy, by binary search on the host offsets).  False if one list alone
// is longer than cap.  Ranges whose lists are all empty are dropped: such a
// vertex is neither an apex nor a middle vertex of any triangle.
bool cut_ranges(int32_t n, const int64_t* off, int64_t cap, std::vector<std::pair<int32_t, int32_t>>& out) {
  out.clear();
  int32_t lo = 0;
  while (lo < n) {
    const int64_t* hi_p = std::upper_bound(off + lo + 1, off + n + 1, off[lo] + cap);
    int32_t hi = static_cast<int32_t>(hi_p - off) - 1;  // largest hi with off[hi] <= off[lo] + cap
    if (hi <= lo) return false;                          // N_lo alone exceeds cap
    if (off[hi] > off[lo]) out.emplace_back(lo, hi);
    lo = hi;
  }
  return true;
}

}  // namespace

cudaError_t ensure_copy_stream(Ctx* ctx) {
  if (ctx->copy_stream) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
  for (int i = 0; e == cudaSuccess && i < 5; ++i) e = cudaEventCreateWithFlags(&ctx->copy_ev[i], cudaEventDisableTiming);
  return e;
}

cudaError_t launch_count_streamed(Ctx* ctx, int32_t n, int64_t m, const int64_t* off_h, const int32_t* cols_h,
                                  uint64_t* total, int64_t* tv, StreamWs w, cudaStream_t s, const char** why) {
  *why = nullptr;
  cudaError_t e;
  if ((e = cudaMemsetAsync(total, 0, sizeof(uint64_t), s)) != cudaSuccess) return e;
  if (tv && n > 0 && (e = cudaMemsetAsync(tv, 0, sizeof(int64_t) * static_cast<size_t>(n), s)) != cudaSuccess)
    return e;
  if (n <= 0 || m <= 0) return cudaSuccess;
  // the host copies are planned from the host offsets: they must describe m ids in order
  if (off_h[0] != 0 || off_h[n] != m) {
    *why = "offsets must start at 0 and end at m";
    return cudaErrorInvalidValue;
  }
  const int64_t resident_cap = w.list_ids / 2, slot_cap = w.list_ids / 4;
  std::vector<std::pair<int32_t, int32_t>> targets, chunks;
  if (!cut_ranges(n, off_h, resident_cap, targets) || !cut_ranges(n, off_h, slot_cap, chunks)) {
    *why = "a list is longer than a quarter of the list buffer";
    return cudaErrorMemoryAllocation;
  }
  for (const auto& r : chunks)  // the copies below read exactly these host ranges
    if (off_h[r.first] < 0 || off_h[r.second] > m || off_h[r.second] < off_h[r.first]) {
      *why = "offsets not monotone or outside [0, m]";
      return cudaErrorInvalidValue;
    }
  for (const auto& r : targets)
    if (off_h[r.first] < 0 || off_h[r.second] > m || off_h[r.second] < off_h[r.first]) {
      *why = "offsets not monotone or outside [0, m]";
      return cudaErrorInvalidValue;
    }
  if ((e = ensure_copy_stream(ctx)) != cudaSuccess) return e;
  cudaStream_t cs = ctx->copy_stream;
  cudaEvent_t copied[2] = {ctx->copy_ev[0], ctx->copy_ev[1]}, freed[2] = {ctx->copy_ev[2], ctx->copy_ev[3]};
  if ((e = cudaMemcpyAsync(w.offsets, off_h, sizeof(int64_t) * (static_cast<size_t>(n) + 1), cudaMemcpyHostToDevice,
                           s)) != cudaSuccess)
    return e;
  // the copy stream starts after everything the caller queued before (the workspace may be in use)
  if ((e = cudaEventRecord(ctx->copy_ev[4], s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(cs, ctx->copy_ev[4], 0)) != cudaSuccess) return e;
  // both slots start free
  for (int i = 0; i < 2; ++i)
    if ((e = cudaEventRecord(freed[i], s)) != cudaSuccess) return e;
  int32_t* resident = w.lists;
  int32_t* slot[2] = {w.lists + resident_cap, w.lists + resident_cap + slot_cap};
  bool off32_ready = false;
  int next = 0;
  for (const auto& t : targets) {
    const int64_t tb = off_h[t.first], tl = off_h[t.second] - tb;
    {
      Stage st(ctx, s, "stream.resident_copy");
      if ((e = cudaMemcpyAsync(resident, cols_h + tb, sizeof(int32_t) * static_cast<size_t>(tl),
                               cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    }
    for (const auto& c : chunks) {
      const int k = next;
      next ^= 1;
      const int64_t cb = off_h[c.first], cl = off_h[c.second] - cb;
      if ((e = cudaStreamWaitEvent(cs, freed[k], 0)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(slot[k], cols_h + cb, sizeof(int32_t) * static_cast<size_t>(cl),
                               cudaMemcpyHostToDevice, cs)) != cudaSuccess)
        return e;
      if ((e = cudaEventRecord(copied[k], cs)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(s, copied[k], 0)) != cudaSuccess) return e;
      CountArgs a{n, m, w.offsets, resident, reinterpret_cast<unsigned long long*>(total), tv, nullptr, 0};
      a.apex_cols = slot[k];
      a.apex_base = cb;
      a.apex_len = cl;
      a.cols_base = tb;
      a.cols_len = tl;
      a.u_lo = t.first;
      a.u_hi = t.second;
      a.v_lo = c.first;
      a.v_hi = c.second;
      a.off32_ready = off32_ready;
      if ((e = launch_count(ctx, tv ? MODE_LOCAL : MODE_COUNT, a, w.count, s)) != cudaSuccess) return e;
      off32_ready = true;
      if ((e = cudaEventRecord(freed[k], s)) != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

}  // namespace tc
