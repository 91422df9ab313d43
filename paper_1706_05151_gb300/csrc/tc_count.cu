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
//                  as one shared-memory tile of up to 256 ids (lists longer
//                  than tile_max are queued for k_count_block).  The tile's
//                  oriented edges (v, u) are processed 32 at a time.  Short
//                  lists N_u are laid end to end and walked in 32-wide windows
//                  (an owner table maps a position to its edge), 8 (or 4)
//                  windows at once so each lane has that many independent
//                  global loads in flight; long lists are walked one edge at a
//                  time.  Every candidate w first meets a bitmap filter of the
//                  tile (one shared load and a bit test); the survivors are
//                  queued and checked exactly, 32 at a time, by binary search
//                  in N_v's slice of the tile.
//   k_count_block  one block per queued vertex: N_v is hashed, in chunks, into
//                  a shared-memory two-choice (cuckoo) table at load factor at
//                  most 1/4, so membership is exact in two independent loads;
//                  the block's warps take the out-neighbour batches in turn.
//   hub side       an edge (v, u) whose N_u is long (>= hub_min ids) and longer
//                  than N_v is counted from u's side: k_count_block<MODE, true>
//                  hashes N_u once per segment of such edges and streams the
//                  short N_v lists (k_hub_list / k_hub_fill / k_hub_items build
//                  the segments).
// Counts are summed per edge and per vertex in shared memory, per warp by
// shuffles and per block by one 64-bit atomicAdd.
//
// Listing is two-pass: pass 1 records the triangles of every oriented edge,
// a scan turns them into output offsets, and pass 2 revisits only edges that
// have triangles, writing edge e's triangles at offset eoff[e] in candidate
// order -- fixed positions, no atomics, the same output every run.
#include <algorithm>

#include <type_traits>

#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kTileWarps = 4;        // warps per block, tile kernel
constexpr int kShortLen = 32;        // N_u shorter than this is walked end to end with others
constexpr int kOwnCap = 32 * kShortLen;
// Shapes of the tile kernel the autotuner chooses among: ids staged per warp,
// candidate windows in flight per lane, filter bits (log2) per tile -- 32 bits
// per staged id, so that at most 1/32 of the candidates pass the filter falsely.
template <int IDS, int UNROLL, int BITS>
struct TileShape {
  static constexpr int kIds = IDS, kUnroll = UNROLL, kBitsLog2 = BITS;
};
using TileShapeA = TileShape<256, 8, 13>;  // the default
using TileShapeB = TileShape<256, 4, 13>;
using TileShapeC = TileShape<128, 8, 12>;
constexpr int kBlockWarps = 8;       // warps per block, block kernel
// walked lists a warp takes at a time in the block and hub kernels: at most the
// kernel's BATCH (32 or 16, chosen by the autotuner), at least this many near
// the end of a chunk
constexpr int kMinHashBatch = 4;
constexpr uint64_t kPtrMask = (uint64_t(1) << 58) - 1;  // packed list address: byte address below bit 58
constexpr uint32_t kSaltMix = 0x7C000000u;              // filter salt (0..31) << 26: bits 58..62 of the packed word
constexpr int kHubMinDefault = 64;   // default hub_min: lists of at least this many ids take their in-edges

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
  if (u < a.u_lo || u >= a.u_hi) return 0;  // N_u is not in this call's part of the lists
  // the int32 copy, when there is one, halves the bytes of this random read; it is read
  // about twice per oriented edge, so its lines are the last this kernel lets L2 evict
  const uint64_t keep = l2_policy_evict_last();
  const int64_t lo = a.off32 ? ld_nc_hint(a.off32 + u, keep) : ld_nc_hint(a.offsets + u, keep);
  const int64_t hi = a.off32 ? ld_nc_hint(a.off32 + u + 1, keep) : ld_nc_hint(a.offsets + u + 1, keep);
  if (lo < 0 || hi < lo || hi > a.m) {
    set_err(err, ERR_BAD_CSR);
    return 0;
  }
  if (hi - lo > kMaxListLen) {
    set_err(err, ERR_TOO_LONG);
    return 0;
  }
  if (lo - a.cols_base < 0 || hi - a.cols_base > a.cols_len) {  // outside the array that holds N_u
    set_err(err, ERR_BAD_CSR);
    return 0;
  }
  b = lo - a.cols_base;
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

// Multiplicative hash of (salt, id) onto a 2^LOG2-bit filter; mix = salt << 26.
template <int LOG2>
__device__ __forceinline__ uint32_t fbit(int32_t w, uint32_t mix) {
  return ((static_cast<uint32_t>(w) ^ mix) * 0x9E3779B1u) >> (32 - LOG2);
}

template <int LOG2>
__device__ __forceinline__ bool ftest(const uint32_t* bits, int32_t w, uint32_t mix) {
  const uint32_t h = fbit<LOG2>(w, mix);
  // the funnel shift takes its amount modulo 32: bit (h & 31) of the word with no mask
  return __funnelshift_r(bits[h >> 5], 0u, h) & 1u;
}

template <int LOG2>
__device__ __forceinline__ void fset(uint32_t* bits, int32_t w, uint32_t mix) {
  const uint32_t h = fbit<LOG2>(w, mix);
  atomicOr(&bits[h >> 5], 1u << (h & 31));
}

// Per-warp state of one batch of up to 32 oriented edges (v, u), one per lane.
// Each kernel keeps only the fields it reads: shared memory and the L1 cache
// share one array per SM, and the tile kernel's candidate reads live in L1.
struct HashBatch {  // block and hub kernels
  static constexpr bool kTile = false, kWrite = false;
  int64_t beg[32];                  // short list: start of N_u minus its flattened offset; long list: start of N_u
  uint32_t cnt[32];                 // matches of the edge
  alignas(4) uint8_t own[kOwnCap];  // flattened position -> edge, short lists
};

struct TileBatch {  // tile kernel, counting passes
  static constexpr bool kTile = true, kWrite = false;
  uint64_t pk[32];    // byte address of the list's first flattened position below bit 58, filter salt above
  int32_t lo[32];     // N_v's slice [lo, lo + len) of the tile
  int32_t len[32];
  int32_t salt[32];   // filter salt (chunk lane of v)
  uint32_t cnt[32];   // matches of the edge
  alignas(4) uint8_t own[kOwnCap];
};

struct TileWriteBatch {  // tile kernel, listing write pass
  static constexpr bool kTile = true, kWrite = true;
  uint64_t pk[32];
  int64_t ebase[32];  // output offset of the edge
  int32_t lo[32];
  int32_t len[32];
  int32_t salt[32];
  uint32_t cnt[32];
  int32_t u[32];
  uint32_t erun[32];  // triples of the edge written so far
  alignas(4) uint8_t own[kOwnCap];
};

// Fills the batch record for this lane's edge; *tot is the flattened length of
// the short lists, *is_short whether this lane's list is one of them, *len its length.
//
// Hub side (hub_mode != 0): an edge (v, u) whose N_u has at least a.hub_min ids
// and more than N_v's dv is left to the hub kernel, which hashes N_u once for
// all such edges of u and walks the shorter N_v instead; hub_mode 2 also
// records the edge (per-hub count, flag on the apex vapex).
template <class BS>
__device__ __forceinline__ void batch_setup(BS& bs, const CountArgs& a, const CountWs& ws, int32_t u,
                                            bool act, int64_t eg, int32_t salt, int32_t lo, int32_t vlen,
                                            int& tot, bool& is_short, int32_t& len, uint32_t* err, bool list_write,
                                            uint32_t erun0, int32_t vapex, int32_t dv, int hub_mode,
                                            int32_t* excl_out = nullptr) {
  const int lane = lane_id();
  int64_t ub = 0;
  len = 0;
  // the listing write pass walks only edges that have triangles
  if (act && (!list_write || ws.ecount[eg] > 0)) len = list_bounds(a, u, ub, err);
  if (hub_mode && len >= a.hub_min && len > dv) {
    const int32_t h = ws.hub_idx[u];
    if (h >= 0) {
      if (hub_mode == 2) {
        atomicAdd(&ws.hub_cnt[h], 1);
        ws.rev_flag[vapex] = 1;
      }
      len = 0;
    }
  }
  is_short = len < kShortLen;
  const int32_t slen = is_short ? len : 0;
  const int32_t incl = warp_incl_scan(slen);
  tot = __shfl_sync(FULL, incl, 31);
  const int32_t excl = incl - slen;
  if (excl_out) *excl_out = excl;
  __syncwarp();
  if constexpr (BS::kTile) {
    bs.lo[lane] = lo;
    bs.len[lane] = vlen;
    bs.salt[lane] = salt;
    // address arithmetic in uint64 (a short list's start may lie below cols by up to its flattened offset)
    bs.pk[lane] = (reinterpret_cast<uintptr_t>(a.cols) + 4u * static_cast<uint64_t>(is_short ? ub - excl : ub)) |
                  (static_cast<uint64_t>(salt) << 58);
  } else {
    bs.beg[lane] = is_short ? ub - excl : ub;
  }
  bs.cnt[lane] = 0;
  if constexpr (BS::kWrite) {
    bs.u[lane] = u;
    bs.erun[lane] = erun0;
    bs.ebase[lane] = act ? ws.eoff[eg] : 0;
  }
  // owner table: this lane's byte range [excl, excl + slen), whole 32-bit words
  // where they fit in the range (no other lane writes those words), bytes at the ends
  int32_t i = 0;
  for (; i < slen && ((excl + i) & 3); ++i) bs.own[excl + i] = static_cast<uint8_t>(lane);
  const uint32_t pat = static_cast<uint32_t>(lane) * 0x01010101u;
  for (; i + 4 <= slen; i += 4) *reinterpret_cast<uint32_t*>(bs.own + excl + i) = pat;
  for (; i < slen; ++i) bs.own[excl + i] = static_cast<uint8_t>(lane);
  __syncwarp();
}

// Lanes in this lane's run of equal keys (runs are contiguous lane ranges).
__device__ __forceinline__ unsigned run_mask(int key) {
  const int lane = lane_id();
  const int prev = __shfl_up_sync(FULL, key, 1);
  const unsigned heads = __ballot_sync(FULL, lane == 0 || key != prev);
  const unsigned upto = lane == 31 ? FULL : (2u << lane) - 1u;   // lanes <= me
  const int head = 31 - __clz(heads & upto);
  const unsigned after = heads & ~upto;
  const unsigned below_next = after ? (1u << (__ffs(after) - 1)) - 1u : FULL;
  return below_next & ~((1u << head) - 1u);
}

// Listing: write this lane's triple (if f) at its edge's offset plus the
// edge's running count; lanes of one edge are contiguous and in candidate order.
__device__ __forceinline__ void write_triples(TileWriteBatch& bs, bool has, bool f, int s, int32_t v, int32_t w,
                                             const CountArgs& a, const CountWs& ws, uint32_t* err) {
  const int lane = lane_id();
  const unsigned fm = __ballot_sync(FULL, f);
  if (!fm) return;
  const unsigned same = run_mask(has ? s : 32 + lane);
  if (f) {
    const int64_t idx = bs.ebase[s] + bs.erun[s] + __popc(fm & same & lanemask_lt());
    if (idx < a.cap) {
      a.tri[3 * idx] = v;
      a.tri[3 * idx + 1] = bs.u[s];
      a.tri[3 * idx + 2] = w;
    } else {
      set_err(err, ERR_CAPACITY);
    }
  }
  __syncwarp();
  if (has && lane == 31 - __clz(same)) bs.erun[s] += __popc(fm & same);
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Tile kernel
// ---------------------------------------------------------------------------

template <int MODE, class SH>
struct TileSmem {
  int32_t tile[SH::kIds];
  uint32_t bits[(1 << SH::kBitsLog2) / 32];
  int32_t vlo[32];     // tile start of each chunk lane's list (-1 before the group, > S after)
  uint32_t vcnt[32];   // triangles with apex v (chunk lane)
  int32_t qw[64];      // filter survivors: candidate id ...
  int32_t qs[64];      // ... and its edge
  std::conditional_t<MODE == MODE_LIST_WRITE, TileWriteBatch, TileBatch> bs;
};

// Exact check of the first `cnt` queued survivors, with the per-mode effects.
template <int MODE, class SH>
__device__ __forceinline__ void exact_flush(TileSmem<MODE, SH>& sm, int cnt, int top, int32_t vbase, const CountArgs& a,
                                            const CountWs& ws, uint32_t* err) {
  auto& bs = sm.bs;
  const int lane = lane_id();
  __syncwarp();
  const bool has = lane < cnt;
  const int s = has ? sm.qs[lane] : 0;
  const int32_t w = has ? sm.qw[lane] : 0;
  const bool f = has && member(sm.tile + bs.lo[s], bs.len[s], top, w);
  if (f && MODE != MODE_LIST_WRITE) {  // the write pass already knows every count
    atomicAdd(&bs.cnt[s], 1u);
    if (MODE == MODE_LOCAL) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + w), 1ull);
  }
  if constexpr (MODE == MODE_LIST_WRITE) write_triples(bs, has, f, s, vbase + bs.salt[s], w, a, ws, err);
  __syncwarp();
}

// Queue this window's survivors; check 32 of them once 32 are waiting.
template <int MODE, class SH>
__device__ __forceinline__ void push(TileSmem<MODE, SH>& sm, bool pass, int32_t w, int s, int& qn, int top, int32_t vbase,
                                     const CountArgs& a, const CountWs& ws, uint32_t* err) {
  const int lane = lane_id();
  const unsigned m = __ballot_sync(FULL, pass);
  if (!m) return;
  if (pass) {
    const int pos = qn + __popc(m & lanemask_lt());
    sm.qw[pos] = w;
    sm.qs[pos] = s;
  }
  qn += __popc(m);
  if (qn >= 32) {
    exact_flush<MODE, SH>(sm, 32, top, vbase, a, ws, err);
    const int rest = qn - 32;
    int32_t tw = 0, ts = 0;
    if (lane < rest) {
      tw = sm.qw[32 + lane];
      ts = sm.qs[32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
      sm.qw[lane] = tw;
      sm.qs[lane] = ts;
    }
    __syncwarp();
    qn = rest;
  }
}

// One batch of the tile's edges; returns the matches of this lane's edge.
template <int MODE, class SH>
__device__ __forceinline__ uint32_t tile_batch(TileSmem<MODE, SH>& sm, int top, int32_t u, bool act, int64_t eg, int32_t vl,
                                               int32_t lo, int32_t vlen, int32_t vbase, const CountArgs& a,
                                               const CountWs& ws, uint32_t* err) {
  auto& bs = sm.bs;
  const int lane = lane_id();
  int tot;
  bool is_short;
  int32_t len;
  // an apex with one out-neighbour closes no triangle (N_v and N_u meet at most in u, and
  // u is not in N_u): its edge reads no list, and the hub side never sees it either
  batch_setup(bs, a, ws, u, act && vlen >= 2, eg, vl, lo, vlen, tot, is_short, len, err, MODE == MODE_LIST_WRITE,
              0u, vbase + vl, vlen, a.hub_min > 0 ? (a.reuse_hub ? 1 : 2) : 0);
  int qn = 0;
  // candidate lists are read evict-first: a list is read again only after many others,
  // and the lines it would keep are better spent on the list bounds (read evict-last)
  for (int32_t p0 = 0; p0 < tot; p0 += 32 * SH::kUnroll) {
    int32_t w[SH::kUnroll];
    uint32_t ss[SH::kUnroll];  // edge (bits 0..4) and its filter salt << 26 (bits 26..30)
#pragma unroll
    for (int k = 0; k < SH::kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      ss[k] = 0;
      w[k] = 0;
      if (p < tot) {
        const int s = bs.own[p];
        const uint64_t pk = bs.pk[s];
        w[k] = ld_nc_hint(reinterpret_cast<const int32_t*>(pk & kPtrMask) + p, l2_policy_evict_first());
        ss[k] = static_cast<uint32_t>(s) | (static_cast<uint32_t>(pk >> 32) & kSaltMix);
      }
    }
#pragma unroll
    for (int k = 0; k < SH::kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      const bool pass = p < tot && ftest<SH::kBitsLog2>(sm.bits, w[k], ss[k] & kSaltMix);
      push<MODE, SH>(sm, pass, w[k], static_cast<int>(ss[k] & 31u), qn, top, vbase, a, ws, err);
    }
  }
  unsigned lm = __ballot_sync(FULL, len > 0 && !is_short);
  while (lm) {
    const int e = __ffs(lm) - 1;
    lm &= lm - 1;
    const int32_t* lb = reinterpret_cast<const int32_t*>(bs.pk[e] & kPtrMask);  // N_u
    const int32_t le = __shfl_sync(FULL, len, e);
    const uint32_t se = static_cast<uint32_t>(bs.salt[e]) << 26;
    for (int32_t p0 = 0; p0 < le; p0 += 32 * SH::kUnroll) {
      int32_t w[SH::kUnroll];
#pragma unroll
      for (int k = 0; k < SH::kUnroll; ++k) {
        const int32_t p = p0 + 32 * k + lane;
        w[k] = p < le ? ld_nc_hint(lb + p, l2_policy_evict_first()) : 0;
      }
#pragma unroll
      for (int k = 0; k < SH::kUnroll; ++k) {
        const int32_t p = p0 + 32 * k + lane;
        const bool pass = p < le && ftest<SH::kBitsLog2>(sm.bits, w[k], se);
        push<MODE, SH>(sm, pass, w[k], e, qn, top, vbase, a, ws, err);
      }
    }
  }
  if (qn) exact_flush<MODE, SH>(sm, qn, top, vbase, a, ws, err);
  __syncwarp();
  return act ? bs.cnt[lane] : 0u;
}

// Batched form: add each apex vertex's count to its graph's total.  Graph ids
// of consecutive vertices form runs; one lane per run adds the run's sum.
__device__ __forceinline__ void add_graph_totals(const CountArgs& a, bool in_group, int32_t v, uint32_t c) {
  const int lane = lane_id();
  const int32_t key = in_group ? a.gid[v] : -1 - lane;
  const uint32_t incl = static_cast<uint32_t>(warp_incl_scan(static_cast<int32_t>(c)));
  const int32_t prev = __shfl_up_sync(FULL, key, 1);
  const bool head = lane == 0 || key != prev;
  const unsigned heads = __ballot_sync(FULL, head);
  const unsigned after = heads & ~(0xffffffffu >> (31 - lane));
  const int end = (after ? __ffs(after) - 1 : 32) - 1;
  const uint32_t at_end = __shfl_sync(FULL, incl, end);
  const uint32_t before = __shfl_sync(FULL, incl, lane > 0 ? lane - 1 : 0);
  const uint32_t sum = at_end - (lane > 0 ? before : 0u);
  if (head && in_group && sum) atomicAdd(a.graph_total + key, static_cast<unsigned long long>(sum));
}

template <int MODE, class SH>
__global__ void __launch_bounds__(kTileWarps * 32, 8) k_count_tile(CountArgs a, CountWs ws, uint32_t* err) {
  __shared__ TileSmem<MODE, SH> s_t[kTileWarps];
  __shared__ unsigned long long s_sum[kTileWarps];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  TileSmem<MODE, SH>& sm = s_t[wid];
  unsigned long long acc = 0;
  const uint64_t stream = l2_policy_evict_first();
  uint32_t claim_next = 0;
  int claim_left = 0;
  for (int32_t chunk = 0; a.tile_quota <= 0 || chunk < a.tile_quota; ++chunk) {
    if (claim_left == 0) {
      // every warp claims its chunks from one counter, and additions to one address
      // serialize in L2: a pass over many vertices claims tile_claim chunks at a time
      uint32_t c0 = 0;
      if (lane == 0) c0 = atomicAdd(&ws.counters[kCtrCursor], 32u * static_cast<uint32_t>(a.tile_claim));
      claim_next = __shfl_sync(FULL, c0, 0);
      claim_left = a.tile_claim;
    }
    const uint32_t off = claim_next;
    claim_next += 32u;
    --claim_left;
    if (off >= static_cast<uint32_t>(a.v_hi - a.v_lo)) break;
    const uint32_t base = static_cast<uint32_t>(a.v_lo) + off;  // apex vertices [v_lo, v_hi) only
    const int32_t v = static_cast<int32_t>(base) + lane;
    const bool valid = v < a.v_hi;
    int64_t b = 0, e = 0;
    if (valid) {  // apex offsets and lists are each read once here: first out of L2
      b = ld_nc_hint(a.offsets + v, stream);
      e = ld_nc_hint(a.offsets + v + 1, stream);
      if (b < 0 || e < b || e > a.m || b - a.apex_base < 0 || e - a.apex_base > a.apex_len) {
        set_err(err, ERR_BAD_CSR);
        b = e = a.apex_base;
      }
    }
    const int64_t d = e - b;
    // the listing write pass only revisits apex vertices that have triangles
    const bool skip = MODE == MODE_LIST_WRITE && valid && ws.eoff[e] == ws.eoff[b];
    const bool big = valid && !skip && d > a.tile_max;
    const unsigned bigmask = __ballot_sync(FULL, big);
    if (bigmask) {
      uint32_t qb = 0;
      if (lane == 0) qb = atomicAdd(&ws.counters[0], static_cast<uint32_t>(__popc(bigmask)));
      qb = __shfl_sync(FULL, qb, 0);
      if (big) ws.big_queue[qb + __popc(bigmask & lanemask_lt())] = v;
    }
    // Groups: maximal runs of consecutive short lists whose ids fit one tile.
    // live: lanes whose list this kernel counts (a live list has <= tile_max <= SH::kIds ids, so it opens a group)
    const unsigned live = __ballot_sync(FULL, valid && !big && !skip);
    int g0 = live ? __ffs(live) - 1 : 32;
    while (g0 < 32) {
      const int32_t len = (lane >= g0 && valid && !big && !skip) ? static_cast<int32_t>(d) : 0;
      const int32_t incl = warp_incl_scan(len);
      const bool stop = lane >= g0 && (!valid || big || skip || incl > SH::kIds);
      const unsigned smask = __ballot_sync(FULL, stop);
      const int g1 = smask ? __ffs(smask) - 1 : 32;
      if (g1 == g0) {  // lane g0 is past the end, a queued long list or skipped: go to the next live lane
        const unsigned after = g0 < 31 ? live & (0xffffffffu << (g0 + 1)) : 0u;
        g0 = after ? __ffs(after) - 1 : 32;
        continue;
      }
      const bool in_group = lane >= g0 && lane < g1;
      const int32_t glen = in_group ? len : 0;
      const int32_t S = __shfl_sync(FULL, incl, g1 - 1);
      const int64_t start = __shfl_sync(FULL, b, g0);
      __syncwarp();
      bool bad = false;
      for (int t = lane; t < S; t += 32) {
        const int32_t x = ld_nc_hint(a.apex_cols + (start - a.apex_base) + t, stream);
        sm.tile[t] = x;
        bad |= static_cast<uint32_t>(x) >= static_cast<uint32_t>(a.n);
      }
      for (int i = lane; i < (1 << SH::kBitsLog2) / 32; i += 32) sm.bits[i] = 0u;
      const int32_t lo = incl - len;
      sm.vlo[lane] = lane < g0 ? -1 : (lane < g1 ? lo : S + 1);
      sm.vcnt[lane] = 0;
      if (__any_sync(FULL, bad)) {
        if (lane == 0) set_err(err, ERR_BAD_ID);
        g0 = g1;
        continue;
      }
      __syncwarp();
      for (int i = 0; i < glen; ++i) fset<SH::kBitsLog2>(sm.bits, sm.tile[lo + i], static_cast<uint32_t>(lane) << 26);
      const int maxlen = __reduce_max_sync(FULL, glen);
      const int top = maxlen > 0 ? 1 << (31 - __clz(maxlen)) : 0;
      __syncwarp();
      for (int t0 = 0; t0 < S; t0 += 32) {
        const int t = t0 + lane;
        const bool act = t < S;
        const int vl = act ? search32(sm.vlo, static_cast<int32_t>(t)) : 0;
        const int32_t u = act ? sm.tile[t] : 0;
        const int32_t vlen = __shfl_sync(FULL, glen, vl);
        const uint32_t c = tile_batch<MODE, SH>(sm, top, u, act, start + t, vl, sm.vlo[vl], vlen,
                                            static_cast<int32_t>(base), a, ws, err);
        if (act && (MODE == MODE_LOCAL || MODE == MODE_LIST_COUNT) && ws.ecount)
          __stcs(ws.ecount + start + t, static_cast<int32_t>(c));  // write-once stream: evict-first
        if (c) {
          if (MODE == MODE_LOCAL)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + u), static_cast<unsigned long long>(c));
          atomicAdd(&sm.vcnt[vl], c);
        }
        __syncwarp();
      }
      const uint32_t cv = in_group ? sm.vcnt[lane] : 0u;
      if (in_group) {
        if (MODE == MODE_LOCAL && cv)
          atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + v), static_cast<unsigned long long>(cv));
        acc += cv;
      }
      if (MODE != MODE_LIST_WRITE && a.graph_total) add_graph_totals(a, in_group, v, cv);
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
// Block kernel (lists longer than tile_max).  Heavy apex vertices get a whole
// block; N_v is hashed into a shared-memory open-addressing table (load factor
// at most 1/4) so that membership is exact in about one probe, with no filter,
// no survivor queue and no binary search.  For per-vertex counts each slot
// also counts its matches, so T_w is added once per (v, w) instead of once
// per triangle (the w of a skewed graph are hubs: one global counter each).
// ---------------------------------------------------------------------------

template <int MODE>
struct HashCfg {
  static constexpr int kLog2 = MODE == MODE_LOCAL ? 12 : 13;   // slots (keys, plus counts when LOCAL)
  static constexpr int kSlots = 1 << kLog2;
  static constexpr int kCap = kSlots / 4;                        // ids of N_v per pass
  static constexpr size_t kBytes = sizeof(int32_t) * kSlots * (MODE == MODE_LOCAL ? 2 : 1);
};

template <int LOG2>
__device__ __forceinline__ uint32_t slot_of(int32_t w) {
  return (static_cast<uint32_t>(w) * 0x9E3779B1u) >> (32 - LOG2);
}

// Second choice of a two-choice (cuckoo) table: slot h's partner for key w is
// h ^ alt_of(w), an odd (so nonzero) offset: the two slots of a key differ and
// each is the other's partner, so an evicted key finds its other slot from
// the one it was evicted from.
template <int LOG2>
__device__ __forceinline__ uint32_t alt_of(int32_t w) {
  return ((static_cast<uint32_t>(w) * 0x85EBCA77u) >> (32 - LOG2)) | 1u;
}

// Cuckoo lookup: slot of w in the table, or -1 -- two independent shared
// loads, no probe loop, so the lanes of a warp never wait on each other.
template <int LOG2>
__device__ __forceinline__ int cuckoo_find(const int32_t* tab, int32_t w) {
  const uint32_t h1 = slot_of<LOG2>(w), h2 = h1 ^ alt_of<LOG2>(w);
  const int32_t x1 = tab[h1], x2 = tab[h2];
  return x1 == w ? static_cast<int>(h1) : (x2 == w ? static_cast<int>(h2) : -1);
}

// Cuckoo insertion by many threads at once: each thread holds one homeless key
// and swaps it into its slot; an evicted key moves to its other slot.  Keys are
// never lost (every move is one atomic exchange).  Returns false if a key is
// still homeless after kCuckooMoves moves (the caller then rebuilds the chunk
// with linear probing).
constexpr int kCuckooMoves = 64;
template <int LOG2>
__device__ __forceinline__ bool cuckoo_insert(int32_t* tab, int32_t w) {
  uint32_t h = slot_of<LOG2>(w);
  for (int i = 0; i < kCuckooMoves; ++i) {
    const int32_t old = atomicExch(&tab[h], w);
    if (old < 0 || old == w) return true;
    w = old;
    h ^= alt_of<LOG2>(w);
  }
  return false;
}

// Linear-probing table (fallback when a cuckoo build fails): slot of w, or -1.
template <int LOG2>
__device__ __forceinline__ int hash_find(const int32_t* tab, int32_t w) {
  if (w < 0) return -1;
  uint32_t h = slot_of<LOG2>(w);
  for (int probe = 0; probe < (1 << LOG2); ++probe) {  // bounded: the table is never full
    const int32_t x = tab[h];
    if (x == w) return static_cast<int>(h);
    if (x < 0) return -1;
    h = (h + 1) & ((1u << LOG2) - 1);
  }
  return -1;
}

template <int LOG2>
__device__ __forceinline__ void hash_insert(int32_t* tab, int32_t w) {
  uint32_t h = slot_of<LOG2>(w);
  for (int probe = 0; probe < (1 << LOG2); ++probe) {
    const int32_t prev = atomicCAS(&tab[h], -1, w);
    if (prev == -1 || prev == w) return;
    h = (h + 1) & ((1u << LOG2) - 1);
  }
}

// Slot of w in the chunk's table (cuckoo, or linear probing after a failed build).
template <int LOG2>
__device__ __forceinline__ int table_find(const int32_t* tab, int32_t w, bool linear) {
  if (w < 0) return -1;
  return linear ? hash_find<LOG2>(tab, w) : cuckoo_find<LOG2>(tab, w);
}

// Counting passes of the hash kernels: a match adds to its edge (and, for
// per-vertex counts, to the slot of w, flushed once per chunk).
template <int MODE>
__device__ __forceinline__ void hash_record(HashBatch& bs, uint32_t* slot_cnt, int slot, int s) {
  if (slot >= 0) {
    atomicAdd(&bs.cnt[s], 1u);
    if (MODE == MODE_LOCAL) atomicAdd(&slot_cnt[slot], 1u);
  }
}

// Write pass of the hash kernels, one window of short lists laid end to end
// (positions wstart .. wstart+31).  The window's lanes map to edges in
// increasing order, so each edge's lanes form one contiguous run; the edge's
// output cursor lives in its owner lane's register (wbase: eoff of the edge
// plus the triples written so far) and a found lane reads its edge's cursor
// and run start with indexed shuffles -- no shared-memory bookkeeping.
// Triples of one edge come out in window order, as in every other pass.
template <bool HUB>
__device__ __forceinline__ void emit_short(bool f, int s, int32_t w, int32_t wstart, int32_t excl, int32_t slen,
                                           int32_t u, int32_t v, int64_t& wbase, const CountArgs& a, uint32_t* err) {
  const int lane = lane_id();
  const unsigned fm = __ballot_sync(FULL, f);
  if (!fm) return;
  // owner lane: its edge's run in this window, clamped to [0, 32)
  const int32_t first = min(max(excl - wstart, 0), 32), end = min(max(excl + slen - wstart, 0), 32);
  const unsigned below_end = end >= 32 ? FULL : ((1u << end) - 1u);
  const unsigned below_first = first >= 32 ? FULL : ((1u << first) - 1u);
  const int cnt = __popc(fm & below_end & ~below_first);
  // found lane: cursor and run start of its edge s
  const int64_t base_s = __shfl_sync(FULL, wbase, s);
  const int32_t first_s = __shfl_sync(FULL, first, s);
  const int32_t u_s = __shfl_sync(FULL, u, s);
  if (f) {
    const unsigned lt = (1u << lane) - 1u;
    const unsigned run_lo = first_s >= 32 ? FULL : ((1u << first_s) - 1u);
    const int64_t idx = base_s + __popc(fm & lt & ~run_lo);
    if (idx < a.cap) {
      a.tri[3 * idx] = HUB ? u_s : v;
      a.tri[3 * idx + 1] = HUB ? v : u_s;
      a.tri[3 * idx + 2] = w;
    } else {
      set_err(err, ERR_CAPACITY);
    }
  }
  wbase += cnt;
}

// Write pass, one window of the long list of edge e (every lane on that edge):
// base_e is the edge's cursor, kept warp-uniform while the list is walked.
template <bool HUB>
__device__ __forceinline__ void emit_long(bool f, int32_t w, int32_t u_e, int32_t v, int64_t& base_e,
                                          const CountArgs& a, uint32_t* err) {
  const unsigned fm = __ballot_sync(FULL, f);
  if (!fm) return;
  if (f) {
    const int64_t idx = base_e + __popc(fm & ((1u << lane_id()) - 1u));
    if (idx < a.cap) {
      a.tri[3 * idx] = HUB ? u_e : v;
      a.tri[3 * idx + 1] = HUB ? v : u_e;
      a.tri[3 * idx + 2] = w;
    } else {
      set_err(err, ERR_CAPACITY);
    }
  }
  base_e += __popc(fm);
}

// One batch of edges against the hashed chunk (ids in [lo, hi]) of the block
// vertex v's list: block kernel, edges (v, u) with u on this lane if `act`,
// walking N_u; hub kernel (HUB), edges (x, v) with x on this lane, walking N_x.
// eg is the lane's edge (its position in cols).  Returns the lane's matches.
template <int MODE, bool HUB, int UNROLL>
__device__ __forceinline__ uint32_t hash_batch(HashBatch& bs, const int32_t* tab, uint32_t* slot_cnt, int32_t lo,
                                               int32_t hi, int32_t u, bool act, int64_t eg, int32_t v,
                                               const CountArgs& a, const CountWs& ws, uint32_t* err,
                                               bool chunked, bool first_chunk, int32_t dv, bool linear) {
  constexpr int L = HashCfg<MODE>::kLog2;
  const int lane = lane_id();
  int tot;
  bool is_short;
  int32_t len;
  // listing a vertex hashed in several chunks: an edge's triples continue where the last chunk stopped
  const uint32_t erun0 = (MODE == MODE_LIST_WRITE && chunked && !first_chunk && act) ? ws.erun[eg] : 0u;
  // block kernel: edges bound for the hub side are recorded once, with the first chunk
  const int hub_mode = (HUB || a.hub_min <= 0) ? 0 : ((first_chunk && !a.reuse_hub) ? 2 : 1);
  int32_t excl = 0;
  batch_setup(bs, a, ws, u, act, eg, 0, 0, 0, tot, is_short, len, err, MODE == MODE_LIST_WRITE, erun0, v, dv,
              hub_mode, &excl);
  constexpr bool kWrite = MODE == MODE_LIST_WRITE;
  // write pass: this lane's edge's output cursor (0 for edges without triangles: they have no lanes)
  int64_t wbase = (kWrite && act && len > 0) ? ws.eoff[eg] + erun0 : 0;
  const int32_t slen = is_short ? len : 0;
  for (int32_t p0 = 0; p0 < tot; p0 += 32 * UNROLL) {
    int32_t w[UNROLL];
    int s[UNROLL];
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      s[k] = 0;
      w[k] = -1;
      if (p < tot) {
        s[k] = bs.own[p];
        w[k] = a.cols[bs.beg[s[k]] + p];
      }
    }
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
      const int slot = (w[k] >= lo && w[k] <= hi) ? table_find<L>(tab, w[k], linear) : -1;
      if (kWrite) emit_short<HUB>(slot >= 0, s[k], w[k], p0 + 32 * k, excl, slen, u, v, wbase, a, err);
      else hash_record<MODE>(bs, slot_cnt, slot, s[k]);
    }
  }
  unsigned lm = __ballot_sync(FULL, len > 0 && !is_short);
  while (lm) {
    const int e = __ffs(lm) - 1;
    lm &= lm - 1;
    const int64_t b = bs.beg[e];
    const int32_t le = __shfl_sync(FULL, len, e);
    const int32_t u_e = __shfl_sync(FULL, u, e);
    int64_t base_e = __shfl_sync(FULL, wbase, e);
    for (int32_t p0 = 0; p0 < le; p0 += 32 * UNROLL) {
      int32_t w[UNROLL];
#pragma unroll
      for (int k = 0; k < UNROLL; ++k) {
        const int32_t p = p0 + 32 * k + lane;
        w[k] = p < le ? a.cols[b + p] : -1;
      }
#pragma unroll
      for (int k = 0; k < UNROLL; ++k) {
        const int slot = (w[k] >= lo && w[k] <= hi) ? table_find<L>(tab, w[k], linear) : -1;
        if (kWrite) emit_long<HUB>(slot >= 0, w[k], u_e, v, base_e, a, err);
        else hash_record<MODE>(bs, slot_cnt, slot, e);
      }
    }
    if (lane == e) wbase = base_e;
  }
  __syncwarp();
  // listing a vertex hashed in several chunks: the next chunk continues at this count
  if (kWrite && chunked && act && len > 0) ws.erun[eg] = static_cast<uint32_t>(wbase - ws.eoff[eg]);
  return act ? bs.cnt[lane] : 0u;
}

// Block kernel (HUB = false): one block per queued apex v with a long N_v.
// Hub kernel (HUB = true): one block per work item (hub u, segment of the
// edges (x, u) recorded for u's side); N_u is hashed and each N_x walked.
// Both: the block vertex's list is hashed in chunks of H::kCap ids; the
// lane's vertex gets its edge's matches, the block vertex their sum.
template <int MODE, bool HUB, int BATCH, int UNROLL>
__global__ void __launch_bounds__(kBlockWarps * 32, 4) k_count_block(CountArgs a, CountWs ws, uint32_t* err) {
  using H = HashCfg<MODE>;
  extern __shared__ int32_t tab[];
  uint32_t* slot_cnt = reinterpret_cast<uint32_t*>(tab + H::kSlots);  // LOCAL only
  __shared__ HashBatch s_b[kBlockWarps];
  __shared__ unsigned long long s_red[kBlockWarps];
  __shared__ int64_t s_next;  // next batch of walked lists (warps take batches as they finish)
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  unsigned long long acc = 0;
  bool clean = false;  // the table holds no key and no count (uniform across the block)
  if (threadIdx.x == 0) s_next = 0;  // reset again after each chunk, behind its last barrier
  const uint32_t qn = HUB ? static_cast<uint32_t>(min64(ws.counters[kCtrItems], ws.items_cap))
                         : ws.counters[kCtrBigQueue];
  for (uint32_t qi = blockIdx.x; qi < qn; qi += gridDim.x) {
    int32_t v;
    int64_t ent_lo = 0, ent_n = 0;  // hub kernel: this item's edges in hub_ent
    if (HUB) {
      const int2 it = ws.hub_items[qi];
      v = ws.hubs[it.x];
      ent_lo = ws.hub_off[it.x] + static_cast<int64_t>(it.y) * kHubSeg;
      ent_n = max64(0, min64(min64(kHubSeg, ws.hub_off[it.x + 1] - ent_lo), a.m - ent_lo));
    } else {
      v = ws.big_queue[qi];
    }
    // the hashed list: the apex's own, or on the hub side the hub's N_u
    const int32_t* hcols = HUB ? a.cols : a.apex_cols;
    const int64_t hbase = HUB ? a.cols_base : a.apex_base, hlen = HUB ? a.cols_len : a.apex_len;
    const int64_t b = a.offsets[v];
    int64_t e = a.offsets[v + 1];
    if (b - hbase < 0 || e < b || e - hbase > hlen) {  // outside the array that holds it: nothing read
      if (threadIdx.x == 0) set_err(err, ERR_BAD_CSR);
      e = b;
    }
    const int32_t* hl = hcols + (b - hbase);  // the hashed list's first id
    const int64_t dv = e - b;
    const int64_t nl = HUB ? ent_n : dv;  // lists walked against v's
    unsigned long long cv = 0;
    for (int64_t c0 = 0; c0 < dv; c0 += H::kCap) {
      const int clen = static_cast<int>(min64(H::kCap, dv - c0));
      __syncthreads();  // the last chunk's clearing and cursor reset are done
      if (!clean) {  // the first chunk of this block, or after a linear-probing chunk or a bad id
        for (int i = threadIdx.x; i < H::kSlots; i += blockDim.x) {
          tab[i] = -1;
          if (MODE == MODE_LOCAL) slot_cnt[i] = 0;
        }
        __syncthreads();
      }
      bool bad = false, homeless = false;
      for (int i = threadIdx.x; i < clen; i += blockDim.x) {
        const int32_t x = hl[c0 + i];
        if (static_cast<uint32_t>(x) >= static_cast<uint32_t>(a.n)) bad = true;
        else if (!cuckoo_insert<H::kLog2>(tab, x)) homeless = true;
      }
      if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) {
          set_err(err, ERR_BAD_ID);
          s_next = 0;
        }
        clean = false;
        break;
      }
      // a cuckoo build that left a key homeless: rebuild this chunk with linear probing
      const bool linear = __syncthreads_or(homeless);
      if (linear) {
        for (int i = threadIdx.x; i < H::kSlots; i += blockDim.x) tab[i] = -1;
        __syncthreads();
        for (int i = threadIdx.x; i < clen; i += blockDim.x) hash_insert<H::kLog2>(tab, hl[c0 + i]);
        __syncthreads();
      }
      // the chunk is a sorted run of the block vertex's list: its ids lie in [lo, hi]
      const int32_t lo = hl[c0], hi = hl[c0 + clen - 1];
      for (;;) {
        // guided batches: a warp takes 32 walked lists while there are many left, then
        // fewer, so that the warps of the block reach the chunk's end together
        int64_t ub = 0;
        int size = BATCH;
        if (lane == 0) {
          const int64_t left = nl - *reinterpret_cast<volatile int64_t*>(&s_next);
          size = static_cast<int>(max64(kMinHashBatch, min64(BATCH, left / (2 * kBlockWarps))));
          ub = atomicAdd(reinterpret_cast<unsigned long long*>(&s_next), static_cast<unsigned long long>(size));
        }
        ub = __shfl_sync(FULL, ub, 0);
        size = __shfl_sync(FULL, size, 0);
        if (ub >= nl) break;
        const int nb = static_cast<int>(min64(size, nl - ub));
        bool act = lane < nb;
        int32_t x = 0;
        int64_t eg = 0;
        if (act) {
          if (HUB) {  // edge (x, v): v sits at position en.y of N_x
            const int2 en = ws.hub_ent[ent_lo + ub + lane];
            x = en.x;
            // N_x's bounds from the int32 offsets when there are some: the same line
            // serves list_bounds right after (the hub side never splits the lists)
            int64_t xb = 0, xe = 0;
            if (static_cast<uint32_t>(x) < static_cast<uint32_t>(a.n)) {
              xb = a.off32 ? a.off32[x] : a.offsets[x];
              xe = a.off32 ? a.off32[x + 1] : a.offsets[x + 1];
            }
            if (static_cast<uint32_t>(x) < static_cast<uint32_t>(a.n) && en.y >= 0 && xb + en.y < xe) {
              eg = xb + en.y;
            } else {  // an entry the fill pass did not write: skip it, report the mismatch
              set_err(err, ERR_BAD_CSR);
              x = 0;
              act = false;
            }
          } else {
            x = hl[ub + lane];
            eg = b + ub + lane;
          }
        }
        const uint32_t c = hash_batch<MODE, HUB, UNROLL>(s_b[wid], tab, slot_cnt, lo, hi, x, act, eg, v, a, ws, err,
                                                 dv > H::kCap, c0 == 0, static_cast<int32_t>(dv), linear);
        cv += c;
        if (act && (MODE == MODE_LOCAL || MODE == MODE_LIST_COUNT) && ws.ecount) {
          // the first chunk sets the edge's count, later chunks add to it
          if (c0 == 0) ws.ecount[eg] = static_cast<int32_t>(c);
          else ws.ecount[eg] += static_cast<int32_t>(c);
        }
        if (MODE == MODE_LOCAL && c)
          atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + x), static_cast<unsigned long long>(c));
      }
      __syncthreads();  // every probe of this chunk is done
      if (linear) {  // T_w once per (block vertex, w) of this chunk, over the whole table
        if (MODE == MODE_LOCAL)
          for (int i = threadIdx.x; i < H::kSlots; i += blockDim.x)
            if (slot_cnt[i])
              atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + tab[i]),
                        static_cast<unsigned long long>(slot_cnt[i]));
        clean = false;
      } else {
        // cuckoo table: each of the chunk's ids sits in one of its two slots, so its
        // count is flushed, and then both slots cleared, from the id alone; reading
        // and clearing are split by a barrier (an id's slot may be another id's partner)
        if (MODE == MODE_LOCAL) {
          for (int i = threadIdx.x; i < clen; i += blockDim.x) {
            const int32_t x = hl[c0 + i];
            const int slot = cuckoo_find<H::kLog2>(tab, x);
            if (slot >= 0 && slot_cnt[slot])
              atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + x),
                        static_cast<unsigned long long>(slot_cnt[slot]));
          }
          __syncthreads();
        }
        for (int i = threadIdx.x; i < clen; i += blockDim.x) {
          const int32_t x = hl[c0 + i];
          const uint32_t h1 = slot_of<H::kLog2>(x), h2 = h1 ^ alt_of<H::kLog2>(x);
          tab[h1] = -1;
          tab[h2] = -1;
          if (MODE == MODE_LOCAL) {
            slot_cnt[h1] = 0;
            slot_cnt[h2] = 0;
          }
        }
        clean = true;
      }
      // every warp has left this chunk's batch loop: the cursor can start over
      if (threadIdx.x == 0) s_next = 0;
    }
    cv = warp_sum64(cv);
    if (lane == 0) s_red[wid] = cv;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kBlockWarps; ++w) t += s_red[w];
      if (MODE == MODE_LOCAL && t) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + v), t);
      if (MODE != MODE_LIST_WRITE && a.graph_total && t) atomicAdd(a.graph_total + a.gid[v], t);
      acc += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && acc && a.total) atomicAdd(a.total, acc);
}

// ---------------------------------------------------------------------------
// Hub side preparation.  Hubs are the vertices with |N_u| >= hub_min; the
// tile and block kernels count, per hub, the edges they leave to its side
// (batch_setup) and flag their apex vertices; the flagged vertices' lists are
// then walked again to place each such edge in its hub's segment of hub_ent.
// ---------------------------------------------------------------------------

// int32 copy of the offsets (m < 2^31); an offset outside [0, m] becomes m + 1
// there, which list_bounds rejects as a broken CSR wherever it is read.
__global__ void k_off32(int32_t n, int64_t m, const int64_t* __restrict__ offsets, int32_t* __restrict__ off32) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v <= n; v += stride) {
    const int64_t o = offsets[v];
    off32[v] = static_cast<int32_t>((o < 0 || o > m) ? m + 1 : o);
  }
}

__global__ void k_hub_list(int32_t n, const int64_t* __restrict__ offsets, int32_t hub_min, CountWs ws) {
  const int lane = lane_id();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; i0 < n; i0 += stride) {
    const int64_t u = i0 + threadIdx.x;
    bool hub = false;
    if (u < n) {
      const int64_t d = offsets[u + 1] - offsets[u];
      hub = d >= hub_min;
      ws.rev_flag[u] = 0;
      if (!hub) ws.hub_idx[u] = -1;
    }
    const unsigned hm = __ballot_sync(FULL, hub);
    if (hm) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&ws.counters[kCtrHubs], static_cast<uint32_t>(__popc(hm)));
      base = __shfl_sync(FULL, base, 0);
      if (hub) {
        const int32_t h = static_cast<int32_t>(base + __popc(hm & lanemask_lt()));
        ws.hub_idx[u] = h;
        ws.hubs[h] = static_cast<int32_t>(u);
        ws.hub_cnt[h] = 0;
        ws.hub_fill[h] = 0;
      }
    }
  }
}

// Walks the lists of the flagged apex vertices (a warp per vertex) and places
// every edge (v, u) that batch_setup left to u's side -- the same test, on
// the same lengths -- at hub_off[h] + (a fill cursor of hub h).
template <int MODE>
__global__ void k_hub_fill(CountArgs a, CountWs ws, uint32_t* err) {
  const int lane = lane_id();
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  for (int64_t base = w0 * 32; base < a.n; base += warps * 32) {
    const int64_t vl = base + lane;
    const bool flagged = vl < a.n && ws.rev_flag[vl];
    unsigned fm = __ballot_sync(FULL, flagged);
    while (fm) {
      const int32_t v = static_cast<int32_t>(base + __ffs(fm) - 1);
      fm &= fm - 1;
      const int64_t b = a.offsets[v], dv = a.offsets[v + 1] - b;
      if (b < 0 || dv < 0 || b + dv > a.m) {
        if (lane == 0) set_err(err, ERR_BAD_CSR);
        continue;
      }
      for (int64_t p = lane; p < dv; p += 32) {
        if (MODE == MODE_LIST_WRITE && ws.ecount[b + p] <= 0) continue;
        const int32_t u = a.cols[b + p];
        int64_t ub;
        const int32_t len = list_bounds(a, u, ub, err);
        if (len < a.hub_min || len <= dv) continue;
        const int32_t h = ws.hub_idx[u];
        if (h < 0) continue;
        const int32_t pos = atomicAdd(&ws.hub_fill[h], 1);
        const int64_t at = ws.hub_off[h] + pos;
        if (pos < ws.hub_cnt[h] && at < a.m) ws.hub_ent[at] = make_int2(v, static_cast<int32_t>(p));
        else set_err(err, ERR_BAD_CSR);  // the two walks disagree: the CSR changed underneath
      }
    }
  }
}

// One work item per kHubSeg edges of each hub.
__global__ void k_hub_items(CountWs ws) {
  const int64_t cap = ws.items_cap;
  const uint32_t hubs = ws.counters[kCtrHubs];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t h = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; h < hubs; h += stride) {
    const int32_t c = ws.hub_cnt[h];
    const int32_t segs = (c + kHubSeg - 1) / kHubSeg;
    if (!segs) continue;
    const uint32_t at = atomicAdd(&ws.counters[kCtrItems], static_cast<uint32_t>(segs));
    for (int32_t j = 0; j < segs; ++j)
      if (at + j < cap) ws.hub_items[at + j] = make_int2(static_cast<int32_t>(h), j);
  }
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

// Dynamic shared memory of k_count_block<MODE, HUB, BATCH, UNROLL> beyond the 48 KB default: opt in once per device.
template <int MODE, bool HUB, int BATCH, int UNROLL>
cudaError_t block_smem_optin(Ctx* ctx, size_t smem) {
  static bool attr_set[64] = {false};
  if (ctx->device >= 0 && ctx->device < 64 && !attr_set[ctx->device]) {
    const cudaError_t e = cudaFuncSetAttribute(k_count_block<MODE, HUB, BATCH, UNROLL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr_set[ctx->device] = true;
  }
  return cudaSuccess;
}

// The tile kernel of shape SH: persistent grid, but no more blocks than there is work
// for (small graphs leave room for other streams); with a chunk quota, enough blocks
// that every chunk is taken although each warp stops after its quota.
template <int MODE, class SH>
cudaError_t launch_tile(Ctx* ctx, const CountArgs& a, CountWs ws, cudaStream_t s, const char* name) {
  const int64_t chunks = (static_cast<int64_t>(a.v_hi) - a.v_lo + 31) / 32;
  const int tgrid = a.tile_quota > 0
      ? static_cast<int>(max64(1, (chunks + static_cast<int64_t>(kTileWarps) * a.tile_quota - 1) /
                                      (static_cast<int64_t>(kTileWarps) * a.tile_quota)))
      : static_cast<int>(min64(
            persistent_blocks(ctx, reinterpret_cast<const void*>(&k_count_tile<MODE, SH>), kTileWarps * 32, 0),
            max64(1, (chunks + kTileWarps - 1) / kTileWarps)));
  // chunks per claim, at most 8: the counting passes keep at least 64 claims per warp (their
  // chunks are heavy, and coarser claims leave the last warps with more work: PA 2^24 per-vertex
  // pass 10.79 -> 10.98 ms with 6 chunks per claim); the listing write pass, which skips almost
  // every apex of a sparse listing, at least 16 (PA 2^27: 8.56 -> 2.64 ms with 8)
  const int64_t min_claims = MODE == MODE_LIST_WRITE ? 16 : 64;
  CountArgs b = a;
  b.tile_claim = a.tile_quota > 0
      ? 1
      : static_cast<int32_t>(min64(8, max64(1, chunks / (static_cast<int64_t>(tgrid) * kTileWarps * min_claims))));
  Stage st(ctx, s, name);
  k_count_tile<MODE, SH><<<tgrid, kTileWarps * 32, 0, s>>>(b, ws, ctx->d_err);
  counted(ctx);
  return cudaSuccess;
}

// The block kernel (apex side) or the hub kernel, taking BATCH walked lists at a time
// with UNROLL candidate windows in flight per lane.
template <int MODE, bool HUB, int BATCH, int UNROLL>
cudaError_t launch_hash(Ctx* ctx, const CountArgs& a, CountWs ws, cudaStream_t s, const char* name) {
  const size_t smem = HashCfg<MODE>::kBytes;
  cudaError_t e = block_smem_optin<MODE, HUB, BATCH, UNROLL>(ctx, smem);
  if (e != cudaSuccess) return e;
  int grid = persistent_blocks(ctx, reinterpret_cast<const void*>(&k_count_block<MODE, HUB, BATCH, UNROLL>),
                               kBlockWarps * 32, smem);
  // the apex side gets at most m / (tile_max + 1) lists
  if (!HUB) grid = static_cast<int>(min64(grid, max64(1, a.m / (a.tile_max + 1))));
  Stage st(ctx, s, name);
  k_count_block<MODE, HUB, BATCH, UNROLL><<<grid, kBlockWarps * 32, smem, s>>>(a, ws, ctx->d_err);
  counted(ctx);
  return cudaSuccess;
}

// The hash kernels' shape: lists per warp batch (32 or 16), windows in flight (4 or 8).
template <int MODE, bool HUB>
cudaError_t launch_hash_shape(Ctx* ctx, const CountArgs& a, CountWs ws, cudaStream_t s, const char* name) {
  const bool w8 = ctx->hash_windows == 8;
  if (ctx->hash_batch == 16) return w8 ? launch_hash<MODE, HUB, 16, 8>(ctx, a, ws, s, name)
                                       : launch_hash<MODE, HUB, 16, 4>(ctx, a, ws, s, name);
  return w8 ? launch_hash<MODE, HUB, 32, 8>(ctx, a, ws, s, name) : launch_hash<MODE, HUB, 32, 4>(ctx, a, ws, s, name);
}

template <int MODE>
cudaError_t launch_mode(Ctx* ctx, const CountArgs& a, CountWs ws, cudaStream_t s) {
  static const char* kNames[4][4] = {
      {"count.tile", "count.block", "count.prep", "count.hub"},
      {"local.tile", "local.block", "local.prep", "local.hub"},
      {"list_count.tile", "list_count.block", "list_count.prep", "list_count.hub"},
      {"list_write.tile", "list_write.block", "list_write.prep", "list_write.hub"}};
  const bool hub = a.hub_min > 0;
  const int n_grid = static_cast<int>(min64((static_cast<int64_t>(a.n) + 256) / 256,
                                            static_cast<int64_t>(ctx->sm_count) * 8));
  if (hub || a.off32) {
    Stage st(ctx, s, kNames[MODE][2]);
    if (a.off32 && !a.off32_ready) {
      k_off32<<<n_grid, 256, 0, s>>>(a.n, a.m, a.offsets, const_cast<int32_t*>(a.off32));
      counted(ctx);
    }
    if (hub && !a.reuse_hub) {
      k_hub_list<<<n_grid, 256, 0, s>>>(a.n, a.offsets, a.hub_min, ws);
      counted(ctx);
    }
  }
  cudaError_t e;
  switch (ctx->tile_shape) {
    case 1: e = launch_tile<MODE, TileShapeB>(ctx, a, ws, s, kNames[MODE][0]); break;
    case 2: e = launch_tile<MODE, TileShapeC>(ctx, a, ws, s, kNames[MODE][0]); break;
    default: e = launch_tile<MODE, TileShapeA>(ctx, a, ws, s, kNames[MODE][0]); break;
  }
  if (e != cudaSuccess) return e;
  e = launch_hash_shape<MODE, false>(ctx, a, ws, s, kNames[MODE][1]);
  if (e != cudaSuccess) return e;
  if (hub) {
    if (!a.reuse_hub) {
      Stage st(ctx, s, kNames[MODE][2]);
      // hub_off = scan of the per-hub counts (as many as there are hubs, read on the device)
      e = exclusive_scan_i32(ws.hub_cnt, ws.hub_off, a.n, ws.hub_scan, s, ws.counters + kCtrHubs);
      if (e != cudaSuccess) return e;
      const int fgrid = static_cast<int>(min64((static_cast<int64_t>(a.n) + 255) / 256,
                                               static_cast<int64_t>(ctx->sm_count) * 16));
      k_hub_fill<MODE><<<fgrid, 256, 0, s>>>(a, ws, ctx->d_err);
      k_hub_items<<<n_grid, 256, 0, s>>>(ws);
      counted(ctx, a.n > 0 ? 5 : 3);
    }
    e = launch_hash_shape<MODE, true>(ctx, a, ws, s, kNames[MODE][3]);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace

CountWs carve_count(Carver& c, int32_t n, int64_t m, bool listing) {
  CountWs w{};
  const size_t n1 = static_cast<size_t>(n > 0 ? n : 1), m1 = static_cast<size_t>(m > 0 ? m : 1);
  w.big_queue = c.take<int32_t>(n1);
  w.counters = c.take<uint32_t>(kCtrSlots);
  w.off32 = c.take<int32_t>(n1 + 1);
  w.hub_idx = c.take<int32_t>(n1);
  w.hubs = c.take<int32_t>(n1);
  w.hub_cnt = c.take<int32_t>(n1);
  w.hub_fill = c.take<int32_t>(n1);
  w.hub_off = c.take<int64_t>(n1 + 1);
  w.rev_flag = c.take<uint8_t>(n1);
  w.hub_ent = c.take<int2>(m1);
  w.items_cap = hub_item_cap(n, m);
  w.hub_items = c.take<int2>(static_cast<size_t>(w.items_cap));
  w.hub_scan = carve_scan(c, n);
  if (listing) {
    w.ecount = c.take<int32_t>(static_cast<size_t>(m > 0 ? m : 1));
    w.erun = c.take<uint32_t>(static_cast<size_t>(m > 0 ? m : 1));
    w.eoff = c.take<int64_t>(static_cast<size_t>(m) + 1);
    w.scan = carve_scan(c, m);
  }
  return w;
}

int persistent_blocks(Ctx* ctx, const void* kernel, int threads, size_t dyn_smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int div = ctx->grid_div > 1 ? ctx->grid_div : 1;
  return static_cast<int>(max64(ctx->sm_count, static_cast<int64_t>(per_sm) * ctx->sm_count / div));
}

cudaError_t launch_count(Ctx* ctx, CountMode mode, const CountArgs& a_in, CountWs ws, cudaStream_t s) {
  // a write pass reusing the hub schedule keeps the hub and item counts of the counting pass
  cudaError_t e = cudaMemsetAsync(ws.counters, 0, sizeof(uint32_t) * (a_in.reuse_hub ? kCtrHubs : kCtrSlots), s);
  if (e != cudaSuccess) return e;
  if (a_in.n <= 0) return cudaGetLastError();
  CountArgs a = a_in;
  if (a.v_hi < 0) a.v_hi = a.n;
  if (a.cols_len < 0) a.cols_len = a.m;
  if (!a.apex_cols) {
    a.apex_cols = a.cols;
    a.apex_base = a.cols_base;
    a.apex_len = a.cols_len;
  } else if (a.apex_len < 0) {
    return cudaErrorInvalidValue;
  }
  if (a.u_hi < 0) a.u_hi = a.n;
  const bool split = a.apex_cols != a.cols || a.apex_base != a.cols_base || a.u_lo > 0 || a.u_hi < a.n;
  if (a.v_lo < 0 || a.v_lo > a.v_hi || a.v_hi > a.n) return cudaErrorInvalidValue;
  // the tile kernel packs a byte address of cols below bit 58 (virtual addresses are far narrower)
  if ((reinterpret_cast<uintptr_t>(a.cols) + 4u * static_cast<uint64_t>(a.cols_len)) >> 58) return cudaErrorInvalidValue;
  const int tile_ids = ctx->tile_shape == 2 ? TileShapeC::kIds : TileShapeA::kIds;
  a.tile_max = (ctx->tile_max > 0 && ctx->tile_max < tile_ids) ? ctx->tile_max : tile_ids;
  a.tile_quota = ctx->tile_quota;
  if (ws.off32 && a.m < (int64_t(1) << 31) - 1) a.off32 = ws.off32;  // filled by launch_mode
  // hub side: needs its workspace (absent in the allocation-free entry point)
  a.hub_min = (ws.hub_idx && ctx->hub_min >= 0) ? (ctx->hub_min > 0 ? ctx->hub_min : kHubMinDefault) : 0;
  // lists in two arrays: the apex-side kernels only (the hub side would hash N_u and
  // walk apex lists from the wrong array), and no listing
  if (split) {
    if (mode == MODE_LIST_COUNT || mode == MODE_LIST_WRITE) return cudaErrorInvalidValue;
    a.hub_min = 0;
  }
  switch (mode) {
    case MODE_COUNT: return launch_mode<MODE_COUNT>(ctx, a, ws, s);
    case MODE_LOCAL: return launch_mode<MODE_LOCAL>(ctx, a, ws, s);
    case MODE_LIST_COUNT: return launch_mode<MODE_LIST_COUNT>(ctx, a, ws, s);
    case MODE_LIST_WRITE: return launch_mode<MODE_LIST_WRITE>(ctx, a, ws, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_list_offsets(Ctx* ctx, int64_t m, CountWs ws, cudaStream_t s) {
  Stage st(ctx, s, "list.scan");
  counted(ctx, m > 0 ? 3 : 1);
  return exclusive_scan_i32(ws.ecount, ws.eoff, m, ws.scan, s);
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
