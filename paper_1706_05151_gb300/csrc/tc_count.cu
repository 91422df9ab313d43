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

constexpr int kTile = 512;           // ids staged per warp; longer lists go to the block kernel
constexpr int kTileWarps = 4;        // warps per block, tile kernel
constexpr int kTileBitsLog2 = 14;    // filter bits per tile (2 KB): <= 512 / 16384 false positives
constexpr int kUnroll = 4;           // candidate windows in flight per lane
constexpr int kShortLen = 32;        // N_u shorter than this is walked end to end with others
constexpr int kOwnCap = 32 * kShortLen;
constexpr int kBlockWarps = 8;       // warps per block, block kernel

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
// Shared batch machinery.  A batch is up to 32 oriented edges (v, u), one per
// lane.  Short lists N_u (< kShortLen ids) are laid end to end and walked in
// 32-wide windows (an owner table maps a position to its edge); long lists are
// walked one edge at a time.  Every candidate w first meets a bitmap filter of
// the staged lists (one shared load and a bit test); the few that pass (true
// matches and about S / 2^bits false positives) are queued and checked exactly,
// 32 at a time, by binary search in the staged N_v.
// ---------------------------------------------------------------------------

// Multiplicative hash of (salt, id) onto a 2^LOG2-bit filter.
template <int LOG2>
__device__ __forceinline__ uint32_t fbit(int32_t w, int32_t salt) {
  return ((static_cast<uint32_t>(w) ^ (static_cast<uint32_t>(salt) << 26)) * 0x9E3779B1u) >> (32 - LOG2);
}

template <int LOG2>
__device__ __forceinline__ bool ftest(const uint32_t* bits, int32_t w, int32_t salt) {
  const uint32_t h = fbit<LOG2>(w, salt);
  return (bits[h >> 5] >> (h & 31)) & 1u;
}

template <int LOG2>
__device__ __forceinline__ void fset(uint32_t* bits, int32_t w, int32_t salt) {
  const uint32_t h = fbit<LOG2>(w, salt);
  atomicOr(&bits[h >> 5], 1u << (h & 31));
}

struct BatchSmem {
  int64_t beg[32];        // short list: start of N_u minus its flattened offset; long list: start of N_u
  int32_t u[32];
  int32_t lo[32];         // tile kernel: N_v's slice [lo, lo + len) of the tile
  int32_t len[32];
  int32_t salt[32];       // filter salt: chunk lane of v (tile kernel), 0 (block kernel)
  uint32_t cnt[32];       // matches of the edge
  int32_t qw[64];         // filter survivors: candidate id ...
  int32_t qs[64];         // ... and its edge
  uint8_t own[kOwnCap];   // flattened position -> edge, short lists
};

struct Probe {            // what the candidates are tested against
  const int32_t* sv;      // tile kernel: the tile; block kernel: the staged chunk of N_v
  const uint32_t* bits;   // filter of sv
  int top;                // binary-search span (power of two)
  int len;                // block kernel: chunk length
  int32_t lo, hi;         // block kernel: id range of the chunk
};

template <bool TILE>
__device__ __forceinline__ bool passes(const Probe& pr, int32_t salt, int32_t w) {
  return ftest<kTileBitsLog2>(pr.bits, w, salt);
}

// Exact check of the first `cnt` queued survivors, with the per-mode effects.
template <int MODE, bool TILE>
__device__ __forceinline__ void exact_flush(BatchSmem& bs, const Probe& pr, int cnt, int32_t vbase_or_v, int32_t* vrun,
                                            unsigned long long* cursor, const CountArgs& a, const CountWs& ws,
                                            uint32_t* err) {
  const int lane = lane_id();
  __syncwarp();
  const bool has = lane < cnt;
  const int s = has ? bs.qs[lane] : 0;
  const int32_t w = has ? bs.qw[lane] : 0;
  bool f = false;
  if (has) f = TILE ? member(pr.sv + bs.lo[s], bs.len[s], pr.top, w) : member(pr.sv, pr.len, pr.top, w);
  if (f) {
    atomicAdd(&bs.cnt[s], 1u);
    if (MODE == MODE_LOCAL) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + w), 1ull);
  }
  if (MODE == MODE_LIST_WRITE) {
    const unsigned fm = __ballot_sync(FULL, f);
    if (fm) {
      if (TILE) {
        // triples of one apex vertex are written in queue order at voff[v] + running count
        const int vl = bs.salt[s];
        const unsigned same = __match_any_sync(FULL, has ? vl : 32 + lane);
        if (f) {
          const int32_t v = vbase_or_v + vl;
          const int64_t idx = ws.voff[v] + vrun[vl] + __popc(fm & same & lanemask_lt());
          if (idx < a.cap) {
            a.tri[3 * idx] = v;
            a.tri[3 * idx + 1] = bs.u[s];
            a.tri[3 * idx + 2] = w;
          } else {
            set_err(err, ERR_CAPACITY);
          }
        }
        __syncwarp();
        if (has && lane == 31 - __clz(same)) vrun[vl] += __popc(fm & same);
      } else {
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(cursor, static_cast<unsigned long long>(__popc(fm)));
        const int64_t base = static_cast<int64_t>(__shfl_sync(FULL, b0, 0));
        if (f) {
          const int64_t idx = base + __popc(fm & lanemask_lt());
          if (idx < a.cap) {
            a.tri[3 * idx] = vbase_or_v;
            a.tri[3 * idx + 1] = bs.u[s];
            a.tri[3 * idx + 2] = w;
          } else {
            set_err(err, ERR_CAPACITY);
          }
        }
      }
    }
  }
  __syncwarp();
}

// Queue this window's survivors; check 32 of them once 32 are waiting.
template <int MODE, bool TILE>
__device__ __forceinline__ void push(BatchSmem& bs, const Probe& pr, bool pass, int32_t w, int s, int& qn,
                                     int32_t vbase_or_v, int32_t* vrun, unsigned long long* cursor,
                                     const CountArgs& a, const CountWs& ws, uint32_t* err) {
  const int lane = lane_id();
  const unsigned m = __ballot_sync(FULL, pass);
  if (!m) return;
  if (pass) {
    const int pos = qn + __popc(m & lanemask_lt());
    bs.qw[pos] = w;
    bs.qs[pos] = s;
  }
  qn += __popc(m);
  if (qn >= 32) {
    exact_flush<MODE, TILE>(bs, pr, 32, vbase_or_v, vrun, cursor, a, ws, err);
    const int rest = qn - 32;
    int32_t tw = 0, ts = 0;
    if (lane < rest) {
      tw = bs.qw[32 + lane];
      ts = bs.qs[32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
      bs.qw[lane] = tw;
      bs.qs[lane] = ts;
    }
    __syncwarp();
    qn = rest;
  }
}

// One batch of edges (v, u): u on this lane if `act`.  Returns the matches of
// this lane's edge.  salt/lo/vlen describe this lane's N_v (tile kernel).
template <int MODE, bool TILE>
__device__ __forceinline__ uint32_t process_batch(BatchSmem& bs, const Probe& pr, int32_t u, bool act, int32_t salt,
                                                  int32_t lo, int32_t vlen, int32_t vbase_or_v, int32_t* vrun,
                                                  unsigned long long* cursor, const CountArgs& a,
                                                  const CountWs& ws, uint32_t* err) {
  const int lane = lane_id();
  int64_t ub = 0;
  int32_t len = 0;
  if (act) len = list_bounds(a, u, ub, err);
  const bool is_short = len < kShortLen;
  const int32_t slen = is_short ? len : 0;
  const int32_t incl = warp_incl_scan(slen);
  const int32_t tot = __shfl_sync(FULL, incl, 31);
  const int32_t excl = incl - slen;
  __syncwarp();
  bs.beg[lane] = is_short ? ub - excl : ub;
  bs.u[lane] = u;
  bs.lo[lane] = lo;
  bs.len[lane] = vlen;
  bs.salt[lane] = salt;
  bs.cnt[lane] = 0;
  for (int i = 0; i < slen; ++i) bs.own[excl + i] = static_cast<uint8_t>(lane);
  __syncwarp();
  int qn = 0;
  // short lists, end to end
  for (int32_t p0 = 0; p0 < tot; p0 += 32 * kUnroll) {
    int32_t w[kUnroll];
    int s[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      s[k] = 0;
      w[k] = 0;
      if (p < tot) {
        s[k] = bs.own[p];
        w[k] = a.cols[bs.beg[s[k]] + p];
      }
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      const bool pass = p < tot && passes<TILE>(pr, bs.salt[s[k]], w[k]);
      push<MODE, TILE>(bs, pr, pass, w[k], s[k], qn, vbase_or_v, vrun, cursor, a, ws, err);
    }
  }
  // long lists, one edge at a time
  unsigned lm = __ballot_sync(FULL, act && !is_short);
  while (lm) {
    const int e = __ffs(lm) - 1;
    lm &= lm - 1;
    const int64_t b = bs.beg[e];
    const int32_t le = __shfl_sync(FULL, len, e);
    const int32_t se = bs.salt[e];
    for (int32_t p0 = 0; p0 < le; p0 += 32 * kUnroll) {
      int32_t w[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int32_t p = p0 + 32 * k + lane;
        w[k] = p < le ? a.cols[b + p] : 0;
      }
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int32_t p = p0 + 32 * k + lane;
        const bool pass = p < le && passes<TILE>(pr, se, w[k]);
        push<MODE, TILE>(bs, pr, pass, w[k], e, qn, vbase_or_v, vrun, cursor, a, ws, err);
      }
    }
  }
  if (qn) exact_flush<MODE, TILE>(bs, pr, qn, vbase_or_v, vrun, cursor, a, ws, err);
  __syncwarp();
  return act ? bs.cnt[lane] : 0u;
}

// ---------------------------------------------------------------------------
// Tile kernel
// ---------------------------------------------------------------------------

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

struct TileSmem {
  int32_t tile[kTile];
  uint32_t bits[(1 << kTileBitsLog2) / 32];
  int32_t vlo[32];     // tile start of each chunk lane's list (-1 before the group, > S after)
  uint32_t vcnt[32];   // triangles with apex v (chunk lane)
  int32_t vrun[32];    // listing: triples written so far per chunk lane
  BatchSmem bs;
};

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
    // the listing write pass only revisits apex vertices that have triangles
    const bool skip = MODE == MODE_LIST_WRITE && valid && ws.vcount[v] == 0;
    const bool big = valid && !skip && d > a.tile_max;
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
      const int32_t len = (lane >= g0 && valid && !big && !skip) ? static_cast<int32_t>(d) : 0;
      const int32_t incl = warp_incl_scan(len);
      const bool stop = lane >= g0 && (!valid || big || skip || incl > kTile);
      const unsigned smask = __ballot_sync(FULL, stop);
      const int g1 = smask ? __ffs(smask) - 1 : 32;
      if (g1 == g0) {  // lane g0 is past the end, a queued long list or skipped
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
      for (int i = lane; i < (1 << kTileBitsLog2) / 32; i += 32) sm.bits[i] = 0u;
      const int32_t lo = incl - len;
      sm.vlo[lane] = lane < g0 ? -1 : (lane < g1 ? lo : S + 1);
      sm.vcnt[lane] = 0;
      sm.vrun[lane] = 0;
      if (__any_sync(FULL, bad)) {
        if (lane == 0) set_err(err, ERR_BAD_ID);
        g0 = g1;
        continue;
      }
      __syncwarp();
      for (int i = 0; i < glen; ++i) fset<kTileBitsLog2>(sm.bits, sm.tile[lo + i], lane);
      const int maxlen = __reduce_max_sync(FULL, glen);
      const Probe pr{sm.tile, sm.bits, maxlen > 0 ? 1 << (31 - __clz(maxlen)) : 0, 0, 0, 0};
      __syncwarp();
      for (int t0 = 0; t0 < S; t0 += 32) {
        const int t = t0 + lane;
        const bool act = t < S;
        const int vl = act ? search32(sm.vlo, static_cast<int32_t>(t)) : 0;
        const int32_t u = act ? sm.tile[t] : 0;
        const int32_t vlen = __shfl_sync(FULL, glen, vl);
        const uint32_t c = process_batch<MODE, true>(sm.bs, pr, u, act, vl, sm.vlo[vl], vlen,
                                                     static_cast<int32_t>(base), sm.vrun, nullptr, a, ws, err);
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
        if ((MODE == MODE_LIST_COUNT || MODE == MODE_LOCAL) && ws.vcount) ws.vcount[v] = cv;
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
// no survivor queue and no binary search.
// ---------------------------------------------------------------------------

constexpr int kHashSlotsLog2 = 13;                   // 8192 slots (32 KB)
constexpr int kHashCap = (1 << kHashSlotsLog2) / 4;  // ids of N_v per pass

__device__ __forceinline__ uint32_t slot_of(int32_t w) {
  return (static_cast<uint32_t>(w) * 0x9E3779B1u) >> (32 - kHashSlotsLog2);
}

__device__ __forceinline__ bool hash_member(const int32_t* tab, int32_t w) {
  if (w < 0) return false;
  uint32_t h = slot_of(w);
  for (int probe = 0; probe < (1 << kHashSlotsLog2); ++probe) {  // bounded: the table is never full
    const int32_t x = tab[h];
    if (x == w) return true;
    if (x < 0) return false;
    h = (h + 1) & ((1u << kHashSlotsLog2) - 1);
  }
  return false;
}

__device__ __forceinline__ void hash_insert(int32_t* tab, int32_t w) {
  uint32_t h = slot_of(w);
  for (int probe = 0; probe < (1 << kHashSlotsLog2); ++probe) {
    const int32_t prev = atomicCAS(&tab[h], -1, w);
    if (prev == -1 || prev == w) return;
    h = (h + 1) & ((1u << kHashSlotsLog2) - 1);
  }
}

struct HashBatch {
  int64_t beg[32];        // short list: start of N_u minus its flattened offset; long list: start of N_u
  int32_t u[32];
  uint32_t cnt[32];       // matches of the edge
  uint8_t own[kOwnCap];   // flattened position -> edge, short lists
};

template <int MODE>
__device__ __forceinline__ void hash_record(HashBatch& hb, bool found, int32_t w, int s, int32_t v,
                                            unsigned long long* cursor, const CountArgs& a, uint32_t* err) {
  if (found) {
    atomicAdd(&hb.cnt[s], 1u);
    if (MODE == MODE_LOCAL) atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + w), 1ull);
  }
  if (MODE == MODE_LIST_WRITE) {
    const unsigned fm = __ballot_sync(FULL, found);
    if (fm) {
      unsigned long long b0 = 0;
      if (lane_id() == 0) b0 = atomicAdd(cursor, static_cast<unsigned long long>(__popc(fm)));
      const int64_t base = static_cast<int64_t>(__shfl_sync(FULL, b0, 0));
      if (found) {
        const int64_t idx = base + __popc(fm & lanemask_lt());
        if (idx < a.cap) {
          a.tri[3 * idx] = v;
          a.tri[3 * idx + 1] = hb.u[s];
          a.tri[3 * idx + 2] = w;
        } else {
          set_err(err, ERR_CAPACITY);
        }
      }
    }
  }
}

// One batch of edges (v, u), u on this lane if `act`, against the hashed chunk
// of N_v whose ids lie in [lo, hi].  Returns the matches of this lane's edge.
template <int MODE>
__device__ __forceinline__ uint32_t hash_batch(HashBatch& hb, const int32_t* tab, int32_t lo, int32_t hi, int32_t u,
                                               bool act, int32_t v, unsigned long long* cursor, const CountArgs& a,
                                               uint32_t* err) {
  const int lane = lane_id();
  int64_t ub = 0;
  int32_t len = 0;
  if (act) len = list_bounds(a, u, ub, err);
  const bool is_short = len < kShortLen;
  const int32_t slen = is_short ? len : 0;
  const int32_t incl = warp_incl_scan(slen);
  const int32_t tot = __shfl_sync(FULL, incl, 31);
  const int32_t excl = incl - slen;
  __syncwarp();
  hb.beg[lane] = is_short ? ub - excl : ub;
  hb.u[lane] = u;
  hb.cnt[lane] = 0;
  for (int i = 0; i < slen; ++i) hb.own[excl + i] = static_cast<uint8_t>(lane);
  __syncwarp();
  for (int32_t p0 = 0; p0 < tot; p0 += 32 * kUnroll) {
    int32_t w[kUnroll];
    int s[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int32_t p = p0 + 32 * k + lane;
      s[k] = 0;
      w[k] = -1;
      if (p < tot) {
        s[k] = hb.own[p];
        w[k] = a.cols[hb.beg[s[k]] + p];
      }
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const bool found = w[k] >= lo && w[k] <= hi && hash_member(tab, w[k]);
      hash_record<MODE>(hb, found, w[k], s[k], v, cursor, a, err);
    }
  }
  unsigned lm = __ballot_sync(FULL, act && !is_short);
  while (lm) {
    const int e = __ffs(lm) - 1;
    lm &= lm - 1;
    const int64_t b = hb.beg[e];
    const int32_t le = __shfl_sync(FULL, len, e);
    for (int32_t p0 = 0; p0 < le; p0 += 32 * kUnroll) {
      int32_t w[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int32_t p = p0 + 32 * k + lane;
        w[k] = p < le ? a.cols[b + p] : -1;
      }
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const bool found = w[k] >= lo && w[k] <= hi && hash_member(tab, w[k]);
        hash_record<MODE>(hb, found, w[k], e, v, cursor, a, err);
      }
    }
  }
  __syncwarp();
  return act ? hb.cnt[lane] : 0u;
}

template <int MODE>
__global__ void __launch_bounds__(kBlockWarps * 32, 4) k_count_block(CountArgs a, CountWs ws, uint32_t* err) {
  extern __shared__ int32_t tab[];
  __shared__ HashBatch s_hb[kBlockWarps];
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
    for (int64_t c0 = 0; c0 < dv; c0 += kHashCap) {
      const int clen = static_cast<int>(min64(kHashCap, dv - c0));
      __syncthreads();
      for (int i = threadIdx.x; i < (1 << kHashSlotsLog2); i += blockDim.x) tab[i] = -1;
      __syncthreads();
      bool bad = false;
      for (int i = threadIdx.x; i < clen; i += blockDim.x) {
        const int32_t x = a.cols[b + c0 + i];
        if (static_cast<uint32_t>(x) >= static_cast<uint32_t>(a.n)) bad = true;
        else hash_insert(tab, x);
      }
      if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) set_err(err, ERR_BAD_ID);
        break;
      }
      // the chunk is a sorted run of N_v: its ids lie in [lo, hi]
      const int32_t lo = a.cols[b + c0], hi = a.cols[b + c0 + clen - 1];
      for (int64_t ub = static_cast<int64_t>(wid) * 32; ub < dv; ub += kBlockWarps * 32) {
        const int nb = static_cast<int>(min64(32, dv - ub));
        const bool act = lane < nb;
        const int32_t u = act ? a.cols[b + ub + lane] : 0;
        const uint32_t c = hash_batch<MODE>(s_hb[wid], tab, lo, hi, u, act, v, &s_cursor, a, err);
        cv += c;
        if (MODE == MODE_LOCAL && c)
          atomicAdd(reinterpret_cast<unsigned long long*>(a.tv + u), static_cast<unsigned long long>(c));
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
      if (MODE != MODE_LIST_WRITE && a.graph_total && t) atomicAdd(a.graph_total + a.gid[v], t);
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
  // persistent grids, but no more blocks than there is work for (small graphs leave room for other streams)
  const int tgrid = static_cast<int>(min64(
      persistent_blocks(ctx, reinterpret_cast<const void*>(&k_count_tile<MODE>), kTileWarps * 32, 0),
      max64(1, (static_cast<int64_t>(a.n) + 32 * kTileWarps - 1) / (32 * kTileWarps))));
  {
    Stage st(ctx, s, kNames[MODE][0]);
    k_count_tile<MODE><<<tgrid, kTileWarps * 32, 0, s>>>(a, ws, ctx->d_err);
  }
  const size_t smem = sizeof(int32_t) << kHashSlotsLog2;
  const int bgrid = static_cast<int>(min64(
      persistent_blocks(ctx, reinterpret_cast<const void*>(&k_count_block<MODE>), kBlockWarps * 32, smem),
      max64(1, a.m / (a.tile_max + 1))));  // at most m / (tile_max + 1) lists go to this kernel
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
  const int div = ctx->grid_div > 1 ? ctx->grid_div : 1;
  return static_cast<int>(max64(ctx->sm_count, static_cast<int64_t>(per_sm) * ctx->sm_count / div));
}

cudaError_t launch_count(Ctx* ctx, CountMode mode, const CountArgs& a_in, CountWs ws, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ws.counters, 0, sizeof(uint32_t) * 4, s);
  if (e != cudaSuccess) return e;
  if (a_in.n <= 0) return cudaGetLastError();
  CountArgs a = a_in;
  a.tile_max = (ctx->tile_max > 0 && ctx->tile_max < kTile) ? ctx->tile_max : kTile;
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
