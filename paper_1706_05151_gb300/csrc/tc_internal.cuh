// Internal declarations shared by the libtc translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tc.h"

namespace tc {

// Bits of the device error word.  Kernels OR them in instead of faulting.
enum : uint32_t {
  ERR_BAD_ID = 1u << 0,     // vertex id outside [0, n)
  ERR_SELF_LOOP = 1u << 1,  // edge (v, v)
  ERR_DUPLICATE = 1u << 2,  // the same edge twice
  ERR_BAD_CSR = 1u << 3,    // offsets not monotone / outside [0, m]
  ERR_TOO_LONG = 1u << 4,   // a list longer than a documented limit
  ERR_CAPACITY = 1u << 5,   // listing output too small
  ERR_TIMEOUT = 1u << 6,    // a bounded wait ran out
};

constexpr unsigned FULL = 0xffffffffu;
constexpr int kSortBlockCap = 32768;     // longest list tc_orient sorts (ints in shared memory)
constexpr int kSortWarpCap = 1024;       // lists up to this length are sorted by one warp
constexpr int kMaxListLen = 1 << 24;     // longest list the counting kernels accept

// Optional per-stage timing: CUDA events recorded around each kernel group on
// the launching stream, resolved when the caller asks for the totals.
struct StageTotal {
  std::string name;
  double ms = 0.0;
  int64_t calls = 0;
};
struct PendingStage {
  int index;
  cudaEvent_t start, stop;
};
struct Profiler {
  bool on = false;
  std::vector<StageTotal> totals;
  std::vector<PendingStage> pending;
  std::vector<cudaEvent_t> pool;
};

// Context state (opaque to callers).
struct Ctx {
  int device = 0;
  int sm_count = 0;
  int async = 0;
  size_t smem_optin = 0;      // max dynamic shared memory per block (opt-in)
  uint32_t* d_err = nullptr;  // device error word
  uint32_t* h_err = nullptr;  // pinned host mirror
  int64_t launches = 0;       // kernels this context has launched
  int32_t tile_max = 0;       // tuning: longest N_v counted by the tile kernel (0 = its capacity)
  int32_t grid_div = 1;       // tuning: persistent grids use 1/grid_div of the resident capacity
  int32_t hub_min = 0;        // tuning: hub side for |N_u| >= hub_min (0: default, -1: off)
  int32_t tile_quota = 0;     // vertex chunks per warp before a tile-kernel block retires (0: persistent)
  int32_t tile_shape = 0;     // tuning: tile kernel shape (0: 256 ids x 8 windows, 1: 256 x 4, 2: 128 x 8)
  int32_t hash_batch = 32;    // tuning: walked lists per warp batch in the block and hub kernels (32 or 16)
  int32_t hash_windows = 4;   // tuning: candidate windows in flight per lane in those kernels (4 or 8)
  int capturing = 0;          // inside tc_capture_begin .. tc_capture_end
  int saved_async = 0;        // async flag before the capture
  int capture_status = 0;     // first failure inside the capture (0 = none)
  Profiler prof;
  cudaStream_t copy_stream = nullptr;  // tc_count_streamed: host-to-device list copies (created on first use)
  cudaEvent_t copy_ev[5] = {};         // ... two slots' "copied" and "free" events, one start event
  char last_error[256] = {0};
};

// Brackets one kernel group with profiling events (no-op when profiling is off).
class Stage {
 public:
  Stage(Ctx* ctx, cudaStream_t s, const char* name);
  ~Stage();
 private:
  Ctx* ctx_;
  cudaStream_t s_;
  int index_ = -1;
  cudaEvent_t start_ = nullptr;
};

// Count one kernel launch of this context.
inline void counted(Ctx* ctx, int n = 1) { ctx->launches += n; }

// Bump allocator over a caller workspace; with base == nullptr it only measures.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return (off + 255) & ~size_t(255); }
};

// ---- workspace layouts ----------------------------------------------------

struct ScanWs {
  int64_t* block_sums;  // one per scan tile, plus the total
};
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int64_t kScanTile = kScanThreads * kScanItems;
inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }
inline ScanWs carve_scan(Carver& c, int64_t n) { return ScanWs{c.take<int64_t>(scan_tiles(n) + 2)}; }

// Counter slots of CountWs::counters.
enum CountCounter : int {
  kCtrBigQueue = 0,  // vertices queued for the block kernel
  kCtrCursor = 1,    // vertex cursor of the tile kernel
  kCtrHubs = 2,      // hub vertices (|N_u| >= hub_min)
  kCtrItems = 3,     // work items of the hub kernel
  kCtrSlots = 8
};
constexpr int kHubSeg = 1024;  // in-edges of a hub per work item of the hub kernel

struct CountWs {
  int32_t* big_queue;   // vertices left to the block kernel
  uint32_t* counters;   // kCtrSlots counters (CountCounter)
  int32_t* ecount;      // listing: triangles per oriented edge (m)
  uint32_t* erun;       // listing: triples written per edge, carried across hash chunks (m)
  int64_t* eoff;        // listing: output offset per oriented edge (m + 1; eoff[m] = T)
  ScanWs scan;          // listing: scan over the m edge counts
  // hub side: edges (v, u) with |N_u| >= hub_min and |N_u| > |N_v| are counted
  // from u's side (NULL hub_idx: off)
  int32_t* off32;       // offsets as int32 when m < 2^31 (n + 1): half the bytes, L2-resident longer
  int32_t* hub_idx;     // per vertex: its index among the hubs, or -1 (n)
  int32_t* hubs;        // hub vertex of each index (n)
  int32_t* hub_cnt;     // edges counted from each hub's side (n)
  int32_t* hub_fill;    // fill cursor per hub (n)
  int64_t* hub_off;     // exclusive scan of hub_cnt (n + 1)
  uint8_t* rev_flag;    // per vertex v: some edge (v, u) goes to u's side (n)
  int2* hub_ent;        // per hub, its edges as (v, position of u in N_v) (m)
  int2* hub_items;      // work items (hub index, segment of kHubSeg edges) ...
  int64_t items_cap;    // ... room for this many
  ScanWs hub_scan;      // scan over hub_cnt
};
inline int64_t hub_item_cap(int32_t n, int64_t m) { return static_cast<int64_t>(n) + m / kHubSeg + 1; }
CountWs carve_count(Carver& c, int32_t n, int64_t m, bool listing);

struct OrientWs {
  int32_t* cursor;      // fill cursor per vertex
  uint8_t* deg8;        // min(d_v, 255): the order's comparisons gather these bytes (n)
  uint32_t* fwd;        // bit e: edge e is stored in the list of its first endpoint ((m + 31) / 32 words)
  int32_t* big_queue;   // vertices whose lists the block sorter takes (> kSortWarpCap ids)
  int32_t* mid_queue;   // vertices whose lists the warp sorter takes (33 .. kSortWarpCap ids)
  uint32_t* counters;   // [0] big queue length, [1] mid queue length
  ScanWs scan;
};
OrientWs carve_orient(Carver& c, int32_t n, int64_t m);

struct SparsifyWs {
  uint8_t* keep;        // coin per oriented edge (m)
  int32_t* kept_count;  // kept edges per vertex (n)
  int64_t* offsets;     // kept CSR offsets (n + 1)
  int32_t* cols;        // kept CSR columns (m)
  ScanWs scan;
  CountWs count;
};
SparsifyWs carve_sparsify(Carver& c, int32_t n, int64_t m);

// tc_count_streamed: the offsets' device copy, the counting kernels' scratch
// (no hub side) and the list buffer (half resident range, two quarter slots).
struct StreamWs {
  int64_t* offsets;     // n + 1
  CountWs count;
  int32_t* lists;       // list_ids
  int64_t list_ids;
};
StreamWs carve_stream(Carver& c, int32_t n, int64_t m, size_t list_bytes);
cudaError_t launch_count_streamed(Ctx* ctx, int32_t n, int64_t m, const int64_t* offsets_host,
                                  const int32_t* cols_host, uint64_t* total, int64_t* tv, StreamWs ws,
                                  cudaStream_t s, const char** why);

struct PartitionWs {
  int64_t* f;           // cost of each vertex (n)
  int64_t* F;           // exclusive scan of f (n + 1)
  ScanWs scan;
};
PartitionWs carve_partition(Carver& c, int32_t n);
cudaError_t launch_partition(Ctx* ctx, int32_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                             const int32_t* deg, int cost, int32_t parts, int64_t* bounds, uint64_t* part_cost,
                             PartitionWs ws, cudaStream_t s);

struct BatchWs {
  int32_t* edges;       // union edge list with global ids (2E)
  int32_t* gid;         // graph id per global vertex (N)
  OrientWs orient;
  CountWs count;
};
BatchWs carve_batch(Carver& c, int32_t n, int64_t m);
cudaError_t launch_batch_prepare(Ctx* ctx, int32_t G, int32_t N, int64_t E, const int64_t* vbase,
                                 const int64_t* ebase, const int32_t* edges_local, BatchWs ws, cudaStream_t s);

// ---- launchers (stream-ordered, no synchronisation) -------------------------

// With n_dev, the scan covers min(n, *n_dev) entries (a length a kernel earlier in the stream wrote).
cudaError_t exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, ScanWs ws, cudaStream_t s,
                               const uint32_t* n_dev = nullptr);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, ScanWs ws, cudaStream_t s);

// keys: NULL for the degree order of Eq. (1), else v precedes u iff (keys[v], v) < (keys[u], u).
// edges_host: when set, `edges` is filled from this page-locked copy in chunks on the
// context's copy stream, each chunk counted by the degree pass as soon as it lands.
cudaError_t launch_orient(Ctx* ctx, int32_t n, int64_t m, const int32_t* edges, int64_t* offsets,
                          int32_t* cols, int32_t* deg, int32_t* dhat, OrientWs ws, cudaStream_t s,
                          const int64_t* keys = nullptr, const int32_t* edges_host = nullptr);
// The context's copy stream and its five events (created on first use).
cudaError_t ensure_copy_stream(Ctx* ctx);

enum CountMode { MODE_COUNT = 0, MODE_LOCAL = 1, MODE_LIST_COUNT = 2, MODE_LIST_WRITE = 3 };

struct CountArgs {
  int32_t n;
  int64_t m;
  const int64_t* offsets;
  const int32_t* cols;
  unsigned long long* total;  // MODE_COUNT / MODE_LOCAL / MODE_LIST_COUNT
  int64_t* tv;                // MODE_LOCAL
  int32_t* tri;               // MODE_LIST_WRITE
  int64_t cap;                // MODE_LIST_WRITE
  unsigned long long* graph_total = nullptr;  // batched form: T per graph ...
  const int32_t* gid = nullptr;               // ... indexed by the graph id of the apex vertex
  int32_t tile_max = 0;                       // lists longer than this go to the block kernel (set by launch_count)
  int32_t hub_min = 0;                        // hub side for lists of at least this length (0: off; set by launch_count)
  int32_t tile_quota = 0;                     // chunks per warp before its block retires (0: until the work ends)
  int32_t tile_claim = 1;                     // 32-vertex chunks a warp of the tile kernel claims at once (set by launch_count)
  const int32_t* off32 = nullptr;             // int32 copy of offsets (set by launch_count when m < 2^31)
  int32_t v_lo = 0, v_hi = -1;                // apex vertices counted: [v_lo, v_hi) (-1: n)
  bool off32_ready = false;                   // off32 already holds these offsets (a sequence of calls on one graph)
  bool reuse_hub = false;                     // listing write pass: the hub schedule of the counting pass that
                                              // ran just before on the same workspace and thresholds is still valid
  // Lists held in two places (counting a CSR streamed from host memory): the apex
  // lists N_v are read at apex_cols[offsets[v] - apex_base] (apex_len ids), the lists
  // N_u at cols[offsets[u] - cols_base] (cols_len ids), and only edges (v, u) with u in
  // [u_lo, u_hi) are counted.  Defaults (set by launch_count): one array, every u.
  const int32_t* apex_cols = nullptr;
  int64_t apex_base = 0, apex_len = -1;
  int64_t cols_base = 0, cols_len = -1;
  int32_t u_lo = 0, u_hi = -1;
};
cudaError_t launch_count(Ctx* ctx, CountMode mode, const CountArgs& a, CountWs ws, cudaStream_t s);
// Listing: eoff = exclusive scan of ecount (after a MODE_LIST_COUNT or MODE_LOCAL pass).
cudaError_t launch_list_offsets(Ctx* ctx, int64_t m, CountWs ws, cudaStream_t s);
cudaError_t launch_clustering(Ctx* ctx, int32_t n, const int32_t* deg, const int64_t* tv, double* cc, cudaStream_t s);

cudaError_t launch_sparsify(Ctx* ctx, int32_t n, int64_t m, const int64_t* offsets, const int32_t* cols,
                            uint64_t threshold53, uint64_t seed, uint32_t part, SparsifyWs ws, int64_t* kept_edges,
                            cudaStream_t s);

// Grid of a persistent kernel: resident blocks per SM times the SM count.
int persistent_blocks(Ctx* ctx, const void* kernel, int threads, size_t dyn_smem);

// ---- device helpers -------------------------------------------------------------

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ void set_err(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

// L2 eviction priorities as per-instruction cache hints (createpolicy + .L2::cache_hint):
// they rank this kernel's lines against each other in L2 and change no device setting.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Read-only loads with an L2 policy (data that no kernel writes while the reader runs).
__device__ __forceinline__ int32_t ld_nc_hint(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int32_t ld_nc_l1na_hint(const int32_t* p, uint64_t pol) {  // and no L1 allocation
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int64_t ld_nc_hint(const int64_t* p, uint64_t pol) {
  int64_t v;
  asm("ld.global.nc.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}

}  // namespace tc
