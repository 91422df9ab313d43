/*
 * tc.h -- C ABI of libtc, exact triangle counting on one GPU (sm_103a).
 *
 * The library implements the hot path of Arifuzzaman, Khan and Marathe,
 * "Distributed-Memory Parallel Algorithms for Counting and Listing Triangles
 * in Big Graphs": orient an undirected simple graph by the degree order of
 * Eq. (1) into sorted out-neighbour lists N_v (Definition 1, the preprocessing
 * of NodeIteratorN, Figure 2), then sum |N_v intersect N_u| over every
 * oriented edge (v, u) (Figure 2, counting loop; Theorem 1 shows each triangle
 * is found once).  The same pass gives per-vertex counts T_v (Section 11,
 * Figure "localcount"), local clustering coefficients C_v (Preliminaries),
 * the triangle list (Section 10, Figure "tlisting") and the edge-sparsified
 * estimate T'/q^3 (Section 9.1, Figure "sparsification").
 *
 * Conventions shared by every call:
 *   - Vertex ids are int32 in [0, n); CSR offsets are int64; counts are
 *     64-bit integers and exact.
 *   - Pointers documented "device" must point to memory of the context's
 *     device (cudaMalloc'd, e.g. by PyTorch); "host" pointers to host memory.
 *   - The caller owns every buffer.  Calls that need scratch memory take a
 *     device workspace `ws` of `ws_bytes` bytes, at least what
 *     tc_workspace_size() reports for that operation and graph size, aligned
 *     to 256 bytes.  No call allocates device memory after tc_ctx_create.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     device work is enqueued on it.  In the default synchronous mode a call
 *     returns after that work has finished and reports input errors found on
 *     the device; after tc_ctx_set_async(ctx, 1) calls only enqueue and return
 *     TC_OK, and tc_ctx_status() reports the device-side checks later.
 *   - Errors are returned as tc_status, never by abort; tc_last_error(ctx)
 *     gives a one-line description of the last failure on that context.
 *   - A tc_ctx is not thread-safe: use one per host thread (or per stream).
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter (checked on the host) */
  TC_ERR_INVALID_GRAPH = 2, /* id outside [0, n), self-loop, repeated edge or broken CSR */
  TC_ERR_WORKSPACE = 3,     /* ws_bytes smaller than tc_workspace_size() */
  TC_ERR_CAPACITY = 4,      /* listing output buffer too small */
  TC_ERR_CUDA = 5,          /* a CUDA runtime call failed (see tc_last_error) */
  TC_ERR_UNSUPPORTED = 6,   /* a size beyond a documented limit */
  TC_ERR_TIMEOUT = 7,       /* a bounded wait ran out */
  TC_ERR_REJECTED = 8,      /* admission refused (serving) */
  TC_ERR_NOT_READY = 9      /* result not finished yet (serving) */
} tc_status;

/* Operations whose workspace size tc_workspace_size() reports. */
typedef enum {
  TC_OP_ORIENT = 0,
  TC_OP_COUNT = 1,       /* tc_count and tc_count_local */
  TC_OP_LIST = 2,        /* tc_list, tc_list_count, tc_list_write, tc_analyze */
  TC_OP_SPARSIFY = 3,    /* tc_sparsify_count */
  TC_OP_BATCH = 4,       /* tc_batch: n = total vertices N, m = total edges E */
  TC_OP_PARTITION = 5    /* tc_partition */
} tc_op;

typedef struct tc_ctx tc_ctx;
typedef void* tc_stream; /* cudaStream_t */

/*
 * An oriented graph in device memory, as tc_orient produces it:
 *   offsets[n+1]  int64, offsets[0] = 0, offsets[n] = m, non-decreasing;
 *   cols[m]       int32, cols[offsets[v] .. offsets[v+1]) = N_v, the ids u with
 *                 v preceding u in the order of Eq. (1), sorted ascending;
 *   deg[n]        int32, the undirected degree d_v (may be NULL for tc_count,
 *                 tc_list and tc_sparsify_count; required for clustering);
 *   dhat[n]       int32, the effective degree |N_v| (Definition 1; optional).
 * The counting calls need only a CSR whose lists are sorted, strictly
 * increasing and form an acyclic orientation; they check offsets and ids
 * against n and m and report TC_ERR_INVALID_GRAPH instead of reading out of
 * bounds.  The four arrays may also live in host memory the GPU can address
 * (page-locked memory, or system memory on a coherent CPU-GPU node): the
 * kernels then read the graph over the CPU-GPU link, for graphs larger than
 * the device memory left free (outputs and workspace stay on the device).
 */
typedef struct {
  int32_t n;
  int64_t m;
  const int64_t* offsets;
  const int32_t* cols;
  const int32_t* deg;
  const int32_t* dhat;
} tc_graph;

/* ---- context ----------------------------------------------------------- */

/* Create a context bound to CUDA device `device` (sets it current on this thread). */
tc_status tc_ctx_create(int device, tc_ctx** out);
void tc_ctx_destroy(tc_ctx* ctx);
/* async = 1: calls only enqueue work; async = 0 (default): calls wait and check. */
tc_status tc_ctx_set_async(tc_ctx* ctx, int async);
/* Wait for `stream` and report the device-side checks of the calls enqueued since the last report. */
tc_status tc_ctx_status(tc_ctx* ctx, tc_stream stream);
const char* tc_status_string(tc_status s);
const char* tc_last_error(const tc_ctx* ctx);
/* Number of SMs of the context's device (sizes persistent grids). */
int tc_ctx_sm_count(const tc_ctx* ctx);
/* Library version string. */
const char* tc_version(void);

/*
 * Tuning (no counterpart in the paper; the paper balances processors with the
 * cost functions of Table "lbscheme", this balances one GPU).  tile_max: apex
 * vertices with |N_v| > tile_max are counted one thread block per vertex, the
 * others 32 to a warp (0 = 256, the warp tile's capacity; values up to 512 are
 * accepted and act as 256).  grid_div: persistent
 * grids use 1/grid_div of the GPU's resident capacity (0 or 1 = all of it),
 * leaving room for work on other streams.  Results do not depend on either.
 */
tc_status tc_ctx_set_tuning(tc_ctx* ctx, int32_t tile_max, int32_t grid_div);

/*
 * Kernel shapes (no counterpart in the paper; chosen by the autotuner).  The
 * warp-tile kernel stages tile_ids ids per warp and keeps tile_windows
 * candidate windows in flight per lane: 256 x 8 (the default, also 0 x 0),
 * 256 x 4 or 128 x 8 (with 128, apex lists longer than 128 ids go to the block
 * kernel whatever tile_max says).  hash_batch: walked lists a warp takes at a
 * time in the block and hub kernels, 32 (default, also 0) or 16; hash_windows:
 * candidate windows each lane of those kernels keeps in flight, 4 (default,
 * also 0) or 8.  Other values: TC_ERR_INVALID_ARG.  Results do not depend on
 * the shapes.
 */
tc_status tc_ctx_set_kernel_shape(tc_ctx* ctx, int32_t tile_ids, int32_t tile_windows, int32_t hash_batch,
                                  int32_t hash_windows);

/*
 * Hub side of the intersection (a cost split; results never depend on it).
 * Theorem 2's work for an oriented edge (v, u) is reading N_v and N_u; the
 * counting kernels keep the apex list N_v on chip and stream N_u.  When N_u
 * is long (at least hub_min ids) and longer than N_v, the edge is instead
 * counted from u's side: N_u is hashed into shared memory once for all such
 * edges of u and each short N_v is streamed, so the per-edge read falls from
 * |N_u| to |N_v|.  hub_min = 0 restores the default (64); -1 turns the hub
 * side off; other negative values give TC_ERR_INVALID_ARG.
 */
tc_status tc_ctx_set_hub_min(tc_ctx* ctx, int32_t hub_min);

/*
 * Per-stage timing and launch accounting (no counterpart in the paper; it
 * measures this library).  With profiling on, each kernel group a call
 * launches is bracketed by CUDA events on the call's stream; the totals are
 * resolved (waiting on those events) when read.  Stage names are
 * "<operation>.<kernel>", e.g. "local.warp" for the per-vertex counting kernel.
 */
tc_status tc_ctx_set_profiling(tc_ctx* ctx, int on);
/* Number of stages seen so far (waits for pending stage events). */
int tc_ctx_stage_count(tc_ctx* ctx);
/* Stage i: *name (owned by ctx), total milliseconds and number of timed calls. */
tc_status tc_ctx_stage(tc_ctx* ctx, int i, const char** name, double* ms, int64_t* calls);
/* Clear stage totals and the launch counter. */
tc_status tc_ctx_reset_stats(tc_ctx* ctx);
/* Kernels this context has launched since creation or the last reset. */
int64_t tc_ctx_launches(const tc_ctx* ctx);

/*
 * Bytes of device workspace operation `op` needs for a graph of n vertices
 * and m edges (m undirected edges = m oriented edges).  Writes *bytes.
 */
tc_status tc_workspace_size(tc_op op, int32_t n, int64_t m, size_t* bytes);

/* ---- orientation (Eq. (1), Definition 1, Figure 2 preprocessing) -------- */

/*
 * Build the oriented CSR of the undirected simple graph given as an edge list.
 *   edges   device int32[m][2]: each undirected edge exactly once, either
 *           direction, any order.
 *   offsets device int64[n+1], cols device int32[m], deg device int32[n],
 *   dhat    device int32[n]: outputs as described for tc_graph.
 * The order is u precedes v iff d_u < d_v, or d_u = d_v and u < v (Eq. (1));
 * each N_v is sorted ascending by id (Figure 2).  Ids outside [0, n),
 * self-loops and repeated edges give TC_ERR_INVALID_GRAPH (outputs are then
 * unspecified but every access stays in bounds).  Lists longer than 2^24 ids
 * give TC_ERR_UNSUPPORTED (the degree order bounds |N_v| by sqrt(2m); lists
 * beyond 32768 ids are sorted in global memory; under the degree order a list
 * holds at most about sqrt(2m) ids, which passes 32768 once m exceeds ~5.4e8).
 */
tc_status tc_orient(tc_ctx* ctx, int32_t n, int64_t m, const int32_t* edges, int64_t* offsets,
                    int32_t* cols, int32_t* deg, int32_t* dhat, void* ws, size_t ws_bytes,
                    tc_stream stream);

/*
 * Orientation by another total order (Section "An Optimal Node Ordering": any
 * order counts each triangle once; Theorem 3: the degree order minimises the
 * counting cost sum_v d_v * dhat_v).  u precedes v iff keys[u] < keys[v], or
 * keys[u] = keys[v] and u < v.  keys_dev: device int64[n]; NULL gives the
 * degree order (= tc_orient).  Examples: all keys equal -- the id order; a
 * random permutation -- a random order; d_v -- Eq. (1).  Everything else as
 * tc_orient (deg is still the degree).  The counting calls work on any such
 * orientation.
 */
tc_status tc_orient_by(tc_ctx* ctx, int32_t n, int64_t m, const int32_t* edges, const int64_t* keys_dev,
                       int64_t* offsets, int32_t* cols, int32_t* deg, int32_t* dhat, void* ws, size_t ws_bytes,
                       tc_stream stream);

/*
 * tc_orient from an edge list in host memory (the same orientation; the
 * upload overlap has no counterpart in the paper).  edges_host: page-locked
 * host int32[m][2] (cudaHostAlloc or cudaHostRegister; other host memory gives
 * TC_ERR_INVALID_ARG); it must stay valid until the stream has passed this
 * call.  edges_dev: device int32[m][2], 8-byte aligned, caller-owned, which
 * receives the copy (overwritten; afterwards it holds the edge list).  The list
 * is copied in chunks of 2^24 edges on a stream of the context's own, and the
 * degree pass counts each chunk as soon as it has landed, so the copy and the
 * degree pass overlap; the rest of the orientation runs after the last chunk.
 * The copies start only after the work queued on `stream` before this call.
 * Outputs, workspace (TC_OP_ORIENT) and errors as tc_orient.
 */
tc_status tc_orient_host(tc_ctx* ctx, int32_t n, int64_t m, const int32_t* edges_host, int32_t* edges_dev,
                         int64_t* offsets, int32_t* cols, int32_t* deg, int32_t* dhat, void* ws, size_t ws_bytes,
                         tc_stream stream);

/* ---- counting (Figure 2 counting loop; Theorems 1-2) --------------------- */

/*
 * T = sum over oriented edges (v, u) of |N_v intersect N_u|.
 *   total_dev  device uint64[1], overwritten with T.
 */
tc_status tc_count(tc_ctx* ctx, const tc_graph* g, uint64_t* total_dev, void* ws, size_t ws_bytes,
                   tc_stream stream);

/*
 * T plus per-vertex counts (Section 11, Figure "localcount": each triangle
 * adds one to each of its three vertices) and, if cc_dev is not NULL, the
 * local clustering coefficients C_v = 2 T_v / (d_v (d_v - 1)) in float64,
 * one IEEE division, C_v = 0 when d_v < 2 (needs g->deg).
 *   total_dev device uint64[1]; tv_dev device int64[n]; cc_dev device double[n] or NULL.
 */
tc_status tc_count_local(tc_ctx* ctx, const tc_graph* g, uint64_t* total_dev, int64_t* tv_dev,
                         double* cc_dev, void* ws, size_t ws_bytes, tc_stream stream);

/* ---- listing (Section 10, Figure "tlisting") ------------------------------ */

/*
 * Two-pass listing.  tc_list_count counts the triangles of each apex vertex v
 * (the lowest of the three in the order), scans them into output positions
 * kept in `ws`, and writes the total to total_dev (device int64[1]).
 * tc_list_write, given the same g and ws right after tc_list_count, writes
 * every triangle as an int32 triple (v, u, w) with v < u < w in the order,
 * u in N_v and w in N_v intersect N_u, into tri_dev (device int32[cap][3]).
 * Triples of one apex vertex are contiguous; apex vertices appear in id order.
 * If the total exceeds cap nothing is written and the device-side check
 * reports TC_ERR_CAPACITY.
 */
tc_status tc_list_count(tc_ctx* ctx, const tc_graph* g, int64_t* total_dev, void* ws, size_t ws_bytes,
                        tc_stream stream);
tc_status tc_list_write(tc_ctx* ctx, const tc_graph* g, int32_t* tri_dev, int64_t cap, void* ws,
                        size_t ws_bytes, tc_stream stream);
/*
 * Both passes in one call.  Waits for the count (even in async mode) to check
 * it against cap.  *count_out (host) receives the number of triangles; with
 * TC_ERR_CAPACITY it holds the capacity needed and nothing was written.
 */
tc_status tc_list(tc_ctx* ctx, const tc_graph* g, int32_t* tri_dev, int64_t cap, int64_t* count_out,
                  void* ws, size_t ws_bytes, tc_stream stream);

/*
 * T, per-vertex counts, clustering coefficients and the triangle list in two
 * passes of the intersection instead of three: pass 1 computes T, T_v
 * (Section 11) and the triangles of each apex vertex; C_v follows
 * (Preliminaries); a scan turns the apex counts into output positions; pass 2
 * writes the triples as tc_list_write does (Section 10).  Waits after pass 1
 * (even in async mode) to check the total against cap.
 *   total_dev device uint64[1]; tv_dev device int64[n]; cc_dev device double[n]
 *   or NULL (needs g->deg); tri_dev device int32[cap][3]; *count_out (host)
 *   receives T.  With TC_ERR_CAPACITY, T, T_v and C_v are complete, *count_out
 *   holds the capacity needed and no triple was written.  Workspace: TC_OP_LIST.
 */
tc_status tc_analyze(tc_ctx* ctx, const tc_graph* g, uint64_t* total_dev, int64_t* tv_dev, double* cc_dev,
                     int32_t* tri_dev, int64_t cap, int64_t* count_out, void* ws, size_t ws_bytes,
                     tc_stream stream);

/* ---- sparsification (Section 9.1, Figure "sparsification") ---------------- */

/*
 * Keep each undirected edge {a, b} independently with probability q and
 * count the triangles T' of the kept graph, whose orientation is the one of
 * the ORIGINAL degrees (the order is fixed before sampling).  The coin of
 * {a, b} is Philox4x32-10 (Salmon et al., SC'11) with 32-bit counter words
 * (min(a,b), max(a,b), 0, 0) and key (lo32(seed), hi32(seed)): with r the top 53
 * bits of the first two output words (r = x0 * 2^21 + (x1 >> 11)), keep iff
 * r < ceil(q * 2^53), i.e. r * 2^-53 < q.
 *   q in [0, 1]; kept_tri_dev device uint64[1] (T'); kept_edges_dev device
 *   int64[1] (edges kept).  The unbiased estimate of T is T' / q^3 (Section 9.1),
 *   computed by the caller on the host.
 */
tc_status tc_sparsify_count(tc_ctx* ctx, const tc_graph* g, double q, uint64_t seed,
                            uint64_t* kept_tri_dev, int64_t* kept_edges_dev, void* ws, size_t ws_bytes,
                            tc_stream stream);

/*
 * Sparsification with partition-local coins (Section 9.2: each processor
 * sparsifies the partition it loads, Figure "sparsification"): the triangles
 * whose apex (first vertex in the order of Eq. (1)) lies in [v_begin, v_end),
 * counted on the graph in which this part keeps each edge with probability q
 * by its own coin -- Philox4x32-10 with counter words (min(a,b), max(a,b), part, 0)
 * and the key above, keep iff r < ceil(q * 2^53).  part = 0 draws the
 * coins of tc_sparsify_count.  Run over the parts of a partition, each with its
 * own index, sum T'/q^3 is unbiased, and two triangles of different parts that
 * share an edge survive independently, so the variance is Eq. var2's (k' <= k).
 *   kept_tri_dev   device uint64[1]: ADDS this part's kept triangles
 *   kept_edges_dev device int64[1]: overwritten with the edges this part's coins keep
 * Workspace: tc_workspace_size(TC_OP_SPARSIFY, n, m).
 */
tc_status tc_sparsify_count_part(tc_ctx* ctx, const tc_graph* g, double q, uint64_t seed, int32_t part,
                                 int32_t v_begin, int32_t v_end, uint64_t* kept_tri_dev, int64_t* kept_edges_dev,
                                 void* ws, size_t ws_bytes, tc_stream stream);

/* ---- cost-balanced partition of the apex vertices (Section "load balancing") --- */

/*
 * Cost functions f(v) of Table "lbscheme" (the paper's load-balancing schemes).
 * WORK is the scheme whose f(v) = sum over u in N_v of (dhat_v + dhat_u): the
 * reads of Theorem 2 charged to apex v, the per-vertex counting work.
 */
typedef enum {
  TC_COST_VERTICES = 0,  /* f(v) = 1 */
  TC_COST_DEGREE = 1,    /* f(v) = d_v (needs g->deg) */
  TC_COST_DHAT = 2,      /* f(v) = dhat_v */
  TC_COST_DEG_DHAT = 3,  /* f(v) = d_v * dhat_v (needs g->deg) */
  TC_COST_DHAT_SQ = 4,   /* f(v) = dhat_v^2 */
  TC_COST_WORK = 5       /* f(v) = sum_{u in N_v} (dhat_v + dhat_u) */
} tc_cost;

/*
 * Split the vertices into `parts` contiguous ranges of about equal cost, as the
 * paper's partitioning step does: F(t) = f(0) + ... + f(t), alpha = F(n-1) /
 * parts, and the boundary node of part j (0 < j < parts) is the smallest v
 * with F(v) >= j * alpha (compared exactly in integers); part j is
 * [bounds[j], bounds[j+1]), bounds[0] = 0, bounds[parts] = n.  dhat is taken
 * from the offsets.
 *   parts          1 .. 65536
 *   bounds_dev     device int64[parts + 1]
 *   part_cost_dev  device uint64[parts] (sum of f over each part) or NULL
 * Workspace: tc_workspace_size(TC_OP_PARTITION, n, m).
 */
tc_status tc_partition(tc_ctx* ctx, const tc_graph* g, int32_t parts, int cost, int64_t* bounds_dev,
                       uint64_t* part_cost_dev, void* ws, size_t ws_bytes, tc_stream stream);

/*
 * The triangles whose first vertex in the order of Eq. (1) -- the apex v of
 * the counting loop of Figure 2 -- lies in [v_begin, v_end): one part of a
 * partition, as one processor of the paper counts its core vertices.  Summed
 * over the parts of any partition of [0, n) they give T and T_v exactly.
 * ADDS to its outputs (the caller clears them once, then runs the parts):
 *   total_dev device uint64[1] += the part's triangles;
 *   tv_dev    device int64[n] or NULL: += each vertex's triangles of the part.
 * Workspace: tc_workspace_size(TC_OP_COUNT, n, m).
 */
tc_status tc_count_range(tc_ctx* ctx, const tc_graph* g, int32_t v_begin, int32_t v_end, uint64_t* total_dev,
                         int64_t* tv_dev, void* ws, size_t ws_bytes, tc_stream stream);

/*
 * Counting a graph whose oriented lists stay in HOST memory, for a CSR larger
 * than the device memory the caller can spare -- the single-GPU form of the
 * paper's space-efficient algorithm (Section "A Space-efficient Parallel
 * Algorithm with Non-overlapping Partitioning", its surrogate approach): the
 * vertices are cut into target ranges whose lists N_u fit half of a device
 * list buffer; one range at a time is copied in and stays resident while the
 * apex lists N_v of every vertex stream past it, chunk by chunk, in large
 * contiguous copies on a second stream (double-buffered, overlapping the
 * counting), and each chunk counts the triangles (v, u, w) whose middle vertex
 * u lies in the resident range -- as the surrogate processor of u computes
 * N_v intersected with N_u for the N_v sent to it.  Every triangle is counted
 * once (at its apex v and its middle u, Theorem 1), so the sums are exact.
 *   n, m          graph size; offsets_host int64[n+1], cols_host int32[m]: the
 *                 oriented CSR in host memory (page-locked for the copies to
 *                 overlap; pageable memory is copied synchronously)
 *   total_dev     device uint64[1], overwritten with T
 *   tv_dev        device int64[n] or NULL: overwritten with T_v
 *   list_bytes    device bytes for lists inside the workspace: half holds the
 *                 resident range, a quarter each of two apex chunks; every
 *                 list must fit a quarter (else TC_ERR_WORKSPACE)
 *   ws            device workspace of tc_count_streamed_workspace_size(n, m,
 *                 list_bytes) bytes, 256-byte aligned: the offsets' device
 *                 copy, the counting kernels' scratch and the list buffer
 * Host traffic: the whole of cols once per target range plus once more for
 * the ranges themselves, (ranges + 1) * 4m bytes.  Returns TC_ERR_INVALID_ARG
 * during a capture.  Stream-ordered like every call; synchronous mode waits
 * and returns the device checks (TC_ERR_INVALID_GRAPH for a broken CSR).
 */
tc_status tc_count_streamed_workspace_size(int32_t n, int64_t m, size_t list_bytes, size_t* bytes);
tc_status tc_count_streamed(tc_ctx* ctx, int32_t n, int64_t m, const int64_t* offsets_host,
                            const int32_t* cols_host, uint64_t* total_dev, int64_t* tv_dev, size_t list_bytes,
                            void* ws, size_t ws_bytes, tc_stream stream);

/* ---- batched form ------------------------------------------------------------ */

/*
 * Many independent graphs in one launch sequence (no counterpart in the
 * paper, which counts one graph; the counting per graph is Figure 2's).  The
 * G graphs are laid side by side as a disjoint union: graph g owns the global
 * vertex ids [vbase[g], vbase[g+1]).  The union is oriented once (a graph's
 * orientation does not depend on the others: degrees and the order of Eq. (1)
 * are per vertex) and counted by one persistent launch whose device-side work
 * cursor and queue of long lists span all graphs.
 *   G          number of graphs (> 0); N, E: total vertices and edges (host)
 *   vbase_dev  device int64[G+1], non-decreasing, vbase[0] = 0, vbase[G] = N
 *   ebase_dev  device int64[G+1], non-decreasing, ebase[0] = 0, ebase[G] = E;
 *              graph g's edges are edges_dev[ebase[g] .. ebase[g+1])
 *   edges_dev  device int32[E][2]: LOCAL ids in [0, n_g), each undirected edge
 *              of graph g once (either direction, any order)
 * Outputs (device):
 *   offsets int64[N+1], cols int32[E], deg int32[N], dhat int32[N]: the
 *     oriented union; graph g's lists are those of its global ids, with
 *     global ids (subtract vbase[g] for local ones)
 *   totals_dev uint64[G]: T of each graph
 *   tv_dev     int64[N] or NULL: per-vertex counts (graph g's in tv[vbase[g] ..))
 * Workspace: tc_workspace_size(TC_OP_BATCH, N, E).  A local id outside
 * [0, n_g), a self-loop, a repeated edge or malformed bases give
 * TC_ERR_INVALID_GRAPH.
 */
tc_status tc_batch(tc_ctx* ctx, int32_t G, int32_t N, int64_t E, const int64_t* vbase_dev, const int64_t* ebase_dev,
                   const int32_t* edges_dev, int64_t* offsets, int32_t* cols, int32_t* deg, int32_t* dhat,
                   uint64_t* totals_dev, int64_t* tv_dev, void* ws, size_t ws_bytes, tc_stream stream);

/* ---- captured launch sequences ------------------------------------------------ */

/*
 * CUDA-graph capture of a sequence of calls (no counterpart in the paper).  A
 * sequence such as tc_batch (orientation + counting of thousands of graphs,
 * about twenty kernels) or tc_orient + tc_count is recorded once and replayed
 * with one cudaGraphLaunch, which removes the per-kernel launch cost from the
 * replays.  A replay re-runs the recorded kernels on the SAME device buffers
 * and sizes; the caller refills the inputs in place between replays.
 *
 * tc_capture_begin starts stream capture on `stream` (a created stream, not
 * the legacy default stream) and puts ctx in capture mode until
 * tc_capture_end: calls only enqueue (as in asynchronous mode) and profiling
 * events are not recorded.  Calls that must synchronize to return a result on
 * the host (tc_list, tc_analyze) return TC_ERR_INVALID_ARG while capturing.
 * Input errors found on the device during a replay accumulate in the
 * context's error word: read them with tc_ctx_status.
 * tc_capture_end ends the capture and instantiates it into *out (owned by the
 * caller, freed by tc_exec_destroy); on a failed call inside the capture it
 * returns that failure and discards the capture.
 */
typedef struct tc_exec tc_exec;

tc_status tc_capture_begin(tc_ctx* ctx, tc_stream stream);
tc_status tc_capture_end(tc_ctx* ctx, tc_stream stream, tc_exec** out);
/* Replay the captured sequence on `stream` (any stream of the same device). */
tc_status tc_exec_launch(tc_exec* x, tc_stream stream);
/* Kernels in one replay (kernel nodes of the captured graph). */
int64_t tc_exec_kernels(const tc_exec* x);
void tc_exec_destroy(tc_exec* x);

/* ---- serving ----------------------------------------------------------------- */

/*
 * A request server over resident graphs (no counterpart in the paper, whose
 * per-graph computations it serves: Figure 2's count, Section 11's per-vertex
 * counts and clustering coefficients, Section 10's listing).  It does
 * continuous batching: a worker thread admits requests as soon as one of its
 * slots (a CUDA stream each) and enough pool memory are free, so requests that
 * arrive while others run join the device at once and overlap with them.
 *
 * Memory: the caller gives the server a device pool (pool_dev, pool_bytes,
 * e.g. 150 GB of HBM); every device byte the server uses -- resident oriented
 * graphs, per-request workspaces and results -- comes from it.  Admission is
 * by footprint: a graph that does not fit is refused with TC_ERR_REJECTED; a
 * request that does not fit yet waits until running requests finish or results
 * are released, for at most the admission timeout, and one larger than all the
 * memory the pool could ever free is refused at once.
 *
 * Threading: every tc_serve_* call is thread-safe.  Results stay valid (and
 * their memory held) until tc_serve_release.
 */
typedef struct tc_server tc_server;

typedef enum {
  TC_REQ_COUNT = 0,  /* T */
  TC_REQ_LOCAL = 1,  /* T, T_v and C_v */
  TC_REQ_LIST = 2    /* T and the triangle list (v, u, w) */
} tc_request_kind;

/*
 * Slots come in two classes.  Requests on graphs of at most small_edges edges
 * are small: they run on high-priority streams and may take any free slot.
 * Large requests take only the low-priority slots; their persistent grids use
 * 1/grid_div of the GPU each, and their warp-tile blocks retire after a few
 * vertex chunks, so that the blocks of a small request arriving behind them
 * are scheduled first as SMs free up.
 */
typedef struct {
  int32_t slots;            /* requests on the GPU at once (0 = 8, at most 64) */
  int64_t admit_timeout_ms; /* how long a request may wait for memory before TC_ERR_REJECTED (0 = 10 s) */
  int32_t grid_div;         /* a large request's persistent grids use 1/grid_div of the GPU (0 = 2) */
  int32_t tile_max;         /* as tc_ctx_set_tuning (0 = default) */
  int32_t high_slots;       /* slots on high-priority streams (0 = half of the slots; < slots) */
  int64_t small_edges;      /* largest graph (edges) of a small request (0 = 2^21) */
} tc_serve_config;

typedef struct {
  tc_status status;  /* TC_OK, or why the request failed (TC_ERR_REJECTED: did not fit) */
  int32_t kind;      /* tc_request_kind */
  int64_t graph_id;
  int32_t n;         /* vertices of the graph */
  uint64_t triangles;
  const int64_t* tv; /* TC_REQ_LOCAL: device int64[n] */
  const double* cc;  /* TC_REQ_LOCAL: device double[n] */
  const int32_t* tri;/* TC_REQ_LIST: device int32[triangles][3] */
  double queue_ms;   /* submit -> admitted */
  double latency_ms; /* submit -> result ready */
} tc_result;

typedef struct {
  int64_t admitted, completed, rejected, pending, running;
  size_t pool_used, pool_capacity;
  int64_t edges_done; /* oriented edges of the graphs of completed requests */
} tc_serve_stats_t;

/* Create a server on CUDA device `device` using the caller's device pool (>= 64 KiB). */
tc_status tc_serve_create(int device, const tc_serve_config* cfg, void* pool_dev, size_t pool_bytes,
                          tc_server** out);
/* Stop the worker, wait for the slots and free the server (the pool stays the caller's). */
void tc_serve_destroy(tc_server* s);
const char* tc_serve_last_error(const tc_server* s);
/*
 * Copy an edge list (host int32[m][2], the input of tc_orient) to the device,
 * orient it (Eq. (1), Figure 2 preprocessing) and keep the CSR resident.
 * Blocks until the graph is ready; writes its id.
 */
tc_status tc_serve_add_graph(tc_server* s, int32_t n, int64_t m, const int32_t* edges_host, int64_t* graph_id);
/* Free a resident graph (TC_ERR_NOT_READY while requests on it are unfinished). */
tc_status tc_serve_remove_graph(tc_server* s, int64_t graph_id);
/* Queue a request (tc_request_kind) on a resident graph; writes its ticket. */
tc_status tc_serve_submit(tc_server* s, int64_t graph_id, int kind, int64_t* ticket);
/* Result of a finished request, or TC_ERR_NOT_READY. */
tc_status tc_serve_poll(tc_server* s, int64_t ticket, tc_result* out);
/* Wait up to timeout_ms for a request; TC_ERR_TIMEOUT if it is still unfinished. */
tc_status tc_serve_wait(tc_server* s, int64_t ticket, int64_t timeout_ms, tc_result* out);
/* Drop a finished request and the device memory of its result. */
tc_status tc_serve_release(tc_server* s, int64_t ticket);
tc_status tc_serve_stats(tc_server* s, tc_serve_stats_t* out);

/* ---- counting without allocation --------------------------------------- */

/*
 * No counterpart in the paper: an entry point for callers that cannot
 * allocate device memory -- a process whose device memory belongs to another
 * allocator (a framework's caching allocator that has reserved the device),
 * a latency-critical path where cudaMalloc/cudaFree would synchronize the
 * device, or code held to a memory budget declared up front.  tc_count needs a
 * caller workspace and tc_ctx_create allocates; this call needs neither.
 *
 * Computes the same T as tc_count, with the same kernels.  Their scratch (the
 * queue of long lists and the work cursors) is a file-scope device array of
 * TC_STATIC_MAX_N * 4 + 256 bytes (about 4 MiB) that every GPU loading the
 * library holds until the process exits.  The caller still passes inputs and
 * outputs:
 *   g          the oriented graph (device pointers, as for tc_count); n must
 *              not exceed TC_STATIC_MAX_N (else TC_ERR_UNSUPPORTED, nothing run)
 *   total_dev  device uint64[1], overwritten with T
 *   check_dev  device uint32[1], overwritten with 0, or with nonzero bits if the
 *              graph failed the kernels' checks (the TC_ERR_INVALID_GRAPH cases)
 *   stream     cudaStream_t on the current device (NULL = legacy default stream)
 * The call only enqueues work: read total_dev and check_dev after the stream
 * has finished.  It returns TC_ERR_INVALID_ARG for NULL or negative arguments
 * and for misaligned pointers (offsets and total_dev must be 8-byte aligned,
 * cols and check_dev 4-byte aligned; nothing is enqueued then), and
 * TC_ERR_CUDA if a CUDA call fails.  The first call on a device does a
 * one-time set-up (it looks up the array's device address), so make that first
 * call before any stream capture begins.  Every call on a device shares the
 * one array and leaves its contents behind (each call clears the cursors it
 * needs): calls that overlap on the GPU race on it, so order them.
 */
#define TC_STATIC_MAX_N (1 << 20)
tc_status tc_count_static(const tc_graph* g, uint64_t* total_dev, uint32_t* check_dev, tc_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
