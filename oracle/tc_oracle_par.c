/*
 * PARALLEL CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * The same definitions as the serial oracle (tc_oracle.c), restated for the
 * host's cores so that the full-size configurations (preferential attachment
 * with 2^24 and 2^27 vertices, R-MAT scale 24) can be checked against a full
 * oracle result instead of samples.  Only the tests, the package's smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does.  It shares no code with the CUDA sources.  Every function is pinned by
 * equality with its serial counterpart (tests/test_oracle_par.py), which is
 * pinned in turn by brute force, trace(A^3) and closed forms.
 *
 * Functions and the passages they follow:
 *   orp_build_adjacency - N(v) sorted (Preliminaries); same result and same
 *                         error codes as orc_build_adjacency
 *   orp_orient          - the oriented lists N_v of Definition 1 under the
 *                         order of Eq. (1) (or a caller key), sorted (Figure 2,
 *                         preprocessing)
 *   orp_count           - NodeIteratorN (Figure 2): for every v and every
 *                         u in N_v, the triangles {v, u, w} are the w in
 *                         N_v intersected with N_u, found here by a two-pointer
 *                         merge of the two sorted lists.  Each triangle is found
 *                         once, from its first vertex in the order (Theorem 1).
 *                         Per-vertex counts are summed per processor and then
 *                         over processors as in Section 11 (Figure
 *                         "localcount"): each thread owns its apexes' sums and
 *                         adds the other two vertices' shares once per (v, u)
 *                         and once per (v, w) into the shared array.
 *   orp_list            - the triples of Figure "tlisting", written per apex at
 *                         offsets the caller derives from orp_count's per-apex
 *                         counts, in the same order as they are found
 *   orp_fingerprint     - two hashes of a triple, summed over all triangles, so
 *                         that a listing too large to store on the host can be
 *                         compared as a set (see the comment there)
 *   orp_sparsify_count  - Section 9.1 / Figure "sparsification": keep each edge
 *                         by the serial oracle's coin, count the kept graph
 *                         under the order of the original degrees
 *
 * Threads: OpenMP, the default team (OMP_NUM_THREADS).  Integer sums only, so
 * every result is the same for any thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

enum {
  ORC_OK = 0,
  ORC_BAD_ID = 1,
  ORC_SELF_LOOP = 2,
  ORC_DUPLICATE = 3,
  ORC_NOMEM = 4,
  ORC_CAPACITY = 5,
};

/* the serial oracle's coin (tc_oracle.c, Section 9.1), linked into this library */
int orc_sparsify_keep(int32_t a, int32_t b, uint64_t seed, double q);

int orp_num_threads(void) { return omp_get_max_threads(); }

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void sort_list(int32_t* a, int64_t len) {
  if (len <= 24) { /* insertion sort for the many short lists */
    for (int64_t i = 1; i < len; ++i) {
      int32_t x = a[i];
      int64_t j = i - 1;
      while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
      a[j + 1] = x;
    }
  } else {
    qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

/*
 * Full adjacency N(v), each list sorted ascending; adj_off[n+1], adj[2m].
 * Rejects ids outside [0, n), self-loops (the code of the first offending
 * edge in input order, as the serial builder reports) and repeated edges.
 */
int orp_build_adjacency(int32_t n, int64_t m, const int32_t* edges, int64_t* adj_off, int32_t* adj) {
  int64_t first_bad = m;
#pragma omp parallel for schedule(static) reduction(min : first_bad)
  for (int64_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b)
      if (e < first_bad) first_bad = e;
  }
  if (first_bad < m) {
    int32_t a = edges[2 * first_bad], b = edges[2 * first_bad + 1];
    return (a < 0 || a >= n || b < 0 || b >= n) ? ORC_BAD_ID : ORC_SELF_LOOP;
  }
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v <= (int64_t)n; ++v) adj_off[v] = 0;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    __atomic_fetch_add(&adj_off[edges[2 * e] + 1], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&adj_off[edges[2 * e + 1] + 1], 1, __ATOMIC_RELAXED);
  }
  for (int32_t v = 0; v < n; ++v) adj_off[v + 1] += adj_off[v];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) return ORC_NOMEM;
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < n; ++v) fill[v] = adj_off[v];
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    adj[__atomic_fetch_add(&fill[a], 1, __ATOMIC_RELAXED)] = b;
    adj[__atomic_fetch_add(&fill[b], 1, __ATOMIC_RELAXED)] = a;
  }
  free(fill);
  int dup = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : dup)
  for (int32_t v = 0; v < n; ++v) {
    int64_t lo = adj_off[v], hi = adj_off[v + 1];
    sort_list(adj + lo, hi - lo);
    for (int64_t i = lo + 1; i < hi; ++i)
      if (adj[i] == adj[i - 1]) dup = 1;
  }
  return dup ? ORC_DUPLICATE : ORC_OK;
}

/* u precedes v: by key (ties by the smaller id); key NULL = the degrees, Eq. (1). */
static inline int precedes(const int64_t* adj_off, const int64_t* key, int32_t u, int32_t v) {
  int64_t ku = key ? key[u] : adj_off[u + 1] - adj_off[u];
  int64_t kv = key ? key[v] : adj_off[v + 1] - adj_off[v];
  return ku < kv || (ku == kv && u < v);
}

/*
 * Oriented lists N_v = {u in N(v) : v precedes u} (Definition 1), in the
 * ascending id order N(v) already has.  off[n+1], cols[m], dhat[n].
 */
void orp_orient(int32_t n, const int64_t* adj_off, const int32_t* adj, const int64_t* key,
                int64_t* off, int32_t* cols, int32_t* dhat) {
#pragma omp parallel for schedule(dynamic, 4096)
  for (int32_t v = 0; v < n; ++v) {
    int32_t c = 0;
    for (int64_t i = adj_off[v]; i < adj_off[v + 1]; ++i) c += precedes(adj_off, key, v, adj[i]);
    dhat[v] = c;
  }
  off[0] = 0;
  for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + dhat[v];
#pragma omp parallel for schedule(dynamic, 4096)
  for (int32_t v = 0; v < n; ++v) {
    int64_t pos = off[v];
    for (int64_t i = adj_off[v]; i < adj_off[v + 1]; ++i)
      if (precedes(adj_off, key, v, adj[i])) cols[pos++] = adj[i];
  }
}

/*
 * Listing fingerprint.  A listing of 10^10 triangles does not fit in host
 * memory, so it is compared as a set through sums of hashes: with
 * P = 2^31 - 1, a triple (v, u, w) written in the order v, u, w is mapped to
 *   x = ((v * A + u) mod P * A + w) mod P,
 *   y = (x * x + B) mod P,   h = (y * y + C) mod P,
 * a polynomial of degree 4 in x; two constant sets give two hashes, and the
 * fingerprint is the pair of their sums mod P over all triangles.  Two lists
 * of the same length that differ (with no repeated triple, which the tests
 * check separately) give the same pair only by a collision of both sums.
 * Every intermediate stays below 2^62, so the same arithmetic runs in signed
 * 64-bit tensor operations on the device side of a test.
 */
#define FP_P 2147483647ULL
static const uint64_t FP_A[2] = {1103515245ULL, 1664525ULL};
static const uint64_t FP_B[2] = {12345ULL, 1013904223ULL};
static const uint64_t FP_C[2] = {2147480009ULL, 305419896ULL};

static inline uint64_t fp_hash(int k, uint64_t v, uint64_t u, uint64_t w) {
  uint64_t x = ((v * FP_A[k]) % FP_P + u) % FP_P;
  x = ((x * FP_A[k]) % FP_P + w) % FP_P;
  uint64_t y = (x * x + FP_B[k]) % FP_P;
  return (y * y + FP_C[k]) % FP_P;
}

/* the fingerprint of one triple, for a test to check the constants on both sides */
void orp_fingerprint(int32_t v, int32_t u, int32_t w, uint64_t out[2]) {
  out[0] = fp_hash(0, (uint64_t)v, (uint64_t)u, (uint64_t)w);
  out[1] = fp_hash(1, (uint64_t)v, (uint64_t)u, (uint64_t)w);
}

/*
 * NodeIteratorN (Figure 2) on the oriented CSR (off[n+1], cols[m], each N_v
 * sorted ascending):
 *   for v in V, for u in N_v: S = N_v intersected with N_u (two-pointer merge);
 *   T += |S|, and each w in S closes the triangle (v, u, w).
 * Outputs (each nullable except T_out):
 *   tv[n]    - T_v: triangles containing v (Section 11);
 *   apex[n]  - triangles whose first vertex in the order is v;
 *   fp[2]    - the listing fingerprint (above) over all triangles.
 */
int orp_count(int32_t n, const int64_t* off, const int32_t* cols, uint64_t* T_out, int64_t* tv,
              int64_t* apex, uint64_t* fp) {
  int64_t max_dhat = 0;
#pragma omp parallel for schedule(static) reduction(max : max_dhat)
  for (int32_t v = 0; v < n; ++v)
    if (off[v + 1] - off[v] > max_dhat) max_dhat = off[v + 1] - off[v];
  if (tv) {
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; ++v) tv[v] = 0;
  }
  uint64_t T = 0, fp0 = 0, fp1 = 0;
  int nomem = 0;
#pragma omp parallel reduction(+ : T) reduction(| : nomem)
  {
    /* per-thread counter of each position of N_v: triangles (v, ., w) per w */
    int64_t* per_w = (int64_t*)calloc((size_t)(max_dhat > 0 ? max_dhat : 1), sizeof(int64_t));
    uint64_t s0 = 0, s1 = 0;
    if (!per_w) nomem = 1;
#pragma omp for schedule(dynamic, 256)
    for (int32_t v = 0; v < n; ++v) {
      if (!per_w) continue;
      int64_t lo = off[v], hi = off[v + 1];
      int64_t t_v = 0;
      for (int64_t i = lo; i < hi; ++i) {
        int32_t u = cols[i];
        int64_t a = lo, b = off[u], be = off[u + 1], t_e = 0;
        while (a < hi && b < be) {
          if (cols[a] < cols[b]) ++a;
          else if (cols[a] > cols[b]) ++b;
          else {
            if (fp) {
              s0 = (s0 + fp_hash(0, (uint64_t)v, (uint64_t)u, (uint64_t)cols[a])) % FP_P;
              s1 = (s1 + fp_hash(1, (uint64_t)v, (uint64_t)u, (uint64_t)cols[a])) % FP_P;
            }
            per_w[a - lo] += 1;
            ++t_e; ++a; ++b;
          }
        }
        t_v += t_e;
        if (tv && t_e) __atomic_fetch_add(&tv[u], t_e, __ATOMIC_RELAXED);
      }
      T += (uint64_t)t_v;
      if (apex) apex[v] = t_v;
      if (tv && t_v) __atomic_fetch_add(&tv[v], t_v, __ATOMIC_RELAXED);
      for (int64_t j = 0; j < hi - lo; ++j) {
        if (per_w[j] && tv) __atomic_fetch_add(&tv[cols[lo + j]], per_w[j], __ATOMIC_RELAXED);
        per_w[j] = 0;
      }
    }
#pragma omp critical
    {
      fp0 = (fp0 + s0) % FP_P;
      fp1 = (fp1 + s1) % FP_P;
    }
    free(per_w);
  }
  if (nomem) return ORC_NOMEM;
  *T_out = T;
  if (fp) { fp[0] = fp0; fp[1] = fp1; }
  return ORC_OK;
}

/*
 * The triples (v, u, w) of Figure "tlisting", those of apex v written from
 * tri[3 * apex_off[v]] on, per u in N_v order and per w ascending (the order
 * the merge finds them).  apex_off[n+1] is the exclusive prefix sum of
 * orp_count's per-apex counts.
 */
void orp_list(int32_t n, const int64_t* off, const int32_t* cols, const int64_t* apex_off, int32_t* tri) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t v = 0; v < n; ++v) {
    int64_t lo = off[v], hi = off[v + 1], pos = apex_off[v];
    for (int64_t i = lo; i < hi; ++i) {
      int32_t u = cols[i];
      int64_t a = lo, b = off[u], be = off[u + 1];
      while (a < hi && b < be) {
        if (cols[a] < cols[b]) ++a;
        else if (cols[a] > cols[b]) ++b;
        else {
          tri[3 * pos] = v;
          tri[3 * pos + 1] = u;
          tri[3 * pos + 2] = cols[a];
          ++pos; ++a; ++b;
        }
      }
    }
  }
}

/*
 * Section 9.1 / Figure "sparsification" on the host's cores: keep edge e iff
 * the serial oracle's coin keeps it, build the kept graph's adjacency, orient
 * it by `deg` (the ORIGINAL degrees, so that the order is the one fixed while
 * loading) and count it with NodeIteratorN.  Writes T' and the kept count.
 */
int orp_sparsify_count(int32_t n, int64_t m, const int32_t* edges, const int32_t* deg, uint64_t seed,
                       double q, uint64_t* T_kept, int64_t* m_kept) {
  uint8_t* keep = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
  if (!keep) return ORC_NOMEM;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) keep[e] = (uint8_t)orc_sparsify_keep(edges[2 * e], edges[2 * e + 1], seed, q);
  int64_t mk = 0;
  for (int64_t e = 0; e < m; ++e) mk += keep[e];
  int32_t* kept = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * mk > 0 ? 2 * mk : 1));
  int64_t* adj_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * mk > 0 ? 2 * mk : 1));
  int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * (size_t)(mk > 0 ? mk : 1));
  int32_t* dhat = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int rc = ORC_NOMEM;
  if (!kept || !adj_off || !adj || !key || !off || !cols || !dhat) goto done;
  {
    int64_t c = 0;
    for (int64_t e = 0; e < m; ++e)
      if (keep[e]) { kept[2 * c] = edges[2 * e]; kept[2 * c + 1] = edges[2 * e + 1]; ++c; }
  }
  rc = orp_build_adjacency(n, mk, kept, adj_off, adj);
  if (rc != ORC_OK) goto done;
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < n; ++v) key[v] = deg[v];
  orp_orient(n, adj_off, adj, key, off, cols, dhat);
  rc = orp_count(n, off, cols, T_kept, NULL, NULL, NULL);
  *m_kept = mk;
done:
  free(keep); free(kept); free(adj_off); free(adj); free(key); free(off); free(cols); free(dhat);
  return rc;
}
