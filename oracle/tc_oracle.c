/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, serial, obviously-correct restatement of what Arifuzzaman, Khan and
 * Marathe, "Distributed-Memory Parallel Algorithms for Counting and Listing
 * Triangles in Big Graphs", compute.  It is what the CUDA library is checked
 * against.  Only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no
 * code, header, table or helper with the CUDA sources.
 *
 * Notation follows the paper's Section "Preliminaries": G(V, E) undirected,
 * n vertices labelled 0..n-1, m edges, neighbour set N(v) (calligraphic N_v),
 * degree d_v = |N(v)|, T_v = triangles containing v, C_v the local clustering
 * coefficient.
 *
 * Functions and the passages they follow:
 *   orc_build_adjacency  - N(v) sorted (Preliminaries; Section 3 assumes the
 *                          lists sorted for binary search)
 *   orc_node_iterator_pp - Algorithm NodeIterator++ (Figure 1) with the degree
 *                          order of Eq. (1); also per-vertex counts (Figure
 *                          "localcount", Section 11) and listing (Figure
 *                          "tlisting", Section 10)
 *   orc_orient           - the oriented lists N_v of Definition 1 (effective
 *                          degree), i.e. the preprocessing of NodeIteratorN
 *                          (Figure 2): u in N_v iff v precedes u, sorted
 *   orc_cost             - sum_v d_v * dhat_v, the bound of Theorem 2
 *   orc_clustering       - C_v = 2 T_v / (d_v (d_v - 1)) (Preliminaries, Sec. 11)
 *   orc_sparsify_keep /
 *   orc_sparsify_count   - edge sparsification of Section 9.1 / Figure
 *                          "sparsification": keep each edge with probability q,
 *                          count the kept graph, estimate = T' / q^3
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   - the order's degree is the undirected degree of the simple graph;
 *   - ties of the order are broken by the smaller id first;
 *   - C_v = 0 when d_v < 2;
 *   - sparsification's coin for the undirected edge {a, b} is Philox4x32-10
 *     (Salmon et al., SC'11) with 32-bit counter words (min(a,b), max(a,b),
 *     0, 0) and key (low, high 32 bits of the seed); with x0, x1 the first two
 *     output words, r = x0 * 2^21 + (x1 >> 11) is the top 53 bits of the
 *     64-bit word x0:x1, and the edge is kept iff r * 2^-53 < q;
 *   - the sparsified graph keeps the order of the ORIGINAL degrees (Figure
 *     "sparsification" compares with the order fixed while loading).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  ORC_OK = 0,
  ORC_BAD_ID = 1,
  ORC_SELF_LOOP = 2,
  ORC_DUPLICATE = 3,
  ORC_NOMEM = 4,
  ORC_CAPACITY = 5,
};

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Full adjacency N(v), each list sorted ascending.  adj_off has n+1 entries,
 * adj has 2m.  Rejects ids outside [0, n), self-loops and repeated edges: the
 * paper's G is a simple undirected graph (Preliminaries).
 */
int orc_build_adjacency(int32_t n, int64_t m, const int32_t* edges, int64_t* adj_off, int32_t* adj) {
  for (int32_t v = 0; v <= n; ++v) adj_off[v] = 0;
  for (int64_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || a >= n || b < 0 || b >= n) return ORC_BAD_ID;
    if (a == b) return ORC_SELF_LOOP;
    adj_off[a + 1]++;
    adj_off[b + 1]++;
  }
  for (int32_t v = 0; v < n; ++v) adj_off[v + 1] += adj_off[v];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) return ORC_NOMEM;
  for (int32_t v = 0; v < n; ++v) fill[v] = adj_off[v];
  for (int64_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    adj[fill[a]++] = b;
    adj[fill[b]++] = a;
  }
  free(fill);
  for (int32_t v = 0; v < n; ++v) {
    int64_t lo = adj_off[v], hi = adj_off[v + 1];
    qsort(adj + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_i32);
    for (int64_t i = lo + 1; i < hi; ++i)
      if (adj[i] == adj[i - 1]) return ORC_DUPLICATE;
  }
  return ORC_OK;
}

/* d_v = |N(v)| (Preliminaries). */
void orc_degrees(int32_t n, const int64_t* adj_off, int32_t* deg) {
  for (int32_t v = 0; v < n; ++v) deg[v] = (int32_t)(adj_off[v + 1] - adj_off[v]);
}

/*
 * The total order.  Eq. (1): u precedes v iff d_u < d_v, or d_u = d_v and
 * u < v.  `key` plays the role of d; passing other keys gives the other total
 * orders of Section 4 (id order: all keys equal; random order: random keys),
 * under which Theorem 1 still counts each triangle once.
 */
static int precedes(const int64_t* key, int32_t u, int32_t v) {
  return key[u] < key[v] || (key[u] == key[v] && u < v);
}

/* is w in the sorted list N(u)?  (Section 3: binary search on sorted lists) */
static int adjacent(const int64_t* adj_off, const int32_t* adj, int32_t u, int32_t w) {
  int64_t lo = adj_off[u], hi = adj_off[u + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (adj[mid] < w) lo = mid + 1;
    else if (adj[mid] > w) hi = mid;
    else return 1;
  }
  return 0;
}

/*
 * Algorithm NodeIterator++ (Figure 1):
 *   T = 0
 *   for v in V:
 *     for u in N(v) with v < u (in the order):
 *       for w in N(v) with u < w:
 *         if (u, w) in E: T = T + 1
 * The triangle found is {v, u, w} with v < u < w in the order; it is counted
 * exactly once (Theorem 1).
 *
 * order_key: per-vertex key of the order (NULL = the degrees d_v, Eq. (1)).
 * tv (nullable, n entries): per-vertex counts, each found triangle adds one to
 *   each of its three vertices (Figure "localcount").
 * tri (nullable, 3*tri_cap entries): each found triangle is written as the
 *   triple (v, u, w) (Figure "tlisting"); *tri_count receives the number found
 *   and ORC_CAPACITY is returned if it exceeds tri_cap.
 */
int orc_node_iterator_pp(int32_t n, const int64_t* adj_off, const int32_t* adj,
                         const int64_t* order_key, uint64_t* T_out, int64_t* tv,
                         int32_t* tri, int64_t tri_cap, int64_t* tri_count) {
  int64_t* key = NULL;
  if (!order_key) {
    key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!key) return ORC_NOMEM;
    for (int32_t v = 0; v < n; ++v) key[v] = adj_off[v + 1] - adj_off[v];
    order_key = key;
  }
  if (tv)
    for (int32_t v = 0; v < n; ++v) tv[v] = 0;
  uint64_t T = 0;
  for (int32_t v = 0; v < n; ++v) {
    for (int64_t i = adj_off[v]; i < adj_off[v + 1]; ++i) {
      int32_t u = adj[i];
      if (!precedes(order_key, v, u)) continue;
      for (int64_t j = adj_off[v]; j < adj_off[v + 1]; ++j) {
        int32_t w = adj[j];
        if (!precedes(order_key, u, w)) continue;
        if (!adjacent(adj_off, adj, u, w)) continue;
        if (tri && (int64_t)T < tri_cap) {
          tri[3 * T] = v;
          tri[3 * T + 1] = u;
          tri[3 * T + 2] = w;
        }
        T += 1;
        if (tv) {
          tv[v] += 1;
          tv[u] += 1;
          tv[w] += 1;
        }
      }
    }
  }
  free(key);
  *T_out = T;
  if (tri_count) *tri_count = (int64_t)T;
  if (tri && (int64_t)T > tri_cap) return ORC_CAPACITY;
  return ORC_OK;
}

/*
 * Oriented lists N_v = {u in N(v) : v precedes u} (Definition 1), sorted
 * ascending by id (Figure 2, preprocessing).  Because N(v) is already sorted,
 * keeping the qualifying entries in order keeps N_v sorted.  Writes
 * off[n+1], cols[m] and dhat[n] = |N_v| (the effective degree).
 */
void orc_orient(int32_t n, const int64_t* adj_off, const int32_t* adj, const int64_t* order_key,
                int64_t* off, int32_t* cols, int32_t* dhat) {
  int64_t pos = 0;
  for (int32_t v = 0; v < n; ++v) {
    off[v] = pos;
    for (int64_t i = adj_off[v]; i < adj_off[v + 1]; ++i) {
      int32_t u = adj[i];
      int64_t dv = adj_off[v + 1] - adj_off[v], du = adj_off[u + 1] - adj_off[u];
      int keep;
      if (order_key) keep = precedes(order_key, v, u);
      else keep = dv < du || (dv == du && v < u);
      if (keep) cols[pos++] = u;
    }
    dhat[v] = (int32_t)(pos - off[v]);
  }
  off[n] = pos;
}

/* Theorem 2's cost sum_v d_v * dhat_v for the order given by order_key (NULL = Eq. (1)). */
uint64_t orc_cost(int32_t n, const int64_t* adj_off, const int32_t* adj, const int64_t* order_key) {
  uint64_t W = 0;
  for (int32_t v = 0; v < n; ++v) {
    int64_t dv = adj_off[v + 1] - adj_off[v], dhat = 0;
    for (int64_t i = adj_off[v]; i < adj_off[v + 1]; ++i) {
      int32_t u = adj[i];
      int64_t du = adj_off[u + 1] - adj_off[u];
      int keep = order_key ? precedes(order_key, v, u) : (dv < du || (dv == du && v < u));
      dhat += keep;
    }
    W += (uint64_t)(dv * dhat);
  }
  return W;
}

/*
 * C_v = T_v / binom(d_v, 2) = 2 T_v / (d_v (d_v - 1)) (Preliminaries and
 * Section 11), one IEEE double division of two exactly representable values;
 * 0 when d_v < 2 (the ratio is undefined there).
 */
void orc_clustering(int32_t n, const int32_t* deg, const int64_t* tv, double* cc) {
  for (int32_t v = 0; v < n; ++v) {
    int64_t d = deg[v];
    if (d < 2) cc[v] = 0.0;
    else cc[v] = (2.0 * (double)tv[v]) / (double)(d * (d - 1));
  }
}

/*
 * T_v by its definition (Preliminaries): the number of edges among the
 * neighbours of v, i.e. pairs u < w of N(v) with (u, w) in E.  Used on
 * sampled vertices of graphs too large for a full oracle run.
 */
int64_t orc_vertex_triangles(const int64_t* adj_off, const int32_t* adj, int32_t v) {
  int64_t t = 0;
  for (int64_t i = adj_off[v]; i < adj_off[v + 1]; ++i)
    for (int64_t j = i + 1; j < adj_off[v + 1]; ++j)
      t += adjacent(adj_off, adj, adj[i], adj[j]);
  return t;
}

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------
 * Ten rounds; each multiplies words 0 and 2 by the round multipliers into
 * 64-bit products, xors the high halves with words 1 and 3 and the round key,
 * permutes the words, and bumps the key by the Weyl constants. */
static void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p = (uint64_t)mul0 * x0;
    uint64_t r = (uint64_t)mul1 * x2;
    uint32_t y0 = (uint32_t)(r >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)r;
    uint32_t y2 = (uint32_t)(p >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += weyl0;
    k1 += weyl1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Exposed so a test can compare it against the published known answers. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  orc_philox4x32_10(ctr, key, out);
}

int orc_sparsify_keep_part(int32_t a, int32_t b, uint64_t seed, double q, uint32_t part);

/*
 * The sparsification coin of Section 9.1: edge {a, b} is retained with
 * probability q, independently of the others, and the coin depends only on
 * the edge (not on any storage order).
 */
int orc_sparsify_keep(int32_t a, int32_t b, uint64_t seed, double q) {
  return orc_sparsify_keep_part(a, b, seed, q, 0);
}

/*
 * The coin of edge {a, b} drawn by processor `part` when it sparsifies the
 * partition it loads (Section 9.2): the same generator with the part's index
 * as the third counter word; part 0 is the coin above.
 */
int orc_sparsify_keep_part(int32_t a, int32_t b, uint64_t seed, double q, uint32_t part) {
  uint32_t ctr[4] = {(uint32_t)(a < b ? a : b), (uint32_t)(a < b ? b : a), part, 0};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  uint64_t r = ((uint64_t)out[0] << 21) | (out[1] >> 11); /* top 53 bits of x0:x1 */
  double u = (double)r * 0x1.0p-53;
  return u < q;
}

/*
 * Figure "sparsification": keep each edge with probability q, count the
 * triangles T' of the kept graph G' with the order fixed by the ORIGINAL
 * degrees, and estimate T = T' / q^3 (Section 9.1; the estimator is unbiased
 * because a triangle survives with probability q^3).  Writes T', the number of
 * kept edges and the estimate.
 */
int orc_sparsify_count(int32_t n, int64_t m, const int32_t* edges, uint64_t seed, double q,
                       uint64_t* T_kept, int64_t* m_kept, double* estimate) {
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m > 0 ? 2 * m : 1));
  int32_t* kept = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m > 0 ? 2 * m : 1));
  int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int rc = ORC_NOMEM;
  if (!off || !adj || !kept || !key) goto done;
  rc = orc_build_adjacency(n, m, edges, off, adj);
  if (rc != ORC_OK) goto done;
  for (int32_t v = 0; v < n; ++v) key[v] = off[v + 1] - off[v]; /* original d_v */
  int64_t mk = 0;
  for (int64_t e = 0; e < m; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if (orc_sparsify_keep(a, b, seed, q)) {
      kept[2 * mk] = a;
      kept[2 * mk + 1] = b;
      ++mk;
    }
  }
  rc = orc_build_adjacency(n, mk, kept, off, adj);
  if (rc != ORC_OK) goto done;
  rc = orc_node_iterator_pp(n, off, adj, key, T_kept, NULL, NULL, 0, NULL);
  *m_kept = mk;
  *estimate = (double)(*T_kept) / (q * q * q);
done:
  free(off); free(adj); free(kept); free(key);
  return rc;
}
