/*
 * Seeded synthetic graph generators: the inputs shared by the CPU oracle and
 * the CUDA path.  This file holds no triangle-counting arithmetic; it only
 * produces undirected simple edge lists (each edge once, as (lo, hi) with
 * lo < hi) from a counter-based random stream.
 *
 * Random stream: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), keyed by (seed, generator tag) and
 * counted by (item index, draw index, 0, 0).  Every draw is a pure function of
 * its counter, so the OpenMP loops below give the same graph for any thread
 * count.
 *
 * Workload shapes (the paper's dataset classes, Section "Preliminaries",
 * Datasets paragraph): Gnp / G(n, M) Erdos-Renyi, preferential attachment
 * PA(n, d), plus R-MAT and Chung-Lu as stand-ins for skewed real graphs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

enum { TAG_ER = 0x4552, TAG_BA = 0x4241, TAG_RMAT = 0x524d, TAG_CL = 0x434c, TAG_BATCH = 0x4254 };

/* ---- Philox4x64-10 ------------------------------------------------------ */
static inline void gen_philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                              uint64_t k0, uint64_t k1, uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  for (int r = 0; r < 10; ++r) {
    u128 p0 = (u128)M0 * c0, p1 = (u128)M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform integer in [0, n) from a 64-bit word (multiply-high). */
static inline uint64_t below(uint64_t r, uint64_t n) { return (uint64_t)(((u128)r * n) >> 64); }
/* uniform double in [0, 1) with 53 random bits. */
static inline double unit53(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

/* ---- parallel LSD radix sort of uint64 keys ------------------------------ */
/* threads: 0 = OpenMP default */
static void sort_u64(uint64_t* a, uint64_t* tmp, int64_t cnt, int bits, int threads) {
  if (cnt <= 1) return;
  int nt = 1;
#ifdef _OPENMP
  nt = threads > 0 ? threads : omp_get_max_threads();
  if (cnt < 65536) nt = 1;
#endif
  int64_t* hist = (int64_t*)calloc((size_t)nt * 256, sizeof(int64_t));
  uint64_t *src = a, *dst = tmp;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int sh = 8 * p;
    memset(hist, 0, (size_t)nt * 256 * sizeof(int64_t));
#pragma omp parallel num_threads(nt)
    {
      int t = 0;
#ifdef _OPENMP
      t = omp_get_thread_num();
#endif
      int64_t lo = cnt * t / nt, hi = cnt * (t + 1) / nt;
      int64_t* h = hist + (size_t)t * 256;
      for (int64_t i = lo; i < hi; ++i) h[(src[i] >> sh) & 255]++;
#pragma omp barrier
#pragma omp single
      {
        int64_t run = 0;
        for (int d = 0; d < 256; ++d)
          for (int tt = 0; tt < nt; ++tt) {
            int64_t c = hist[(size_t)tt * 256 + d];
            hist[(size_t)tt * 256 + d] = run;
            run += c;
          }
      }
      for (int64_t i = lo; i < hi; ++i) dst[h[(src[i] >> sh) & 255]++] = src[i];
    }
    uint64_t* s = src; src = dst; dst = s;
  }
  if (src != a) memcpy(a, src, (size_t)cnt * sizeof(uint64_t));
  free(hist);
}

static int bits_for(int64_t n) {
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) < n) ++b;
  return b;
}

/* keys = (lo << 32) | hi; sort, unique, write int32 pairs. Returns edge count. */
static int64_t keys_to_edges(uint64_t* keys, int64_t cnt, int32_t n, int32_t* out, int64_t cap, int threads) {
  uint64_t* tmp = (uint64_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(uint64_t));
  if (!tmp) return -2;
  int b = bits_for(n);
  /* the low word holds hi (< n), the high word lo (< n): sort on both */
  for (int64_t i = 0; i < cnt; ++i) keys[i] = ((keys[i] >> 32) << b) | (keys[i] & 0xffffffffULL);
  sort_u64(keys, tmp, cnt, 2 * b, threads);
  free(tmp);
  int64_t m = 0;
  uint64_t mask = ((uint64_t)1 << b) - 1;
  for (int64_t i = 0; i < cnt; ++i) {
    if (i > 0 && keys[i] == keys[i - 1]) continue;
    if (m >= cap) return -1;
    out[2 * m] = (int32_t)(keys[i] >> b);
    out[2 * m + 1] = (int32_t)(keys[i] & mask);
    ++m;
  }
  return m;
}

/*
 * Erdos-Renyi G(n, M) by sampling: `draws` endpoint pairs, each endpoint
 * uniform in [0, n); self-loops dropped, duplicates merged.  Returns m, or -1
 * if `cap` (edges) is too small.
 */
int64_t gen_er(int32_t n, int64_t draws, uint64_t seed, int32_t* out, int64_t cap) {
  uint64_t* keys = (uint64_t*)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(uint64_t));
  if (!keys) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < draws; ++i) {
    uint64_t r[4];
    gen_philox((uint64_t)i, 0, 0, 0, seed, TAG_ER, r);
    uint64_t a = below(r[0], (uint64_t)n), b = below(r[1], (uint64_t)n);
    if (a == b) { keys[i] = ~0ULL; continue; }
    uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    keys[i] = (lo << 32) | hi;
  }
  int64_t c = 0;
  for (int64_t i = 0; i < draws; ++i)
    if (keys[i] != ~0ULL) keys[c++] = keys[i];
  int64_t m = keys_to_edges(keys, c, n, out, cap, 0);
  free(keys);
  return m;
}

/*
 * Preferential attachment PA(n, k) in the Batagelj-Brandes endpoint-copy
 * form.  Vertices 0..k-1 form a clique K_k.  Each later vertex v adds k
 * edges; the target of each is the vertex at a uniformly drawn position of
 * the endpoint sequence of all edges added before v (so a vertex is chosen
 * with probability proportional to its degree).  A position on the target
 * side of an earlier edge is resolved by following that edge's own draw,
 * which makes every target a pure function of the counter and lets the loop
 * run in parallel.  Repeated targets of one vertex are merged, so m is a
 * little under k(n-k) + k(k-1)/2.  Edges are written (target, v), target < v.
 */
int64_t gen_ba(int32_t n, int32_t k, uint64_t seed, int32_t* out, int64_t cap) {
  if (k < 2) return -3; /* k = 1 leaves vertex 1 no earlier endpoint to copy */
  if (n < 1) return 0;
  int32_t kc = n < k ? n : k;
  int64_t nclique = (int64_t)kc * (kc - 1) / 2;
  int32_t* cs = (int32_t*)malloc((size_t)(nclique > 0 ? nclique : 1) * sizeof(int32_t));
  int32_t* cd = (int32_t*)malloc((size_t)(nclique > 0 ? nclique : 1) * sizeof(int32_t));
  int64_t e = 0;
  for (int32_t i = 0; i < kc; ++i)
    for (int32_t j = i + 1; j < kc; ++j) { cs[e] = i; cd[e] = j; ++e; }
  int64_t m = 0;
  for (int64_t i = 0; i < nclique; ++i) {
    if (m >= cap) { free(cs); free(cd); return -1; }
    out[2 * m] = cs[i]; out[2 * m + 1] = cd[i]; ++m;
  }
  if (n <= k) { free(cs); free(cd); return m; }
  int64_t nv = (int64_t)n - k;
  int32_t* tgt = (int32_t*)malloc((size_t)nv * k * sizeof(int32_t));
  int32_t* cnt = (int32_t*)malloc((size_t)nv * sizeof(int32_t));
  if (!tgt || !cnt) { free(cs); free(cd); free(tgt); free(cnt); return -2; }
#pragma omp parallel for schedule(static)
  for (int64_t vi = 0; vi < nv; ++vi) {
    int64_t first = nclique + vi * k; /* index of v's first edge */
    int32_t kept = 0;
    for (int32_t j = 0; j < k; ++j) {
      /* draw for edge (first + j): a position in [0, 2*first) */
      uint64_t r4[4];
      gen_philox((uint64_t)(first + j), 0, 0, 0, seed, TAG_BA, r4);
      uint64_t pos = below(r4[0], (uint64_t)(2 * first));
      int32_t t;
      for (;;) {
        int64_t ed = (int64_t)(pos >> 1);
        if (ed < nclique) { t = (pos & 1) ? cd[ed] : cs[ed]; break; }
        int64_t owner = k + (ed - nclique) / k; /* vertex that added edge ed */
        if ((pos & 1) == 0) { t = (int32_t)owner; break; }
        int64_t ofirst = nclique + (owner - k) * k;
        gen_philox((uint64_t)ed, 0, 0, 0, seed, TAG_BA, r4);
        pos = below(r4[0], (uint64_t)(2 * ofirst));
      }
      int dup = 0;
      for (int32_t q = 0; q < kept; ++q)
        if (tgt[vi * k + q] == t) { dup = 1; break; }
      if (!dup) tgt[vi * k + kept++] = t;
    }
    cnt[vi] = kept;
  }
  int64_t total = m;
  for (int64_t vi = 0; vi < nv; ++vi) total += cnt[vi];
  if (total > cap) { free(cs); free(cd); free(tgt); free(cnt); return -1; }
  /* prefix over per-vertex kept counts, then parallel write */
  int64_t* base = (int64_t*)malloc((size_t)nv * sizeof(int64_t));
  int64_t run = m;
  for (int64_t vi = 0; vi < nv; ++vi) { base[vi] = run; run += cnt[vi]; }
#pragma omp parallel for schedule(static)
  for (int64_t vi = 0; vi < nv; ++vi)
    for (int32_t q = 0; q < cnt[vi]; ++q) {
      out[2 * (base[vi] + q)] = tgt[vi * k + q];
      out[2 * (base[vi] + q) + 1] = (int32_t)(k + vi);
    }
  free(base); free(cs); free(cd); free(tgt); free(cnt);
  return total;
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004): ef * 2^scale samples, each
 * descending `scale` levels of the adjacency matrix; at each level one 32-bit
 * draw picks quadrant a, b, c or d by integer thresholds floor(p * 2^32).  No
 * noise and no vertex permutation.  Self-loops dropped, pairs symmetrised to
 * (lo, hi) and merged.
 */
int64_t gen_rmat(int32_t scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                 int32_t* out, int64_t cap) {
  int64_t samples = edge_factor << scale;
  int32_t n = (int32_t)1 << scale;
  uint64_t ta = (uint64_t)floor(a * 4294967296.0);
  uint64_t tab = (uint64_t)floor((a + b) * 4294967296.0);
  uint64_t tabc = (uint64_t)floor((a + b + c) * 4294967296.0);
  uint64_t* keys = (uint64_t*)malloc((size_t)(samples > 0 ? samples : 1) * sizeof(uint64_t));
  if (!keys) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < samples; ++i) {
    uint64_t row = 0, col = 0, r4[4];
    for (int32_t lev = 0; lev < scale; ++lev) {
      if ((lev & 7) == 0) gen_philox((uint64_t)i, (uint64_t)(lev >> 3), 0, 0, seed, TAG_RMAT, r4);
      int w = lev & 7;
      uint64_t x = (r4[w >> 1] >> ((w & 1) * 32)) & 0xffffffffULL;
      uint64_t rb = 0, cb = 0;
      if (x < ta) { rb = 0; cb = 0; }
      else if (x < tab) { rb = 0; cb = 1; }
      else if (x < tabc) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      row = (row << 1) | rb;
      col = (col << 1) | cb;
    }
    if (row == col) { keys[i] = ~0ULL; continue; }
    uint64_t lo = row < col ? row : col, hi = row < col ? col : row;
    keys[i] = (lo << 32) | hi;
  }
  int64_t cnt = 0;
  for (int64_t i = 0; i < samples; ++i)
    if (keys[i] != ~0ULL) keys[cnt++] = keys[i];
  int64_t m = keys_to_edges(keys, cnt, n, out, cap, 0);
  free(keys);
  return m;
}

/*
 * Chung-Lu power-law graph: weight w_i = (i+1)^(-1/(gamma-1)); floor(n*dbar/2)
 * endpoint pairs, each endpoint drawn with probability proportional to w by
 * inverse CDF; self-loops dropped, duplicates merged.  `stream` separates
 * independent graphs drawn with the same seed.
 */
int64_t gen_chung_lu(int32_t n, double dbar, double gamma, uint64_t seed, uint64_t stream,
                     int32_t* out, int64_t cap, int threads) {
  if (n < 2) return 0;
  int64_t pairs = (int64_t)floor((double)n * dbar / 2.0);
  double* cum = (double*)malloc((size_t)n * sizeof(double));
  int32_t* guide = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  double run = 0.0, ex = -1.0 / (gamma - 1.0);
  for (int32_t i = 0; i < n; ++i) { run += pow((double)(i + 1), ex); cum[i] = run; }
  /* guide table (indexed search): guide[k] = first i with cum[i] > k * run / n */
  for (int32_t k = 0, i = 0; k < n; ++k) {
    double t = (double)k * run / (double)n;
    while (i < n - 1 && cum[i] <= t) ++i;
    guide[k] = i;
  }
  uint64_t* keys = (uint64_t*)malloc((size_t)(pairs > 0 ? pairs : 1) * sizeof(uint64_t));
  if (!keys) { free(cum); free(guide); return -2; }
  int nt = threads > 0 ? threads : 1;
#ifdef _OPENMP
  if (threads <= 0) nt = omp_get_max_threads();
#endif
#pragma omp parallel for schedule(static) num_threads(nt) if (pairs > 65536 && nt > 1)
  for (int64_t i = 0; i < pairs; ++i) {
    uint64_t r4[4];
    gen_philox((uint64_t)i, stream, 0, 0, seed, TAG_CL, r4);
    int32_t ends[2];
    for (int s = 0; s < 2; ++s) {
      double u = unit53(r4[s]);
      double x = u * run;
      int64_t k = (int64_t)(u * (double)n);
      if (k >= n) k = n - 1;
      int32_t j = guide[k]; /* first index with cum > x, walking forward from the guide */
      while (j < n - 1 && cum[j] <= x) ++j;
      ends[s] = j;
    }
    if (ends[0] == ends[1]) { keys[i] = ~0ULL; continue; }
    uint64_t lo = (uint64_t)(ends[0] < ends[1] ? ends[0] : ends[1]);
    uint64_t hi = (uint64_t)(ends[0] < ends[1] ? ends[1] : ends[0]);
    keys[i] = (lo << 32) | hi;
  }
  int64_t cnt = 0;
  for (int64_t i = 0; i < pairs; ++i)
    if (keys[i] != ~0ULL) keys[cnt++] = keys[i];
  int64_t m = keys_to_edges(keys, cnt, n, out, cap, threads);
  free(keys); free(cum); free(guide);
  return m;
}

/*
 * Parameters of the batched workload: graph g gets n_g = round(exp(U(ln nlo,
 * ln nhi))) vertices and a target mean degree dbar_g ~ U[dlo, dhi].
 */
void gen_batch_params(int32_t num_graphs, uint64_t seed, double nlo, double nhi, double dlo,
                      double dhi, int32_t* n_out, double* dbar_out) {
  for (int32_t g = 0; g < num_graphs; ++g) {
    uint64_t r4[4];
    gen_philox((uint64_t)g, 0, 0, 0, seed, TAG_BATCH, r4);
    double u0 = unit53(r4[0]), u1 = unit53(r4[1]);
    double ln = log(nlo) + u0 * (log(nhi) - log(nlo));
    n_out[g] = (int32_t)llround(exp(ln));
    dbar_out[g] = dlo + u1 * (dhi - dlo);
  }
}

/* Upper bounds on edge counts, for sizing output buffers. */
int64_t gen_ba_max_edges(int32_t n, int32_t k) {
  int32_t kc = n < k ? n : k;
  int64_t m = (int64_t)kc * (kc - 1) / 2;
  if (n > k) m += (int64_t)(n - k) * k;
  return m;
}

int gen_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
