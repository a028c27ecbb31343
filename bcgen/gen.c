/*
 * bcgen: seeded synthetic graph inputs for betweenness-centrality runs.
 *
 * This module only PRODUCES inputs (edge lists, canonical CSR, source lists).
 * It contains none of the centrality arithmetic, so both the CPU oracle and
 * the CUDA library can be fed from it without sharing any method code.
 *
 * Random numbers come from two published generators, written from their
 * definitions:
 *   - splitmix64 (Steele, Lea & Flood, OOPSLA 2014): used for seeding and
 *     for single hashed draws;
 *   - xoshiro256** (Blackman & Vigna, 2018): the bulk stream.
 *
 * Graph models:
 *   - R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004): every edge picks one
 *     of the four adjacency-matrix quadrants per bit with probabilities
 *     (a, b, c, d), no noise; a seeded vertex relabelling spreads the hubs
 *     (Graph500 practice).
 *   - Directed preferential attachment (Barabasi-Albert growth): a complete
 *     digraph on m0 seed vertices, then every new vertex u draws `mout`
 *     distinct existing targets with probability proportional to their total
 *     degree and adds u -> target.  This is the paper's input family
 *     (Section II.C) with every edge oriented new -> old.
 *
 * Canonical CSR: rows sorted ascending, duplicate edges and self-loops
 * removed, int32 row_ptr[n+1] / col_idx[m].
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- generators ------------------------------------------------------- */

static inline uint64_t sm64_next(uint64_t *state) {
  uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* splitmix64 applied once to x: the value a fresh splitmix64 stream with
 * state x returns first.  Used for per-graph / per-block seeds. */
uint64_t bcg_splitmix64(uint64_t x) {
  uint64_t s = x;
  return sm64_next(&s);
}

typedef struct { uint64_t s[4]; } xo256;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void xo_seed(xo256 *g, uint64_t seed) {
  uint64_t st = seed;
  for (int i = 0; i < 4; ++i) g->s[i] = sm64_next(&st);
}

static inline uint64_t xo_next(xo256 *g) {
  uint64_t *s = g->s;
  const uint64_t result = rotl64(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return result;
}

/* uniform double in [0, 1) from the top 53 bits */
static inline double xo_unif(xo256 *g) { return (double)(xo_next(g) >> 11) * 0x1.0p-53; }

/* integer in [0, range) by the multiply-high method (bias < range / 2^64) */
static inline uint64_t bounded(uint64_t r, uint64_t range) {
  return (uint64_t)(((unsigned __int128)r * range) >> 64);
}

/* ---- R-MAT ------------------------------------------------------------ */

#define RMAT_BLOCK 65536

/* Seeded Fisher-Yates permutation of [0, n). */
void bcg_permutation(int32_t n, uint64_t seed, int32_t *perm) {
  uint64_t st = seed ^ 0x7065726d75746521ULL;
  for (int32_t i = 0; i < n; ++i) perm[i] = i;
  for (int32_t i = n - 1; i > 0; --i) {
    int32_t j = (int32_t)bounded(sm64_next(&st), (uint64_t)i + 1);
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}

/* Writes nedges raw R-MAT edges (self-loops and duplicates included).
 * Edges are produced in independent blocks of RMAT_BLOCK, block b seeded by
 * splitmix64(seed ^ (b * golden)), so the output does not depend on the
 * number of threads.  permute != 0 relabels vertices with a seeded
 * permutation.  Returns nedges, or -1 on bad arguments. */
int64_t bcg_rmat_edges(int32_t scale, int64_t nedges, double a, double b, double c,
                       uint64_t seed, int32_t permute, int32_t *src, int32_t *dst) {
  if (scale < 1 || scale > 30 || nedges < 0) return -1;
  const double ab = a + b, abc = a + b + c;
  const int64_t nblocks = (nedges + RMAT_BLOCK - 1) / RMAT_BLOCK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t blk = 0; blk < nblocks; ++blk) {
    xo256 g;
    xo_seed(&g, bcg_splitmix64(seed ^ ((uint64_t)blk * 0x9e3779b97f4a7c15ULL)));
    int64_t e0 = blk * RMAT_BLOCK, e1 = e0 + RMAT_BLOCK;
    if (e1 > nedges) e1 = nedges;
    for (int64_t e = e0; e < e1; ++e) {
      uint32_t u = 0, v = 0;
      for (int32_t bit = 0; bit < scale; ++bit) {
        double r = xo_unif(&g);
        uint32_t bu, bv;
        if (r < a) { bu = 0; bv = 0; }
        else if (r < ab) { bu = 0; bv = 1; }
        else if (r < abc) { bu = 1; bv = 0; }
        else { bu = 1; bv = 1; }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
      }
      src[e] = (int32_t)u;
      dst[e] = (int32_t)v;
    }
  }
  if (permute) {
    int32_t n = (int32_t)1 << scale;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!perm) return -1;
    bcg_permutation(n, seed, perm);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
      src[e] = perm[src[e]];
      dst[e] = perm[dst[e]];
    }
    free(perm);
  }
  return nedges;
}

/* ---- directed preferential attachment ---------------------------------- */

/* Returns the number of edges written (m0*(m0-1) + mout*(n-m0)), or -1.
 * Edge list capacity must be at least that. */
int64_t bcg_ba_edges(int32_t n, int32_t m0, int32_t mout, uint64_t seed, int32_t *src,
                     int32_t *dst) {
  if (m0 < 2 || mout < 1 || mout > m0 || n < m0) return -1;
  const int64_t total = (int64_t)m0 * (m0 - 1) + (int64_t)mout * (n - m0);
  /* every edge contributes both endpoints to the urn */
  int32_t *urn = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * total));
  int32_t *picked = (int32_t *)malloc(sizeof(int32_t) * (size_t)mout);
  if (!urn || !picked) { free(urn); free(picked); return -1; }
  int64_t ne = 0, nu = 0;
  for (int32_t u = 0; u < m0; ++u)
    for (int32_t v = 0; v < m0; ++v)
      if (u != v) {
        src[ne] = u; dst[ne] = v; ++ne;
        urn[nu++] = u; urn[nu++] = v;
      }
  xo256 g;
  xo_seed(&g, seed);
  for (int32_t u = m0; u < n; ++u) {
    int32_t got = 0;
    while (got < mout) {
      int32_t t = urn[bounded(xo_next(&g), (uint64_t)nu)];
      int dup = 0;
      for (int32_t i = 0; i < got; ++i) dup |= (picked[i] == t);
      if (!dup) picked[got++] = t;
    }
    for (int32_t i = 0; i < mout; ++i) {
      src[ne] = u; dst[ne] = picked[i]; ++ne;
      urn[nu++] = u; urn[nu++] = picked[i];
    }
  }
  free(urn);
  free(picked);
  return ne;
}

/* ---- canonical CSR ----------------------------------------------------- */

static int cmp_i32(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

/* Builds canonical CSR from an edge list: self-loops dropped, each row
 * sorted and de-duplicated.  row_ptr has n+1 entries; col_idx must hold m
 * entries (the raw count).  Returns the canonical edge count, or -1. */
int64_t bcg_csr_from_edges(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           int32_t *row_ptr, int32_t *col_idx) {
  if (n < 0 || m < 0) return -1;
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -1;
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) { free(cnt); return -1; }
    if (u != v) cnt[u + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!fill) { free(cnt); return -1; }
  memcpy(fill, cnt, sizeof(int64_t) * ((size_t)n + 1));
  for (int64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) col_idx[fill[src[e]]++] = dst[e];
  free(fill);
  int64_t *uniq = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!uniq) { free(cnt); return -1; }
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t i = 0; i < n; ++i) {
    int32_t *row = col_idx + cnt[i];
    int64_t len = cnt[i + 1] - cnt[i];
    if (len > 1) qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t k = 0;
    for (int64_t j = 0; j < len; ++j)
      if (k == 0 || row[j] != row[k - 1]) row[k++] = row[j];
    uniq[i] = k;
  }
  /* compact rows in place, left to right */
  int64_t out = 0;
  row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int64_t base = cnt[i];
    if (out != base) memmove(col_idx + out, col_idx + base, sizeof(int32_t) * (size_t)uniq[i]);
    out += uniq[i];
    row_ptr[i + 1] = (int32_t)out;
  }
  free(uniq);
  free(cnt);
  return out;
}

/* ---- source lists ------------------------------------------------------ */

/* k distinct vertices of [0, n) drawn uniformly without replacement by a
 * partial Fisher-Yates shuffle driven by splitmix64(seed); k <= n. */
int32_t bcg_sample_sources(int32_t n, int32_t k, uint64_t seed, int32_t *out) {
  if (k < 0 || k > n) return -1;
  int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!a) return -1;
  for (int32_t i = 0; i < n; ++i) a[i] = i;
  uint64_t st = seed;
  for (int32_t i = 0; i < k; ++i) {
    int32_t j = i + (int32_t)bounded(sm64_next(&st), (uint64_t)(n - i));
    int32_t t = a[i];
    a[i] = a[j];
    a[j] = t;
    out[i] = a[i];
  }
  free(a);
  return k;
}

/* Draws `count` integers uniformly from [lo, hi] with a splitmix64 stream. */
void bcg_uniform_ints(int64_t count, int32_t lo, int32_t hi, uint64_t seed, int32_t *out) {
  uint64_t st = seed;
  for (int64_t i = 0; i < count; ++i)
    out[i] = lo + (int32_t)bounded(sm64_next(&st), (uint64_t)(hi - lo + 1));
}
