/*
 * CPU oracle for exact betweenness centrality: TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * use this file.  The product path (the CUDA library) never calls it, links
 * it or shares code with it.
 *
 * What it computes (paper, Section I): the betweenness of v is the sum, over
 * ordered pairs s != v != t, of the fraction of shortest s->t paths that pass
 * through v.  The paper cites Brandes' algorithm (Section I) for the exact
 * O(nm) computation without printing it; this file is the classical
 * sequential form of that algorithm (Brandes 2001, Algorithm 1), unweighted
 * and directed, with no normalisation:
 *
 *   for each source s (in the order given):
 *     1. FIFO BFS from s.  d[s] = 0, sigma[s] = 1.  For a popped v and each
 *        out-neighbour w: if d[w] < 0 then d[w] = d[v] + 1 and w is queued;
 *        if d[w] == d[v] + 1 then sigma[w] += sigma[v] and v is recorded as a
 *        predecessor of w.  Popped vertices are pushed on a stack S.
 *     2. delta = 0.  Pop S (non-increasing distance).  For a popped w and
 *        each predecessor v of w:
 *            delta[v] += sigma[v] / sigma[w] * (1 + delta[w]).
 *        If w != s, BC[w] += delta[w].
 *
 * Readings where the paper is silent:
 *   - the source and the target are excluded (s != v != t); delta_s(s) is
 *     computed but never added;
 *   - input CSR is canonicalised here, independently of any other code:
 *     self-loops and duplicate edges are dropped (a duplicate edge would
 *     double path counts; a self-loop cannot lie on a shortest path);
 *   - sigma is an exact uint64; every add is checked for carry.  Since all
 *     addends are non-negative, the first carrying add happens exactly when
 *     the true count reaches 2^64; the count then saturates and the source is
 *     flagged;
 *   - delta is IEEE double, division is the plain operator;
 *   - BC[v] is summed over sources with Neumaier's compensated summation
 *     (Neumaier 1974), so the oracle's own rounding stays far below the
 *     parity tolerances; no long double is used (its width differs between
 *     x86-64 and aarch64 hosts).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n;
  int64_t m;
  int32_t *off;  /* out-neighbour offsets, n+1 */
  int32_t *adj;  /* out-neighbours, sorted, unique, no self-loops */
  int32_t *poff; /* in-degree offsets (capacity of predecessor lists), n+1 */
} og_graph;

static int cmp_int(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Validates a CSR and builds the oracle's own canonical copy. */
static int og_build(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, og_graph *g) {
  memset(g, 0, sizeof(*g));
  if (n < 0) return -1;
  if (row_ptr[0] != 0) return -1;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return -1;
  int64_t mraw = row_ptr[n];
  for (int64_t e = 0; e < mraw; ++e)
    if (col_idx[e] < 0 || col_idx[e] >= n) return -1;
  g->n = n;
  g->off = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mraw > 0 ? mraw : 1));
  g->poff = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  if (!g->off || !g->adj || !g->poff) return -2;
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mraw > 0 ? mraw : 1));
  if (!tmp) return -2;
  int64_t out = 0;
  g->off[0] = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t len = 0;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
      if (col_idx[e] != v) tmp[len++] = col_idx[e];
    qsort(tmp, (size_t)len, sizeof(int32_t), cmp_int);
    for (int32_t i = 0; i < len; ++i)
      if (i == 0 || tmp[i] != tmp[i - 1]) g->adj[out++] = tmp[i];
    g->off[v + 1] = (int32_t)out;
  }
  free(tmp);
  g->m = out;
  for (int64_t e = 0; e < out; ++e) g->poff[g->adj[e] + 1]++;
  for (int32_t v = 0; v < n; ++v) g->poff[v + 1] += g->poff[v];
  return 0;
}

static void og_free(og_graph *g) {
  free(g->off);
  free(g->adj);
  free(g->poff);
}

typedef struct {
  int32_t *d;
  uint64_t *sigma;
  double *delta;
  int32_t *queue;  /* BFS order; read back to front it is the stack S */
  int32_t *pcnt;   /* predecessors recorded per vertex */
  int32_t *pred;   /* predecessor lists, capacity = in-degree */
} og_work;

static int og_work_alloc(const og_graph *g, og_work *w) {
  size_t n = (size_t)(g->n > 0 ? g->n : 1);
  w->d = (int32_t *)malloc(sizeof(int32_t) * n);
  w->sigma = (uint64_t *)malloc(sizeof(uint64_t) * n);
  w->delta = (double *)malloc(sizeof(double) * n);
  w->queue = (int32_t *)malloc(sizeof(int32_t) * n);
  w->pcnt = (int32_t *)malloc(sizeof(int32_t) * n);
  w->pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m > 0 ? g->m : 1));
  return (w->d && w->sigma && w->delta && w->queue && w->pcnt && w->pred) ? 0 : -2;
}

static void og_work_free(og_work *w) {
  free(w->d);
  free(w->sigma);
  free(w->delta);
  free(w->queue);
  free(w->pcnt);
  free(w->pred);
}

/* Steps 1 and 2 for one source.  Returns the number of reached vertices;
 * *overflow is set when some sigma reached 2^64. */
static int32_t og_one_source(const og_graph *g, og_work *w, int32_t s, int *overflow) {
  const int32_t n = g->n;
  for (int32_t v = 0; v < n; ++v) {
    w->d[v] = -1;
    w->sigma[v] = 0;
    w->delta[v] = 0.0;
    w->pcnt[v] = 0;
  }
  *overflow = 0;
  int32_t head = 0, tail = 0;
  w->d[s] = 0;
  w->sigma[s] = 1;
  w->queue[tail++] = s;
  /* step 1: BFS, path counts, predecessor lists */
  while (head < tail) {
    int32_t v = w->queue[head++];
    for (int32_t e = g->off[v]; e < g->off[v + 1]; ++e) {
      int32_t x = g->adj[e];
      if (w->d[x] < 0) {
        w->d[x] = w->d[v] + 1;
        w->queue[tail++] = x;
      }
      if (w->d[x] == w->d[v] + 1) {
        uint64_t before = w->sigma[x];
        uint64_t after = before + w->sigma[v];
        if (after < before) { /* carry out of 64 bits */
          *overflow = 1;
          after = UINT64_MAX;
        }
        w->sigma[x] = after;
        w->pred[g->poff[x] + w->pcnt[x]++] = v;
      }
    }
  }
  /* step 2: dependencies in reverse BFS order */
  for (int32_t i = tail - 1; i >= 0; --i) {
    int32_t x = w->queue[i];
    for (int32_t p = 0; p < w->pcnt[x]; ++p) {
      int32_t v = w->pred[g->poff[x] + p];
      w->delta[v] += (double)w->sigma[v] / (double)w->sigma[x] * (1.0 + w->delta[x]);
    }
  }
  return tail;
}

/* Number of edges after canonicalisation, or a negative code for an invalid
 * CSR. */
int64_t oracle_canonical_edges(int32_t n, const int32_t *row_ptr, const int32_t *col_idx) {
  og_graph g;
  int rc = og_build(n, row_ptr, col_idx, &g);
  int64_t m = rc == 0 ? g.m : rc;
  og_free(&g);
  return m;
}

/* Copies the oracle's canonical CSR out (row_ptr n+1, col_idx m). */
int64_t oracle_canonicalise(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                            int32_t *out_row_ptr, int32_t *out_col_idx) {
  og_graph g;
  int rc = og_build(n, row_ptr, col_idx, &g);
  if (rc != 0) { og_free(&g); return rc; }
  memcpy(out_row_ptr, g.off, sizeof(int32_t) * ((size_t)n + 1));
  memcpy(out_col_idx, g.adj, sizeof(int32_t) * (size_t)g.m);
  int64_t m = g.m;
  og_free(&g);
  return m;
}

/* Exact BC summed over the given sources (all n vertices in id order when
 * sources == NULL).  bc_out[n]; overflow_out[k] (nullable) receives 1 for a
 * source whose path counts overflowed.  Returns 0, -1 (bad input) or -2
 * (out of memory). */
int oracle_bc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
              const int32_t *sources, int32_t k, double *bc_out, int32_t *overflow_out) {
  og_graph g;
  int rc = og_build(n, row_ptr, col_idx, &g);
  if (rc != 0) { og_free(&g); return rc; }
  if (sources == NULL) k = n;
  for (int32_t i = 0; i < k; ++i)
    if (sources && (sources[i] < 0 || sources[i] >= n)) { og_free(&g); return -1; }
  og_work w;
  double *comp = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (og_work_alloc(&g, &w) != 0 || !comp) {
    og_work_free(&w);
    free(comp);
    og_free(&g);
    return -2;
  }
  for (int32_t v = 0; v < n; ++v) bc_out[v] = 0.0;
  for (int32_t i = 0; i < k; ++i) {
    int32_t s = sources ? sources[i] : i;
    int ovf = 0;
    int32_t reached = og_one_source(&g, &w, s, &ovf);
    if (overflow_out) overflow_out[i] = ovf;
    for (int32_t r = 0; r < reached; ++r) {
      int32_t v = w.queue[r];
      if (v == s) continue;
      /* Neumaier compensated add of delta[v] into bc_out[v] */
      double x = w.delta[v], sum = bc_out[v], t = sum + x;
      if ((sum >= 0 ? sum : -sum) >= (x >= 0 ? x : -x))
        comp[v] += (sum - t) + x;
      else
        comp[v] += (x - t) + sum;
      bc_out[v] = t;
    }
  }
  for (int32_t v = 0; v < n; ++v) bc_out[v] += comp[v];
  free(comp);
  og_work_free(&w);
  og_free(&g);
  return 0;
}

/* One source's distance, path count and dependency vectors (d = -1,
 * sigma = 0, delta = 0 for unreached vertices).  Returns the number of
 * reached vertices, or a negative code; *overflow as in oracle_bc. */
int32_t oracle_single_source(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                             int32_t s, int32_t *d_out, uint64_t *sigma_out, double *delta_out,
                             int32_t *overflow) {
  og_graph g;
  int rc = og_build(n, row_ptr, col_idx, &g);
  if (rc != 0) { og_free(&g); return rc; }
  if (s < 0 || s >= n) { og_free(&g); return -1; }
  og_work w;
  if (og_work_alloc(&g, &w) != 0) { og_work_free(&w); og_free(&g); return -2; }
  int ovf = 0;
  int32_t reached = og_one_source(&g, &w, s, &ovf);
  memcpy(d_out, w.d, sizeof(int32_t) * (size_t)n);
  memcpy(sigma_out, w.sigma, sizeof(uint64_t) * (size_t)n);
  memcpy(delta_out, w.delta, sizeof(double) * (size_t)n);
  if (overflow) *overflow = ovf;
  og_work_free(&w);
  og_free(&g);
  return reached;
}
