/*
 * bc_gb300.h -- C ABI of the GB300 (sm_103a) exact betweenness-centrality
 * library.
 *
 * Method.  Betweenness centrality of a vertex v is the sum, over ordered
 * pairs of distinct vertices s != v != t, of the fraction of shortest s->t
 * paths that pass through v (paper, Section I).  Exact values come from
 * Brandes' algorithm, which the paper names (Section I) and studies on the GPU
 * (Section II.A): per source s, a level-synchronous BFS gives the depth d[]
 * and the shortest-path counts sigma[]; a reverse-level sweep then gives the
 * dependencies
 *     delta[v] = sum over successors w (edge v->w, d[w] = d[v] + 1) of
 *                sigma[v] / sigma[w] * (1 + delta[w]),
 * and BC[v] accumulates delta[v] over all sources s != v.  Graphs are
 * unweighted and directed (paper, Section II.C); BC values are raw sums with
 * no normalisation unless an option asks for it.
 *
 * Conventions shared by every entry point.
 *   - Return values are bc_status codes: 0 on success, BC_PENDING (1) for an
 *     unfinished job, negative on error.  Nothing aborts the process and no
 *     device code traps; a device-side failure is reported as a status.
 *   - Input arrays are copied before the call returns; the caller keeps
 *     ownership and may free them immediately.  Output buffers are always
 *     owned by the caller.
 *   - Output BC vectors are float64[n].  bc_opts.out_device selects whether
 *     bc_out is host memory (0) or device memory on the context's GPU (1).
 *   - Vertex ids are int32 in [0, n); edge counts are int64 but must stay
 *     below 2^31.
 *   - Depths and path counts are exact integers (int32 / uint64).  A source
 *     whose path count reaches 2^64 makes the call return
 *     BC_ERR_SIGMA_OVERFLOW; bc_out is still written but is not valid for the
 *     flagged sources (bc_stats.overflow_sources counts them).
 *   - A context is not thread-safe: calls on one context must not overlap,
 *     except that bc_submit / bc_poll may be called while jobs run on the
 *     context's internal scheduler thread.
 */
#ifndef BC_GB300_H
#define BC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bc_ctx bc_ctx; /* opaque; one per GPU */
typedef int64_t bc_graph;     /* graph handle, > 0 */
typedef int64_t bc_job;       /* job handle, > 0 */

typedef enum {
  BC_OK = 0,
  BC_PENDING = 1,             /* bc_poll: job not finished yet */
  BC_ERR_ARG = -1,            /* bad argument (null pointer, source id out of range, bad option) */
  BC_ERR_GRAPH = -2,          /* malformed CSR, or unknown graph handle */
  BC_ERR_OOM = -3,            /* device or host allocation failed */
  BC_ERR_CUDA = -4,           /* a CUDA runtime call failed */
  BC_ERR_TIMEOUT = -5,        /* a bounded device-side wait ran out */
  BC_ERR_SIGMA_OVERFLOW = -6, /* some shortest-path count reached 2^64 */
  BC_ERR_NOT_FOUND = -7,      /* unknown or already consumed job handle */
  BC_ERR_ADMISSION = -8,      /* job footprint exceeds the context's HBM budget */
  BC_ERR_INTERNAL = -9        /* device-side capacity check failed (a bug) */
} bc_status;

/* Work schedules.  AUTO is BATCH. */
enum {
  BC_SCHED_AUTO = 0,
  BC_SCHED_PLAIN = 1,        /* one source per kernel launch, level-synchronous: the whole GPU
                                per source, or one thread block per source on small graphs */
  BC_SCHED_BATCH = 2,        /* up to 256 sources per launch, bitset frontiers, per-level
                                frontier queues, [n][k] state.  The first job on a graph with
                                enough sources times trial batches and keeps, per graph, the
                                fastest batch width (when batch_k = 0) and work split */
  BC_SCHED_BATCH_QUEUE = 3,  /* the same as BATCH */
  BC_SCHED_BATCH_VERTEX = 4, /* BATCH with a fixed vertex-centric split: one warp per frontier
                                entry whatever its degree */
  BC_SCHED_BATCH_WARP = 5,   /* BATCH, warp-centric: entries with more than 256 in- plus
                                out-edges cut into 256-edge chunks, one warp each */
  BC_SCHED_BATCH_EDGE = 6    /* BATCH, edge-centric leaning: 128-edge chunks */
};

typedef struct {
  int32_t delta_fp64;    /* 0: dependencies in FP32 (fast path); 1: FP64 */
  int32_t batch_k;       /* sources per batch of the batched schedules: 0 = the library picks
                            64, 128 or 256 (the widest that still gives the job eight batches;
                            64 for debug exports; per graph in bc_exact_many); else 1..256 for
                            BC_SCHED_AUTO / BATCH / BATCH_QUEUE, 1..64 for bc_exact_many.  Bit j of a batch's source masks is its j-th
                            source; masks are 1, 2 or 4 64-bit words.  Wider batches size
                            their frontier queue for 64 distinct depths per vertex; a job
                            that overruns it reruns with 64 sources per batch, and so do
                            later jobs on that graph */
  int32_t schedule;      /* BC_SCHED_* */
  int32_t normalize;     /* 0: raw sums; 1: divide by (n-1)(n-2) when n > 2 */
  int32_t scale_sampled; /* 0: raw sum over the given sources; 1: multiply by n/k */
  int32_t out_device;    /* 0: bc_out is host memory; 1: device memory */
  int32_t source_order;  /* batched schedules: 0 (default) = the library composes the batches,
                            grouping sources whose traversals line up (sources without
                            out-edges last, the others by the number of two-hop walks,
                            descending), so fewer (vertex, level) frontier entries and
                            edge scans are shared by more sources; 1 = batches take the
                            sources in the given order.  The result is the same sum over
                            the sources, up to floating-point summation order. */
  int32_t direction;     /* path-count step of each forward level l >= 1 of the batched
                            schedules: 0 (default) = per level, pull over the in-edges of
                            level l unless pushing from level l-1 along its out-edges scans
                            several times fewer edges; 1 = always pull; 2 = always push.
                            Pulling adds in a fixed order, pushing with 64-bit integer
                            atomics; both give the same exact counts.  A pushed count of
                            2^32 or more makes the job rerun pulling (and later jobs on
                            that graph pull) */
  int32_t count_bits;    /* storage of the batched schedules' path counts: 0 (default) = 32
                            bits, and a job in which a count reaches 2^32 reruns with 64 bits
                            (so do later jobs on that graph); 64 = always 64 bits.  Sums and
                            results are the same; 32-bit rows halve the bytes each
                            shortest-path edge moves.  bc_exact_many follows it per graph:
                            a graph whose count reaches 2^32 continues with 64 bits from
                            that batch.  Estimator calls use 64 bits */
} bc_opts;

/* Per-call statistics.  Counters feed the bytes model of the roofline. */
typedef struct {
  int64_t n;                 /* vertices */
  int64_t m;                 /* canonical edges */
  int64_t sources;           /* sources processed */
  int64_t batches;           /* kernel passes (one per batch, or per source for PLAIN); batched
                                calls in the library's source order do not launch sources
                                without out-edges (their traversal adds nothing to BC) */
  int64_t kernel_launches;   /* kernels launched by the call */
  int32_t max_levels;        /* deepest BFS level count over all sources */
  int32_t overflow_sources;  /* sources whose path count reached 2^64 */
  double device_ms;          /* device time of the BC kernels (CUDA events) */
  int64_t frontier_entries;  /* (vertex, level) pairs with a non-empty frontier mask */
  int64_t scanned_out_edges; /* out-edges scanned, forward discovery plus backward */
  int64_t scanned_in_edges;  /* in-edges scanned by the path-count pull */
  int64_t dag_pairs;         /* sum over sources of shortest-path DAG edges */
  int64_t reached_pairs;     /* sum over sources of reached vertices (incl. source) */
  int64_t heavy_chunks;      /* edge chunks of high-degree vertices split across warps */
  int32_t kernel_kind;       /* kernel of the last launch: 1 plain, 2 batch (frontier queue) */
  int32_t levels_sum;        /* BFS level counts summed over all batches */
  int32_t chunk_edges;       /* edges per chunk of a high-degree vertex in the last launch */
  int32_t grab;              /* work items a warp fetched at a time in the last launch */
  int32_t batch_sources;     /* sources per batch of the call's full batches (a last batch of at
                                most half as many runs with fewer mask words) */
  int32_t mask_words;        /* 64-bit words per source mask of those batches (1, 2 or 4) */
  int32_t push_levels;       /* forward levels whose path counts were pushed, over all batches */
  int32_t batch_groups;      /* batches the last launches ran at once (concurrent groups) */
} bc_stats;

/* Creates a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * to order work on, or NULL for a stream the context creates and owns.
 * hbm_budget_bytes caps the device memory the context may hold for job
 * state (0 = 90% of the memory free at creation); graphs count against it.
 * Errors: BC_ERR_ARG (null out), BC_ERR_CUDA (no such device). */
bc_status bc_init(int device, void *cuda_stream, size_t hbm_budget_bytes, bc_ctx **out);

/* Waits for outstanding jobs, frees every graph and buffer, destroys the
 * context.  The handle is invalid afterwards. */
bc_status bc_shutdown(bc_ctx *ctx);

/* Uploads a directed graph given as host CSR: out-neighbours of v are
 * col_idx[row_ptr[v] .. row_ptr[v+1]).  Rejected with BC_ERR_GRAPH when
 * n < 0, row_ptr[0] != 0, row_ptr decreases, row_ptr[n] != m, m >= 2^31 or
 * a column is outside [0, n).  The graph is canonicalised (rows sorted,
 * duplicate edges and self-loops dropped; paper Section II.D stores graphs
 * as adjacency lists, and a duplicate edge would double path counts); the
 * resulting edge count is written to *m_effective (nullable).  Both arrays
 * are copied; the graph stays resident in HBM until bc_destroy_graph. */
bc_status bc_create_graph(bc_ctx *ctx, const int32_t *row_ptr, const int32_t *col_idx,
                          int32_t n, int64_t m, bc_graph *out, int64_t *m_effective);

/* Uploads `count` graphs at once, as bc_create_graph does one by one:
 * graph i is row_ptrs[i] (ns[i]+1 entries) and col_idxs[i] (ms[i] entries),
 * host memory, validated and canonicalised the same way.  Graphs of up to
 * 2^18 edges are prepared on host threads in parallel and uploaded in
 * groups (one transfer per graph, one synchronisation per group), which is
 * what makes creating many small graphs cheap; larger ones take the device
 * path one by one.  All or nothing: on any error no graph is kept and the
 * status is that of the first failing step (BC_ERR_GRAPH for a malformed
 * graph, BC_ERR_ADMISSION past the HBM budget).  out[i] receives graph i's
 * handle and m_effective[i] (may be NULL) its canonical edge count. */
bc_status bc_create_graphs(bc_ctx *ctx, int32_t count, const int32_t *const *row_ptrs,
                           const int32_t *const *col_idxs, const int32_t *ns, const int64_t *ms,
                           bc_graph *out, int64_t *m_effective);

/* Frees a graph.  Fails with BC_ERR_ARG while a submitted job still uses it. */
bc_status bc_destroy_graph(bc_ctx *ctx, bc_graph g);

/* Exact BC over all n sources (paper, Section I).  bc_out: float64[n].
 * opts may be NULL (FP32 dependencies, automatic schedule, raw output to
 * host memory).  Blocks until the result is written.  Errors (this and the
 * other BC calls): BC_ERR_ARG also when a batched schedule meets a graph
 * whose 2n + 2 x (heavy-vertex chunks) reaches 2^31 (the kernels index a
 * level step's work items in 32 bits; such a graph's workspace would not
 * fit one GPU anyway). */
bc_status bc_exact(bc_ctx *ctx, bc_graph g, const bc_opts *opts, double *bc_out);

/* BC summed over the k given sources (host int32[k], each in [0, n);
 * a repeated source counts once per occurrence).  With scale_sampled the
 * sum is multiplied by n/k, the usual estimator of exact BC from sampled
 * sources (paper, Section I cites approximate BC by sampling).  Errors:
 * BC_ERR_ARG for k < 0 or a source out of range. */
bc_status bc_sources(bc_ctx *ctx, bc_graph g, const int32_t *src, int32_t k,
                     const bc_opts *opts, double *bc_out);

/* Estimate of BC from k sources taken as a uniform sample without
 * replacement from the n vertices, with its standard error (paper, Section I
 * cites approximate BC by source sampling without fixing an estimator).
 * With x_s(v) = delta_s(v) for v != s and 0 for v == s, m(v) their mean over
 * the k sources and S2(v) their sample variance (k - 1 denominator):
 *   est_out[v]    = n * m(v)
 *   stderr_out[v] = n * sqrt((1 - k/n) * S2(v) / k)
 * (NaN for k < 2; the finite-population factor 1 - k/n is taken as 0 when
 * k >= n, so all n distinct sources give the exact BC with zero error).  The
 * kernels accumulate sums of x and x^2 per vertex in FP64; opts.normalize
 * scales both outputs by 1/((n-1)(n-2)); opts.scale_sampled is ignored.
 * est_out / stderr_out: float64[n] each, host or device per opts.out_device.
 * Errors as bc_sources; BC_ERR_SIGMA_OVERFLOW still writes the outputs. */
bc_status bc_sources_estimate(bc_ctx *ctx, bc_graph g, const int32_t *src, int32_t k,
                              const bc_opts *opts, double *est_out, double *stderr_out);

/* Adaptive source sampling: takes sources from `order` (host int32[max_k],
 * each in [0, n), a sample order drawn by the caller, e.g. a seeded
 * permutation) in rounds of `round`, and stops after the first round at
 * which every vertex whose estimate (in output units) is at least min_est
 * has stderr <= rel_err * estimate, or when max_k sources are used.  Writes
 * the estimate and standard error over the sources used (as
 * bc_sources_estimate over order[0 .. *k_used)) and their number to k_used.
 * Errors: BC_ERR_ARG for max_k < 1, round < 1, rel_err <= 0, null outputs or
 * a source out of range. */
bc_status bc_sources_adaptive(bc_ctx *ctx, bc_graph g, const int32_t *order, int32_t max_k,
                              int32_t round, double rel_err, double min_est,
                              const bc_opts *opts, double *est_out, double *stderr_out,
                              int32_t *k_used);

/* Queues a BC job (src == NULL: all sources; else k host sources, copied)
 * for the context's scheduler thread and returns at once.  Jobs are admitted
 * when their device footprint fits the HBM budget next to the jobs already
 * running; jobs run concurrently on separate streams.  A job that could never
 * fit is refused with BC_ERR_ADMISSION.  opts is copied (out_device must be
 * 0: results are handed over by bc_poll). */
bc_status bc_submit(bc_ctx *ctx, bc_graph g, const int32_t *src, int32_t k, const bc_opts *opts,
                    bc_job *out);

/* Non-blocking.  Returns BC_PENDING while the job runs; otherwise writes the
 * job's float64[n] result to host bc_out, its statistics to stats
 * (nullable), forgets the job and returns the job's final status.  A
 * consumed or unknown handle gives BC_ERR_NOT_FOUND. */
bc_status bc_poll(bc_ctx *ctx, bc_job job, double *bc_out, bc_stats *stats);

/* Like bc_poll but waits up to timeout_ms (<0: no limit) for completion;
 * BC_ERR_TIMEOUT when the limit passes first (the job keeps running). */
bc_status bc_wait(bc_ctx *ctx, bc_job job, int64_t timeout_ms, double *bc_out, bc_stats *stats);

/* Statistics of the last completed synchronous call (bc_exact / bc_sources /
 * bc_exact_many / bc_debug_*) on this context. */
bc_status bc_last_stats(bc_ctx *ctx, bc_stats *stats);

/* The sources whose shortest-path count reached 2^64 in the last synchronous
 * call on this context (bc_exact, bc_sources, bc_sources_estimate and the
 * like; each flagged occurrence of a repeated source listed), ascending.
 * Writes up to `capacity` ids to src_out (host int32) and the full number to
 * count.  Errors: BC_ERR_ARG for null count or a null src_out with
 * capacity > 0. */
bc_status bc_last_overflow_sources(bc_ctx *ctx, int32_t *src_out, int32_t capacity,
                                   int32_t *count);

/* Per-source vectors of one source through the PLAIN schedule: depth d
 * (int32, -1 unreached), path count sigma (uint64, 0 unreached) and
 * dependency delta (float64; delta[s] is the source's own dependency, which
 * BC excludes).  Host arrays of n entries each; any may be NULL. */
bc_status bc_debug_source(bc_ctx *ctx, bc_graph g, int32_t s, int32_t *d_out,
                          uint64_t *sigma_out, double *delta_out);

/* Same vectors for k sources through the schedule opts selects, laid out
 * source-major: entry [j*n + v].  Host arrays; any may be NULL. */
bc_status bc_debug_sources(bc_ctx *ctx, bc_graph g, const int32_t *src, int32_t k,
                           const bc_opts *opts, int32_t *d_out, uint64_t *sigma_out,
                           double *delta_out);

/* The graph as the library holds it on the device: the canonical out-CSR
 * row_ptr[n+1], col_idx[m] (m = the canonical edge count; every row
 * ascending, no duplicates or self-loops) and its transpose in_ptr[n+1],
 * in_idx[m] (in-neighbours of v in in_idx[in_ptr[v] .. in_ptr[v+1]),
 * ascending).  Host arrays owned by the caller; any may be NULL.  For tests
 * and debugging.  Errors: BC_ERR_ARG (null ctx), BC_ERR_GRAPH (unknown
 * handle), BC_ERR_CUDA. */
bc_status bc_debug_graph(bc_ctx *ctx, bc_graph g, int32_t *row_ptr, int32_t *col_idx,
                         int32_t *in_ptr, int32_t *in_idx);

/* Exact BC of `count` resident graphs.  Graphs of up to 8192 vertices run in
 * ONE persistent launch: each thread block takes the next graph (largest
 * n*(m+n) first), runs all of its source batches (opts.batch_k sources each;
 * with batch_k = 0 each graph gets 64, 128 or 256 by the automatic rule on
 * its vertex count, and a wide batch that overruns its frontier queue
 * continues 64 per batch) with block-level barriers between BFS levels and
 * writes that graph's BC itself (path counts in 32-bit rows unless
 * opts.count_bits = 64; with batches composed by the library, source_order = 0,
 * a graph's sources without out-edges, whose terms are all zero, are not run);
 * larger graphs run one after another through the grid-wide batched kernel.  bc_out receives the vectors back to back (graph
 * i at offset sum_{j<i} n_j), host or device memory per opts.out_device;
 * normalize applies per graph, scale_sampled has no effect (all sources).
 * BC_ERR_ADMISSION when the per-block workspaces do not fit the budget. */
bc_status bc_exact_many(bc_ctx *ctx, const bc_graph *graphs, int32_t count, const bc_opts *opts,
                        double *bc_out);

/* Test hook for failure detection: with block >= 0 the next BATCH launch on
 * this context has that thread block skip its first grid-barrier arrival
 * and the others give up after timeout_ms, so the call returns
 * BC_ERR_TIMEOUT and the context stays usable.  block < 0 disables it. */
bc_status bc_debug_inject_barrier_skip(bc_ctx *ctx, int32_t block, int32_t timeout_ms);

/* Largest vertex count bc_sources_noalloc accepts. */
#define BC_NOALLOC_MAX_N 8192

/* BC summed over k sources for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment variant of bc_sources.
 *
 * Who needs it: code that may not call cudaMalloc when it needs the result,
 * e.g. a service running under a device-memory budget reserved at start-up,
 * a framework whose caching allocator owns all device memory, or a callback
 * where an allocation could stall on device synchronisation.  The call
 * allocates nothing: no cudaMalloc / cudaFree / cudaMallocAsync and no
 * allocating library routine.  Its working state is one fixed array of about
 * 15 MB compiled into the library, which every GPU that loads the library
 * holds until the process exits; that array bounds n to BC_NOALLOC_MAX_N.
 *
 * Inputs: the graph as DEVICE memory owned by the caller, already canonical
 * (rows sorted, no duplicate edges, no self-loops): out-CSR row_ptr[n+1],
 * col_idx[m] and its transpose in_ptr[n+1], in_idx[m] (in-neighbours of v are
 * in_idx[in_ptr[v] .. in_ptr[v+1])); these are not validated beyond their
 * sizes.  src: HOST int32[k], each in [0, n) (checked).  delta_fp64 as in
 * bc_opts.  Output: bc_out, DEVICE float64[n], overwritten with raw sums.
 * cuda_stream: the cudaStream_t to run on (NULL: the legacy default stream).
 * The call returns after the result is written.
 *
 * Limits and sharing: n > BC_NOALLOC_MAX_N, m >= 2^31, k < 0, a null pointer
 * or a source out of range give BC_ERR_ARG before any work.  Every call on a
 * GPU uses the same array and leaves its contents behind; each call clears
 * what must start at zero, so sequential calls are independent, but calls
 * that overlap on the GPU (other host threads, other streams) race on the
 * array and give wrong results.  High-degree vertices are not split across
 * warps, so hubs run slower than through bc_sources.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) and the
 * kernel's grid size with that device current; make that first call before
 * any stream capture.  Only a successful look-up is kept: if it fails (also
 * when a CUDA error from earlier, unrelated work is still pending on the
 * calling thread, which this call reports as BC_ERR_CUDA and does not clear)
 * the next call tries again.  If fewer thread blocks can run at once than at
 * that first call (the GPU shared differently, e.g. under MPS), the launch
 * is retried with half the grid until it fits. */
bc_status bc_sources_noalloc(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *in_ptr,
                             const int32_t *in_idx, int32_t n, int64_t m, const int32_t *src,
                             int32_t k, int32_t delta_fp64, double *bc_out, void *cuda_stream);

/* Static description of a status code. */
const char *bc_status_str(bc_status status);

#ifdef __cplusplus
}
#endif

#endif /* BC_GB300_H */
