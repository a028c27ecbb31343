// Internal declarations of the GB300 betweenness-centrality library: device
// control block, graph and workspace descriptors, kernel parameters and the
// host-side launchers.  Not part of the C ABI (see include/bc_gb300.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bcgpu {

constexpr int kWarp = 32;
// Threads per CTA of the persistent kernels: one 1024-thread CTA per SM (32
// warps, 64 registers each).  Measured against 4 x 256 and 2 x 512 with the
// same warps per SM: fewer CTAs make the grid barrier cheaper and give the
// many-graph launch more threads per graph (+4% on R-MAT scale 16 exact
// BC, +17% on 10,000 small graphs, equal elsewhere).
constexpr int kBlock = 1024;
constexpr int kWarpsPerBlock = kBlock / kWarp; // 32
constexpr int kK = 64;                         // sources per mask word (one bit each in a u64)
constexpr int kMaxWords = 4;                   // queue kernel: up to 4 words = 256 sources per batch
constexpr int kWideMinBatches = 8;             // automatic width: batches a job must still have

// Mask words of a job of k sources when the library picks the width: the
// widest batch (64 sources per word, up to max_words words) that still gives
// the job kWideMinBatches batches; wider batches share each (vertex, level)
// entry and edge scan among more sources.
__host__ __device__ constexpr int auto_words(int64_t k, int max_words) {
  return max_words >= 4 && k >= (int64_t)kWideMinBatches * kK * 4   ? 4
         : max_words >= 2 && k >= (int64_t)kWideMinBatches * kK * 2 ? 2
                                                                    : 1;
}
// Work split of a level's entries among warps (the per-graph tuner picks
// one; the first is the default before tuning): an entry with more in- plus
// out-edges than the chunk size is cut into chunks of about that many edges,
// each taken by its own warp; smaller entries take one warp each.  128 edges
// leans towards edge-centric balance, 256 and 512 are warp-centric, and 2^30
// never splits (vertex-centric: one warp per entry, whatever its degree).
constexpr int kChunkCandidates[4] = {256, 128, 512, 1 << 30}; // 1 << 30: never split
constexpr int kChunkVariants = 4;
constexpr int kSplitWarp = 0, kSplitEdge = 1, kSplitWarp512 = 2, kSplitVertex = 3;
constexpr int kChunk = kChunkCandidates[0];    // chunk size of the plain and no-alloc paths
#ifndef BC_HEAVY_MIN
#define BC_HEAVY_MIN 256
#endif
// Entries listed with the heavy ones, which a step takes first: more in- plus
// out-edges than the chunk size (split into chunks of about that many), or,
// with a split, than BC_HEAVY_MIN (one chunk, not split).  Starting the long
// unsplit entries early leaves short ones for the end of the step, where
// warps that are done wait for the last: R-MAT scale 20 with 512-edge
// chunks, +2% with 256 (no vertex there has 193 to 320 edges, so 192..320
// are one setting), +1% with 128.  The vertex-centric split keeps its
// order (-2% on the directed preferential-attachment graph).
__host__ __device__ constexpr int64_t heavy_threshold(int64_t chunk) {
  return BC_HEAVY_MIN > 0 && BC_HEAVY_MIN < chunk && chunk < (1 << 30) ? BC_HEAVY_MIN : chunk;
}
#ifndef BC_PREFETCH_GROUPS
#define BC_PREFETCH_GROUPS 0 // 1: fetch the next item group before processing the current one
#endif
constexpr int kGrabDefault = 2;                // work items a warp takes per counter fetch
constexpr int kGrabMax = 2;                    // largest fetch the kernels' header rounds hold
#ifndef BC_BATCH_MIN_BLOCKS
#define BC_BATCH_MIN_BLOCKS 1                  // resident CTAs per SM the batch kernel is built for
#endif
constexpr int kBatchMinBlocks = BC_BATCH_MIN_BLOCKS;

// Device-side error codes (sticky in Ctl::err).
enum : int {
  KERR_NONE = 0,
  KERR_TIMEOUT = 1,  // a grid-barrier wait ran out
  KERR_QUEUE = 2,    // frontier queue capacity exceeded
  KERR_HEAVY = 3,    // heavy-entry list capacity exceeded
  KERR_CHUNKS = 4,   // heavy chunk scratch exceeded
  KERR_GRAB = 6,     // more work items per fetch than a header round holds (host bug)
  KERR_PUSH = 7,     // a pushed path count was 2^32 or more: the job reruns pulling counts
  KERR_WIDE = 8,     // a path count did not fit 32-bit storage: the job reruns with 64 bits
};

// Job-level counters (uint64 each), accumulated by the kernels.
enum : int {
  CNT_ENTRIES = 0,   // (vertex, level) frontier entries
  CNT_OUT_EDGES = 1, // out-edges scanned (discovery + backward)
  CNT_IN_EDGES = 2,  // in-edges scanned (path-count pull)
  CNT_DAG = 3,       // (source, DAG edge) pairs
  CNT_REACHED = 4,   // (source, reached vertex) pairs
  CNT_HEAVY = 5,     // heavy chunks processed (forward + backward)
  CNT_MAXLEV = 6,    // max level count (atomicMax)
  CNT_LEVELS = 7,    // level counts summed over batches
  CNT_BUSY = 8,      // phase-clock builds: warp cycles spent on step items
  CNT_IDLE = 9,      // phase-clock builds: warp cycles from a warp's last item to the step's end
  CNT_PUSH = 10,     // forward levels whose path counts were pushed (summed over batches)
  CNT_N = 11
};


// Per-workspace control block; the host zeroes it once per job.
struct Ctl {
  unsigned int bar_count; // grid barrier arrivals
  unsigned int bar_gen;   // grid barrier generation
  int err;                // first device error (KERR_*), sticky for the job
  int nlevels;            // levels of the current batch
  unsigned long long tail; // frontier queue tail (entries)
  unsigned long long ovf[kMaxWords]; // batch: sources (bits) whose count reached 2^64; plain: [0] 0/1
  unsigned long long work[4]; // work-item counters of consecutive steps (ring)
};

// A resident graph: out-CSR, in-CSR and the per-vertex chunk count
// (0 = light vertex handled by one warp, else ceil((in+out)/kChunk)).
struct GraphDev {
  int32_t n = 0;
  int64_t m = 0;
  const int32_t *row_ptr = nullptr;
  const int32_t *col_idx = nullptr;
  const int32_t *in_ptr = nullptr;
  const int32_t *in_idx = nullptr;
  const int32_t *nchunks = nullptr;
  int64_t heavy_vertices = 0; // vertices with nchunks > 0
  int64_t heavy_chunks = 0;   // sum of nchunks
  const int32_t *order = nullptr; // all vertices in batch-composition order (exact BC)
};

// Device workspace of one in-flight batch (or one plain source).
struct Work {
  int32_t n = 0;
  int32_t k_max = 0;          // 64 * words for the batch kernels, 1 for plain
  int32_t words = 1;          // batch: 64-bit words per source mask
  uint64_t *vis = nullptr;    // batch: [n][words] visited masks
  uint64_t *fr = nullptr;     // batch: [4][n][words] rotating dense frontier masks
  int32_t *claim = nullptr;   // queue kernel, words > 1: [n] 1 + the deepest level a vertex was
                              // queued at (first-toucher claims)
  int32_t *d = nullptr;       // plain: [n] depth (-1 unreached)
  int32_t *qv = nullptr;      // [cap] frontier entries (vertex ids), levels back to back
  uint64_t *qm = nullptr;     // batch: [cap][words] entry masks
  int64_t cap = 0;
  int64_t *qoff = nullptr;    // [n+3] start of each level in qv
  unsigned long long *hpack = nullptr; // [n+3] per level: (heavy count << 32) | chunk total
  int64_t *hoff = nullptr;    // [n+3] start of each level's heavy list
  int64_t *hq_e = nullptr;    // [hcap] queue position
                              // of each heavy entry
  int64_t *hq_c = nullptr;    // [hcap] first chunk of each heavy entry within its level
  unsigned *harrive = nullptr; // [hcap] chunk arrivals per heavy entry
  int64_t hcap = 0;
  void *partial = nullptr;    // [chunk_cap][k_max] chunk partial sums (u64 or float type)
  uint64_t *partial_ovf = nullptr; // [chunk_cap][words] overflow bits of forward partials
  int64_t chunk_cap = 0;
  unsigned long long *lsum = nullptr; // batch: [n+3][2] per level: summed in- and out-degree of
                              // its vertices (the scan lengths of pulling and pushing counts)
  uint64_t *sigma = nullptr;  // [n][k_max] path counts
  void *cdep = nullptr;       // [n][k_max] (1 + delta) / sigma, float or double
  Ctl *ctl = nullptr;
};

struct KParams {
  GraphDev g;
  Work w;
  const int32_t *src = nullptr; // device [k] sources of this batch
  int32_t k = 0;
  int64_t src_base = 0;         // position of src[0] in the job's source list
  double *bc = nullptr;         // [n] accumulator (float64)
  double *bc2 = nullptr;        // [n] optional accumulator of squared per-source terms
  int8_t *ovf_flags = nullptr;  // [job sources] 1 = count reached 2^64
  unsigned long long *job_cnt = nullptr; // [CNT_N]
  int32_t *dbg_d = nullptr;     // [k][n] or null
  uint64_t *dbg_sigma = nullptr;
  double *dbg_delta = nullptr;
  long long timeout_ns = 2000000000LL;
  int32_t skip_block = -1;      // failure-injection hook (-1: none)
  unsigned long long *trace = nullptr; // optional [trace_cap][4] per-step records
  int32_t trace_cap = 0;
  int32_t grab = kGrabDefault;  // work items per counter fetch
  // Direction of the path-count step of forward level l >= 1: 0 = always
  // pull over the in-edges of level l; r > 0 = push from level l-1 along its
  // out-edges when r x (their out-degree sum) < (level l's in-degree sum);
  // -1 = push at every level >= 1.  Needs Work::lsum.
  int32_t push_ratio = 0;
};

// Parameters of the many-small-graphs launch: one thread block per graph at a
// time, graphs taken from *next in the order given.
struct ManyParams {
  KParams base;                   // counters, flags, timeout (graph/batch fields unused)
  const GraphDev *graphs = nullptr; // [count]
  const int32_t *order = nullptr; // [count] graph indices, largest work first
  const int64_t *out_off = nullptr; // [count] offset of each graph's BC (and source flags)
  int32_t count = 0;
  const Work *works = nullptr;    // [grid] one workspace per thread block
  const int32_t *iota = nullptr;  // [max n] 0, 1, 2, ...: the sources of exact BC in given order
  int32_t grouped = 1;            // 1: batches take the sources in GraphDev::order
  const int32_t *traverse = nullptr; // [count] sources each graph runs: with grouped
                                  // batches its vertices with out-edges (first in
                                  // GraphDev::order; the others add nothing), else n
  int32_t max_words = 1;          // widest source masks a graph may use (auto_words)
  int32_t counts64 = 0;           // 1: 64-bit path-count rows throughout; 0: 32-bit rows,
                                  // and a graph with a count of 2^32 or more continues
                                  // (from the batch that found it) with 64-bit rows
  double *out = nullptr;          // [sum of n]
  unsigned *next = nullptr;       // graph counter
  int32_t kb = kK;                // sources per batch when max_words == 1
};

// Parameters of a launch that runs a job's batches in concurrent groups of
// thread blocks: group g (blocks g*gsize .. g*gsize+gsize-1) takes batches
// g, g+groups, ... of the job's sources from `first` on, with workspace
// works[g] and BC partial vector parts[g][n].
struct MultiParams {
  KParams base;                 // src = the job's source list; bc unused
  const Work *works = nullptr;  // [groups]
  double *parts = nullptr;      // [groups][n]
  int32_t groups = 1;
  int32_t gsize = 1;
  int32_t kb = kK;              // sources per batch
  int64_t k = 0;                // sources of the job
  int64_t first = 0;            // first source of the grouped range
};

// Host launchers (bc_kernels.cu; the many-graph launch in bc_many.cu).
// Return a cudaError_t.
cudaError_t launch_many(const ManyParams &mp, bool fp64, int grid, cudaStream_t st);
int max_grid_many(bool fp64, int device);
cudaError_t launch_batch(const KParams &p, bool fp64, int grid, cudaStream_t st, int words = 1,
                         bool counts32 = false);
cudaError_t launch_multi(const MultiParams &mp, bool fp64, int words, bool counts32,
                         cudaStream_t st);
// A batch of `words` mask words in a workspace laid out for layout_words >
// words (bc_narrow.cu); plain BC only (no squared terms).
cudaError_t launch_batch_narrow(const KParams &p, bool fp64, int grid, cudaStream_t st,
                                int words, int layout_words, bool counts32);
cudaError_t launch_plain(const KParams &p, bool fp64, int grid, cudaStream_t st);
cudaError_t launch_plain_block(const KParams *slots, int slot, int64_t b, bool fp64,
                               cudaStream_t st);
cudaError_t launch_sum_parts(const double *parts, int nparts, int64_t n, double *out,
                             cudaStream_t st, bool add_to_out = false);
cudaError_t launch_gather_err(Ctl *first, size_t stride_bytes, int count, cudaStream_t st);
cudaError_t launch_scale(const double *in, double *out, int64_t n, double factor, cudaStream_t st);
cudaError_t launch_estimate(const double *sum, const double *sumsq, int64_t n, int64_t k,
                            double factor, double *est, double *err, cudaStream_t st);
cudaError_t launch_max_rel_err(const double *est, const double *err, int64_t n, double min_est,
                               unsigned long long *out, cudaStream_t st);
cudaError_t launch_accumulate(double *acc, double *acc2, const double *add, const double *add2,
                              int64_t n, const int *err, cudaStream_t st);

// Graph preparation (bc_graph.cu).
cudaError_t launch_check_csr(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int *flags,
                             cudaStream_t st);
cudaError_t launch_in_degree(const int32_t *col_idx, int64_t m, int32_t n, int32_t *cnt,
                             cudaStream_t st);
int64_t scan_scratch_elems(int64_t len);
cudaError_t launch_scan_inclusive(int32_t *a, int64_t len, int32_t *scratch, cudaStream_t st);
cudaError_t launch_in_scatter(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                              int32_t *fill, int32_t *in_idx, cudaStream_t st);
cudaError_t launch_sort_rows(const int32_t *in_ptr, int32_t *in_idx, int32_t n, int64_t m,
                             int32_t *rows, int32_t *counts, cudaStream_t st);
cudaError_t launch_graph_keys(const int32_t *row_ptr, const int32_t *col_idx,
                              const int32_t *in_ptr, int32_t n, int32_t *nchunks, int64_t *two,
                              unsigned long long *totals, cudaStream_t st);
int max_grid_batch(bool fp64, int device, int words = 1);
int max_grid_plain(bool fp64, int device);

} // namespace bcgpu
