// Host side of the GB300 betweenness-centrality library: the C ABI declared
// in include/bc_gb300.h.
//
//  - graph registry: validation, canonicalisation (sorted rows, no duplicate
//    edges or self-loops), in-CSR construction and chunk counts, one device
//    allocation per graph, resident until destroyed;
//  - workspaces: device state of one in-flight batch, cached and reused; the
//    kernels leave a workspace zeroed, so reuse needs no clearing;
//  - jobs: a source list split into batches of up to 64 (BATCH schedule) or
//    single sources (PLAIN), one cooperative launch each, stream-ordered,
//    followed by one scaling pass and one copy of the float64 result;
//  - scheduler: a host thread that admits submitted jobs when their device
//    footprint fits the HBM budget next to running jobs, launches each on a
//    stream of its own so their kernels overlap, and retires them by event.
#include "bc_internal.cuh"
#include "bc_gb300.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace bcgpu;

namespace {

constexpr int kMaxSlots = 8; // concurrently running submitted jobs

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves typed arrays out of one device allocation.
struct Carver {
  size_t off = 0;
  char *base = nullptr;
  template <typename T> T *take(size_t count) {
    off = align_up(off, 256);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += sizeof(T) * (count ? count : 1);
    return p;
  }
};

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (prev_ != dev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0, dev_ = 0;
};

struct GraphRec {
  int64_t handle = 0;
  GraphDev dev;
  void *mem = nullptr;
  size_t bytes = 0;
  int active_jobs = 0;
  // chunk counts of the high-degree vertices for each candidate chunk size
  const int32_t *nch_variant[kChunkVariants] = {};
  int64_t heavy_v[kChunkVariants] = {}, heavy_c[kChunkVariants] = {};
  // per-graph tuning of the batched kernel, per batch width (1, 2, 4 mask
  // words): chunk variant and grab size (-1: not tuned yet)
  std::atomic<int> tuned[3] = {-1, -1, -1};
  // mask words the width trial found fastest per source (0: not tried yet)
  std::atomic<int> tuned_words{0};
  // concurrent batch groups the groups trial found fastest, per width (0: not tried yet)
  std::atomic<int> tuned_groups[3] = {0, 0, 0};
  // a batch wider than 64 sources overran its frontier queue or heavy list
  // (sized for 64 distinct depths per vertex): later jobs use 64 sources
  std::atomic<bool> narrow{false};
  // a pushed path count was 2^32 or more: later jobs pull every level
  std::atomic<bool> no_push{false};
  // a path count reached 2^32: later jobs store counts in 64 bits
  std::atomic<bool> wide_counts{false};
  // batch composition (see order_key): host copies of the out-CSR
  // offsets and of the two-hop walk counts; every vertex in batch order, made
  // on first need (kept on the host and in d_order)
  std::vector<int32_t> row_ptr;
  std::vector<int64_t> two;
  std::vector<int32_t> order;
  int32_t *d_order = nullptr;
  std::mutex order_mu;
  uint64_t fingerprint = 0; // of the CSR as given (0: tuning not remembered, see TuneMemo)
  std::atomic<int32_t> with_out{-1}; // vertices with out-edges (-1: not counted yet)
};

// Tuning results of a graph, remembered by its context beyond the graph's
// destruction and keyed by a fingerprint of the CSR as given (n, m and evenly
// spaced samples of the offsets and column ids): a graph created again (a
// service reloading it, or a benchmark's fresh copies) starts with the width,
// split and group choices and the fallbacks (64-source batches, pulled
// counts, 64-bit counts) that its earlier copies found, instead of running
// the timed trials again.  Every choice computes the same BC, so a different
// graph with the same fingerprint only inherits launch choices.  Kept for
// graphs of kTuneMemoMinEdges edges or more, where the trials cost the most.
struct TuneMemo {
  int tuned[3];
  int tuned_words;
  int tuned_groups[3];
  bool narrow, no_push, wide_counts;
};
constexpr int64_t kTuneMemoMinEdges = 1 << 18;
constexpr size_t kTuneMemoMax = 4096; // entries (the memo is cleared when full)

uint64_t memo_mix(uint64_t h, uint64_t v) {
  // splitmix64 finaliser over the running hash and the next value
  uint64_t z = h ^ (v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2));
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

uint64_t graph_fingerprint(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int64_t m) {
  constexpr int kSamples = 512;
  uint64_t h = memo_mix(memo_mix(0x6a09e667f3bcc908ull, (uint64_t)n), (uint64_t)m);
  for (int i = 0; i <= kSamples; ++i) {
    h = memo_mix(h, (uint64_t)(uint32_t)row_ptr[(int64_t)n * i / kSamples]);
    if (m > 0 && i < kSamples) h = memo_mix(h, (uint64_t)(uint32_t)col_idx[m * i / kSamples]);
  }
  return h ? h : 1;
}

// Batch composition order of the vertices as sources.  A batch advances
// the union of its sources' frontiers, so its cost grows with the (vertex,
// level) entries and edge scans of that union; sources whose traversals
// reach the same vertices at the same depths share them.  The key: sources
// without out-edges (a traversal of one vertex) last, the others by the
// number of two-hop walks leaving them (a proxy for how fast the traversal
// fans out into the graph's core), descending; ties by out-degree, then
// vertex id.  Packed as two words compared in turn (smaller first): the
// no-out-edge flag and the descending two-hop count, then the descending
// out-degree and the id.
struct OrderKey {
  uint64_t hi, lo;
  bool operator<(const OrderKey &o) const { return hi != o.hi ? hi < o.hi : lo < o.lo; }
};
inline OrderKey order_key(const std::vector<int32_t> &row_ptr, const std::vector<int64_t> &two,
                          int32_t v) {
  const int32_t d = row_ptr[(size_t)v + 1] - row_ptr[(size_t)v];
  const uint64_t t = (uint64_t)std::max<int64_t>(two[(size_t)v], 0); // < 2^63
  return {(d == 0 ? 1ull << 63 : 0ull) | ((uint64_t)INT64_MAX - t),
          ((uint64_t)(uint32_t)(INT32_MAX - d) << 32) | (uint32_t)v};
}

// Every vertex in batch order (order_key): packed keys sorted in
// chunks on up to eight threads, then merged pairwise.
std::vector<int32_t> batch_order(const std::vector<int32_t> &row_ptr,
                                 const std::vector<int64_t> &two, int32_t n) {
  std::vector<OrderKey> keys((size_t)n);
  for (int32_t v = 0; v < n; ++v) keys[(size_t)v] = order_key(row_ptr, two, v);
  const int chunks = (int)std::min<int64_t>(8, std::max<int64_t>(1, n / 8192));
  std::vector<size_t> cut((size_t)chunks + 1);
  for (int c = 0; c <= chunks; ++c) cut[(size_t)c] = (size_t)n * (size_t)c / (size_t)chunks;
  auto run = [](int count, const std::function<void(int)> &f) {
    std::vector<std::thread> th;
    for (int i = 1; i < count; ++i) th.emplace_back(f, i);
    f(0);
    for (auto &t : th) t.join();
  };
  run(chunks, [&](int c) {
    std::sort(keys.begin() + (ptrdiff_t)cut[(size_t)c], keys.begin() + (ptrdiff_t)cut[(size_t)c + 1]);
  });
  for (int width = 1; width < chunks; width *= 2) {
    const int pairs = (chunks + 2 * width - 1) / (2 * width);
    run(pairs, [&](int p_) {
      const int c0 = 2 * width * p_;
      const int c1 = std::min(c0 + width, chunks), c2 = std::min(c0 + 2 * width, chunks);
      if (c1 < c2)
        std::inplace_merge(keys.begin() + (ptrdiff_t)cut[(size_t)c0],
                           keys.begin() + (ptrdiff_t)cut[(size_t)c1],
                           keys.begin() + (ptrdiff_t)cut[(size_t)c2]);
    });
  }
  std::vector<int32_t> ord((size_t)n);
  for (int32_t i = 0; i < n; ++i) ord[(size_t)i] = (int32_t)(uint32_t)keys[(size_t)i].lo;
  return ord;
}

// Graphs up to this many vertices get their batch order at creation.
constexpr int32_t kEagerOrderN = 1 << 16;

// Launch configurations the tuner compares: (work split, items per fetch).
// The splits are kChunkCandidates: warp-centric with 256-edge chunks of hubs
// (the default), edge-centric leaning 128-edge chunks, coarser 512-edge
// chunks, vertex-centric (no split); the fourth candidate takes one item per
// counter fetch instead of two.
struct TuneCandidate {
  int variant;
  int grab;
};
constexpr TuneCandidate kTuneCandidates[] = {
    {kSplitWarp, 2}, {kSplitEdge, 2}, {kSplitWarp512, 2}, {kSplitWarp, 1}, {kSplitVertex, 2}};
constexpr bool grabs_fit() {
  for (const TuneCandidate &c : kTuneCandidates)
    if (c.grab < 1 || c.grab > kGrabMax) return false;
  return kGrabDefault <= kGrabMax;
}
static_assert(grabs_fit(), "a fetch larger than the kernels' header rounds hold");
constexpr int kNumTune = 5;
constexpr int kTuneRounds = 2; // trial batches per candidate
constexpr double kTuneMargin = 1.05; // throughput a split must beat the default by
// Batch widths (mask words) the width trial compares, widest first.
constexpr int kWidthTrial[3] = {4, 2, 1};

enum WsKind { WS_PLAIN = 0, WS_QUEUE = 1 };

struct WsRec {
  bool batch = true;
  int kind = WS_QUEUE;
  int words = 1; // 64-bit words per source mask (queue kernel: 1, 2 or 4)
  int slots = 1; // plain, one block per source: copies for concurrent launches
  int32_t n = 0;
  int64_t cap = 0, hcap = 0, chunk_cap = 0;
  Work w;                   // the workspace (slot 0)
  size_t slot_bytes = 0;    // stride between slot copies
  double *parts = nullptr;  // slots > 1: [slots][n] BC partial sums, one per slot
  KParams *slot_params = nullptr; // slots > 1: [slots] launch parameters, rewritten per job
  // slots > 1: the one-block launches of a job of plain_k sources on plain_s
  // streams, captured once as a CUDA graph (the launches read everything that
  // changes between jobs from slot_params)
  cudaGraphExec_t plain_exec = nullptr;
  int64_t plain_k = 0;
  int plain_s = 0;
  bool plain_fp64 = false;
  void *mem = nullptr;
  size_t bytes = 0;
  bool dirty = false;
};

struct WsNeed {
  int kind;
  int words;
  int slots;
  int32_t n;
  int64_t cap, hcap, chunk_cap;
  bool fits(const WsRec &r) const {
    if (r.kind != kind || r.words != words || r.slots < slots || r.n < n || r.hcap < hcap ||
        r.chunk_cap < chunk_cap)
      return false;
    return r.cap >= cap;
  }
};

// Sources per batch and mask words of a job.  Explicit batch_k: that many
// sources, in as many words as they need.  Automatic: the queue kernel takes
// 64 sources per mask word and the widest batch (up to 256 sources) that
// still gives the job kWideMinBatches batches; wider batches share each
// (vertex, level) entry and edge scan among more sources.  Debug exports and
// graphs that overran a wide batch's queue use 64.
struct BatchShape {
  int kb;
  int words;
};
BatchShape batch_shape(const bc_opts &o, int kind, int64_t k, bool narrow, bool dbg) {
  if (kind == WS_PLAIN) return {1, 1};
  if (narrow && kind == WS_QUEUE) return {o.batch_k > 0 && o.batch_k < kK ? o.batch_k : kK, 1};
  if (o.batch_k > 0) return {o.batch_k, o.batch_k <= kK ? 1 : o.batch_k <= 2 * kK ? 2 : 4};
  const int w = kind == WS_QUEUE && !narrow && !dbg ? auto_words(k, kMaxWords) : 1;
  return {kK * w, w};
}

int word_index(int words) { return words == 1 ? 0 : words == 2 ? 1 : 2; }

WsNeed ws_need(const GraphDev &g, int kind, int kb, int words, int slots = 1) {
  WsNeed nd;
  nd.kind = kind;
  nd.words = kind == WS_QUEUE ? words : 1;
  nd.slots = slots;
  nd.n = g.n;
  // a vertex is queued at most once per distinct depth among the batch's
  // sources; wider batches are sized for 64 depths (overruns are detected)
  const int64_t kk = kind == WS_PLAIN ? 1 : std::min<int64_t>(kb, kK);
  nd.cap = std::max<int64_t>(1, (int64_t)g.n * kk);
  nd.hcap = std::max<int64_t>(1, g.heavy_vertices * kk);
  nd.chunk_cap = std::max<int64_t>(1, g.heavy_chunks);
  return nd;
}

// Lays out (mem == nullptr: only sizes) the arrays of one workspace copy.
size_t ws_layout_one(WsRec &r, char *mem) {
  Carver c;
  c.base = mem;
  const size_t n = (size_t)r.n;
  const size_t words = r.batch ? (size_t)r.words : 1;
  const size_t kk = r.batch ? kK * words : 1;
  Work &w = r.w;
  w = Work();
  w.n = r.n;
  w.k_max = (int32_t)kk;
  w.words = (int32_t)words;
  w.ctl = c.take<Ctl>(1);
  if (r.batch) {
    w.vis = c.take<uint64_t>(n * words);
    w.fr = c.take<uint64_t>(4 * n * words);
    w.qm = c.take<uint64_t>((size_t)r.cap * words);
    w.claim = words > 1 ? c.take<int32_t>(n) : nullptr;
    w.lsum = c.take<unsigned long long>(2 * (n + 3));
    w.d = nullptr;
  } else {
    w.d = c.take<int32_t>(n);
    w.vis = nullptr;
    w.fr = nullptr;
    w.qm = nullptr;
  }
  w.qv = c.take<int32_t>((size_t)r.cap);
  w.cap = r.cap;
  w.qoff = c.take<int64_t>(n + 3);
  w.hpack = c.take<unsigned long long>(n + 3);
  w.hoff = c.take<int64_t>(n + 3);
  w.hq_e = c.take<int64_t>((size_t)r.hcap);
  w.hq_c = c.take<int64_t>((size_t)r.hcap);
  w.harrive = c.take<unsigned>((size_t)r.hcap);
  w.hcap = r.hcap;
  w.partial = c.take<uint64_t>((size_t)r.chunk_cap * kk);
  w.partial_ovf = c.take<uint64_t>((size_t)r.chunk_cap * words);
  w.chunk_cap = r.chunk_cap;
  w.sigma = c.take<uint64_t>(n * kk);
  w.cdep = c.take<double>(n * kk);
  return align_up(c.off, 256);
}

// Lays out a workspace: one copy, or for the one-block plain form `slots`
// copies back to back and then one BC partial vector per copy.
size_t ws_layout(WsRec &r, char *mem) {
  const size_t one = ws_layout_one(r, mem);
  if (r.slots <= 1) {
    r.slot_bytes = one;
    r.parts = nullptr;
    return one;
  }
  r.slot_bytes = one;
  const size_t parts_at = one * (size_t)r.slots;
  const size_t params_at = align_up(parts_at + sizeof(double) * (size_t)r.n * (size_t)r.slots, 256);
  r.parts = mem ? reinterpret_cast<double *>(mem + parts_at) : nullptr;
  r.slot_params = mem ? reinterpret_cast<KParams *>(mem + params_at) : nullptr;
  return align_up(params_at + sizeof(KParams) * (size_t)r.slots, 256);
}

// Releases a workspace's device memory and captured launches.
void ws_free(WsRec &r) {
  if (r.plain_exec) cudaGraphExecDestroy(r.plain_exec);
  r.plain_exec = nullptr;
  cudaFree(r.mem);
  r.mem = nullptr;
}

// The workspace copy of slot i (plain, one block per source).
Work slot_work(const WsRec &r, int i) {
  WsRec t = r;
  t.slots = 1;
  ws_layout_one(t, static_cast<char *>(r.mem) + r.slot_bytes * (size_t)i);
  return t.w;
}

// Brings a workspace to its resting state: all masks, counts and arrival
// counters zero, depths -1.
cudaError_t ws_clear(WsRec &r, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(r.mem, 0, r.bytes, st);
  for (int i = 0; i < r.slots && e == cudaSuccess && !r.batch; ++i)
    e = cudaMemsetAsync(slot_work(r, i).d, 0xff, sizeof(int32_t) * r.n, st);
  return e;
}

struct JobRec;

} // namespace

struct bc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  std::atomic<size_t> used{0};
  int sm_count = 0;
  int grid_batch[3][2] = {}; // [mask words 1/2/4][fp64]
  int grid_many[2] = {0, 0};
  int grid_plain[2] = {0, 0};
  // Stream-ordered allocations of this context (graphs, job buffers, prep
  // scratch) come from its own pool, which keeps up to kPoolKeepBytes of
  // freed memory mapped: with the default pool's threshold of 0 every
  // synchronisation returns freed memory to the system and the next
  // allocation maps it again (about 0.1 ms per graph or job).
  cudaMemPool_t pool = nullptr;
  // pinned staging for the single upload of a host-prepared graph
  void *stage = nullptr;
  size_t stage_bytes = 0;
  // pinned host blocks of finished jobs kept for reuse (power-of-two size
  // classes, up to kPinKeepBytes): pinning and unpinning cost tens to
  // hundreds of microseconds per call
  std::mutex pin_mu;
  std::multimap<size_t, void *> pin_free;
  size_t pin_free_bytes = 0;

  std::mutex memo_mu;
  std::unordered_map<uint64_t, TuneMemo> tune_memo; // by graph fingerprint

  std::mutex mu;
  std::unordered_map<int64_t, std::unique_ptr<GraphRec>> graphs;
  int64_t next_graph = 1;
  std::vector<std::unique_ptr<WsRec>> free_ws;

  bc_stats last{};
  std::vector<int32_t> last_ovf; // sources whose path count reached 2^64 in the last call
  // streams (and their events) of the one-block plain launches, made on first use
  std::mutex aux_mu;
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> aux_ev;
  cudaStream_t aux_root = nullptr; // stream the launches are captured on
  int32_t inject_block = -1;
  int32_t inject_timeout_ms = 0;

  // scheduler
  std::thread sched;
  std::condition_variable cv;
  bool stop = false;
  std::deque<JobRec *> pending;
  std::vector<JobRec *> running;
  std::map<int64_t, std::unique_ptr<JobRec>> jobs;
  int64_t next_job = 1;
  cudaStream_t slot_stream[kMaxSlots] = {};
  bool slot_busy[kMaxSlots] = {};
};

namespace {

constexpr uint64_t kPoolKeepBytes = (uint64_t)2 << 30;

constexpr size_t kPinKeepBytes = (size_t)64 << 20;

size_t pin_class(size_t bytes) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  return c;
}

// Pinned host block of at least `bytes`, from the context's cache if one of
// its size class is free.
template <typename T> cudaError_t pin_get(bc_ctx *ctx, T **p, size_t bytes) {
  const size_t cls = pin_class(bytes);
  {
    std::lock_guard<std::mutex> lk(ctx->pin_mu);
    auto it = ctx->pin_free.find(cls);
    if (it != ctx->pin_free.end()) {
      *p = static_cast<T *>(it->second);
      ctx->pin_free.erase(it);
      ctx->pin_free_bytes -= cls;
      return cudaSuccess;
    }
  }
  void *q = nullptr;
  const cudaError_t e = cudaMallocHost(&q, cls);
  *p = static_cast<T *>(q);
  return e;
}

// Returns a block from pin_get (asked for `bytes`) to the cache, or unpins
// it when the cache is full.
void pin_put(bc_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  const size_t cls = pin_class(bytes);
  {
    std::lock_guard<std::mutex> lk(ctx->pin_mu);
    if (ctx->pin_free_bytes + cls <= kPinKeepBytes) {
      ctx->pin_free.emplace(cls, p);
      ctx->pin_free_bytes += cls;
      return;
    }
  }
  cudaFreeHost(p);
}

// Stream-ordered allocation from the context's pool.
template <typename T> cudaError_t pool_alloc(bc_ctx *ctx, T **p, size_t bytes, cudaStream_t st) {
  return cudaMallocFromPoolAsync(reinterpret_cast<void **>(p), bytes, ctx->pool, st);
}

// One BC job: a graph, a source list and options; runs on one stream.
struct JobRec {
  int64_t handle = 0;
  GraphRec *g = nullptr;
  std::vector<int32_t> src; // empty + all_sources: 0..n-1
  bool all_sources = false;
  bc_opts opts{};
  int64_t k = 0;            // number of sources
  // sources the batched kernels traverse: in grouped order the sources
  // without out-edges come last, and their traversal (the source alone)
  // adds nothing to any BC value, so they are not launched
  int64_t k_traverse = 0;
  int64_t n = 0;            // vertices of the graph (result length)
  // run state
  int slot = -1;
  cudaStream_t st = nullptr;
  std::unique_ptr<WsRec> ws;
  int32_t *d_src = nullptr;
  double *d_bc = nullptr;
  double *d_bc2 = nullptr;  // squared per-source terms (estimator jobs)
  double *acc_sum = nullptr, *acc_sumsq = nullptr; // estimator jobs: running sums to add into
  int8_t *d_ovf = nullptr;
  unsigned long long *d_cnt = nullptr;
  KParams *h_slots = nullptr; // one-block plain form: pinned staging of the launch parameters
  int32_t *h_src = nullptr;   // pinned staging
  double *h_out = nullptr;    // pinned result (async jobs)
  unsigned long long *h_cnt = nullptr; // pinned: counters + err + ovf count
  int *h_err = nullptr;
  int8_t *h_ovf = nullptr;
  std::vector<int32_t> ovf_sources; // flagged source ids, ascending (set by job_finish)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evdone = nullptr;
  unsigned long long *d_trace = nullptr; // per-step trace of one batch (BC_TRACE)
  unsigned long long *h_trace = nullptr;
  int64_t trace_batch = -1;
  int64_t launches = 0;
  int64_t batches = 0;
  int kind = 0;              // workspace / kernel kind of the last launch
  int kb = 0;                // sources per batch of the last launch
  int words = 1;             // mask words of the last launch
  int cand = 0;              // tuning candidate of the last launch
  int ws_slots = 0;          // one-block plain form: streams (entries of h_slots)
  int groups = 1;            // concurrent batch groups the job's workspace holds
  int groups_used = 1;       // concurrent batch groups of the job's last batches
  Work *h_works = nullptr;   // grouped batches: pinned staging of the groups' workspaces
  int works_n = 0;           // entries of h_works
  size_t footprint = 0;
  bc_status status = BC_PENDING;
  bc_stats stats{};
  bool done = false;
};

// internal: the job must be launched again (a wide batch overran its queue,
// a count needed 64 bits or a pushed count was too large to push)
constexpr bc_status kStatusRetry = static_cast<bc_status>(100);

bc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BC_OK;
  if (e == cudaErrorMemoryAllocation) return BC_ERR_OOM;
  return BC_ERR_CUDA;
}

#define BC_TRY(expr)                                \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return cuda_status(_e);  \
  } while (0)

bc_opts default_opts() {
  bc_opts o;
  std::memset(&o, 0, sizeof(o));
  return o;
}

bool opts_valid(const bc_opts &o) {
  return (o.delta_fp64 == 0 || o.delta_fp64 == 1) && o.batch_k >= 0 &&
         o.batch_k <= kK * kMaxWords &&
         (o.batch_k <= kK || o.schedule != BC_SCHED_PLAIN) &&
         o.schedule >= BC_SCHED_AUTO && o.schedule <= BC_SCHED_BATCH_EDGE &&
         (o.normalize == 0 || o.normalize == 1) &&
         (o.scale_sampled == 0 || o.scale_sampled == 1) &&
         (o.out_device == 0 || o.out_device == 1) &&
         (o.source_order == 0 || o.source_order == 1) &&
         (o.direction >= 0 && o.direction <= 2) &&
         (o.count_bits == 0 || o.count_bits == 32 || o.count_bits == 64);
}

int resolve_schedule(const bc_opts &o, const GraphDev &) {
  if (o.schedule != BC_SCHED_AUTO) return o.schedule;
  return BC_SCHED_BATCH;
}

// Work split a batched schedule fixes (-1: tuned per graph).
int fixed_split(int sched) {
  return sched == BC_SCHED_BATCH_VERTEX ? kSplitVertex
         : sched == BC_SCHED_BATCH_WARP ? kSplitWarp
         : sched == BC_SCHED_BATCH_EDGE ? kSplitEdge
                                        : -1;
}


// Direction rule of the forward path-count step (KParams::push_ratio): by
// default a level pushes from the previous level when that scans at least
// kPushRatio times fewer edges than pulling (BC_PUSH_RATIO overrides it for
// experiments); bc_opts.direction forces either form.
constexpr int kPushRatio = 8;
int push_ratio(const bc_opts &o, const GraphRec &g) {
  if (o.direction == 1 || g.no_push) return 0;
  if (o.direction == 2) return -1;
  if (const char *env = std::getenv("BC_PUSH_RATIO")) return std::atoi(env);
  return kPushRatio;
}

// Grid of a persistent launch: the co-resident maximum for large graphs, a
// smaller share of the GPU for small ones so that concurrent jobs overlap.
int pick_grid(const bc_ctx *ctx, const GraphDev &g, int kind, bool fp64, int words) {
  const int gmax =
      kind == WS_QUEUE ? ctx->grid_batch[word_index(words)][fp64] : ctx->grid_plain[fp64];
  if (const char *env = std::getenv("BC_GRID")) {
    int v = std::atoi(env);
    if (v > 0) return std::min(v, gmax);
  }
  // about eight threads per vertex, at least two CTAs (graphs of 16K+
  // vertices take every SM)
  const int64_t want = std::max<int64_t>(2, ((int64_t)g.n * 8 + kBlock - 1) / kBlock);
  return (int)std::min<int64_t>(gmax, want);
}

// ---- graphs -----------------------------------------------------------------

// Makes the graph's batch order (host and device copies) if it has none yet.
bc_status ensure_order(GraphRec *g, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g->order_mu);
  const int32_t n = g->dev.n;
  if (!g->order.empty() || n == 0) return BC_OK;
  g->order = batch_order(g->row_ptr, g->two, n);
  // the source stays alive with the graph, which outlives the copy (it is
  // freed on the context's stream, and never while a job uses it)
  BC_TRY(cudaMemcpyAsync(g->d_order, g->order.data(), sizeof(int32_t) * (size_t)n,
                         cudaMemcpyHostToDevice, st));
  return BC_OK;
}

// Graphs up to this many edges are prepared on the host: a few microseconds
// of host work and one upload beat the device path's launches and
// synchronisations (many small graphs are created one after another).
constexpr int64_t kHostPrepMaxEdges = (int64_t)1 << 18;

// A graph prepared on the host (offsets already checked): validated,
// canonicalised, in-CSR by counting sort, chunk counts, two-hop keys and the
// batch order.  Touches no CUDA state, so several run at once.
struct HostPrep {
  int32_t n = 0;
  int64_t me = 0;
  size_t bytes = 0;                  // device block size
  std::vector<int32_t> crp, cci;     // canonical CSR when the input was not canonical
  const int32_t *rp = nullptr, *ci = nullptr;
  std::vector<int32_t> ip, ii, nc, ord;
  std::vector<int64_t> two;
  int64_t heavy_v[kChunkVariants] = {}, heavy_c[kChunkVariants] = {}, hv = 0, hc = 0;
};

// The device block of a graph: offsets of its arrays (Carver order).
template <typename F> void block_layout(int32_t n, int64_t me, F &&take) {
  take((size_t)n + 1);             // row_ptr
  take((size_t)me);                // col_idx
  take((size_t)n + 1);             // in_ptr
  take((size_t)me);                // in_idx
  take((size_t)n * kChunkVariants); // nchunks
  take((size_t)n);                 // order
}

bc_status prep_host(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int64_t m,
                    HostPrep &h) {
  bool canonical = true;
  for (int32_t v = 0; v < n; ++v)
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      const int32_t x = col_idx[e];
      if (x < 0 || x >= n) return BC_ERR_GRAPH;
      if (x == v || (e > row_ptr[v] && x <= col_idx[e - 1])) canonical = false;
    }
  h.n = n;
  h.rp = row_ptr;
  h.ci = col_idx;
  if (!canonical) {
    h.crp.resize((size_t)n + 1);
    h.cci.reserve((size_t)m);
    h.crp[0] = 0;
    std::vector<int32_t> row;
    for (int32_t v = 0; v < n; ++v) {
      row.assign(col_idx + row_ptr[v], col_idx + row_ptr[v + 1]);
      std::sort(row.begin(), row.end());
      int32_t prev = -1;
      for (int32_t x : row)
        if (x != v && x != prev) {
          h.cci.push_back(x);
          prev = x;
        }
      h.crp[(size_t)v + 1] = (int32_t)h.cci.size();
    }
    h.rp = h.crp.data();
    h.ci = h.cci.data();
  }
  const int32_t *rp = h.rp, *ci = h.ci;
  const int64_t me = (int64_t)rp[n];
  h.me = me;
  // in-CSR by counting sort over destinations (sources stay ascending)
  h.ip.assign((size_t)n + 1, 0);
  h.ii.resize((size_t)std::max<int64_t>(me, 1));
  for (int64_t e = 0; e < me; ++e) h.ip[(size_t)ci[e] + 1]++;
  for (int32_t v = 0; v < n; ++v) h.ip[(size_t)v + 1] += h.ip[v];
  {
    std::vector<int32_t> fill(h.ip.begin(), h.ip.end() - 1);
    for (int32_t v = 0; v < n; ++v)
      for (int32_t e = rp[v]; e < rp[(size_t)v + 1]; ++e) h.ii[(size_t)fill[ci[e]]++] = v;
  }
  h.nc.assign((size_t)n * kChunkVariants, 0);
  for (int c = 0; c < kChunkVariants; ++c) {
    const int64_t ch = kChunkCandidates[c];
    for (int32_t v = 0; v < n; ++v) {
      const int64_t cost = (int64_t)(rp[(size_t)v + 1] - rp[v]) + (h.ip[(size_t)v + 1] - h.ip[v]);
      if (cost > heavy_threshold(ch)) {
        const int32_t k = (int32_t)((cost + ch - 1) / ch);
        h.nc[(size_t)c * n + v] = k;
        h.heavy_v[c]++;
        h.heavy_c[c] += k;
      }
    }
    h.hv = std::max(h.hv, h.heavy_v[c]);
    h.hc = std::max(h.hc, h.heavy_c[c]);
  }
  h.two.assign((size_t)n, 0);
  for (int32_t v = 0; v < n; ++v) {
    int64_t t = 0;
    for (int32_t e = rp[v]; e < rp[(size_t)v + 1]; ++e) t += rp[(size_t)ci[e] + 1] - rp[ci[e]];
    h.two[(size_t)v] = t;
  }
  {
    std::vector<int32_t> rpv(rp, rp + (size_t)n + 1);
    h.ord = batch_order(rpv, h.two, n);
  }
  Carver c;
  block_layout(n, me, [&](size_t cnt) { (void)c.take<int32_t>(cnt); });
  h.bytes = align_up(c.off, 256);
  return BC_OK;
}

// Writes the device image of a prepared graph (its arrays at their block
// offsets) to dst, which holds h.bytes.
void prep_image(const HostPrep &h, char *dst) {
  Carver c;
  c.base = dst;
  const int32_t *src[6] = {h.rp, h.ci, h.ip.data(), h.ii.data(), h.nc.data(), h.ord.data()};
  int a = 0;
  block_layout(h.n, h.me, [&](size_t cnt) {
    int32_t *d = c.take<int32_t>(cnt);
    const size_t real = a == 1 || a == 3 ? (size_t)h.me : cnt; // edge arrays may be empty
    if (real) std::memcpy(d, src[a], sizeof(int32_t) * real);
    ++a;
  });
}

// The resident graph of a prepared one whose image was copied to mem.
std::unique_ptr<GraphRec> prep_graph(HostPrep &h, void *mem) {
  auto g = std::make_unique<GraphRec>();
  int32_t *ptr[6];
  Carver c;
  c.base = static_cast<char *>(mem);
  int a = 0;
  block_layout(h.n, h.me, [&](size_t cnt) { ptr[a++] = c.take<int32_t>(cnt); });
  const int32_t n = h.n;
  for (int v = 0; v < kChunkVariants; ++v) {
    g->heavy_v[v] = h.heavy_v[v];
    g->heavy_c[v] = h.heavy_c[v];
    g->nch_variant[v] = ptr[4] + (size_t)v * n;
  }
  g->row_ptr.assign(h.rp, h.rp + (size_t)n + 1);
  g->two = std::move(h.two);
  g->mem = mem;
  g->bytes = h.bytes;
  g->dev.n = n;
  g->dev.m = h.me;
  g->dev.row_ptr = ptr[0];
  g->dev.col_idx = ptr[1];
  g->dev.in_ptr = ptr[2];
  g->dev.in_idx = ptr[3];
  g->dev.nchunks = ptr[4];
  g->dev.heavy_vertices = h.hv;
  g->dev.heavy_chunks = h.hc;
  g->dev.order = ptr[5];
  g->d_order = ptr[5];
  g->order = std::move(h.ord);
  return g;
}

// Room for `bytes` in the context's pinned staging buffer.
bc_status ensure_stage(bc_ctx *ctx, size_t bytes) {
  if (ctx->stage_bytes >= bytes) return BC_OK;
  if (ctx->stage) cudaFreeHost(ctx->stage);
  ctx->stage = nullptr;
  ctx->stage_bytes = 0;
  const size_t want = std::max<size_t>(bytes, (size_t)1 << 20);
  BC_TRY(cudaMallocHost(&ctx->stage, want));
  ctx->stage_bytes = want;
  return BC_OK;
}

// Host preparation of a small graph, then one upload of its image from the
// pinned staging buffer.
bc_status build_graph_small(bc_ctx *ctx, const int32_t *row_ptr, const int32_t *col_idx,
                            int32_t n, int64_t m, std::unique_ptr<GraphRec> &out,
                            int64_t *m_eff) {
  HostPrep h;
  bc_status s = prep_host(row_ptr, col_idx, n, m, h);
  if (s != BC_OK) return s;
  if (ctx->used + h.bytes > ctx->budget) return BC_ERR_ADMISSION;
  s = ensure_stage(ctx, h.bytes);
  if (s != BC_OK) return s;
  prep_image(h, static_cast<char *>(ctx->stage));
  cudaStream_t st = ctx->stream;
  void *mem = nullptr;
  BC_TRY(pool_alloc(ctx, &mem, h.bytes, st));
  cudaError_t e = cudaMemcpyAsync(mem, ctx->stage, h.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, st);
    return cuda_status(e);
  }
  if (m_eff) *m_eff = h.me;
  ctx->used += h.bytes;
  out = prep_graph(h, mem);
  return BC_OK;
}

// Host checks of a CSR's sizes and offsets (column ids are checked where the
// graph is prepared).
bc_status check_offsets(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int64_t m) {
  if (n < 0 || m < 0 || m >= ((int64_t)1 << 31)) return BC_ERR_GRAPH;
  if (!row_ptr || (m > 0 && !col_idx)) return BC_ERR_ARG;
  if (row_ptr[0] != 0 || (int64_t)row_ptr[n] != m) return BC_ERR_GRAPH;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return BC_ERR_GRAPH;
  return BC_OK;
}

bc_status build_graph(bc_ctx *ctx, const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                      int64_t m, std::unique_ptr<GraphRec> &out, int64_t *m_eff) {
  const bc_status chk = check_offsets(row_ptr, col_idx, n, m);
  if (chk != BC_OK) return chk;
  if (m <= kHostPrepMaxEdges) return build_graph_small(ctx, row_ptr, col_idx, n, m, out, m_eff);
  cudaStream_t st = ctx->stream;
  // BC_PREP_TRACE=1: per-phase times of the preparation to stderr (each mark
  // synchronises the stream, so the traced run is slower than a plain one)
  const bool trace = std::getenv("BC_PREP_TRACE") != nullptr;
  const auto t_start = std::chrono::steady_clock::now();
  auto mark = [&](const char *what) {
    if (!trace) return;
    cudaStreamSynchronize(st);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                                 t_start).count();
    std::fprintf(stderr, "# graph prep n=%d m=%lld: %-28s %8.3f ms\n", n, (long long)m, what, ms);
  };
  mark("host offsets checked");
  // The graph's device block, laid out for `me` canonical edges.
  struct Block {
    void *mem = nullptr;
    size_t bytes = 0;
    int32_t *rp = nullptr, *ci = nullptr, *ip = nullptr, *ii = nullptr, *nc = nullptr,
            *ord = nullptr;
  };
  auto carve = [n](Block &b, int64_t me, char *base) {
    Carver c;
    c.base = base;
    b.rp = c.take<int32_t>((size_t)n + 1);
    b.ci = c.take<int32_t>((size_t)me);
    b.ip = c.take<int32_t>((size_t)n + 1);
    b.ii = c.take<int32_t>((size_t)me);
    b.nc = c.take<int32_t>((size_t)n * kChunkVariants);
    b.ord = c.take<int32_t>((size_t)n);
    b.bytes = align_up(c.off, 256);
  };
  auto alloc_upload = [&](Block &b, const int32_t *rp, const int32_t *ci, int64_t me) -> bc_status {
    carve(b, me, nullptr);
    if (ctx->used + b.bytes > ctx->budget) return BC_ERR_ADMISSION;
    BC_TRY(pool_alloc(ctx, &b.mem, b.bytes, st));
    carve(b, me, static_cast<char *>(b.mem));
    cudaError_t r = cudaMemcpyAsync(b.rp, rp, sizeof(int32_t) * ((size_t)n + 1),
                                    cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess && me)
      r = cudaMemcpyAsync(b.ci, ci, sizeof(int32_t) * (size_t)me, cudaMemcpyHostToDevice, st);
    if (r != cudaSuccess) {
      cudaFreeAsync(b.mem, st);
      b.mem = nullptr;
      return cuda_status(r);
    }
    return BC_OK;
  };
  // The whole device pipeline on the uploaded block, read back with one
  // synchronisation: validation flags (id out of range, row not canonical),
  // in-degrees -> scan -> in-CSR scatter, row sorts, chunk counts and totals,
  // two-hop keys.  Every kernel skips out-of-range ids, so a bad graph is only
  // reported.
  auto prepare = [&](Block &b, int64_t me, int (&flags)[2], std::vector<int64_t> &two,
                     unsigned long long (&totals)[2 * kChunkVariants]) -> cudaError_t {
    int *d_flags = nullptr;
    int32_t *d_fill = nullptr, *d_rows = nullptr, *d_scan = nullptr;
    int64_t *d_two = nullptr;
    unsigned long long *d_tot = nullptr;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t r) {
      if (e == cudaSuccess) e = r;
    };
    step(pool_alloc(ctx, &d_flags, sizeof(int) * 2 + 3 * sizeof(int32_t), st));
    step(pool_alloc(ctx, &d_fill, sizeof(int32_t) * ((size_t)n + 1), st));
    step(pool_alloc(ctx, &d_rows, sizeof(int32_t) * 3 * (size_t)n, st));
    step(pool_alloc(ctx, &d_two, sizeof(int64_t) * (size_t)n, st));
    step(pool_alloc(ctx, &d_tot, sizeof(totals), st));
    step(pool_alloc(ctx, &d_scan, sizeof(int32_t) * (size_t)scan_scratch_elems((int64_t)n + 1), st));
    if (e == cudaSuccess) {
      int32_t *d_rcnt = reinterpret_cast<int32_t *>(d_flags + 2);
      step(cudaMemsetAsync(d_flags, 0, sizeof(int) * 2, st));
      step(cudaMemsetAsync(d_tot, 0, sizeof(totals), st));
      step(launch_check_csr(b.rp, b.ci, n, d_flags, st));
      step(cudaMemsetAsync(b.ip, 0, sizeof(int32_t) * ((size_t)n + 1), st));
      step(launch_in_degree(b.ci, me, n, b.ip, st));
      mark("checked, in-degrees counted");
      step(launch_scan_inclusive(b.ip, (int64_t)n + 1, d_scan, st));
      step(cudaMemcpyAsync(d_fill, b.ip, sizeof(int32_t) * ((size_t)n + 1),
                           cudaMemcpyDeviceToDevice, st));
      mark("in-degrees scanned");
      step(launch_in_scatter(b.rp, b.ci, n, d_fill, b.ii, st));
      mark("in-edges scattered");
      step(launch_graph_keys(b.rp, b.ci, b.ip, n, b.nc, d_two, d_tot, st));
      mark("chunk counts and keys");
      // in-rows back in ascending source order (the scatter's atomics left
      // them in arbitrary order)
      step(launch_sort_rows(b.ip, b.ii, n, me, d_rows, d_rcnt, st));
      mark("in-rows sorted");
      step(cudaMemcpyAsync(flags, d_flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
      step(cudaMemcpyAsync(two.data(), d_two, sizeof(int64_t) * (size_t)n,
                           cudaMemcpyDeviceToHost, st));
      step(cudaMemcpyAsync(totals, d_tot, sizeof(totals), cudaMemcpyDeviceToHost, st));
    }
    if (d_flags) cudaFreeAsync(d_flags, st);
    if (d_fill) cudaFreeAsync(d_fill, st);
    if (d_rows) cudaFreeAsync(d_rows, st);
    if (d_two) cudaFreeAsync(d_two, st);
    if (d_tot) cudaFreeAsync(d_tot, st);
    if (d_scan) cudaFreeAsync(d_scan, st);
    step(cudaStreamSynchronize(st));
    mark("flags, keys and totals read");
    return e;
  };
  auto g = std::make_unique<GraphRec>();
  g->two.assign((size_t)n, 0);
  unsigned long long totals[2 * kChunkVariants] = {};
  Block blk;
  bc_status bs = alloc_upload(blk, row_ptr, col_idx, m);
  if (bs != BC_OK) return bs;
  mark("uploaded");
  int flags_h[2] = {0, 0};
  {
    const cudaError_t r = prepare(blk, m, flags_h, g->two, totals);
    if (r != cudaSuccess) {
      cudaFreeAsync(blk.mem, st);
      return cuda_status(r);
    }
  }
  if (flags_h[0]) {
    cudaFreeAsync(blk.mem, st);
    return BC_ERR_GRAPH;
  }
  // canonical out-CSR: the caller's arrays as they are, else sorted,
  // de-duplicated rows without self-loops (made on the host, uploaded and
  // prepared again)
  std::vector<int32_t> crp, cci;
  const int32_t *rp = row_ptr;
  if (flags_h[1]) {
    cudaFreeAsync(blk.mem, st);
    crp.resize((size_t)n + 1);
    cci.reserve((size_t)m);
    crp[0] = 0;
    std::vector<int32_t> row;
    for (int32_t v = 0; v < n; ++v) {
      row.assign(col_idx + row_ptr[v], col_idx + row_ptr[v + 1]);
      std::sort(row.begin(), row.end());
      int32_t prev = -1;
      for (int32_t x : row)
        if (x != v && x != prev) {
          cci.push_back(x);
          prev = x;
        }
      crp[(size_t)v + 1] = (int32_t)cci.size();
    }
    rp = crp.data();
    blk = Block();
    bs = alloc_upload(blk, rp, cci.data(), (int64_t)crp[n]);
    if (bs != BC_OK) return bs;
    int again[2] = {0, 0};
    const cudaError_t r = prepare(blk, (int64_t)crp[n], again, g->two, totals);
    if (r != cudaSuccess) {
      cudaFreeAsync(blk.mem, st);
      return cuda_status(r);
    }
  }
  const int64_t me = (int64_t)rp[n];
  void *mem = blk.mem;
  const size_t bytes = blk.bytes;
  int32_t *d_rp = blk.rp, *d_ci = blk.ci, *d_ip = blk.ip, *d_ii = blk.ii, *d_nc = blk.nc,
          *d_ord = blk.ord;
  g->row_ptr.assign(rp, rp + (size_t)n + 1);
  int64_t hv = 0, hc = 0; // maxima over the variants (workspace sizing)
  for (int v = 0; v < kChunkVariants; ++v) {
    g->heavy_v[v] = (int64_t)totals[2 * v];
    g->heavy_c[v] = (int64_t)totals[2 * v + 1];
    hv = std::max(hv, g->heavy_v[v]);
    hc = std::max(hc, g->heavy_c[v]);
    g->nch_variant[v] = d_nc + (size_t)v * n;
  }
  g->mem = mem;
  g->bytes = bytes;
  g->dev.n = n;
  g->dev.m = me;
  g->dev.row_ptr = d_rp;
  g->dev.col_idx = d_ci;
  g->dev.in_ptr = d_ip;
  g->dev.in_idx = d_ii;
  g->dev.nchunks = d_nc; // variant 0 until tuned
  g->dev.heavy_vertices = hv;
  g->dev.heavy_chunks = hc;
  g->dev.order = d_ord;
  g->d_order = d_ord;
  // small graphs (the many-graph launch reads the order on the device) get
  // their batch order now; larger ones on their first exact job
  if (n <= kEagerOrderN) {
    const bc_status so = ensure_order(g.get(), st);
    if (so != BC_OK) {
      cudaFreeAsync(mem, st);
      return so;
    }
  }
  mark("done");
  ctx->used += bytes;
  if (m_eff) *m_eff = me;
  out = std::move(g);
  return BC_OK;
}

GraphRec *find_graph(bc_ctx *ctx, bc_graph h) {
  auto it = ctx->graphs.find(h);
  return it == ctx->graphs.end() ? nullptr : it->second.get();
}

// ---- workspaces -------------------------------------------------------------

bc_status ws_acquire(bc_ctx *ctx, const WsNeed &nd, cudaStream_t st, std::unique_ptr<WsRec> &out) {
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (size_t i = 0; i < ctx->free_ws.size(); ++i)
      if (nd.fits(*ctx->free_ws[i])) {
        out = std::move(ctx->free_ws[i]);
        ctx->free_ws.erase(ctx->free_ws.begin() + (ptrdiff_t)i);
        break;
      }
  }
  if (out) {
    if (out->dirty) {
      BC_TRY(ws_clear(*out, st));
      out->dirty = false;
    }
    return BC_OK;
  }
  auto r = std::make_unique<WsRec>();
  r->kind = nd.kind;
  r->words = nd.words;
  r->slots = nd.slots;
  r->batch = nd.kind != WS_PLAIN;
  r->n = nd.n;
  r->cap = nd.cap;
  r->hcap = nd.hcap;
  r->chunk_cap = nd.chunk_cap;
  r->bytes = ws_layout(*r, nullptr);
  // make room: drop cached workspaces until the new one fits the budget
  while (ctx->used + r->bytes > ctx->budget) {
    std::unique_ptr<WsRec> victim;
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      if (ctx->free_ws.empty()) break;
      victim = std::move(ctx->free_ws.back());
      ctx->free_ws.pop_back();
    }
    ws_free(*victim);
    ctx->used -= victim->bytes;
  }
  if (ctx->used + r->bytes > ctx->budget) return BC_ERR_ADMISSION;
  void *mem = nullptr;
  BC_TRY(cudaMalloc(&mem, r->bytes));
  r->mem = mem;
  ws_layout(*r, static_cast<char *>(mem));
  ctx->used += r->bytes;
  cudaError_t e = ws_clear(*r, st);
  if (e != cudaSuccess) {
    cudaFree(mem);
    ctx->used -= r->bytes;
    return cuda_status(e);
  }
  out = std::move(r);
  return BC_OK;
}

void ws_release(bc_ctx *ctx, std::unique_ptr<WsRec> ws) {
  if (!ws) return;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->free_ws.push_back(std::move(ws));
}

// ---- jobs -------------------------------------------------------------------

// The one-source-per-launch schedule on small graphs: each source is a
// one-block launch (block barriers between levels) instead of a launch over
// the whole GPU, whose grid barriers dominate when a level holds a few
// hundred vertices; launches go round-robin to this many streams, so that
// many sources run at once, each stream adding into its own BC partial
// vector (summed in stream order at the end).
constexpr int32_t kPlainBlockMaxN = 1 << 16;
constexpr int kPlainStreams = 64;
int plain_slots(const GraphDev &g, int64_t k) {
  if (g.n > kPlainBlockMaxN || k < 2) return 1;
  return (int)std::min<int64_t>(kPlainStreams, k);
}

// Concurrent batch groups of a batched job (MultiParams): the job's batches
// after its trials run G at a time, each group on 1/G of the SMs.  G is
// tried per graph and width (kGroupTrial); BC_GROUPS fixes it for
// experiments.  A job's workspace holds one copy per group it may use.
constexpr int kGroupTrial[3] = {1, 2, 4};
constexpr int kNumGroupTrial = 3;
int forced_groups() {
  if (const char *env = std::getenv("BC_GROUPS")) return std::max(1, std::min(std::atoi(env), 8));
  return 0;
}
int batch_groups(const GraphRec &gr, int words, int64_t k, int kb) {
  int want = forced_groups();
  if (!want) {
    const int t = gr.tuned_groups[word_index(words)].load();
    want = t > 0 ? t : kGroupTrial[kNumGroupTrial - 1];
  }
  // at least two batches per group
  while (want > 1 && k < (int64_t)2 * want * kb) want /= 2;
  return want;
}

// Bytes a stretch of batches moved by this design's model, from the job
// counters before (c0) and after (c1) it.
double moved_bytes(const unsigned long long *c0, const unsigned long long *c1, int words, bool fp64,
                   bool c32) {
  auto d = [&](int c) { return (double)(c1[c] - c0[c]); };
  const double b = fp64 ? 8.0 : 4.0, cb = c32 ? 4.0 : 8.0;
  return 124.0 * d(CNT_ENTRIES) + (4.0 + 8.0 * words) * (d(CNT_IN_EDGES) + d(CNT_OUT_EDGES)) +
         (cb + b) * d(CNT_DAG) + (3.0 * cb + b) * d(CNT_REACHED);
}

size_t job_footprint(const GraphRec &gr, int sched, const bc_opts &o, int64_t k) {
  const GraphDev &g = gr.dev;
  WsRec r;
  const int kind = sched == BC_SCHED_PLAIN ? WS_PLAIN : WS_QUEUE;
  const BatchShape bs = batch_shape(o, kind, k, gr.narrow, false);
  WsNeed nd = ws_need(g, kind, bs.kb, bs.words,
                      kind == WS_PLAIN ? plain_slots(g, k) : batch_groups(gr, bs.words, k, bs.kb));
  r.kind = nd.kind;
  r.words = nd.words;
  r.slots = nd.slots;
  r.batch = nd.kind != WS_PLAIN;
  r.n = nd.n;
  r.cap = nd.cap;
  r.hcap = nd.hcap;
  r.chunk_cap = nd.chunk_cap;
  return ws_layout(r, nullptr) + sizeof(double) * (size_t)g.n + (size_t)k * 5 + 4096;
}

void job_free_buffers(bc_ctx *ctx, JobRec *j) {
  if (j->d_src) cudaFreeAsync(j->d_src, j->st);
  if (j->d_bc) cudaFreeAsync(j->d_bc, j->st);
  if (j->d_bc2) cudaFreeAsync(j->d_bc2, j->st);
  j->d_bc2 = nullptr;
  if (j->d_ovf) cudaFreeAsync(j->d_ovf, j->st);
  if (j->d_cnt) cudaFreeAsync(j->d_cnt, j->st);
  if (j->h_slots) pin_put(ctx, j->h_slots, sizeof(KParams) * (size_t)std::max(j->ws_slots, 1));
  j->h_slots = nullptr;
  if (j->h_works) pin_put(ctx, j->h_works, sizeof(Work) * (size_t)std::max(j->works_n, 1));
  j->h_works = nullptr;
  j->d_src = nullptr;
  j->d_bc = nullptr;
  j->d_ovf = nullptr;
  j->d_cnt = nullptr;
  pin_put(ctx, j->h_src, sizeof(int32_t) * (size_t)std::max<int64_t>(j->k, 1));
  pin_put(ctx, j->h_cnt, sizeof(unsigned long long) * (CNT_N + 1));
  pin_put(ctx, j->h_ovf, (size_t)std::max<int64_t>(j->k, 1));
  j->h_src = nullptr;
  j->h_cnt = nullptr;
  j->h_ovf = nullptr;
  j->h_err = nullptr;
  if (j->d_trace) cudaFreeAsync(j->d_trace, j->st);
  if (j->h_trace) cudaFreeHost(j->h_trace);
  j->d_trace = nullptr;
  j->h_trace = nullptr;
  if (j->ev0) cudaEventDestroy(j->ev0);
  if (j->ev1) cudaEventDestroy(j->ev1);
  if (j->evdone) cudaEventDestroy(j->evdone);
  j->ev0 = j->ev1 = j->evdone = nullptr;
}

struct DebugOut {
  int32_t *d = nullptr; // device [k][n]
  uint64_t *sigma = nullptr;
  double *delta = nullptr;
};

// Tuning candidate of a fixed work split (items per fetch at the default).
int cand_of_split(int variant) {
  for (int c = 0; c < kNumTune; ++c)
    if (kTuneCandidates[c].variant == variant && kTuneCandidates[c].grab == kGrabDefault) return c;
  return 0;
}

// BC_SPLIT fixes the tuning candidate (an index into kTuneCandidates) of
// every batched job and skips the split trial, for experiments and for
// profiling a tuned configuration under a profiler, whose launch overheads
// would skew the timed trials (-1: not set).
int forced_split() {
  if (const char *env = std::getenv("BC_SPLIT")) {
    const int c = std::atoi(env);
    if (c >= 0 && c < kNumTune) return c;
  }
  return -1;
}

// Times the batches launched between consecutive events of `ev` (all of them
// enqueued already) and returns, per slot of `slot_of`, the summed time per
// source; the events are destroyed.
bc_status trial_times(std::vector<cudaEvent_t> &ev, const std::vector<int> &slot_of,
                      const std::vector<int64_t> &sources, std::vector<double> &per_slot) {
  bc_status s = BC_OK;
  if (cudaEventSynchronize(ev.back()) != cudaSuccess) s = BC_ERR_CUDA;
  for (size_t t = 0; t + 1 < ev.size() && s == BC_OK; ++t) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[t], ev[t + 1]) != cudaSuccess) s = BC_ERR_CUDA;
    per_slot[(size_t)slot_of[t]] += (double)ms / (double)std::max<int64_t>(sources[t], 1);
  }
  for (cudaEvent_t &e : ev)
    if (e) cudaEventDestroy(e);
  ev.clear();
  return s;
}

// The one-block plain form: source i of the job runs as its own one-block
// launch on stream i mod S (S = the workspace's slots), with that slot's
// workspace copy and BC partial vector; the job's stream waits for all of
// them, sums the partial vectors in slot order and collects the first
// device error of any slot.
bc_status run_plain_blocks(bc_ctx *ctx, JobRec *j, KParams p, const DebugOut *dbg) {
  WsRec *ws = j->ws.get();
  const int64_t n = j->g->dev.n, k = j->k;
  const bool fp64 = j->opts.delta_fp64 != 0;
  const int S = (int)std::min<int64_t>(ws->slots, k);
  cudaStream_t st = j->st;
  // one job at a time uses the extra streams (jobs of other threads wait)
  std::lock_guard<std::mutex> lk(ctx->aux_mu);
  while ((int)ctx->aux.size() < S) {
    cudaStream_t a = nullptr;
    cudaEvent_t e = nullptr;
    BC_TRY(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    BC_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->aux.push_back(a);
    ctx->aux_ev.push_back(e);
  }
  if (!ctx->aux_root) BC_TRY(cudaStreamCreateWithFlags(&ctx->aux_root, cudaStreamNonBlocking));
  // each slot's parameters (a launch adds its source's position b),
  // staged in pinned memory and copied in stream order
  p.g.nchunks = j->g->nch_variant[kSplitWarp];
  p.grab = kGrabDefault;
  p.k = 1;
  p.src = j->d_src;
  p.src_base = 0;
  p.trace = nullptr;
  p.trace_cap = 0;
  if (dbg) {
    p.dbg_d = dbg->d;
    p.dbg_sigma = dbg->sigma;
    p.dbg_delta = dbg->delta;
  }
  j->ws_slots = S;
  BC_TRY(pin_get(ctx, &j->h_slots, sizeof(KParams) * (size_t)S));
  for (int i = 0; i < S; ++i) {
    j->h_slots[i] = p;
    j->h_slots[i].w = slot_work(*ws, i);
    j->h_slots[i].bc = ws->parts + (size_t)i * (size_t)n;
  }
  BC_TRY(cudaMemcpyAsync(ws->slot_params, j->h_slots, sizeof(KParams) * (size_t)S,
                         cudaMemcpyHostToDevice, st));
  BC_TRY(cudaMemsetAsync(ws->parts, 0, sizeof(double) * (size_t)n * (size_t)S, st));
  // the k launches over S streams, captured once per (k, S, precision) and
  // replayed: one graph launch costs the host far less than k launches
  if (!ws->plain_exec || ws->plain_k != k || ws->plain_s != S || ws->plain_fp64 != fp64) {
    if (ws->plain_exec) cudaGraphExecDestroy(ws->plain_exec);
    ws->plain_exec = nullptr;
    cudaStream_t cs = ctx->aux_root;
    BC_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaEventRecord(ctx->aux_ev[0], cs);
    for (int i = 0; i < S && e == cudaSuccess; ++i)
      e = cudaStreamWaitEvent(ctx->aux[(size_t)i], ctx->aux_ev[0], 0);
    for (int64_t b = 0; b < k && e == cudaSuccess; ++b)
      e = launch_plain_block(ws->slot_params, (int)(b % S), b, fp64, ctx->aux[(size_t)(b % S)]);
    for (int i = 0; i < S && e == cudaSuccess; ++i) {
      e = cudaEventRecord(ctx->aux_ev[(size_t)i], ctx->aux[(size_t)i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->aux_ev[(size_t)i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ws->plain_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    BC_TRY(e);
    ws->plain_k = k;
    ws->plain_s = S;
    ws->plain_fp64 = fp64;
  }
  BC_TRY(cudaGraphLaunch(ws->plain_exec, st));
  j->batches += k;
  j->launches += k;
  BC_TRY(launch_sum_parts(ws->parts, S, n, j->d_bc, st));
  BC_TRY(launch_gather_err(ws->w.ctl, ws->slot_bytes, S, st));
  j->launches += 2;
  j->cand = cand_of_split(kSplitWarp);
  return BC_OK;
}

// Launches a job's batches on j->st in source order.  A graph's first job
// with enough sources also tunes, on its own batches (every configuration
// computes the same sums; only the work layout differs):
//   - with the automatic width, the width trial: two rounds of one batch at
//     each width from the automatic one down to 64 sources (rounds in
//     opposite orders, so a trend in cost along the grouped source order
//     weighs every width alike); the fastest per source is kept for the
//     graph.  A width runs in the same workspace in its own layout, which is
//     cleared (all but the control block, which keeps errors) when the width
//     changes;
//   - then, unless the schedule fixes it, the work-split trial at the chosen
//     width: kTuneRounds batches per candidate, fastest kept per graph and
//     width.
// Records graph g's current tuning results in its context's memo.
void remember_tuning(bc_ctx *ctx, const GraphRec &g) {
  if (!g.fingerprint) return;
  TuneMemo t;
  for (int i = 0; i < 3; ++i) {
    t.tuned[i] = g.tuned[i].load();
    t.tuned_groups[i] = g.tuned_groups[i].load();
  }
  t.tuned_words = g.tuned_words.load();
  t.narrow = g.narrow.load();
  t.no_push = g.no_push.load();
  t.wide_counts = g.wide_counts.load();
  std::lock_guard<std::mutex> lk(ctx->memo_mu);
  if (ctx->tune_memo.size() >= kTuneMemoMax && !ctx->tune_memo.count(g.fingerprint))
    ctx->tune_memo.clear();
  ctx->tune_memo[g.fingerprint] = t;
}

// Gives a new graph the tuning results remembered for its fingerprint, if any.
void recall_tuning(bc_ctx *ctx, GraphRec &g) {
  if (!g.fingerprint) return;
  std::lock_guard<std::mutex> lk(ctx->memo_mu);
  auto it = ctx->tune_memo.find(g.fingerprint);
  if (it == ctx->tune_memo.end()) return;
  const TuneMemo &t = it->second;
  for (int i = 0; i < 3; ++i) {
    g.tuned[i] = t.tuned[i];
    g.tuned_groups[i] = t.tuned_groups[i];
  }
  g.tuned_words = t.tuned_words;
  g.narrow = t.narrow;
  g.no_push = t.no_push;
  g.wide_counts = t.wide_counts;
}

bc_status run_batches(bc_ctx *ctx, JobRec *j, KParams p, const DebugOut *dbg, bool wtrial,
                      int trace_cap) {
  const GraphDev &g = j->g->dev;
  const bool fp64 = j->opts.delta_fp64 != 0;
  const int64_t n = g.n, k = j->k;
  cudaStream_t st = j->st;
  const int kind = j->kind;
  const int fixed = fixed_split(resolve_schedule(j->opts, g));
  const bool notune = dbg || kind != WS_QUEUE || std::getenv("BC_NO_TUNE");
  // 32-bit path-count rows unless asked for 64 bits or this graph needed them
  const bool c32 = j->opts.count_bits != 64 && !j->g->wide_counts && !j->acc_sum;
  WsRec *ws = j->ws.get();
  if (kind == WS_PLAIN && ws->slots > 1) return run_plain_blocks(ctx, j, p, dbg);
  const size_t ctl_bytes = align_up(sizeof(Ctl), 256);
  int cur_words = j->words; // layout the workspace holds
  int64_t bi = 0, b0 = 0;

  auto launch = [&](int kb, int words, int cand) -> bc_status {
    if (words != cur_words) {
      WsRec r = *ws;
      r.words = words;
      ws_layout(r, static_cast<char *>(ws->mem));
      p.w = r.w;
      // trials run in the first copy only (the others stay clean)
      BC_TRY(cudaMemsetAsync(static_cast<char *>(ws->mem) + ctl_bytes, 0,
                             ws->slot_bytes - ctl_bytes, st));
      cur_words = words;
    }
    p.g.nchunks = j->g->nch_variant[kTuneCandidates[cand].variant];
    p.grab = kTuneCandidates[cand].grab;
    p.src = j->d_src + b0;
    p.k = (int32_t)std::min<int64_t>(kb, k - b0);
    p.src_base = b0;
    p.trace = (j->d_trace && bi == j->trace_batch) ? j->d_trace : nullptr;
    p.trace_cap = p.trace ? trace_cap : 0;
    if (dbg) {
      p.dbg_d = dbg->d + b0 * n;
      p.dbg_sigma = dbg->sigma + b0 * n;
      p.dbg_delta = dbg->delta + b0 * n;
    }
    const int grid = pick_grid(ctx, g, kind, fp64, words);
    if (grid <= 0) return BC_ERR_CUDA;
    BC_TRY(kind == WS_QUEUE ? launch_batch(p, fp64, grid, st, words, c32)
                            : launch_plain(p, fp64, grid, st));
    b0 += p.k;
    ++bi;
    ++j->batches;
    ++j->launches;
    j->cand = cand;
    return BC_OK;
  };
  auto record = [&](std::vector<cudaEvent_t> &ev) -> bc_status {
    cudaEvent_t e = nullptr;
    BC_TRY(cudaEventCreate(&e));
    ev.push_back(e);
    BC_TRY(cudaEventRecord(e, st));
    return BC_OK;
  };

  int words = j->words;
  int kb = j->kb;
  const int split_cand = fixed >= 0 ? cand_of_split(fixed) : 0;
  // ---- width trial ----
  if (wtrial && !notune) {
    std::vector<int> widths;
    for (int w : kWidthTrial)
      if (w <= words) widths.push_back(w);
    int64_t need = 0;
    for (int w : widths) need += 2 * (int64_t)kK * w;
    if (widths.size() > 1 && k - need >= 2 * (int64_t)kK * words) {
      std::vector<cudaEvent_t> ev;
      std::vector<int> slot_of;
      std::vector<int64_t> srcs;
      const int nw = (int)widths.size();
      for (int t = 0; t < 2 * nw; ++t) {
        const int i = t < nw ? t : 2 * nw - 1 - t;
        const int w = widths[(size_t)i];
        bc_status s = record(ev);
        if (s != BC_OK) return s;
        slot_of.push_back(i);
        srcs.push_back(std::min<int64_t>((int64_t)kK * w, k - b0));
        s = launch(kK * w, w, split_cand);
        if (s != BC_OK) return s;
      }
      bc_status s = record(ev);
      if (s != BC_OK) return s;
      std::vector<double> per((size_t)nw, 0.0);
      s = trial_times(ev, slot_of, srcs, per);
      if (s != BC_OK) return s;
      int best = 0;
      for (int i = 1; i < nw; ++i)
        if (per[(size_t)i] < per[(size_t)best]) best = i;
      words = widths[(size_t)best];
      kb = kK * words;
      j->g->tuned_words = words;
    }
  }
  j->words = words;
  j->kb = kb;
  // ---- work-split trial ----
  // Candidates are compared by throughput, not time: the trial batches take
  // consecutive sources of the grouped order, whose work per batch varies
  // several-fold (and drops to nothing for sources without out-edges), so
  // each batch's time is set against the bytes its own counters say it
  // moved (the design's bytes model, from counter snapshots taken between
  // the trial batches).
  std::atomic<int> &tuned_slot = j->g->tuned[word_index(words)];
  const int forced_cand = forced_split();
  int cand = fixed >= 0 ? split_cand
             : forced_cand >= 0 ? forced_cand
                                : std::max(tuned_slot.load(), 0);
  if (kind != WS_QUEUE) cand = 0;
  const int64_t left = (k - b0 + kb - 1) / kb;
  if (!notune && fixed < 0 && forced_cand < 0 && tuned_slot.load() < 0 &&
      left >= kNumTune * kTuneRounds + 4) {
    constexpr int kTrials = kNumTune * kTuneRounds;
    unsigned long long *d_snap = nullptr;
    BC_TRY(pool_alloc(ctx, &d_snap, sizeof(unsigned long long) * CNT_N * (kTrials + 1), st));
    auto snap = [&](int t) {
      return cudaMemcpyAsync(d_snap + (size_t)t * CNT_N, j->d_cnt,
                             sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToDevice, st);
    };
    std::vector<cudaEvent_t> ev;
    std::vector<int> slot_of;
    std::vector<int64_t> ones;
    bc_status s = BC_OK;
    if (snap(0) != cudaSuccess) s = BC_ERR_CUDA;
    for (int t = 0; t < kTrials && s == BC_OK; ++t) {
      // rounds alternate direction (c0 c1 .. c4 c4 .. c0)
      const int r = t / kNumTune, c = t % kNumTune;
      const int cc = r % 2 == 0 ? c : kNumTune - 1 - c;
      s = record(ev);
      if (s == BC_OK) s = launch(kb, words, cc);
      if (s == BC_OK && snap(t + 1) != cudaSuccess) s = BC_ERR_CUDA;
      slot_of.push_back(t); // one slot per trial batch
      ones.push_back(1);
    }
    if (s == BC_OK) s = record(ev);
    std::vector<double> ms((size_t)kTrials, 0.0);
    if (s == BC_OK) s = trial_times(ev, slot_of, ones, ms);
    std::vector<unsigned long long> h((size_t)CNT_N * (kTrials + 1), 0);
    if (s == BC_OK &&
        (cudaMemcpyAsync(h.data(), d_snap, sizeof(unsigned long long) * h.size(),
                         cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
      s = BC_ERR_CUDA;
    cudaFreeAsync(d_snap, st);
    if (s != BC_OK) return s;
    std::vector<double> bytes((size_t)kNumTune, 0.0), time((size_t)kNumTune, 0.0);
    for (int t = 0; t < kTrials; ++t) {
      const int r = t / kNumTune, c = t % kNumTune;
      const int cc = r % 2 == 0 ? c : kNumTune - 1 - c;
      bytes[(size_t)cc] += moved_bytes(h.data() + (size_t)t * CNT_N, h.data() + (size_t)(t + 1) * CNT_N,
                                       words, j->opts.delta_fp64 != 0, c32);
      time[(size_t)cc] += ms[(size_t)t];
    }
    // the default split stays unless another is clearly faster: the trial
    // batches differ in content, so small differences are noise
    int best = 0;
    auto rate = [&](int c) { return time[(size_t)c] > 0.0 ? bytes[(size_t)c] / time[(size_t)c] : 0.0; };
    for (int c = 1; c < kNumTune; ++c)
      if (rate(c) > rate(best) && rate(c) > kTuneMargin * rate(0)) best = c;
    tuned_slot = best;
    cand = best;
  }
  // ---- concurrent batch groups ----
  // Sources [b0, end) in groups of G concurrent batches (G = 1: one launch
  // per batch).  G > 1 runs one launch, group g on its own slot workspace
  // and BC partial vector, the partials added to the job's BC in group order.
  const bool groups_ok = kind == WS_QUEUE && !dbg && cur_words == ws->words && words == ws->words;
  auto run_range = [&](int G, int64_t end) -> bc_status {
    const int gsize = G > 1 ? ctx->grid_batch[word_index(words)][fp64] / G : 0;
    if (G <= 1 || gsize < 1 || !groups_ok || G > ws->slots) {
      if (b0 < end) j->groups_used = 1;
      while (b0 < end) {
        const bc_status s = launch(kb, words, cand);
        if (s != BC_OK) return s;
      }
      return BC_OK;
    }
    if (!j->h_works) {
      BC_TRY(pin_get(ctx, &j->h_works, sizeof(Work) * (size_t)ws->slots));
      j->works_n = ws->slots;
      for (int i = 0; i < ws->slots; ++i) j->h_works[i] = slot_work(*ws, i);
      // room for `slots` entries where the one-block plain form keeps its parameters
      BC_TRY(cudaMemcpyAsync(ws->slot_params, j->h_works, sizeof(Work) * (size_t)ws->slots,
                             cudaMemcpyHostToDevice, st));
    }
    BC_TRY(cudaMemsetAsync(ws->parts, 0, sizeof(double) * (size_t)n * (size_t)G, st));
    MultiParams mp;
    mp.base = p;
    mp.base.g.nchunks = j->g->nch_variant[kTuneCandidates[cand].variant];
    mp.base.grab = kTuneCandidates[cand].grab;
    mp.base.src = j->d_src;
    mp.base.dbg_d = nullptr;
    mp.works = reinterpret_cast<const Work *>(ws->slot_params);
    mp.parts = ws->parts;
    mp.groups = G;
    mp.gsize = gsize;
    mp.kb = kb;
    mp.k = end;
    mp.first = b0;
    BC_TRY(launch_multi(mp, fp64, words, c32, st));
    j->groups_used = G;
    BC_TRY(launch_sum_parts(ws->parts, G, n, j->d_bc, st, true));
    BC_TRY(launch_gather_err(ws->w.ctl, ws->slot_bytes, G, st));
    j->batches += (end - b0 + kb - 1) / kb;
    j->launches += 3;
    j->cand = cand;
    b0 = end;
    return BC_OK;
  };
  const int forced = forced_groups();
  std::atomic<int> &tuned_g = j->g->tuned_groups[word_index(words)];
  int G = forced ? forced : std::max(1, tuned_g.load());
  // the groups trial: 2G batches with each G of kGroupTrial, compared by
  // throughput like the split trial; the fastest is kept per graph and
  // width (one group unless another is more than kTuneMargin faster)
  int64_t need = 0;
  for (int g : kGroupTrial) need += 2 * (int64_t)g * kb;
  if (!notune && !forced && tuned_g.load() < 1 && groups_ok &&
      ws->slots >= kGroupTrial[kNumGroupTrial - 1] && k - b0 >= need) {
    unsigned long long *d_snap = nullptr;
    BC_TRY(pool_alloc(ctx, &d_snap, sizeof(unsigned long long) * CNT_N * (kNumGroupTrial + 1), st));
    std::vector<cudaEvent_t> ev;
    std::vector<int> slot_of;
    std::vector<int64_t> ones;
    bc_status s = BC_OK;
    for (int t = 0; t <= kNumGroupTrial && s == BC_OK; ++t) {
      if (cudaMemcpyAsync(d_snap + (size_t)t * CNT_N, j->d_cnt, sizeof(unsigned long long) * CNT_N,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        s = BC_ERR_CUDA;
      if (s == BC_OK) s = record(ev);
      if (s == BC_OK && t < kNumGroupTrial) {
        slot_of.push_back(t);
        ones.push_back(1);
        s = run_range(kGroupTrial[t], std::min<int64_t>(k, b0 + 2 * (int64_t)kGroupTrial[t] * kb));
      }
    }
    std::vector<double> ms((size_t)kNumGroupTrial, 0.0);
    if (s == BC_OK) s = trial_times(ev, slot_of, ones, ms);
    std::vector<unsigned long long> h((size_t)CNT_N * (kNumGroupTrial + 1), 0);
    if (s == BC_OK &&
        (cudaMemcpyAsync(h.data(), d_snap, sizeof(unsigned long long) * h.size(),
                         cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
      s = BC_ERR_CUDA;
    cudaFreeAsync(d_snap, st);
    if (s != BC_OK) return s;
    std::vector<double> rate((size_t)kNumGroupTrial, 0.0);
    for (int t = 0; t < kNumGroupTrial; ++t)
      rate[(size_t)t] = ms[(size_t)t] > 0.0 ? moved_bytes(h.data() + (size_t)t * CNT_N,
                                                         h.data() + (size_t)(t + 1) * CNT_N,
                                                         words, j->opts.delta_fp64 != 0, c32) /
                                                  ms[(size_t)t]
                                            : 0.0;
    int best = 0;
    for (int t = 1; t < kNumGroupTrial; ++t)
      if (rate[(size_t)t] > rate[(size_t)best] && rate[(size_t)t] > kTuneMargin * rate[0]) best = t;
    G = kGroupTrial[best];
    tuned_g = G;
  }
  // Full batches up to the sources without out-edges (the tuning trials
  // above may have taken some of those already; the rest are not launched),
  // then the last, partly filled batch: with at most half its sources it
  // runs with fewer mask words in the same layout (bc_narrow.cu).
  const int64_t kt = std::max(b0, j->k_traverse);
  const int64_t full_end = b0 + (kt - b0) / kb * kb;
  {
    const bc_status s = run_range(G, kind == WS_QUEUE && !dbg ? full_end : kt);
    if (s != BC_OK) return s;
  }
  if (b0 < kt) {
    const int64_t rem = kt - b0;
    int nw = words;
    while (nw > 1 && rem <= (int64_t)kK * (nw / 2)) nw /= 2;
    if (nw < words && cur_words == words && !j->acc_sum && kind == WS_QUEUE && !dbg) {
      p.g.nchunks = j->g->nch_variant[kTuneCandidates[cand].variant];
      p.grab = kTuneCandidates[cand].grab;
      p.src = j->d_src + b0;
      p.k = (int32_t)rem;
      p.src_base = b0;
      p.trace = (j->d_trace && bi == j->trace_batch) ? j->d_trace : nullptr;
      p.trace_cap = p.trace ? trace_cap : 0;
      const int grid = pick_grid(ctx, g, kind, fp64, words);
      if (grid <= 0) return BC_ERR_CUDA;
      BC_TRY(launch_batch_narrow(p, fp64, grid, st, nw, words, c32));
      b0 = kt;
      ++bi;
      ++j->batches;
      ++j->launches;
      j->cand = cand;
    } else {
      while (b0 < kt) {
        const bc_status s = launch(kb, words, cand);
        if (s != BC_OK) return s;
      }
    }
  }
  if (cur_words != ws->words) // back to the workspace's own layout, clean
    BC_TRY(cudaMemsetAsync(static_cast<char *>(ws->mem) + ctl_bytes, 0, ws->slot_bytes - ctl_bytes,
                           st));
  if (!notune) remember_tuning(ctx, *j->g);
  return BC_OK;
}

// Enqueues a whole job on j->st: inputs, one launch per batch, scaling, copy
// of the result to `out` (device or host pointer per opts.out_device; an
// async job passes its pinned buffer) and of the job counters.
bc_status job_launch(bc_ctx *ctx, JobRec *j, double *out, const DebugOut *dbg) {
  const GraphDev &g = j->g->dev;
  const int sched = resolve_schedule(j->opts, g);
  const bool batch = sched != BC_SCHED_PLAIN;
  const bool fp64 = j->opts.delta_fp64 != 0;
  const int64_t n = g.n, k = j->k;
  cudaStream_t st = j->st;
  const int kind = batch ? WS_QUEUE : WS_PLAIN;
  j->kind = kind;
  // the batched kernels index a step's work items (two levels' entries and
  // heavy chunks) in 32 bits
  if (batch && 2 * n + 2 * g.heavy_chunks >= (int64_t)INT32_MAX) return BC_ERR_ARG;
  BatchShape bs = batch_shape(j->opts, kind, k, j->g->narrow, dbg != nullptr);
  // wider than one mask word: the queue kernel only
  if (bs.words > 1 && kind != WS_QUEUE) return BC_ERR_ARG;
  // automatic width: the graph's width trial, once run, caps it
  const bool auto_width = batch && j->opts.batch_k == 0 && !j->g->narrow && !dbg;
  const int tw = j->g->tuned_words.load();
  if (auto_width && tw > 0 && tw < bs.words) bs = {kK * tw, tw};
  // the width trial runs on the first job of a graph whose automatic width
  // has narrower alternatives and enough sources to try each twice
  const bool wtrial = auto_width && tw == 0 && bs.words > 1 && !std::getenv("BC_NO_TUNE");
  const int kb = bs.kb, words = bs.words;
  j->kb = kb;
  j->words = words;

  j->groups = batch && !dbg ? batch_groups(*j->g, words, k, kb) : 1;
  bc_status s = ws_acquire(ctx, ws_need(g, kind, kb, words, batch ? j->groups : plain_slots(g, k)),
                           st, j->ws);
  if (s != BC_OK) return s;
  BC_TRY(pin_get(ctx, &j->h_src, sizeof(int32_t) * (size_t)std::max<int64_t>(k, 1)));
  BC_TRY(pin_get(ctx, &j->h_cnt, sizeof(unsigned long long) * (CNT_N + 1)));
  BC_TRY(pin_get(ctx, &j->h_ovf, (size_t)std::max<int64_t>(k, 1)));
  j->h_err = reinterpret_cast<int *>(j->h_cnt + CNT_N);
  // batch composition (bc_opts.source_order); debug exports keep the given
  // order, since their rows follow it
  const bool grouped = batch && !dbg && j->opts.source_order == 0 && k > kb;
  if (j->all_sources) {
    if (grouped) {
      s = ensure_order(j->g, st);
      if (s != BC_OK) return s;
      std::memcpy(j->h_src, j->g->order.data(), sizeof(int32_t) * (size_t)k);
    } else {
      for (int64_t i = 0; i < k; ++i) j->h_src[i] = (int32_t)i;
    }
  } else if (k) {
    std::memcpy(j->h_src, j->src.data(), sizeof(int32_t) * (size_t)k);
    if (grouped) {
      GraphRec *g = j->g;
      if (k >= (int64_t)n / 8) {
        // many sources: walk the graph's batch order once, emitting each
        // vertex as often as the list holds it (O(n + k))
        s = ensure_order(g, st);
        if (s != BC_OK) return s;
        std::vector<int32_t> cnt((size_t)n, 0);
        for (int64_t i = 0; i < k; ++i) cnt[(size_t)j->h_src[i]]++;
        int64_t w = 0;
        for (int32_t v : g->order)
          for (int32_t c = cnt[(size_t)v]; c > 0; --c) j->h_src[w++] = v;
      } else {
        // few sources: their packed keys, sorted (equal keys are equal ids)
        std::vector<OrderKey> keys((size_t)k);
        for (int64_t i = 0; i < k; ++i) keys[(size_t)i] = order_key(g->row_ptr, g->two, j->h_src[i]);
        std::sort(keys.begin(), keys.end());
        for (int64_t i = 0; i < k; ++i) j->h_src[i] = (int32_t)(uint32_t)keys[(size_t)i].lo;
      }
    }
  }
  j->k_traverse = k;
  if (grouped && !j->acc_sum) {
    const std::vector<int32_t> &rp = j->g->row_ptr;
    while (j->k_traverse > 0) {
      const int32_t v = j->h_src[j->k_traverse - 1];
      if (rp[(size_t)v + 1] != rp[(size_t)v]) break;
      --j->k_traverse;
    }
  }
  BC_TRY(pool_alloc(ctx, &j->d_src, sizeof(int32_t) * (size_t)std::max<int64_t>(k, 1), st));
  BC_TRY(pool_alloc(ctx, &j->d_bc, sizeof(double) * (size_t)std::max<int64_t>(n, 1), st));
  BC_TRY(pool_alloc(ctx, &j->d_ovf, (size_t)std::max<int64_t>(k, 1), st));
  BC_TRY(pool_alloc(ctx, &j->d_cnt, sizeof(unsigned long long) * CNT_N, st));
  if (k) BC_TRY(cudaMemcpyAsync(j->d_src, j->h_src, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st));
  BC_TRY(cudaMemsetAsync(j->d_bc, 0, sizeof(double) * (size_t)std::max<int64_t>(n, 1), st));
  BC_TRY(cudaMemsetAsync(j->d_ovf, 0, (size_t)std::max<int64_t>(k, 1), st));
  BC_TRY(cudaMemsetAsync(j->d_cnt, 0, sizeof(unsigned long long) * CNT_N, st));
  BC_TRY(cudaMemsetAsync(j->ws->w.ctl, 0, sizeof(Ctl), st));
  BC_TRY(cudaEventCreate(&j->ev0));
  BC_TRY(cudaEventCreate(&j->ev1));
  BC_TRY(cudaEventCreateWithFlags(&j->evdone, cudaEventDisableTiming));

  if (j->acc_sum) {
    BC_TRY(pool_alloc(ctx, &j->d_bc2, sizeof(double) * (size_t)std::max<int64_t>(n, 1), st));
    BC_TRY(cudaMemsetAsync(j->d_bc2, 0, sizeof(double) * (size_t)std::max<int64_t>(n, 1), st));
  }
  KParams p;
  p.g = g;
  p.w = j->ws->w;
  p.bc = j->d_bc;
  p.bc2 = j->d_bc2;
  p.ovf_flags = j->d_ovf;
  p.job_cnt = j->d_cnt;
  p.push_ratio = push_ratio(j->opts, *j->g);
  if (ctx->inject_block >= 0 && batch) {
    p.skip_block = ctx->inject_block;
    p.timeout_ns = (long long)ctx->inject_timeout_ms * 1000000LL;
    ctx->inject_block = -1;
  }
  if (pick_grid(ctx, g, kind, fp64, words) <= 0) return BC_ERR_CUDA;
  constexpr int kTraceCap = 8192;
  if (const char *tr = std::getenv("BC_TRACE")) {
    // per-step timing of one batch (index BC_TRACE, -1 = last) to stderr
    j->trace_batch = std::atoll(tr);
    if (j->trace_batch < 0) j->trace_batch = (k + kb - 1) / kb - 1;
    BC_TRY(pool_alloc(ctx, &j->d_trace, sizeof(unsigned long long) * 4 * kTraceCap, st));
    BC_TRY(cudaMemsetAsync(j->d_trace, 0, sizeof(unsigned long long) * 4 * kTraceCap, st));
    BC_TRY(cudaMallocHost(&j->h_trace, sizeof(unsigned long long) * 4 * kTraceCap));
  }
  BC_TRY(cudaEventRecord(j->ev0, st));
  j->batches = 0;
  j->launches = 0;
  s = run_batches(ctx, j, p, dbg, wtrial, kTraceCap);
  if (s != BC_OK) return s;
  BC_TRY(cudaEventRecord(j->ev1, st));
  double factor = 1.0;
  if (j->opts.normalize && n > 2) factor /= (double)(n - 1) * (double)(n - 2);
  if (j->opts.scale_sampled && k > 0) factor *= (double)n / (double)k;
  if (j->acc_sum) {
    // estimator job: add this job's sums into the running ones (skipped on a
    // device error, so a rerun never double counts)
    BC_TRY(launch_accumulate(j->acc_sum, j->acc_sumsq, j->d_bc, j->d_bc2, n, &j->ws->w.ctl->err,
                             st));
    ++j->launches;
  } else if (out && n > 0) {
    if (j->opts.out_device) {
      BC_TRY(launch_scale(j->d_bc, out, n, factor, st));
    } else {
      BC_TRY(launch_scale(j->d_bc, j->d_bc, n, factor, st));
      BC_TRY(cudaMemcpyAsync(out, j->d_bc, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    }
    ++j->launches;
  }
  BC_TRY(cudaMemcpyAsync(j->h_cnt, j->d_cnt, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, st));
  BC_TRY(cudaMemcpyAsync(j->h_err, &j->ws->w.ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (k) BC_TRY(cudaMemcpyAsync(j->h_ovf, j->d_ovf, (size_t)k, cudaMemcpyDeviceToHost, st));
  if (j->d_trace)
    BC_TRY(cudaMemcpyAsync(j->h_trace, j->d_trace, sizeof(unsigned long long) * 4 * kTraceCap,
                           cudaMemcpyDeviceToHost, st));
  BC_TRY(cudaEventRecord(j->evdone, st));
  return BC_OK;
}

// After evdone completed: statistics, status, workspace hand-back.
bc_status job_finish(bc_ctx *ctx, JobRec *j) {
  bc_stats &s = j->stats;
  std::memset(&s, 0, sizeof(s));
  s.n = j->g->dev.n;
  s.m = j->g->dev.m;
  s.sources = j->k;
  s.batches = j->batches;
  s.kernel_launches = j->launches;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, j->ev0, j->ev1) == cudaSuccess) s.device_ms = ms;
  s.frontier_entries = (int64_t)j->h_cnt[CNT_ENTRIES];
  s.scanned_out_edges = (int64_t)j->h_cnt[CNT_OUT_EDGES];
  s.scanned_in_edges = (int64_t)j->h_cnt[CNT_IN_EDGES];
  s.dag_pairs = (int64_t)j->h_cnt[CNT_DAG];
  s.reached_pairs = (int64_t)j->h_cnt[CNT_REACHED];
  s.heavy_chunks = (int64_t)j->h_cnt[CNT_HEAVY];
  s.max_levels = (int32_t)j->h_cnt[CNT_MAXLEV];
  s.kernel_kind = j->kind == WS_QUEUE ? 2 : 1;
  s.levels_sum = (int32_t)j->h_cnt[CNT_LEVELS];
  s.chunk_edges = kTuneCandidates[j->cand].variant == kSplitVertex
                      ? 0
                      : kChunkCandidates[kTuneCandidates[j->cand].variant];
  s.batch_sources = j->kb;
  s.mask_words = j->words;
  s.grab = kTuneCandidates[j->cand].grab;
  s.push_levels = (int32_t)j->h_cnt[CNT_PUSH];
  s.batch_groups = j->groups_used;
  int32_t novf = 0;
  j->ovf_sources.clear();
  for (int64_t i = 0; i < j->k; ++i)
    if (j->h_ovf[i]) {
      ++novf;
      j->ovf_sources.push_back(j->h_src[i]); // flags follow the launched source order
    }
  std::sort(j->ovf_sources.begin(), j->ovf_sources.end());
  if (j->h_trace && (j->h_cnt[CNT_BUSY] || j->h_cnt[CNT_IDLE])) {
    const double b = (double)j->h_cnt[CNT_BUSY], i = (double)j->h_cnt[CNT_IDLE];
    std::fprintf(stderr, "# phase clocks: items %.1f%%, waiting for the step end %.1f%%\n",
                 100.0 * b / (b + i), 100.0 * i / (b + i));
  }
  if (j->h_trace) {
    std::fprintf(stderr, "# trace batch %lld: step level items heavy_chunks us\n",
                 (long long)j->trace_batch);
    for (int i = 0; i + 1 < 8192 && j->h_trace[4 * i]; ++i) {
      const unsigned long long *t = j->h_trace + 4 * i;
      const long long lvl = (long long)t[1];
      if (lvl == (1 << 20)) break;
      const double us = t[4] ? (double)(t[4] - t[0]) / 1000.0 : 0.0;
      std::fprintf(stderr, "%d %lld %llu %llu %.2f\n", i, lvl, t[2], t[3], us);
    }
  }
  s.overflow_sources = novf;
  bc_status st = BC_OK;
  const int kerr = *j->h_err;
  if (kerr == KERR_WIDE) {
    // a path count reached 2^32: rerun the job with 64-bit counts (and keep
    // them for this graph)
    j->g->wide_counts = true;
    st = kStatusRetry;
    j->ws->dirty = true;
  } else if (kerr == KERR_PUSH) {
    // a pushed path count reached 2^32, so a pushed sum could have carried:
    // rerun the job pulling every level (and keep pulling on this graph)
    j->g->no_push = true;
    st = kStatusRetry;
    j->ws->dirty = true;
  } else if ((kerr == KERR_QUEUE || kerr == KERR_HEAVY) && j->words > 1) {
    // a wide batch queued vertices at more distinct depths than its queue
    // holds: rerun the job with 64 sources per batch
    j->g->narrow = true;
    st = kStatusRetry;
    j->ws->dirty = true;
  } else if (kerr != KERR_NONE) {
    st = kerr == KERR_TIMEOUT ? BC_ERR_TIMEOUT : BC_ERR_INTERNAL;
    j->ws->dirty = true;
  } else if (novf) {
    st = BC_ERR_SIGMA_OVERFLOW;
  }
  ws_release(ctx, std::move(j->ws));
  job_free_buffers(ctx, j);
  return st;
}

bc_status run_sync(bc_ctx *ctx, GraphRec *g, const int32_t *src, int64_t k, bool all,
                   const bc_opts *opts_in, double *out, const DebugOut *dbg,
                   double *acc_sum = nullptr, double *acc_sumsq = nullptr) {
  bc_opts opts = opts_in ? *opts_in : default_opts();
  if (!opts_valid(opts)) return BC_ERR_ARG;
  JobRec j;
  j.g = g;
  j.opts = opts;
  j.k = k;
  j.all_sources = all;
  if (!all && k) j.src.assign(src, src + k);
  j.st = ctx->stream;
  j.acc_sum = acc_sum;
  j.acc_sumsq = acc_sumsq;
  bc_status s = kStatusRetry;
  for (int attempt = 0; attempt < 5 && s == kStatusRetry; ++attempt) {
    s = job_launch(ctx, &j, out, dbg);
    if (s != BC_OK) {
      cudaStreamSynchronize(j.st);
      if (j.ws) {
        j.ws->dirty = true;
        ws_release(ctx, std::move(j.ws));
      }
      job_free_buffers(ctx, &j);
      return s;
    }
    cudaError_t e = cudaEventSynchronize(j.evdone);
    if (e != cudaSuccess) {
      job_free_buffers(ctx, &j);
      return cuda_status(e);
    }
    s = job_finish(ctx, &j);
  }
  if (s == kStatusRetry) s = BC_ERR_INTERNAL;
  ctx->last = j.stats;
  ctx->last_ovf = j.ovf_sources;
  return s;
}

bc_status check_sources(const GraphRec *g, const int32_t *src, int64_t k) {
  if (k < 0) return BC_ERR_ARG;
  if (k > 0 && !src) return BC_ERR_ARG;
  for (int64_t i = 0; i < k; ++i)
    if (src[i] < 0 || src[i] >= g->dev.n) return BC_ERR_ARG;
  return BC_OK;
}

// ---- scheduler ----------------------------------------------------------------

void scheduler_loop(bc_ctx *ctx) {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->mu);
  while (true) {
    if (ctx->stop && ctx->pending.empty() && ctx->running.empty()) break;
    bool progressed = false;
    // admit pending jobs in arrival order while a slot and memory are free
    while (!ctx->pending.empty()) {
      JobRec *j = ctx->pending.front();
      int slot = -1;
      for (int i = 0; i < kMaxSlots; ++i)
        if (!ctx->slot_busy[i]) {
          slot = i;
          break;
        }
      if (slot < 0) break;
      if (ctx->used + j->footprint > ctx->budget && !ctx->running.empty()) break;
      ctx->pending.pop_front();
      ctx->slot_busy[slot] = true;
      j->slot = slot;
      j->st = ctx->slot_stream[slot];
      lk.unlock();
      bc_status s = job_launch(ctx, j, j->h_out, nullptr);
      lk.lock();
      if (s != BC_OK) {
        lk.unlock();
        cudaStreamSynchronize(j->st);
        if (j->ws) {
          j->ws->dirty = true;
          ws_release(ctx, std::move(j->ws));
        }
        job_free_buffers(ctx, j);
        lk.lock();
        j->status = s;
        j->done = true;
        j->g->active_jobs--;
        ctx->slot_busy[slot] = false;
      } else {
        ctx->running.push_back(j);
      }
      progressed = true;
    }
    // retire finished jobs
    for (size_t i = 0; i < ctx->running.size();) {
      JobRec *j = ctx->running[i];
      if (cudaEventQuery(j->evdone) == cudaSuccess) {
        lk.unlock();
        bc_status s = job_finish(ctx, j);
        if (s == kStatusRetry) {
          s = job_launch(ctx, j, j->h_out, nullptr);
          if (s == BC_OK) {
            lk.lock();
            ++i;
            continue;
          }
          cudaStreamSynchronize(j->st);
          if (j->ws) {
            j->ws->dirty = true;
            ws_release(ctx, std::move(j->ws));
          }
          job_free_buffers(ctx, j);
        }
        lk.lock();
        j->status = s;
        j->done = true;
        j->g->active_jobs--;
        ctx->slot_busy[j->slot] = false;
        ctx->running.erase(ctx->running.begin() + (ptrdiff_t)i);
        progressed = true;
      } else {
        ++i;
      }
    }
    if (progressed) ctx->cv.notify_all();
    if (ctx->pending.empty() && ctx->running.empty()) {
      if (ctx->stop) break;
      ctx->cv.wait(lk);
    } else if (!progressed) {
      ctx->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

} // namespace

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

const char *bc_status_str(bc_status s) {
  switch (s) {
    case BC_OK: return "ok";
    case BC_PENDING: return "pending";
    case BC_ERR_ARG: return "invalid argument";
    case BC_ERR_GRAPH: return "malformed graph or unknown graph handle";
    case BC_ERR_OOM: return "out of memory";
    case BC_ERR_CUDA: return "CUDA runtime error";
    case BC_ERR_TIMEOUT: return "bounded device wait ran out";
    case BC_ERR_SIGMA_OVERFLOW: return "shortest-path count reached 2^64";
    case BC_ERR_NOT_FOUND: return "unknown or consumed job handle";
    case BC_ERR_ADMISSION: return "job does not fit the HBM budget";
    case BC_ERR_INTERNAL: return "device capacity check failed";
  }
  return "unknown status";
}

bc_status bc_init(int device, void *cuda_stream, size_t hbm_budget_bytes, bc_ctx **out) {
  if (!out) return BC_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return BC_ERR_CUDA;
  DeviceGuard dg(device);
  std::unique_ptr<bc_ctx> ctx(new (std::nothrow) bc_ctx());
  if (!ctx) return BC_ERR_OOM;
  ctx->device = device;
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    BC_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  size_t freeb = 0, totalb = 0;
  BC_TRY(cudaMemGetInfo(&freeb, &totalb));
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)freeb);
  {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    BC_TRY(cudaMemPoolCreate(&ctx->pool, &props));
    uint64_t keep = std::min<uint64_t>(kPoolKeepBytes, ctx->budget);
    BC_TRY(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep));
  }
  BC_TRY(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
  for (int f = 0; f < 2; ++f) {
    for (int wi = 0; wi < 3; ++wi) {
      ctx->grid_batch[wi][f] = max_grid_batch(f != 0, device, 1 << wi);
      if (ctx->grid_batch[wi][f] <= 0) return BC_ERR_CUDA;
    }
    ctx->grid_many[f] = max_grid_many(f != 0, device);
    ctx->grid_plain[f] = max_grid_plain(f != 0, device);
    if (ctx->grid_plain[f] <= 0 || ctx->grid_many[f] <= 0)
      return BC_ERR_CUDA;
  }
  for (int i = 0; i < kMaxSlots; ++i)
    BC_TRY(cudaStreamCreateWithFlags(&ctx->slot_stream[i], cudaStreamNonBlocking));
  bc_ctx *raw = ctx.get();
  ctx->sched = std::thread(scheduler_loop, raw);
  *out = ctx.release();
  return BC_OK;
}

bc_status bc_shutdown(bc_ctx *ctx) {
  if (!ctx) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stop = true;
  }
  ctx->cv.notify_all();
  if (ctx->sched.joinable()) ctx->sched.join();
  cudaDeviceSynchronize();
  for (auto &kv : ctx->jobs) {
    if (kv.second->h_out) cudaFreeHost(kv.second->h_out);
  }
  ctx->jobs.clear();
  for (auto &w : ctx->free_ws) ws_free(*w);
  ctx->free_ws.clear();
  for (auto &kv : ctx->graphs) cudaFreeAsync(kv.second->mem, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  ctx->graphs.clear();
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->stage) cudaFreeHost(ctx->stage);
  for (auto &kv : ctx->pin_free) cudaFreeHost(kv.second);
  ctx->pin_free.clear();
  for (int i = 0; i < kMaxSlots; ++i)
    if (ctx->slot_stream[i]) cudaStreamDestroy(ctx->slot_stream[i]);
  for (cudaStream_t a : ctx->aux) cudaStreamDestroy(a);
  if (ctx->aux_root) cudaStreamDestroy(ctx->aux_root);
  for (cudaEvent_t e : ctx->aux_ev) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return BC_OK;
}

bc_status bc_create_graph(bc_ctx *ctx, const int32_t *row_ptr, const int32_t *col_idx,
                          int32_t n, int64_t m, bc_graph *out, int64_t *m_effective) {
  if (!ctx || !out) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  std::unique_ptr<GraphRec> g;
  bc_status s = build_graph(ctx, row_ptr, col_idx, n, m, g, m_effective);
  if (s != BC_OK) return s;
  if (m >= kTuneMemoMinEdges) {
    g->fingerprint = graph_fingerprint(row_ptr, col_idx, n, m);
    recall_tuning(ctx, *g);
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  g->handle = ctx->next_graph++;
  *out = g->handle;
  ctx->graphs.emplace(g->handle, std::move(g));
  return BC_OK;
}

bc_status bc_create_graphs(bc_ctx *ctx, int32_t count, const int32_t *const *row_ptrs,
                           const int32_t *const *col_idxs, const int32_t *ns, const int64_t *ms,
                           bc_graph *out, int64_t *m_effective) {
  if (!ctx || count < 0) return BC_ERR_ARG;
  if (count > 0 && (!row_ptrs || !col_idxs || !ns || !ms || !out)) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  cudaStream_t st = ctx->stream;
  std::vector<std::unique_ptr<GraphRec>> made((size_t)count);
  std::vector<int64_t> meff((size_t)count, 0);
  auto fail = [&](bc_status s) {
    cudaStreamSynchronize(st);
    for (auto &g : made)
      if (g) {
        cudaFreeAsync(g->mem, st);
        ctx->used -= g->bytes;
      }
    cudaStreamSynchronize(st);
    return s;
  };
  for (int32_t i = 0; i < count; ++i) {
    const bc_status s = check_offsets(row_ptrs[i], col_idxs[i], ns[i], ms[i]);
    if (s != BC_OK) return s;
  }
  // Graphs prepared on the host go in groups of up to kGroupBytes of device
  // image: prepared on up to 16 threads, written to the pinned staging
  // buffer, copied with one transfer each and one synchronisation per group.
  // Larger graphs take the device path one by one.
  constexpr size_t kGroupBytes = (size_t)64 << 20;
  const int threads = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  auto parallel = [&](int items, const std::function<void(int)> &f) {
    std::atomic<int> next{0};
    auto work = [&]() {
      for (int t = next++; t < items; t = next++) f(t);
    };
    std::vector<std::thread> th;
    for (int i = 1; i < std::min(threads, items); ++i) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
  };
  int32_t i = 0;
  while (i < count) {
    if (ms[i] > kHostPrepMaxEdges) {
      const bc_status s = build_graph(ctx, row_ptrs[i], col_idxs[i], ns[i], ms[i], made[(size_t)i],
                                      &meff[(size_t)i]);
      if (s != BC_OK) return fail(s);
      ++i;
      continue;
    }
    int32_t j = i;
    size_t bound = 0;
    while (j < count && ms[j] <= kHostPrepMaxEdges) {
      Carver c;
      block_layout(ns[j], ms[j], [&](size_t cnt) { (void)c.take<int32_t>(cnt); });
      if (j > i && bound + c.off > kGroupBytes) break;
      bound += align_up(c.off, 256);
      ++j;
    }
    const int items = j - i;
    std::vector<HostPrep> hp((size_t)items);
    std::vector<bc_status> res((size_t)items, BC_OK);
    parallel(items, [&](int t) {
      res[(size_t)t] = prep_host(row_ptrs[i + t], col_idxs[i + t], ns[i + t], ms[i + t], hp[(size_t)t]);
    });
    for (bc_status s : res)
      if (s != BC_OK) return fail(s);
    std::vector<size_t> off((size_t)items + 1, 0);
    for (int t = 0; t < items; ++t) off[(size_t)t + 1] = off[(size_t)t] + hp[(size_t)t].bytes;
    bc_status s = ensure_stage(ctx, off[(size_t)items]);
    if (s != BC_OK) return fail(s);
    char *stage = static_cast<char *>(ctx->stage);
    parallel(items, [&](int t) { prep_image(hp[(size_t)t], stage + off[(size_t)t]); });
    std::vector<void *> mem((size_t)items, nullptr);
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < items && e == cudaSuccess && s == BC_OK; ++t) {
      if (ctx->used + hp[(size_t)t].bytes > ctx->budget) {
        s = BC_ERR_ADMISSION;
        break;
      }
      e = pool_alloc(ctx, &mem[(size_t)t], hp[(size_t)t].bytes, st);
      if (e == cudaSuccess) {
        ctx->used += hp[(size_t)t].bytes;
        e = cudaMemcpyAsync(mem[(size_t)t], stage + off[(size_t)t], hp[(size_t)t].bytes,
                            cudaMemcpyHostToDevice, st);
      } else {
        mem[(size_t)t] = nullptr;
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || s != BC_OK) {
      for (int t = 0; t < items; ++t)
        if (mem[(size_t)t]) {
          cudaFreeAsync(mem[(size_t)t], st);
          ctx->used -= hp[(size_t)t].bytes;
        }
      return fail(s != BC_OK ? s : cuda_status(e));
    }
    for (int t = 0; t < items; ++t) {
      meff[(size_t)(i + t)] = hp[(size_t)t].me;
      made[(size_t)(i + t)] = prep_graph(hp[(size_t)t], mem[(size_t)t]);
    }
    i = j;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  for (int32_t t = 0; t < count; ++t) {
    made[(size_t)t]->handle = ctx->next_graph++;
    out[t] = made[(size_t)t]->handle;
    if (m_effective) m_effective[t] = meff[(size_t)t];
    ctx->graphs.emplace(out[t], std::move(made[(size_t)t]));
  }
  return BC_OK;
}

bc_status bc_destroy_graph(bc_ctx *ctx, bc_graph h) {
  if (!ctx) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  std::unique_ptr<GraphRec> g;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->graphs.find(h);
    if (it == ctx->graphs.end()) return BC_ERR_GRAPH;
    if (it->second->active_jobs > 0) return BC_ERR_ARG;
    g = std::move(it->second);
    ctx->graphs.erase(it);
  }
  // graph memory comes from the stream-ordered pool: freed after every
  // earlier operation on the context's stream
  cudaFreeAsync(g->mem, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  ctx->used -= g->bytes;
  return BC_OK;
}

bc_status bc_exact(bc_ctx *ctx, bc_graph h, const bc_opts *opts, double *bc_out) {
  if (!ctx || !bc_out) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  GraphRec *g;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    g = find_graph(ctx, h);
  }
  if (!g) return BC_ERR_GRAPH;
  return run_sync(ctx, g, nullptr, g->dev.n, true, opts, bc_out, nullptr);
}

bc_status bc_sources(bc_ctx *ctx, bc_graph h, const int32_t *src, int32_t k, const bc_opts *opts,
                     double *bc_out) {
  if (!ctx || !bc_out) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  GraphRec *g;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    g = find_graph(ctx, h);
  }
  if (!g) return BC_ERR_GRAPH;
  bc_status s = check_sources(g, src, k);
  if (s != BC_OK) return s;
  return run_sync(ctx, g, src, k, false, opts, bc_out, nullptr);
}

namespace {

// Device buffers of the sampled-source estimator: running sums of the
// per-source terms and of their squares, the estimate and its error.
struct EstimateBufs {
  bc_ctx *ctx = nullptr;
  cudaStream_t st = nullptr;
  double *sum = nullptr, *sumsq = nullptr, *est = nullptr, *err = nullptr;
  unsigned long long *stat = nullptr;
  bc_status alloc(int64_t n) {
    const size_t b = sizeof(double) * (size_t)std::max<int64_t>(n, 1);
    BC_TRY(pool_alloc(ctx, &sum, b, st));
    BC_TRY(pool_alloc(ctx, &sumsq, b, st));
    BC_TRY(pool_alloc(ctx, &est, b, st));
    BC_TRY(pool_alloc(ctx, &err, b, st));
    BC_TRY(pool_alloc(ctx, &stat, sizeof(unsigned long long), st));
    BC_TRY(cudaMemsetAsync(sum, 0, b, st));
    BC_TRY(cudaMemsetAsync(sumsq, 0, b, st));
    return BC_OK;
  }
  ~EstimateBufs() {
    for (double *q : {sum, sumsq, est, err})
      if (q) cudaFreeAsync(q, st);
    if (stat) cudaFreeAsync(stat, st);
    if (st) cudaStreamSynchronize(st);
  }
};

// Output scale of the estimate: 1, or 1/((n-1)(n-2)) when normalising.
double estimate_factor(const bc_opts &o, int64_t n) {
  return o.normalize && n > 2 ? 1.0 / ((double)(n - 1) * (double)(n - 2)) : 1.0;
}

bc_status estimate_out(bc_ctx *ctx, EstimateBufs &b, int64_t n, int64_t k, const bc_opts &o,
                       double *est_out, double *err_out) {
  cudaStream_t st = ctx->stream;
  BC_TRY(launch_estimate(b.sum, b.sumsq, n, k, estimate_factor(o, n), b.est, b.err, st));
  const cudaMemcpyKind kind = o.out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (n > 0) {
    BC_TRY(cudaMemcpyAsync(est_out, b.est, sizeof(double) * (size_t)n, kind, st));
    BC_TRY(cudaMemcpyAsync(err_out, b.err, sizeof(double) * (size_t)n, kind, st));
  }
  BC_TRY(cudaStreamSynchronize(st));
  return BC_OK;
}

} // namespace

bc_status bc_sources_estimate(bc_ctx *ctx, bc_graph h, const int32_t *src, int32_t k,
                              const bc_opts *opts, double *est_out, double *stderr_out) {
  if (!ctx || !est_out || !stderr_out) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  GraphRec *g;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    g = find_graph(ctx, h);
  }
  if (!g) return BC_ERR_GRAPH;
  bc_status s = check_sources(g, src, k);
  if (s != BC_OK) return s;
  bc_opts o = opts ? *opts : default_opts();
  if (!opts_valid(o)) return BC_ERR_ARG;
  o.scale_sampled = 0; // the estimate carries its own n/k
  const int64_t n = g->dev.n;
  EstimateBufs b;
  b.ctx = ctx;
  b.st = ctx->stream;
  s = b.alloc(n);
  if (s != BC_OK) return s;
  if (k > 0) {
    s = run_sync(ctx, g, src, k, false, &o, nullptr, nullptr, b.sum, b.sumsq);
    if (s != BC_OK && s != BC_ERR_SIGMA_OVERFLOW) return s;
  }
  const bc_status so = estimate_out(ctx, b, n, k, o, est_out, stderr_out);
  return so != BC_OK ? so : s;
}

bc_status bc_sources_adaptive(bc_ctx *ctx, bc_graph h, const int32_t *order, int32_t max_k,
                              int32_t round, double rel_err, double min_est, const bc_opts *opts,
                              double *est_out, double *stderr_out, int32_t *k_used) {
  if (!ctx || !est_out || !stderr_out || !k_used || max_k < 1 || round < 1 || !(rel_err > 0.0))
    return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  GraphRec *g;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    g = find_graph(ctx, h);
  }
  if (!g) return BC_ERR_GRAPH;
  bc_status s = check_sources(g, order, max_k);
  if (s != BC_OK) return s;
  bc_opts o = opts ? *opts : default_opts();
  if (!opts_valid(o)) return BC_ERR_ARG;
  o.scale_sampled = 0;
  const int64_t n = g->dev.n;
  const double factor = estimate_factor(o, n);
  EstimateBufs b;
  b.ctx = ctx;
  b.st = ctx->stream;
  s = b.alloc(n);
  if (s != BC_OK) return s;
  cudaStream_t st = ctx->stream;
  int64_t done = 0;
  bc_status worst = BC_OK;
  std::vector<int32_t> flagged; // overflowing sources of every round
  while (done < max_k) {
    const int64_t r = std::min<int64_t>(round, max_k - done);
    s = run_sync(ctx, g, order + done, r, false, &o, nullptr, nullptr, b.sum, b.sumsq);
    if (s != BC_OK && s != BC_ERR_SIGMA_OVERFLOW) return s;
    if (s != BC_OK) worst = s;
    flagged.insert(flagged.end(), ctx->last_ovf.begin(), ctx->last_ovf.end());
    done += r;
    if (done < 2) continue;
    // stop once every vertex whose estimate reaches min_est has a standard
    // error of at most rel_err times its estimate
    unsigned long long bits = 0;
    BC_TRY(launch_estimate(b.sum, b.sumsq, n, done, factor, b.est, b.err, st));
    BC_TRY(cudaMemsetAsync(b.stat, 0, sizeof(unsigned long long), st));
    BC_TRY(launch_max_rel_err(b.est, b.err, n, min_est, b.stat, st));
    BC_TRY(cudaMemcpyAsync(&bits, b.stat, sizeof(bits), cudaMemcpyDeviceToHost, st));
    BC_TRY(cudaStreamSynchronize(st));
    double worst_rel;
    std::memcpy(&worst_rel, &bits, sizeof(double));
    if (worst_rel <= rel_err) break;
  }
  *k_used = (int32_t)done;
  std::sort(flagged.begin(), flagged.end());
  ctx->last_ovf = std::move(flagged);
  const bc_status so = estimate_out(ctx, b, n, done, o, est_out, stderr_out);
  return so != BC_OK ? so : worst;
}

bc_status bc_submit(bc_ctx *ctx, bc_graph h, const int32_t *src, int32_t k, const bc_opts *opts,
                    bc_job *out) {
  if (!ctx || !out) return BC_ERR_ARG;
  bc_opts o = opts ? *opts : default_opts();
  if (!opts_valid(o) || o.out_device) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  auto j = std::make_unique<JobRec>();
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    GraphRec *g = find_graph(ctx, h);
    if (!g) return BC_ERR_GRAPH;
    j->g = g;
  }
  if (src) {
    bc_status s = check_sources(j->g, src, k);
    if (s != BC_OK) return s;
    j->src.assign(src, src + k);
    j->k = k;
  } else {
    j->all_sources = true;
    j->k = j->g->dev.n;
  }
  j->opts = o;
  j->n = j->g->dev.n;
  const int sched = resolve_schedule(o, j->g->dev);
  j->footprint = job_footprint(*j->g, sched, o, j->k);
  if (j->footprint > ctx->budget) return BC_ERR_ADMISSION;
  if (pin_get(ctx, &j->h_out, sizeof(double) * (size_t)std::max<int64_t>(j->n, 1)) != cudaSuccess)
    return BC_ERR_OOM;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->stop) {
    pin_put(ctx, j->h_out, sizeof(double) * (size_t)std::max<int64_t>(j->n, 1));
    return BC_ERR_ARG;
  }
  j->handle = ctx->next_job++;
  *out = j->handle;
  j->g->active_jobs++;
  ctx->pending.push_back(j.get());
  ctx->jobs.emplace(j->handle, std::move(j));
  ctx->cv.notify_all();
  return BC_OK;
}

static bc_status take_result(bc_ctx *ctx, std::map<int64_t, std::unique_ptr<JobRec>>::iterator it,
                             double *bc_out, bc_stats *stats) {
  JobRec *j = it->second.get();
  // the graph may be gone by now (destroyed after the job finished)
  if (bc_out && j->n) std::memcpy(bc_out, j->h_out, sizeof(double) * (size_t)j->n);
  if (stats) *stats = j->stats;
  bc_status s = j->status;
  pin_put(ctx, j->h_out, sizeof(double) * (size_t)std::max<int64_t>(j->n, 1));
  ctx->jobs.erase(it);
  return s;
}

bc_status bc_poll(bc_ctx *ctx, bc_job job, double *bc_out, bc_stats *stats) {
  if (!ctx) return BC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->jobs.find(job);
  if (it == ctx->jobs.end()) return BC_ERR_NOT_FOUND;
  if (!it->second->done) return BC_PENDING;
  return take_result(ctx, it, bc_out, stats);
}

bc_status bc_wait(bc_ctx *ctx, bc_job job, int64_t timeout_ms, double *bc_out, bc_stats *stats) {
  if (!ctx) return BC_ERR_ARG;
  std::unique_lock<std::mutex> lk(ctx->mu);
  auto it = ctx->jobs.find(job);
  if (it == ctx->jobs.end()) return BC_ERR_NOT_FOUND;
  JobRec *j = it->second.get();
  auto ready = [&] { return j->done; };
  if (timeout_ms < 0) {
    ctx->cv.wait(lk, ready);
  } else if (!ctx->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return BC_ERR_TIMEOUT;
  }
  return take_result(ctx, ctx->jobs.find(job), bc_out, stats);
}

bc_status bc_last_stats(bc_ctx *ctx, bc_stats *stats) {
  if (!ctx || !stats) return BC_ERR_ARG;
  *stats = ctx->last;
  return BC_OK;
}

bc_status bc_last_overflow_sources(bc_ctx *ctx, int32_t *src_out, int32_t capacity,
                                   int32_t *count) {
  if (!ctx || !count || capacity < 0 || (capacity > 0 && !src_out)) return BC_ERR_ARG;
  *count = (int32_t)ctx->last_ovf.size();
  const size_t w = std::min<size_t>((size_t)capacity, ctx->last_ovf.size());
  if (w) std::memcpy(src_out, ctx->last_ovf.data(), sizeof(int32_t) * w);
  return BC_OK;
}

bc_status bc_debug_sources(bc_ctx *ctx, bc_graph h, const int32_t *src, int32_t k,
                           const bc_opts *opts, int32_t *d_out, uint64_t *sigma_out,
                           double *delta_out) {
  if (!ctx) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  GraphRec *g;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    g = find_graph(ctx, h);
  }
  if (!g) return BC_ERR_GRAPH;
  bc_status s = check_sources(g, src, k);
  if (s != BC_OK) return s;
  bc_opts o = opts ? *opts : default_opts();
  o.out_device = 0;
  const size_t cells = (size_t)k * (size_t)g->dev.n;
  DebugOut dbg;
  cudaStream_t st = ctx->stream;
  BC_TRY(pool_alloc(ctx, &dbg.d, sizeof(int32_t) * std::max<size_t>(cells, 1), st));
  BC_TRY(pool_alloc(ctx, &dbg.sigma, sizeof(uint64_t) * std::max<size_t>(cells, 1), st));
  BC_TRY(pool_alloc(ctx, &dbg.delta, sizeof(double) * std::max<size_t>(cells, 1), st));
  BC_TRY(cudaMemsetAsync(dbg.d, 0xff, sizeof(int32_t) * cells, st));
  BC_TRY(cudaMemsetAsync(dbg.sigma, 0, sizeof(uint64_t) * cells, st));
  BC_TRY(cudaMemsetAsync(dbg.delta, 0, sizeof(double) * cells, st));
  std::vector<double> tmp((size_t)std::max<int32_t>(g->dev.n, 1));
  s = run_sync(ctx, g, src, k, false, &o, tmp.data(), &dbg);
  if (s == BC_OK || s == BC_ERR_SIGMA_OVERFLOW) {
    cudaError_t e = cudaSuccess;
    if (d_out && cells) e = cudaMemcpyAsync(d_out, dbg.d, sizeof(int32_t) * cells, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && sigma_out && cells) e = cudaMemcpyAsync(sigma_out, dbg.sigma, sizeof(uint64_t) * cells, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && delta_out && cells) e = cudaMemcpyAsync(delta_out, dbg.delta, sizeof(double) * cells, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e);
  }
  cudaFreeAsync(dbg.d, st);
  cudaFreeAsync(dbg.sigma, st);
  cudaFreeAsync(dbg.delta, st);
  cudaStreamSynchronize(st);
  return s;
}

bc_status bc_debug_source(bc_ctx *ctx, bc_graph h, int32_t s, int32_t *d_out, uint64_t *sigma_out,
                          double *delta_out) {
  bc_opts o = default_opts();
  o.schedule = BC_SCHED_PLAIN;
  o.delta_fp64 = 1;
  return bc_debug_sources(ctx, h, &s, 1, &o, d_out, sigma_out, delta_out);
}

bc_status bc_debug_graph(bc_ctx *ctx, bc_graph h, int32_t *row_ptr, int32_t *col_idx,
                         int32_t *in_ptr, int32_t *in_idx) {
  if (!ctx) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  GraphRec *g = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    g = find_graph(ctx, h);
  }
  if (!g) return BC_ERR_GRAPH;
  const GraphDev &d = g->dev;
  cudaStream_t st = ctx->stream;
  const size_t np1 = sizeof(int32_t) * ((size_t)d.n + 1), mb = sizeof(int32_t) * (size_t)d.m;
  if (row_ptr) BC_TRY(cudaMemcpyAsync(row_ptr, d.row_ptr, np1, cudaMemcpyDeviceToHost, st));
  if (col_idx && mb) BC_TRY(cudaMemcpyAsync(col_idx, d.col_idx, mb, cudaMemcpyDeviceToHost, st));
  if (in_ptr) BC_TRY(cudaMemcpyAsync(in_ptr, d.in_ptr, np1, cudaMemcpyDeviceToHost, st));
  if (in_idx && mb) BC_TRY(cudaMemcpyAsync(in_idx, d.in_idx, mb, cudaMemcpyDeviceToHost, st));
  BC_TRY(cudaStreamSynchronize(st));
  return BC_OK;
}

bc_status bc_exact_many(bc_ctx *ctx, const bc_graph *graphs, int32_t count, const bc_opts *opts,
                        double *bc_out) {
  if (!ctx || (count > 0 && (!graphs || !bc_out)) || count < 0) return BC_ERR_ARG;
  DeviceGuard dg(ctx->device);
  bc_opts o = opts ? *opts : default_opts();
  if (!opts_valid(o)) return BC_ERR_ARG;
  std::vector<GraphRec *> gs((size_t)count);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (int32_t i = 0; i < count; ++i)
      if (!(gs[(size_t)i] = find_graph(ctx, graphs[i]))) return BC_ERR_GRAPH;
  }
  const bool fp64 = o.delta_fp64 != 0;
  if (o.batch_k > kK) return BC_ERR_ARG; // one block per graph: up to 64 sources per batch
  const int kb = o.batch_k == 0 ? kK : o.batch_k;
  std::vector<int64_t> off((size_t)count + 1, 0);
  for (int32_t i = 0; i < count; ++i) off[(size_t)i + 1] = off[(size_t)i] + gs[(size_t)i]->dev.n;
  const int64_t total_n = off[(size_t)count];
  // schedule per graph: graphs up to kManyMaxN vertices share the persistent
  // many-graph launch; larger ones use the grid-wide batched kernel
  constexpr int32_t kManyMaxN = 8192;
  std::vector<int32_t> small, big;
  int32_t max_n = 1;
  int64_t max_hv = 1, max_hc = 1;
  for (int32_t i = 0; i < count; ++i) {
    const GraphDev &gd = gs[(size_t)i]->dev;
    if (gd.n <= kManyMaxN) {
      small.push_back(i);
      max_n = std::max(max_n, gd.n);
      max_hv = std::max(max_hv, gd.heavy_vertices);
      max_hc = std::max(max_hc, gd.heavy_chunks);
    } else {
      big.push_back(i);
    }
  }
  // largest work first (longest-processing-time order)
  std::sort(small.begin(), small.end(), [&](int32_t a, int32_t b) {
    const GraphDev &x = gs[(size_t)a]->dev, &y = gs[(size_t)b]->dev;
    return (double)x.n * (double)(x.m + x.n) > (double)y.n * (double)(y.m + y.n);
  });
  cudaStream_t st = ctx->stream;
  double *d_out = nullptr;
  int8_t *d_ovf = nullptr;
  unsigned long long *d_cnt = nullptr;
  BC_TRY(pool_alloc(ctx, &d_out, sizeof(double) * (size_t)std::max<int64_t>(total_n, 1), st));
  BC_TRY(pool_alloc(ctx, &d_ovf, (size_t)std::max<int64_t>(total_n, 1), st));
  BC_TRY(pool_alloc(ctx, &d_cnt, sizeof(unsigned long long) * (CNT_N + 1), st));
  BC_TRY(cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)std::max<int64_t>(total_n, 1), st));
  BC_TRY(cudaMemsetAsync(d_ovf, 0, (size_t)std::max<int64_t>(total_n, 1), st));
  BC_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * (CNT_N + 1), st));
  bc_stats total{};
  total.kernel_kind = 2;
  float many_ms = 0.f;
  bc_status status = BC_OK;
  void *ws_mem = nullptr;
  Work *d_works = nullptr;
  GraphDev *d_graphs = nullptr;
  int32_t *d_order = nullptr, *d_iota = nullptr, *d_trav = nullptr;
  int64_t *d_off = nullptr;
  // sources each small graph runs: with grouped batches, its vertices with
  // out-edges (first in its batch order; a source without out-edges reaches
  // nothing and adds nothing to BC)
  const bool grouped = o.source_order == 0;
  std::vector<int32_t> trav((size_t)count, 0);
  for (int32_t i : small) {
    GraphRec &gr = *gs[(size_t)i];
    int32_t t = gr.dev.n;
    if (grouped && gr.dev.order && !gr.order.empty()) {
      t = gr.with_out.load();
      if (t < 0) { // counted once per graph (concurrent callers store the same count)
        t = 0;
        for (int32_t v = 0; v < gr.dev.n; ++v) t += gr.row_ptr[(size_t)v + 1] != gr.row_ptr[(size_t)v];
        gr.with_out = t;
      }
    }
    trav[(size_t)i] = t;
  }
  unsigned *d_next = nullptr;
  if (!small.empty()) {
    // one workspace per thread block, sized for the largest small graph
    WsRec proto;
    // widest masks any of the graphs takes (each picks its own in the kernel)
    const int max_words = o.batch_k == 0 ? kMaxWords : 1;
    int ws_words = 1;
    for (int32_t i : small) ws_words = std::max(ws_words, auto_words(gs[(size_t)i]->dev.n, max_words));
    proto.kind = WS_QUEUE;
    proto.words = ws_words;
    proto.batch = true;
    proto.n = max_n;
    proto.cap = (int64_t)max_n * kb;
    proto.hcap = max_hv * kb;
    proto.chunk_cap = max_hc;
    const size_t stride = ws_layout(proto, nullptr);
    int grid = ctx->grid_many[fp64];
    const size_t ws_budget = (ctx->budget > ctx->used ? ctx->budget - ctx->used : 0) / 2;
    grid = (int)std::min<int64_t>(grid, std::max<int64_t>(1, (int64_t)(ws_budget / stride)));
    grid = (int)std::min<int64_t>(grid, (int64_t)small.size());
    auto release = [&] {
      cudaFreeAsync(d_out, st);
      cudaFreeAsync(d_ovf, st);
      cudaFreeAsync(d_cnt, st);
    };
    if (grid < 1 || stride * (size_t)grid > ws_budget) {
      release();
      return BC_ERR_ADMISSION;
    }
    const cudaError_t ea = cudaMalloc(&ws_mem, stride * (size_t)grid);
    if (ea != cudaSuccess) {
      ws_mem = nullptr;
      release();
      return cuda_status(ea);
    }
    std::vector<Work> works((size_t)grid);
    for (int c = 0; c < grid; ++c) {
      WsRec r = proto;
      ws_layout(r, static_cast<char *>(ws_mem) + stride * (size_t)c);
      works[(size_t)c] = r.w;
    }
    std::vector<GraphDev> table((size_t)count);
    for (int32_t i = 0; i < count; ++i) table[(size_t)i] = gs[(size_t)i]->dev;
    std::vector<int32_t> iota((size_t)max_n);
    for (int32_t i = 0; i < max_n; ++i) iota[(size_t)i] = i;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
      if (e == cudaSuccess) e = pool_alloc(ctx, ptr, std::max<size_t>(bytes, 1), st);
    };
    alloc(reinterpret_cast<void **>(&d_works), sizeof(Work) * works.size());
    alloc(reinterpret_cast<void **>(&d_graphs), sizeof(GraphDev) * table.size());
    alloc(reinterpret_cast<void **>(&d_order), sizeof(int32_t) * small.size());
    alloc(reinterpret_cast<void **>(&d_iota), sizeof(int32_t) * iota.size());
    alloc(reinterpret_cast<void **>(&d_off), sizeof(int64_t) * off.size());
    alloc(reinterpret_cast<void **>(&d_trav), sizeof(int32_t) * trav.size());
    alloc(reinterpret_cast<void **>(&d_next), sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(ws_mem, 0, stride * (size_t)grid, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_works, works.data(), sizeof(Work) * works.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_graphs, table.data(), sizeof(GraphDev) * table.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, small.data(), sizeof(int32_t) * small.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_iota, iota.data(), sizeof(int32_t) * iota.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && count) e = cudaMemcpyAsync(d_trav, trav.data(), sizeof(int32_t) * trav.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, sizeof(unsigned), st);
    ManyParams mp;
    mp.base.ovf_flags = d_ovf;
    mp.base.job_cnt = d_cnt;
    mp.graphs = d_graphs;
    mp.order = d_order;
    mp.out_off = d_off;
    mp.count = (int32_t)small.size();
    mp.works = d_works;
    mp.iota = d_iota;
    mp.out = d_out;
    mp.next = d_next;
    mp.kb = kb;
    mp.max_words = ws_words;
    total.mask_words = std::max(total.mask_words, ws_words);
    mp.grouped = grouped ? 1 : 0;
    mp.traverse = d_trav;
    mp.counts64 = o.count_bits == 64 ? 1 : 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_many(mp, fp64, grid, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    // the block workspaces' control words carry any device error: the first
    // one found is gathered into block 0's and read back once
    int err0 = 0;
    if (e == cudaSuccess) e = launch_gather_err(works[0].ctl, stride, grid, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&err0, &works[0].ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) cudaEventElapsedTime(&many_ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) status = cuda_status(e);
    if (status == BC_OK && err0) status = BC_ERR_INTERNAL;
    for (int32_t i : small) {
      const int64_t gn = gs[(size_t)i]->dev.n;
      const int64_t gkb = ws_words > 1 ? kK * auto_words(gn, ws_words) : kb;
      total.batches += (trav[(size_t)i] + gkb - 1) / gkb;
    }
    total.kernel_launches += 2;
  }
  // larger graphs, one grid-wide job each, straight into the device result
  for (int32_t i : big) {
    if (status != BC_OK) break;
    bc_opts od = o;
    od.out_device = 1;
    od.normalize = 0;
    od.schedule = BC_SCHED_BATCH;
    status = run_sync(ctx, gs[(size_t)i], nullptr, gs[(size_t)i]->dev.n, true, &od,
                      d_out + off[(size_t)i], nullptr);
    if (status == BC_OK) {
      total.batches += ctx->last.batches;
      total.kernel_launches += ctx->last.kernel_launches;
      total.device_ms += ctx->last.device_ms;
      total.max_levels = std::max(total.max_levels, ctx->last.max_levels);
      total.frontier_entries += ctx->last.frontier_entries;
      total.scanned_out_edges += ctx->last.scanned_out_edges;
      total.scanned_in_edges += ctx->last.scanned_in_edges;
      total.dag_pairs += ctx->last.dag_pairs;
      total.reached_pairs += ctx->last.reached_pairs;
      total.heavy_chunks += ctx->last.heavy_chunks;
      total.levels_sum += ctx->last.levels_sum;
      total.push_levels += ctx->last.push_levels;
      total.mask_words = std::max(total.mask_words, ctx->last.mask_words);
    }
  }
  // per-graph normalisation, result copy, counters of the persistent launch
  std::vector<unsigned long long> cnt(CNT_N + 1, 0);
  std::vector<int8_t> ovf((size_t)std::max<int64_t>(total_n, 1), 0);
  if (status == BC_OK) {
    cudaError_t e = cudaSuccess;
    if (o.normalize)
      for (int32_t i = 0; i < count && e == cudaSuccess; ++i) {
        const int64_t n = gs[(size_t)i]->dev.n;
        if (n > 2)
          e = launch_scale(d_out + off[(size_t)i], d_out + off[(size_t)i], n,
                           1.0 / ((double)(n - 1) * (double)(n - 2)), st);
      }
    if (e == cudaSuccess && total_n)
      e = cudaMemcpyAsync(bc_out, d_out, sizeof(double) * (size_t)total_n,
                          o.out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && total_n)
      e = cudaMemcpyAsync(ovf.data(), d_ovf, (size_t)total_n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) status = cuda_status(e);
  }
  cudaFreeAsync(d_out, st);
  cudaFreeAsync(d_ovf, st);
  cudaFreeAsync(d_cnt, st);
  if (d_works) cudaFreeAsync(d_works, st);
  if (d_graphs) cudaFreeAsync(d_graphs, st);
  if (d_order) cudaFreeAsync(d_order, st);
  if (d_iota) cudaFreeAsync(d_iota, st);
  if (d_off) cudaFreeAsync(d_off, st);
  if (d_trav) cudaFreeAsync(d_trav, st);
  if (d_next) cudaFreeAsync(d_next, st);
  cudaStreamSynchronize(st);
  if (ws_mem) cudaFree(ws_mem);
  if (status != BC_OK) return status;
  for (int32_t i = 0; i < count; ++i) {
    total.n += gs[(size_t)i]->dev.n;
    total.m += gs[(size_t)i]->dev.m;
  }
  total.sources = total_n;
  total.device_ms += many_ms;
  total.frontier_entries += (int64_t)cnt[CNT_ENTRIES];
  total.scanned_out_edges += (int64_t)cnt[CNT_OUT_EDGES];
  total.scanned_in_edges += (int64_t)cnt[CNT_IN_EDGES];
  total.dag_pairs += (int64_t)cnt[CNT_DAG];
  total.reached_pairs += (int64_t)cnt[CNT_REACHED];
  total.heavy_chunks += (int64_t)cnt[CNT_HEAVY];
  total.levels_sum += (int32_t)cnt[CNT_LEVELS];
  total.max_levels = std::max(total.max_levels, (int32_t)cnt[CNT_MAXLEV]);
  int32_t novf = 0;
  for (int64_t i = 0; i < total_n; ++i) novf += ovf[(size_t)i] ? 1 : 0;
  total.overflow_sources += novf;
  ctx->last = total;
  return novf ? BC_ERR_SIGMA_OVERFLOW : BC_OK;
}

bc_status bc_debug_inject_barrier_skip(bc_ctx *ctx, int32_t block, int32_t timeout_ms) {
  if (!ctx || timeout_ms < 0) return BC_ERR_ARG;
  ctx->inject_block = block;
  ctx->inject_timeout_ms = timeout_ms;
  return BC_OK;
}

} // extern "C"
