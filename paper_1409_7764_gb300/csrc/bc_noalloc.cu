// bc_sources_noalloc: betweenness centrality over a source list for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need BC: code
// that runs under a fixed, pre-reserved memory budget (embedded or
// safety-certified deployments where every allocation happens at start-up),
// frameworks whose own caching allocator owns all device memory and forbids
// side allocations, or callbacks where an allocation could stall on a device
// synchronisation.  This entry point takes the graph and the output as
// device memory the caller already owns and keeps all of its working state in
// one fixed array compiled into this library, so a call allocates nothing.
//
// The working state lives in g_noalloc_scratch below (about 15 MB per GPU,
// held by every GPU that loads this library for the life of the process).
// Its size fixes the largest graph: n <= BC_NOALLOC_MAX_N vertices.  It runs
// the same batched kernel as bc_sources (64 sources per launch), with every
// vertex handled by a single warp (no splitting of high-degree vertices,
// which would need scratch proportional to the edge count).
#include "bc_internal.cuh"
#include "bc_gb300.h"

#include <algorithm>
#include <cstring>
#include <atomic>
#include <mutex>

using namespace bcgpu;

namespace {

constexpr int64_t kNoAllocMaxN = BC_NOALLOC_MAX_N;
constexpr int64_t kNoAllocCap = kNoAllocMaxN * kK; // frontier entries: each vertex, each source
constexpr int kMaxDevices = 64;

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of every array inside the scratch block.
struct ScratchLayout {
  size_t ctl, vis, fr, qm, qv, qoff, hpack, hoff, hq_e, hq_c, harrive, partial, partial_ovf,
      sigma, cdep, src, ovf, cnt, nch, total;
};

constexpr ScratchLayout make_layout() {
  ScratchLayout o{};
  size_t at = 0;
  auto take = [&at](size_t bytes) {
    size_t here = at;
    at = al256(at + bytes);
    return here;
  };
  const size_t n = (size_t)kNoAllocMaxN;
  o.ctl = take(sizeof(Ctl));
  o.vis = take(8 * n);
  o.fr = take(8 * 4 * n);
  o.qm = take(8 * (size_t)kNoAllocCap);
  o.qv = take(4 * (size_t)kNoAllocCap);
  o.qoff = take(8 * (n + 3));
  o.hpack = take(8 * (n + 3));
  o.hoff = take(8 * (n + 3));
  o.hq_e = take(8);
  o.hq_c = take(8);
  o.harrive = take(4);
  o.partial = take(8 * kK);
  o.partial_ovf = take(8);
  o.sigma = take(8 * n * kK);
  o.cdep = take(8 * n * kK);
  o.src = take(4 * kK);
  o.ovf = take(kK);
  o.cnt = take(8 * CNT_N);
  o.nch = take(4 * n);
  o.total = at;
  return o;
}

constexpr ScratchLayout kLay = make_layout();

// The fixed working state.  In host code this name is only a stand-in for
// the device array, never a usable address: the address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kLay.total];

struct DeviceSetup {
  std::mutex mu;
  std::atomic<bool> ready{false}; // set once, only after a successful set-up
  unsigned char *base = nullptr;
  int grid[2] = {0, 0};
};

DeviceSetup g_setup[kMaxDevices];

// Per-device set-up, run with the device current by the first call on that
// device that finds it missing: resolve the scratch array's device address
// and the co-resident grid size of the batched kernel.  Neither allocates.
// Only success is remembered; a failed attempt is retried by the next call.
// An error already pending on this thread (left by earlier, unrelated work)
// is reported as it is and not cleared, so the lookup below is never blamed
// for it and the caller still sees it.
cudaError_t ensure_setup(int dev) {
  DeviceSetup &s = g_setup[dev];
  if (s.ready.load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(s.mu);
  if (s.ready.load(std::memory_order_relaxed)) return cudaSuccess;
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return e;
  void *ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  int grid[2];
  for (int f = 0; f < 2; ++f) {
    grid[f] = max_grid_batch(f != 0, dev);
    if (grid[f] <= 0) return cudaErrorUnknown;
  }
  s.base = static_cast<unsigned char *>(ptr);
  s.grid[0] = grid[0];
  s.grid[1] = grid[1];
  s.ready.store(true, std::memory_order_release);
  return cudaSuccess;
}

bc_status to_status(cudaError_t e) {
  return e == cudaSuccess ? BC_OK : BC_ERR_CUDA;
}

} // namespace

extern "C" bc_status bc_sources_noalloc(const int32_t *row_ptr, const int32_t *col_idx,
                                        const int32_t *in_ptr, const int32_t *in_idx, int32_t n,
                                        int64_t m, const int32_t *src, int32_t k,
                                        int32_t delta_fp64, double *bc_out, void *cuda_stream) {
  if (n < 0 || n > kNoAllocMaxN) return BC_ERR_ARG;
  if (m < 0 || m >= ((int64_t)1 << 31) || k < 0) return BC_ERR_ARG;
  if (delta_fp64 != 0 && delta_fp64 != 1) return BC_ERR_ARG;
  if (k > 0 && !src) return BC_ERR_ARG;
  if (n > 0 && (!row_ptr || !in_ptr || !bc_out)) return BC_ERR_ARG;
  if (m > 0 && (!col_idx || !in_idx)) return BC_ERR_ARG;
  for (int32_t i = 0; i < k; ++i)
    if (src[i] < 0 || src[i] >= n) return BC_ERR_ARG;
  if (n == 0) return BC_OK;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BC_ERR_CUDA;
  if (ensure_setup(dev) != cudaSuccess) return BC_ERR_CUDA;
  DeviceSetup &ds = g_setup[dev];

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char *b = ds.base;
  const bool fp64 = delta_fp64 != 0;
  const size_t nn = (size_t)n;

  KParams p;
  p.g.n = n;
  p.g.m = m;
  p.g.row_ptr = row_ptr;
  p.g.col_idx = col_idx;
  p.g.in_ptr = in_ptr;
  p.g.in_idx = in_idx;
  p.g.nchunks = reinterpret_cast<const int32_t *>(b + kLay.nch);
  p.g.heavy_vertices = 0;
  p.g.heavy_chunks = 0;
  Work &w = p.w;
  w.n = n;
  w.k_max = kK;
  w.ctl = reinterpret_cast<Ctl *>(b + kLay.ctl);
  w.vis = reinterpret_cast<uint64_t *>(b + kLay.vis);
  w.fr = reinterpret_cast<uint64_t *>(b + kLay.fr);
  w.qm = reinterpret_cast<uint64_t *>(b + kLay.qm);
  w.qv = reinterpret_cast<int32_t *>(b + kLay.qv);
  w.cap = (int64_t)n * kK;
  w.qoff = reinterpret_cast<int64_t *>(b + kLay.qoff);
  w.hpack = reinterpret_cast<unsigned long long *>(b + kLay.hpack);
  w.hoff = reinterpret_cast<int64_t *>(b + kLay.hoff);
  w.hq_e = reinterpret_cast<int64_t *>(b + kLay.hq_e);
  w.hq_c = reinterpret_cast<int64_t *>(b + kLay.hq_c);
  w.harrive = reinterpret_cast<unsigned *>(b + kLay.harrive);
  w.hcap = 1;
  w.partial = b + kLay.partial;
  w.partial_ovf = reinterpret_cast<uint64_t *>(b + kLay.partial_ovf);
  w.chunk_cap = 1;
  w.sigma = reinterpret_cast<uint64_t *>(b + kLay.sigma);
  w.cdep = b + kLay.cdep;
  int32_t *d_src = reinterpret_cast<int32_t *>(b + kLay.src);
  int8_t *d_ovf = reinterpret_cast<int8_t *>(b + kLay.ovf);
  p.bc = bc_out;
  p.ovf_flags = d_ovf;
  p.job_cnt = reinterpret_cast<unsigned long long *>(b + kLay.cnt);
  p.src_base = 0;

  // The array keeps whatever the previous call left; everything the kernel
  // expects to start at zero is cleared here, as is the output.  (Path counts
  // and coefficients are only read where the same batch wrote them.)
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.vis, 0, 8 * nn, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.fr, 0, 8 * 4 * nn, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.harrive, 0, 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ovf, 0, kK, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.job_cnt, 0, 8 * CNT_N, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + kLay.nch, 0, 4 * nn, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bc_out, 0, 8 * nn, st);
  if (e != cudaSuccess) return to_status(e);

  const int64_t want = ((int64_t)n * 8 + kBlock - 1) / kBlock; // ~8 threads per vertex
  int grid = (int)std::min<int64_t>(ds.grid[fp64], std::max<int64_t>(2, want));
  for (int32_t b0 = 0; b0 < k; b0 += kK) {
    const int32_t kb = std::min<int32_t>(kK, k - b0);
    // stream-ordered after the previous batch's kernel, so the slot is free
    e = cudaMemcpyAsync(d_src, src + b0, sizeof(int32_t) * (size_t)kb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return to_status(e);
    p.src = d_src;
    p.k = kb;
    e = launch_batch(p, fp64, grid, st);
    while (e == cudaErrorCooperativeLaunchTooLarge && grid > 1) {
      // fewer blocks fit at once than at set-up (e.g. the GPU is partitioned
      // differently now): the launch was refused before running; clear that
      // error and retry with half the grid (the kernel works with any grid)
      (void)cudaGetLastError();
      grid /= 2;
      e = launch_batch(p, fp64, grid, st);
    }
    if (e != cudaSuccess) return to_status(e);
  }

  int kerr = 0;
  int8_t ovf[kK];
  e = cudaMemcpyAsync(&kerr, &w.ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ovf, d_ovf, sizeof(ovf), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return to_status(e);
  if (kerr == KERR_TIMEOUT) return BC_ERR_TIMEOUT;
  if (kerr != KERR_NONE) return BC_ERR_INTERNAL;
  for (int j = 0; j < kK; ++j)
    if (ovf[j]) return BC_ERR_SIGMA_OVERFLOW;
  return BC_OK;
}
