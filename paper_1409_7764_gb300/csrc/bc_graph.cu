// Device-side preparation of a resident graph: the in-CSR (transpose) of the
// canonical out-CSR, the per-vertex chunk counts of high-degree vertices for
// every candidate chunk size, and the batch-composition key (two-hop walk
// counts).  All linear in n + m; the host only validates, canonicalises when
// needed and prefix-sums the in-degrees.
#include "bc_internal.cuh"

#include <algorithm>

namespace bcgpu {
namespace {

constexpr int kPrepBlock = 256;

// Validation of an uploaded out-CSR (offsets already checked on the host):
// flags[0] |= 1 for a neighbour id outside [0, n); flags[1] |= 1 when a row
// is not canonical (unsorted, duplicate, or a self-loop).  One warp per row.
__global__ void check_csr_kernel(const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col_idx, int32_t n,
                                 int *__restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool bad = false, noncanon = false;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t b = row_ptr[v], e = row_ptr[v + 1];
    for (int32_t i = b + lane; i < e; i += 32) {
      const int32_t x = col_idx[i];
      if (x < 0 || x >= n) bad = true;
      if (x == v || (i > b && x <= col_idx[i - 1])) noncanon = true;
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, 1);
  if (__any_sync(0xffffffffu, noncanon) && lane == 0) atomicOr(flags + 1, 1);
}

// In-degree counts: cnt[x + 1] += 1 for every edge into x.
__global__ void in_degree_kernel(const int32_t *__restrict__ col_idx, int64_t m,
                                 int32_t *__restrict__ cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + col_idx[e] + 1, 1);
}

// Scatter of the edges into the in-CSR, one warp per source vertex (lanes
// over its out-edges); fill[x] starts at in_ptr[x].  The order inside an
// in-row depends on the atomics' order, so the rows are sorted afterwards
// (sort_rows_*: ascending sources, as a sequential transpose would give).
__global__ void in_scatter_kernel(const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col_idx, int32_t n,
                                  int32_t *__restrict__ fill, int32_t *__restrict__ in_idx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t b = row_ptr[v], e = row_ptr[v + 1];
    for (int32_t i = b + lane; i < e; i += 32) {
      const int32_t x = col_idx[i];
      in_idx[atomicAdd(fill + x, 1)] = (int32_t)v;
    }
  }
}

// Per vertex: chunk counts for each candidate chunk size (0 when in+out
// degree fits one chunk), the heavy-vertex and chunk totals per size, and the
// number of two-hop walks leaving it (sum of its out-neighbours' out-degrees).
__global__ void graph_keys_kernel(const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col_idx,
                                  const int32_t *__restrict__ in_ptr, int32_t n,
                                  int32_t *__restrict__ nchunks, int64_t *__restrict__ two,
                                  unsigned long long *__restrict__ totals) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t b = row_ptr[v], e = row_ptr[v + 1];
    long long t = 0;
    for (int32_t i = b + lane; i < e; i += 32) {
      const int32_t x = col_idx[i];
      t += row_ptr[x + 1] - row_ptr[x];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) {
      two[v] = t;
      const int64_t cost = (int64_t)(e - b) + (in_ptr[v + 1] - in_ptr[v]);
      constexpr int64_t kSizes[kChunkVariants] = {kChunkCandidates[0], kChunkCandidates[1],
                                                   kChunkCandidates[2]};
#pragma unroll
      for (int c = 0; c < kChunkVariants; ++c) {
        const int64_t ch = kSizes[c];
        int32_t nc = 0;
        if (cost > ch) {
          nc = (int32_t)((cost + ch - 1) / ch);
          atomicAdd(totals + 2 * c, 1ull);
          atomicAdd(totals + 2 * c + 1, (unsigned long long)nc);
        }
        nchunks[(size_t)c * n + v] = nc;
      }
    }
  }
}

// Sorts the in-rows listed in rows[] (2..32 entries each), one warp per row:
// a bitonic network over the lanes, padded with INT_MAX.
__global__ void sort_rows_warp_kernel(const int32_t *__restrict__ in_ptr,
                                      int32_t *__restrict__ in_idx,
                                      const int32_t *__restrict__ rows, int32_t nrows) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < nrows; r += nwarps) {
    const int32_t x = rows[r];
    const int32_t b = in_ptr[x], len = in_ptr[x + 1] - b;
    int32_t v = lane < len ? in_idx[b + lane] : 0x7fffffff;
    for (int k = 2; k <= 32; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int32_t o = __shfl_xor_sync(0xffffffffu, v, j);
        const bool up = (lane & k) == 0;
        const bool lower = (lane & j) == 0;
        // keep the smaller value in the lower lane of an ascending pair
        v = (lower == up) ? min(v, o) : max(v, o);
      }
    if (lane < len) in_idx[b + lane] = v;
  }
}

constexpr int kSortBlockMax = 8192; // longest in-row sorted in shared memory

// Sorts the in-rows listed in rows[] (33..kSortBlockMax entries), one block
// per row: a bitonic network in shared memory over the next power of two.
__global__ void sort_rows_block_kernel(const int32_t *__restrict__ in_ptr,
                                       int32_t *__restrict__ in_idx,
                                       const int32_t *__restrict__ rows, int32_t nrows) {
  __shared__ int32_t buf[kSortBlockMax];
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int32_t x = rows[r];
    const int32_t b = in_ptr[x], len = in_ptr[x + 1] - b;
    int p2 = 64;
    while (p2 < len) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) buf[i] = i < len ? in_idx[b + i] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < p2; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) {
            const bool up = (i & k) == 0;
            const int32_t a = buf[i], c = buf[l];
            if ((a > c) == up) {
              buf[i] = c;
              buf[l] = a;
            }
          }
        }
        __syncthreads();
      }
    for (int i = threadIdx.x; i < len; i += blockDim.x) in_idx[b + i] = buf[i];
    __syncthreads();
  }
}

int prep_grid(int64_t work) {
  int64_t g = (work + kPrepBlock - 1) / kPrepBlock;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (int)g;
}

} // namespace

cudaError_t launch_check_csr(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int *flags,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  check_csr_kernel<<<prep_grid((int64_t)n * 32), kPrepBlock, 0, st>>>(row_ptr, col_idx, n, flags);
  return cudaGetLastError();
}

cudaError_t launch_in_degree(const int32_t *col_idx, int64_t m, int32_t *cnt, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  in_degree_kernel<<<prep_grid(m), kPrepBlock, 0, st>>>(col_idx, m, cnt);
  return cudaGetLastError();
}

cudaError_t launch_in_scatter(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                              int32_t *fill, int32_t *in_idx, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  in_scatter_kernel<<<prep_grid((int64_t)n * 32), kPrepBlock, 0, st>>>(row_ptr, col_idx, n, fill,
                                                                        in_idx);
  return cudaGetLastError();
}

cudaError_t launch_sort_rows(const int32_t *in_ptr, int32_t *in_idx, const int32_t *warp_rows,
                             int32_t n_warp_rows, const int32_t *block_rows, int32_t n_block_rows,
                             cudaStream_t st) {
  if (n_warp_rows > 0)
    sort_rows_warp_kernel<<<prep_grid((int64_t)n_warp_rows * 32), kPrepBlock, 0, st>>>(
        in_ptr, in_idx, warp_rows, n_warp_rows);
  if (n_block_rows > 0)
    sort_rows_block_kernel<<<(int)std::min<int64_t>(n_block_rows, 4096), kPrepBlock, 0, st>>>(
        in_ptr, in_idx, block_rows, n_block_rows);
  return cudaGetLastError();
}

int sort_block_max() { return kSortBlockMax; }

cudaError_t launch_graph_keys(const int32_t *row_ptr, const int32_t *col_idx,
                              const int32_t *in_ptr, int32_t n, int32_t *nchunks, int64_t *two,
                              unsigned long long *totals, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  graph_keys_kernel<<<prep_grid((int64_t)n * 32), kPrepBlock, 0, st>>>(row_ptr, col_idx, in_ptr,
                                                                        n, nchunks, two, totals);
  return cudaGetLastError();
}

} // namespace bcgpu
