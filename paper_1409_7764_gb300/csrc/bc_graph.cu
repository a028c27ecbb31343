// Device-side preparation of a resident graph: the in-CSR (transpose) of the
// canonical out-CSR with every in-row in ascending source order, the
// per-vertex chunk counts of high-degree vertices for every candidate chunk
// size, and the batch-composition key (two-hop walk counts).  The whole
// pipeline runs on one stream with no host round trip; the host reads the
// validation flags at its end (and canonicalises on the host, then runs the
// pipeline again, when a row was not canonical).  Every kernel that indexes
// by a column id skips ids outside [0, n), so an invalid graph is only
// reported, never followed out of bounds.
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

// In-degree counts: cnt[x + 1] += 1 for every edge into x (ids outside
// [0, n) skipped; check_csr reports them).
__global__ void in_degree_kernel(const int32_t *__restrict__ col_idx, int64_t m, int32_t n,
                                 int32_t *__restrict__ cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = col_idx[e];
    if ((uint32_t)x < (uint32_t)n) atomicAdd(cnt + x + 1, 1);
  }
}

constexpr int kScanBlock = 1024;
constexpr int kScanTile = 2 * kScanBlock; // elements per block

// Inclusive scan of a[0, len) in tiles of kScanTile (two elements per
// thread); tile totals go to sums[blockIdx.x].
__global__ void scan_tiles_kernel(int32_t *__restrict__ a, int64_t len,
                                  int32_t *__restrict__ sums) {
  __shared__ int32_t warp_tot[kScanBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * kScanTile + 2 * threadIdx.x;
  const int32_t x0 = i0 < len ? a[i0] : 0;
  const int32_t x1 = i0 + 1 < len ? a[i0 + 1] : 0;
  int32_t v = x0 + x1;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int32_t o = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += o;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int32_t t = lane < kScanBlock / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int32_t o = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= off) t += o;
    }
    if (lane < kScanBlock / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  const int32_t before = (wid > 0 ? warp_tot[wid - 1] : 0) + v - (x0 + x1);
  if (i0 < len) a[i0] = before + x0;
  if (i0 + 1 < len) a[i0 + 1] = before + x0 + x1;
  if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = warp_tot[kScanBlock / 32 - 1];
}

// Adds the scanned total of the tiles before it to every element of a tile.
__global__ void scan_add_kernel(int32_t *__restrict__ a, int64_t len,
                                const int32_t *__restrict__ sums) {
  if (blockIdx.x == 0) return;
  const int32_t add = sums[blockIdx.x - 1];
  const int64_t i0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  if (i0 < len) a[i0] += add;
  if (i0 + kScanBlock < len) a[i0 + kScanBlock] += add;
}

// Scatter of the edges into the in-CSR, one warp per source vertex (lanes
// over its out-edges); fill[x] starts at in_ptr[x].  The order inside an
// in-row depends on the atomics' order, so the rows are sorted afterwards
// (sort_rows_*: ascending sources, as a sequential transpose would give).
// Ids outside [0, n) are skipped.
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
      if ((uint32_t)x < (uint32_t)n) in_idx[atomicAdd(fill + x, 1)] = (int32_t)v;
    }
  }
}

// Per vertex: chunk counts for each candidate chunk size (0 when in+out
// degree fits one chunk), the heavy-vertex and chunk totals per size, and the
// number of two-hop walks leaving it (sum of its out-neighbours'
// out-degrees; neighbour ids outside [0, n) skipped).
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
      if ((uint32_t)x < (uint32_t)n) t += row_ptr[x + 1] - row_ptr[x];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) {
      two[v] = t;
      const int64_t cost = (int64_t)(e - b) + (in_ptr[v + 1] - in_ptr[v]);
      static_assert(kChunkVariants == 4, "one size per work-split variant");
      constexpr int64_t kSizes[kChunkVariants] = {kChunkCandidates[0], kChunkCandidates[1],
                                                   kChunkCandidates[2], kChunkCandidates[3]};
#pragma unroll
      for (int c = 0; c < kChunkVariants; ++c) {
        const int64_t ch = kSizes[c];
        int32_t nc = 0;
        if (cost > heavy_threshold(ch)) {
          nc = (int32_t)((cost + ch - 1) / ch);
          atomicAdd(totals + 2 * c, 1ull);
          atomicAdd(totals + 2 * c + 1, (unsigned long long)nc);
        }
        nchunks[(size_t)c * n + v] = nc;
      }
    }
  }
}

constexpr int kSortBlockMax = 8192; // longest in-row sorted in shared memory

// Lists the in-rows to sort by length: rows[0 ..) of 2..32 entries (count
// in counts[0]), rows[n ..) of 33..kSortBlockMax (counts[1]), rows[2n ..)
// longer ones (counts[2]); warp-aggregated appends, in no particular order.
__global__ void classify_rows_kernel(const int32_t *__restrict__ in_ptr, int32_t n,
                                     int32_t *__restrict__ rows, int32_t *__restrict__ counts) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = b + threadIdx.x;
    int cls = -1;
    if (x < n) {
      const int32_t len = in_ptr[x + 1] - in_ptr[x];
      cls = len < 2 ? -1 : len <= 32 ? 0 : len <= kSortBlockMax ? 1 : 2;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const unsigned bal = __ballot_sync(0xffffffffu, cls == c);
      if (!bal) continue;
      int32_t base = 0;
      if (lane == 0) base = atomicAdd(counts + c, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (cls == c) rows[(size_t)c * n + base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)x;
    }
  }
}

// Sorts the in-rows listed in rows[0, *nrows) (2..32 entries each), one warp
// per row: a bitonic network over the lanes, padded with INT_MAX.
__global__ void sort_rows_warp_kernel(const int32_t *__restrict__ in_ptr,
                                      int32_t *__restrict__ in_idx,
                                      const int32_t *__restrict__ rows,
                                      const int32_t *__restrict__ nrows_p) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t nrows = *nrows_p;
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

// Sorts the in-rows listed in rows[0, *nrows) (33..kSortBlockMax entries),
// one block per row: a bitonic network in shared memory over the next power
// of two.
__global__ void sort_rows_block_kernel(const int32_t *__restrict__ in_ptr,
                                       int32_t *__restrict__ in_idx,
                                       const int32_t *__restrict__ rows,
                                       const int32_t *__restrict__ nrows_p) {
  __shared__ int32_t buf[kSortBlockMax];
  const int32_t nrows = *nrows_p;
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

constexpr int kLongSortBlock = 1024;

// One compare-exchange pass of the merge network over the pairs (i, l) of
// a[0, len): with the first step of stage k (flip) l = i ^ (k-1), the
// mirror of i in its k-block, else l = i + j; i runs over the lower halves
// of the j-blocks of [0, span).  Ascending everywhere, so positions at or
// past len act as +infinity and are never touched.
__device__ __forceinline__ void merge_pass(int32_t *a, int64_t len, int64_t span, int64_t k,
                                           int64_t j, bool flip) {
  const int lj = __ffsll((long long)j) - 1; // j is a power of two
  for (int64_t t = threadIdx.x; t < span / 2; t += blockDim.x) {
    const int64_t i = ((t >> lj) << (lj + 1)) | (t & (j - 1));
    const int64_t l = flip ? (i ^ (k - 1)) : (i + j);
    if (l < len) {
      const int32_t u = a[i], w = a[l];
      if (u > w) {
        a[i] = w;
        a[l] = u;
      }
    }
  }
}

// Sorts the in-rows listed in rows[0, *nrows) (longer than kSortBlockMax),
// one block per row, in place: a bitonic network whose merge steps compare
// every element with its mirror in the merged block and then with i + j,
// all towards ascending order (so no padding is stored).  Every pass with
// j < kSortBlockMax stays inside a kSortBlockMax-aligned tile and runs in
// shared memory (all stages up to the tile size at once, then the tail of
// each larger stage); only the passes with j >= kSortBlockMax run over the
// row in global memory.
__global__ void __launch_bounds__(kLongSortBlock)
    sort_rows_long_kernel(const int32_t *__restrict__ in_ptr, int32_t *__restrict__ in_idx,
                          const int32_t *__restrict__ rows, const int32_t *__restrict__ nrows_p) {
  constexpr int T = kSortBlockMax;
  __shared__ int32_t buf[T];
  const int32_t nrows = *nrows_p;
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int32_t x = rows[r];
    int32_t *a = in_idx + in_ptr[x];
    const int64_t len = in_ptr[x + 1] - in_ptr[x];
    int64_t p2 = T;
    while (p2 < len) p2 <<= 1;
    // passes inside each tile, in shared memory: stages k <= T (kmin = 2),
    // or the passes j < T of stage kmin (> T)
    auto tile_passes = [&](int64_t kmin) {
      for (int64_t tb = 0; tb < len; tb += T) {
        const int64_t tl = len - tb < T ? len - tb : T; // real entries in the tile
        for (int i = threadIdx.x; i < T; i += blockDim.x) buf[i] = i < tl ? a[tb + i] : 0x7fffffff;
        __syncthreads();
        const int64_t k0 = kmin <= T ? 2 : kmin, k1 = kmin <= T ? T : kmin;
        for (int64_t k = k0; k <= k1; k <<= 1) {
          for (int64_t j = (k <= T ? k : T) >> 1; j > 0; j >>= 1) {
            merge_pass(buf, tl, T, k, j, k <= T && j == (k >> 1));
            __syncthreads();
          }
        }
        for (int i = threadIdx.x; i < tl; i += blockDim.x) a[tb + i] = buf[i];
        __syncthreads();
      }
    };
    tile_passes(2);
    for (int64_t k = 2 * T; k <= p2; k <<= 1) {
      for (int64_t j = k >> 1; j >= T; j >>= 1) {
        merge_pass(a, len, p2, k, j, j == (k >> 1));
        __syncthreads();
      }
      tile_passes(k);
    }
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

cudaError_t launch_in_degree(const int32_t *col_idx, int64_t m, int32_t n, int32_t *cnt,
                             cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  in_degree_kernel<<<prep_grid(m), kPrepBlock, 0, st>>>(col_idx, m, n, cnt);
  return cudaGetLastError();
}

// Scratch (int32 elements) the scan of len elements needs: the tile totals
// of every level.
int64_t scan_scratch_elems(int64_t len) {
  int64_t total = 0;
  while (len > 1) {
    len = (len + kScanTile - 1) / kScanTile;
    total += len;
  }
  return total > 0 ? total : 1;
}

// In-place inclusive scan of a[0, len): tiles, then (recursively) the tile
// totals, then the carry into each tile.  scratch holds
// scan_scratch_elems(len) int32.
cudaError_t launch_scan_inclusive(int32_t *a, int64_t len, int32_t *scratch, cudaStream_t st) {
  if (len <= 0) return cudaSuccess;
  const int64_t tiles = (len + kScanTile - 1) / kScanTile;
  int32_t *sums = scratch;
  scan_tiles_kernel<<<(unsigned)tiles, kScanBlock, 0, st>>>(a, len, sums);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && tiles > 1) {
    e = launch_scan_inclusive(sums, tiles, scratch + tiles, st);
    if (e == cudaSuccess) {
      scan_add_kernel<<<(unsigned)tiles, kScanBlock, 0, st>>>(a, len, sums);
      e = cudaGetLastError();
    }
  }
  return e;
}

cudaError_t launch_in_scatter(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                              int32_t *fill, int32_t *in_idx, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  in_scatter_kernel<<<prep_grid((int64_t)n * 32), kPrepBlock, 0, st>>>(row_ptr, col_idx, n, fill,
                                                                        in_idx);
  return cudaGetLastError();
}

// Sorts every in-row: classification by length, then the warp, block and
// long-row sorts, each reading its row count on the device (grids sized for
// the most rows there can be; surplus blocks find no row).  rows: scratch
// of 3n int32, counts: 3 int32 (zeroed here).
cudaError_t launch_sort_rows(const int32_t *in_ptr, int32_t *in_idx, int32_t n, int64_t m,
                             int32_t *rows, int32_t *counts, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  classify_rows_kernel<<<prep_grid(n), kPrepBlock, 0, st>>>(in_ptr, n, rows, counts);
  // at most n rows of each kind; rows of 33+ entries number at most m / 33,
  // rows of kSortBlockMax+ entries at most m / (kSortBlockMax + 1)
  sort_rows_warp_kernel<<<prep_grid((int64_t)n * 32), kPrepBlock, 0, st>>>(in_ptr, in_idx, rows,
                                                                          counts);
  const int64_t nb = std::min<int64_t>(n, m / 33 + 1);
  sort_rows_block_kernel<<<(int)std::min<int64_t>(nb, 4096), kPrepBlock, 0, st>>>(
      in_ptr, in_idx, rows + n, counts + 1);
  const int64_t nl = std::min<int64_t>(n, m / (kSortBlockMax + 1) + 1);
  sort_rows_long_kernel<<<(int)std::min<int64_t>(nl, 1024), kLongSortBlock, 0, st>>>(
      in_ptr, in_idx, rows + 2 * (size_t)n, counts + 2);
  return cudaGetLastError();
}

cudaError_t launch_graph_keys(const int32_t *row_ptr, const int32_t *col_idx,
                              const int32_t *in_ptr, int32_t n, int32_t *nchunks, int64_t *two,
                              unsigned long long *totals, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  graph_keys_kernel<<<prep_grid((int64_t)n * 32), kPrepBlock, 0, st>>>(row_ptr, col_idx, in_ptr,
                                                                        n, nchunks, two, totals);
  return cudaGetLastError();
}

} // namespace bcgpu
