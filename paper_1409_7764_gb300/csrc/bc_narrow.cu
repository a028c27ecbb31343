// Narrow batches in a wide workspace: the batched kernel instantiated with
// fewer mask words per source set (W) than the workspace is laid out for
// (S).  A job's last batch that holds sources with out-edges is usually
// partly filled; running it with W words instead of S skips the mask words
// and state slots that no source of the batch uses (about half a full
// batch's gather work when 128 sources or fewer remain), without laying out
// or clearing the workspace again: the words and slots a narrow batch never
// touches stay zero, as every batch leaves them.
#include "bc_batch.cuh"

namespace bcgpu {
namespace {

template <typename K> cudaError_t coop_launch_narrow(K kernel, const KParams &p, int grid,
                                                     cudaStream_t st) {
  void *args[] = {const_cast<KParams *>(&p)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kernel), dim3(grid),
                                     dim3(kBlock), args, 0, st);
}

template <typename DT, typename CT>
cudaError_t narrow_dt_ct(const KParams &p, int grid, cudaStream_t st, int words, int layout) {
  if (layout == 4 && words == 2)
    return coop_launch_narrow(batch_kernel<DT, 2, false, CT, 4>, p, grid, st);
  if (layout == 4 && words == 1)
    return coop_launch_narrow(batch_kernel<DT, 1, false, CT, 4>, p, grid, st);
  if (layout == 2 && words == 1)
    return coop_launch_narrow(batch_kernel<DT, 1, false, CT, 2>, p, grid, st);
  return cudaErrorInvalidValue;
}

} // namespace

cudaError_t launch_batch_narrow(const KParams &p, bool fp64, int grid, cudaStream_t st,
                                int words, int layout_words, bool counts32) {
  if (p.bc2 || words >= layout_words) return cudaErrorInvalidValue;
  if (counts32)
    return fp64 ? narrow_dt_ct<double, uint32_t>(p, grid, st, words, layout_words)
                : narrow_dt_ct<float, uint32_t>(p, grid, st, words, layout_words);
  return fp64 ? narrow_dt_ct<double, uint64_t>(p, grid, st, words, layout_words)
              : narrow_dt_ct<float, uint64_t>(p, grid, st, words, layout_words);
}

} // namespace bcgpu
