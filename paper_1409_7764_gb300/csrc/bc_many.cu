// The many-small-graphs launch (many_kernel in bc_batch.cuh) in its own
// translation unit: each precision instantiates the batched sweep for every
// mask width with 32- and 64-bit path-count rows under block barriers.
#include "bc_batch.cuh"

namespace bcgpu {

cudaError_t launch_many(const ManyParams &mp, bool fp64, int grid, cudaStream_t st) {
  if (fp64) many_kernel<double><<<grid, kBlock, 0, st>>>(mp);
  else many_kernel<float><<<grid, kBlock, 0, st>>>(mp);
  return cudaGetLastError();
}

int max_grid_many(bool fp64, int device) {
  int per_sm = 0, sms = 0;
  const cudaError_t e =
      fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, many_kernel<double>, kBlock, 0)
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, many_kernel<float>, kBlock, 0);
  if (e != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

} // namespace bcgpu
