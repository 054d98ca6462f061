// nr_fp64.cu -- the Newton-Raphson backward-Euler reference solver of
// Sec. 2.2.8 on the GPU (FP64), in the same persistent lane-refill kernel
// as the LI method.
#include "nr_device.cuh"
#include "launch.h"

namespace sfc {

// One kernel for every launch shape (64 or 128 threads per CTA).
__global__ void __launch_bounds__(128) sfchem_nr_fp64(KArgs a) { li_persistent_body<double, false, true>(a); }

cudaError_t launch_nr_fp64(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  sfchem_nr_fp64<<<grid, tpb, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_nr_fp64(int tpb, int *ctas_per_sm) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_nr_fp64, tpb, 0);
}

}  // namespace sfc
