// nr_fp64.cu -- the Newton-Raphson backward-Euler reference solver of
// Sec. 2.2.8 on the GPU (FP64), in the same persistent lane-refill kernel
// as the LI method.
#include "nr_device.cuh"
#include "launch.h"

namespace sfc {

template <int TPB>
__global__ void __launch_bounds__(TPB) sfchem_nr_fp64(KArgs a) {
  li_persistent_body<double, false, true>(a);
}

cudaError_t launch_nr_fp64(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb == 256) sfchem_nr_fp64<256><<<grid, 256, 0, s>>>(a);
  else if (tpb == 64) sfchem_nr_fp64<64><<<grid, 64, 0, s>>>(a);
  else sfchem_nr_fp64<128><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_nr_fp64(int tpb, int *ctas_per_sm) {
  if (tpb == 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_nr_fp64<256>, 256, 0);
  if (tpb == 64) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_nr_fp64<64>, 64, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_nr_fp64<128>, 128, 0);
}

}  // namespace sfc
