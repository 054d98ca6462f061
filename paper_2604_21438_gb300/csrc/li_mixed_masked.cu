// li_mixed_masked.cu -- the general mixed-precision LI kernel: every mask and
// flag tested at run time (configurations with reactions or processes
// switched off, freeze or split flags); see li_mixed.cu.
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

__global__ void __launch_bounds__(128, 5) sfchem_li_mixed_masked(KArgs a) { li_persistent_body<float, true>(a); }

cudaError_t launch_li_mixed_masked(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  sfchem_li_mixed_masked<<<grid, tpb, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_li_mixed_masked(int tpb, int *ctas_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_mixed_masked, tpb, 0);
}

}  // namespace sfc
