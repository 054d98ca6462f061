// li_mixed_ff.cu -- the all-on mixed-precision LI kernel with the refinement
// residual of every row in error-free FP32 arithmetic (SFCHEM_F_REFINE_FF);
// see li_mixed.cu.
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

__global__ void __launch_bounds__(128, 5) sfchem_li_mixed_ff(KArgs a) {
  li_persistent_body<float, true, false, true, 1>(a);
}

cudaError_t launch_li_mixed_ff(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  sfchem_li_mixed_ff<<<grid, tpb, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_li_mixed_ff(int tpb, int *ctas_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_mixed_ff, tpb, 0);
}

}  // namespace sfc
