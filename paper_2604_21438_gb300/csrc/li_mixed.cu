// li_mixed.cu -- the mixed-precision LI kernel: rate coefficients, heating
// and cooling, Jacobian assembly and the 5x5 LU in FP32; the state, the time
// accounting, one residual-refinement pass of the solve, the update and the
// conservation projection in FP64.
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

// One kernel for every launch shape, so that a cell's arithmetic does not
// depend on the block size the autotuner picks (ptxas may fuse a multiply
// and an add differently under different register limits).  The register cap
// (96 per thread, 64 or 128 threads per CTA) raises residency to 20 warps/SM:
// about 150 bytes spill to L1, and the kernel is 2-3 % faster than at 16
// warps/SM (128 registers) and 5 % faster than uncapped (12 warps/SM); 24
// warps/SM (80 registers) gains nothing more.
__global__ void __launch_bounds__(128, 5) sfchem_li_mixed(KArgs a) { li_persistent_body<float, true>(a); }

cudaError_t launch_li_mixed(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  sfchem_li_mixed<<<grid, tpb, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_li_mixed(int tpb, int *ctas_per_sm) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_mixed, tpb, 0);
}

}  // namespace sfc
