// li_mixed.cu -- the mixed-precision LI kernel: rate coefficients, heating
// and cooling, Jacobian assembly and the 5x5 LU in FP32; the state, the time
// accounting, one residual-refinement pass of the solve, the update and the
// conservation projection in FP64.
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

// Register caps (96 per thread) that raise residency to 20 warps/SM at 64 or
// 128 threads per CTA: about 150 bytes spill to L1, and the kernel is 2-3 %
// faster than at 16 warps/SM (128 registers) and 5 % faster than uncapped
// (12 warps/SM); 24 warps/SM (80 registers) gains nothing more.
template <int TPB>
__global__ void __launch_bounds__(TPB, (TPB == 64 ? 10 : (TPB == 128 ? 5 : 2))) sfchem_li_mixed(KArgs a) {
  li_persistent_body<float, true>(a);
}

cudaError_t launch_li_mixed(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb == 256) sfchem_li_mixed<256><<<grid, 256, 0, s>>>(a);
  else if (tpb == 64) sfchem_li_mixed<64><<<grid, 64, 0, s>>>(a);
  else sfchem_li_mixed<128><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_li_mixed(int tpb, int *ctas_per_sm) {
  if (tpb == 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_mixed<256>, 256, 0);
  if (tpb == 64) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_mixed<64>, 64, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_mixed<128>, 128, 0);
}

}  // namespace sfc
