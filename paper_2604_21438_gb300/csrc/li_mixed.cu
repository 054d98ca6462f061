// li_mixed.cu -- the mixed-precision LI kernel: rate coefficients, heating
// and cooling, Jacobian assembly and the 5x5 LU in FP32; the state, the time
// accounting, one residual-refinement pass of the solve, the update and the
// conservation projection in FP64.
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

// One kernel for every launch shape, so that a cell's arithmetic does not
// depend on the block size the autotuner picks (ptxas may fuse a multiply
// and an add differently under different register limits).  Two instances:
// sfchem_li_mixed for the all-on configuration of production calls, and
// sfchem_li_mixed_masked for configurations with reactions or processes
// switched off or test flags set; the configuration alone picks one, so every
// launch path of a given configuration runs the same kernel.  The register cap (96 per thread, 64 or 128 threads per CTA)
// raises residency to 20 warps/SM: about 200 bytes spill to L1, and on the
// GMC-like workload the kernel is 3 % faster than at 16 warps/SM (128
// registers) and 2 % faster than at 24 warps/SM (80 registers, ~450 bytes of
// spills).
__global__ void __launch_bounds__(128, 5) sfchem_li_mixed(KArgs a) {
  li_persistent_body<float, true, false, true>(a);
}
__global__ void __launch_bounds__(128, 5) sfchem_li_mixed_masked(KArgs a) { li_persistent_body<float, true>(a); }

static bool all_on(const DevCfg &c) {
  return c.rmask == R_ALL && c.pmask == P_ALL && (c.flags & ~F_REFINE_FF) == 0u;
}

cudaError_t launch_li_mixed(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  if (all_on(a.cfg)) sfchem_li_mixed<<<grid, tpb, 0, s>>>(a);
  else sfchem_li_mixed_masked<<<grid, tpb, 0, s>>>(a);
  return cudaGetLastError();
}

// the smaller residency of the two instances, so that one launch shape fits both
cudaError_t occupancy_li_mixed(int tpb, int *ctas_per_sm) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, sfchem_li_mixed, tpb, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sfchem_li_mixed_masked, tpb, 0);
  *ctas_per_sm = a < b ? a : b;
  return e;
}

}  // namespace sfc
