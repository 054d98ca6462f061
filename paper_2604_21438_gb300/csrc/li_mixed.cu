// li_mixed.cu -- the mixed-precision LI kernel: rate coefficients, heating
// and cooling, Jacobian assembly and the 5x5 LU in FP32; the state, the time
// accounting, one residual-refinement pass of the solve, the update and the
// conservation projection in FP64.
//
// One kernel for every launch shape, so that a cell's arithmetic does not
// depend on the block size the autotuner picks (ptxas may fuse a multiply
// and an add differently under different register limits).  Three
// instances, one per translation unit (compiled in parallel):
//   sfchem_li_mixed         all-on configuration, default refinement (this file)
//   sfchem_li_mixed_ff      all-on configuration, SFCHEM_F_REFINE_FF (li_mixed_ff.cu)
//   sfchem_li_mixed_masked  reactions or processes switched off, or test
//                           flags set; refinement chosen at run time
//                           (li_mixed_masked.cu)
// The configuration alone picks the instance, so every launch path of a
// given configuration runs the same kernel.  The register cap (96 per
// thread, 64 or 128 threads per CTA) gives 20 warps/SM; on the GMC-like
// workload this is faster than 16 warps/SM (128 registers) and than
// 24 warps/SM (80 registers, more spills).
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

__global__ void __launch_bounds__(128, 5) sfchem_li_mixed(KArgs a) {
  li_persistent_body<float, true, false, true, 0>(a);
}

static bool all_on(const DevCfg &c) {
  return c.rmask == R_ALL && c.pmask == P_ALL && (c.flags & ~(F_REFINE_FF | F_NO_REJECT)) == 0u;
}

cudaError_t launch_li_mixed(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  cudaError_t e;
  if (!all_on(a.cfg)) {
    e = launch_li_mixed_masked(a, grid, tpb, s);
  } else if (a.cfg.flags & F_REFINE_FF) {
    e = launch_li_mixed_ff(a, grid, tpb, s);
  } else {
    sfchem_li_mixed<<<grid, tpb, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? launch_hminus(a, true, s) : e;
}

// the smallest residency of the three instances, so that one launch shape fits all
cudaError_t occupancy_li_mixed(int tpb, int *ctas_per_sm) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  int a = 0, b = 0, c = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, sfchem_li_mixed, tpb, 0);
  if (e == cudaSuccess) e = occupancy_li_mixed_ff(tpb, &b);
  if (e == cudaSuccess) e = occupancy_li_mixed_masked(tpb, &c);
  *ctas_per_sm = a < b ? (a < c ? a : c) : (b < c ? b : c);
  return e;
}

}  // namespace sfc
