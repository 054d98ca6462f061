// li_fp64.cu -- the plain FP64 LI kernel: rates, Jacobian and 5x5 solve in
// FP64 (the paper runs every real quantity in FP64, Sec. 3 and Sec. 4).
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

// One kernel for every launch shape (64 or 128 threads per CTA), so that a
// cell's arithmetic does not depend on the block size.  (A 256-thread bound
// makes ptxas cap the kernel at 150 registers, 4 % slower.)
__global__ void __launch_bounds__(128) sfchem_li_fp64(KArgs a) { li_persistent_body<double, false>(a); }

cudaError_t launch_li_fp64(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  sfchem_li_fp64<<<grid, tpb, 0, s>>>(a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_hminus(a, false, s) : e;
}

cudaError_t occupancy_li_fp64(int tpb, int *ctas_per_sm) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_fp64, tpb, 0);
}

}  // namespace sfc
