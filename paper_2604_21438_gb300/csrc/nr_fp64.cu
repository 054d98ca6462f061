// nr_fp64.cu -- the Newton-Raphson backward-Euler reference solver of
// Sec. 2.2.8 on the GPU (FP64), in the same persistent lane-refill kernel
// as the LI method.
#include "nr_device.cuh"
#include "launch.h"

namespace sfc {

// One kernel for every launch shape (64 or 128 threads per CTA), at full
// occupancy (32 registers, 64 warps per SM).  The nested Newton loops are a
// long body whose lanes take different iteration counts, so warps wait for
// instruction fetch far more than for the FP64 pipe: more warps hide it
// despite the spills (GMC-like 256^3, first 512 blocks: 186 ms with 166
// registers and 12 warps per SM, 164 / 138 / 114 ms with 96 / 64 / 32
// registers).  The FP64 LI kernel, bound by its FP64 pipe, gains nothing
// from the same change (it slows down).
__global__ void __launch_bounds__(128, 16) sfchem_nr_fp64(KArgs a) { li_persistent_body<double, false, true>(a); }

cudaError_t launch_nr_fp64(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  sfchem_nr_fp64<<<grid, tpb, 0, s>>>(a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_hminus(a, false, s) : e;
}

cudaError_t occupancy_nr_fp64(int tpb, int *ctas_per_sm) {
  if (tpb != 64 && tpb != 128) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_nr_fp64, tpb, 0);
}

}  // namespace sfc
