// li_fp64.cu -- the plain FP64 LI kernel: rates, Jacobian and 5x5 solve in
// FP64 (the paper runs every real quantity in FP64, Sec. 3 and Sec. 4).
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

template <int TPB>
__global__ void __launch_bounds__(TPB) sfchem_li_fp64(KArgs a) {
  li_persistent_body<double, false>(a);
}

cudaError_t launch_li_fp64(const KArgs &a, int grid, int tpb, cudaStream_t s) {
  if (tpb == 256) sfchem_li_fp64<256><<<grid, 256, 0, s>>>(a);
  else if (tpb == 64) sfchem_li_fp64<64><<<grid, 64, 0, s>>>(a);
  else sfchem_li_fp64<128><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_li_fp64(int tpb, int *ctas_per_sm) {
  if (tpb == 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_fp64<256>, 256, 0);
  if (tpb == 64) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_fp64<64>, 64, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sfchem_li_fp64<128>, 128, 0);
}

}  // namespace sfc
