// derived.cu -- y_H- (the H- abundance in equilibrium between reactions H2 and
// H3 of Table 3, at the final gas temperature and electron fraction) of every
// cell of a call, formed after the solver kernel on the same stream.
//
// The solver writes 0 into y_Hm for a cell it advanced and NaN for a cell
// with invalid inputs; this kernel replaces every value that is not NaN.  One
// thread per cell: 24 B read, 8 B written, about a hundred FP32 (mixed) or
// FP64 instructions.  In the solver's refill phase each finished cell formed
// its y_H- with a few lanes of its warp active; on the 16.8M cells of a 256^3
// GMC-like grid, taking that out of the solver took the mixed kernel from
// 77.1 to 74.1 ms and the FP64 step from 3.32 to 3.09 s (the same results
// bit for bit).
#include "li_kernels.cuh"
#include "launch.h"

namespace sfc {

template <typename W>
__global__ void __launch_bounds__(256) sfchem_hminus(const double *__restrict__ Tg, const double *__restrict__ ye,
                                                     double *__restrict__ yHm, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (((__double2hiint(yHm[i]) >> 20) & 0x7ff) == 0x7ff) continue;   // NaN: invalid inputs, left as it is
    yHm[i] = y_hminus<W>(Tg[i], ye[i]);
  }
}

cudaError_t launch_hminus(const KArgs &a, bool fp32, cudaStream_t s) {
  if (!a.yHm || a.n_cells <= 0) return cudaSuccess;
  const int64_t blocks = (a.n_cells + 255) / 256;
  const int grid = (int)(blocks < (int64_t)(1 << 20) ? blocks : (int64_t)(1 << 20));
  if (fp32) sfchem_hminus<float><<<grid, 256, 0, s>>>(a.Tg, a.ye, a.yHm, a.n_cells);
  else sfchem_hminus<double><<<grid, 256, 0, s>>>(a.Tg, a.ye, a.yHm, a.n_cells);
  return cudaGetLastError();
}

}  // namespace sfc
