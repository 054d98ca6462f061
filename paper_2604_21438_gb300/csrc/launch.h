// launch.h -- host-side entry points of the kernels (internal to libsfchem).
#pragma once
#include <cuda_runtime.h>
#include "li_kernels.cuh"

namespace sfc {
cudaError_t launch_li_fp64(const KArgs &a, int grid, int tpb, cudaStream_t s);
cudaError_t launch_li_mixed(const KArgs &a, int grid, int tpb, cudaStream_t s);
cudaError_t occupancy_li_fp64(int tpb, int *ctas_per_sm);
cudaError_t occupancy_li_mixed(int tpb, int *ctas_per_sm);
// the instances behind launch_li_mixed (li_mixed_ff.cu, li_mixed_masked.cu)
cudaError_t launch_li_mixed_ff(const KArgs &a, int grid, int tpb, cudaStream_t s);
cudaError_t launch_li_mixed_masked(const KArgs &a, int grid, int tpb, cudaStream_t s);
cudaError_t occupancy_li_mixed_ff(int tpb, int *ctas_per_sm);
cudaError_t occupancy_li_mixed_masked(int tpb, int *ctas_per_sm);
cudaError_t launch_nr_fp64(const KArgs &a, int grid, int tpb, cudaStream_t s);
cudaError_t occupancy_nr_fp64(int tpb, int *ctas_per_sm);
// y_H- of the cells [0, a.n_cells) after a solver launch (derived.cu); every
// solver launcher above ends with it.  fp32: the mixed path's precision.
cudaError_t launch_hminus(const KArgs &a, bool fp32, cudaStream_t s);
// One-CTA schedule kernel of the batched path (cost order and chunk table).
cudaError_t launch_schedule(const int64_t *block_offset, float *block_cost, int32_t n_blocks, int32_t chunk,
                            int64_t *ch_start, int32_t *ch_count, int32_t *ch_block, cudaStream_t s);
}  // namespace sfc
