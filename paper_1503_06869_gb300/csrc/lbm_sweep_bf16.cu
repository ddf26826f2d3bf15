// lbm_sweep_bf16.cu -- the sweep kernels of the LBM_BF16_OFFSET storage form.
#include "lbm_sweep.cuh"

namespace lbm {
template cudaError_t launch_sweep_prec<LBM_BF16_OFFSET>(int, int, const SweepArgs &, int, int, int, cudaStream_t);
template int sweep_max_blocks_prec<LBM_BF16_OFFSET>(int, int, int);
}  // namespace lbm
