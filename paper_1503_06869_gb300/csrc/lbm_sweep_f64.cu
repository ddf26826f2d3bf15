// lbm_sweep_f64.cu -- the sweep kernels of the LBM_F64 storage form.
#include "lbm_sweep.cuh"

namespace lbm {
template cudaError_t launch_sweep_prec<LBM_F64>(int, int, const SweepArgs &, int, int, int, cudaStream_t);
template int sweep_max_blocks_prec<LBM_F64>(int, int, int);
}  // namespace lbm
