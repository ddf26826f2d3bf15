// lbm_sweep.cu -- dispatch of the sweep launchers by storage form (the kernels
// are in lbm_sweep.cuh, instantiated per form by lbm_sweep_<form>.cu) and the
// tile -> lattice map of batches.
#include "lbm_internal.cuh"

namespace lbm {

namespace {

// Lattice of every sweep tile (batches): tiles are numbered lattice by
// lattice, lattice l owning [tile0_l, tile0_{l+1}); one binary search per tile
// here instead of one per block in every sweep.
__global__ void tile_map_kernel(const LatDev *lat, int nlat, int ntiles, int *map) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int lo = 0, hi = nlat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lat[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    map[t] = lo;
}

}  // namespace

cudaError_t launch_tile_map(const LatDev *lat, int nlat, int ntiles, int *map, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    tile_map_kernel<<<(ntiles + 255) / 256, 256, 0, s>>>(lat, nlat, ntiles, map);
    return cudaGetLastError();
}

cudaError_t launch_sweep(int prec, int parity, int variant, const SweepArgs &a, int grid, int block, int cpt,
                         cudaStream_t s) {
    if (!sweep_cpt_supported(prec, variant == SWEEP_DIRECT ? cpt : 1)) return cudaErrorInvalidValue;
    switch (prec) {
    case LBM_F64: return launch_sweep_prec<LBM_F64>(parity, variant, a, grid, block, cpt, s);
    case LBM_F32: return launch_sweep_prec<LBM_F32>(parity, variant, a, grid, block, cpt, s);
    case LBM_F16_OFFSET: return launch_sweep_prec<LBM_F16_OFFSET>(parity, variant, a, grid, block, cpt, s);
    case LBM_BF16_OFFSET: return launch_sweep_prec<LBM_BF16_OFFSET>(parity, variant, a, grid, block, cpt, s);
    }
    return cudaErrorInvalidValue;
}

int sweep_max_active_blocks(int prec, int variant, int block, int cpt) {
    switch (prec) {
    case LBM_F64: return sweep_max_blocks_prec<LBM_F64>(variant, block, cpt);
    case LBM_F32: return sweep_max_blocks_prec<LBM_F32>(variant, block, cpt);
    case LBM_F16_OFFSET: return sweep_max_blocks_prec<LBM_F16_OFFSET>(variant, block, cpt);
    case LBM_BF16_OFFSET: return sweep_max_blocks_prec<LBM_BF16_OFFSET>(variant, block, cpt);
    }
    return 0;
}

}  // namespace lbm
