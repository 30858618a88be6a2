// nyx_fused_mixed.cu -- the fused persistent advance in mixed precision:
// FP32 primitives, PPM, tracing, Riemann solves and corner coupling; FP64
// state, flux-divergence accumulation, update and dual-energy sync.
#define NYX_NS nyx_mixed
#include "nyx_fused.cuh"

namespace nyx {

int launch_fused_mixed(int shape, const FusedArgs &a, int grid, cudaStream_t st) {
  switch (shape) {
    case 0: return nyx_mixed::launch_one<float, 16, 16>(a, grid, st);
    case 1: return nyx_mixed::launch_one<float, 32, 8>(a, grid, st);
    case 2: return nyx_mixed::launch_one<float, 16, 8>(a, grid, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

int max_grid_mixed(int shape) {
  switch (shape) {
    case 0: return nyx_mixed::max_grid_one<float, 16, 16>();
    case 1: return nyx_mixed::max_grid_one<float, 32, 8>();
    case 2: return nyx_mixed::max_grid_one<float, 16, 8>();
    default: return 1;
  }
}

}  // namespace nyx
