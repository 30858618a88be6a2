// nyx_fused_mixed.cu -- the fused persistent advance in mixed precision:
// FP32 primitives, PPM, tracing, Riemann solves and corner coupling; FP64
// state, flux-divergence accumulation, update and dual-energy sync.
// Shapes 0-2: column-owning form (nyx_fused.cuh); 3-5: task form
// (nyx_fused2.cuh).
#define NYX_NS nyx_mixed
#include "nyx_fused.cuh"
#include "nyx_fused2.cuh"

namespace nyx {

int launch_fused_mixed(int shape, const FusedArgs &a, int grid, cudaStream_t st) {
  switch (shape) {
    case 0: return nyx_mixed::launch_one<float, 16, 16>(a, grid, st);
    case 1: return nyx_mixed::launch_one<float, 32, 8>(a, grid, st);
    case 2: return nyx_mixed::launch_one<float, 16, 8>(a, grid, st);
    case 3: return nyx_mixed::launch_two<16, 8, 1>(a, grid, st);
    case 4: return nyx_mixed::launch_two<8, 8, 2>(a, grid, st);
    case 5: return nyx_mixed::launch_two<32, 4, 1>(a, grid, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

int max_grid_mixed(int shape) {
  switch (shape) {
    case 0: return nyx_mixed::max_grid_one<float, 16, 16>();
    case 1: return nyx_mixed::max_grid_one<float, 32, 8>();
    case 2: return nyx_mixed::max_grid_one<float, 16, 8>();
    case 3: return nyx_mixed::max_grid_two<16, 8, 1>();
    case 4: return nyx_mixed::max_grid_two<8, 8, 2>();
    case 5: return nyx_mixed::max_grid_two<32, 4, 1>();
    default: return 1;
  }
}

}  // namespace nyx
