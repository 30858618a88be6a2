// nyx_fused_f64.cu -- the fused persistent advance in FP64 (built with
// --fmad=false, so it reproduces the per-box FP64 form bit for bit).
#define NYX_NS nyx_fused64
#include "nyx_fused.cuh"

namespace nyx {

int launch_fused_f64(int shape, const FusedArgs &a, int grid, cudaStream_t st) {
  switch (shape) {
    case 0: return nyx_fused64::launch_one<double, 16, 16>(a, grid, st);
    case 1: return nyx_fused64::launch_one<double, 32, 8>(a, grid, st);
    case 2: return nyx_fused64::launch_one<double, 16, 8>(a, grid, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_flatten_f64(const BoxDev *boxes, const FlatTile *tiles, int ntiles, const double *S,
                       const SchemeConsts *K, void *fl, cudaStream_t st) {
  return nyx_fused64::launch_flatten_t<double>(boxes, tiles, ntiles, S, K, fl, st);
}

int flatten_init_f64() { return nyx_fused64::flatten_init_t<double>(); }

int flat_ones_f64(void *fl, long long n, cudaStream_t st) {
  nyx_fused64::k_flat_ones<double><<<1216, 256, 0, st>>>(static_cast<double *>(fl), n);
  return (int)cudaGetLastError();
}

int max_grid_f64(int shape) {
  switch (shape) {
    case 0: return nyx_fused64::max_grid_one<double, 16, 16>();
    case 1: return nyx_fused64::max_grid_one<double, 32, 8>();
    case 2: return nyx_fused64::max_grid_one<double, 16, 8>();
    default: return 1;
  }
}

}  // namespace nyx
