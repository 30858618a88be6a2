// nyx_fused_mixed.cu -- the fused persistent advance in mixed precision:
// FP32 primitives, PPM, tracing, Riemann solves and corner coupling; FP64
// state, flux-divergence accumulation, update and dual-energy sync.
// Shapes 0-2: column-owning form (nyx_fused.cuh); 3-5: task form
// (nyx_fused2.cuh).
#include <algorithm>

#define NYX_NS nyx_mixed
#include "nyx_fused.cuh"
#include "nyx_fused2.cuh"

namespace nyx {

int launch_fused_mixed(int shape, const FusedArgs &a, int grid, cudaStream_t st) {
  switch (shape) {
    case 0: return nyx_mixed::launch_one<float, 16, 16>(a, grid, st);
    case 1: return nyx_mixed::launch_one<float, 32, 8>(a, grid, st);
    case 2: return nyx_mixed::launch_one<float, 16, 8>(a, grid, st);
    case 3:  // the default shape: one instantiation per scheme variant (flattening with
             // PLM or the linearised solver: the one with run-time variant flags)
      if (a.variant == 4) return nyx_mixed::launch_two<16, 8, 1, 4>(a, grid, st);
      if (a.variant & 4) return nyx_mixed::launch_two<16, 8, 1, -1>(a, grid, st);
      switch (a.variant) {
        case 1: return nyx_mixed::launch_two<16, 8, 1, 1>(a, grid, st);
        case 2: return nyx_mixed::launch_two<16, 8, 1, 2>(a, grid, st);
        case 3: return nyx_mixed::launch_two<16, 8, 1, 3>(a, grid, st);
        default: return nyx_mixed::launch_two<16, 8, 1, 0>(a, grid, st);
      }
    case 4: return nyx_mixed::launch_two<8, 8, 2, -1>(a, grid, st);
    case 5: return nyx_mixed::launch_two<32, 4, 1, -1>(a, grid, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

int max_grid_mixed(int shape) {
  switch (shape) {
    case 0: return nyx_mixed::max_grid_one<float, 16, 16>();
    case 1: return nyx_mixed::max_grid_one<float, 32, 8>();
    case 2: return nyx_mixed::max_grid_one<float, 16, 8>();
    case 3: {  // every variant instantiation, the smallest grid
      int g = nyx_mixed::max_grid_two<16, 8, 1, 0>();
      g = std::min(g, nyx_mixed::max_grid_two<16, 8, 1, 1>());
      g = std::min(g, nyx_mixed::max_grid_two<16, 8, 1, 2>());
      g = std::min(g, nyx_mixed::max_grid_two<16, 8, 1, -1>());
      g = std::min(g, nyx_mixed::max_grid_two<16, 8, 1, 4>());
      return std::min(g, nyx_mixed::max_grid_two<16, 8, 1, 3>());
    }
    case 4: return nyx_mixed::max_grid_two<8, 8, 2, -1>();
    case 5: return nyx_mixed::max_grid_two<32, 4, 1, -1>();
    default: return 1;
  }
}

int launch_flatten_mixed(const BoxDev *boxes, const FlatTile *tiles, int ntiles, const double *S,
                         const SchemeConsts *K, void *fl, cudaStream_t st) {
  return nyx_mixed::launch_flatten_t<float>(boxes, tiles, ntiles, S, K, fl, st);
}

int flatten_init_mixed() { return nyx_mixed::flatten_init_t<float>(); }

int flat_ones_mixed(void *fl, long long n, cudaStream_t st) {
  nyx_mixed::k_flat_ones<float><<<1216, 256, 0, st>>>(static_cast<float *>(fl), n);
  return (int)cudaGetLastError();
}

}  // namespace nyx

namespace nyx {
namespace {

// CFL step of a state in FP32 (mixed plans): the same minimum as the FP64
// reduction, with the primitives and the ratios formed in FP32.
__global__ void k_estdt_mixed(const BoxDev *boxes, const long long *cell_pref, int nbox,
                              long long total, const double *state, const SchemeConsts *K,
                              const double *a_dev, unsigned long long *dtacc) {
  const float gm1 = nyx_mixed::d2f_rn(K->gm1), gamma = nyx_mixed::d2f_rn(K->gamma);
  const float small_pres = nyx_mixed::d2f_rn(K->small_pres);
  const double a = *a_dev;
  float local_min = __int_as_float(0x7f800000);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (cell_pref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const BoxDev b = boxes[lo];
    const long long f = t - cell_pref[lo];
    const int i = (int)(f % b.n[0]);
    const long long u = f / b.n[0];
    const int j = (int)(u % b.n[1]);
    const int kk = (int)(u / b.n[1]);
    const double *S = state + NCONS * b.pref;
    const long long id = cell_index(b, i, j, kk);
    const float rho = nyx_mixed::d2f_rn(S[id]);
    const float ir = 1.0f / rho;
    float p = gm1 * nyx_mixed::d2f_rn(S[5 * b.stride + id]);
    if (p < small_pres) p = small_pres;
    const float c2 = gamma * p * ir;
    const float c = c2 * rsqrtf(c2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float adx = nyx_mixed::d2f_rn(a * b.dx[d]);
      const float tt = adx / (fabsf(nyx_mixed::d2f_rn(S[(1 + d) * b.stride + id]) * ir) + c);
      local_min = fminf(local_min, tt);
    }
  }
  for (int o = 16; o > 0; o >>= 1) local_min = fminf(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
  if ((threadIdx.x & 31) == 0 && local_min < __int_as_float(0x7f800000))
    atomic_min_pos(dtacc, (double)local_min);
}

}  // namespace

void launch_estdt_mixed(const BoxDev *boxes, const long long *cell_pref, int nbox, long long total,
                        const double *state, const SchemeConsts *K, const double *a_dev,
                        unsigned long long *dtacc, cudaStream_t st) {
  long long g = (total + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  k_estdt_mixed<<<(int)g, 256, 0, st>>>(boxes, cell_pref, nbox, total, state, K, a_dev, dtacc);
}

}  // namespace nyx
