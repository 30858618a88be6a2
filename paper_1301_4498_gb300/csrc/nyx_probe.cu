// nyx_probe.cu -- nyx_alu_peak: the FP32 and FP64 fused multiply-add
// throughput of the current device, measured with CUDA events.  These are
// the ALU denominators of the advance's roofline (the update is FP64, the
// reconstruction, tracing and Riemann solves of the mixed path FP32).
//
// Each thread runs CH independent multiply-add chains a = a*b + c (b just
// below 1, c small, so the values stay normal and bounded) for a fixed
// number of iterations; the chains are summed at the end and stored only if
// the sum takes an impossible value, which keeps every operation live
// without any memory traffic.  The grid holds 8 blocks of 256 threads per
// SM, enough warps to hide the pipes' latency with CH chains per thread.
#include <cuda_runtime.h>

#include <string>

#include "nyx_hydro.h"
#include "nyx_kernels.h"

namespace {

constexpr int CH = 8;        // independent chains per thread
constexpr int THREADS = 256;
constexpr int BLOCKS_PER_SM = 8;

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <class T>
__global__ void __launch_bounds__(THREADS) k_fma_chains(T *sink, int iters, T b, T c) {
  T a[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = T(threadIdx.x & 7) * T(0.125) + T(k + 1);
#pragma unroll 1
  for (int i = 0; i < iters; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int k = 0; k < CH; ++k) a[k] = fma_t(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  if (s == T(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true
}

int fail(int code, const std::string &m) {
  nyx::record_error(m.c_str());
  return code;
}

}  // namespace

extern "C" int nyx_alu_peak(int pipe, double seconds, void *stream, double *fma_per_s) {
  nyx::record_error("");
  if (!fma_per_s || (pipe != 0 && pipe != 1) || !(seconds > 0.0) || seconds > 10.0)
    return fail(NYX_EINVAL, "nyx_alu_peak: pipe must be 0 (FP32) or 1 (FP64), 0 < seconds <= 10");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(NYX_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  const int blocks = nsm * BLOCKS_PER_SM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(NYX_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
  }
  // the sink is never written (the store's condition is never met)
  auto launch = [&](int iters) {
    if (pipe == 0)
      k_fma_chains<float><<<blocks, THREADS, 0, st>>>(nullptr, iters, 0.99999994f, 1e-7f);
    else
      k_fma_chains<double><<<blocks, THREADS, 0, st>>>(nullptr, iters, 0.9999999999999999, 1e-15);
  };
  // calibrate the iteration count so that one launch takes about 1/5 of the time asked for
  int iters = pipe == 0 ? 1 << 14 : 1 << 9;
  float ms = 0.f;
  for (int rep = 0; rep < 12; ++rep) {
    launch(iters);  // warm-up at this size
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= 200.0 * seconds || iters >= (1 << 26)) break;
    iters *= 2;
  }
  double best = 0.0;
  if (e == cudaSuccess) {
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, st);
      launch(iters);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      const double rate = (double)blocks * THREADS * CH * (double)iters / (ms * 1e-3);
      if (rate > best) best = rate;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(NYX_ECUDA, std::string("nyx_alu_peak: ") + cudaGetErrorString(e));
  *fma_per_s = best;
  return NYX_OK;
}
