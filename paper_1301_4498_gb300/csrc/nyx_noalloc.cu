// nyx_noalloc.cu -- nyx_hydro_estdt_noalloc: the level CFL reduction without
// any device allocation, for callers that cannot call cudaMalloc (for example
// code that runs where a framework owns every device allocation, or a
// real-time loop that must not enter the allocator).
//
// Its scratch (box table, per-box cell offsets, the min accumulator and the
// scheme constants) lives in one file-scope __device__ array of fixed size,
// so every GPU that loads this library holds it until the process exits.
// All calls share that array, and it keeps the contents of the last call.
// Two calls that overlap on the GPU (on different streams, or from several
// host threads) therefore race; calls on one stream are ordered and safe.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "nyx_hydro.h"
#include "nyx_internal.cuh"
#include "nyx_kernels.h"

namespace {

using namespace nyx;

constexpr int kMaxBoxes = NYX_NOALLOC_MAX_BOXES;

// Byte layout of the scratch array.
constexpr size_t kBoxBytes = sizeof(BoxDev) * kMaxBoxes;
constexpr size_t kPrefOff = (kBoxBytes + 255) / 256 * 256;
constexpr size_t kAccOff = (kPrefOff + sizeof(long long) * kMaxBoxes + 255) / 256 * 256;
constexpr size_t kConstOff = kAccOff + 256;
constexpr size_t kScratchBytes = (kConstOff + sizeof(SchemeConsts) + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_estdt_scratch[kScratchBytes];

// Host staging for the tables (kept static so the call allocates nothing).
struct Staging {
  std::mutex mu;
  BoxDev boxes[kMaxBoxes];
  long long pref[kMaxBoxes];
  unsigned char *dev_ptr[64] = {nullptr};  // device address of the array, per device
};
Staging &staging() {
  static Staging s;
  return s;
}

int fail(int code, const std::string &m) {
  record_error(m.c_str());
  return code;
}

}  // namespace

extern "C" int nyx_hydro_estdt_noalloc(const nyx_level_desc *level, const nyx_hydro_params *params,
                                       const double *state, const double *a_dev, double *dt_dev,
                                       void *stream) {
  record_error("");
  if (!level || !params || !state || !a_dev || !dt_dev)
    return fail(NYX_EINVAL, "null argument");
  if (level->nboxes <= 0 || !level->boxes) return fail(NYX_EINVAL, "level has no boxes");
  if (level->nboxes > kMaxBoxes)
    return fail(NYX_EINVAL, "level has " + std::to_string(level->nboxes) +
                                " boxes; the allocation-free CFL reduction takes at most " +
                                std::to_string(kMaxBoxes));
  if (level->ng != 4) return fail(NYX_EINVAL, "ghost width must be 4");
  if (!(params->gamma > 1.0) || !std::isfinite(params->gamma) || !(params->cfl > 0.0) ||
      !std::isfinite(params->cfl) || !(params->small_pres > 0.0) ||
      !std::isfinite(params->small_pres))
    return fail(NYX_EINVAL, "invalid scheme parameters");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(NYX_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return fail(NYX_EINVAL, "device index out of range");
  cudaStream_t st = (cudaStream_t)stream;
  // The tables are copied from host memory on every call, which a stream
  // that is being captured into a graph cannot take.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess)
    return fail(NYX_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(NYX_EINVAL, "the stream is capturing; call nyx_hydro_estdt_noalloc outside stream capture");

  Staging &S = staging();
  std::lock_guard<std::mutex> lock(S.mu);
  if (!S.dev_ptr[dev]) {
    // Set-up, once per device, with that device current: the array's name is
    // only a host-side stand-in, the kernels need its device address.
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_estdt_scratch);
    if (e != cudaSuccess)
      return fail(NYX_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    S.dev_ptr[dev] = (unsigned char *)p;
  }
  unsigned char *base = S.dev_ptr[dev];

  long long pref = 0, cells = 0;
  for (int b = 0; b < level->nboxes; ++b) {
    const nyx_box &X = level->boxes[b];
    BoxDev &D = S.boxes[b];
    for (int a = 0; a < 3; ++a) {
      const int n = X.hi[a] - X.lo[a] + 1;
      if (n <= 0 || (n & 1) || !(X.dx[a] > 0.0) || !std::isfinite(X.dx[a]))
        return fail(NYX_EINVAL, "box " + std::to_string(b) + " has a bad extent or dx");
      D.n[a] = n;
      D.N[a] = n + 8;
      D.dx[a] = X.dx[a];
      D.idx[a] = 1.0 / X.dx[a];
    }
    const long long vol = (long long)D.N[0] * D.N[1] * D.N[2];
    D.stride = (vol + 31) / 32 * 32;  // the layout of nyx_hydro_layout
    D.pref = pref;
    pref += D.stride;
    S.pref[b] = cells;
    cells += (long long)D.n[0] * D.n[1] * D.n[2];
  }
  SchemeConsts K{};
  K.gamma = params->gamma;
  K.gm1 = params->gamma - 1.0;
  K.igm1 = 1.0 / K.gm1;
  K.small_pres = params->small_pres;
  K.cfl = params->cfl;
  const unsigned long long inf = 0x7ff0000000000000ULL;  // the accumulator starts at +inf

  BoxDev *d_boxes = (BoxDev *)base;
  long long *d_pref = (long long *)(base + kPrefOff);
  unsigned long long *d_acc = (unsigned long long *)(base + kAccOff);
  SchemeConsts *d_K = (SchemeConsts *)(base + kConstOff);
  const int nb = level->nboxes;
  if ((e = cudaMemcpyAsync(d_boxes, S.boxes, sizeof(BoxDev) * nb, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(d_pref, S.pref, sizeof(long long) * nb, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(d_acc, &inf, sizeof(inf), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(d_K, &K, sizeof(K), cudaMemcpyHostToDevice, st)))
    return fail(NYX_ECUDA, std::string("copy to the scratch array: ") + cudaGetErrorString(e));
  launch_estdt(d_boxes, d_pref, nb, cells, state, d_K, a_dev, d_acc, st);
  launch_dt_finalize(d_K, d_acc, dt_dev, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NYX_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  // Copies from pageable host memory return once their source has been
  // staged, so the host tables may be rewritten by the next call.
  return NYX_OK;
}
