// nyx_fill.cu -- ghost-cell exchange of a level field (Sec. 4.1: every grid
// carries the same number of ghost cells on every side).  The host builds a
// list of copy rectangles once per plan (neighbour and periodic copies first,
// then the outflow passes x, y, z); one launch per pass copies them.
#include "nyx_internal.cuh"
#include "nyx_kernels.h"

namespace nyx {
namespace {

// One thread per (cell of a rectangle); rect_pref[r] = cells before rect r.
__global__ void k_fill(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects,
                       const long long *rect_pref, int nrect, long long total) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nrect - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (rect_pref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const FillRect R = rects[lo];
    long long f = t - rect_pref[lo];
    int i = (int)(f % R.ext[0]);
    long long u = f / R.ext[0];
    int j = (int)(u % R.ext[1]);
    int k = (int)(u / R.ext[1]);
    const BoxDev bd = boxes[R.dst_box];
    const BoxDev bs = boxes[R.src_box];
    long long di = cell_index(bd, R.dlo[0] + i, R.dlo[1] + j, R.dlo[2] + k);
    long long si = cell_index(bs, R.slo[0] + R.sstep[0] * i, R.slo[1] + R.sstep[1] * j,
                              R.slo[2] + R.sstep[2] * k);
    double *D = field + (long long)ncomp * bd.pref;
    const double *S = field + (long long)ncomp * bs.pref;
    for (int c = 0; c < ncomp; ++c) D[c * bd.stride + di] = S[c * bs.stride + si];
  }
}

}  // namespace

void launch_fill(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects,
                 const long long *rect_pref, int nrect, long long total, cudaStream_t st) {
  if (nrect <= 0 || total <= 0) return;
  long long g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_fill<<<(int)g, 256, 0, st>>>(field, ncomp, boxes, rects, rect_pref, nrect, total);
}

}  // namespace nyx
