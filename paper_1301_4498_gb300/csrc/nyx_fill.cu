// nyx_fill.cu -- ghost-cell exchange of a level field (Sec. 4.1: every grid
// carries the same number of ghost cells on every side).  The host builds a
// list of copy rectangles once per plan (neighbour and periodic copies first,
// then the outflow passes x, y, z); one launch per pass copies them.
#include "nyx_internal.cuh"
#include "nyx_kernels.h"

namespace nyx {
namespace {

// One CTA per rectangle (grid-strided): consecutive threads copy
// consecutive x cells of a row, so both sides are read and written in
// coalesced runs, and no thread searches the rectangle list.  (One warp per
// rectangle measured slower on the large level: 6.8 against 6.0 ms.)  A ghost cell
// never overlaps the valid cell it copies, so each thread loads every
// component of its cell before storing any (NC > 0: that many components;
// 0: ncomp at run time, one at a time), instead of one dependent load and
// store per component.
template <int NC>
__global__ void k_fill_rects(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects,
                             int nrect) {
  for (int r = blockIdx.x; r < nrect; r += gridDim.x) {
    const FillRect R = rects[r];
    const BoxDev bd = boxes[R.dst_box];
    const BoxDev bs = boxes[R.src_box];
    double *D = field + (long long)ncomp * bd.pref;
    const double *S = field + (long long)ncomp * bs.pref;
    const int n = R.ext[0] * R.ext[1] * R.ext[2];
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
      const int i = f % R.ext[0];
      const int u = f / R.ext[0];
      const int j = u % R.ext[1];
      const int k = u / R.ext[1];
      const long long di = cell_index(bd, R.dlo[0] + i, R.dlo[1] + j, R.dlo[2] + k);
      const long long si = cell_index(bs, R.slo[0] + R.sstep[0] * i, R.slo[1] + R.sstep[1] * j,
                                      R.slo[2] + R.sstep[2] * k);
      if constexpr (NC > 0) {
        double v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = __ldg(S + c * bs.stride + si);
#pragma unroll
        for (int c = 0; c < NC; ++c) D[c * bd.stride + di] = v[c];
      } else {
        for (int c = 0; c < ncomp; ++c) D[c * bd.stride + di] = S[c * bs.stride + si];
      }
    }
  }
}

// Copy between a level field (6 components, with ghosts) and its valid cells
// packed box by box (box b at 6 cell_pref[b], component-major, x fastest).
// One block per plane of each box (plane_pref[b]: the first block of box
// b); consecutive threads take consecutive x cells on both sides.
__global__ void k_valid_copy(double *field, double *packed, const BoxDev *boxes,
                             const long long *cell_pref, const int *plane_pref, int nbox,
                             int blk0, int to_field) {
  const int blk = blk0 + (int)blockIdx.x;
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (plane_pref[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const BoxDev X = boxes[lo];
  const int k = blk - plane_pref[lo];
  const int nxy = X.n[0] * X.n[1];
  const long long vol = (long long)nxy * X.n[2];
  double *F = field + NCONS * X.pref;
  double *Pk = packed + NCONS * cell_pref[lo] + (long long)k * nxy;
  for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
    const int i = t % X.n[0], j = t / X.n[0];
    const long long id = cell_index(X, i, j, k);
    if (to_field) {
#pragma unroll
      for (int c = 0; c < NCONS; ++c) F[c * X.stride + id] = Pk[c * vol + t];
    } else {
#pragma unroll
      for (int c = 0; c < NCONS; ++c) Pk[c * vol + t] = F[c * X.stride + id];
    }
  }
}

}  // namespace

void launch_valid_copy(double *field, double *packed, const BoxDev *boxes,
                       const long long *cell_pref, const int *plane_pref, int nbox, int nblocks,
                       int blk0, int to_field, cudaStream_t st) {
  if (nblocks < 1) return;
  k_valid_copy<<<nblocks, 256, 0, st>>>(field, packed, boxes, cell_pref, plane_pref, nbox, blk0,
                                       to_field);
}

void launch_fill(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects,
                 const long long *rect_pref, int nrect, long long total, cudaStream_t st) {
  (void)rect_pref;
  if (nrect <= 0 || total <= 0) return;
  const int grid = nrect < 152 * 16 ? nrect : 152 * 16;
  if (ncomp == NCONS)
    k_fill_rects<NCONS><<<grid, 256, 0, st>>>(field, ncomp, boxes, rects, nrect);
  else if (ncomp == NGRAV)
    k_fill_rects<NGRAV><<<grid, 256, 0, st>>>(field, ncomp, boxes, rects, nrect);
  else
    k_fill_rects<0><<<grid, 256, 0, st>>>(field, ncomp, boxes, rects, nrect);
}

}  // namespace nyx
