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
//
// Launch shapes: the ghost fill of a whole level runs alone, 256 threads per
// block.  The copies of the overlapped host step (scatter, per-group fill,
// gather) run 128 threads per block at no more than 32 registers per
// thread: the fused advance holds 80 registers x 768 threads of every SM
// (61,440 of 65,536), which leaves room for exactly one such block beside
// it, so one box group's copies run on the SMs while another group advances
// instead of waiting for its end.
constexpr int COPY_THREADS = 128;

template <int NC, int BESIDE>
__global__ void __launch_bounds__(BESIDE ? COPY_THREADS : 256, BESIDE ? 16 : 4)
    k_fill_rects(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects, int nrect) {
  for (int r = blockIdx.x; r < nrect; r += gridDim.x) {
    const FillRect &R = rects[r];
    const BoxDev &bd = boxes[R.dst_box];
    const BoxDev &bs = boxes[R.src_box];
    // only what the copy needs, so that it fits in 32 registers
    const long long dstr = bd.stride, sstr = bs.stride;
    double *D = field + (long long)ncomp * bd.pref;
    const double *S = field + (long long)ncomp * bs.pref;
    const int dN0 = bd.N[0], dN1 = bd.N[1], sN0 = bs.N[0], sN1 = bs.N[1];
    const int e0 = R.ext[0], e1 = R.ext[1], n = R.ext[0] * R.ext[1] * R.ext[2];
    const int d0 = R.dlo[0] + 4, d1 = R.dlo[1] + 4, d2 = R.dlo[2] + 4;
    const int s0 = R.slo[0] + 4, s1 = R.slo[1] + 4, s2 = R.slo[2] + 4;
    const int t0 = R.sstep[0], t1 = R.sstep[1], t2 = R.sstep[2];
    if constexpr (NC > 0 && !BESIDE) {
      // 16-byte copies (two x cells per thread, double2 loads and stores)
      // when both sides' rows start and stay on 16-byte boundaries: an even
      // x extent copied forward, even row starts (box offset + first x),
      // row lengths and component strides, a 16-byte aligned field
      const long long dref = (long long)ncomp * bd.pref + d0, sref = (long long)ncomp * bs.pref + s0;
      const bool vec = t0 == 1 && !(e0 & 1) && !(dref & 1) && !(sref & 1) && !(dN0 & 1) &&
                       !(sN0 & 1) && !(dstr & 1) && !(sstr & 1) &&
                       !(reinterpret_cast<unsigned long long>(field) & 15ull);
      if (vec) {
        const int h0 = e0 >> 1, nv = n >> 1;
        for (int f = threadIdx.x; f < nv; f += blockDim.x) {
          const int i = 2 * (f % h0);
          const int u = f / h0;
          const int j = u % e1;
          const int k = u / e1;
          const long long di = ((long long)(d2 + k) * dN1 + (d1 + j)) * dN0 + (d0 + i);
          const long long si = ((long long)(s2 + t2 * k) * sN1 + (s1 + t1 * j)) * sN0 + (s0 + i);
          double2 v[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) v[c] = __ldg(reinterpret_cast<const double2 *>(S + c * sstr + si));
#pragma unroll
          for (int c = 0; c < NC; ++c) *reinterpret_cast<double2 *>(D + c * dstr + di) = v[c];
        }
        continue;
      }
    }
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
      const int i = f % e0;
      const int u = f / e0;
      const int j = u % e1;
      const int k = u / e1;
      const long long di = ((long long)(d2 + k) * dN1 + (d1 + j)) * dN0 + (d0 + i);
      const long long si = ((long long)(s2 + t2 * k) * sN1 + (s1 + t1 * j)) * sN0 + (s0 + t0 * i);
      if constexpr (NC > 0) {
        double v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = __ldg(S + c * sstr + si);
#pragma unroll
        for (int c = 0; c < NC; ++c) D[c * dstr + di] = v[c];
      } else {
        for (int c = 0; c < ncomp; ++c) D[c * dstr + di] = S[c * sstr + si];
      }
    }
  }
}

// Copy between a level field (6 components, with ghosts) and its valid cells
// packed box by box (box b at 6 cell_pref[b], component-major, x fastest).
// One block per plane of each box (plane_pref[b]: the first block of box
// b); consecutive threads take consecutive x cells on both sides.
__global__ void __launch_bounds__(COPY_THREADS, 16)
    k_valid_copy(double *field, double *packed, const BoxDev *boxes, const long long *cell_pref,
                 const int *plane_pref, int nbox, int blk0, int to_field) {
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

// Load the copy kernels of the overlapped host step (with lazy module
// loading, a kernel's first launch may wait for every kernel and copy in
// flight, which would stall the first overlapped step behind its inputs).
int preload_copy_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_fill_rects<NCONS, 1>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_valid_copy);
  return (int)e;
}

void launch_valid_copy(double *field, double *packed, const BoxDev *boxes,
                       const long long *cell_pref, const int *plane_pref, int nbox, int nblocks,
                       int blk0, int to_field, cudaStream_t st) {
  if (nblocks < 1) return;
  k_valid_copy<<<nblocks, COPY_THREADS, 0, st>>>(field, packed, boxes, cell_pref, plane_pref,
                                                 nbox, blk0, to_field);
}

template <int BESIDE>
void fill_launch(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects, int nrect,
                 cudaStream_t st) {
  const int threads = BESIDE ? COPY_THREADS : 256;
  const int cap = BESIDE ? 152 * 32 : 152 * 16;
  const int grid = nrect < cap ? nrect : cap;
  if (ncomp == NCONS)
    k_fill_rects<NCONS, BESIDE><<<grid, threads, 0, st>>>(field, ncomp, boxes, rects, nrect);
  else if (ncomp == NGRAV)
    k_fill_rects<NGRAV, BESIDE><<<grid, threads, 0, st>>>(field, ncomp, boxes, rects, nrect);
  else
    k_fill_rects<0, BESIDE><<<grid, threads, 0, st>>>(field, ncomp, boxes, rects, nrect);
}

void launch_fill(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects,
                 const long long *rect_pref, int nrect, long long total, cudaStream_t st,
                 bool beside) {
  (void)rect_pref;
  if (nrect <= 0 || total <= 0) return;
  if (beside)
    fill_launch<1>(field, ncomp, boxes, rects, nrect, st);
  else
    fill_launch<0>(field, ncomp, boxes, rects, nrect, st);
}

}  // namespace nyx
