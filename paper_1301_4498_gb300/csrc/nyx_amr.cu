// nyx_amr.cu -- coupling of a fine level to the coarse level it refines by 2,
// with no subcycling (Sec. 4.2: both levels take the same dt).
//
//  * Interpolation (Sec. 4.1): in each coarse cell a linear profile from the
//    MC-limited slopes along the three axes, all scaled by one factor so that
//    no fine value leaves the range of the coarse cell and its six face
//    neighbours, evaluated at the fine cell centres.  It fills the fine ghost
//    cells from the coarse state at t^n (Sec. 4.3 Step 2: coarse Dirichlet
//    data) and makes initial fine data.
//  * Reflux (Sec. 4.3 Steps 2 and 8): coarse cells outside the fine level
//    that share a face with it take the mean of the 4 fine fluxes through
//    that face instead of their own, with the update's coefficients.
//  * Average down (Sec. 4.3 Step 8): coarse cells under the fine level take
//    the mean of their 8 fine cells.
//
// The host cuts each operation into rectangles that lie in one fine box and
// one coarse box (after periodic wrap); one CTA takes one rectangle, its
// threads consecutive cells (x fastest), so both sides are read in
// coalesced runs.  Reflux runs in six launches, one per face orientation:
// within one orientation no coarse cell is met twice, so there are no
// atomics and the corrections of a cell are added in a fixed order.  The
// arithmetic is FP64 with the expression order of the update (this unit is
// built without FMA contraction).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "nyx_hydro.h"
#include "nyx_internal.cuh"
#include "nyx_kernels.h"
#include "nyx_plan.h"

using namespace nyx;
using namespace nyx::host;

namespace {

// Fine cells [flo, flo+ext) (local to fine box fbox, ghosts negative) whose
// coarse cells lie in coarse box cbox: rel = local + base >= 0 is the fine
// offset from the fine domain origin after the periodic shift; the coarse
// cell is rel/2 + coff (local to cbox), the fine offset inside it rel & 1.
struct InterpRect {
  int fbox, cbox;
  int flo[3], ext[3];
  int base[3], coff[3];
};

// Coarse cells P outside fine box fbox across its face of axis d (high: past
// the high face), P in coarse box cbox: first P plo (local to cbox), extents
// along the tangential axes t1 < t2, and the fine tangential face index of
// the first P (local to the fine box's flux arrays).
struct FaceRect {
  int fbox, cbox, d, high;
  int plo[3];
  int ext[2];
  int ft0[2];
};

// Coarse cells [clo, clo+ext) of coarse box cbox under fine box fbox; the
// first one's first fine cell is flo (local to fbox).
struct AvgRect {
  int fbox, cbox;
  int clo[3], ext[3], flo[3];
};

constexpr int kMaxGrid = 152 * 16;

__device__ __forceinline__ double mc_slope_d(double sm, double s0, double sp) {
  double dc = 0.5 * (sp - sm);
  double dl = s0 - sm;
  double dr = sp - s0;
  if (dl * dr > 0.0) {
    double m = fabs(dc);
    double b = 2.0 * fabs(dl);
    double c = 2.0 * fabs(dr);
    if (b < m) m = b;
    if (c < m) m = c;
    return copysign(m, dc);
  }
  return 0.0;
}

// One thread per coarse cell of the rectangle's footprint: the slopes and the
// limiter factor of a coarse cell are formed once and give its (up to 8)
// fine cells, each evaluated with the same expression as cell by cell.
__global__ void k_amr_interp(const double *cf, double *ff, int ncomp, const BoxDev *cboxes,
                             const BoxDev *fboxes, const InterpRect *rects, int nrect) {
  for (int r = blockIdx.x; r < nrect; r += gridDim.x) {
    const InterpRect R = rects[r];
    const BoxDev bc = cboxes[R.cbox];
    const BoxDev bf = fboxes[R.fbox];
    const double *C = cf + (long long)ncomp * bc.pref;
    double *F = ff + (long long)ncomp * bf.pref;
    const long long s1 = bc.N[0], s2 = (long long)bc.N[0] * bc.N[1];
    int c0[3], ne[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c0[d] = (R.flo[d] + R.base[d]) >> 1;
      ne[d] = ((R.flo[d] + R.ext[d] - 1 + R.base[d]) >> 1) - c0[d] + 1;
    }
    const int n = ne[0] * ne[1] * ne[2];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int cr[3] = {c0[0] + q % ne[0], c0[1] + (q / ne[0]) % ne[1], c0[2] + q / (ne[0] * ne[1])};
      const long long cid = cell_index(bc, cr[0] + R.coff[0], cr[1] + R.coff[1], cr[2] + R.coff[2]);
      const long long st[3] = {1, s1, s2};
      for (int c = 0; c < ncomp; ++c) {
        const double *u_ = C + c * bc.stride;
        const double uc = u_[cid];
        double s[3], umin = uc, umax = uc;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double um = u_[cid - st[d]], up = u_[cid + st[d]];
          s[d] = mc_slope_d(um, uc, up);
          if (um < umin) umin = um;
          if (up < umin) umin = up;
          if (um > umax) umax = um;
          if (up > umax) umax = up;
        }
        const double dev = 0.25 * (fabs(s[0]) + fabs(s[1]) + fabs(s[2]));
        double alpha = 1.0;
        if (dev > 0.0) {
          if (uc + dev > umax) alpha = fmin(alpha, (umax - uc) / dev);
          if (uc - dev < umin) alpha = fmin(alpha, (uc - umin) / dev);
        }
        double *o_ = F + c * bf.stride;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          const int f0 = 2 * cr[0] + (o & 1) - R.base[0];
          const int f1 = 2 * cr[1] + ((o >> 1) & 1) - R.base[1];
          const int f2 = 2 * cr[2] + (o >> 2) - R.base[2];
          if (f0 < R.flo[0] || f0 >= R.flo[0] + R.ext[0] || f1 < R.flo[1] ||
              f1 >= R.flo[1] + R.ext[1] || f2 < R.flo[2] || f2 >= R.flo[2] + R.ext[2])
            continue;
          const double xo = (o & 1) ? 0.25 : -0.25, yo = ((o >> 1) & 1) ? 0.25 : -0.25,
                       zo = (o >> 2) ? 0.25 : -0.25;
          o_[cell_index(bf, f0, f1, f2)] = uc + alpha * (s[0] * xo + s[1] * yo + s[2] * zo);
        }
      }
    }
  }
}

// Offset of the direction-d block of a box's flux store: x block (6, nz, ny,
// nx+1), then y (6, nz, ny+1, nx), then z (6, nz+1, ny, nx).
__device__ __forceinline__ long long flux_block(const BoxDev &b, int d, int e[3]) {
  long long off = 0;
  for (int a = 0; a < d; ++a) {
    int ea[3] = {b.n[0], b.n[1], b.n[2]};
    ea[a] += 1;
    off += 6LL * ea[0] * ea[1] * ea[2];
  }
  e[0] = b.n[0];
  e[1] = b.n[1];
  e[2] = b.n[2];
  e[d] += 1;
  return off;
}

__global__ void k_amr_reflux(double *cs, const double *cflux, const long long *cflux_off,
                             const double *fflux, const long long *fflux_off,
                             const BoxDev *cboxes, const BoxDev *fboxes,
                             const unsigned char *covered, const long long *ccell_pref,
                             const StepConsts *SC, const FaceRect *rects, int nrect) {
  const StepConsts sc = *SC;
  const double coef[6] = {sc.dtp, sc.dt * sc.ian, sc.dt * sc.ian, sc.dt * sc.ian,
                          sc.ahdt * sc.ian2, sc.ahdt * sc.ian2};
  for (int r = blockIdx.x; r < nrect; r += gridDim.x) {
    const FaceRect R = rects[r];
    const BoxDev bc = cboxes[R.cbox];
    const BoxDev bf = fboxes[R.fbox];
    const int d = R.d, t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    int ce[3], fe[3];
    const double *Fc = cflux + cflux_off[R.cbox] + flux_block(bc, d, ce);
    const double *Ff = fflux + fflux_off[R.fbox] + flux_block(bf, d, fe);
    const long long cv = (long long)ce[0] * ce[1] * ce[2];
    const long long fv = (long long)fe[0] * fe[1] * fe[2];
    const int ffi = R.high ? bf.n[d] : 0;
    const double idx = bc.idx[d];
    double *U = cs + 6LL * bc.pref;
    const int n = R.ext[0] * R.ext[1];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int a1 = q % R.ext[0], a2 = q / R.ext[0];
      int P[3];
      P[d] = R.plo[d];
      P[t1] = R.plo[t1] + a1;
      P[t2] = R.plo[t2] + a2;
      if (covered[ccell_pref[R.cbox] + ((long long)P[2] * bc.n[1] + P[1]) * bc.n[0] + P[0]]) continue;
      int cfi[3] = {P[0], P[1], P[2]};
      if (!R.high) cfi[d] += 1;  // the outside cell's high face
      const long long cid = ((long long)cfi[2] * ce[1] + cfi[1]) * ce[0] + cfi[0];
      const long long sid = cell_index(bc, P[0], P[1], P[2]);
      const int f1 = R.ft0[0] + 2 * a1, f2 = R.ft0[1] + 2 * a2;
      for (int c = 0; c < 6; ++c) {
        double fsum = 0.0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          int fi[3];
          fi[d] = ffi;
          fi[t1] = f1 + (s & 1);
          fi[t2] = f2 + (s >> 1);
          const double v = Ff[c * fv + ((long long)fi[2] * fe[1] + fi[1]) * fe[0] + fi[0]];
          fsum = (s == 0) ? v : fsum + v;
        }
        const double favg = 0.25 * fsum;
        const double corr = coef[c] * ((favg - Fc[c * cv + cid]) * idx);
        double *u_ = U + c * bc.stride + sid;
        *u_ = R.high ? *u_ + corr : *u_ - corr;
      }
    }
  }
}

__global__ void k_amr_avgdown(const double *ff, double *cf, int ncomp, const BoxDev *cboxes,
                              const BoxDev *fboxes, const AvgRect *rects, int nrect) {
  for (int r = blockIdx.x; r < nrect; r += gridDim.x) {
    const AvgRect R = rects[r];
    const BoxDev bc = cboxes[R.cbox];
    const BoxDev bf = fboxes[R.fbox];
    const double *F = ff + (long long)ncomp * bf.pref;
    double *C = cf + (long long)ncomp * bc.pref;
    const int n = R.ext[0] * R.ext[1] * R.ext[2];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int i = q % R.ext[0];
      const int u = q / R.ext[0];
      const int j = u % R.ext[1];
      const int k = u / R.ext[1];
      const long long cid = cell_index(bc, R.clo[0] + i, R.clo[1] + j, R.clo[2] + k);
      const int f0 = R.flo[0] + 2 * i, f1 = R.flo[1] + 2 * j, f2 = R.flo[2] + 2 * k;
      for (int c = 0; c < ncomp; ++c) {
        const double *v_ = F + c * bf.stride;
        double s = 0.0;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          const double v = v_[cell_index(bf, f0 + (o & 1), f1 + ((o >> 1) & 1), f2 + (o >> 2))];
          s = (o == 0) ? v : s + v;
        }
        C[c * bc.stride + cid] = 0.125 * s;
      }
    }
  }
}

int grid_of(int n) { return std::max(1, std::min(n, kMaxGrid)); }

// Coarse boxes of one domain in a uniform bin grid (bins of the largest box
// extent), for rectangle queries in the coarse index space.
struct CoarseBins {
  int bs = 1, nb[3] = {1, 1, 1}, lo[3] = {0, 0, 0};
  std::vector<std::vector<int>> cell;
};

}  // namespace

// Graph cache key: both levels' buffers and cur, the scalar arrays, nsteps.
using AmrKey = std::tuple<const void *, const void *, const void *, const void *, const void *,
                          const void *, int, const void *, const void *, int, int>;

struct nyx_amr {
  nyx_plan *C = nullptr, *F = nullptr;
  InterpRect *d_ig = nullptr, *d_ia = nullptr;
  int n_ig = 0, n_ia = 0;
  FaceRect *d_face[6] = {nullptr};
  int n_face[6] = {0};
  AvgRect *d_avg = nullptr;
  int n_avg = 0;
  unsigned char *d_cov = nullptr;
  std::map<AmrKey, std::pair<cudaGraphExec_t, long long>> graphs;
};

namespace {

void free_amr(nyx_amr *A) {
  if (!A) return;
  cudaFree(A->d_ig);
  cudaFree(A->d_ia);
  for (int o = 0; o < 6; ++o) cudaFree(A->d_face[o]);
  cudaFree(A->d_avg);
  cudaFree(A->d_cov);
  for (auto &kv : A->graphs) cudaGraphExecDestroy(kv.second.first);
  delete A;
}

template <class T>
int upload(const std::vector<T> &h, T **d) {
  *d = nullptr;
  if (h.empty()) return NYX_OK;
  cudaError_t e = cudaMalloc(d, sizeof(T) * h.size());
  if (e != cudaSuccess)
    return e == cudaErrorMemoryAllocation ? fail(NYX_ENOMEM, "amr table allocation failed")
                                          : cuda_fail(e, "cudaMalloc");
  CK(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return NYX_OK;
}

bool box_intersect(const int alo[3], const int ahi[3], const int blo[3], const int bhi[3],
                   int olo[3], int ohi[3]) {
  for (int d = 0; d < 3; ++d) {
    olo[d] = std::max(alo[d], blo[d]);
    ohi[d] = std::min(ahi[d], bhi[d]);
    if (olo[d] > ohi[d]) return false;
  }
  return true;
}

int floor2(int x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); }

// Split [lo, hi] (at most one domain length past either end) at the domain
// bounds: pieces with their shift into the domain.
void wrap_pieces(int lo, int hi, int dlo, int dhi, std::vector<std::pair<std::pair<int, int>, int>> &out) {
  const int L = dhi - dlo + 1;
  out.clear();
  if (lo < dlo) out.push_back({{lo, std::min(hi, dlo - 1)}, L});
  if (hi >= dlo && lo <= dhi) out.push_back({{std::max(lo, dlo), std::min(hi, dhi)}, 0});
  if (hi > dhi) out.push_back({{std::max(lo, dhi + 1), hi}, -L});
}

struct Builder {
  const nyx_plan &C, &F;
  std::vector<CoarseBins> bins;
  explicit Builder(const nyx_plan &c, const nyx_plan &f) : C(c), F(f) {
    bins.resize(C.doms.size());
    for (size_t dm = 0; dm < C.doms.size(); ++dm) {
      CoarseBins &B = bins[dm];
      for (int a = 0; a < 3; ++a) B.lo[a] = C.doms[dm].lo[a];
      int bs = 1;
      for (int b = 0; b < C.nbox; ++b)
        if (C.boxes[b].domain == (int)dm)
          for (int a = 0; a < 3; ++a) bs = std::max(bs, C.boxes[b].hi[a] - C.boxes[b].lo[a] + 1);
      B.bs = bs;
      for (int a = 0; a < 3; ++a) B.nb[a] = (C.doms[dm].hi[a] - C.doms[dm].lo[a] + 1 + bs - 1) / bs;
      B.cell.assign((size_t)B.nb[0] * B.nb[1] * B.nb[2], {});
      for (int b = 0; b < C.nbox; ++b) {
        if (C.boxes[b].domain != (int)dm) continue;
        int l[3], h[3];
        for (int a = 0; a < 3; ++a) {
          l[a] = (C.boxes[b].lo[a] - B.lo[a]) / bs;
          h[a] = (C.boxes[b].hi[a] - B.lo[a]) / bs;
        }
        for (int k = l[2]; k <= h[2]; ++k)
          for (int j = l[1]; j <= h[1]; ++j)
            for (int i = l[0]; i <= h[0]; ++i)
              B.cell[((size_t)k * B.nb[1] + j) * B.nb[0] + i].push_back(b);
      }
    }
  }
  // coarse boxes of domain dm meeting [lo, hi] (inside the domain)
  std::vector<int> query(int dm, const int lo[3], const int hi[3]) const {
    const CoarseBins &B = bins[dm];
    std::vector<int> out;
    int l[3], h[3];
    for (int a = 0; a < 3; ++a) {
      l[a] = std::max(0, (lo[a] - B.lo[a]) / B.bs);
      h[a] = std::min(B.nb[a] - 1, (hi[a] - B.lo[a]) / B.bs);
    }
    for (int k = l[2]; k <= h[2]; ++k)
      for (int j = l[1]; j <= h[1]; ++j)
        for (int i = l[0]; i <= h[0]; ++i)
          for (int b : B.cell[((size_t)k * B.nb[1] + j) * B.nb[0] + i]) {
            int ol[3], oh[3];
            if (std::find(out.begin(), out.end(), b) == out.end() &&
                box_intersect(lo, hi, C.boxes[b].lo, C.boxes[b].hi, ol, oh))
              out.push_back(b);
          }
    std::sort(out.begin(), out.end());
    return out;
  }
  // interpolation rectangles of the fine cells [glo, ghi] (fine global, may
  // reach one domain length outside) of fine box fb
  void interp_rects(int fb, const int glo[3], const int ghi[3], std::vector<InterpRect> &out) const {
    const nyx_box &X = F.boxes[fb];
    const nyx_domain &DF = F.doms[X.domain];
    const nyx_domain &DC = C.doms[X.domain];
    std::vector<std::pair<std::pair<int, int>, int>> pc[3];
    for (int a = 0; a < 3; ++a) wrap_pieces(glo[a], ghi[a], DF.lo[a], DF.hi[a], pc[a]);
    for (auto &pz : pc[2])
      for (auto &py : pc[1])
        for (auto &px : pc[0]) {
          const std::pair<std::pair<int, int>, int> *p3[3] = {&px, &py, &pz};
          int sl[3], sh[3], shift[3], clo[3], chi[3];
          for (int a = 0; a < 3; ++a) {
            shift[a] = p3[a]->second;
            sl[a] = p3[a]->first.first + shift[a];
            sh[a] = p3[a]->first.second + shift[a];
            clo[a] = DC.lo[a] + floor2(sl[a] - DF.lo[a]);
            chi[a] = DC.lo[a] + floor2(sh[a] - DF.lo[a]);
          }
          for (int cb : query(X.domain, clo, chi)) {
            const nyx_box &Y = C.boxes[cb];
            int ol[3], oh[3];
            if (!box_intersect(clo, chi, Y.lo, Y.hi, ol, oh)) continue;
            InterpRect R;
            R.fbox = fb;
            R.cbox = cb;
            for (int a = 0; a < 3; ++a) {
              const int f0 = std::max(sl[a], DF.lo[a] + 2 * (ol[a] - DC.lo[a]));
              const int f1 = std::min(sh[a], DF.lo[a] + 2 * (oh[a] - DC.lo[a]) + 1);
              R.flo[a] = f0 - shift[a] - X.lo[a];
              R.ext[a] = f1 - f0 + 1;
              R.base[a] = X.lo[a] + shift[a] - DF.lo[a];
              R.coff[a] = DC.lo[a] - Y.lo[a];
            }
            out.push_back(R);
          }
        }
  }
};

// Rectangles of at most about kChunk cells, so that small hierarchies still
// give every SM work: interpolation rectangles are cut along z at coarse
// cell boundaries (each coarse cell stays in one piece), face and average
// rectangles along their slowest axis.
constexpr int kChunk = 4096;

void split_interp(const InterpRect &R, std::vector<InterpRect> &out) {
  const long long plane = (long long)R.ext[0] * R.ext[1];
  int step = (int)std::max<long long>(2, kChunk / std::max<long long>(1, plane)) & ~1;
  int z = R.flo[2];
  const int zend = R.flo[2] + R.ext[2];
  while (z < zend) {
    // the first piece ends on a coarse boundary: (z + base) even after it
    int e = std::min(zend, z + step);
    if (e < zend && ((e + R.base[2]) & 1)) ++e;
    InterpRect P = R;
    P.flo[2] = z;
    P.ext[2] = e - z;
    out.push_back(P);
    z = e;
  }
}

void split_face(const FaceRect &R, std::vector<FaceRect> &out) {
  const int t2 = (R.d == 2) ? 1 : 2;
  const int step = std::max(1, kChunk / std::max(1, R.ext[0]));
  for (int a = 0; a < R.ext[1]; a += step) {
    FaceRect P = R;
    P.plo[t2] = R.plo[t2] + a;
    P.ext[1] = std::min(step, R.ext[1] - a);
    P.ft0[1] = R.ft0[1] + 2 * a;
    out.push_back(P);
  }
}

void split_avg(const AvgRect &R, std::vector<AvgRect> &out) {
  const int step = std::max(1, kChunk / std::max(1, R.ext[0] * R.ext[1]));
  for (int a = 0; a < R.ext[2]; a += step) {
    AvgRect P = R;
    P.clo[2] = R.clo[2] + a;
    P.ext[2] = std::min(step, R.ext[2] - a);
    P.flo[2] = R.flo[2] + 2 * a;
    out.push_back(P);
  }
}

int build_tables(nyx_amr *A) {
  const nyx_plan &C = *A->C, &F = *A->F;
  Builder B(C, F);
  const int ng = 4;
  std::vector<InterpRect> ig, ia;
  std::vector<FaceRect> face[6];
  std::vector<AvgRect> avg;
  std::vector<unsigned char> cov((size_t)C.total_cells, 0);
  for (int fb = 0; fb < F.nbox; ++fb) {
    const nyx_box &X = F.boxes[fb];
    const nyx_domain &DF = F.doms[X.domain];
    const nyx_domain &DC = C.doms[X.domain];
    int glo[3], ghi[3], cl[3], ch[3];
    for (int a = 0; a < 3; ++a) {
      glo[a] = X.lo[a] - ng;
      ghi[a] = X.hi[a] + ng;
      cl[a] = DC.lo[a] + (X.lo[a] - DF.lo[a]) / 2;
      ch[a] = DC.lo[a] + (X.hi[a] + 1 - DF.lo[a]) / 2 - 1;
    }
    // every cell, and the six ghost slabs (z slabs whole, y slabs within the
    // valid z range, x slabs within the valid y and z ranges)
    B.interp_rects(fb, glo, ghi, ia);
    for (int a = 2; a >= 0; --a)
      for (int side = 0; side < 2; ++side) {
        int sl[3], sh[3];
        for (int e = 0; e < 3; ++e) {
          if (e == a) {
            sl[e] = side ? X.hi[e] + 1 : X.lo[e] - ng;
            sh[e] = side ? X.hi[e] + ng : X.lo[e] - 1;
          } else if (e > a) {
            sl[e] = X.lo[e];
            sh[e] = X.hi[e];
          } else {
            sl[e] = glo[e];
            sh[e] = ghi[e];
          }
        }
        B.interp_rects(fb, sl, sh, ig);
      }
    // average down, covered mask
    for (int cb : B.query(X.domain, cl, ch)) {
      const nyx_box &Y = C.boxes[cb];
      int ol[3], oh[3];
      if (!box_intersect(cl, ch, Y.lo, Y.hi, ol, oh)) continue;
      AvgRect R;
      R.fbox = fb;
      R.cbox = cb;
      for (int a = 0; a < 3; ++a) {
        R.clo[a] = ol[a] - Y.lo[a];
        R.ext[a] = oh[a] - ol[a] + 1;
        R.flo[a] = 2 * (ol[a] - cl[a]);
      }
      avg.push_back(R);
      const int nx = Y.hi[0] - Y.lo[0] + 1, ny = Y.hi[1] - Y.lo[1] + 1;
      for (int k = ol[2]; k <= oh[2]; ++k)
        for (int j = ol[1]; j <= oh[1]; ++j)
          for (int i = ol[0]; i <= oh[0]; ++i)
            cov[(size_t)C.cell_pref[cb] +
                ((size_t)(k - Y.lo[2]) * ny + (j - Y.lo[1])) * nx + (i - Y.lo[0])] = 1;
    }
    // reflux faces: the coarse layer outside each face of the footprint
    for (int d = 0; d < 3; ++d) {
      const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
      const int L = DC.hi[d] - DC.lo[d] + 1;
      for (int high = 0; high < 2; ++high) {
        int ll[3] = {cl[0], cl[1], cl[2]}, hh[3] = {ch[0], ch[1], ch[2]};
        int pd = high ? ch[d] + 1 : cl[d] - 1;
        if (pd < DC.lo[d]) pd += L;
        if (pd > DC.hi[d]) pd -= L;
        ll[d] = hh[d] = pd;
        for (int cb : B.query(X.domain, ll, hh)) {
          const nyx_box &Y = C.boxes[cb];
          int ol[3], oh[3];
          if (!box_intersect(ll, hh, Y.lo, Y.hi, ol, oh)) continue;
          FaceRect R;
          R.fbox = fb;
          R.cbox = cb;
          R.d = d;
          R.high = high;
          for (int a = 0; a < 3; ++a) R.plo[a] = ol[a] - Y.lo[a];
          R.ext[0] = oh[t1] - ol[t1] + 1;
          R.ext[1] = oh[t2] - ol[t2] + 1;
          R.ft0[0] = 2 * (ol[t1] - cl[t1]);
          R.ft0[1] = 2 * (ol[t2] - cl[t2]);
          face[2 * d + high].push_back(R);
        }
      }
    }
  }
  std::vector<InterpRect> ig2, ia2;
  for (const InterpRect &R : ig) split_interp(R, ig2);
  for (const InterpRect &R : ia) split_interp(R, ia2);
  ig.swap(ig2);
  ia.swap(ia2);
  for (int o = 0; o < 6; ++o) {
    std::vector<FaceRect> f2;
    for (const FaceRect &R : face[o]) split_face(R, f2);
    face[o].swap(f2);
  }
  std::vector<AvgRect> avg2;
  for (const AvgRect &R : avg) split_avg(R, avg2);
  avg.swap(avg2);
  int rc;
  if ((rc = upload(ig, &A->d_ig))) return rc;
  if ((rc = upload(ia, &A->d_ia))) return rc;
  A->n_ig = (int)ig.size();
  A->n_ia = (int)ia.size();
  for (int o = 0; o < 6; ++o) {
    if ((rc = upload(face[o], &A->d_face[o]))) return rc;
    A->n_face[o] = (int)face[o].size();
  }
  if ((rc = upload(avg, &A->d_avg))) return rc;
  A->n_avg = (int)avg.size();
  if ((rc = upload(cov, &A->d_cov))) return rc;
  return NYX_OK;
}

int check_pair(const nyx_plan &C, const nyx_plan &F) {
  if (C.doms.size() != F.doms.size())
    return fail(NYX_EINVAL, "the fine plan must have one domain per coarse domain");
  for (size_t d = 0; d < C.doms.size(); ++d)
    for (int a = 0; a < 3; ++a) {
      if (F.doms[d].lo[a] != 2 * C.doms[d].lo[a] || F.doms[d].hi[a] != 2 * C.doms[d].hi[a] + 1)
        return fail(NYX_EINVAL, "fine domain " + std::to_string(d) +
                                    " is not the ratio-2 refinement of the coarse one");
      for (int s = 0; s < 2; ++s)
        if (C.doms[d].bc[3 * s + a] != NYX_BC_PERIODIC || F.doms[d].bc[3 * s + a] != NYX_BC_PERIODIC)
          return fail(NYX_EINVAL, "coarse-fine coupling needs periodic domains");
    }
  for (int b = 0; b < F.nbox; ++b)
    for (int a = 0; a < 3; ++a)
      if (F.boxes[b].lo[a] % 2 != 0 || (F.boxes[b].hi[a] + 1) % 2 != 0)
        return fail(NYX_EINVAL, "fine box " + std::to_string(b) +
                                    " does not start and end on coarse cell boundaries");
  if (!C.prm.keep_fluxes || !F.prm.keep_fluxes)
    return fail(NYX_EINVAL, "both plans need keep_fluxes = 1 for the reflux");
  if (!F.prm.coarse_fine) return fail(NYX_EINVAL, "the fine plan needs coarse_fine = 1");
  if (C.prm.coarse_fine) return fail(NYX_EINVAL, "the coarse plan must cover its domains");
  if (C.prm.precision != F.prm.precision)
    return fail(NYX_EINVAL, "both plans need the same precision");
  if (C.stream != F.stream) return fail(NYX_EINVAL, "both plans need the same stream");
  return NYX_OK;
}

int enqueue_reflux(nyx_amr *A, double *coarse_new) {
  nyx_plan &C = *A->C, &F = *A->F;
  for (int o = 0; o < 6; ++o) {
    if (!A->n_face[o]) continue;
    k_amr_reflux<<<grid_of(A->n_face[o]), 128, 0, C.stream>>>(
        coarse_new, C.d_flux, C.d_flux_off, F.d_flux, F.d_flux_off, C.d_boxes, F.d_boxes, A->d_cov,
        C.d_cell_pref, C.d_SC, A->d_face[o], A->n_face[o]);
    C.launches += 1;
  }
  return NYX_OK;
}

int enqueue_interp(nyx_amr *A, const double *cf, double *ff, int ncomp, int region) {
  nyx_plan &C = *A->C, &F = *A->F;
  const InterpRect *r = region == NYX_AMR_ALL ? A->d_ia : A->d_ig;
  const int n = region == NYX_AMR_ALL ? A->n_ia : A->n_ig;
  if (!n) return NYX_OK;
  k_amr_interp<<<grid_of(n), 256, 0, C.stream>>>(cf, ff, ncomp, C.d_boxes, F.d_boxes, r, n);
  C.launches += 1;
  return NYX_OK;
}

int enqueue_avgdown(nyx_amr *A, const double *ff, double *cf, int ncomp) {
  nyx_plan &C = *A->C, &F = *A->F;
  if (!A->n_avg) return NYX_OK;
  k_amr_avgdown<<<grid_of(A->n_avg), 256, 0, C.stream>>>(ff, cf, ncomp, C.d_boxes, F.d_boxes,
                                                         A->d_avg, A->n_avg);
  C.launches += 1;
  return NYX_OK;
}

int enqueue_estdt(nyx_amr *A, const double *cstate, const double *fstate, const double *a_dev,
                  double *dt_dev) {
  nyx_plan &C = *A->C, &F = *A->F;
  plan_estdt_accumulate(&C, cstate, a_dev, C.d_dtacc);
  plan_estdt_accumulate(&F, fstate, a_dev, C.d_dtacc);
  launch_dt_finalize(C.d_K, C.d_dtacc, dt_dev, C.stream);
  C.launches += 1;
  return NYX_OK;
}

int enqueue_step(nyx_amr *A, nyx_level *Lc, nyx_level *Lf, const double *a_old,
                 const double *a_new, const double *dt, double *dt_next) {
  int rc = plan_advance(A->C, Lc, a_old, a_new, dt, nullptr, nullptr);
  if (rc) return rc;
  // the coarse state at t^n (its ghosts filled by that advance) -> fine ghosts
  if ((rc = enqueue_interp(A, Lc->state[1 - Lc->cur], Lf->state[Lf->cur], NCONS, NYX_AMR_GHOSTS)))
    return rc;
  if ((rc = plan_advance(A->F, Lf, a_old, a_new, dt, nullptr, nullptr))) return rc;
  if ((rc = enqueue_reflux(A, Lc->state[Lc->cur]))) return rc;
  if ((rc = enqueue_avgdown(A, Lf->state[Lf->cur], Lc->state[Lc->cur], NCONS))) return rc;
  if (dt_next) return enqueue_estdt(A, Lc->state[Lc->cur], Lf->state[Lf->cur], a_new, dt_next);
  return NYX_OK;
}

int check_level(const nyx_level *L) {
  if (!L || (L->cur != 0 && L->cur != 1) || !L->state[0] || !L->state[1] ||
      L->state[0] == L->state[1])
    return fail(NYX_EINVAL, "level needs two distinct state buffers and cur in {0,1}");
  return NYX_OK;
}

int last_cuda(const char *what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NYX_OK : cuda_fail(e, what);
}

}  // namespace

extern "C" {

int nyx_amr_create(nyx_plan *coarse, nyx_plan *fine, nyx_amr **out) {
  if (!coarse || !fine || !out) return fail(NYX_EINVAL, "null argument");
  *out = nullptr;
  int rc = check_pair(*coarse, *fine);
  if (rc) return rc;
  nyx_amr *A = new nyx_amr;
  A->C = coarse;
  A->F = fine;
  if ((rc = build_tables(A))) {
    free_amr(A);
    return rc;
  }
  *out = A;
  return NYX_OK;
}

int nyx_amr_interp(nyx_amr *A, const double *coarse_field, double *fine_field, int ncomp,
                   int region) {
  if (!A || !coarse_field || !fine_field || ncomp < 1) return fail(NYX_EINVAL, "bad argument");
  if (region != NYX_AMR_GHOSTS && region != NYX_AMR_ALL) return fail(NYX_EINVAL, "bad region");
  int rc = enqueue_interp(A, coarse_field, fine_field, ncomp, region);
  return rc ? rc : last_cuda("amr interpolation launch");
}

int nyx_amr_reflux(nyx_amr *A, double *coarse_new) {
  if (!A || !coarse_new) return fail(NYX_EINVAL, "null argument");
  if (!A->C->flux_valid || !A->F->flux_valid)
    return fail(NYX_EINVAL, "both plans need an advance (with kept fluxes) before a reflux");
  int rc = enqueue_reflux(A, coarse_new);
  return rc ? rc : last_cuda("reflux launch");
}

int nyx_amr_average_down(nyx_amr *A, const double *fine_field, double *coarse_field, int ncomp) {
  if (!A || !fine_field || !coarse_field || ncomp < 1) return fail(NYX_EINVAL, "bad argument");
  int rc = enqueue_avgdown(A, fine_field, coarse_field, ncomp);
  return rc ? rc : last_cuda("average-down launch");
}

int nyx_amr_estdt(nyx_amr *A, const nyx_level *Lc, const nyx_level *Lf, const double *a_dev,
                  double *dt_dev) {
  if (!A || !a_dev || !dt_dev) return fail(NYX_EINVAL, "null argument");
  int rc = check_level(Lc);
  if (!rc) rc = check_level(Lf);
  if (rc) return rc;
  rc = enqueue_estdt(A, Lc->state[Lc->cur], Lf->state[Lf->cur], a_dev, dt_dev);
  return rc ? rc : last_cuda("amr estdt launch");
}

int nyx_amr_step(nyx_amr *A, nyx_level *Lc, nyx_level *Lf, const double *a_old_dev,
                 const double *a_new_dev, const double *dt_dev, double *dt_next_dev) {
  if (!A || !a_old_dev || !a_new_dev || !dt_dev) return fail(NYX_EINVAL, "null argument");
  int rc = check_level(Lc);
  if (!rc) rc = check_level(Lf);
  if (rc) return rc;
  rc = enqueue_step(A, Lc, Lf, a_old_dev, a_new_dev, dt_dev, dt_next_dev);
  return rc ? rc : last_cuda("amr step launch");
}

int nyx_amr_run(nyx_amr *A, nyx_level *Lc, nyx_level *Lf, const double *a_dev, double *dt_dev,
                int nsteps, int compute_dt0, int use_graph) {
  if (!A || !a_dev || !dt_dev || nsteps < 0) return fail(NYX_EINVAL, "null argument");
  int rc = check_level(Lc);
  if (!rc) rc = check_level(Lf);
  if (rc) return rc;
  auto run = [&](nyx_level *c, nyx_level *f) -> int {
    if (compute_dt0) {
      int r = enqueue_estdt(A, c->state[c->cur], f->state[f->cur], a_dev, dt_dev);
      if (r) return r;
    }
    for (int s = 0; s < nsteps; ++s) {
      int r = enqueue_step(A, c, f, a_dev + s, a_dev + s + 1, dt_dev + s, dt_dev + s + 1);
      if (r) return r;
    }
    return NYX_OK;
  };
  if (!use_graph) {
    rc = run(Lc, Lf);
    return rc ? rc : last_cuda("amr run launch");
  }
  nyx_plan &C = *A->C, &F = *A->F;
  const bool tune_c = C.prm.batching == NYX_PERSISTENT && C.prm.autotune && !C.tuned;
  const bool tune_f = F.prm.batching == NYX_PERSISTENT && F.prm.autotune && !F.tuned;
  if (tune_c || tune_f) {
    // time the tile shapes outside the capture, on the first step's data
    // (the tuning launches write only state[1-cur] of each level)
    if (compute_dt0 && (rc = enqueue_estdt(A, Lc->state[Lc->cur], Lf->state[Lf->cur], a_dev, dt_dev)))
      return rc;
    if ((rc = plan_tune(&C, Lc, a_dev, dt_dev))) return rc;
    plan_fill(&C, Lc->state[Lc->cur], NCONS);
    if ((rc = enqueue_interp(A, Lc->state[Lc->cur], Lf->state[Lf->cur], NCONS, NYX_AMR_GHOSTS)))
      return rc;
    if ((rc = plan_tune(&F, Lf, a_dev, dt_dev))) return rc;
  }
  AmrKey key(Lc->state[0], Lc->state[1], Lf->state[0], Lf->state[1], Lc->grav, Lf->grav,
             Lc->cur * 2 + Lf->cur, a_dev, dt_dev, nsteps, compute_dt0);
  auto it = A->graphs.find(key);
  if (it == A->graphs.end()) {
    nyx_level tc = *Lc, tf = *Lf;
    const long long before_c = C.launches, before_f = F.launches;
    CK(cudaStreamBeginCapture(C.stream, cudaStreamCaptureModeThreadLocal));
    rc = run(&tc, &tf);
    const long long in_graph = (C.launches - before_c) + (F.launches - before_f);
    C.launches = before_c;
    F.launches = before_f;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(C.stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "amr graph capture");
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "amr graph instantiate");
    it = A->graphs.emplace(key, std::make_pair(ge, in_graph)).first;
  }
  CK(cudaGraphLaunch(it->second.first, C.stream));
  C.launches += it->second.second;
  Lc->cur = (Lc->cur + nsteps) & 1;
  Lf->cur = (Lf->cur + nsteps) & 1;
  C.flux_valid = C.d_flux != nullptr;
  F.flux_valid = F.d_flux != nullptr;
  return NYX_OK;
}

int nyx_amr_destroy(nyx_amr *A) {
  free_amr(A);
  return NYX_OK;
}

}  // extern "C"
