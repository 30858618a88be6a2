// nyx_poisson.cu -- self-gravity of one level (Sec. 3.4): the periodic
// 7-point Poisson equation L phi = 4 pi G / a (rho - mean rho) solved by
// geometric multigrid (V-cycles with red-black Gauss-Seidel relaxation,
// tolerance 1e-12 by default, warm start from the previous potential), then
// g = -grad phi by centred differences between adjacent cell centres.
//
// One GPU holds the whole level, so the solve runs on the dense periodic
// grid of its domain (gathered from the boxes): no ghost exchange between
// boxes at any multigrid level.  Transfer operators (reading): restriction
// = mean of the 8 fine residuals, prolongation = the coarse correction
// (piecewise constant).  Every sum runs in a fixed order (rows, planes,
// domain; the 8 children in index order) and the residual norm is a max,
// so the result does not depend on scheduling.  FP64 throughout by default;
// this unit is built without FMA contraction.  Mixed precision (on request):
// iterative refinement, each cycle an FP64 residual r = f - L phi, one FP32
// V-cycle of the same multigrid on L e = r from e = 0, and phi += e in FP64;
// the stopping test is the max norm of that residual (rounded to float).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "nyx_hydro.h"
#include "nyx_internal.cuh"
#include "nyx_kernels.h"
#include "nyx_plan.h"

using namespace nyx;
using namespace nyx::host;

namespace {

struct Dims {
  int n[3];
};

__device__ __forceinline__ long long didx(const Dims &d, int i, int j, int k) {
  return ((long long)k * d.n[1] + j) * d.n[0] + i;
}
__device__ __forceinline__ int wrp(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <class T>
__device__ __forceinline__ T nbsum(const T *u, const Dims &d, int i, int j, int k) {
  T s = u[didx(d, wrp(i - 1, d.n[0]), j, k)];
  s = s + u[didx(d, wrp(i + 1, d.n[0]), j, k)];
  s = s + u[didx(d, i, wrp(j - 1, d.n[1]), k)];
  s = s + u[didx(d, i, wrp(j + 1, d.n[1]), k)];
  s = s + u[didx(d, i, j, wrp(k - 1, d.n[2]))];
  s = s + u[didx(d, i, j, wrp(k + 1, d.n[2]))];
  return s;
}

template <class T>
__device__ __forceinline__ T resid_at(const T *phi, const T *f, const Dims &d, T ih2, int i, int j,
                                      int k) {
  const long long id = didx(d, i, j, k);
  return f[id] - (nbsum(phi, d, i, j, k) - T(6) * phi[id]) * ih2;
}

// valid cell t of the level (box by binary search of the cell offsets)
__device__ __forceinline__ void level_cell(const BoxDev *boxes, const long long *cell_pref,
                                           int nbox, long long t, int &b, int &i, int &j,
                                           int &k) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cell_pref[mid] <= t) lo = mid; else hi = mid - 1;
  }
  b = lo;
  const BoxDev &X = boxes[lo];
  const long long f = t - cell_pref[lo];
  i = (int)(f % X.n[0]);
  const long long u = f / X.n[0];
  j = (int)(u % X.n[1]);
  k = (int)(u / X.n[1]);
}

__global__ void k_pg_gather(const double *state, const BoxDev *boxes, const long long *cell_pref,
                            const int *box_lo, int nbox, long long total, Dims d, double *f) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int b, i, j, k;
    level_cell(boxes, cell_pref, nbox, t, b, i, j, k);
    const BoxDev X = boxes[b];
    f[didx(d, box_lo[3 * b] + i, box_lo[3 * b + 1] + j, box_lo[3 * b + 2] + k)] =
        state[NCONS * X.pref + cell_index(X, i, j, k)];
  }
}

__global__ void k_pg_add(double *f, const double *r, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    f[q] = f[q] + r[q];
}

// g = -grad phi on the dense grid (3 consecutive dense arrays)
__global__ void k_pg_grav_dense(const double *u, Dims d, double hdx, double *g) {
  const long long n = (long long)d.n[0] * d.n[1] * d.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % d.n[0]);
    const long long v = t / d.n[0];
    const int J = (int)(v % d.n[1]);
    const int K = (int)(v / d.n[1]);
    g[t] = -((u[didx(d, wrp(I + 1, d.n[0]), J, K)] - u[didx(d, wrp(I - 1, d.n[0]), J, K)]) * hdx);
    g[n + t] =
        -((u[didx(d, I, wrp(J + 1, d.n[1]), K)] - u[didx(d, I, wrp(J - 1, d.n[1]), K)]) * hdx);
    g[2 * n + t] =
        -((u[didx(d, I, J, wrp(K + 1, d.n[2]))] - u[didx(d, I, J, wrp(K - 1, d.n[2]))]) * hdx);
  }
}

// ---------------------------------------------------------------- dark matter
// Cloud in cell (Sec. 3.4): cell-centred coordinate s = x/dx - 1/2, the
// particle's cube overlaps cells floor(s) (weight 1 - frac(s)) and floor(s)+1.
// The particle kernels compare with the oracle within round-off (the deposit
// adds with atomics), so they multiply by host reciprocals instead of
// dividing and accumulate with fused multiply-adds: the FP64 pipe is their
// bound.
__device__ __forceinline__ void cic(double x, double idx, int n, int &i0, double &w0) {
  const double s = x * idx - 0.5;
  const double fl = floor(s);
  w0 = 1.0 - (s - fl);
  i0 = wrp((int)fl, n);
}

__device__ __forceinline__ void g_at(const double *g, const Dims &d, double idx, double x0,
                                     double x1, double x2, double (&out)[3]) {
  const long long N = (long long)d.n[0] * d.n[1] * d.n[2];
  int i0, j0, k0;
  double wx, wy, wz;
  cic(x0, idx, d.n[0], i0, wx);
  cic(x1, idx, d.n[1], j0, wy);
  cic(x2, idx, d.n[2], k0, wz);
  const int i1 = wrp(i0 + 1, d.n[0]), j1 = wrp(j0 + 1, d.n[1]), k1 = wrp(k0 + 1, d.n[2]);
  const double vx = 1.0 - wx, vy = 1.0 - wy, vz = 1.0 - wz;
  out[0] = out[1] = out[2] = 0.0;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int I = (o & 1) ? i1 : i0;
    const int J = ((o >> 1) & 1) ? j1 : j0;
    const int K = (o >> 2) ? k1 : k0;
    const double w = ((o & 1) ? vx : wx) * (((o >> 1) & 1) ? vy : wy) * ((o >> 2) ? vz : wz);
    const long long id = didx(d, I, J, K);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = fma(w, g[c * N + id], out[c]);
  }
}

__global__ void k_pm_deposit(const double *x, const double *m, long long np, Dims d, double idx,
                             double iv, double *rho) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int i0, j0, k0;
    double wx, wy, wz;
    cic(x[p], idx, d.n[0], i0, wx);
    cic(x[np + p], idx, d.n[1], j0, wy);
    cic(x[2 * np + p], idx, d.n[2], k0, wz);
    const int i1 = wrp(i0 + 1, d.n[0]), j1 = wrp(j0 + 1, d.n[1]), k1 = wrp(k0 + 1, d.n[2]);
    const double vx = 1.0 - wx, vy = 1.0 - wy, vz = 1.0 - wz;
    const double mp = m[p] * iv;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int I = (o & 1) ? i1 : i0;
      const int J = ((o >> 1) & 1) ? j1 : j0;
      const int K = (o >> 2) ? k1 : k0;
      const double w = ((o & 1) ? vx : wx) * (((o >> 1) & 1) ? vy : wy) * ((o >> 2) ? vz : wz);
      atomicAdd(&rho[didx(d, I, J, K)], mp * w);
    }
  }
}

// Step 3: kick by dt/2 with g^n, drift by dt at a^{n+1/2}, periodic wrap.
// ia_half = 1/a_half, dta = dt/a_half.
__global__ void k_pm_kick_drift(double *x, double *u, long long np, const double *g, Dims d,
                                double dx, double idx, double a_old, double ia_half, double hdt,
                                double dta) {
  const double L[3] = {d.n[0] * dx, d.n[1] * dx, d.n[2] * dx};
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double gp[3];
    const double xp[3] = {x[p], x[np + p], x[2 * np + p]};
    g_at(g, d, idx, xp[0], xp[1], xp[2], gp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double uh = fma(a_old, u[c * np + p], hdt * gp[c]) * ia_half;
      u[c * np + p] = uh;
      double xn = fma(dta, uh, xp[c]);
      if (xn < 0.0) xn = xn + L[c];
      if (xn >= L[c]) xn = xn - L[c];
      x[c * np + p] = xn;
    }
  }
}

// Step 5: kick by dt/2 with g^{n+1} (ia_new = 1/a_new).  With mx, also the
// maxima of |u_d| and |g_d| of the kicked particles (Sec. 3.5), for the
// particle time step of the next step: the same values k_pm_maxes forms.
__global__ void k_pm_kick(const double *x, double *u, long long np, const double *g, Dims d,
                          double idx, double a_half, double ia_new, double hdt,
                          unsigned long long *mx) {
  double um = 0.0, gm = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double gp[3];
    g_at(g, d, idx, x[p], x[np + p], x[2 * np + p], gp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double un = fma(a_half, u[c * np + p], hdt * gp[c]) * ia_new;
      u[c * np + p] = un;
      um = fmax(um, fabs(un));
      gm = fmax(gm, fabs(gp[c]));
    }
  }
  if (!mx) return;
  for (int o = 16; o > 0; o >>= 1) {
    um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
    gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&mx[0], (unsigned long long)__double_as_longlong(um));
    atomicMax(&mx[1], (unsigned long long)__double_as_longlong(gm));
  }
}

// Sec. 3.5: maxima of |u_d| and |g_d| at the particles (ordered bits)
__global__ void k_pm_maxes(const double *x, const double *u, long long np, const double *g,
                           Dims d, double idx, unsigned long long *mx) {
  double um = 0.0, gm = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double gp[3];
    g_at(g, d, idx, x[p], x[np + p], x[2 * np + p], gp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      um = fmax(um, fabs(u[c * np + p]));
      gm = fmax(gm, fabs(gp[c]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
    gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&mx[0], (unsigned long long)__double_as_longlong(um));
    atomicMax(&mx[1], (unsigned long long)__double_as_longlong(gm));
  }
}

__global__ void k_pm_dt(const unsigned long long *mx, double a, double dx, double cfl_dm,
                        double *dt_out) {
  const double um = __longlong_as_double((long long)mx[0]);
  const double gm = __longlong_as_double((long long)mx[1]);
  double dt = __longlong_as_double(0x7ff0000000000000LL);
  if (um > 0.0) dt = cfl_dm * (a * dx / um);
  if (gm > 0.0) {
    const double dg = sqrt(dx / gm);
    if (dg < dt) dt = dg;
  }
  *dt_out = dt;
}

// row sums (one thread per row, in index order), then plane sums, then the total
__global__ void k_pg_rows(const double *f, Dims d, double *rows) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= (long long)d.n[1] * d.n[2]) return;
  const double *p = f + r * d.n[0];
  double s = p[0];
  for (int i = 1; i < d.n[0]; ++i) s = s + p[i];
  rows[r] = s;
}
__global__ void k_pg_planes(const double *rows, Dims d, double *planes) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.n[2]) return;
  const double *p = rows + (long long)k * d.n[1];
  double s = p[0];
  for (int j = 1; j < d.n[1]; ++j) s = s + p[j];
  planes[k] = s;
}
__global__ void k_pg_mean(const double *planes, Dims d, double *mean) {
  double s = planes[0];
  for (int k = 1; k < d.n[2]; ++k) s = s + planes[k];
  *mean = s / ((double)d.n[0] * d.n[1] * d.n[2]);
}

__global__ void k_pg_rhs(double *f, long long n, const double *mean, double c,
                         unsigned long long *fmax_bits) {
  const double m = *mean;
  double loc = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double v = c * (f[q] - m);
    f[q] = v;
    loc = fmax(loc, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) loc = fmax(loc, __shfl_xor_sync(0xffffffffu, loc, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(fmax_bits, (unsigned long long)__double_as_longlong(loc));
}

// one colour of a red-black sweep: cells with (i + j + k) % 2 == color
// (launched on a grid3 of (n_x / 2, n_y, n_z): no index division)
template <class T>
__global__ void k_pg_sweep(T *phi, const T *f, Dims d, T h2, int color) {
  const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
  if (i2 >= d.n[0] / 2) return;
  const int j = blockIdx.y, k = blockIdx.z;
  const int i = 2 * i2 + ((j + k + color) & 1);
  const long long id = didx(d, i, j, k);
  phi[id] = (nbsum(phi, d, i, j, k) - h2 * f[id]) * (T(1) / T(6));
}

// (grid3 of (n_x, n_y, n_z))
__global__ void k_pg_resid_max(const double *phi, const double *f, Dims d, double ih2,
                               unsigned long long *out) {
  double loc = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.n[0]) loc = fabs(resid_at(phi, f, d, ih2, i, (int)blockIdx.y, (int)blockIdx.z));
  for (int o = 16; o > 0; o >>= 1) loc = fmax(loc, __shfl_xor_sync(0xffffffffu, loc, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(loc));
}

// coarse f = mean of the 8 fine residuals (index order), coarse phi = 0
// (grid3 of the coarse grid)
template <class T>
__global__ void k_pg_restrict(const T *phi, const T *f, Dims d, T ih2, T *fc, T *phic, Dims dc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < dc.n[0]) {
    const int j = blockIdx.y, k = blockIdx.z;
    const long long t = didx(dc, i, j, k);
    T s = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const T r =
          resid_at(phi, f, d, ih2, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + (o >> 2));
      s = (o == 0) ? r : s + r;
    }
    fc[t] = T(0.125) * s;
    phic[t] = T(0);
  }
}

// (grid3 of the fine grid)
template <class T>
__global__ void k_pg_prolong(T *phi, Dims d, const T *phic, Dims dc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n[0]) return;
  const int j = blockIdx.y, k = blockIdx.z;
  const long long t = didx(d, i, j, k);
  phi[t] = phi[t] + phic[didx(dc, i / 2, j / 2, k / 2)];
}

// double -> float on the integer pipe (the FP64 pipe, which also runs the
// F2F conversion, bounds the residual kernel): truncates the mantissa; below
// the float range gives 0, above it (or NaN) +-inf.  The right-hand side of
// the FP32 correction needs no correct rounding.
__device__ __forceinline__ float d2f_trunc(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// Mixed precision: the FP64 residual r = f - L phi of the finest grid as
// float (the right-hand side of the FP32 correction solve), the max norm of
// that float residual, and the correction's start e = 0.  The Laplacian is
// formed as f + 6 ih2 phi - ih2 (sum of the neighbours) with two fused
// multiply-adds: 7 FP64 operations per cell (c6 = 6 ih2).
// (grid3 of (n_x, n_y, n_z))
__global__ void k_pg_resid32(const double *phi, const double *f, Dims d, double ih2, double c6,
                             float *r, float *e, unsigned long long *out) {
  float loc = 0.0f;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.n[0]) {
    const int j = blockIdx.y, k = blockIdx.z;
    const long long t = didx(d, i, j, k);
    const double v = fma(-ih2, nbsum(phi, d, i, j, k), fma(c6, phi[t], f[t]));
    const float v32 = d2f_trunc(v);
    r[t] = v32;
    e[t] = 0.0f;
    loc = fabsf(v32);
  }
  for (int o = 16; o > 0; o >>= 1) loc = fmaxf(loc, __shfl_xor_sync(0xffffffffu, loc, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(out, (unsigned long long)__double_as_longlong((double)loc));
}

// phi += e (the FP32 correction), in FP64
__global__ void k_pg_correct(double *phi, const float *e, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    phi[t] = phi[t] + (double)e[t];
}

// g = -grad phi (centred) into the level's gravity field, valid cells
__global__ void k_pg_grav(const double *u, Dims d, double hdx, const BoxDev *boxes,
                          const long long *cell_pref, const int *box_lo, int nbox,
                          long long total, double *grav) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int b, i, j, k;
    level_cell(boxes, cell_pref, nbox, t, b, i, j, k);
    const BoxDev X = boxes[b];
    const int I = box_lo[3 * b] + i, J = box_lo[3 * b + 1] + j, K = box_lo[3 * b + 2] + k;
    double *G = grav + NGRAV * X.pref + cell_index(X, i, j, k);
    G[0] = -((u[didx(d, wrp(I + 1, d.n[0]), J, K)] - u[didx(d, wrp(I - 1, d.n[0]), J, K)]) * hdx);
    G[X.stride] =
        -((u[didx(d, I, wrp(J + 1, d.n[1]), K)] - u[didx(d, I, wrp(J - 1, d.n[1]), K)]) * hdx);
    G[2 * X.stride] =
        -((u[didx(d, I, J, wrp(K + 1, d.n[2]))] - u[didx(d, I, J, wrp(K - 1, d.n[2]))]) * hdx);
  }
}

int gridn(long long n, int block) {
  long long g = (n + block - 1) / block;
  return (int)std::max<long long>(1, std::min<long long>(g, 152 * 32));
}

// Launch shape covering an (nx, ny, nz) index box: x in blocks of up to 128
// threads, y and z one block row each (extents are at most 65535).
struct Grid3 {
  dim3 g, b;
};
Grid3 grid3(int nx, int ny, int nz) {
  Grid3 r;
  const int bx = std::min(128, (nx + 31) / 32 * 32);
  r.b = dim3(bx, 1, 1);
  r.g = dim3((nx + bx - 1) / bx, ny, nz);
  return r;
}

template <class T>
struct LevelT {
  Dims d;
  T h2, ih2;
  T *phi = nullptr, *f = nullptr;
};
using Level = LevelT<double>;

}  // namespace

struct nyx_poisson {
  nyx_plan *P = nullptr;
  nyx_poisson_params prm{};
  std::vector<Level> L;
  std::vector<LevelT<float>> L32;  // mixed precision: the FP32 correction grids
  int *d_box_lo = nullptr;       // box lo relative to the domain origin
  double *d_rows = nullptr, *d_planes = nullptr, *d_scal = nullptr;  // scal: mean
  unsigned long long *d_max = nullptr;
  double dx = 0.0;
  long long launches = 0;
};

namespace {

void free_poisson(nyx_poisson *S) {
  if (!S) return;
  for (auto &l : S->L) {
    if (l.phi) cudaFree(l.phi);
    if (l.f) cudaFree(l.f);
  }
  for (auto &l : S->L32) {
    if (l.phi) cudaFree(l.phi);
    if (l.f) cudaFree(l.f);
  }
  cudaFree(S->d_box_lo);
  cudaFree(S->d_rows);
  cudaFree(S->d_planes);
  cudaFree(S->d_scal);
  cudaFree(S->d_max);
  delete S;
}

int read_max(nyx_poisson *S, double *out) {
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, S->d_max, sizeof(v), cudaMemcpyDeviceToHost, S->P->stream));
  CK(cudaStreamSynchronize(S->P->stream));
  std::memcpy(out, &v, sizeof(double));
  return NYX_OK;
}

template <class T>
void sweep(nyx_poisson *S, LevelT<T> &l) {
  const Grid3 G = grid3(l.d.n[0] / 2, l.d.n[1], l.d.n[2]);
  for (int c = 0; c < 2; ++c)
    k_pg_sweep<T><<<G.g, G.b, 0, S->P->stream>>>(l.phi, l.f, l.d, l.h2, c);
  S->launches += 2;
}

template <class T>
void vcycle(nyx_poisson *S, std::vector<LevelT<T>> &L, size_t l) {
  LevelT<T> &g = L[l];
  if (l + 1 == L.size()) {
    for (int s = 0; s < S->prm.coarse_sweeps; ++s) sweep(S, g);
    return;
  }
  for (int s = 0; s < S->prm.pre; ++s) sweep(S, g);
  LevelT<T> &c = L[l + 1];
  const Grid3 Gc = grid3(c.d.n[0], c.d.n[1], c.d.n[2]);
  k_pg_restrict<T><<<Gc.g, Gc.b, 0, S->P->stream>>>(g.phi, g.f, g.d, g.ih2, c.f, c.phi, c.d);
  S->launches += 1;
  vcycle(S, L, l + 1);
  const Grid3 Gf = grid3(g.d.n[0], g.d.n[1], g.d.n[2]);
  k_pg_prolong<T><<<Gf.g, Gf.b, 0, S->P->stream>>>(g.phi, g.d, c.phi, c.d);
  S->launches += 1;
  for (int s = 0; s < S->prm.post; ++s) sweep(S, g);
}

int resid_max(nyx_poisson *S, double *out) {
  Level &g = S->L[0];
  CK(cudaMemsetAsync(S->d_max, 0, sizeof(unsigned long long), S->P->stream));
  const Grid3 G = grid3(g.d.n[0], g.d.n[1], g.d.n[2]);
  if (S->L32.empty()) {
    k_pg_resid_max<<<G.g, G.b, 0, S->P->stream>>>(g.phi, g.f, g.d, g.ih2, S->d_max);
  } else {  // also the FP32 right-hand side of the next correction, and e = 0
    LevelT<float> &g32 = S->L32[0];
    k_pg_resid32<<<G.g, G.b, 0, S->P->stream>>>(g.phi, g.f, g.d, g.ih2, 6.0 * g.ih2, g32.f,
                                                g32.phi, S->d_max);
  }
  S->launches += 1;
  return read_max(S, out);
}

// One cycle: a V-cycle on phi (FP64), or a refinement step (FP32 V-cycle on
// the correction equation whose right-hand side resid_max left, then phi +=
// e in FP64).
void cycle(nyx_poisson *S) {
  if (S->L32.empty()) {
    vcycle(S, S->L, 0);
    return;
  }
  vcycle(S, S->L32, 0);
  Level &g = S->L[0];
  const long long n = (long long)g.d.n[0] * g.d.n[1] * g.d.n[2];
  k_pg_correct<<<gridn(n, 256), 256, 0, S->P->stream>>>(g.phi, S->L32[0].phi, n);
  S->launches += 1;
}

}  // namespace

extern "C" {

void nyx_poisson_default_params(nyx_poisson_params *p) {
  if (!p) return;
  p->tol = 1e-12;
  p->max_cycles = 50;
  p->pre = 2;
  p->post = 2;
  p->coarse_sweeps = 40;
  p->min_size = 2;
  p->four_pi_G = 1.0;
  p->precision = NYX_FP64;
}

int nyx_poisson_create(nyx_plan *P, const nyx_poisson_params *prm, nyx_poisson **out) {
  if (!P || !prm || !out) return fail(NYX_EINVAL, "null argument");
  *out = nullptr;
  if (P->doms.size() != 1) return fail(NYX_EINVAL, "the Poisson solve needs a one-domain level");
  const nyx_domain &D = P->doms[0];
  int n[3];
  for (int a = 0; a < 3; ++a) {
    n[a] = D.hi[a] - D.lo[a] + 1;
    if (n[a] % 2) return fail(NYX_EINVAL, "the Poisson solve needs even domain extents");
    if (D.bc[a] != NYX_BC_PERIODIC || D.bc[3 + a] != NYX_BC_PERIODIC)
      return fail(NYX_EINVAL, "the Poisson solve needs a periodic domain");
  }
  const double dx = P->boxes[0].dx[0];
  for (const nyx_box &X : P->boxes)
    for (int a = 0; a < 3; ++a)
      if (X.dx[a] != dx) return fail(NYX_EINVAL, "the Poisson solve needs equal cubic cells");
  if (P->total_cells != (long long)n[0] * n[1] * n[2])
    return fail(NYX_EINVAL, "the level's boxes must tile its domain");
  if (prm->pre < 0 || prm->post < 0 || prm->coarse_sweeps < 1 || prm->max_cycles < 0 ||
      prm->min_size < 1 || !(prm->tol > 0.0) ||
      (prm->precision != NYX_FP64 && prm->precision != NYX_MIXED))
    return fail(NYX_EINVAL, "bad Poisson parameters");
  nyx_poisson *S = new nyx_poisson;
  S->P = P;
  S->prm = *prm;
  S->dx = dx;
  int m[3] = {n[0], n[1], n[2]};
  double h = dx;
  int rc = NYX_OK;
  for (;;) {
    Level l;
    for (int a = 0; a < 3; ++a) l.d.n[a] = m[a];
    l.h2 = h * h;
    l.ih2 = 1.0 / (h * h);
    const size_t v = (size_t)m[0] * m[1] * m[2];
    if (cudaMalloc(&l.phi, v * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&l.f, v * sizeof(double)) != cudaSuccess) {
      S->L.push_back(l);
      rc = fail(NYX_ENOMEM, "Poisson grid allocation failed");
      break;
    }
    cudaMemset(l.phi, 0, v * sizeof(double));
    S->L.push_back(l);
    if (prm->precision == NYX_MIXED) {
      LevelT<float> l32;
      l32.d = l.d;
      l32.h2 = (float)l.h2;
      l32.ih2 = (float)l.ih2;
      if (cudaMalloc(&l32.phi, v * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&l32.f, v * sizeof(float)) != cudaSuccess) {
        S->L32.push_back(l32);
        rc = fail(NYX_ENOMEM, "Poisson grid allocation failed");
        break;
      }
      S->L32.push_back(l32);
    }
    bool ok = S->L.size() < 32;
    for (int a = 0; a < 3; ++a)
      if (m[a] % 4 || m[a] < 2 * prm->min_size) ok = false;
    if (!ok) break;
    for (int a = 0; a < 3; ++a) m[a] /= 2;
    h *= 2.0;
  }
  if (!rc) {
    std::vector<int> lo(3 * P->nbox);
    for (int b = 0; b < P->nbox; ++b)
      for (int a = 0; a < 3; ++a) lo[3 * b + a] = P->boxes[b].lo[a] - D.lo[a];
    if (cudaMalloc(&S->d_box_lo, lo.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&S->d_rows, sizeof(double) * (size_t)n[1] * n[2]) != cudaSuccess ||
        cudaMalloc(&S->d_planes, sizeof(double) * n[2]) != cudaSuccess ||
        cudaMalloc(&S->d_scal, sizeof(double) * 2) != cudaSuccess ||
        cudaMalloc(&S->d_max, 2 * sizeof(unsigned long long)) != cudaSuccess)
      rc = fail(NYX_ENOMEM, "Poisson scratch allocation failed");
    else if (cudaMemcpy(S->d_box_lo, lo.data(), lo.size() * sizeof(int), cudaMemcpyHostToDevice) !=
             cudaSuccess)
      rc = fail(NYX_ECUDA, "Poisson table upload failed");
  }
  if (rc) {
    free_poisson(S);
    return rc;
  }
  *out = S;
  return NYX_OK;
}

int nyx_poisson_solve(nyx_poisson *S, const double *state, const double *rho_dm, double a,
                      double *grav_out, double *g_dense_out, int warm_start, int *cycles_out,
                      double *resid_out) {
  if (!S || !state || !(a > 0.0)) return fail(NYX_EINVAL, "bad argument");
  nyx_plan &P = *S->P;
  Level &g0 = S->L[0];
  const long long N = (long long)g0.d.n[0] * g0.d.n[1] * g0.d.n[2];
  cudaStream_t st = P.stream;
  if (!warm_start) CK(cudaMemsetAsync(g0.phi, 0, N * sizeof(double), st));
  k_pg_gather<<<gridn(P.total_cells, 256), 256, 0, st>>>(state, P.d_boxes, P.d_cell_pref,
                                                        S->d_box_lo, P.nbox, P.total_cells, g0.d,
                                                        g0.f);
  if (rho_dm) {
    k_pg_add<<<gridn(N, 256), 256, 0, st>>>(g0.f, rho_dm, N);
    S->launches += 1;
  }
  const long long nrow = (long long)g0.d.n[1] * g0.d.n[2];
  k_pg_rows<<<gridn(nrow, 128), 128, 0, st>>>(g0.f, g0.d, S->d_rows);
  k_pg_planes<<<gridn(g0.d.n[2], 128), 128, 0, st>>>(S->d_rows, g0.d, S->d_planes);
  k_pg_mean<<<1, 1, 0, st>>>(S->d_planes, g0.d, S->d_scal);
  CK(cudaMemsetAsync(S->d_max, 0, sizeof(unsigned long long), st));
  k_pg_rhs<<<gridn(N, 256), 256, 0, st>>>(g0.f, N, S->d_scal, S->prm.four_pi_G / a, S->d_max);
  S->launches += 5;
  double fmax = 0.0, res = 0.0;
  int rc = read_max(S, &fmax);
  if (rc) return rc;
  if ((rc = resid_max(S, &res))) return rc;
  const double target = S->prm.tol * fmax;
  int cyc = 0;
  while (res > target && cyc < S->prm.max_cycles) {
    cycle(S);
    ++cyc;
    if ((rc = resid_max(S, &res))) return rc;
  }
  if (grav_out) {
    k_pg_grav<<<gridn(P.total_cells, 256), 256, 0, st>>>(g0.phi, g0.d, 0.5 / S->dx, P.d_boxes,
                                                        P.d_cell_pref, S->d_box_lo, P.nbox,
                                                        P.total_cells, grav_out);
    S->launches += 1;
    plan_fill(&P, grav_out, NGRAV);
  }
  if (g_dense_out) {
    k_pg_grav_dense<<<gridn(N, 256), 256, 0, st>>>(g0.phi, g0.d, 0.5 / S->dx, g_dense_out);
    S->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "Poisson launch");
  P.launches += S->launches;
  S->launches = 0;
  if (cycles_out) *cycles_out = cyc;
  if (resid_out) *resid_out = fmax > 0.0 ? res / fmax : 0.0;
  if (res > target) return fail(NYX_ETIMEOUT, "Poisson solve did not reach the tolerance");
  return NYX_OK;
}

int nyx_pm_deposit(nyx_poisson *S, const double *x, const double *m, long long np,
                   double *rho_dm) {
  if (!S || !rho_dm || np < 0 || (np && (!x || !m))) return fail(NYX_EINVAL, "bad argument");
  Level &g0 = S->L[0];
  const long long N = (long long)g0.d.n[0] * g0.d.n[1] * g0.d.n[2];
  CK(cudaMemsetAsync(rho_dm, 0, N * sizeof(double), S->P->stream));
  if (np) {
    const double iv = 1.0 / (S->dx * S->dx * S->dx);
    k_pm_deposit<<<gridn(np, 256), 256, 0, S->P->stream>>>(x, m, np, g0.d, 1.0 / S->dx, iv,
                                                           rho_dm);
    S->P->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NYX_OK : cuda_fail(e, "deposit launch");
}

int nyx_pm_kick_drift(nyx_poisson *S, double *x, double *u, long long np, const double *g_dense,
                      double a_old, double a_half, double dt) {
  if (!S || !g_dense || np < 0 || (np && (!x || !u)) || !(a_half > 0.0))
    return fail(NYX_EINVAL, "bad argument");
  if (np) {
    k_pm_kick_drift<<<gridn(np, 256), 256, 0, S->P->stream>>>(
        x, u, np, g_dense, S->L[0].d, S->dx, 1.0 / S->dx, a_old, 1.0 / a_half, 0.5 * dt,
        dt / a_half);
    S->P->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NYX_OK : cuda_fail(e, "kick-drift launch");
}

static int pm_kick_impl(nyx_poisson *S, const double *x, double *u, long long np,
                        const double *g_dense, double a_half, double a_new, double dt,
                        unsigned long long *mx) {
  if (!S || !g_dense || np < 0 || (np && (!x || !u)) || !(a_new > 0.0))
    return fail(NYX_EINVAL, "bad argument");
  if (np) {
    k_pm_kick<<<gridn(np, 256), 256, 0, S->P->stream>>>(x, u, np, g_dense, S->L[0].d,
                                                        1.0 / S->dx, a_half, 1.0 / a_new,
                                                        0.5 * dt, mx);
    S->P->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NYX_OK : cuda_fail(e, "kick launch");
}

int nyx_pm_kick(nyx_poisson *S, const double *x, double *u, long long np, const double *g_dense,
                double a_half, double a_new, double dt) {
  return pm_kick_impl(S, x, u, np, g_dense, a_half, a_new, dt, nullptr);
}

int nyx_pm_kick_estdt(nyx_poisson *S, const double *x, double *u, long long np,
                      const double *g_dense, double a_half, double a_new, double dt,
                      double cfl_dm, double *dt_dev) {
  if (!S || !dt_dev) return fail(NYX_EINVAL, "bad argument");
  CK(cudaMemsetAsync(S->d_max, 0, 2 * sizeof(unsigned long long), S->P->stream));
  int rc = pm_kick_impl(S, x, u, np, g_dense, a_half, a_new, dt, S->d_max);
  if (rc) return rc;
  k_pm_dt<<<1, 1, 0, S->P->stream>>>(S->d_max, a_new, S->dx, cfl_dm, dt_dev);
  S->P->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NYX_OK : cuda_fail(e, "particle dt launch");
}

int nyx_pm_estdt(nyx_poisson *S, const double *x, const double *u, long long np,
                 const double *g_dense, double a, double cfl_dm, double *dt_dev) {
  if (!S || !g_dense || !dt_dev || np < 0 || (np && (!x || !u)))
    return fail(NYX_EINVAL, "bad argument");
  CK(cudaMemsetAsync(S->d_max, 0, 2 * sizeof(unsigned long long), S->P->stream));
  if (np)
    k_pm_maxes<<<gridn(np, 256), 256, 0, S->P->stream>>>(x, u, np, g_dense, S->L[0].d,
                                                         1.0 / S->dx, S->d_max);
  k_pm_dt<<<1, 1, 0, S->P->stream>>>(S->d_max, a, S->dx, cfl_dm, dt_dev);
  S->P->launches += np ? 2 : 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NYX_OK : cuda_fail(e, "particle dt launch");
}

int nyx_poisson_phi(nyx_poisson *S, double *phi_out) {
  if (!S || !phi_out) return fail(NYX_EINVAL, "null argument");
  Level &g0 = S->L[0];
  const size_t N = (size_t)g0.d.n[0] * g0.d.n[1] * g0.d.n[2];
  CK(cudaMemcpyAsync(phi_out, g0.phi, N * sizeof(double), cudaMemcpyDeviceToDevice, S->P->stream));
  return NYX_OK;
}

int nyx_poisson_destroy(nyx_poisson *S) {
  free_poisson(S);
  return NYX_OK;
}

}  // extern "C"
