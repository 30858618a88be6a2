// nyx_staged.cu -- the plain FP64 per-box form of the advance: one kernel per
// stage (primitives, PPM + tracing, normal solves, corner-coupling
// corrections, intermediate solves, final states, final solves, update),
// one thread per cell or face, intermediates in global FP64 arrays.  Built
// with --fmad=false: every value is the correctly rounded result of the
// expression forms in nyx_scheme.cuh.  Also holds the FP64 step-scalar
// set-up, the CFL reduction and its finalisation.
#define NYX_NS nyx_f64
#include "nyx_scheme.cuh"
#include "nyx_internal.cuh"
#include "nyx_finish.cuh"
#include "nyx_kernels.h"

namespace nyx {
using nyx_f64::Eos;
using nyx_f64::TraceSrc;
using nyx_f64::TFlux;

namespace {

__device__ __forceinline__ Eos<double> eos64(const SchemeConsts &k) {
  Eos<double> e;
  e.gamma = k.gamma;
  e.gm1 = k.gm1;
  e.igm1 = k.igm1;
  e.kshock = k.kshock;
  e.small_dens = k.small_dens;
  e.small_pres = k.small_pres;
  e.tol = k.tol;
  e.max_iter = k.max_iter;
  e.plm = k.plm;
  e.linear = k.linear_rs;
  e.flat = k.flat;
  return e;
}

struct Range {
  int lo[3], ext[3];
  long long count;
};

Range make_range(const int lo[3], const int hi[3]) {
  Range r;
  r.count = 1;
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = lo[d];
    r.ext[d] = hi[d] - lo[d] + 1;
    if (r.ext[d] < 0) r.ext[d] = 0;
    r.count *= r.ext[d];
  }
  return r;
}

__device__ __forceinline__ void range_ijk(const Range &r, long long t, int &i, int &j, int &k) {
  i = r.lo[0] + (int)(t % r.ext[0]);
  long long u = t / r.ext[0];
  j = r.lo[1] + (int)(u % r.ext[1]);
  k = r.lo[2] + (int)(u / r.ext[1]);
}

#define RANGE_FOR(r)                                                                       \
  for (long long t_ = blockIdx.x * (long long)blockDim.x + threadIdx.x; t_ < (r).count;  \
       t_ += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ long long stride_of(const BoxDev &b, int d) {
  return d == 0 ? 1LL : (d == 1 ? (long long)b.N[0] : (long long)b.N[0] * b.N[1]);
}

// ------------------------------------------------------------ O1 primitives
__global__ void k_prims(BoxDev b, const SchemeConsts *K, const double *S, double *q, long long V,
                        Range r) {
  const SchemeConsts k = *K;
  RANGE_FOR(r) {
    int i, j, kk;
    range_ijk(r, t_, i, j, kk);
    long long id = cell_index(b, i, j, kk);
    double rho = S[id];
    double p = k.gm1 * S[5 * b.stride + id];
    if (p < k.small_pres) p = k.small_pres;
    q[id] = rho;
    q[V + id] = S[b.stride + id] / rho;
    q[2 * V + id] = S[2 * b.stride + id] / rho;
    q[3 * V + id] = S[3 * b.stride + id] / rho;
    q[4 * V + id] = p;
    q[5 * V + id] = sqrt(k.gamma * p / rho);
  }
}

// ------------------------------------------------------------ O2+O3 PPM and tracing
template <int DIR>
__global__ void k_trace(BoxDev b, const SchemeConsts *K, const StepConsts *SC, const BoxStep *BS,
                        const double *q, const double *G, const double *FL, double *qm,
                        double *qp, long long V, Range r) {
  const Eos<double> E = eos64(*K);
  TraceSrc<double> src;
  src.hdtp = SC->hdtp;
  src.src_u = SC->src_u;
  src.src_p = SC->src_p;
  const double dtdx = BS->dtdx[DIR];
  const long long s = stride_of(b, DIR);
  RANGE_FOR(r) {
    int i, j, kk;
    range_ijk(r, t_, i, j, kk);
    long long id = cell_index(b, i, j, kk);
    double sv[5][5];
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int o = 0; o < 5; ++o) sv[v][o] = q[v * V + id + (o - 2) * s];
    double g3[3] = {0.0, 0.0, 0.0};
    if (G) {
      g3[0] = G[id];
      g3[1] = G[b.stride + id];
      g3[2] = G[2 * b.stride + id];
    }
    double a5[5], b5[5];
    const double fl = FL ? FL[id] : 1.0;
    nyx_f64::trace_cell<double, DIR>(E, sv, q[5 * V + id], g3, dtdx, src, fl, a5, b5);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      qm[v * V + id] = a5[v];
      qp[v * V + id] = b5[v];
    }
  }
}

// ------------------------------------------------------------ Riemann solves on DIR faces
// face f-1/2 stored at cell f; left state = high-face state of cell f-1.
template <int DIR>
__global__ void k_riemann(BoxDev b, const SchemeConsts *K, const double *qhi, const double *qlo,
                          double *F, long long V, Range r) {
  const Eos<double> E = eos64(*K);
  const long long s = stride_of(b, DIR);
  RANGE_FOR(r) {
    int i, j, kk;
    range_ijk(r, t_, i, j, kk);
    long long id = cell_index(b, i, j, kk);
    double ql[5], qr[5], f8[8];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      ql[v] = qhi[v * V + id - s];
      qr[v] = qlo[v * V + id];
    }
    nyx_f64::face_flux<double, DIR>(E, ql, qr, f8);
#pragma unroll
    for (int c = 0; c < 8; ++c) F[c * V + id] = f8[c];
  }
}

__device__ __forceinline__ TFlux<double> load_tflux(const double *F, long long V, long long id) {
  TFlux<double> t;
  t.f[0] = F[id];
  t.f[1] = F[V + id];
  t.f[2] = F[2 * V + id];
  t.f[3] = F[3 * V + id];
  t.f[4] = F[5 * V + id];
  t.f[5] = F[6 * V + id];
  t.f[6] = F[7 * V + id];
  return t;
}

// ------------------------------------------------------------ q_{D|T}, theta = 1/3
template <int D, int T>
__global__ void k_trans(BoxDev b, const SchemeConsts *K, const BoxStep *BS, const double *qm,
                        const double *qp, const double *Fn, double *tm, double *tp, long long V,
                        Range r) {
  const Eos<double> E = eos64(*K);
  const double cdt = BS->cdt3[T];
  const long long st = stride_of(b, T);
  RANGE_FOR(r) {
    int i, j, kk;
    range_ijk(r, t_, i, j, kk);
    long long id = cell_index(b, i, j, kk);
    TFlux<double> fm = load_tflux(Fn, V, id), fp = load_tflux(Fn, V, id + st);
    double a5[5], b5[5], o5[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a5[v] = qm[v * V + id];
      b5[v] = qp[v * V + id];
    }
    nyx_f64::transverse1(E, a5, cdt, fp, fm, o5);
#pragma unroll
    for (int v = 0; v < 5; ++v) tm[v * V + id] = o5[v];
    nyx_f64::transverse1(E, b5, cdt, fp, fm, o5);
#pragma unroll
    for (int v = 0; v < 5; ++v) tp[v * V + id] = o5[v];
  }
}

// ------------------------------------------------------------ final states, theta = 1/2
template <int D>
__global__ void k_final(BoxDev b, const SchemeConsts *K, const BoxStep *BS, const double *qm,
                        const double *qp, const double *A, const double *B, double *fm5,
                        double *fp5, long long V, Range r) {
  constexpr int T1 = nyx_f64::Tan<D>::t1, T2 = nyx_f64::Tan<D>::t2;
  const Eos<double> E = eos64(*K);
  const double c1 = BS->chalf[T1], c2 = BS->chalf[T2];
  const long long s1 = stride_of(b, T1), s2 = stride_of(b, T2);
  RANGE_FOR(r) {
    int i, j, kk;
    range_ijk(r, t_, i, j, kk);
    long long id = cell_index(b, i, j, kk);
    TFlux<double> am = load_tflux(A, V, id), ap = load_tflux(A, V, id + s1);
    TFlux<double> bm = load_tflux(B, V, id), bp = load_tflux(B, V, id + s2);
    double a5[5], b5[5], o5[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a5[v] = qm[v * V + id];
      b5[v] = qp[v * V + id];
    }
    nyx_f64::transverse2(E, a5, c1, ap, am, c2, bp, bm, o5);
#pragma unroll
    for (int v = 0; v < 5; ++v) fm5[v * V + id] = o5[v];
    nyx_f64::transverse2(E, b5, c1, ap, am, c2, bp, bm, o5);
#pragma unroll
    for (int v = 0; v < 5; ++v) fp5[v * V + id] = o5[v];
  }
}

// ------------------------------------------------------------ O6-O9 update
__global__ void k_update(BoxDev b, const SchemeConsts *K, const StepConsts *SC, const double *S,
                         const double *G, const double *F0, const double *F1, const double *F2,
                         double *Sn, long long V, Range r, unsigned long long *dtacc,
                         unsigned *status, double *flux_keep, int predict_only) {
  const SchemeConsts k = *K;
  const StepConsts sc = *SC;
  const long long s0 = 1, s1 = b.N[0], s2 = (long long)b.N[0] * b.N[1];
  const long long bs = b.stride;
  double local_min = __longlong_as_double(0x7ff0000000000000LL);
  unsigned flags = 0;
  RANGE_FOR(r) {
    int i, j, kk;
    range_ijk(r, t_, i, j, kk);
    long long id = cell_index(b, i, j, kk);
    double div[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double acc = (F0[c * V + id + s0] - F0[c * V + id]) * b.idx[0];
      acc = acc + (F1[c * V + id + s1] - F1[c * V + id]) * b.idx[1];
      acc = acc + (F2[c * V + id + s2] - F2[c * V + id]) * b.idx[2];
      div[c] = acc;
    }
    double pdivu = 0.5 * (F0[7 * V + id + s0] + F0[7 * V + id]) *
                   (F0[6 * V + id + s0] - F0[6 * V + id]) * b.idx[0];
    pdivu = pdivu + 0.5 * (F1[7 * V + id + s1] + F1[7 * V + id]) *
                        (F1[6 * V + id + s1] - F1[6 * V + id]) * b.idx[1];
    pdivu = pdivu + 0.5 * (F2[7 * V + id + s2] + F2[7 * V + id]) *
                        (F2[6 * V + id + s2] - F2[6 * V + id]) * b.idx[2];
    const double rho = S[id];
    const double m0 = S[bs + id], m1 = S[2 * bs + id], m2 = S[3 * bs + id];
    const double rE = S[4 * bs + id], re = S[5 * bs + id];
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (G) {
      g0 = G[id];
      g1 = G[bs + id];
      g2 = G[2 * bs + id];
    }
    // predictor (Step 2): U* = U^n - dt div F + dt S_e + dt S_g^n, comoving weights
    const double rho_s = rho - sc.dtp * div[0];
    const double ms0 = (sc.a_old * m0 - sc.dt * div[1] + sc.dt * rho * g0) * sc.ian;
    const double ms1 = (sc.a_old * m1 - sc.dt * div[2] + sc.dt * rho * g1) * sc.ian;
    const double ms2 = (sc.a_old * m2 - sc.dt * div[3] + sc.dt * rho * g2) * sc.ian;
    const double rE_s = predictor_energy(k, sc, rE, re, div[4], m0, m1, m2, g0, g1, g2, div[1],
                                         div[2], div[3], rho_s, ms0, ms1, ms2);
    const double re_s =
        (sc.ao2 * re - sc.ahdt * div[5] - sc.ahdt * pdivu + sc.expn * re) * sc.ian2;
    // corrector (Step 6): + dt/2 (S_g^{n+1,*} - S_g^n), then the dual-energy sync
    double o6[6];
    finish_cell(k, sc, rho, m0, m1, m2, g0, g1, g2, g0, g1, g2, rho_s, ms0, ms1, ms2, rE_s, re_s,
                k.grav_corrector && !predict_only, !predict_only, o6);
    const double mn0 = o6[1], mn1 = o6[2], mn2 = o6[3], rEn = o6[4], ren = o6[5];
    if (!(rho_s > 0.0)) flags |= ST_NEGATIVE;
    if (!isfinite(rho_s) || !isfinite(rEn) || !isfinite(ren) || !isfinite(mn0) ||
        !isfinite(mn1) || !isfinite(mn2))
      flags |= ST_NONFINITE;
    Sn[id] = rho_s;
    Sn[bs + id] = mn0;
    Sn[2 * bs + id] = mn1;
    Sn[3 * bs + id] = mn2;
    Sn[4 * bs + id] = rEn;
    Sn[5 * bs + id] = ren;
    // CFL step of the new state at a_new (Sec. 3.5)
    if (dtacc && !predict_only) {
      double p = k.gm1 * ren;
      if (p < k.small_pres) p = k.small_pres;
      const double c = sqrt(k.gamma * p / rho_s);
      double t0 = sc.a_new * b.dx[0] / (fabs(mn0 / rho_s) + c);
      double t1 = sc.a_new * b.dx[1] / (fabs(mn1 / rho_s) + c);
      double t2 = sc.a_new * b.dx[2] / (fabs(mn2 / rho_s) + c);
      if (t0 < local_min) local_min = t0;
      if (t1 < local_min) local_min = t1;
      if (t2 < local_min) local_min = t2;
    }
  }
  if (dtacc) {
    for (int o = 16; o > 0; o >>= 1) {
      double v = __shfl_xor_sync(0xffffffffu, local_min, o);
      if (v < local_min) local_min = v;
    }
    if ((threadIdx.x & 31) == 0) atomic_min_pos(dtacc, local_min);
  }
  if (flags) atomicOr(status, flags);
}

// ------------------------------------------------------------ Step 6 alone
// The corrector with g^n and g^{n+1} and the dual-energy sync over every
// valid cell of the level, in place on the predictor; one thread per cell,
// cells of a box in x-fastest order (coalesced), the box found by a binary
// search of the cell offsets.  CFL minimum of the result as in k_update (in
// FP32 for mixed plans, as their CFL reduction is: FP64 division and square
// root run at a small fraction of the FP32 rate on this part).
template <bool F32DT>
__global__ void k_correct(const BoxDev *boxes, const long long *cell_pref, int nbox,
                          long long total, const SchemeConsts *K, const StepConsts *SC,
                          const double *S, double *Sp, const double *Go, const double *Gn,
                          unsigned long long *dtacc, unsigned *status) {
  const SchemeConsts k = *K;
  const StepConsts sc = *SC;
  double local_min = __longlong_as_double(0x7ff0000000000000LL);
  unsigned flags = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cell_pref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const BoxDev b = boxes[lo];
    const long long f = t - cell_pref[lo];
    const int i = (int)(f % b.n[0]);
    const long long u = f / b.n[0];
    const int j = (int)(u % b.n[1]);
    const int kk = (int)(u / b.n[1]);
    const long long bs = b.stride;
    const long long id = NCONS * b.pref + cell_index(b, i, j, kk);
    const long long ig = NGRAV * b.pref + cell_index(b, i, j, kk);
    double go0 = 0.0, go1 = 0.0, go2 = 0.0, gn0 = 0.0, gn1 = 0.0, gn2 = 0.0;
    if (Go) {
      go0 = Go[ig];
      go1 = Go[bs + ig];
      go2 = Go[2 * bs + ig];
    }
    if (Gn) {
      gn0 = Gn[ig];
      gn1 = Gn[bs + ig];
      gn2 = Gn[2 * bs + ig];
    }
    double o6[6];
    finish_cell(k, sc, S[id], S[bs + id], S[2 * bs + id], S[3 * bs + id], go0, go1, go2, gn0, gn1,
                gn2, Sp[id], Sp[bs + id], Sp[2 * bs + id], Sp[3 * bs + id], Sp[4 * bs + id],
                Sp[5 * bs + id], true, true, o6);
    const double rho_s = o6[0];
    if (!(rho_s > 0.0)) flags |= ST_NEGATIVE;
    if (!isfinite(rho_s) || !isfinite(o6[4]) || !isfinite(o6[5]) || !isfinite(o6[1]) ||
        !isfinite(o6[2]) || !isfinite(o6[3]))
      flags |= ST_NONFINITE;
#pragma unroll
    for (int c = 1; c < 6; ++c) Sp[c * bs + id] = o6[c];
    if (dtacc) {
      if constexpr (F32DT) {
        const float r = (float)rho_s, ir = 1.0f / r;
        float p = (float)k.gm1 * (float)o6[5];
        if (p < (float)k.small_pres) p = (float)k.small_pres;
        const float c = sqrtf((float)k.gamma * p * ir);
        const float an = (float)sc.a_new;
        const float t0 = an * (float)b.dx[0] / (fabsf((float)o6[1] * ir) + c);
        const float t1 = an * (float)b.dx[1] / (fabsf((float)o6[2] * ir) + c);
        const float t2 = an * (float)b.dx[2] / (fabsf((float)o6[3] * ir) + c);
        const double tm = (double)fminf(t0, fminf(t1, t2));
        if (tm < local_min) local_min = tm;
      } else {
        double p = k.gm1 * o6[5];
        if (p < k.small_pres) p = k.small_pres;
        const double c = sqrt(k.gamma * p / rho_s);
        double t0 = sc.a_new * b.dx[0] / (fabs(o6[1] / rho_s) + c);
        double t1 = sc.a_new * b.dx[1] / (fabs(o6[2] / rho_s) + c);
        double t2 = sc.a_new * b.dx[2] / (fabs(o6[3] / rho_s) + c);
        if (t0 < local_min) local_min = t0;
        if (t1 < local_min) local_min = t1;
        if (t2 < local_min) local_min = t2;
      }
    }
  }
  if (dtacc) {
    for (int o = 16; o > 0; o >>= 1) {
      double v = __shfl_xor_sync(0xffffffffu, local_min, o);
      if (v < local_min) local_min = v;
    }
    if ((threadIdx.x & 31) == 0 && local_min < __longlong_as_double(0x7ff0000000000000LL))
      atomic_min_pos(dtacc, local_min);
  }
  if (flags) atomicOr(status, flags);
}

// copy the valid faces of the final fluxes of direction d into the flux store
__global__ void k_keep_flux(BoxDev b, const double *F, long long V, int d, double *out) {
  int e[3] = {b.n[0], b.n[1], b.n[2]};
  e[d] += 1;
  long long nf = (long long)e[0] * e[1] * e[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 6 * nf;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t / nf);
    long long f = t % nf;
    int i = (int)(f % e[0]);
    long long u = f / e[0];
    int j = (int)(u % e[1]);
    int kk = (int)(u / e[1]);
    out[t] = F[c * V + cell_index(b, i, j, kk)];
  }
}

// ------------------------------------------------------------ standalone CFL reduction
__global__ void k_estdt(const BoxDev *boxes, const long long *cell_pref, int nbox, long long total,
                        const double *state, const SchemeConsts *K, const double *a_dev,
                        unsigned long long *dtacc) {
  const SchemeConsts k = *K;
  const double a = *a_dev;
  double local_min = __longlong_as_double(0x7ff0000000000000LL);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (cell_pref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const BoxDev b = boxes[lo];
    long long f = t - cell_pref[lo];
    int i = (int)(f % b.n[0]);
    long long u = f / b.n[0];
    int j = (int)(u % b.n[1]);
    int kk = (int)(u / b.n[1]);
    const double *S = state + NCONS * b.pref;
    long long id = cell_index(b, i, j, kk);
    const double rho = S[id];
    double p = k.gm1 * S[5 * b.stride + id];
    if (p < k.small_pres) p = k.small_pres;
    const double c = sqrt(k.gamma * p / rho);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double tt = a * b.dx[d] / (fabs(S[(1 + d) * b.stride + id] / rho) + c);
      if (tt < local_min) local_min = tt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_xor_sync(0xffffffffu, local_min, o);
    if (v < local_min) local_min = v;
  }
  if ((threadIdx.x & 31) == 0) atomic_min_pos(dtacc, local_min);
}

__global__ void k_dt_finalize(const SchemeConsts *K, unsigned long long *dtacc, double *dt_out) {
  double m = __longlong_as_double((long long)*dtacc);
  if (dt_out) *dt_out = K->cfl * m;
  *dtacc = 0x7ff0000000000000ULL;
}

// ------------------------------------------------------------ step scalars
__global__ void k_step_setup(const SchemeConsts *K, const double *a_old_p, const double *a_new_p,
                             const double *dt_p, StepConsts *SC, const BoxDev *boxes, int nbox,
                             BoxStep *BS) {
  const double a_old = *a_old_p, a_new = *a_new_p, dt = *dt_p;
  const double gm1 = K->gm1;
  const double a_half = 0.5 * (a_old + a_new);
  const double dtp = dt / a_half;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    StepConsts s;
    s.a_old = a_old;
    s.a_new = a_new;
    s.dt = dt;
    s.a_half = a_half;
    s.dtp = dtp;
    s.adot = (a_new - a_old) / a_half;
    s.hdtp = 0.5 * dtp;
    s.src_u = 0.5 * s.adot;
    s.src_p = 1.5 * gm1 * s.adot;
    s.ao2 = a_old * a_old;
    s.an2 = a_new * a_new;
    s.ian = 1.0 / a_new;
    s.ian2 = 1.0 / s.an2;
    s.ahdt = a_half * dt;
    s.dta = dt * a_old;
    s.expn = a_half * (a_new - a_old) * K->kappa;
    s.hdt = 0.5 * dt;
    *SC = s;
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    BoxStep t;
    for (int d = 0; d < 3; ++d) {
      t.dtdx[d] = dtp / boxes[b].dx[d];
      t.cdt3[d] = dtp / (3.0 * boxes[b].dx[d]);
      t.chalf[d] = 0.5 * dtp / boxes[b].dx[d];
    }
    BS[b] = t;
  }
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ------------------------------------------------------------ host launchers
void launch_step_setup(const SchemeConsts *K, const double *a_old, const double *a_new,
                       const double *dt, StepConsts *SC, const BoxDev *boxes, int nbox,
                       BoxStep *BS, cudaStream_t st) {
  k_step_setup<<<grid_for(nbox, 128), 128, 0, st>>>(K, a_old, a_new, dt, SC, boxes, nbox, BS);
}

void launch_estdt(const BoxDev *boxes, const long long *cell_pref, int nbox, long long total,
                  const double *state, const SchemeConsts *K, const double *a_dev,
                  unsigned long long *dtacc, cudaStream_t st) {
  k_estdt<<<grid_for(total, 256), 256, 0, st>>>(boxes, cell_pref, nbox, total, state, K, a_dev,
                                                 dtacc);
}

void launch_correct(const BoxDev *boxes, const long long *cell_pref, int nbox, long long total,
                    const SchemeConsts *K, const StepConsts *SC, const double *S, double *Sp,
                    const double *Go, const double *Gn, unsigned long long *dtacc,
                    unsigned *status, bool f32_dt, cudaStream_t st) {
  if (total <= 0) return;
  if (f32_dt)
    k_correct<true><<<grid_for(total, 256), 256, 0, st>>>(boxes, cell_pref, nbox, total, K, SC, S,
                                                           Sp, Go, Gn, dtacc, status);
  else
    k_correct<false><<<grid_for(total, 256), 256, 0, st>>>(boxes, cell_pref, nbox, total, K, SC, S,
                                                            Sp, Go, Gn, dtacc, status);
}

void launch_dt_finalize(const SchemeConsts *K, unsigned long long *dtacc, double *dt_out,
                        cudaStream_t st) {
  k_dt_finalize<<<1, 1, 0, st>>>(K, dtacc, dt_out);
}

size_t staged_scratch_doubles(long long V) { return (size_t)222 * (size_t)V; }

// One box, all stages.  Sbox/Snbox/Gbox point at the box's blocks.
void launch_staged_box(const BoxDev &b, const BoxDev *b_dev, const SchemeConsts *K,
                       const StepConsts *SC, const BoxStep *BSb, const double *Sbox,
                       const double *Gbox, const double *FLbox, double *Snbox, double *scratch,
                       long long V, unsigned long long *dtacc, unsigned *status,
                       double *flux_keep, int predict_only, cudaStream_t st) {
  (void)b_dev;
  const int BLK = 256;
  double *q = scratch;
  double *qm[3], *qp[3], *Fn[3], *qtm[3][3], *qtp[3][3], *Ft[3][3], *qfm[3], *qfp[3], *Ff[3];
  double *p = scratch + 6 * V;
  for (int d = 0; d < 3; ++d) {
    qm[d] = p; p += 5 * V;
    qp[d] = p; p += 5 * V;
    Fn[d] = p; p += 8 * V;
    qfm[d] = p; p += 5 * V;
    qfp[d] = p; p += 5 * V;
    Ff[d] = p; p += 8 * V;
  }
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 3; ++t) {
      if (t == d) { qtm[d][t] = qtp[d][t] = Ft[d][t] = nullptr; continue; }
      qtm[d][t] = p; p += 5 * V;
      qtp[d][t] = p; p += 5 * V;
      Ft[d][t] = p; p += 8 * V;
    }
  int L[3], H[3];
  for (int d = 0; d < 3; ++d) {
    L[d] = -4;
    H[d] = b.n[d] + 3;
  }
  {
    Range r = make_range(L, H);
    k_prims<<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, Sbox, q, V, r);
  }
  // tracing
  {
    int lo[3] = {L[0] + 2, L[1], L[2]}, hi[3] = {H[0] - 2, H[1], H[2]};
    Range r = make_range(lo, hi);
    k_trace<0><<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, SC, BSb, q, Gbox, FLbox, qm[0],
                                                        qp[0], V, r);
  }
  {
    int lo[3] = {L[0], L[1] + 2, L[2]}, hi[3] = {H[0], H[1] - 2, H[2]};
    Range r = make_range(lo, hi);
    k_trace<1><<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, SC, BSb, q, Gbox, FLbox, qm[1],
                                                        qp[1], V, r);
  }
  {
    int lo[3] = {L[0], L[1], L[2] + 2}, hi[3] = {H[0], H[1], H[2] - 2};
    Range r = make_range(lo, hi);
    k_trace<2><<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, SC, BSb, q, Gbox, FLbox, qm[2],
                                                        qp[2], V, r);
  }
  // normal solves
#define NORMAL(D)                                                                                \
  {                                                                                              \
    int lo[3] = {L[0], L[1], L[2]}, hi[3] = {H[0], H[1], H[2]};                                  \
    lo[D] += 3;                                                                                  \
    hi[D] -= 2;                                                                                  \
    Range r = make_range(lo, hi);                                                                \
    k_riemann<D><<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, qp[D], qm[D], Fn[D], V, r);       \
  }
  NORMAL(0) NORMAL(1) NORMAL(2)
#undef NORMAL
  // corner coupling, theta = 1/3, and intermediate solves
#define TRANS(D, T)                                                                              \
  {                                                                                              \
    int lo[3] = {L[0], L[1], L[2]}, hi[3] = {H[0], H[1], H[2]};                                  \
    lo[D] += 2;                                                                                  \
    hi[D] -= 2;                                                                                  \
    lo[T] += 3;                                                                                  \
    hi[T] -= 3;                                                                                  \
    Range r = make_range(lo, hi);                                                                \
    k_trans<D, T><<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, BSb, qm[D], qp[D], Fn[T],        \
                                                          qtm[D][T], qtp[D][T], V, r);           \
    lo[D] += 1;                                                                                  \
    Range rf = make_range(lo, hi);                                                               \
    k_riemann<D><<<grid_for(rf.count, BLK), BLK, 0, st>>>(b, K, qtp[D][T], qtm[D][T], Ft[D][T],  \
                                                          V, rf);                                \
  }
  TRANS(0, 1) TRANS(0, 2) TRANS(1, 0) TRANS(1, 2) TRANS(2, 0) TRANS(2, 1)
#undef TRANS
  // final states (theta = 1/2) and final solves
#define FINAL(D, T1, T2)                                                                         \
  {                                                                                              \
    int lo[3] = {L[0], L[1], L[2]}, hi[3] = {H[0], H[1], H[2]};                                  \
    lo[D] += 2;                                                                                  \
    hi[D] -= 2;                                                                                  \
    lo[T1] += 3;                                                                                 \
    hi[T1] -= 3;                                                                                 \
    lo[T2] += 3;                                                                                 \
    hi[T2] -= 3;                                                                                 \
    Range r = make_range(lo, hi);                                                                \
    k_final<D><<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, BSb, qm[D], qp[D], Ft[T1][T2],      \
                                                       Ft[T2][T1], qfm[D], qfp[D], V, r);        \
    lo[D] += 1;                                                                                  \
    Range rf = make_range(lo, hi);                                                               \
    k_riemann<D><<<grid_for(rf.count, BLK), BLK, 0, st>>>(b, K, qfp[D], qfm[D], Ff[D], V, rf);   \
  }
  FINAL(0, 1, 2) FINAL(1, 0, 2) FINAL(2, 0, 1)
#undef FINAL
  {
    int lo[3] = {0, 0, 0}, hi[3] = {b.n[0] - 1, b.n[1] - 1, b.n[2] - 1};
    Range r = make_range(lo, hi);
    k_update<<<grid_for(r.count, BLK), BLK, 0, st>>>(b, K, SC, Sbox, Gbox, Ff[0], Ff[1], Ff[2],
                                                     Snbox, V, r, dtacc, status, flux_keep,
                                                     predict_only);
  }
  if (flux_keep) {
    double *o = flux_keep;
    for (int d = 0; d < 3; ++d) {
      long long nf = 6LL * (b.n[0] + (d == 0)) * (b.n[1] + (d == 1)) * (b.n[2] + (d == 2));
      k_keep_flux<<<grid_for(nf, BLK), BLK, 0, st>>>(b, Ff[d], V, d, o);
      o += nf;
    }
  }
}

}  // namespace nyx
