// nyx_fused.cuh -- the fused, persistent single-level advance.
//
// One CTA takes a work item, a TX x TY column tile of one box, and streams
// it along z.  Its threads own the (TX+2) x (TY+2) columns of the tile plus
// a one-cell halo: the region where traced edge states are needed for the
// corner-coupled fluxes of the tile's faces.  Each thread keeps the z-history
// of its own column in registers (the 5-plane primitive window of the z-PPM
// stencil and the few upstream-plane states and fluxes the z-direction
// corner coupling needs); x/y neighbour data goes through shared memory,
// one plane at a time.  Per plane c (c = -1 .. nz) the stages are:
//
//   0 primitives of plane c+2 (own column) and of the x/y PPM halo of plane c
//   1 PPM + characteristic tracing at plane c in x, y, z
//   2 normal solves: x, y faces of plane c; z face c-1/2
//   3 corner-coupling corrections (theta = 1/3): in-plane ones at plane c,
//     z-flux ones at plane c-1
//   4 six intermediate solves (x|y, y|x at c; x|z, y|z at c-1; z|x, z|y at c-1/2)
//   5 final states (theta = 1/2): z at plane c, x and y at plane c-1
//   6 final solves: x, y faces of plane c-1; z face c-1/2
//   7 conservative comoving update of plane c-1 in FP64, gravity
//     predictor-corrector, dual-energy sync, CFL minimum
//
// The arithmetic is nyx_scheme.cuh's, in type R (double: FP64 path, float:
// mixed path); the state, the flux-divergence accumulation and the update
// are FP64 in both.  NYX_NS is defined by the including translation unit.
#pragma once
#include "nyx_internal.cuh"
#include "nyx_kernels.h"
#include "nyx_scheme.cuh"
#include "nyx_finish.cuh"

namespace NYX_NS {

template <class R, int TX, int TY>
struct FusedGeom {
  static constexpr int W = TX + 2, H = TY + 2, NC = W * H;  // owned columns
  static constexpr int WE = TX + 6, HE = TY + 6, NE = WE * HE;  // primitive plane
  static constexpr int NT = (NC + 31) / 32 * 32;
  static constexpr int NA = 20, NB = 28;  // shared planes in the two ping-pong buffers
  static constexpr size_t SMEM = sizeof(R) * (size_t)(5 * NE + (NA + NB) * NC);
};

template <class R>
__device__ __forceinline__ Eos<R> make_eos(const nyx::SchemeConsts &k, bool mixed) {
  Eos<R> e;
  e.gamma = (R)k.gamma;
  e.gm1 = (R)k.gm1;
  e.igm1 = (R)k.igm1;
  e.kshock = (R)k.kshock;
  e.small_dens = (R)k.small_dens;
  e.small_pres = (R)k.small_pres;
  e.tol = (R)(mixed ? k.tol_mixed : k.tol);
  e.max_iter = k.max_iter;
  e.plm = k.plm;
  e.linear = k.linear_rs;
  e.flat = k.flat;
  return e;
}

// double -> float, round to nearest even, flushing results below the
// smallest normal float to zero (the mixed unit runs with flush-to-zero),
// computed on the integer pipe: the FP64 pipe of this part is 1/64 of the
// FP32 rate and also executes the F2F conversion.
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);
  const int e = E - 896;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  unsigned bits = ((unsigned)e << 23) + m;
  bits += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  if (e <= 0) bits = 0u;
  if (e >= 255) bits = (E == 0x7ff && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
  return __uint_as_float(bits | sign);
}

template <class R>
__device__ __forceinline__ R to_r(double x) {
  if constexpr (sizeof(R) == 4)
    return d2f_rn(x);
  else
    return x;
}

// primitives (rho, u, v, w, p) of one cell of the state
template <class R>
__device__ __forceinline__ void prims_of(const double *S, long long bs, long long id, const Eos<R> &E,
                                         R (&q)[5]) {
  const R rho = to_r<R>(S[id]);
  q[0] = rho;
  if constexpr (sizeof(R) == 4) {
    const R ir = R(1) / rho;
    q[1] = to_r<R>(S[bs + id]) * ir;
    q[2] = to_r<R>(S[2 * bs + id]) * ir;
    q[3] = to_r<R>(S[3 * bs + id]) * ir;
  } else {
    q[1] = (R)S[bs + id] / rho;
    q[2] = (R)S[2 * bs + id] / rho;
    q[3] = (R)S[3 * bs + id] / rho;
  }
  R p = E.gm1 * to_r<R>(S[5 * bs + id]);
  if (p < E.small_pres) p = E.small_pres;
  q[4] = p;
}

template <class R>
__device__ __forceinline__ void put7(R *buf, int nc, int base, int cell, const TFlux<R> &t) {
#pragma unroll
  for (int k = 0; k < 7; ++k) buf[(base + k) * nc + cell] = t.f[k];
}
template <class R>
__device__ __forceinline__ TFlux<R> get7(const R *buf, int nc, int base, int cell) {
  TFlux<R> t;
#pragma unroll
  for (int k = 0; k < 7; ++k) t.f[k] = buf[(base + k) * nc + cell];
  return t;
}
template <class R>
__device__ __forceinline__ void put5(R *buf, int nc, int base, int cell, const R (&q)[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) buf[(base + k) * nc + cell] = q[k];
}
template <class R>
__device__ __forceinline__ void get5(const R *buf, int nc, int base, int cell, R (&q)[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) q[k] = buf[(base + k) * nc + cell];
}
template <class R>
__device__ __forceinline__ void copy5(R (&d)[5], const R (&s)[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) d[k] = s[k];
}
template <class R>
__device__ __forceinline__ void copy8(R (&d)[8], const R (&s)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) d[k] = s[k];
}

// FP64 conservative update of one cell (Step 2 predictor + Step 6 corrector
// and sync, Sec. 3.6), from the final fluxes on its six faces.  The flux
// differences are taken in FP64 (exact for FP32 inputs), so the divergence
// telescopes like the FP64 path.
template <class R>
__device__ __forceinline__ void update_cell(const nyx::SchemeConsts &k, const nyx::StepConsts &sc,
                                            const nyx::BoxDev &b, const double *S, const double *G,
                                            double *Sn, long long id, const R (&Fxm)[8],
                                            const R (&Fxp)[8], const R (&Fym)[8],
                                            const R (&Fyp)[8], const R (&Fzm)[8],
                                            const R (&Fzp)[8], double &dtmin, unsigned &flags,
                                            bool want_dt, bool full) {
  const long long bs = b.stride;
  double div[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double acc = ((double)Fxp[c] - (double)Fxm[c]) * b.idx[0];
    acc = acc + ((double)Fyp[c] - (double)Fym[c]) * b.idx[1];
    acc = acc + ((double)Fzp[c] - (double)Fzm[c]) * b.idx[2];
    div[c] = acc;
  }
  double pdivu = 0.5 * ((double)Fxp[7] + (double)Fxm[7]) * ((double)Fxp[6] - (double)Fxm[6]) * b.idx[0];
  pdivu = pdivu + 0.5 * ((double)Fyp[7] + (double)Fym[7]) * ((double)Fyp[6] - (double)Fym[6]) * b.idx[1];
  pdivu = pdivu + 0.5 * ((double)Fzp[7] + (double)Fzm[7]) * ((double)Fzp[6] - (double)Fzm[6]) * b.idx[2];
  const double rho = S[id];
  const double m0 = S[bs + id], m1 = S[2 * bs + id], m2 = S[3 * bs + id];
  const double rE = S[4 * bs + id], re = S[5 * bs + id];
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  if (G) {
    g0 = G[id];
    g1 = G[bs + id];
    g2 = G[2 * bs + id];
  }
  const double rho_s = rho - sc.dtp * div[0];
  const double ms0 = (sc.a_old * m0 - sc.dt * div[1] + sc.dt * rho * g0) * sc.ian;
  const double ms1 = (sc.a_old * m1 - sc.dt * div[2] + sc.dt * rho * g1) * sc.ian;
  const double ms2 = (sc.a_old * m2 - sc.dt * div[3] + sc.dt * rho * g2) * sc.ian;
  const double rE_s = nyx::predictor_energy(k, sc, rE, re, div[4], m0, m1, m2, g0, g1, g2, div[1],
                                              div[2], div[3], rho_s, ms0, ms1, ms2);
  const double re_s = (sc.ao2 * re - sc.ahdt * div[5] - sc.ahdt * pdivu + sc.expn * re) * sc.ian2;
  double o6[6];
  nyx::finish_cell(k, sc, rho, m0, m1, m2, g0, g1, g2, g0, g1, g2, rho_s, ms0, ms1, ms2, rE_s, re_s,
                   k.grav_corrector && full, full, o6);
  const double mn0 = o6[1], mn1 = o6[2], mn2 = o6[3], rEn = o6[4], ren = o6[5];
  if (!(rho_s > 0.0)) flags |= nyx::ST_NEGATIVE;
  if (!isfinite(rho_s) || !isfinite(rEn) || !isfinite(ren) || !isfinite(mn0) || !isfinite(mn1) ||
      !isfinite(mn2))
    flags |= nyx::ST_NONFINITE;
  Sn[id] = rho_s;
  Sn[bs + id] = mn0;
  Sn[2 * bs + id] = mn1;
  Sn[3 * bs + id] = mn2;
  Sn[4 * bs + id] = rEn;
  Sn[5 * bs + id] = ren;
  if (want_dt && full) {
    // CFL step of the new state at a_new (Sec. 3.5), in the path's precision
    const R r = (R)rho_s;
    R p = (R)k.gm1 * (R)ren;
    if (p < (R)k.small_pres) p = (R)k.small_pres;
    const R c = sqrt_r((R)k.gamma * p / r);
    const R an = (R)sc.a_new;
    R t0 = an * (R)b.dx[0] / (rabs((R)mn0 / r) + c);
    R t1 = an * (R)b.dx[1] / (rabs((R)mn1 / r) + c);
    R t2 = an * (R)b.dx[2] / (rabs((R)mn2 / r) + c);
    if ((double)t0 < dtmin) dtmin = (double)t0;
    if ((double)t1 < dtmin) dtmin = (double)t1;
    if ((double)t2 < dtmin) dtmin = (double)t2;
  }
}

// Exact float -> double conversion on the integer pipe (FP32 results are
// never subnormal here: the mixed unit is built with flush-to-zero).  The
// FP64 pipe of this part runs at 1/64 of the FP32 rate and also executes the
// F2F conversion, so keeping conversions off it matters.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned bias = (e == 0u) ? 0u : ((e == 0xffu) ? 0x70000000u : 0x38000000u);
  const unsigned hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + bias);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// finite test on the high word (integer pipe)
__device__ __forceinline__ bool finite_hi(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}

// Mixed-precision update of one cell: the same FP64 update (flux divergence
// accumulated in FP64 from exactly converted FP32 fluxes, comoving weights,
// gravity predictor-corrector, FP64 kinetic-energy subtraction), arranged so
// that the FP64 pipe does as little as possible: the p div U source term is
// formed in FP32, 1/rho is an FP32 reciprocal refined by one FP64 Newton step.
// FP32 constants of the mixed update (converted once per work item).
struct MixK {
  float idx0, idx1, idx2, gm1, gamma, small_pres, an_dx0, an_dx1, an_dx2;
};

__device__ __forceinline__ MixK make_mixk(const nyx::SchemeConsts &k, const nyx::StepConsts &sc,
                                          const nyx::BoxDev &b) {
  MixK m;
  m.idx0 = d2f_rn(b.idx[0]);
  m.idx1 = d2f_rn(b.idx[1]);
  m.idx2 = d2f_rn(b.idx[2]);
  m.gm1 = d2f_rn(k.gm1);
  m.gamma = d2f_rn(k.gamma);
  m.small_pres = d2f_rn(k.small_pres);
  m.an_dx0 = d2f_rn(sc.a_new * b.dx[0]);
  m.an_dx1 = d2f_rn(sc.a_new * b.dx[1]);
  m.an_dx2 = d2f_rn(sc.a_new * b.dx[2]);
  return m;
}

__device__ __forceinline__ void update_cell_mixed(
    const nyx::SchemeConsts &k, const nyx::StepConsts &sc, const nyx::BoxDev &b, const MixK &mk,
    const double *S, const double *G, double *Sn, long long id, const float (&Fxm)[8],
    const float (&Fxp)[8], const float (&Fym)[8], const float (&Fyp)[8], const float (&Fzm)[8],
    const float (&Fzp)[8], float &dtmin, unsigned &flags, bool want_dt, bool full) {
  const long long bs = b.stride;
  double div[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const double dx_ = f2d_exact(Fxp[c]) - f2d_exact(Fxm[c]);
    const double dy_ = f2d_exact(Fyp[c]) - f2d_exact(Fym[c]);
    const double dz_ = f2d_exact(Fzp[c]) - f2d_exact(Fzm[c]);
    div[c] = dx_ * b.idx[0] + dy_ * b.idx[1] + dz_ * b.idx[2];
  }
  const float pdivu_f = 0.5f * (Fxp[7] + Fxm[7]) * (Fxp[6] - Fxm[6]) * mk.idx0 +
                        0.5f * (Fyp[7] + Fym[7]) * (Fyp[6] - Fym[6]) * mk.idx1 +
                        0.5f * (Fzp[7] + Fzm[7]) * (Fzp[6] - Fzm[6]) * mk.idx2;
  const double pdivu = f2d_exact(pdivu_f);
  const double rho = S[id];
  const double m0 = S[bs + id], m1 = S[2 * bs + id], m2 = S[3 * bs + id];
  const double rE = S[4 * bs + id], re = S[5 * bs + id];
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  if (G) {
    g0 = G[id];
    g1 = G[bs + id];
    g2 = G[2 * bs + id];
  }
  const double rho_s = rho - sc.dtp * div[0];
  const double dtrho = sc.dt * rho;
  const double ms0 = (sc.a_old * m0 - sc.dt * div[1] + dtrho * g0) * sc.ian;
  const double ms1 = (sc.a_old * m1 - sc.dt * div[2] + dtrho * g1) * sc.ian;
  const double ms2 = (sc.a_old * m2 - sc.dt * div[3] + dtrho * g2) * sc.ian;
  // 1/rho: FP32 reciprocal, one Newton step in FP64 (relative error ~1e-14)
  const float rho_f = d2f_rn(rho_s);
  double ir = f2d_exact(1.0f / rho_f);
  ir = ir * (2.0 - rho_s * ir);
  const double mg = m0 * g0 + m1 * g1 + m2 * g2;
  double rE_s;
  if (k.grav_energy) {
    // Sec. 3.2, second alternative: the kinetic-energy change of the gravity update
    const double mh0 = (sc.a_old * m0 - sc.dt * div[1]) * sc.ian;
    const double mh1 = (sc.a_old * m1 - sc.dt * div[2]) * sc.ian;
    const double mh2 = (sc.a_old * m2 - sc.dt * div[3]) * sc.ian;
    const double kh = mh0 * mh0 + mh1 * mh1 + mh2 * mh2;
    const double ks = ms0 * ms0 + ms1 * ms1 + ms2 * ms2;
    rE_s = (sc.ao2 * rE - sc.ahdt * div[4] + sc.expn * re) * sc.ian2 + 0.5 * (ks - kh) * ir;
  } else {
    rE_s = (sc.ao2 * rE - sc.ahdt * div[4] + sc.dta * mg + sc.expn * re) * sc.ian2;
  }
  const double re_s = (sc.ao2 * re - sc.ahdt * (div[5] + pdivu) + sc.expn * re) * sc.ian2;
  double mn0 = ms0, mn1 = ms1, mn2 = ms2, rEn = rE_s;
  if (k.grav_corrector && full) {
    const double cr = sc.hdt * (rho_s - rho) * sc.ian;
    mn0 = ms0 + cr * g0;
    mn1 = ms1 + cr * g1;
    mn2 = ms2 + cr * g2;
    if (k.grav_energy) {
      const double ks = ms0 * ms0 + ms1 * ms1 + ms2 * ms2;
      const double kn = mn0 * mn0 + mn1 * mn1 + mn2 * mn2;
      rEn = rE_s + 0.5 * (kn - ks) * ir;
    } else {
      const double msg = ms0 * g0 + ms1 * g1 + ms2 * g2;
      rEn = rE_s + sc.hdt * (sc.a_new * msg - sc.a_old * mg) * sc.ian2;
    }
  }
  double ren = re_s;
  if (full) {
    const double ke = 0.5 * (mn0 * mn0 + mn1 * mn1 + mn2 * mn2) * ir;
    if (rEn - ke > k.eta_de * rEn) {
      ren = rEn - ke;
    } else {
      rEn = ren + ke;
    }
    if (ren < k.efloor) {
      ren = k.efloor;
      rEn = ren + ke;
    }
  }
  if (!(rho_f > 0.0f)) flags |= nyx::ST_NEGATIVE;
  if (!finite_hi(rho_s) || !finite_hi(rEn) || !finite_hi(ren) || !finite_hi(mn0) ||
      !finite_hi(mn1) || !finite_hi(mn2))
    flags |= nyx::ST_NONFINITE;
  Sn[id] = rho_s;
  Sn[bs + id] = mn0;
  Sn[2 * bs + id] = mn1;
  Sn[3 * bs + id] = mn2;
  Sn[4 * bs + id] = rEn;
  Sn[5 * bs + id] = ren;
  if (want_dt && full) {
    const float irf = 1.0f / rho_f;
    float p = mk.gm1 * d2f_rn(ren);
    if (p < mk.small_pres) p = mk.small_pres;
    const float c2 = mk.gamma * p * irf;
    const float c = c2 * rsqrtf(c2);
    const float t0 = mk.an_dx0 / (fabsf(d2f_rn(mn0) * irf) + c);
    const float t1 = mk.an_dx1 / (fabsf(d2f_rn(mn1) * irf) + c);
    const float t2 = mk.an_dx2 / (fabsf(d2f_rn(mn2) * irf) + c);
    dtmin = fminf(dtmin, fminf(t0, fminf(t1, t2)));
  }
}

template <class R, int TX, int TY>
__global__ void __launch_bounds__(FusedGeom<R, TX, TY>::NT, 1) k_fused(nyx::FusedArgs a) {
  using FG = FusedGeom<R, TX, TY>;
  constexpr int NC = FG::NC, NE = FG::NE, W = FG::W, WE = FG::WE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *Ps = reinterpret_cast<R *>(smem_raw);  // [5][NE] primitives of plane c
  R *A = Ps + 5 * NE;                        // [NA][NC]
  R *B = A + FG::NA * NC;                    // [NB][NC]
  __shared__ int s_item;

  const nyx::SchemeConsts KK = *a.K;
  const nyx::StepConsts sc = *a.SC;
  const bool mixed = sizeof(R) == 4;
  const Eos<R> E = make_eos<R>(KK, mixed);
  TraceSrc<R> src;
  src.hdtp = (R)sc.hdtp;
  src.src_u = (R)sc.src_u;
  src.src_p = (R)sc.src_p;

  const int tid = threadIdx.x;
  const bool in_r1 = tid < NC;
  const int i = tid % W - 1;
  const int j = tid / W - 1;
  const int me = tid;  // == (j+1)*W + (i+1) for owned columns
  const int me_e = (j + 3) * WE + (i + 3);
  double dtmin = __longlong_as_double(0x7ff0000000000000LL);
  unsigned flags = 0;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= a.nitems) break;
    const nyx::WorkItem w = a.items[item];
    const nyx::BoxDev b = a.boxes[w.box];
    const nyx::BoxStep bst = a.BS[w.box];
    const int nxt = w.nx, nyt = w.ny, nz = b.n[2];
    const int zb = w.z0, ze = w.z0 + w.nz;  // this item's planes [zb, ze)
    const long long bs = b.stride;
    const long long ps = (long long)b.N[0] * b.N[1];
    const double *S = a.S + nyx::NCONS * b.pref;
    const double *G = a.G ? a.G + nyx::NGRAV * b.pref : nullptr;
    const R *FL = E.flat ? static_cast<const R *>(a.flat) + b.pref : nullptr;
    double *Sn = a.Sn + nyx::NCONS * b.pref;
    const bool act = in_r1 && i <= nxt && j <= nyt;
    const bool inX = i >= 0 && i < nxt, inY = j >= 0 && j < nyt;
    const bool fxf = i >= 0 && i <= nxt, fyf = j >= 0 && j <= nyt;
    const long long col = (long long)(w.y0 + j + 4) * b.N[0] + (w.x0 + i + 4);
    const R dtdx0 = (R)bst.dtdx[0], dtdx1 = (R)bst.dtdx[1], dtdx2 = (R)bst.dtdx[2];
    const R c30 = (R)bst.cdt3[0], c31 = (R)bst.cdt3[1], c32 = (R)bst.cdt3[2];
    const R ch0 = (R)bst.chalf[0], ch1 = (R)bst.chalf[1], ch2 = (R)bst.chalf[2];
    const MixK mixk = make_mixk(KK, sc, b);

    // own-column z window: planes c-2 .. c+2
    R win[5][5];
    if (act) {
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        R q[5];
        prims_of<R>(S, bs, col + (long long)(zb + o - 3 + 4) * ps, E, q);
#pragma unroll
        for (int v = 0; v < 5; ++v) win[o][v] = q[v];
      }
    }
    // values carried from plane c-1 to plane c
    R qzp_prev[5], qx_prev_m[5], qx_prev_p[5], qy_prev_m[5], qy_prev_p[5];
    R qzx_prev[5], qzy_prev[5], qzf_prev[5];
    TFlux<R> Fz_prev, Fzx_prev, Fzy_prev;
    R Ffz_prev[8];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      qzp_prev[k] = qx_prev_m[k] = qx_prev_p[k] = qy_prev_m[k] = qy_prev_p[k] = R(0);
      qzx_prev[k] = qzy_prev[k] = qzf_prev[k] = R(0);
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) Fz_prev.f[k] = Fzx_prev.f[k] = Fzy_prev.f[k] = R(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) Ffz_prev[k] = R(0);

    const int nstrip = 4 * (nxt + 2) + 4 * (nyt + 2);

    for (int c = zb - 1; c <= ze; ++c) {
      // ---------------- stage 0: primitives
      if (act) {
        R q[5];
        prims_of<R>(S, bs, col + (long long)(c + 2 + 4) * ps, E, q);
#pragma unroll
        for (int v = 0; v < 5; ++v) win[4][v] = q[v];
#pragma unroll
        for (int v = 0; v < 5; ++v) Ps[v * NE + me_e] = win[2][v];
      }
      for (int t = tid; t < nstrip; t += FG::NT) {
        int x, y;
        if (t < 4 * (nyt + 2)) {  // left / right strips, rows -1..nyt
          int r = t % (nyt + 2), s = t / (nyt + 2);
          y = r - 1;
          x = (s < 2) ? (-3 + s) : (nxt + 1 + (s - 2));
        } else {  // bottom / top strips, columns -1..nxt
          int u = t - 4 * (nyt + 2);
          int r = u % (nxt + 2), s = u / (nxt + 2);
          x = r - 1;
          y = (s < 2) ? (-3 + s) : (nyt + 1 + (s - 2));
        }
        long long id = ((long long)(c + 4) * b.N[1] + (w.y0 + y + 4)) * b.N[0] + (w.x0 + x + 4);
        R q[5];
        prims_of<R>(S, bs, id, E, q);
        const int e = (y + 3) * WE + (x + 3);
#pragma unroll
        for (int v = 0; v < 5; ++v) Ps[v * NE + e] = q[v];
      }
      __syncthreads();

      // ---------------- stage 1: PPM + tracing at plane c
      R qx_m[5], qx_p[5], qy_m[5], qy_p[5], qz_m[5], qz_p[5];
      if (act) {
        const R rho = win[2][0], p = win[2][4];
        const R cs = sqrt_r(E.gamma * p / rho);
        R g3[3] = {R(0), R(0), R(0)};
        if (G) {
          const long long id = col + (long long)(c + 4) * ps;
          g3[0] = to_r<R>(G[id]);
          g3[1] = to_r<R>(G[bs + id]);
          g3[2] = to_r<R>(G[2 * bs + id]);
        }
        const R fl = FL ? FL[col + (long long)(c + 4) * ps] : R(1);
        R s[5][5];
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
          for (int o = 0; o < 5; ++o) s[v][o] = Ps[v * NE + me_e + (o - 2)];
        trace_cell<R, 0>(E, s, cs, g3, dtdx0, src, fl, qx_m, qx_p);
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
          for (int o = 0; o < 5; ++o) s[v][o] = Ps[v * NE + me_e + (o - 2) * WE];
        trace_cell<R, 1>(E, s, cs, g3, dtdx1, src, fl, qy_m, qy_p);
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
          for (int o = 0; o < 5; ++o) s[v][o] = win[o][v];
        trace_cell<R, 2>(E, s, cs, g3, dtdx2, src, fl, qz_m, qz_p);
        put5(A, NC, 0, me, qx_p);
        put5(A, NC, 5, me, qy_p);
      }
      __syncthreads();

      // ---------------- stage 2: normal solves
      TFlux<R> Fz;
      if (act) {
        R F8[8], l[5];
        if (fxf) {
          get5(A, NC, 0, me - 1, l);
          face_flux<R, 0>(E, l, qx_m, F8);
          put7(B, NC, 0, me, tflux_of(F8));
        }
        if (fyf) {
          get5(A, NC, 5, me - W, l);
          face_flux<R, 1>(E, l, qy_m, F8);
          put7(B, NC, 7, me, tflux_of(F8));
        }
        if (c >= zb) {
          face_flux<R, 2>(E, qzp_prev, qz_m, F8);
          Fz = tflux_of(F8);
        }
      }
      __syncthreads();

      // ---------------- stage 3: corner coupling, theta = 1/3
      R qxy_m[5], qxy_p[5], qyx_m[5], qyx_p[5], qzx_m[5], qzx_p[5], qzy_m[5], qzy_p[5];
      R qxz_m[5], qxz_p[5], qyz_m[5], qyz_p[5];
      const bool zc = (c >= zb + 1);  // plane c-1 is one of the item's planes
      if (act) {
        if (inY) {
          TFlux<R> Fm = get7(B, NC, 7, me), Fp = get7(B, NC, 7, me + W);
          transverse1(E, qx_m, c31, Fp, Fm, qxy_m);
          transverse1(E, qx_p, c31, Fp, Fm, qxy_p);
          transverse1(E, qz_m, c31, Fp, Fm, qzy_m);
          transverse1(E, qz_p, c31, Fp, Fm, qzy_p);
          put5(A, NC, 0, me, qxy_p);
        }
        if (inX) {
          TFlux<R> Fm = get7(B, NC, 0, me), Fp = get7(B, NC, 0, me + 1);
          transverse1(E, qy_m, c30, Fp, Fm, qyx_m);
          transverse1(E, qy_p, c30, Fp, Fm, qyx_p);
          transverse1(E, qz_m, c30, Fp, Fm, qzx_m);
          transverse1(E, qz_p, c30, Fp, Fm, qzx_p);
          put5(A, NC, 5, me, qyx_p);
        }
        if (zc) {
          transverse1(E, qx_prev_m, c32, Fz, Fz_prev, qxz_m);
          transverse1(E, qx_prev_p, c32, Fz, Fz_prev, qxz_p);
          transverse1(E, qy_prev_m, c32, Fz, Fz_prev, qyz_m);
          transverse1(E, qy_prev_p, c32, Fz, Fz_prev, qyz_p);
          put5(A, NC, 10, me, qxz_p);
          put5(A, NC, 15, me, qyz_p);
        }
      }
      __syncthreads();

      // ---------------- stage 4: intermediate solves
      TFlux<R> Fzx, Fzy;
      if (act) {
        R F8[8], l[5];
        if (fxf && inY) {  // F^{x|y} at plane c
          get5(A, NC, 0, me - 1, l);
          face_flux<R, 0>(E, l, qxy_m, F8);
          put7(B, NC, 0, me, tflux_of(F8));
        }
        if (fyf && inX) {  // F^{y|x} at plane c
          get5(A, NC, 5, me - W, l);
          face_flux<R, 1>(E, l, qyx_m, F8);
          put7(B, NC, 7, me, tflux_of(F8));
        }
        if (zc && fxf) {  // F^{x|z} at plane c-1
          get5(A, NC, 10, me - 1, l);
          face_flux<R, 0>(E, l, qxz_m, F8);
          put7(B, NC, 14, me, tflux_of(F8));
        }
        if (zc && fyf) {  // F^{y|z} at plane c-1
          get5(A, NC, 15, me - W, l);
          face_flux<R, 1>(E, l, qyz_m, F8);
          put7(B, NC, 21, me, tflux_of(F8));
        }
        if (c >= zb && inX) {  // F^{z|x} at face c-1/2
          face_flux<R, 2>(E, qzx_prev, qzx_m, F8);
          Fzx = tflux_of(F8);
        }
        if (c >= zb && inY) {  // F^{z|y} at face c-1/2
          face_flux<R, 2>(E, qzy_prev, qzy_m, F8);
          Fzy = tflux_of(F8);
        }
      }
      __syncthreads();

      // ---------------- stage 5: final states, theta = 1/2
      R qzf_m[5], qzf_p[5], qxf_m[5], qxf_p[5], qyf_m[5], qyf_p[5];
      if (act) {
        if (inX && inY) {  // z states at plane c: by F^{x|y} in x, F^{y|x} in y
          TFlux<R> Am = get7(B, NC, 0, me), Ap = get7(B, NC, 0, me + 1);
          TFlux<R> Bm = get7(B, NC, 7, me), Bp = get7(B, NC, 7, me + W);
          transverse2(E, qz_m, ch0, Ap, Am, ch1, Bp, Bm, qzf_m);
          transverse2(E, qz_p, ch0, Ap, Am, ch1, Bp, Bm, qzf_p);
        }
        if (zc && inY) {  // x states at plane c-1: by F^{y|z} in y, F^{z|y} in z
          TFlux<R> Am = get7(B, NC, 21, me), Ap = get7(B, NC, 21, me + W);
          transverse2(E, qx_prev_m, ch1, Ap, Am, ch2, Fzy, Fzy_prev, qxf_m);
          transverse2(E, qx_prev_p, ch1, Ap, Am, ch2, Fzy, Fzy_prev, qxf_p);
          put5(A, NC, 0, me, qxf_p);
        }
        if (zc && inX) {  // y states at plane c-1: by F^{x|z} in x, F^{z|x} in z
          TFlux<R> Am = get7(B, NC, 14, me), Ap = get7(B, NC, 14, me + 1);
          transverse2(E, qy_prev_m, ch0, Ap, Am, ch2, Fzx, Fzx_prev, qyf_m);
          transverse2(E, qy_prev_p, ch0, Ap, Am, ch2, Fzx, Fzx_prev, qyf_p);
          put5(A, NC, 5, me, qyf_p);
        }
      }
      __syncthreads();

      // ---------------- stage 6: final solves
      R Ffz[8];
      if (act) {
        R F8[8], l[5];
        if (zc && fxf && inY) {
          get5(A, NC, 0, me - 1, l);
          face_flux<R, 0>(E, l, qxf_m, F8);
#pragma unroll
          for (int k = 0; k < 8; ++k) B[k * NC + me] = F8[k];
        }
        if (zc && fyf && inX) {
          get5(A, NC, 5, me - W, l);
          face_flux<R, 1>(E, l, qyf_m, F8);
#pragma unroll
          for (int k = 0; k < 8; ++k) B[(8 + k) * NC + me] = F8[k];
        }
        if (c >= zb && inX && inY) face_flux<R, 2>(E, qzf_prev, qzf_m, Ffz);
      }
      __syncthreads();

      // ---------------- stage 7: update of plane c-1
      if (act && zc && inX && inY) {
        R Fxm[8], Fxp[8], Fym[8], Fyp[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          Fxm[k] = B[k * NC + me];
          Fxp[k] = B[k * NC + me + 1];
          Fym[k] = B[(8 + k) * NC + me];
          Fyp[k] = B[(8 + k) * NC + me + W];
        }
        const long long id = col + (long long)(c - 1 + 4) * ps;
        if constexpr (sizeof(R) == 4) {
          float dtf = __int_as_float(0x7f800000);
          update_cell_mixed(KK, sc, b, mixk, S, G, Sn, id, Fxm, Fxp, Fym, Fyp, Ffz_prev, Ffz, dtf,
                            flags, a.dtacc != nullptr, !a.predict_only);
          if ((double)dtf < dtmin) dtmin = (double)dtf;
        } else
          update_cell<R>(KK, sc, b, S, G, Sn, id, Fxm, Fxp, Fym, Fyp, Ffz_prev, Ffz, dtmin, flags,
                         a.dtacc != nullptr, !a.predict_only);
        if (a.flux_keep) {
          double *fk = a.flux_keep + a.flux_off[w.box];
          const int nx = b.n[0], ny = b.n[1];
          const int gx = w.x0 + i, gy = w.y0 + j, p = c - 1;
          // x faces (6, nz, ny, nx+1): face gx-1/2, and gx+1/2 on the box's last column
          long long fx = (long long)(nx + 1) * ny * nz;
          long long ix = ((long long)p * ny + gy) * (nx + 1) + gx;
#pragma unroll
          for (int k = 0; k < 6; ++k) fk[k * fx + ix] = (double)Fxm[k];
          if (gx == nx - 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) fk[k * fx + ix + 1] = (double)Fxp[k];
          fk += 6 * fx;
          long long fy = (long long)nx * (ny + 1) * nz;
          long long iy = ((long long)p * (ny + 1) + gy) * nx + gx;
#pragma unroll
          for (int k = 0; k < 6; ++k) fk[k * fy + iy] = (double)Fym[k];
          if (gy == ny - 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) fk[k * fy + iy + nx] = (double)Fyp[k];
          fk += 6 * fy;
          long long fz = (long long)nx * ny * (nz + 1);
          long long iz = ((long long)p * ny + gy) * nx + gx;
#pragma unroll
          for (int k = 0; k < 6; ++k) fk[k * fz + iz] = (double)Ffz_prev[k];
          if (p == nz - 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) fk[k * fz + iz + (long long)nx * ny] = (double)Ffz[k];
        }
      }

      // ---------------- carry plane c to plane c+1
      if (act) {
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
          for (int v = 0; v < 5; ++v) win[o][v] = win[o + 1][v];
        copy5(qzp_prev, qz_p);
        copy5(qx_prev_m, qx_m);
        copy5(qx_prev_p, qx_p);
        copy5(qy_prev_m, qy_m);
        copy5(qy_prev_p, qy_p);
        if (c >= zb) Fz_prev = Fz;
        if (inX) copy5(qzx_prev, qzx_p);
        if (inY) copy5(qzy_prev, qzy_p);
        if (c >= zb && inX) Fzx_prev = Fzx;
        if (c >= zb && inY) Fzy_prev = Fzy;
        if (inX && inY) copy5(qzf_prev, qzf_p);
        if (c >= zb && inX && inY) copy8(Ffz_prev, Ffz);
      }
    }
    __syncthreads();
  }

  if (a.dtacc) {
    for (int o = 16; o > 0; o >>= 1) {
      double v = __shfl_xor_sync(0xffffffffu, dtmin, o);
      if (v < dtmin) dtmin = v;
    }
    if ((tid & 31) == 0 && dtmin < __longlong_as_double(0x7ff0000000000000LL))
      nyx::atomic_min_pos(a.dtacc, dtmin);
  }
  if (flags) atomicOr(a.status, flags);
}

// The dynamic shared-memory attribute is set by max_grid_one, which every
// plan calls for its shapes when it is created (outside any graph capture).
// ---------------------------------------------------------------- shock flattening
// Coefficient 1 - max_d flat_d of every cell of [-1, n]^3 of every box (the
// cells the advance traces; the +-3 stencil fits in the 4 ghost cells), from
// the primitives exactly as the advance forms them in type R.  One block per
// tile of output columns (nyx::FlatTile) walks the planes c = -1 .. n_z: it
// keeps p and u_z of planes c-3 .. c+3 at the output columns in a ring, and
// p, u_x, u_y of plane c on the tile's frame (+-3 in x and y), so that each
// cell's primitives are formed about once per tile instead of once per
// stencil point.  The other cells keep the 1 they were set to when the
// buffer was made.
constexpr int FLAT_TX = 34, FLAT_TY = 17;  // largest output tile
constexpr int FLAT_NO = FLAT_TX * FLAT_TY;
constexpr int FLAT_NF = (FLAT_TX + 6) * (FLAT_TY + 6);
constexpr int FLAT_THREADS = 512;

template <class R>
constexpr size_t flat_smem() {
  return sizeof(R) * (size_t)(14 * FLAT_NO + 3 * FLAT_NF);
}

__device__ __forceinline__ int flat_slot(int k) { return (k + 7) % 7; }  // k >= -7

template <class R>
__global__ void __launch_bounds__(FLAT_THREADS) k_flatten(const nyx::BoxDev *boxes,
                                                          const nyx::FlatTile *tiles,
                                                          const double *Sall,
                                                          const nyx::SchemeConsts *K, R *FLall) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *ringp = reinterpret_cast<R *>(smem_raw);  // [7][FLAT_NO] p at the output columns
  R *ringw = ringp + 7 * FLAT_NO;               // [7][FLAT_NO] u_z at the output columns
  R *fp = ringw + 7 * FLAT_NO;                  // [FLAT_NF] p of plane c on the frame
  R *fu = fp + FLAT_NF;                         // [FLAT_NF] u_x
  R *fv = fu + FLAT_NF;                         // [FLAT_NF] u_y
  const nyx::FlatTile T = tiles[blockIdx.x];
  const nyx::BoxDev b = boxes[T.box];
  const Eos<R> E = make_eos<R>(*K, sizeof(R) == 4);
  const double *S = Sall + nyx::NCONS * b.pref;
  R *FL = FLall + b.pref;
  const long long bs = b.stride;
  const int N0 = b.N[0], N1 = b.N[1];
  const int NO = T.nx * T.ny, FW = T.nx + 6, NF = FW * (T.ny + 6);
  auto cell = [&](int i, int j, int k) {
    return ((long long)(k + 4) * N1 + (j + 4)) * N0 + (i + 4);
  };
  auto ring_plane = [&](int k) {
    R *P = ringp + flat_slot(k) * FLAT_NO, *U = ringw + flat_slot(k) * FLAT_NO;
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
      R q[5];
      prims_of<R>(S, bs, cell(T.x0 + o % T.nx, T.y0 + o / T.nx, k), E, q);
      P[o] = q[4];
      U[o] = q[3];
    }
  };
  for (int k = -4; k <= 1; ++k) ring_plane(k);
  for (int c = -1; c <= b.n[2]; ++c) {
    ring_plane(c + 3);
    for (int e = threadIdx.x; e < NF; e += blockDim.x) {
      R q[5];
      prims_of<R>(S, bs, cell(T.x0 - 3 + e % FW, T.y0 - 3 + e / FW, c), E, q);
      fp[e] = q[4];
      fu[e] = q[1];
      fv[e] = q[2];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
      const int ox = o % T.nx, oy = o / T.nx;
      const int fe = (oy + 3) * FW + (ox + 3);
      R p[7], u[5];
      R fmax;
#pragma unroll
      for (int s = 0; s < 7; ++s) p[s] = fp[fe + s - 3];
#pragma unroll
      for (int s = 0; s < 5; ++s) u[s] = fu[fe + s - 2];
      fmax = flat_dir(p, u, E.small_pres);
#pragma unroll
      for (int s = 0; s < 7; ++s) p[s] = fp[fe + (s - 3) * FW];
#pragma unroll
      for (int s = 0; s < 5; ++s) u[s] = fv[fe + (s - 2) * FW];
      R f = flat_dir(p, u, E.small_pres);
      if (f > fmax) fmax = f;
#pragma unroll
      for (int s = 0; s < 7; ++s) p[s] = ringp[flat_slot(c + s - 3) * FLAT_NO + o];
#pragma unroll
      for (int s = 0; s < 5; ++s) u[s] = ringw[flat_slot(c + s - 2) * FLAT_NO + o];
      f = flat_dir(p, u, E.small_pres);
      if (f > fmax) fmax = f;
      FL[cell(T.x0 + ox, T.y0 + oy, c)] = R(1) - fmax;
    }
    __syncthreads();
  }
}

template <class R>
int launch_flatten_t(const nyx::BoxDev *boxes, const nyx::FlatTile *tiles, int ntiles,
                     const double *S, const nyx::SchemeConsts *K, void *fl, cudaStream_t st) {
  if (ntiles < 1) return 0;
  k_flatten<R><<<ntiles, FLAT_THREADS, flat_smem<R>(), st>>>(boxes, tiles, S, K,
                                                              static_cast<R *>(fl));
  return (int)cudaGetLastError();
}

template <class R>
int flatten_init_t() {
  return (int)cudaFuncSetAttribute(k_flatten<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)flat_smem<R>());
}

// Set every value of a coefficient buffer to 1 (no flattening).
template <class R>
__global__ void k_flat_ones(R *fl, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    fl[t] = R(1);
}

template <class R, int TX, int TY>
int launch_one(const nyx::FusedArgs &a, int grid, cudaStream_t st) {
  using FG = FusedGeom<R, TX, TY>;
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return (int)e;
  k_fused<R, TX, TY><<<grid, FG::NT, FG::SMEM, st>>>(a);
  return (int)cudaGetLastError();
}

template <class R, int TX, int TY>
int max_grid_one() {
  using FG = FusedGeom<R, TX, TY>;
  cudaFuncSetAttribute(k_fused<R, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)FG::SMEM);
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<R, TX, TY>, FG::NT, FG::SMEM);
  if (per_sm < 1) per_sm = 1;
  return per_sm * nsm;
}

}  // namespace NYX_NS
