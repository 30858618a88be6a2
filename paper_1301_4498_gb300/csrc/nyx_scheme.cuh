// nyx_scheme.cuh -- per-cell and per-face arithmetic of the comoving PPM
// Godunov advance (Nyx, Almgren et al. 2013, Sec. 2.2 and 3.2), templated on
// the arithmetic type R.  R = double is the FP64 path: every expression has
// one fixed form and the translation units that use it are compiled with
// --fmad=false, so results are reproducible to the last bit.  R = float is the
// reduced-precision part of the mixed path.
//
// The header is included by several translation units with different
// floating-point flags; NYX_NS gives each its own namespace so that no
// instantiation is shared across them.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#ifndef NYX_NS
#error "define NYX_NS before including nyx_scheme.cuh"
#endif

namespace NYX_NS {

template <class R>
struct Eos {
  R gamma, gm1, igm1, kshock, small_dens, small_pres, tol;
  int max_iter;
  int plm;     // PLM profiles instead of PPM (Sec. 3.2)
  int linear;  // the linearised Riemann solver instead of the two-shock one (Sec. 3.2)
  int flat;    // Colella-Woodward shock flattening (coefficients from k_flatten)
};

template <class R>
__device__ __forceinline__ R sqrt_r(R x);
template <>
__device__ __forceinline__ double sqrt_r<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float sqrt_r<float>(float x) { return sqrtf(x); }

template <class R>
__device__ __forceinline__ R rabs(R x) { return fabs(x); }
template <class R>
__device__ __forceinline__ R rcopysign(R m, R s) { return copysign(m, s); }

// ---------------------------------------------------------------- PPM
// MC-limited slope, fourth-order interface value, CW84 parabola limiter
// (Colella & Woodward 1984, named in Sec. 3.2).  Here and in the corner
// coupling below, the FP32 instantiation takes the same values in select form
// (every lane computes both outcomes, so lanes that take different limiter
// branches do not split their warp); the FP64 one keeps the branch form, the
// oracle's expressions one for one.
template <class R>
__device__ __forceinline__ R mc_slope(R sm, R s0, R sp) {
  if constexpr (sizeof(R) == 4) {
    const float dc = 0.5f * (sp - sm), dl = s0 - sm, dr = sp - s0;
    const float m = fminf(fabsf(dc), fminf(2.0f * fabsf(dl), 2.0f * fabsf(dr)));
    return (dl * dr > 0.0f) ? copysignf(m, dc) : 0.0f;
  }
  R dc = R(0.5) * (sp - sm);
  R dl = s0 - sm;
  R dr = sp - s0;
  if (dl * dr > R(0)) {
    R m = rabs(dc);
    R b = R(2) * rabs(dl);
    R c = R(2) * rabs(dr);
    if (b < m) m = b;
    if (c < m) m = c;
    return rcopysign(m, dc);
  }
  return R(0);
}

template <class R>
__device__ __forceinline__ R interface_value(R s0, R s1, R d0, R d1) {
  return R(0.5) * (s0 + s1) - (d1 - d0) * R(1.0 / 6.0);
}

// s0..s4 = s_{i-2}..s_{i+2}
template <class R>
__device__ __forceinline__ void ppm_coeffs(R s0, R s1, R s2, R s3, R s4, R &sLo, R &sRo, R &s6o) {
  R dm = mc_slope(s0, s1, s2);
  R d0 = mc_slope(s1, s2, s3);
  R dp = mc_slope(s2, s3, s4);
  R sL = interface_value(s1, s2, dm, d0);
  R sR = interface_value(s2, s3, d0, dp);
  R si = s2;
  if constexpr (sizeof(R) == 4) {
    const bool flat = (sR - si) * (si - sL) <= 0.0f;
    const float D = sR - sL, M = si - 0.5f * (sL + sR);
    const float DM = D * M, D26 = D * D * (1.0f / 6.0f);
    const bool cl = DM > D26, cr = !cl && (-D26 > DM);
    const float nL = flat ? si : (cl ? 3.0f * si - 2.0f * sR : sL);
    const float nR = flat ? si : (cr ? 3.0f * si - 2.0f * sL : sR);
    sLo = nL;
    sRo = nR;
    s6o = 6.0f * (si - 0.5f * (nL + nR));
    return;
  }
  if ((sR - si) * (si - sL) <= R(0)) {
    sL = si;
    sR = si;
  } else {
    R D = sR - sL;
    R M = si - R(0.5) * (sL + sR);
    if (D * M > D * D * R(1.0 / 6.0)) {
      sL = R(3) * si - R(2) * sR;
    } else if (-(D * D * R(1.0 / 6.0)) > D * M) {
      sR = R(3) * si - R(2) * sL;
    }
  }
  sLo = sL;
  sRo = sR;
  s6o = R(6) * (si - R(0.5) * (sL + sR));
}

// PLM (Sec. 3.2): the linear profile with the cell's MC-limited slope d,
// written as a parabola with edge values s_i -+ d/2 and no curvature, so that
// ppm_ip / ppm_im below give the averages of the linear profile.
template <class R>
__device__ __forceinline__ void plm_coeffs(R s1, R s2, R s3, R &sLo, R &sRo, R &s6o) {
  const R d = mc_slope(s1, s2, s3);
  sLo = s2 - R(0.5) * d;
  sRo = s2 + R(0.5) * d;
  s6o = R(0);
}

template <class R>
__device__ __forceinline__ R ppm_ip(R sL, R sR, R s6, R sig) {
  return sR - R(0.5) * sig * ((sR - sL) - (R(1) - R(2.0 / 3.0) * sig) * s6);
}
template <class R>
__device__ __forceinline__ R ppm_im(R sL, R sR, R s6, R sig) {
  return sL + R(0.5) * sig * ((sR - sL) + (R(1) - R(2.0 / 3.0) * sig) * s6);
}

// ---------------------------------------------------------------- tracing
// Characteristic tracing with a reference state (Sec. 3.2): the reference is
// the average of the parabola over the domain of dependence of the fastest
// wave moving toward the face (the edge value if it moves away); the other
// waves moving toward the face are projected with the primitive-system
// eigenvectors at the cell centre.  Half-step comoving sources (Sec. 2.2 in
// primitive form) are added to both edge states.
// ---------------------------------------------------------------- shock flattening
// Colella & Woodward (1984), the PPM that Sec. 3.2 cites.  Along one
// direction, a cell is in a shock when the pressure across it (cells -1,
// +1) differs by more than 0.33 of the smaller of the two and the flow
// converges (u(-1) > u(+1)); its steepness chi = clamp(10 (z - 0.75), 0, 1),
// z = |p(+1) - p(-1)| / max(|p(+2) - p(-2)|, small_pres), is 0 outside a
// shock.  The cell's flattening is the larger chi of itself and of its
// neighbour on the low-pressure side (the +1 one when p(+1) = p(-1)).
template <class R>
__device__ __forceinline__ R shock_chi(R pm2, R pm1, R pp1, R pp2, R um1, R up1, R small_pres) {
  const R dp1 = pp1 - pm1;
  const R lo = (pp1 < pm1) ? pp1 : pm1;
  if (!(rabs(dp1) > R(0.33) * lo)) return R(0);
  if (!(um1 - up1 > R(0))) return R(0);
  R den = rabs(pp2 - pm2);
  if (den < small_pres) den = small_pres;
  const R z = rabs(dp1) / den;
  R w = R(10) * (z - R(0.75));
  if (w < R(0)) w = R(0);
  if (w > R(1)) w = R(1);
  return w;
}

// Flattening along one direction: p[o] at offsets o - 3 (o = 0..6), u[o] the
// velocity along it at offsets o - 2 (o = 0..4).
template <class R>
__device__ __forceinline__ R flat_dir(const R (&p)[7], const R (&u)[5], R small_pres) {
  const R c0 = shock_chi(p[1], p[2], p[4], p[5], u[1], u[3], small_pres);
  const R cn = (p[4] - p[2] > R(0)) ? shock_chi(p[0], p[1], p[3], p[4], u[0], u[2], small_pres)
                                    : shock_chi(p[2], p[3], p[5], p[6], u[2], u[4], small_pres);
  return (c0 > cn) ? c0 : cn;
}

template <class R>
struct TraceSrc {
  R hdtp;   // dt'/2
  R src_u;  // (a_new - a_old)/a_half / 2
  R src_p;  // 3 (gamma-1) (a_new - a_old)/a_half / 2
};

// s[v][o]: variable v of (rho, u_x, u_y, u_z, p) at cells i-2..i+2 along DIR.
// fl: the cell's shock-flattening coefficient (1: none).
// Outputs qm (low face i-1/2) and qp (high face i+1/2), lab frame.
template <class R, int DIR>
__device__ __forceinline__ void trace_cell(const Eos<R> &E, const R (&s)[5][5], R c,
                                           const R (&g3)[3], R dtdx, const TraceSrc<R> &src,
                                           R fl, R (&qm)[5], R (&qp)[5]) {
  constexpr int NV = 1 + DIR;
  R sL[5], sR[5], s6[5];
  if (E.plm) {
#pragma unroll
    for (int v = 0; v < 5; ++v) plm_coeffs(s[v][1], s[v][2], s[v][3], sL[v], sR[v], s6[v]);
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v)
      ppm_coeffs(s[v][0], s[v][1], s[v][2], s[v][3], s[v][4], sL[v], sR[v], s6[v]);
  }
  // shock flattening: each profile pulled toward the cell value
  if (fl < R(1)) {
    const R gl = R(1) - fl;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sL[v] = fl * sL[v] + gl * s[v][2];
      sR[v] = fl * sR[v] + gl * s[v][2];
      s6[v] = fl * s6[v];
    }
  }
  const R rho = s[0][2];
  const R un = s[NV][2];
  const R pr = s[4][2];
  const R lam0 = un - c, lam1 = un, lam2 = un + c;
  const R sig0 = rabs(lam0) * dtdx, sig1 = rabs(lam1) * dtdx, sig2 = rabs(lam2) * dtdx;
  const R c2 = c * c;
  const R ic2 = R(1) / c2;
  const R hc2 = R(0.5) * ic2;
  const R rc = rho * c;
  const R cor = c / rho;

  // The fastest wave toward a face is the reference itself, so its own
  // amplitude is identically zero (beta_+ on the high face, beta_- on the
  // low face) and is not formed.  Each remaining wave needs the parabola
  // integral only of the variables its projection uses: (p, u_n) for the
  // acoustic waves, (rho, p, u_t1, u_t2) for the entropy/shear wave.
  constexpr int T1 = (DIR == 0) ? 1 : 0;
  constexpr int T2 = (DIR == 2) ? 1 : 2;
  constexpr int TV1 = 1 + T1, TV2 = 1 + T2;
  // ---- high face i+1/2: waves with lam > 0
  {
    R ref[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) ref[v] = (lam2 > R(0)) ? ppm_ip(sL[v], sR[v], s6[v], sig2) : sR[v];
    R d0p = R(0), d0n = R(0), d1r = R(0), d1p = R(0), d1a = R(0), d1b = R(0);
    if (lam0 > R(0)) {
      d0p = ref[4] - ppm_ip(sL[4], sR[4], s6[4], sig0);
      d0n = ref[NV] - ppm_ip(sL[NV], sR[NV], s6[NV], sig0);
    }
    if constexpr (sizeof(R) == 4) {
      // the entropy/shear wave's direction varies from lane to lane: selects
      const bool w1 = lam1 > R(0);
      const R e0 = ref[0] - ppm_ip(sL[0], sR[0], s6[0], sig1);
      const R e4 = ref[4] - ppm_ip(sL[4], sR[4], s6[4], sig1);
      const R ea = ref[TV1] - ppm_ip(sL[TV1], sR[TV1], s6[TV1], sig1);
      const R eb = ref[TV2] - ppm_ip(sL[TV2], sR[TV2], s6[TV2], sig1);
      d1r = w1 ? e0 : R(0);
      d1p = w1 ? e4 : R(0);
      d1a = w1 ? ea : R(0);
      d1b = w1 ? eb : R(0);
    } else
    if (lam1 > R(0)) {
      d1r = ref[0] - ppm_ip(sL[0], sR[0], s6[0], sig1);
      d1p = ref[4] - ppm_ip(sL[4], sR[4], s6[4], sig1);
      d1a = ref[TV1] - ppm_ip(sL[TV1], sR[TV1], s6[TV1], sig1);
      d1b = ref[TV2] - ppm_ip(sL[TV2], sR[TV2], s6[TV2], sig1);
    }
    const R bm = (d0p - rc * d0n) * hc2;
    const R b0 = d1r - d1p * ic2;
    qp[0] = ref[0] - bm - b0;
    qp[NV] = ref[NV] - cor * (R(0) - bm);
    qp[TV1] = ref[TV1] - d1a;
    qp[TV2] = ref[TV2] - d1b;
    qp[4] = ref[4] - c2 * bm;
  }
  // ---- low face i-1/2: waves with lam < 0
  {
    R ref[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) ref[v] = (lam0 < R(0)) ? ppm_im(sL[v], sR[v], s6[v], sig0) : sL[v];
    R d2p = R(0), d2n = R(0), d1r = R(0), d1p = R(0), d1a = R(0), d1b = R(0);
    if (lam2 < R(0)) {
      d2p = ref[4] - ppm_im(sL[4], sR[4], s6[4], sig2);
      d2n = ref[NV] - ppm_im(sL[NV], sR[NV], s6[NV], sig2);
    }
    if constexpr (sizeof(R) == 4) {
      const bool w1 = lam1 < R(0);
      const R e0 = ref[0] - ppm_im(sL[0], sR[0], s6[0], sig1);
      const R e4 = ref[4] - ppm_im(sL[4], sR[4], s6[4], sig1);
      const R ea = ref[TV1] - ppm_im(sL[TV1], sR[TV1], s6[TV1], sig1);
      const R eb = ref[TV2] - ppm_im(sL[TV2], sR[TV2], s6[TV2], sig1);
      d1r = w1 ? e0 : R(0);
      d1p = w1 ? e4 : R(0);
      d1a = w1 ? ea : R(0);
      d1b = w1 ? eb : R(0);
    } else
    if (lam1 < R(0)) {
      d1r = ref[0] - ppm_im(sL[0], sR[0], s6[0], sig1);
      d1p = ref[4] - ppm_im(sL[4], sR[4], s6[4], sig1);
      d1a = ref[TV1] - ppm_im(sL[TV1], sR[TV1], s6[TV1], sig1);
      d1b = ref[TV2] - ppm_im(sL[TV2], sR[TV2], s6[TV2], sig1);
    }
    const R bp = (d2p + rc * d2n) * hc2;
    const R b0 = d1r - d1p * ic2;
    qm[0] = ref[0] - b0 - bp;
    qm[NV] = ref[NV] - cor * bp;
    qm[TV1] = ref[TV1] - d1a;
    qm[TV2] = ref[TV2] - d1b;
    qm[4] = ref[4] - c2 * bp;
  }
  // ---- half-step sources from cell-centre values, then floors
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const R add = src.hdtp * g3[d] - src.src_u * s[1 + d][2];
    qp[1 + d] = qp[1 + d] + add;
    qm[1 + d] = qm[1 + d] + add;
  }
  qp[4] = qp[4] - src.src_p * pr;
  qm[4] = qm[4] - src.src_p * pr;
  if (qp[0] < E.small_dens) qp[0] = E.small_dens;
  if (qm[0] < E.small_dens) qm[0] = E.small_dens;
  if (qp[4] < E.small_pres) qp[4] = E.small_pres;
  if (qm[4] < E.small_pres) qm[4] = E.small_pres;
}

// ---------------------------------------------------------------- Riemann
// Two-shock approximate Riemann solver (Colella & Glaz 1985, named in
// Sec. 3.2): Newton iteration on u*_R(p) = u*_L(p) along the two shock
// curves, then sampling at x/t = 0 with a linear fan across rarefactions.
template <class R>
__device__ __forceinline__ R shock_w(const Eos<R> &E, R C, R ps, R p) {
  R x = R(1) + E.kshock * (p - ps) / ps;
  if (x < R(1e-10)) x = R(1e-10);
  return C * sqrt_r(x);
}

// Godunov state (rho, u_n, u_t1, u_t2, p) sampled from side o.
template <class R>
__device__ __forceinline__ void sample_side(const Eos<R> &E, R ro, R uo, R t1o, R t2o, R po, R Wo,
                                            R co, R s, R pstar, R ustar, R (&g)[5]) {
  // star density across the shock curve, or from dp = c^2 d rho (linearised)
  R rhos = E.linear ? ro + (pstar - po) / (co * co)
                    : R(1) / (R(1) / ro - (pstar - po) / (Wo * Wo));
  if (rhos < E.small_dens) rhos = E.small_dens;
  R cs = sqrt_r(E.gamma * pstar / rhos);
  int star;
  R w = R(-1);
  if (pstar > po) {
    R S = uo - s * (Wo / ro);
    star = (s * S < R(0)) ? 1 : 0;
  } else {
    R H = uo - s * co;
    R T = ustar - s * cs;
    if (s * H >= R(0)) {
      star = 0;
    } else if (s * T < R(0)) {
      star = 1;
    } else {
      star = 2;
      w = (R(0) - H) / (T - H);
    }
  }
  if (star == 0) {
    g[0] = ro;
    g[1] = uo;
    g[4] = po;
  } else if (star == 1) {
    g[0] = rhos;
    g[1] = ustar;
    g[4] = pstar;
  } else {
    g[0] = (R(1) - w) * ro + w * rhos;
    g[1] = (R(1) - w) * uo + w * ustar;
    g[4] = (R(1) - w) * po + w * pstar;
  }
  g[2] = t1o;
  g[3] = t2o;
}

// Normal-frame solve.  out = (F_rho, F_mn, F_mt1, F_mt2, F_rhoE, F_rhoe, u_g, p_g).
template <class R>
__device__ __forceinline__ void riemann(const Eos<R> &E, const R (&qL)[5], const R (&qR)[5],
                                        R (&out)[8]) {
  const R cL = sqrt_r(E.gamma * qL[4] / qL[0]);
  const R cR = sqrt_r(E.gamma * qR[4] / qR[0]);
  const R CL = qL[0] * cL;
  const R CR = qR[0] * cR;
  const R pL = qL[4], pR = qR[4], uL = qL[1], uR = qR[1];
  R p = (CR * pL + CL * pR + CL * CR * (uL - uR)) / (CL + CR);
  if (p < E.small_pres) p = E.small_pres;
  // the linearised solver stops at this acoustic estimate (W = C)
  for (int it = 0; it < (E.linear ? 0 : E.max_iter); ++it) {
    R WL = shock_w(E, CL, pL, p);
    R WR = shock_w(E, CR, pR, p);
    R usL = uL - (p - pL) / WL;
    R usR = uR + (p - pR) / WR;
    R ZL = R(2) * WL * WL * WL / (WL * WL + CL * CL);
    R ZR = R(2) * WR * WR * WR / (WR * WR + CR * CR);
    R pn = p - ZL * ZR * (usR - usL) / (ZL + ZR);
    if (pn < E.small_pres) pn = E.small_pres;
    bool conv = rabs(pn - p) <= E.tol * pn;
    p = pn;
    if (conv) break;
  }
  const R WL = E.linear ? CL : shock_w(E, CL, pL, p);
  const R WR = E.linear ? CR : shock_w(E, CR, pR, p);
  const R ustar = (pL - pR + WL * uL + WR * uR) / (WL + WR);
  const R pstar = p;
  R g[5];
  if (ustar > R(0)) {
    sample_side(E, qL[0], qL[1], qL[2], qL[3], qL[4], WL, cL, R(1), pstar, ustar, g);
  } else if (ustar < R(0)) {
    sample_side(E, qR[0], qR[1], qR[2], qR[3], qR[4], WR, cR, R(-1), pstar, ustar, g);
  } else {
    R gl[5], gr[5];
    sample_side(E, qL[0], qL[1], qL[2], qL[3], qL[4], WL, cL, R(1), pstar, ustar, gl);
    sample_side(E, qR[0], qR[1], qR[2], qR[3], qR[4], WR, cR, R(-1), pstar, ustar, gr);
#pragma unroll
    for (int v = 0; v < 5; ++v) g[v] = R(0.5) * (gl[v] + gr[v]);
  }
  if (g[0] < E.small_dens) g[0] = E.small_dens;
  if (g[4] < E.small_pres) g[4] = E.small_pres;
  const R rg = g[0], ug = g[1], t1 = g[2], t2 = g[3], pg = g[4];
  const R frho = rg * ug;
  const R rhoeg = pg * E.igm1;
  const R ke = R(0.5) * rg * (ug * ug + t1 * t1 + t2 * t2);
  out[0] = frho;
  out[1] = frho * ug + pg;
  out[2] = frho * t1;
  out[3] = frho * t2;
  out[4] = ug * (rhoeg + ke + pg);
  out[5] = ug * rhoeg;
  out[6] = ug;
  out[7] = pg;
}

// FP32 Godunov state sampled from side o (sign s = +1 for the left side, -1
// for the right one), written with selects instead of branches: every lane
// forms the shock and the rarefaction quantities and picks its case, so a
// warp whose faces meet different wave patterns does not split.
__device__ __forceinline__ void sample_side_fast(const Eos<float> &E, float ro, float iro, float uo,
                                                 float t1o, float t2o, float po, float Wo, float iWo,
                                                 float co, float s, float pstar, float ustar,
                                                 float (&g)[5]) {
  const float d = E.linear ? 1.0f / (ro + (pstar - po) / (co * co)) : iro - (pstar - po) * (iWo * iWo);
  const float rq = 1.0f / d;
  const bool low = !(rq >= E.small_dens);
  const float rhos = low ? E.small_dens : rq;
  const float ird = low ? 1.0f / E.small_dens : d;
  const float cs2 = E.gamma * pstar * ird;
  const float cs = cs2 * rsqrtf(cs2);
  const bool shock = pstar > po;
  const float S = uo - s * (Wo * iro);
  const float H = uo - s * co;
  const float T = ustar - s * cs;
  const bool side_r = s * H >= 0.0f;     // rarefaction: head moving away
  const bool star_r = s * T < 0.0f;      // rarefaction: tail moving away
  const bool star = shock ? (s * S < 0.0f) : (!side_r && star_r);
  const bool fan = !shock && !side_r && !star_r;
  const float w = H / (H - T);
  const float lr = (1.0f - w) * ro + w * rhos;
  const float lu = (1.0f - w) * uo + w * ustar;
  const float lp = (1.0f - w) * po + w * pstar;
  g[0] = fan ? lr : (star ? rhos : ro);
  g[1] = fan ? lu : (star ? ustar : uo);
  g[4] = fan ? lp : (star ? pstar : po);
  g[2] = t1o;
  g[3] = t2o;
}

// The same two-shock solve for the FP32 path, written with reciprocals and
// reciprocal square roots (MUFU) instead of divisions and square roots.  With
// x = max(1 + K (p - p_s)/p_s, 1e-10) and r = x^{-1/2}: W = C x r, 1/W = r/C,
// and the Newton slope 1/Z = (W^2 + C^2)/(2 W^3) = (x + 1) r^3 / (2 C).  Each
// lane leaves the Newton loop when it has converged: the lanes that are done
// go on to sample while the others iterate, which hides the loop's latency
// better than holding the whole warp to its slowest lane.
__device__ __forceinline__ void riemann_fast(const Eos<float> &E, const float (&qL)[5],
                                             const float (&qR)[5], float (&out)[8]) {
  const float iRL = 1.0f / qL[0], iRR = 1.0f / qR[0];
  const float c2L = E.gamma * qL[4] * iRL, c2R = E.gamma * qR[4] * iRR;
  const float cL = c2L * rsqrtf(c2L), cR = c2R * rsqrtf(c2R);
  const float CL = qL[0] * cL, CR = qR[0] * cR;
  const float iCL = 1.0f / CL, iCR = 1.0f / CR;
  const float pL = qL[4], pR = qR[4], uL = qL[1], uR = qR[1];
  const float kL = E.kshock / pL, kR = E.kshock / pR;
  float p = (CR * pL + CL * pR + CL * CR * (uL - uR)) / (CL + CR);
  if (p < E.small_pres) p = E.small_pres;
  for (int it = 0; it < (E.linear ? 0 : E.max_iter); ++it) {
    const float xL = fmaxf(1.0f + (p - pL) * kL, 1e-10f);
    const float xR = fmaxf(1.0f + (p - pR) * kR, 1e-10f);
    const float rL = rsqrtf(xL), rR = rsqrtf(xR);
    const float usL = uL - (p - pL) * (rL * iCL);
    const float usR = uR + (p - pR) * (rR * iCR);
    const float izL = (xL + 1.0f) * (rL * rL * rL) * (0.5f * iCL);
    const float izR = (xR + 1.0f) * (rR * rR * rR) * (0.5f * iCR);
    float pn = p - (usR - usL) / (izL + izR);
    if (pn < E.small_pres) pn = E.small_pres;
    const bool conv = fabsf(pn - p) <= E.tol * pn;
    p = pn;
    if (conv) break;
  }
  // final wave speeds W = C sqrt(x), x = 1 for the linearised solver (W = C)
  const float xL = E.linear ? 1.0f : fmaxf(1.0f + (p - pL) * kL, 1e-10f);
  const float xR = E.linear ? 1.0f : fmaxf(1.0f + (p - pR) * kR, 1e-10f);
  const float rL = E.linear ? 1.0f : rsqrtf(xL), rR = E.linear ? 1.0f : rsqrtf(xR);
  const float WL = CL * xL * rL, WR = CR * xR * rR;
  const float ustar = (pL - pR + WL * uL + WR * uR) / (WL + WR);
  const float pstar = p;
  float g[5];
  {
    // upwind side: left for u* >= 0 (u* = 0 also samples the right side below)
    const bool rs = ustar < 0.0f;
    sample_side_fast(E, rs ? qR[0] : qL[0], rs ? iRR : iRL, rs ? qR[1] : qL[1],
                     rs ? qR[2] : qL[2], rs ? qR[3] : qL[3], rs ? qR[4] : qL[4], rs ? WR : WL,
                     rs ? rR * iCR : rL * iCL, rs ? cR : cL, rs ? -1.0f : 1.0f, pstar, ustar, g);
    if (ustar == 0.0f) {
      float gr[5];
      sample_side_fast(E, qR[0], iRR, qR[1], qR[2], qR[3], qR[4], WR, rR * iCR, cR, -1.0f,
                       pstar, ustar, gr);
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v] = 0.5f * (g[v] + gr[v]);
    }
  }
  if (g[0] < E.small_dens) g[0] = E.small_dens;
  if (g[4] < E.small_pres) g[4] = E.small_pres;
  const float rg = g[0], ug = g[1], t1 = g[2], t2 = g[3], pg = g[4];
  const float frho = rg * ug;
  const float rhoeg = pg * E.igm1;
  const float ke = 0.5f * rg * (ug * ug + t1 * t1 + t2 * t2);
  out[0] = frho;
  out[1] = frho * ug + pg;
  out[2] = frho * t1;
  out[3] = frho * t2;
  out[4] = ug * (rhoeg + ke + pg);
  out[5] = ug * rhoeg;
  out[6] = ug;
  out[7] = pg;
}

// Tangential axes of face direction DIR, increasing order.
template <int DIR>
struct Tan {
  static constexpr int t1 = (DIR == 0) ? 1 : 0;
  static constexpr int t2 = (DIR == 2) ? 1 : 2;
};

// Lab-frame face flux: F = (F_rho, F_mx, F_my, F_mz, F_rhoE, F_rhoe, u_g, p_g).
template <class R, int DIR>
__device__ __forceinline__ void face_flux(const Eos<R> &E, const R (&qLl)[5], const R (&qRl)[5],
                                          R (&F)[8]) {
  constexpr int T1 = Tan<DIR>::t1, T2 = Tan<DIR>::t2;
  R qL[5] = {qLl[0], qLl[1 + DIR], qLl[1 + T1], qLl[1 + T2], qLl[4]};
  R qR[5] = {qRl[0], qRl[1 + DIR], qRl[1 + T1], qRl[1 + T2], qRl[4]};
  R o[8];
  if constexpr (sizeof(R) == 4)
    riemann_fast(E, qL, qR, o);
  else
    riemann(E, qL, qR, o);
  F[0] = o[0];
  F[1 + DIR] = o[1];
  F[1 + T1] = o[2];
  F[1 + T2] = o[3];
  F[4] = o[4];
  F[5] = o[5];
  F[6] = o[6];
  F[7] = o[7];
}

// ---------------------------------------------------------------- corner coupling
// Transverse correction of an edge state from cell C by the Godunov data on
// C's two faces normal to t (full corner coupling, Saltzman 1994, named in
// Sec. 3.2), in (rho, m, rho e) with the p div U term; the corrected state is
// dropped for the uncorrected one if its density falls below the floor.
// Flux records used here hold 7 numbers: (F_rho, F_mx, F_my, F_mz, F_rhoe, u_g, p_g).
template <class R>
struct TFlux {
  R f[7];
};

template <class R>
__device__ __forceinline__ TFlux<R> tflux_of(const R (&F)[8]) {
  TFlux<R> t;
  t.f[0] = F[0];
  t.f[1] = F[1];
  t.f[2] = F[2];
  t.f[3] = F[3];
  t.f[4] = F[5];
  t.f[5] = F[6];
  t.f[6] = F[7];
  return t;
}

template <class R>
__device__ __forceinline__ R rhoe_flux_diff(const TFlux<R> &Fp, const TFlux<R> &Fm) {
  return (Fp.f[4] - Fm.f[4]) + R(0.5) * (Fp.f[6] + Fm.f[6]) * (Fp.f[5] - Fm.f[5]);
}

template <class R>
__device__ __forceinline__ void transverse1(const Eos<R> &E, const R (&q)[5], R cdt, const TFlux<R> &Fp,
                                            const TFlux<R> &Fm, R (&out)[5]) {
  const R rho = q[0];
  R m0 = rho * q[1], m1 = rho * q[2], m2 = rho * q[3];
  const R rhoe = q[4] * E.igm1;
  R rn = rho - cdt * (Fp.f[0] - Fm.f[0]);
  m0 = m0 - cdt * (Fp.f[1] - Fm.f[1]);
  m1 = m1 - cdt * (Fp.f[2] - Fm.f[2]);
  m2 = m2 - cdt * (Fp.f[3] - Fm.f[3]);
  R en = rhoe - cdt * rhoe_flux_diff(Fp, Fm);
  if constexpr (sizeof(R) == 4) {
    const bool bad = rn < E.small_dens;
    const R irn = R(1) / rn;
    R p = E.gm1 * en;
    if (p < E.small_pres) p = E.small_pres;
    out[0] = bad ? q[0] : rn;
    out[1] = bad ? q[1] : m0 * irn;
    out[2] = bad ? q[2] : m1 * irn;
    out[3] = bad ? q[3] : m2 * irn;
    out[4] = bad ? q[4] : p;
    return;
  }
  if (rn < E.small_dens) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = q[v];
    return;
  }
  out[0] = rn;
  if constexpr (sizeof(R) == 4) {
    const R irn = R(1) / rn;
    out[1] = m0 * irn;
    out[2] = m1 * irn;
    out[3] = m2 * irn;
  } else {
    out[1] = m0 / rn;
    out[2] = m1 / rn;
    out[3] = m2 / rn;
  }
  R p = E.gm1 * en;
  if (p < E.small_pres) p = E.small_pres;
  out[4] = p;
}

template <class R>
__device__ __forceinline__ void transverse2(const Eos<R> &E, const R (&q)[5], R c1, const TFlux<R> &Ap,
                                            const TFlux<R> &Am, R c2, const TFlux<R> &Bp,
                                            const TFlux<R> &Bm, R (&out)[5]) {
  const R rho = q[0];
  R m0 = rho * q[1], m1 = rho * q[2], m2 = rho * q[3];
  const R rhoe = q[4] * E.igm1;
  R rn = rho - c1 * (Ap.f[0] - Am.f[0]);
  m0 = m0 - c1 * (Ap.f[1] - Am.f[1]);
  m1 = m1 - c1 * (Ap.f[2] - Am.f[2]);
  m2 = m2 - c1 * (Ap.f[3] - Am.f[3]);
  R en = rhoe - c1 * rhoe_flux_diff(Ap, Am);
  rn = rn - c2 * (Bp.f[0] - Bm.f[0]);
  m0 = m0 - c2 * (Bp.f[1] - Bm.f[1]);
  m1 = m1 - c2 * (Bp.f[2] - Bm.f[2]);
  m2 = m2 - c2 * (Bp.f[3] - Bm.f[3]);
  en = en - c2 * rhoe_flux_diff(Bp, Bm);
  if constexpr (sizeof(R) == 4) {
    const bool bad = rn < E.small_dens;
    const R irn = R(1) / rn;
    R p = E.gm1 * en;
    if (p < E.small_pres) p = E.small_pres;
    out[0] = bad ? q[0] : rn;
    out[1] = bad ? q[1] : m0 * irn;
    out[2] = bad ? q[2] : m1 * irn;
    out[3] = bad ? q[3] : m2 * irn;
    out[4] = bad ? q[4] : p;
    return;
  }
  if (rn < E.small_dens) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = q[v];
    return;
  }
  out[0] = rn;
  if constexpr (sizeof(R) == 4) {
    const R irn = R(1) / rn;
    out[1] = m0 * irn;
    out[2] = m1 * irn;
    out[3] = m2 * irn;
  } else {
    out[1] = m0 / rn;
    out[2] = m1 / rn;
    out[3] = m2 / rn;
  }
  R p = E.gm1 * en;
  if (p < E.small_pres) p = E.small_pres;
  out[4] = p;
}

}  // namespace NYX_NS
