/*
 * nyx_oracle.c -- TEST INFRASTRUCTURE, not product code.
 *
 * A plain FP64 CPU restatement of the single-level comoving gas advance of
 * the Nyx paper (Almgren et al. 2013).  It follows the scheme stage by stage,
 * one loop nest per stage over whole boxes, in the order the method states
 * it; nothing is fused, blocked or reordered.  Every expression is written in
 * one fixed form and evaluated left to right; the library is compiled with
 * -ffp-contract=off so no multiply-add is fused.
 *
 * Where the paper names a method but does not spell it out (PPM limiter,
 * tracing, two-shock solver, corner coupling) the standard published form is
 * restated here; each such reading is marked "reading:".
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this code.
 */
#include "nyx_oracle.h"

#include <math.h>
#include <omp.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* Two-shock solve statistics (calls, Newton iterations), one cache-line
 * slot per OpenMP thread; read by orc_riemann_counts. */
#define ORC_MAX_THREADS 512
static long long orc_rcount[ORC_MAX_THREADS * 8][2];

#define SIXTH (1.0 / 6.0)
#define TWO_THIRDS (2.0 / 3.0)
#define THIRD (1.0 / 3.0)

/* Derived constants of the gamma-law EOS, Sec. 2.2: p = (gamma-1) rho e. */
typedef struct {
  double gamma, gm1, igm1, kshock, small_dens, small_pres, tol;
  int max_iter;
  int plm, linear;  /* PLM profiles; linearised Riemann solver */
} eos_t;

static eos_t make_eos(const orc_params *p) {
  eos_t e;
  e.gamma = p->gamma;
  e.gm1 = p->gamma - 1.0;
  e.igm1 = 1.0 / e.gm1;
  e.kshock = (p->gamma + 1.0) / (2.0 * p->gamma);
  e.small_dens = p->small_dens;
  e.small_pres = p->small_pres;
  e.tol = p->riemann_tol;
  e.max_iter = p->riemann_max_iter;
  e.plm = p->reconstruction == 1;
  e.linear = p->riemann_solver == 1;
  return e;
}

/* ------------------------------------------------------------------ */
/* PPM reconstruction with limiting (Sec. 3.2; Colella & Woodward 1984).
 * reading: van Leer / MC-limited slopes, fourth-order interface values,
 * then the CW84 monotonicity constraint on each parabola.  s[0..4] holds
 * s_{i-2} .. s_{i+2}. */
static double mc_slope(double sm, double s0, double sp) {
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

static double interface_value(double s0, double s1, double d0, double d1) {
  /* s_{i+1/2} = (s_i + s_{i+1})/2 - (ds_{i+1} - ds_i)/6 */
  return 0.5 * (s0 + s1) - (d1 - d0) * SIXTH;
}

static void ppm_coeffs(const double s[5], double *sLo, double *sRo, double *s6o) {
  double dm = mc_slope(s[0], s[1], s[2]);
  double d0 = mc_slope(s[1], s[2], s[3]);
  double dp = mc_slope(s[2], s[3], s[4]);
  double sL = interface_value(s[1], s[2], dm, d0);
  double sR = interface_value(s[2], s[3], d0, dp);
  double si = s[2];
  if ((sR - si) * (si - sL) <= 0.0) {
    sL = si;
    sR = si;
  } else {
    double D = sR - sL;
    double M = si - 0.5 * (sL + sR);
    if (D * M > D * D * SIXTH) {
      sL = 3.0 * si - 2.0 * sR;
    } else if (-(D * D * SIXTH) > D * M) {
      sR = 3.0 * si - 2.0 * sL;
    }
  }
  *sLo = sL;
  *sRo = sR;
  *s6o = 6.0 * (si - 0.5 * (sL + sR));
}

/* PLM (Sec. 3.2, the piecewise linear option): the linear profile with the
 * MC-limited slope d of the cell, written in the parabola's coefficients --
 * edge values s_i -+ d/2 and no curvature -- so that the integrals below
 * are the averages of the linear profile.  reading: the plain MC slope (the
 * PPM slope of cell i), not a fourth-order slope. */
static void plm_coeffs(const double s[5], double *sLo, double *sRo, double *s6o) {
  double d = mc_slope(s[1], s[2], s[3]);
  *sLo = s[2] - 0.5 * d;
  *sRo = s[2] + 0.5 * d;
  *s6o = 0.0;
}

/* Average of the parabola over the sigma-fraction of the cell next to the
 * right (Ip) or left (Im) edge. */
static double ppm_ip(double sL, double sR, double s6, double sig) {
  return sR - 0.5 * sig * ((sR - sL) - (1.0 - TWO_THIRDS * sig) * s6);
}
static double ppm_im(double sL, double sR, double s6, double sig) {
  return sL + 0.5 * sig * ((sR - sL) + (1.0 - TWO_THIRDS * sig) * s6);
}

/* ------------------------------------------------------------------ */
/* Shock flattening (Colella & Woodward 1984; the PPM that Sec. 3.2 cites).
 * reading: along each direction d, a cell is inside a shock when the
 * pressure differs across it (cells i-1, i+1) by more than eps times the
 * smaller of the two pressures and the flow converges there
 * (u_d(i-1) > u_d(i+1)).  The shock's steepness is the ratio z of that
 * pressure difference to the one across cells i-2, i+2 (the latter not
 * below the pressure floor): a jump spread over one cell gives z near 1,
 * smooth data z near 1/2.  chi = clamp(omega2 (z - omega1), 0, 1) inside
 * a shock, 0 outside.  A cell's flattening along d is the larger chi of
 * itself and its neighbour on the low-pressure side (the side the shock
 * moves into; the right-hand one when both pressures are equal).  The
 * cell's coefficient is 1 minus its largest flattening over the three
 * directions; each profile of the cell is pulled toward the cell value by
 * it (edge values s_c + f (s_edge - s_c), curvature f s6).  Constants of
 * CW84: eps = 0.33, omega1 = 0.75, omega2 = 10. */
#define FLAT_EPS 0.33
#define FLAT_OMEGA1 0.75
#define FLAT_OMEGA2 10.0

/* chi of the cell at pr[0], u[0]; neighbours at multiples of stride s */
static double shock_chi(const double *pr, const double *u, ptrdiff_t s, double small_pres) {
  double dp1 = pr[s] - pr[-s];
  double dp2 = pr[2 * s] - pr[-2 * s];
  double lo = (pr[s] < pr[-s]) ? pr[s] : pr[-s];
  if (!(fabs(dp1) > FLAT_EPS * lo)) return 0.0;
  if (!(u[-s] - u[s] > 0.0)) return 0.0;
  double den = fabs(dp2);
  if (den < small_pres) den = small_pres;
  double z = fabs(dp1) / den;
  double w = FLAT_OMEGA2 * (z - FLAT_OMEGA1);
  if (w < 0.0) w = 0.0;
  if (w > 1.0) w = 1.0;
  return w;
}

/* flattening along one direction (needs pr at -3..3, u at -2..2) */
static double flat_dir(const double *pr, const double *u, ptrdiff_t s, double small_pres) {
  double chi0 = shock_chi(pr, u, s, small_pres);
  ptrdiff_t t = (pr[s] - pr[-s] > 0.0) ? -s : s;
  double chin = shock_chi(pr + t, u + t, s, small_pres);
  return (chi0 > chin) ? chi0 : chin;
}

/* ------------------------------------------------------------------ */
/* Characteristic tracing with a reference state (Sec. 3.2): the reference
 * is the average of the parabola over the domain of dependence of the
 * fastest wave moving toward the face (the edge value if it moves away);
 * the remaining waves moving toward the face are projected with the
 * eigenvectors of the primitive system at the cell centre.  reading: the
 * paper states this for PLM; it is used with PPM here.
 *
 * s5[v][o]: variable v in (rho, u_x, u_y, u_z, p), offset o = 0..4 for
 * cells i-2..i+2 along direction dir.  Half-step sources from the
 * primitive form of the comoving equations (Sec. 2.2) are added to both
 * edge states: gravity g/a and the expansion drag -(adot/a)U on every
 * velocity component, -3(gamma-1)(adot/a)p on pressure. */
typedef struct {
  double hdtp;  /* dt'/2, dt' = dt/a_half */
  double src_u; /* (a_new - a_old)/a_half / 2 */
  double src_p; /* 3 (gamma-1) (a_new - a_old)/a_half / 2 */
} trace_src_t;

static void trace_cell(const eos_t *E, double s5[5][5], double c, const double g3[3],
                       double dtdx, const trace_src_t *src, double fl, int dir, double qm[5],
                       double qp[5], double bm_out[3], double bp_out[3]) {
  double sL[5], sR[5], s6[5];
  for (int v = 0; v < 5; ++v) {
    if (E->plm)
      plm_coeffs(s5[v], &sL[v], &sR[v], &s6[v]);
    else
      ppm_coeffs(s5[v], &sL[v], &sR[v], &s6[v]);
  }
  /* shock flattening: fl = 1 leaves the profiles as they are */
  if (fl < 1.0)
    for (int v = 0; v < 5; ++v) {
      double si = s5[v][2];
      sL[v] = fl * sL[v] + (1.0 - fl) * si;
      sR[v] = fl * sR[v] + (1.0 - fl) * si;
      s6[v] = fl * s6[v];
    }
  const int nv = 1 + dir;
  const double rho = s5[0][2];
  const double un = s5[nv][2];
  const double pr = s5[4][2];
  double lam[3], sig[3];
  lam[0] = un - c;
  lam[1] = un;
  lam[2] = un + c;
  for (int k = 0; k < 3; ++k) sig[k] = fabs(lam[k]) * dtdx;
  const double c2 = c * c;
  const double ic2 = 1.0 / c2;
  const double hc2 = 0.5 * ic2;
  const double rc = rho * c;
  const double cor = c / rho;

  for (int side = 0; side < 2; ++side) {
    /* side 0: high face i+1/2 (waves with lam > 0 reach it);
     * side 1: low face i-1/2 (waves with lam < 0 reach it). */
    double ref[5], dq[3][5];
    for (int v = 0; v < 5; ++v) {
      if (side == 0)
        ref[v] = (lam[2] > 0.0) ? ppm_ip(sL[v], sR[v], s6[v], sig[2]) : sR[v];
      else
        ref[v] = (lam[0] < 0.0) ? ppm_im(sL[v], sR[v], s6[v], sig[0]) : sL[v];
    }
    for (int k = 0; k < 3; ++k) {
      int moving = (side == 0) ? (lam[k] > 0.0) : (lam[k] < 0.0);
      for (int v = 0; v < 5; ++v) {
        if (moving)
          dq[k][v] = ref[v] - ((side == 0) ? ppm_ip(sL[v], sR[v], s6[v], sig[k])
                                           : ppm_im(sL[v], sR[v], s6[v], sig[k]));
        else
          dq[k][v] = 0.0;
      }
    }
    /* wave amplitudes: beta_- (u-c), beta_0 (entropy / shear), beta_+ (u+c) */
    double bm = (dq[0][4] - rc * dq[0][nv]) * hc2;
    double bp = (dq[2][4] + rc * dq[2][nv]) * hc2;
    double b0 = dq[1][0] - dq[1][4] * ic2;
    double *q = (side == 0) ? qp : qm;
    q[0] = ref[0] - bm - b0 - bp;
    for (int v = 1; v <= 3; ++v) {
      if (v == nv)
        q[v] = ref[v] - cor * (bp - bm);
      else
        q[v] = ref[v] - dq[1][v];
    }
    q[4] = ref[4] - c2 * (bm + bp);
    double *bo = (side == 0) ? bp_out : bm_out;
    if (bo) {
      bo[0] = bm;
      bo[1] = b0;
      bo[2] = bp;
    }
    /* half-step sources, cell-centre values */
    for (int d = 0; d < 3; ++d) q[1 + d] = q[1 + d] + (src->hdtp * g3[d] - src->src_u * s5[1 + d][2]);
    q[4] = q[4] - src->src_p * pr;
    if (q[0] < E->small_dens) q[0] = E->small_dens;
    if (q[4] < E->small_pres) q[4] = E->small_pres;
  }
}

/* ------------------------------------------------------------------ */
/* Two-shock approximate Riemann solver (Sec. 3.2; Colella & Glaz 1985).
 * reading: Newton iteration on u*_R(p) - u*_L(p) = 0 along the two shock
 * curves (W = Lagrangian shock speed, Z = |dp/du| on the curve), then the
 * Godunov state is sampled at x/t = 0 with a linear fan across
 * rarefactions.  States are (rho, u_n, u_t1, u_t2, p).  out[8] =
 * (F_rho, F_mn, F_mt1, F_mt2, F_rhoE, F_rhoe, u_g, p_g). */
static double shock_w(const eos_t *E, double C, double ps, double p) {
  double x = 1.0 + E->kshock * (p - ps) / ps;
  if (x < 1e-10) x = 1e-10;
  return C * sqrt(x);
}

static void sample_side(const eos_t *E, const double *qo, double Wo, double co, double s,
                        double pstar, double ustar, double g[5]) {
  /* star density: across the shock curve (two-shock), or from the
   * linearised relation dp = c^2 d rho (linearised solver) */
  double rhos = E->linear ? qo[0] + (pstar - qo[4]) / (co * co)
                          : 1.0 / (1.0 / qo[0] - (pstar - qo[4]) / (Wo * Wo));
  if (rhos < E->small_dens) rhos = E->small_dens;
  double cs = sqrt(E->gamma * pstar / rhos);
  int star;
  double w = -1.0;
  if (pstar > qo[4]) {
    double S = qo[1] - s * (Wo / qo[0]);
    star = (s * S < 0.0);
  } else {
    double H = qo[1] - s * co;
    double T = ustar - s * cs;
    if (s * H >= 0.0)
      star = 0;
    else if (s * T < 0.0)
      star = 1;
    else {
      star = 2;
      w = (0.0 - H) / (T - H);
    }
  }
  if (star == 0) {
    g[0] = qo[0];
    g[1] = qo[1];
    g[4] = qo[4];
  } else if (star == 1) {
    g[0] = rhos;
    g[1] = ustar;
    g[4] = pstar;
  } else {
    g[0] = (1.0 - w) * qo[0] + w * rhos;
    g[1] = (1.0 - w) * qo[1] + w * ustar;
    g[4] = (1.0 - w) * qo[4] + w * pstar;
  }
  g[2] = qo[2];
  g[3] = qo[3];
}

static void riemann_solve(const eos_t *E, const double *qL, const double *qR, double out[8],
                          double *pstar_o, double *ustar_o, double *g_o) {
  const double cL = sqrt(E->gamma * qL[4] / qL[0]);
  const double cR = sqrt(E->gamma * qR[4] / qR[0]);
  const double CL = qL[0] * cL;
  const double CR = qR[0] * cR;
  const double pL = qL[4], pR = qR[4], uL = qL[1], uR = qR[1];
  double p = (CR * pL + CL * pR + CL * CR * (uL - uR)) / (CL + CR);
  if (p < E->small_pres) p = E->small_pres;
  long long nit = 0;
  /* the linearised solver stops at the acoustic estimate: p* above, the
   * wave speeds the acoustic impedances C (no Newton iteration) */
  for (int it = 0; it < (E->linear ? 0 : E->max_iter); ++it) {
    double WL = shock_w(E, CL, pL, p);
    double WR = shock_w(E, CR, pR, p);
    double usL = uL - (p - pL) / WL;
    double usR = uR + (p - pR) / WR;
    double ZL = 2.0 * WL * WL * WL / (WL * WL + CL * CL);
    double ZR = 2.0 * WR * WR * WR / (WR * WR + CR * CR);
    double pn = p - ZL * ZR * (usR - usL) / (ZL + ZR);
    if (pn < E->small_pres) pn = E->small_pres;
    int conv = fabs(pn - p) <= E->tol * pn;
    p = pn;
    nit++;
    if (conv) break;
  }
  {
    int t = omp_get_thread_num();
    if (t < ORC_MAX_THREADS) {
      orc_rcount[t * 8][0] += 1;
      orc_rcount[t * 8][1] += nit;
    }
  }
  const double WL = E->linear ? CL : shock_w(E, CL, pL, p);
  const double WR = E->linear ? CR : shock_w(E, CR, pR, p);
  const double ustar = (pL - pR + WL * uL + WR * uR) / (WL + WR);
  const double pstar = p;
  double g[5];
  if (ustar > 0.0) {
    sample_side(E, qL, WL, cL, 1.0, pstar, ustar, g);
  } else if (ustar < 0.0) {
    sample_side(E, qR, WR, cR, -1.0, pstar, ustar, g);
  } else {
    double gl[5], gr[5];
    sample_side(E, qL, WL, cL, 1.0, pstar, ustar, gl);
    sample_side(E, qR, WR, cR, -1.0, pstar, ustar, gr);
    for (int v = 0; v < 5; ++v) g[v] = 0.5 * (gl[v] + gr[v]);
  }
  if (g[0] < E->small_dens) g[0] = E->small_dens;
  if (g[4] < E->small_pres) g[4] = E->small_pres;
  const double rg = g[0], ug = g[1], t1 = g[2], t2 = g[3], pg = g[4];
  const double frho = rg * ug;
  const double rhoeg = pg * E->igm1;
  const double ke = 0.5 * rg * (ug * ug + t1 * t1 + t2 * t2);
  out[0] = frho;
  out[1] = frho * ug + pg;
  out[2] = frho * t1;
  out[3] = frho * t2;
  out[4] = ug * (rhoeg + ke + pg);
  out[5] = ug * rhoeg;
  out[6] = ug;
  out[7] = pg;
  if (pstar_o) *pstar_o = pstar;
  if (ustar_o) *ustar_o = ustar;
  if (g_o)
    for (int v = 0; v < 5; ++v) g_o[v] = g[v];
}

/* Tangential axes of a face direction, in increasing order. */
static void tangential_axes(int dir, int *t1, int *t2) {
  *t1 = (dir == 0) ? 1 : 0;
  *t2 = (dir == 2) ? 1 : 2;
}

/* Godunov flux through a direction-dir face from lab-frame primitive
 * states; F8 = (F_rho, F_mx, F_my, F_mz, F_rhoE, F_rhoe, u_g, p_g). */
static void face_flux(const eos_t *E, int dir, const double *qLl, const double *qRl,
                      double F8[8]) {
  int t1, t2;
  tangential_axes(dir, &t1, &t2);
  double qL[5] = {qLl[0], qLl[1 + dir], qLl[1 + t1], qLl[1 + t2], qLl[4]};
  double qR[5] = {qRl[0], qRl[1 + dir], qRl[1 + t1], qRl[1 + t2], qRl[4]};
  double out[8];
  riemann_solve(E, qL, qR, out, NULL, NULL, NULL);
  F8[0] = out[0];
  F8[1 + dir] = out[1];
  F8[1 + t1] = out[2];
  F8[1 + t2] = out[3];
  F8[4] = out[4];
  F8[5] = out[5];
  F8[6] = out[6];
  F8[7] = out[7];
}

/* ------------------------------------------------------------------ */
/* Transverse (corner-coupling) correction of an edge state that came from
 * cell C by the Godunov data on C's two faces normal to t (Saltzman 1994
 * full corner coupling, as cited in Sec. 3.2).  reading: the update is done
 * on (rho, m, rho e), with the p div U term for rho e; if the corrected
 * density drops below the floor the uncorrected state is kept. */
static double rhoe_flux_diff(const double *Fp, const double *Fm) {
  return (Fp[5] - Fm[5]) + 0.5 * (Fp[7] + Fm[7]) * (Fp[6] - Fm[6]);
}

static void transverse_correct(const eos_t *E, const double q[5], int nterms,
                               const double *cdt, const double *const *Fp,
                               const double *const *Fm, double out[5]) {
  const double rho = q[0];
  double m[3];
  for (int k = 0; k < 3; ++k) m[k] = rho * q[1 + k];
  const double rhoe = q[4] * E->igm1;
  double rn = rho, en = rhoe, mn[3] = {m[0], m[1], m[2]};
  for (int t = 0; t < nterms; ++t) {
    rn = rn - cdt[t] * (Fp[t][0] - Fm[t][0]);
    for (int k = 0; k < 3; ++k) mn[k] = mn[k] - cdt[t] * (Fp[t][1 + k] - Fm[t][1 + k]);
    en = en - cdt[t] * rhoe_flux_diff(Fp[t], Fm[t]);
  }
  if (rn < E->small_dens) {
    for (int v = 0; v < 5; ++v) out[v] = q[v];
    return;
  }
  out[0] = rn;
  for (int k = 0; k < 3; ++k) out[1 + k] = mn[k] / rn;
  out[4] = E->gm1 * en;
  if (out[4] < E->small_pres) out[4] = E->small_pres;
}

/* ------------------------------------------------------------------ */
/* Box geometry helpers. */
typedef struct {
  int n[3], ng, N[3];
  size_t vol, st[3];
} geom_t;

static geom_t make_geom(const int lo[3], const int hi[3], int ng) {
  geom_t g;
  g.ng = ng;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = hi[d] - lo[d] + 1;
    g.N[d] = g.n[d] + 2 * ng;
  }
  g.st[0] = 1;
  g.st[1] = (size_t)g.N[0];
  g.st[2] = (size_t)g.N[0] * g.N[1];
  g.vol = g.st[2] * g.N[2];
  return g;
}

static size_t gidx(const geom_t *g, int i, int j, int k) {
  return ((size_t)(k + g->ng) * g->N[1] + (size_t)(j + g->ng)) * g->N[0] + (size_t)(i + g->ng);
}

/* ------------------------------------------------------------------ */
/* Ghost fill (Sec. 4.1: every grid carries the same number of ghost cells
 * on every side).  Each ghost cell takes the value of the valid cell that
 * covers the same point of its domain, after periodic wrapping; across an
 * outflow face the index is clamped to the last interior cell
 * (zero-gradient extrapolation; reading, the paper is silent). */
static int find_box(const orc_level *L, int dom, const int gi[3], int hint) {
  if (hint >= 0 && L->dom[hint] == dom) {
    const int *lo = L->lo + 3 * hint, *hi = L->hi + 3 * hint;
    if (gi[0] >= lo[0] && gi[0] <= hi[0] && gi[1] >= lo[1] && gi[1] <= hi[1] && gi[2] >= lo[2] &&
        gi[2] <= hi[2])
      return hint;
  }
  for (int b = 0; b < L->nbox; ++b) {
    if (L->dom[b] != dom) continue;
    const int *lo = L->lo + 3 * b, *hi = L->hi + 3 * b;
    if (gi[0] >= lo[0] && gi[0] <= hi[0] && gi[1] >= lo[1] && gi[1] <= hi[1] && gi[2] >= lo[2] &&
        gi[2] <= hi[2])
      return b;
  }
  return -1;
}

int orc_fill_ghosts(const orc_level *L, int ncomp, double *const *f) {
  int err = 0;
  for (int b = 0; b < L->nbox; ++b) {
    geom_t g = make_geom(L->lo + 3 * b, L->hi + 3 * b, L->ng);
    const int dom = L->dom[b];
    const int *dlo = L->dom_lo + 3 * dom, *dhi = L->dom_hi + 3 * dom, *bc = L->dom_bc + 6 * dom;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int k = -g.ng; k < g.n[2] + g.ng; ++k) {
      int hint = -1;
      for (int j = -g.ng; j < g.n[1] + g.ng; ++j)
        for (int i = -g.ng; i < g.n[0] + g.ng; ++i) {
          int loc[3] = {i, j, k};
          int inside = 1;
          for (int d = 0; d < 3; ++d)
            if (loc[d] < 0 || loc[d] >= g.n[d]) inside = 0;
          if (inside) continue;
          int gi[3];
          for (int d = 0; d < 3; ++d) {
            int x = L->lo[3 * b + d] + loc[d];
            int len = dhi[d] - dlo[d] + 1;
            if (x < dlo[d]) {
              if (bc[d] == ORC_BC_PERIODIC)
                x = dlo[d] + ((x - dlo[d]) % len + len) % len;
              else
                x = dlo[d];
            } else if (x > dhi[d]) {
              if (bc[3 + d] == ORC_BC_PERIODIC)
                x = dlo[d] + ((x - dlo[d]) % len + len) % len;
              else
                x = dhi[d];
            }
            gi[d] = x;
          }
          int sb = find_box(L, dom, gi, hint);
          if (sb < 0) {
            err = 1;
            continue;
          }
          hint = sb;
          geom_t gs = make_geom(L->lo + 3 * sb, L->hi + 3 * sb, L->ng);
          size_t src = gidx(&gs, gi[0] - L->lo[3 * sb], gi[1] - L->lo[3 * sb + 1],
                            gi[2] - L->lo[3 * sb + 2]);
          size_t dst = gidx(&g, i, j, k);
          for (int c = 0; c < ncomp; ++c) f[b][c * g.vol + dst] = f[sb][c * gs.vol + src];
        }
    }
  }
  return err ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Primitive variables (Sec. 2.2 EOS; Sec. 3.2: pressure from the evolved
 * internal energy).  q6 = (rho, u_x, u_y, u_z, p, c). */
static void primitives(const eos_t *E, const double *S, size_t vol, size_t id, double q6[6]) {
  double rho = S[id];
  q6[0] = rho;
  q6[1] = S[vol + id] / rho;
  q6[2] = S[2 * vol + id] / rho;
  q6[3] = S[3 * vol + id] / rho;
  double p = E->gm1 * S[5 * vol + id];
  if (p < E->small_pres) p = E->small_pres;
  q6[4] = p;
  q6[5] = sqrt(E->gamma * p / rho);
}

/* Loop helper over an inclusive 3-D range of local cell indices. */
#define RANGE_LOOP(lo, hi, ...)                                     \
  _Pragma("omp parallel for collapse(2) schedule(static)")          \
  for (int k = (lo)[2]; k <= (hi)[2]; ++k)                          \
    for (int j = (lo)[1]; j <= (hi)[1]; ++j)                        \
      for (int i = (lo)[0]; i <= (hi)[0]; ++i) { __VA_ARGS__ }

static double *alloc_arr(size_t n) { return (double *)calloc(n, sizeof(double)); }

/* One box, Steps 2 and 6 of the single-level algorithm (Sec. 3.6). */
/* Scalars of one step (Sec. 2.2, 3.6) used by the corrector. */
typedef struct {
  double a_old, a_new, dt, hdt, ian, ian2, eta_de, efloor;
} step_k;

/* Step 6 for one cell: the gravity corrector U^{n+1} = U^{n+1,*} + dt/2
 * (S_g^{n+1,*} - S_g^n) with g_old at t^n and g_new at t^{n+1} (when
 * P->grav_corrector), then the dual-energy synchronisation (when
 * P->dual_energy_sync).  rho, m: state at t^n; rho_s, ms, rE_s, re_s: the
 * predictor.  out = (rho, m_x, m_y, m_z, rhoE, rhoe) at t^{n+1}. */
static void finish_cell(const orc_params *P, const step_k *s, double rho, const double m[3],
                        const double go[3], const double gn[3], double rho_s, const double ms[3],
                        double rE_s, double re_s, double out[6], long long *n_use_e,
                        long long *n_floor) {
  double mn[3];
  double rEn = rE_s;
  if (P->grav_corrector) {
    for (int c = 0; c < 3; ++c) mn[c] = ms[c] + s->hdt * (rho_s * gn[c] - rho * go[c]) * s->ian;
    if (P->grav_energy) {
      double ks = ms[0] * ms[0] + ms[1] * ms[1] + ms[2] * ms[2];
      double kn = mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2];
      rEn = rE_s + 0.5 * (kn - ks) / rho_s;
    } else {
      double mg = m[0] * go[0] + m[1] * go[1] + m[2] * go[2];
      double msg = ms[0] * gn[0] + ms[1] * gn[1] + ms[2] * gn[2];
      rEn = rE_s + s->hdt * (s->a_new * msg - s->a_old * mg) * s->ian2;
    }
  } else {
    for (int c = 0; c < 3; ++c) mn[c] = ms[c];
  }
  double ren = re_s;
  if (P->dual_energy_sync) {
    double ke = 0.5 * (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) / rho_s;
    if (rEn - ke > s->eta_de * rEn) {
      ren = rEn - ke;
    } else {
      rEn = ren + ke;
      (*n_use_e)++;
    }
    if (ren < s->efloor) {
      ren = s->efloor;
      rEn = ren + ke;
      (*n_floor)++;
    }
  }
  out[0] = rho_s;
  for (int c = 0; c < 3; ++c) out[1 + c] = mn[c];
  out[4] = rEn;
  out[5] = ren;
}

static int advance_box(const eos_t *E, const orc_params *P, const int lo_[3], const int hi_[3],
                       int ng, const double dx[3], const double *S, double *Sn, const double *G,
                       double a_old, double a_new, double dt, double *flux_out[3],
                       orc_stats *st) {
  geom_t g = make_geom(lo_, hi_, ng);
  const size_t V = g.vol;
  const double a_half = 0.5 * (a_old + a_new);
  const double dtp = dt / a_half;
  trace_src_t src;
  const double adot = (a_new - a_old) / a_half;
  src.hdtp = 0.5 * dtp;
  src.src_u = 0.5 * adot;
  src.src_p = 1.5 * E->gm1 * adot;

  /* full extent and shrinking ranges, local coordinates */
  int L[3], H[3];
  for (int d = 0; d < 3; ++d) {
    L[d] = -ng;
    H[d] = g.n[d] + ng - 1;
  }

  /* O1 primitives on every cell */
  double *q = alloc_arr(6 * V);
  RANGE_LOOP(L, H, {
    size_t id = gidx(&g, i, j, k);
    double q6[6];
    primitives(E, S, V, id, q6);
    for (int v = 0; v < 6; ++v) q[v * V + id] = q6[v];
  })

  /* O1b shock-flattening coefficients on [-1, n] in every direction (the
   * cells whose edge states the valid faces use; their +-3 stencil is
   * inside the 4 ghost cells); 1 on the other cells */
  double *fl = NULL;
  if (P->flattening) {
    fl = alloc_arr(V);
    for (size_t t = 0; t < V; ++t) fl[t] = 1.0;
    int lo[3] = {-1, -1, -1}, hi[3] = {g.n[0], g.n[1], g.n[2]};
    RANGE_LOOP(lo, hi, {
      size_t id = gidx(&g, i, j, k);
      double f = 0.0;
      for (int d = 0; d < 3; ++d) {
        double fd = flat_dir(q + 4 * V + id, q + (size_t)(1 + d) * V + id, (ptrdiff_t)g.st[d],
                             E->small_pres);
        if (fd > f) f = fd;
      }
      fl[id] = 1.0 - f;
    })
  }

  /* O2+O3 PPM and tracing, direction d, where +-2 neighbours exist */
  double *qm[3], *qp[3];
  for (int d = 0; d < 3; ++d) {
    qm[d] = alloc_arr(5 * V);
    qp[d] = alloc_arr(5 * V);
    int lo[3] = {L[0], L[1], L[2]}, hi[3] = {H[0], H[1], H[2]};
    lo[d] += 2;
    hi[d] -= 2;
    const size_t s = g.st[d];
    const double dtdx = dtp / dx[d];
    double *qmd = qm[d], *qpd = qp[d];
    RANGE_LOOP(lo, hi, {
      size_t id = gidx(&g, i, j, k);
      double s5[5][5];
      for (int v = 0; v < 5; ++v)
        for (int o = 0; o < 5; ++o) s5[v][o] = q[v * V + id + (size_t)(o - 2) * s];
      double g3[3] = {0.0, 0.0, 0.0};
      if (G)
        for (int c = 0; c < 3; ++c) g3[c] = G[c * V + id];
      double a5[5], b5[5];
      trace_cell(E, s5, q[5 * V + id], g3, dtdx, &src, fl ? fl[id] : 1.0, d, a5, b5, NULL,
                 NULL);
      for (int v = 0; v < 5; ++v) {
        qmd[v * V + id] = a5[v];
        qpd[v * V + id] = b5[v];
      }
    })
  }

  /* O5.1 normal Riemann solves; face f-1/2 stored at cell f */
  double *Fn[3];
  for (int d = 0; d < 3; ++d) {
    Fn[d] = alloc_arr(8 * V);
    int lo[3] = {L[0], L[1], L[2]}, hi[3] = {H[0], H[1], H[2]};
    lo[d] += 3;
    hi[d] -= 2;
    const size_t s = g.st[d];
    double *F = Fn[d], *qpd = qp[d], *qmd = qm[d];
    RANGE_LOOP(lo, hi, {
      size_t id = gidx(&g, i, j, k);
      double ql[5], qr[5], f8[8];
      for (int v = 0; v < 5; ++v) {
        ql[v] = qpd[v * V + id - s];
        qr[v] = qmd[v * V + id];
      }
      face_flux(E, d, ql, qr, f8);
      for (int c = 0; c < 8; ++c) F[c * V + id] = f8[c];
    })
  }

  /* O5.2-3 singly corrected states q_{d|t}, theta = 1/3, and their solves */
  double *Ft[3][3] = {{NULL}};
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 3; ++t) {
      if (t == d) continue;
      double *tm = alloc_arr(5 * V), *tp = alloc_arr(5 * V);
      int lo[3] = {L[0], L[1], L[2]}, hi[3] = {H[0], H[1], H[2]};
      lo[d] += 2;
      hi[d] -= 2;
      lo[t] += 3;
      hi[t] -= 3;
      const size_t stt = g.st[t];
      const double cdt = dtp / (3.0 * dx[t]);
      double *F = Fn[t], *qmd = qm[d], *qpd = qp[d];
      RANGE_LOOP(lo, hi, {
        size_t id = gidx(&g, i, j, k);
        double fm[8], fp[8], a5[5], b5[5], o5[5];
        for (int c = 0; c < 8; ++c) {
          fm[c] = F[c * V + id];
          fp[c] = F[c * V + id + stt];
        }
        const double *Fp1[1] = {fp}, *Fm1[1] = {fm};
        double cd[1] = {cdt};
        for (int v = 0; v < 5; ++v) {
          a5[v] = qmd[v * V + id];
          b5[v] = qpd[v * V + id];
        }
        transverse_correct(E, a5, 1, cd, Fp1, Fm1, o5);
        for (int v = 0; v < 5; ++v) tm[v * V + id] = o5[v];
        transverse_correct(E, b5, 1, cd, Fp1, Fm1, o5);
        for (int v = 0; v < 5; ++v) tp[v * V + id] = o5[v];
      })
      /* F^{d|t} on d-faces */
      Ft[d][t] = alloc_arr(8 * V);
      int flo[3] = {lo[0], lo[1], lo[2]}, fhi[3] = {hi[0], hi[1], hi[2]};
      flo[d] += 1;
      const size_t sd = g.st[d];
      double *FF = Ft[d][t];
      RANGE_LOOP(flo, fhi, {
        size_t id = gidx(&g, i, j, k);
        double ql[5], qr[5], f8[8];
        for (int v = 0; v < 5; ++v) {
          ql[v] = tp[v * V + id - sd];
          qr[v] = tm[v * V + id];
        }
        face_flux(E, d, ql, qr, f8);
        for (int c = 0; c < 8; ++c) FF[c * V + id] = f8[c];
      })
      free(tm);
      free(tp);
    }
  for (int d = 0; d < 3; ++d) free(Fn[d]);

  /* O5.4 final states (theta = 1/2, both transverse directions in one
   * update, t1 terms first) and final solves */
  double *Ff[3];
  for (int d = 0; d < 3; ++d) {
    int t1, t2;
    tangential_axes(d, &t1, &t2);
    double *fm5 = alloc_arr(5 * V), *fp5 = alloc_arr(5 * V);
    int lo[3] = {L[0], L[1], L[2]}, hi[3] = {H[0], H[1], H[2]};
    lo[d] += 2;
    hi[d] -= 2;
    lo[t1] += 3;
    hi[t1] -= 3;
    lo[t2] += 3;
    hi[t2] -= 3;
    const size_t s1 = g.st[t1], s2 = g.st[t2];
    const double c1 = 0.5 * dtp / dx[t1], c2 = 0.5 * dtp / dx[t2];
    double *A = Ft[t1][t2], *B = Ft[t2][t1], *qmd = qm[d], *qpd = qp[d];
    RANGE_LOOP(lo, hi, {
      size_t id = gidx(&g, i, j, k);
      double am[8], ap[8], bm[8], bp[8], a5[5], b5[5], o5[5];
      for (int c = 0; c < 8; ++c) {
        am[c] = A[c * V + id];
        ap[c] = A[c * V + id + s1];
        bm[c] = B[c * V + id];
        bp[c] = B[c * V + id + s2];
      }
      const double *Fp2[2] = {ap, bp}, *Fm2[2] = {am, bm};
      double cd[2] = {c1, c2};
      for (int v = 0; v < 5; ++v) {
        a5[v] = qmd[v * V + id];
        b5[v] = qpd[v * V + id];
      }
      transverse_correct(E, a5, 2, cd, Fp2, Fm2, o5);
      for (int v = 0; v < 5; ++v) fm5[v * V + id] = o5[v];
      transverse_correct(E, b5, 2, cd, Fp2, Fm2, o5);
      for (int v = 0; v < 5; ++v) fp5[v * V + id] = o5[v];
    })
    Ff[d] = alloc_arr(8 * V);
    int flo[3] = {lo[0], lo[1], lo[2]}, fhi[3] = {hi[0], hi[1], hi[2]};
    flo[d] += 1;
    const size_t sd = g.st[d];
    double *FF = Ff[d];
    RANGE_LOOP(flo, fhi, {
      size_t id = gidx(&g, i, j, k);
      double ql[5], qr[5], f8[8];
      for (int v = 0; v < 5; ++v) {
        ql[v] = fp5[v * V + id - sd];
        qr[v] = fm5[v * V + id];
      }
      face_flux(E, d, ql, qr, f8);
      for (int c = 0; c < 8; ++c) FF[c * V + id] = f8[c];
    })
    free(fm5);
    free(fp5);
  }
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 3; ++t) free(Ft[d][t]);
  for (int d = 0; d < 3; ++d) {
    free(qm[d]);
    free(qp[d]);
  }
  free(q);
  free(fl);

  /* O6-O9 conservative update with comoving weights, gravity predictor
   * (Step 2) and corrector (Step 6), dual-energy sync (Step 6). */
  const double idx[3] = {1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2]};
  const double ao2 = a_old * a_old;
  const double an2 = a_new * a_new;
  const double ian = 1.0 / a_new;
  const double ian2 = 1.0 / an2;
  const double ahdt = a_half * dt;
  const double dta = dt * a_old;
  const double kappa = 2.0 - 3.0 * E->gm1;
  const double expn = a_half * (a_new - a_old) * kappa;
  const double hdt = 0.5 * dt;
  const double efloor = P->small_pres * E->igm1;
  const step_k sk = {a_old, a_new, dt, hdt, ian, ian2, P->eta_de, efloor};
  int vlo[3] = {0, 0, 0}, vhi[3] = {g.n[0] - 1, g.n[1] - 1, g.n[2] - 1};
  long long n_use_e = 0, n_floor = 0, n_bad = 0;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : n_use_e, n_floor, n_bad)
  for (int k = vlo[2]; k <= vhi[2]; ++k)
    for (int j = vlo[1]; j <= vhi[1]; ++j)
      for (int i = vlo[0]; i <= vhi[0]; ++i) {
        size_t id = gidx(&g, i, j, k);
        double div[6], pdivu = 0.0;
        for (int c = 0; c < 6; ++c) {
          double acc = 0.0;
          for (int d = 0; d < 3; ++d) {
            double t = (Ff[d][c * V + id + g.st[d]] - Ff[d][c * V + id]) * idx[d];
            acc = (d == 0) ? t : acc + t;
          }
          div[c] = acc;
        }
        for (int d = 0; d < 3; ++d) {
          const double *F = Ff[d];
          double t = 0.5 * (F[7 * V + id + g.st[d]] + F[7 * V + id]) *
                     (F[6 * V + id + g.st[d]] - F[6 * V + id]) * idx[d];
          pdivu = (d == 0) ? t : pdivu + t;
        }
        double rho = S[id];
        double m[3] = {S[V + id], S[2 * V + id], S[3 * V + id]};
        double rE = S[4 * V + id], re = S[5 * V + id];
        double gv[3] = {0.0, 0.0, 0.0};
        if (G)
          for (int c = 0; c < 3; ++c) gv[c] = G[c * V + id];
        /* predictor: U^{n+1,*} = U^n - dt div F + dt S_e + dt S_g^n */
        double rho_s = rho - dtp * div[0];
        double ms[3];
        for (int c = 0; c < 3; ++c) ms[c] = (a_old * m[c] - dt * div[1 + c] + dt * rho * gv[c]) * ian;
        double rE_s;
        if (P->grav_energy) {
          /* Sec. 3.2, second alternative: the gravity part of the energy
           * update is the change of the kinetic energy that the gravity part
           * of the momentum update makes (at the new density) */
          double mh[3];
          for (int c = 0; c < 3; ++c) mh[c] = (a_old * m[c] - dt * div[1 + c]) * ian;
          double kh = mh[0] * mh[0] + mh[1] * mh[1] + mh[2] * mh[2];
          double ks = ms[0] * ms[0] + ms[1] * ms[1] + ms[2] * ms[2];
          rE_s = (ao2 * rE - ahdt * div[4] + expn * re) * ian2 + 0.5 * (ks - kh) / rho_s;
        } else {
          double mg = m[0] * gv[0] + m[1] * gv[1] + m[2] * gv[2];
          rE_s = (ao2 * rE - ahdt * div[4] + dta * mg + expn * re) * ian2;
        }
        double re_s = (ao2 * re - ahdt * div[5] - ahdt * pdivu + expn * re) * ian2;
        /* corrector (Step 6) and dual-energy synchronisation */
        double out[6];
        finish_cell(P, &sk, rho, m, gv, gv, rho_s, ms, rE_s, re_s, out, &n_use_e, &n_floor);
        const double rEn = out[4], ren = out[5];
        double mn[3] = {out[1], out[2], out[3]};
        if (!(rho_s > 0.0) || !isfinite(rho_s) || !isfinite(rEn) || !isfinite(ren)) n_bad++;
        Sn[id] = rho_s;
        for (int c = 0; c < 3; ++c) Sn[(1 + c) * V + id] = mn[c];
        Sn[4 * V + id] = rEn;
        Sn[5 * V + id] = ren;
      }

  if (flux_out) {
    for (int d = 0; d < 3; ++d) {
      if (!flux_out[d]) continue;
      int e[3] = {g.n[0], g.n[1], g.n[2]};
      e[d] += 1;
      size_t fv = (size_t)e[0] * e[1] * e[2];
      double *o = flux_out[d];
      for (int c = 0; c < 6; ++c)
        for (int k = 0; k < e[2]; ++k)
          for (int j = 0; j < e[1]; ++j)
            for (int i = 0; i < e[0]; ++i)
              o[c * fv + ((size_t)k * e[1] + j) * e[0] + i] = Ff[d][c * V + gidx(&g, i, j, k)];
    }
  }
  for (int d = 0; d < 3; ++d) free(Ff[d]);
  if (st) {
    st->use_e += n_use_e;
    st->floor_e += n_floor;
    st->bad += n_bad;
  }
  return n_bad ? -3 : 0;
}

int orc_advance(const orc_level *L, const orc_params *P, double *const *state_in,
                double *const *state_out, double *const *grav, double a_old, double a_new,
                double dt, int fill_ghosts, double *const *flux_out, orc_stats *stats) {
  eos_t E = make_eos(P);
  if (L->ng < 4) return -1;
  if (fill_ghosts) {
    if (orc_fill_ghosts(L, ORC_NCONS, state_in)) return -1;
    if (grav && orc_fill_ghosts(L, 3, grav)) return -1;
  }
  int rc = 0;
  for (int b = 0; b < L->nbox; ++b) {
    double *fo[3] = {NULL, NULL, NULL};
    if (flux_out)
      for (int d = 0; d < 3; ++d) fo[d] = flux_out[3 * b + d];
    int r = advance_box(&E, P, L->lo + 3 * b, L->hi + 3 * b, L->ng, L->dx + 3 * b, state_in[b],
                        state_out[b], grav ? grav[b] : NULL, a_old, a_new, dt,
                        flux_out ? fo : NULL, stats);
    if (r) rc = r;
  }
  return rc;
}

/* Step 6 alone (corrector with g^{n+1}, then the sync), see the header. */
int orc_correct(const orc_level *L, const orc_params *P, double *const *old,
                double *const *pred, double *const *g_old, double *const *g_new, double a_old,
                double a_new, double dt, orc_stats *st) {
  eos_t E = make_eos(P);
  orc_params Pc = *P;
  Pc.grav_corrector = 1;
  const double an2 = a_new * a_new;
  const step_k sk = {a_old, a_new, dt, 0.5 * dt, 1.0 / a_new, 1.0 / an2, P->eta_de,
                     P->small_pres * E.igm1};
  long long n_use_e = 0, n_floor = 0, n_bad = 0;
  for (int b = 0; b < L->nbox; ++b) {
    geom_t g = make_geom(L->lo + 3 * b, L->hi + 3 * b, L->ng);
    const size_t V = g.vol;
    const double *S = old[b];
    double *Sp = pred[b];
    const double *Go = g_old ? g_old[b] : NULL, *Gn = g_new ? g_new[b] : NULL;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : n_use_e, n_floor, n_bad)
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i) {
          size_t id = gidx(&g, i, j, k);
          double m[3] = {S[V + id], S[2 * V + id], S[3 * V + id]};
          double ms[3] = {Sp[V + id], Sp[2 * V + id], Sp[3 * V + id]};
          double go[3] = {0.0, 0.0, 0.0}, gn[3] = {0.0, 0.0, 0.0};
          for (int c = 0; c < 3; ++c) {
            if (Go) go[c] = Go[c * V + id];
            if (Gn) gn[c] = Gn[c * V + id];
          }
          double out[6];
          finish_cell(&Pc, &sk, S[id], m, go, gn, Sp[id], ms, Sp[4 * V + id], Sp[5 * V + id], out,
                      &n_use_e, &n_floor);
          if (!(out[0] > 0.0) || !isfinite(out[0]) || !isfinite(out[4]) || !isfinite(out[5]))
            n_bad++;
          for (int c = 0; c < 6; ++c) Sp[c * V + id] = out[c];
        }
  }
  if (st) {
    st->use_e += n_use_e;
    st->floor_e += n_floor;
    st->bad += n_bad;
  }
  return n_bad ? -3 : 0;
}

/* CFL time step, Sec. 3.5: sigma * min over cells and directions of
 * a dx_d / (|U_d| + c). */
double orc_estdt(const orc_level *L, const orc_params *P, double *const *state, double a) {
  eos_t E = make_eos(P);
  double best = INFINITY;
  for (int b = 0; b < L->nbox; ++b) {
    geom_t g = make_geom(L->lo + 3 * b, L->hi + 3 * b, L->ng);
    const double *dx = L->dx + 3 * b;
    const double *S = state[b];
    double bmin = INFINITY;
#pragma omp parallel for collapse(2) schedule(static) reduction(min : bmin)
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i) {
          double q6[6];
          primitives(&E, S, g.vol, gidx(&g, i, j, k), q6);
          for (int d = 0; d < 3; ++d) {
            double t = a * dx[d] / (fabs(q6[1 + d]) + q6[5]);
            if (t < bmin) bmin = t;
          }
        }
    if (bmin < best) best = bmin;
  }
  return P->cfl * best;
}

void orc_riemann_counts(long long *calls, long long *iters, int reset) {
  long long c = 0, n = 0;
  for (int t = 0; t < ORC_MAX_THREADS; ++t) {
    c += orc_rcount[t * 8][0];
    n += orc_rcount[t * 8][1];
    if (reset) orc_rcount[t * 8][0] = orc_rcount[t * 8][1] = 0;
  }
  *calls = c;
  *iters = n;
}

/* ------------------------------------------------------------------ */
/* Unit-level entry points for the pin tests. */
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }

void orc_flatten_line(const orc_params *p, int n, const double *pr, const double *u, double *fl) {
  for (int i = 0; i < n; ++i) fl[i] = 1.0;
  for (int i = 3; i < n - 3; ++i) fl[i] = 1.0 - flat_dir(pr + i, u + i, 1, p->small_pres);
}

int orc_flatten_field(const orc_level *L, const orc_params *p, double *const *S,
                      double *const *fl) {
  eos_t E = make_eos(p);
  for (int b = 0; b < L->nbox; ++b) {
    geom_t g = make_geom(L->lo + 3 * b, L->hi + 3 * b, L->ng);
    const size_t V = g.vol;
    double *q = alloc_arr(6 * V);
    for (size_t id = 0; id < V; ++id) {
      double q6[6];
      primitives(&E, S[b], V, id, q6);
      for (int v = 0; v < 6; ++v) q[v * V + id] = q6[v];
    }
    for (size_t id = 0; id < V; ++id) fl[b][id] = 1.0;
    for (int k = -1; k <= g.n[2]; ++k)
      for (int j = -1; j <= g.n[1]; ++j)
        for (int i = -1; i <= g.n[0]; ++i) {
          size_t id = gidx(&g, i, j, k);
          double f = 0.0;
          for (int d = 0; d < 3; ++d) {
            double fd = flat_dir(q + 4 * V + id, q + (size_t)(1 + d) * V + id, (ptrdiff_t)g.st[d],
                                 E.small_pres);
            if (fd > f) f = fd;
          }
          fl[b][id] = 1.0 - f;
        }
    free(q);
  }
  return 0;
}

void orc_ppm_line(int n, const double *s, double *sL, double *sR, double *s6) {
  for (int i = 2; i < n - 2; ++i) ppm_coeffs(s + i - 2, &sL[i], &sR[i], &s6[i]);
}

void orc_ppm_integrals(double sL, double sR, double s6, double sigma, double *ip, double *im) {
  *ip = ppm_ip(sL, sR, s6, sigma);
  *im = ppm_im(sL, sR, s6, sigma);
}

int orc_riemann(const orc_params *p, const double *qL, const double *qR, double *flux8,
                double *pstar, double *ustar) {
  eos_t E = make_eos(p);
  riemann_solve(&E, qL, qR, flux8, pstar, ustar, NULL);
  return 0;
}

int orc_riemann_state(const orc_params *p, const double *qL, const double *qR, double *g5) {
  eos_t E = make_eos(p);
  double flux8[8];
  riemann_solve(&E, qL, qR, flux8, NULL, NULL, g5);
  return 0;
}

/* q5: 5 x n primitives (rho,u_x,u_y,u_z,p) along a line in direction dir;
 * gline: 3 x n gravity.  Fills qm, qp (5 x n) and the wave amplitudes
 * (3 x n, may be NULL) for cells 2..n-3. */
void orc_trace_line(const orc_params *p, int n, const double *q5, const double *gline,
                    const double *fl, double dtp, double dx, double adot, int dir, double *qm,
                    double *qp, double *beta_m, double *beta_p) {
  eos_t E = make_eos(p);
  trace_src_t src;
  src.hdtp = 0.5 * dtp;
  src.src_u = 0.5 * adot;
  src.src_p = 1.5 * E.gm1 * adot;
  for (int i = 2; i < n - 2; ++i) {
    double s5[5][5];
    for (int v = 0; v < 5; ++v)
      for (int o = 0; o < 5; ++o) s5[v][o] = q5[v * n + i + o - 2];
    double c = sqrt(E.gamma * s5[4][2] / s5[0][2]);
    double g3[3] = {0.0, 0.0, 0.0};
    if (gline)
      for (int d = 0; d < 3; ++d) g3[d] = gline[d * n + i];
    double a5[5], b5[5], bm[3], bp[3];
    trace_cell(&E, s5, c, g3, dtp / dx, &src, fl ? fl[i] : 1.0, dir, a5, b5, bm, bp);
    for (int v = 0; v < 5; ++v) {
      qm[v * n + i] = a5[v];
      qp[v * n + i] = b5[v];
    }
    if (beta_m)
      for (int w = 0; w < 3; ++w) beta_m[w * n + i] = bm[w];
    if (beta_p)
      for (int w = 0; w < 3; ++w) beta_p[w * n + i] = bp[w];
  }
}

/* ------------------------------------------------------------------ */
/* Coarse-fine coupling, refinement ratio 2, no subcycling.
 *
 * Sec. 4.1: grids are refined by 2 and properly nested; data of a newly
 * refined region comes from a piecewise linear profile in each coarse cell,
 * built from its nearest neighbours and limited so that it makes no new
 * maxima or minima, evaluated at the fine cell centres (so the mean of the
 * 8 fine cells is the coarse value).  Sec. 4.2: no subcycling, both levels
 * take the same dt.  Sec. 4.3, Step 2: the fine ghost cells take coarse
 * (Dirichlet) data where no fine grid covers them; Step 8: reflux the
 * coarse cells next to the fine level, then average the fine solution down.
 *
 * Readings (the paper names the operations without their formulas):
 *  - the slope of the linear profile along d is the MC-limited slope of the
 *    coarse cell and its two neighbours along d (the PPM slope of O2);
 *  - "no new extrema": the three slopes are scaled by one factor alpha so
 *    that the largest and smallest fine values stay inside the range of the
 *    coarse cell and its six face neighbours;
 *  - each conserved component (rho, m, rhoE, rhoe) and each gravity
 *    component is interpolated on its own;
 *  - reflux corrects the flux-divergence terms of the update only, with the
 *    update's coefficients (dt' for rho, dt/a_new for m, a_h dt/a_new^2 for
 *    rhoE and rhoe); the gravity corrector, the pdV term and the dual-energy
 *    switch are not redone, and averaging down does not re-sync e and E.
 */
static int floor_div2(int x) { return (x >= 0) ? x / 2 : -((-x + 1) / 2); }

static int wrap_into(int x, int lo, int hi) {
  int len = hi - lo + 1;
  return lo + ((x - lo) % len + len) % len;
}

int orc_amr_check(const orc_level *C, const orc_level *F) {
  if (C->ng < 4 || F->ng < 4 || F->ndom != C->ndom) return -1;
  for (int d = 0; d < C->ndom; ++d)
    for (int a = 0; a < 3; ++a) {
      if (F->dom_lo[3 * d + a] != 2 * C->dom_lo[3 * d + a]) return -1;
      if (F->dom_hi[3 * d + a] != 2 * C->dom_hi[3 * d + a] + 1) return -1;
      if (C->dom_bc[6 * d + a] != ORC_BC_PERIODIC || C->dom_bc[6 * d + 3 + a] != ORC_BC_PERIODIC)
        return -1;
      if (F->dom_bc[6 * d + a] != ORC_BC_PERIODIC || F->dom_bc[6 * d + 3 + a] != ORC_BC_PERIODIC)
        return -1;
    }
  for (int b = 0; b < F->nbox; ++b)
    for (int a = 0; a < 3; ++a) {
      if (F->lo[3 * b + a] % 2 != 0 || (F->hi[3 * b + a] + 1) % 2 != 0) return -1;
    }
  return 0;
}

/* Interpolated value of one fine cell: coarse cell (I,J,K) (local indices of
 * coarse box geometry g, its ghosts filled), fine offsets o in {0,1}^3. */
static double prolong_value(const double *u, const geom_t *g, int I, int J, int K, const int o[3]) {
  const size_t id = gidx(g, I, J, K);
  const double uc = u[id];
  double s[3], umin = uc, umax = uc;
  for (int d = 0; d < 3; ++d) {
    const double um = u[id - g->st[d]], up = u[id + g->st[d]];
    s[d] = mc_slope(um, uc, up);
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
  const double xo = o[0] ? 0.25 : -0.25, yo = o[1] ? 0.25 : -0.25, zo = o[2] ? 0.25 : -0.25;
  return uc + alpha * (s[0] * xo + s[1] * yo + s[2] * zo);
}

int orc_amr_interp(const orc_level *C, int ncomp, double *const *cf, const orc_level *F,
                   double *const *ff, int region) {
  if (orc_amr_check(C, F)) return -1;
  int err = 0;
  for (int b = 0; b < F->nbox; ++b) {
    geom_t g = make_geom(F->lo + 3 * b, F->hi + 3 * b, F->ng);
    const int dom = F->dom[b];
    const int *flo = F->dom_lo + 3 * dom, *fhi = F->dom_hi + 3 * dom;
    const int *clo = C->dom_lo + 3 * dom;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int k = -g.ng; k < g.n[2] + g.ng; ++k) {
      int hint = -1, chint = -1;
      for (int j = -g.ng; j < g.n[1] + g.ng; ++j)
        for (int i = -g.ng; i < g.n[0] + g.ng; ++i) {
          const int loc[3] = {i, j, k};
          int inside = 1;
          for (int d = 0; d < 3; ++d)
            if (loc[d] < 0 || loc[d] >= g.n[d]) inside = 0;
          if (region == 1 && inside) continue;
          int gi[3];
          for (int d = 0; d < 3; ++d) gi[d] = wrap_into(F->lo[3 * b + d] + loc[d], flo[d], fhi[d]);
          const size_t dst = gidx(&g, i, j, k);
          if (region == 1) {
            const int sb = find_box(F, dom, gi, hint);
            if (sb >= 0) {
              hint = sb;
              geom_t gs = make_geom(F->lo + 3 * sb, F->hi + 3 * sb, F->ng);
              const size_t src = gidx(&gs, gi[0] - F->lo[3 * sb], gi[1] - F->lo[3 * sb + 1],
                                      gi[2] - F->lo[3 * sb + 2]);
              for (int c = 0; c < ncomp; ++c) ff[b][c * g.vol + dst] = ff[sb][c * gs.vol + src];
              continue;
            }
          }
          int ci[3], o[3];
          for (int d = 0; d < 3; ++d) {
            const int rel = gi[d] - flo[d];
            ci[d] = clo[d] + floor_div2(rel);
            o[d] = rel - 2 * floor_div2(rel);
          }
          const int cb = find_box(C, dom, ci, chint);
          if (cb < 0) {
            err = 1;
            continue;
          }
          chint = cb;
          geom_t gc = make_geom(C->lo + 3 * cb, C->hi + 3 * cb, C->ng);
          for (int c = 0; c < ncomp; ++c)
            ff[b][c * g.vol + dst] =
                prolong_value(cf[cb] + c * gc.vol, &gc, ci[0] - C->lo[3 * cb],
                              ci[1] - C->lo[3 * cb + 1], ci[2] - C->lo[3 * cb + 2], o);
        }
    }
  }
  return err ? -1 : 0;
}

/* Coarse cell ci (domain index, wrapped) is under the fine level if a fine
 * box holds its first fine cell. */
static int coarse_covered(const orc_level *C, const orc_level *F, int dom, const int ci[3]) {
  int fi[3];
  for (int d = 0; d < 3; ++d) fi[d] = F->dom_lo[3 * dom + d] + 2 * (ci[d] - C->dom_lo[3 * dom + d]);
  return find_box(F, dom, fi, -1) >= 0;
}

int orc_amr_reflux(const orc_level *C, double *const *cstate, double *const *cflux,
                   const orc_level *F, double *const *fflux, double a_old, double a_new,
                   double dt) {
  if (orc_amr_check(C, F)) return -1;
  const double a_half = 0.5 * (a_old + a_new);
  const double dtp = dt / a_half;
  const double ian = 1.0 / a_new;
  const double ian2 = 1.0 / (a_new * a_new);
  const double ahdt = a_half * dt;
  const double coef[6] = {dtp, dt * ian, dt * ian, dt * ian, ahdt * ian2, ahdt * ian2};
  /* six orientations in a fixed order (x low, x high, y low, ...); within
   * one orientation no coarse cell is met twice */
  for (int orient = 0; orient < 6; ++orient) {
    const int d = orient / 2, high = orient % 2;
    const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    for (int fb = 0; fb < F->nbox; ++fb) {
      const int dom = F->dom[fb];
      const int *clo = C->dom_lo + 3 * dom, *chi = C->dom_hi + 3 * dom;
      const int *flo = F->dom_lo + 3 * dom;
      int fl[3], fn[3], cl[3], ch[3];
      for (int a = 0; a < 3; ++a) {
        fl[a] = F->lo[3 * fb + a];
        fn[a] = F->hi[3 * fb + a] - fl[a] + 1;
        cl[a] = clo[a] + (fl[a] - flo[a]) / 2;
        ch[a] = cl[a] + fn[a] / 2 - 1;
      }
      int fe[3] = {fn[0], fn[1], fn[2]};
      fe[d] += 1;
      const size_t fv = (size_t)fe[0] * fe[1] * fe[2];
      const double *Ff = fflux[3 * fb + d];
      const int ffi = high ? fn[d] : 0; /* fine face index along d */
      for (int q2 = cl[t2]; q2 <= ch[t2]; ++q2)
        for (int q1 = cl[t1]; q1 <= ch[t1]; ++q1) {
          int P[3];
          P[d] = high ? ch[d] + 1 : cl[d] - 1;
          P[t1] = q1;
          P[t2] = q2;
          for (int a = 0; a < 3; ++a) P[a] = wrap_into(P[a], clo[a], chi[a]);
          if (coarse_covered(C, F, dom, P)) continue;
          const int cb = find_box(C, dom, P, -1);
          if (cb < 0) return -1;
          geom_t gc = make_geom(C->lo + 3 * cb, C->hi + 3 * cb, C->ng);
          int pl[3];
          for (int a = 0; a < 3; ++a) pl[a] = P[a] - C->lo[3 * cb + a];
          int ce[3] = {gc.n[0], gc.n[1], gc.n[2]};
          ce[d] += 1;
          const size_t cv = (size_t)ce[0] * ce[1] * ce[2];
          int cf[3] = {pl[0], pl[1], pl[2]};
          if (!high) cf[d] += 1; /* the outside cell's high face */
          const size_t cid = ((size_t)cf[2] * ce[1] + cf[1]) * ce[0] + cf[0];
          const double *Fc = cflux[3 * cb + d];
          const double idx = 1.0 / C->dx[3 * cb + d];
          const size_t sid = gidx(&gc, pl[0], pl[1], pl[2]);
          for (int c = 0; c < 6; ++c) {
            double fsum = 0.0;
            for (int s = 0; s < 4; ++s) {
              int fi[3];
              fi[d] = ffi;
              fi[t1] = 2 * (q1 - cl[t1]) + (s & 1);
              fi[t2] = 2 * (q2 - cl[t2]) + (s >> 1);
              const double v = Ff[c * fv + ((size_t)fi[2] * fe[1] + fi[1]) * fe[0] + fi[0]];
              fsum = (s == 0) ? v : fsum + v;
            }
            const double favg = 0.25 * fsum;
            const double corr = coef[c] * ((favg - Fc[c * cv + cid]) * idx);
            double *U = cstate[cb] + c * gc.vol + sid;
            *U = high ? *U + corr : *U - corr;
          }
        }
    }
  }
  return 0;
}

int orc_amr_average_down(const orc_level *C, int ncomp, double *const *cstate,
                         const orc_level *F, double *const *fstate) {
  if (orc_amr_check(C, F)) return -1;
  for (int fb = 0; fb < F->nbox; ++fb) {
    const int dom = F->dom[fb];
    geom_t g = make_geom(F->lo + 3 * fb, F->hi + 3 * fb, F->ng);
    const int *clo = C->dom_lo + 3 * dom, *flo = F->dom_lo + 3 * dom;
    for (int K = 0; K < g.n[2] / 2; ++K)
      for (int J = 0; J < g.n[1] / 2; ++J)
        for (int I = 0; I < g.n[0] / 2; ++I) {
          int ci[3] = {I, J, K};
          for (int a = 0; a < 3; ++a) ci[a] += clo[a] + (F->lo[3 * fb + a] - flo[a]) / 2;
          const int cb = find_box(C, dom, ci, -1);
          if (cb < 0) return -1;
          geom_t gc = make_geom(C->lo + 3 * cb, C->hi + 3 * cb, C->ng);
          const size_t cid = gidx(&gc, ci[0] - C->lo[3 * cb], ci[1] - C->lo[3 * cb + 1],
                                  ci[2] - C->lo[3 * cb + 2]);
          for (int c = 0; c < ncomp; ++c) {
            double s = 0.0;
            for (int o = 0; o < 8; ++o) {
              const double v = fstate[fb][c * g.vol + gidx(&g, 2 * I + (o & 1), 2 * J + ((o >> 1) & 1),
                                                           2 * K + (o >> 2))];
              s = (o == 0) ? v : s + v;
            }
            cstate[cb][c * gc.vol + cid] = 0.125 * s;
          }
        }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Self-gravity, Sec. 3.4: the 7-point Laplacian on the cell centres of the
 * periodic domain, solved by geometric multigrid (V-cycles with red-black
 * Gauss-Seidel), tolerance 1e-12 by default, warm start from the previous
 * potential; g the centred difference of phi.  The paper uses BoxLib's
 * cell-centred multigrid without stating its transfer operators; reading:
 * restriction = mean of the 8 fine cells, prolongation = the coarse value
 * (piecewise constant), as in standard cell-centred multigrid.
 *
 * All sums run in a fixed order (rows, then planes, then the domain) so
 * that a parallel code can reproduce them exactly. */
typedef struct {
  int n[3];
  double h2, ih2;   /* dx^2 and 1/dx^2 at this grid */
  double *phi, *f;
} mg_grid;

static size_t mg_idx(const mg_grid *g, int i, int j, int k) {
  return ((size_t)k * g->n[1] + j) * g->n[0] + i;
}

static int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

static double mg_nbsum(const mg_grid *g, int i, int j, int k) {
  const double *u = g->phi;
  double s = u[mg_idx(g, wrapi(i - 1, g->n[0]), j, k)];
  s = s + u[mg_idx(g, wrapi(i + 1, g->n[0]), j, k)];
  s = s + u[mg_idx(g, i, wrapi(j - 1, g->n[1]), k)];
  s = s + u[mg_idx(g, i, wrapi(j + 1, g->n[1]), k)];
  s = s + u[mg_idx(g, i, j, wrapi(k - 1, g->n[2]))];
  s = s + u[mg_idx(g, i, j, wrapi(k + 1, g->n[2]))];
  return s;
}

/* one red-black Gauss-Seidel sweep: red cells (i+j+k even), then black */
static void mg_sweep(mg_grid *g) {
  for (int color = 0; color < 2; ++color) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->n[2]; ++k)
      for (int j = 0; j < g->n[1]; ++j)
        for (int i = (j + k + color) & 1; i < g->n[0]; i += 2) {
          const size_t id = mg_idx(g, i, j, k);
          g->phi[id] = (mg_nbsum(g, i, j, k) - g->h2 * g->f[id]) * SIXTH;
        }
  }
}

static double mg_resid(const mg_grid *g, int i, int j, int k) {
  const size_t id = mg_idx(g, i, j, k);
  return g->f[id] - (mg_nbsum(g, i, j, k) - 6.0 * g->phi[id]) * g->ih2;
}

static double mg_resid_max(const mg_grid *g) {
  double m = 0.0;
#pragma omp parallel for collapse(2) schedule(static) reduction(max : m)
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) {
        const double r = fabs(mg_resid(g, i, j, k));
        if (r > m) m = r;
      }
  return m;
}

/* coarse f = mean of the 8 fine residuals; coarse phi = 0 */
static void mg_restrict(const mg_grid *fg, mg_grid *cg) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < cg->n[2]; ++k)
    for (int j = 0; j < cg->n[1]; ++j)
      for (int i = 0; i < cg->n[0]; ++i) {
        double s = 0.0;
        for (int o = 0; o < 8; ++o) {
          const double r = mg_resid(fg, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + (o >> 2));
          s = (o == 0) ? r : s + r;
        }
        const size_t id = mg_idx(cg, i, j, k);
        cg->f[id] = 0.125 * s;
        cg->phi[id] = 0.0;
      }
}

static void mg_prolong_add(const mg_grid *cg, mg_grid *fg) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < fg->n[2]; ++k)
    for (int j = 0; j < fg->n[1]; ++j)
      for (int i = 0; i < fg->n[0]; ++i) {
        const size_t id = mg_idx(fg, i, j, k);
        fg->phi[id] = fg->phi[id] + cg->phi[mg_idx(cg, i / 2, j / 2, k / 2)];
      }
}

static void mg_vcycle(mg_grid *G, int l, int nl, const orc_poisson_params *p) {
  if (l == nl - 1) {
    for (int s = 0; s < p->coarse_sweeps; ++s) mg_sweep(&G[l]);
    return;
  }
  for (int s = 0; s < p->pre; ++s) mg_sweep(&G[l]);
  mg_restrict(&G[l], &G[l + 1]);
  mg_vcycle(G, l + 1, nl, p);
  mg_prolong_add(&G[l + 1], &G[l]);
  for (int s = 0; s < p->post; ++s) mg_sweep(&G[l]);
}

int orc_poisson_solve(const orc_level *L, const orc_poisson_params *p, double *const *state,
                      const double *rho_dm, double a, double *phi, double *const *grav_out,
                      double *g_dense, orc_poisson_stats *st) {
  if (L->ndom != 1) return -1;
  const int *dlo = L->dom_lo, *dhi = L->dom_hi;
  int n[3];
  long long cells = 0;
  for (int d = 0; d < 3; ++d) {
    n[d] = dhi[d] - dlo[d] + 1;
    if (n[d] % 2) return -1;
    if (L->dom_bc[d] != ORC_BC_PERIODIC || L->dom_bc[3 + d] != ORC_BC_PERIODIC) return -1;
  }
  const double dx = L->dx[0];
  for (int b = 0; b < L->nbox; ++b) {
    for (int d = 0; d < 3; ++d)
      if (L->dx[3 * b + d] != dx) return -1;
    long long v = 1;
    for (int d = 0; d < 3; ++d) v *= (L->hi[3 * b + d] - L->lo[3 * b + d] + 1);
    cells += v;
  }
  if (cells != (long long)n[0] * n[1] * n[2]) return -1;
  /* grid hierarchy */
  mg_grid G[32];
  int nl = 0;
  {
    int m[3] = {n[0], n[1], n[2]};
    double h = dx;
    for (;;) {
      G[nl].n[0] = m[0];
      G[nl].n[1] = m[1];
      G[nl].n[2] = m[2];
      G[nl].h2 = h * h;
      G[nl].ih2 = 1.0 / (h * h);
      size_t v = (size_t)m[0] * m[1] * m[2];
      G[nl].phi = nl ? (double *)calloc(v, sizeof(double)) : phi;
      G[nl].f = (double *)calloc(v, sizeof(double));
      ++nl;
      /* coarsen while the coarse extents stay even (a periodic red-black
       * colouring needs even extents) and no smaller than min_size */
      int ok = nl < 32;
      for (int d = 0; d < 3; ++d)
        if (m[d] % 4 || m[d] < 2 * p->min_size) ok = 0;
      if (!ok) break;
      for (int d = 0; d < 3; ++d) m[d] /= 2;
      h *= 2.0;
    }
  }
  /* gather rho into the dense right-hand side */
  double *f0 = G[0].f;
  for (int b = 0; b < L->nbox; ++b) {
    geom_t g = make_geom(L->lo + 3 * b, L->hi + 3 * b, L->ng);
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i)
          f0[mg_idx(&G[0], L->lo[3 * b] - dlo[0] + i, L->lo[3 * b + 1] - dlo[1] + j,
                    L->lo[3 * b + 2] - dlo[2] + k)] = state[b][gidx(&g, i, j, k)];
  }
  /* dark matter (Sec. 3.4): rho_b + rho_dm */
  if (rho_dm)
    for (size_t q = 0; q < (size_t)n[0] * n[1] * n[2]; ++q) f0[q] = f0[q] + rho_dm[q];
  /* mean density: rows, then planes, then the domain, each in index order */
  double tot = 0.0;
  for (int k = 0; k < n[2]; ++k) {
    double plane = 0.0;
    for (int j = 0; j < n[1]; ++j) {
      double row = 0.0;
      for (int i = 0; i < n[0]; ++i) {
        const double v = f0[mg_idx(&G[0], i, j, k)];
        row = (i == 0) ? v : row + v;
      }
      plane = (j == 0) ? row : plane + row;
    }
    tot = (k == 0) ? plane : tot + plane;
  }
  const double mean = tot / ((double)n[0] * n[1] * n[2]);
  const double c = p->four_pi_G / a;
  double fmax = 0.0;
  for (size_t q = 0; q < (size_t)n[0] * n[1] * n[2]; ++q) {
    f0[q] = c * (f0[q] - mean);
    if (fabs(f0[q]) > fmax) fmax = fabs(f0[q]);
  }
  /* V-cycles */
  int cyc = 0;
  double res = mg_resid_max(&G[0]);
  const double target = p->tol * fmax;
  while (res > target && cyc < p->max_cycles) {
    mg_vcycle(G, 0, nl, p);
    ++cyc;
    res = mg_resid_max(&G[0]);
  }
  /* g = -grad phi, centred differences */
  const double hdx = 0.5 / dx;
  if (g_dense) {
    const size_t N = (size_t)n[0] * n[1] * n[2];
    for (int K = 0; K < n[2]; ++K)
      for (int J = 0; J < n[1]; ++J)
        for (int I = 0; I < n[0]; ++I) {
          const double *u = phi;
          const size_t id = mg_idx(&G[0], I, J, K);
          g_dense[id] = -((u[mg_idx(&G[0], wrapi(I + 1, n[0]), J, K)] -
                           u[mg_idx(&G[0], wrapi(I - 1, n[0]), J, K)]) * hdx);
          g_dense[N + id] = -((u[mg_idx(&G[0], I, wrapi(J + 1, n[1]), K)] -
                               u[mg_idx(&G[0], I, wrapi(J - 1, n[1]), K)]) * hdx);
          g_dense[2 * N + id] = -((u[mg_idx(&G[0], I, J, wrapi(K + 1, n[2]))] -
                                   u[mg_idx(&G[0], I, J, wrapi(K - 1, n[2]))]) * hdx);
        }
  }
  for (int b = 0; grav_out && b < L->nbox; ++b) {
    geom_t g = make_geom(L->lo + 3 * b, L->hi + 3 * b, L->ng);
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i) {
          const int I = L->lo[3 * b] - dlo[0] + i, J = L->lo[3 * b + 1] - dlo[1] + j,
                    K = L->lo[3 * b + 2] - dlo[2] + k;
          const double *u = phi;
          const size_t id = gidx(&g, i, j, k);
          grav_out[b][id] = -((u[mg_idx(&G[0], wrapi(I + 1, n[0]), J, K)] -
                               u[mg_idx(&G[0], wrapi(I - 1, n[0]), J, K)]) * hdx);
          grav_out[b][g.vol + id] = -((u[mg_idx(&G[0], I, wrapi(J + 1, n[1]), K)] -
                                       u[mg_idx(&G[0], I, wrapi(J - 1, n[1]), K)]) * hdx);
          grav_out[b][2 * g.vol + id] = -((u[mg_idx(&G[0], I, J, wrapi(K + 1, n[2]))] -
                                           u[mg_idx(&G[0], I, J, wrapi(K - 1, n[2]))]) * hdx);
        }
  }
  for (int l = 0; l < nl; ++l) {
    if (l) free(G[l].phi);
    free(G[l].f);
  }
  if (st) {
    st->cycles = cyc;
    st->resid = fmax > 0.0 ? res / fmax : 0.0;
    st->rho_mean = mean;
  }
  return res <= target ? 0 : -4;
}


/* ------------------------------------------------------------------ */
/* Dark matter as particles (Sec. 3.3, 3.4, 3.5, 3.6 Steps 3 and 5) on the
 * dense periodic grid of n[0] x n[1] x n[2] cells of width dx, positions in
 * [0, n dx) per axis (cell I spans [I dx, (I+1) dx)).
 *
 * Cloud in cell: a particle is a cube of side dx centred on it; the cells it
 * overlaps get its mass in proportion to the overlap, divided by dx^3.  The
 * same weights interpolate g from the cell centres to the particle (Sec. 3.3:
 * linear interpolation from cell centres), which with the centred-difference
 * g makes the self-force vanish (Sec. 3.4). */
static void cic_weights(double x, double dx, int n, int *i0, double *w0) {
  const double s = x / dx - 0.5;
  const double fl = floor(s);
  *w0 = 1.0 - (s - fl);      /* weight of cell i0; i0 + 1 gets 1 - w0 */
  int i = (int)fl;
  *i0 = wrapi(i, n);
}

void orc_pm_deposit(const int n[3], double dx, const double *x, const double *m, long long np,
                    double *rho) {
  const size_t N = (size_t)n[0] * n[1] * n[2];
  for (size_t q = 0; q < N; ++q) rho[q] = 0.0;
  const double iv = 1.0 / (dx * dx * dx);
  for (long long p = 0; p < np; ++p) {
    int i0[3];
    double w0[3];
    for (int d = 0; d < 3; ++d) cic_weights(x[d * np + p], dx, n[d], &i0[d], &w0[d]);
    for (int o = 0; o < 8; ++o) {
      const int I = (o & 1) ? wrapi(i0[0] + 1, n[0]) : i0[0];
      const int J = ((o >> 1) & 1) ? wrapi(i0[1] + 1, n[1]) : i0[1];
      const int K = (o >> 2) ? wrapi(i0[2] + 1, n[2]) : i0[2];
      const double w = ((o & 1) ? 1.0 - w0[0] : w0[0]) * (((o >> 1) & 1) ? 1.0 - w0[1] : w0[1]) *
                       ((o >> 2) ? 1.0 - w0[2] : w0[2]);
      const size_t id = ((size_t)K * n[1] + J) * n[0] + I;
      rho[id] = rho[id] + m[p] * w * iv;
    }
  }
}

/* g at a particle: the cloud-in-cell weights of its position */
static void pm_g_at(const int n[3], double dx, const double *g, const double xp[3], double out[3]) {
  const size_t N = (size_t)n[0] * n[1] * n[2];
  int i0[3];
  double w0[3];
  for (int d = 0; d < 3; ++d) cic_weights(xp[d], dx, n[d], &i0[d], &w0[d]);
  for (int c = 0; c < 3; ++c) out[c] = 0.0;
  for (int o = 0; o < 8; ++o) {
    const int I = (o & 1) ? wrapi(i0[0] + 1, n[0]) : i0[0];
    const int J = ((o >> 1) & 1) ? wrapi(i0[1] + 1, n[1]) : i0[1];
    const int K = (o >> 2) ? wrapi(i0[2] + 1, n[2]) : i0[2];
    const double w = ((o & 1) ? 1.0 - w0[0] : w0[0]) * (((o >> 1) & 1) ? 1.0 - w0[1] : w0[1]) *
                     ((o >> 2) ? 1.0 - w0[2] : w0[2]);
    const size_t id = ((size_t)K * n[1] + J) * n[0] + I;
    for (int c = 0; c < 3; ++c) out[c] = out[c] + w * g[c * N + id];
  }
}

void orc_pm_interp(const int n[3], double dx, const double *g, const double *x, long long np,
                   double *gp) {
  for (long long p = 0; p < np; ++p) {
    double xp[3] = {x[p], x[np + p], x[2 * np + p]}, o[3];
    pm_g_at(n, dx, g, xp, o);
    for (int c = 0; c < 3; ++c) gp[c * np + p] = o[c];
  }
}

/* Step 3: u^{n+1/2} = (a^n u^n + dt/2 g^n) / a^{n+1/2}; x^{n+1} = x^n +
 * dt / a^{n+1/2} u^{n+1/2}, wrapped into the periodic domain. */
void orc_pm_kick_drift(const int n[3], double dx, const double *g, double *x, double *u,
                       long long np, double a_old, double a_half, double dt) {
  const double L[3] = {n[0] * dx, n[1] * dx, n[2] * dx};
  for (long long p = 0; p < np; ++p) {
    double xp[3] = {x[p], x[np + p], x[2 * np + p]}, gp[3];
    pm_g_at(n, dx, g, xp, gp);
    for (int c = 0; c < 3; ++c) {
      const double uh = (a_old * u[c * np + p] + 0.5 * dt * gp[c]) / a_half;
      u[c * np + p] = uh;
      double xn = xp[c] + dt / a_half * uh;
      if (xn < 0.0) xn = xn + L[c];
      if (xn >= L[c]) xn = xn - L[c];
      x[c * np + p] = xn;
    }
  }
}

/* Step 5: u^{n+1} = (a^{n+1/2} u^{n+1/2} + dt/2 g^{n+1}) / a^{n+1}. */
void orc_pm_kick(const int n[3], double dx, const double *g, const double *x, double *u,
                 long long np, double a_half, double a_new, double dt) {
  for (long long p = 0; p < np; ++p) {
    double xp[3] = {x[p], x[np + p], x[2 * np + p]}, gp[3];
    pm_g_at(n, dx, g, xp, gp);
    for (int c = 0; c < 3; ++c) u[c * np + p] = (a_half * u[c * np + p] + 0.5 * dt * gp[c]) / a_new;
  }
}

/* Sec. 3.5: dt_dm = cfl_dm min_d a dx / max_j |u_j,d|, and g_j dt^2 < dx:
 * dt_dm <= sqrt(dx / max_j |g_j,d|) (reading: per component, g at the
 * particle by cloud in cell).  Returns +inf for resting particles in no field. */
double orc_pm_estdt(const int n[3], double dx, const double *g, const double *x, const double *u,
                    long long np, double a, double cfl_dm) {
  double umax = 0.0, gmax = 0.0;
  for (long long p = 0; p < np; ++p) {
    double xp[3] = {x[p], x[np + p], x[2 * np + p]}, gp[3];
    pm_g_at(n, dx, g, xp, gp);
    for (int c = 0; c < 3; ++c) {
      if (fabs(u[c * np + p]) > umax) umax = fabs(u[c * np + p]);
      if (fabs(gp[c]) > gmax) gmax = fabs(gp[c]);
    }
  }
  double dt = INFINITY;
  if (umax > 0.0) dt = cfl_dm * (a * dx / umax);
  if (gmax > 0.0) {
    const double dg = sqrt(dx / gmax);
    if (dg < dt) dt = dg;
  }
  return dt;
}
