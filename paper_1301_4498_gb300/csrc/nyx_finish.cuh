// nyx_finish.cuh -- the FP64 end of the update of one cell (Sec. 3.6 Steps 2
// and 6, Sec. 3.2): the predictor's total energy in either discretisation of
// the gravity source, the gravity corrector with g^n and g^{n+1}, and the
// dual-energy synchronisation.  Shared by the FP64 update kernels and the
// standalone corrector; the translation units that include it are built
// without FMA contraction, in the oracle's expression order.
#pragma once
#include "nyx_internal.cuh"

namespace nyx {

// Predictor total energy (Step 2).  grav_energy 0: the product of the
// cell-centred momentum at t^n and g^n; 1: the change of the kinetic energy
// (at the new density rho_s) that the gravity part of the momentum update
// makes, from mh (hydro only) to ms (with gravity).
__device__ __forceinline__ double predictor_energy(const SchemeConsts &k, const StepConsts &sc,
                                                   double rE, double re, double div4, double m0,
                                                   double m1, double m2, double g0, double g1,
                                                   double g2, double d1, double d2, double d3,
                                                   double rho_s, double ms0, double ms1,
                                                   double ms2) {
  if (k.grav_energy) {
    const double mh0 = (sc.a_old * m0 - sc.dt * d1) * sc.ian;
    const double mh1 = (sc.a_old * m1 - sc.dt * d2) * sc.ian;
    const double mh2 = (sc.a_old * m2 - sc.dt * d3) * sc.ian;
    const double kh = mh0 * mh0 + mh1 * mh1 + mh2 * mh2;
    const double ks = ms0 * ms0 + ms1 * ms1 + ms2 * ms2;
    return (sc.ao2 * rE - sc.ahdt * div4 + sc.expn * re) * sc.ian2 + 0.5 * (ks - kh) / rho_s;
  }
  const double mg = m0 * g0 + m1 * g1 + m2 * g2;
  return (sc.ao2 * rE - sc.ahdt * div4 + sc.dta * mg + sc.expn * re) * sc.ian2;
}

// Step 6 of one cell: the corrector U^{n+1} = U^{n+1,*} + dt/2 (S_g^{n+1,*}
// - S_g^n) with go = g^n and gn = g^{n+1} (when corrector), then the
// dual-energy sync (when sync).  rho, m*: state at t^n; rho_s, ms*, rE_s,
// re_s: the predictor.  out = (rho, m_x, m_y, m_z, rhoE, rhoe).
__device__ __forceinline__ void finish_cell(const SchemeConsts &k, const StepConsts &sc,
                                            double rho, double m0, double m1, double m2,
                                            double go0, double go1, double go2, double gn0,
                                            double gn1, double gn2, double rho_s, double ms0,
                                            double ms1, double ms2, double rE_s, double re_s,
                                            bool corrector, bool sync, double (&out)[6]) {
  double mn0 = ms0, mn1 = ms1, mn2 = ms2, rEn = rE_s;
  if (corrector) {
    mn0 = ms0 + sc.hdt * (rho_s * gn0 - rho * go0) * sc.ian;
    mn1 = ms1 + sc.hdt * (rho_s * gn1 - rho * go1) * sc.ian;
    mn2 = ms2 + sc.hdt * (rho_s * gn2 - rho * go2) * sc.ian;
    if (k.grav_energy) {
      const double ks = ms0 * ms0 + ms1 * ms1 + ms2 * ms2;
      const double kn = mn0 * mn0 + mn1 * mn1 + mn2 * mn2;
      rEn = rE_s + 0.5 * (kn - ks) / rho_s;
    } else {
      const double mg = m0 * go0 + m1 * go1 + m2 * go2;
      const double msg = ms0 * gn0 + ms1 * gn1 + ms2 * gn2;
      rEn = rE_s + sc.hdt * (sc.a_new * msg - sc.a_old * mg) * sc.ian2;
    }
  }
  double ren = re_s;
  if (sync) {
    const double ke = 0.5 * (mn0 * mn0 + mn1 * mn1 + mn2 * mn2) / rho_s;
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
  out[0] = rho_s;
  out[1] = mn0;
  out[2] = mn1;
  out[3] = mn2;
  out[4] = rEn;
  out[5] = ren;
}

}  // namespace nyx
