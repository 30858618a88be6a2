// nyx_internal.cuh -- device-side descriptors shared by the kernels of
// libnyxhydro.so and the host code that builds them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nyx_hydro.h"

namespace nyx {

constexpr int NCONS = 6;  // rho, m_x, m_y, m_z, rhoE, rhoe
constexpr int NGRAV = 3;

// Status bits raised on the device (read by nyx_hydro_status).
constexpr unsigned ST_NEGATIVE = 1u;
constexpr unsigned ST_NONFINITE = 2u;
constexpr unsigned ST_OVERRUN = 4u;
constexpr unsigned ST_TIMEOUT = 8u;

// One box of the level as the kernels see it.
struct BoxDev {
  int n[3];           // valid extents
  int N[3];           // extents with ghosts
  long long pref;     // sum of the strides of the boxes before this one:
                      // the box's block in an ncomp field starts at ncomp*pref
  long long stride;   // component stride (padded volume, multiple of 32)
  double dx[3];
  double idx[3];      // 1/dx
};

// Scheme constants fixed for a plan.
struct SchemeConsts {
  double gamma, gm1, igm1, kshock, small_dens, small_pres, tol, eta_de, cfl, kappa, efloor;
  double tol_mixed;
  int max_iter, grav_corrector;
  int grav_energy;  // S_g in the total energy: 0 rho U . g, 1 kinetic-energy change (Sec. 3.2)
  int plm;          // 1: PLM profiles (Sec. 3.2)
  int linear_rs;    // 1: linearised Riemann solver (Sec. 3.2)
  int flat;         // 1: Colella-Woodward shock flattening (per-cell coefficients)
};

// Scalars of one step, derived on the device from a_old, a_new, dt so that
// a step can be replayed from a CUDA graph without host work.
struct StepConsts {
  double a_old, a_new, dt;
  double a_half, dtp, adot, hdtp, src_u, src_p;
  double ao2, an2, ian, ian2, ahdt, dta, expn, hdt;
};

// Per-box step scalars.
struct BoxStep {
  double dtdx[3];   // dt'/dx_d
  double cdt3[3];   // dt'/(3 dx_d): theta = 1/3 transverse coefficient
  double chalf[3];  // dt'/2 / dx_d: theta = 1/2 final coefficient
};

// Ghost-fill copy rectangle: dst local (dlo + ijk) <- src local (slo + sstep*ijk).
struct FillRect {
  int dst_box, src_box;
  int dlo[3], ext[3], slo[3], sstep[3];
};

// Work item of the fused persistent kernel: a TX x TY column tile of a box.
// Output tile of the shock-flattening pass: columns [x0, x0+nx) x [y0, y0+ny)
// of one box, local coordinates (-1 and n are the one-cell halo); nx <= 34,
// ny <= 17.
struct FlatTile {
  int box, x0, y0, nx, ny;
};

struct WorkItem {
  int box;
  int x0, y0;
  int nx, ny;     // tile extent (<= TX, TY at the box edge)
  int z0, nz;     // planes [z0, z0 + nz) of the box (the task form; whole columns otherwise)
  int pad;
};

__device__ __forceinline__ long long cell_index(const BoxDev &b, int i, int j, int k) {
  // local valid coordinates (may be negative in the ghosts)
  return ((long long)(k + 4) * b.N[1] + (j + 4)) * b.N[0] + (i + 4);
}

// Positive doubles order like their bit patterns as unsigned 64-bit ints.
__device__ __forceinline__ void atomic_min_pos(unsigned long long *acc, double v) {
  atomicMin(acc, (unsigned long long)__double_as_longlong(v));
}

}  // namespace nyx
