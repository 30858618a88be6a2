/*
 * nyx_oracle.h -- TEST INFRASTRUCTURE, not product code.
 *
 * Plain, slow FP64 CPU oracle for the single-level comoving gas advance of
 * the Nyx paper (Almgren et al. 2013): Sec. 2.2 (comoving Euler and dual
 * energy equations), Sec. 3.2 (unsplit PPM Godunov with characteristic
 * tracing, reference states, two-shock Riemann solver, dual-energy switch,
 * gravity predictor-corrector), Sec. 3.5 (CFL time step) and Sec. 3.6
 * (Steps 2 and 6 of the single-level algorithm).
 *
 * Only the test suite, the package's smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA
 * path and includes none of its headers.
 *
 * Coarse-fine coupling (orc_amr_*): a fine level refines a coarse level by
 * 2 in every direction with no subcycling (Sec. 4.2; Sec. 4.3: Step 2 with
 * coarse Dirichlet data for the fine ghosts, Step 8 reflux and average
 * down; Sec. 4.1 for the conservative limited linear interpolation).
 *
 * Layout of every box array: ncomp blocks of (nz+2ng)(ny+2ng)(nx+2ng)
 * doubles, x fastest; cell (i,j,k) of the valid region [0,n) sits at
 * ((c*Nz + k+ng)*Ny + j+ng)*Nx + i+ng.  State components: rho, m_x, m_y,
 * m_z, rhoE, rhoe (m = rho U, unweighted by a).  Gravity: g_x, g_y, g_z.
 */
#ifndef NYX_ORACLE_H
#define NYX_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NCONS 6
#define ORC_BC_PERIODIC 0
#define ORC_BC_OUTFLOW 1

typedef struct {
  double gamma;          /* gamma-law EOS exponent (Sec. 2.2) */
  double cfl;            /* hyperbolic CFL factor sigma (Sec. 3.5) */
  double small_dens;     /* density floor */
  double small_pres;     /* pressure floor */
  double eta_de;         /* dual-energy threshold, 1e-4 (Sec. 3.2 / Step 6) */
  int riemann_max_iter;  /* two-shock iteration cap */
  double riemann_tol;    /* relative pressure convergence tolerance */
  int grav_corrector;    /* 1: apply the Step 6 gravity corrector */
  int dual_energy_sync;  /* 1: apply the Step 6 e/E synchronisation */
  int grav_energy;       /* S_g in the total energy (Sec. 3.2): 0 the product of the
                            cell-centred momentum and g; 1 the change of the kinetic
                            energy that the momentum's gravity update makes */
  int reconstruction;    /* edge-state profiles (Sec. 3.2): 0 PPM, 1 PLM; both with the
                            reference-state tracing */
  int riemann_solver;    /* 0 the iterative two-shock solver; 1 the linearised
                            approximate solver (Sec. 3.2 names both) */
  int flattening;        /* 1: Colella-Woodward shock flattening of the profiles
                            (the PPM the scheme of Sec. 3.2 cites); 0 off */
} orc_params;

typedef struct {
  int nbox, ng;
  const int *lo, *hi;     /* nbox*3 each; inclusive cell bounds in the domain index space */
  const int *dom;         /* nbox: domain id of each box */
  const double *dx;       /* nbox*3: cell widths */
  int ndom;
  const int *dom_lo, *dom_hi; /* ndom*3 each, inclusive */
  const int *dom_bc;      /* ndom*6: bc of lo x,y,z then hi x,y,z */
} orc_level;

typedef struct {
  long long floor_rho;    /* Godunov/edge states raised to small_dens */
  long long floor_e;      /* cells whose rhoe was raised to the floor in the sync */
  long long use_e;        /* cells where the sync kept e and re-derived E */
  long long bad;          /* non-positive or non-finite density after the update */
} orc_stats;

/* Ghost fill (periodic copy / zero-gradient outflow / neighbour copy). */
int orc_fill_ghosts(const orc_level *lev, int ncomp, double *const *f);

/* One advance of every box: state_in (ghosts filled unless fill_ghosts=1,
 * in which case they are filled in place) -> valid cells of state_out.
 * grav may be NULL (zero gravity).  flux_out may be NULL; otherwise
 * flux_out[b*3+d] receives box b's final direction-d fluxes, 6 components
 * each laid out as ((c*nz + k)*ny + j)*(nx+1 on d==0 ...) -- see
 * orc_flux_count. */
int orc_advance(const orc_level *lev, const orc_params *p, double *const *state_in,
                double *const *state_out, double *const *grav, double a_old,
                double a_new, double dt, int fill_ghosts, double *const *flux_out,
                orc_stats *stats);

/* Step 6 on its own, for a gravity field recomputed at t^{n+1} (Sec. 3.6:
 * Step 4 solves for g^{n+1} from the predicted density): pred holds the
 * predictor of orc_advance run with grav_corrector = 0 and
 * dual_energy_sync = 0 (valid cells); old the state at t^n.  The corrector
 * with g_old at t^n and g_new at t^{n+1}, then the dual-energy sync (when
 * p->dual_energy_sync), is applied to pred in place.  g_old / g_new may be
 * NULL (zero).  With g_new = g_old this is the corrector of orc_advance. */
int orc_correct(const orc_level *lev, const orc_params *p, double *const *old,
                double *const *pred, double *const *g_old, double *const *g_new, double a_old,
                double a_new, double dt, orc_stats *stats);

/* CFL time step over valid cells at scale factor a (Sec. 3.5). */
double orc_estdt(const orc_level *lev, const orc_params *p, double *const *state, double a);

/* Two-shock solves and Newton iterations since the last reset (all threads). */
void orc_riemann_counts(long long *calls, long long *iters, int reset);

/* ---- coarse-fine coupling, refinement ratio 2 (Sec. 4.1-4.3) ----------
 * Fine domain k refines coarse domain k: dom_lo_f = 2 dom_lo_c, dom_hi_f =
 * 2 dom_hi_c + 1, every face periodic.  Fine boxes start and end on coarse
 * cell boundaries (even lo, odd hi).  Returns 0, or -1 if the pair is not
 * such a hierarchy. */
int orc_amr_check(const orc_level *C, const orc_level *F);

/* Conservative limited linear interpolation (Sec. 4.1) of the coarse field
 * cf (ghosts filled) into the fine field ff.  region 0: every cell of every
 * fine box, valid and ghost; region 1: the fine ghost cells only -- a ghost
 * cell that lies in the valid region of a fine box (after periodic wrap)
 * takes that cell's value, every other one is interpolated. */
int orc_amr_interp(const orc_level *C, int ncomp, double *const *cf, const orc_level *F,
                   double *const *ff, int region);

/* Reflux (Sec. 4.3, Steps 2 and 8): every coarse cell outside the fine level that
 * shares a face with it gets the difference between the area average of the
 * fine fluxes on that face and its own coarse flux, with the coefficients
 * of the update (a_old, a_new, dt as given to orc_advance).  cflux / fflux
 * are the flux_out arrays of the two advances (box*3 + dir). */
int orc_amr_reflux(const orc_level *C, double *const *cstate, double *const *cflux,
                   const orc_level *F, double *const *fflux, double a_old, double a_new,
                   double dt);

/* Average down (Sec. 4.3, Step 8): every coarse cell under the fine level
 * takes the mean of its 8 fine cells, all ncomp components. */
int orc_amr_average_down(const orc_level *C, int ncomp, double *const *cstate,
                         const orc_level *F, double *const *fstate);

/* ---- self-gravity (Sec. 3.4): periodic 7-point Poisson, multigrid ------
 * The level's boxes must tile one periodic domain (even extents) with equal
 * cubic cells;
 * the solve runs on the dense grid of the domain (x fastest).  RHS f =
 * four_pi_G / a * (rho - mean rho) (no dark matter).  V-cycles with
 * red-black Gauss-Seidel (red: i+j+k even, first), average restriction,
 * piecewise-constant prolongation, a fixed number of sweeps on the
 * coarsest grid; stop when max|f - L phi| <= tol max|f|.  phi (dense,
 * in/out) is the initial guess (warm start) and the result; grav_out (per
 * box, valid cells; may be NULL) receives g = -grad phi by centred
 * differences.  rho_dm (dense, may be NULL) is added to the gas density. */
typedef struct {
  double tol;             /* relative max-norm residual, 1e-12 */
  int max_cycles;         /* V-cycle cap */
  int pre, post;          /* red-black sweeps before / after the coarse correction */
  int coarse_sweeps;      /* sweeps on the coarsest grid */
  int min_size;           /* coarsen while every extent is a multiple of 4 and >= 2 min_size */
  double four_pi_G;       /* 4 pi G in code units */
} orc_poisson_params;

typedef struct {
  int cycles;             /* V-cycles taken */
  double resid;           /* final max|f - L phi| / max|f| */
  double rho_mean;        /* the mean density subtracted */
} orc_poisson_stats;

int orc_poisson_solve(const orc_level *lev, const orc_poisson_params *p, double *const *state,
                      const double *rho_dm, double a, double *phi, double *const *grav_out,
                      double *g_dense, orc_poisson_stats *st);

/* ---- dark matter (Sec. 3.3-3.6): particles on the dense periodic grid --
 * n cells of width dx per axis, positions in [0, n dx); SoA arrays x[3*np],
 * u[3*np] (comoving position, peculiar proper velocity), m[np]; dense
 * fields x fastest, g as 3 consecutive dense arrays.  rho_dm (optional in
 * orc_poisson_solve) is added to rho_b on the right-hand side; g_dense
 * (optional) receives g on the dense grid for the particles. */
void orc_pm_deposit(const int n[3], double dx, const double *x, const double *m, long long np,
                    double *rho);
void orc_pm_interp(const int n[3], double dx, const double *g, const double *x, long long np,
                   double *gp);
void orc_pm_kick_drift(const int n[3], double dx, const double *g, double *x, double *u,
                       long long np, double a_old, double a_half, double dt);
void orc_pm_kick(const int n[3], double dx, const double *g, const double *x, double *u,
                 long long np, double a_half, double a_new, double dt);
double orc_pm_estdt(const int n[3], double dx, const double *g, const double *x, const double *u,
                    long long np, double a, double cfl_dm);

/* OpenMP threads of the oracle's loops (n <= 0: all host processors). */
void orc_set_threads(int n);

/* Unit-level entry points used by the pin tests. */
void orc_ppm_line(int n, const double *s, double *sL, double *sR, double *s6);
void orc_ppm_integrals(double sL, double sR, double s6, double sigma, double *ip, double *im);
int orc_riemann(const orc_params *p, const double *qL, const double *qR, double *flux8,
                double *pstar, double *ustar);
/* The Godunov state (rho, u_n, u_t1, u_t2, p) at x/t = 0 that the fluxes of
 * orc_riemann are formed from, floors applied. */
int orc_riemann_state(const orc_params *p, const double *qL, const double *qR, double *g5);
void orc_trace_line(const orc_params *p, int n, const double *q5, const double *gline,
                    const double *fl, double dtp, double dx, double adot, int dir, double *qm,
                    double *qp, double *beta_m, double *beta_p);
/* Shock-flattening coefficients of cells 3..n-4 of a line (pressure pr,
 * velocity along the line u); the other entries are set to 1. */
void orc_flatten_line(const orc_params *p, int n, const double *pr, const double *u, double *fl);
/* Shock-flattening coefficient of every cell of every box (fl[b]: the
 * box's volume with ghosts) from the state S with its ghosts filled. */
int orc_flatten_field(const orc_level *L, const orc_params *p, double *const *S,
                      double *const *fl);

#ifdef __cplusplus
}
#endif
#endif
