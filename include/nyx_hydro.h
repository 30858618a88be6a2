/*
 * nyx_hydro.h -- C ABI of libnyxhydro.so, the GB300 (sm_103a) single-level
 * comoving gas advance of Nyx (Almgren et al. 2013).
 *
 * The operation is Step 2 (hydro advance) and the hydro part of Step 6
 * (gravity corrector, dual-energy sync) of the single-level algorithm
 * (Sec. 3.6), for the comoving Euler + dual-energy equations of Sec. 2.2 in
 * the discretisation of Sec. 3.2 (unsplit PPM Godunov with characteristic
 * tracing, reference states, full corner coupling, two-shock Riemann
 * solver), over every box of one AMR level (Sec. 4.1), plus the CFL time
 * step of Sec. 3.5.  The nyx_amr_* calls couple two such levels, a fine
 * level refining a coarse one by 2 with no subcycling (Sec. 4.1-4.3):
 * coarse-to-fine interpolation of the fine ghost cells, reflux and average
 * down.
 *
 * Conventions for every entry point:
 *  - Return 0 (NYX_OK) on success or a negative NYX_E* code; the text of
 *    the last error of the calling thread is returned by nyx_last_error().
 *  - Device pointers are plain CUDA device addresses of the current device;
 *    the caller owns every buffer it passes and the library never frees one.
 *  - Work is enqueued on the stream given to nyx_hydro_plan() and is
 *    asynchronous; device-side failures (negative density, non-finite
 *    values) raise a status word that nyx_hydro_status() reads.
 *  - A plan is not thread-safe: one host thread at a time per plan.
 *
 * Level buffers.  A "field" of ncomp components over a level is one device
 * buffer of doubles.  Box b occupies [off[b], off[b+1]) with off from
 * nyx_hydro_layout(); inside it component c is a contiguous array of
 * (nz+2ng)(ny+2ng)(nx+2ng) doubles (x fastest, ghost cells included),
 * starting at off[b] + c*stride[b] (stride[b] is the padded component
 * volume, a multiple of 32 doubles).  The conserved state has 6
 * components (rho, m_x, m_y, m_z, rhoE, rhoe) with m = rho U, not weighted
 * by a (the a, a^2 weights of the paper's U are applied inside the update);
 * gravity has 3 (g_x, g_y, g_z).
 */
#ifndef NYX_HYDRO_H
#define NYX_HYDRO_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

#define NYX_OK 0
#define NYX_EINVAL (-1)    /* bad descriptor, parameter or pointer */
#define NYX_ECUDA (-2)     /* a CUDA call failed */
#define NYX_ENEGATIVE (-3) /* device flag: density <= 0 after an update */
#define NYX_ENONFINITE (-4) /* device flag: NaN/Inf in an updated state */
#define NYX_ETIMEOUT (-5)  /* device flag: a bounded device wait gave up */
#define NYX_ENOMEM (-6)    /* device allocation failed */

#define NYX_BC_PERIODIC 0
#define NYX_BC_OUTFLOW 1   /* zero-gradient extrapolation */

#define NYX_FP64 0         /* all arithmetic FP64 */
#define NYX_MIXED 1        /* FP32 reconstruction/tracing/Riemann; FP64 state,
                              flux-divergence accumulation and dual-energy sync */

#define NYX_PPM 0          /* edge-state profiles: piecewise parabolic (Sec. 3.2) */
#define NYX_PLM 1          /* piecewise linear, MC-limited slope (Sec. 3.2) */
#define NYX_RS_TWO_SHOCK 0 /* iterative two-shock Riemann solver (Sec. 3.2) */
#define NYX_RS_LINEAR 1    /* linearised approximate Riemann solver (Sec. 3.2) */

#define NYX_PERSISTENT 0   /* one persistent fused launch over all (box, tile) items */
#define NYX_PER_BOX 1      /* plain FP64 stage-by-stage kernels, one box at a time */

/* One grid of the level (Sec. 4.1): inclusive cell bounds lo..hi in the
 * index space of its domain, even cell counts, cell widths dx. */
typedef struct {
  int lo[3], hi[3];
  int domain;
  double dx[3];
} nyx_box;

/* A domain: the region the boxes of one index space tile, with the kind of
 * boundary on its lo x,y,z and hi x,y,z faces.  Boxes of one domain must
 * not overlap; every ghost cell must map (after periodic wrap or outflow
 * clamp) to a valid cell of some box of the same domain. */
typedef struct {
  int lo[3], hi[3];
  int bc[6];
} nyx_domain;

typedef struct {
  int nboxes;
  int ng;                  /* ghost width: must be 4 (PPM stencil + corner coupling) */
  const nyx_box *boxes;    /* host array, copied by nyx_hydro_plan */
  int ndomains;
  const nyx_domain *domains;
} nyx_level_desc;

typedef struct {
  double gamma;            /* gamma-law EOS exponent, p = (gamma-1) rho e (Sec. 2.2) */
  double cfl;              /* CFL factor sigma of Sec. 3.5, 0 < cfl < 1 */
  double small_dens;       /* density floor of edge and Godunov states */
  double small_pres;       /* pressure floor */
  double eta_de;           /* dual-energy threshold (1e-4 in Sec. 3.2 / Step 6) */
  int riemann_max_iter;    /* two-shock iteration cap */
  double riemann_tol;      /* relative pressure tolerance (1e-10 FP64, 1e-6 mixed) */
  int precision;           /* NYX_FP64 or NYX_MIXED */
  int grav_corrector;      /* 1: Step 6 gravity corrector */
  int batching;            /* NYX_PERSISTENT or NYX_PER_BOX */
  int autotune;            /* 1: tune the tile shape per box-size class (nyx_hydro_tune_info) */
  int keep_fluxes;         /* 1: keep the final fluxes of the last advance */
  int coarse_fine;         /* 1: the level is the fine level of a nyx_amr pair: ghost
                              cells that no box of the level covers are left to
                              nyx_amr_interp (coarse data, Sec. 4.3 Step 2) instead
                              of being an error */
  int grav_energy;         /* gravity source of the total energy (Sec. 3.2): 0 the
                              product of the cell-centred momentum and g; 1 the change
                              of the kinetic energy that the momentum's gravity update
                              makes (leaves e = E - U^2/2 to the hydro update) */
  int reconstruction;      /* NYX_PPM or NYX_PLM; both trace with the reference state of
                              Sec. 3.2 (the average of the profile over the domain of
                              dependence of the fastest wave toward the face) */
  int riemann_solver;      /* NYX_RS_TWO_SHOCK or NYX_RS_LINEAR (acoustic p*, u* without
                              iteration; star density from dp = c^2 d rho) */
  int flattening;          /* 1: Colella-Woodward shock flattening of the profiles (the
                              PPM that Sec. 3.2 cites): a cell in a steep, converging
                              pressure jump (or next to one, on its low-pressure side)
                              has its profiles pulled toward the cell value.  Costs one
                              extra pass over the level per advance and, per plan, one
                              value per cell (FP64 plans double, mixed plans float). */
  int z_chunks;            /* 1: the fused kernel may cut columns into chunks of planes to
                              even out the CTAs' loads (nyx_task_items), for example when a
                              single box has fewer column tiles than the GPU has SMs; 0 keeps
                              whole columns.  Either gives the same result, bit for bit. */
} nyx_hydro_params;

typedef struct nyx_plan nyx_plan;

/* Caller-owned device buffers of one level: two state versions (a stencil
 * cannot update in place), gravity (may be NULL for g = 0), and which
 * state version is current.  nyx_hydro_advance flips cur. */
typedef struct {
  double *state[2];
  const double *grav;
  int cur;
} nyx_level;

/* Fill *params with the defaults (gamma 5/3, cfl 0.5, small_dens 1e-10,
 * small_pres 1e-12, eta_de 1e-4, 12 iterations, tol 1e-10, FP64,
 * corrector on, persistent, autotune off, keep_fluxes off, coarse_fine off,
 * grav_energy 0, PPM, two-shock solver, no flattening, z_chunks 1). */
void nyx_hydro_default_params(nyx_hydro_params *params);

/* Validate the level (Sec. 4.1: even positive extents, ng == 4, boxes of a
 * domain disjoint and covering every ghost cell's image), copy it to the
 * device, build the ghost-fill copy list and the batched work list, and
 * allocate the plan's scratch.  stream: a cudaStream_t (NULL = legacy
 * default stream).  *out receives the plan; NYX_EINVAL / NYX_ENOMEM /
 * NYX_ECUDA on failure (no plan is returned). */
int nyx_hydro_plan(const nyx_level_desc *level, const nyx_hydro_params *params,
                   void *stream, nyx_plan **out);

/* Offsets (in doubles) of each box's block in a field of ncomp components:
 * off has nboxes+1 entries, off[nboxes] = total doubles to allocate.
 * stride (nboxes entries, may be NULL) receives the component stride. */
int nyx_hydro_layout(const nyx_plan *plan, int ncomp, size_t *off, size_t *stride);

/* Fill the ghost cells of every box of a level field in place (ghost
 * exchange of Sec. 4.1): copy from the box covering the same point after
 * periodic wrap; zero-gradient copy across outflow faces.  Used by the
 * advance on the state; callers use it once on gravity. */
int nyx_hydro_fill(nyx_plan *plan, double *field, int ncomp);

/* CFL time step of Sec. 3.5 for state[cur]:
 *   *dt_dev = cfl * min over valid cells and d of a dx_d / (|U_d| + c)
 * a_dev and dt_dev are device scalars (so the call can be graph captured).
 * FP64 plans evaluate it in FP64, mixed plans in FP32. */
int nyx_hydro_estdt(nyx_plan *plan, const nyx_level *level, const double *a_dev, double *dt_dev);

/* One single-level hydro advance (Sec. 3.6 Steps 2 and 6, hydro part):
 * ghost fill of state[cur], then state[1-cur] (valid cells) =
 * advance(state[cur], g) from a_old to a_new over dt, then cur flips.
 * a_old_dev, a_new_dev, dt_dev: device scalars.  grav_dev: device field of
 * 3 components with ghosts filled; when NULL, level->grav is used, and
 * when that is NULL too, g = 0.  dt_next_dev (may be NULL): receives the
 * CFL step of the new state at a_new, computed in the same pass. */
int nyx_hydro_advance(nyx_plan *plan, nyx_level *level, const double *a_old_dev,
                      const double *a_new_dev, const double *dt_dev, const double *grav_dev,
                      double *dt_next_dev);

/* Step 2 alone (Sec. 3.6), for a caller that recomputes gravity at t^{n+1}
 * (Step 4) before the corrector: ghost fill of state[cur], then
 * state[1-cur] (valid cells) = the predictor U^{n+1,*} of state[cur] with
 * grav_old (g^n; NULL: level->grav, NULL again: g = 0) -- the advance without
 * the gravity corrector and without the dual-energy sync.  cur does not
 * flip.  Scalars are device pointers. */
int nyx_hydro_predict(nyx_plan *plan, nyx_level *level, const double *a_old_dev,
                      const double *a_new_dev, const double *dt_dev, const double *grav_old_dev);

/* Step 6 alone (Sec. 3.6): state[1-cur], a predictor from nyx_hydro_predict
 * with the same scalars, gets the gravity corrector with g^n (grav_old_dev)
 * and g^{n+1} (grav_new_dev) -- in the energy discretisation of the plan's
 * grav_energy -- then the dual-energy sync, in place (FP64 for every plan);
 * cur flips.  Gravity fields are device fields of 3 components (valid cells
 * read; NULL = zero).  dt_next_dev (may be NULL) receives the CFL step of
 * the new state at a_new (FP32 for mixed plans, as nyx_hydro_estdt).  With
 * grav_new = grav_old the pair gives the
 * result of nyx_hydro_advance (bitwise for FP64 plans). */
int nyx_hydro_correct(nyx_plan *plan, nyx_level *level, const double *a_old_dev,
                      const double *a_new_dev, const double *dt_dev, const double *grav_old_dev,
                      const double *grav_new_dev, double *dt_next_dev);

/* nsteps advances back to back.  a_dev holds a_0..a_nsteps; dt_dev holds
 * nsteps+1 scalars: dt_dev[0] is the first step's dt (computed here by
 * nyx_hydro_estdt if compute_dt0 != 0) and step s writes dt_dev[s+1].
 * use_graph != 0 captures the sequence once into a CUDA graph (kept in the
 * plan, keyed by the pointers and nsteps) and replays it.  On a persistent
 * plan whose level has enough work items (4 waves or more) the boxes are cut
 * into the groups of nyx_hydro_step_host_valid (made on the first call):
 * every step runs one advance launch per group, and each group's ghost fill
 * of the next step starts as soon as the groups it reads have advanced,
 * beside the other groups' advances (a flattening plan's coefficient pass
 * then runs over the whole level before the step's advances).  The result is
 * that of nsteps calls of nyx_hydro_advance, bit for bit (a plan with
 * profiling on keeps one fill and one advance launch per step). */
int nyx_hydro_run(nyx_plan *plan, nyx_level *level, const double *a_dev, double *dt_dev,
                  int nsteps, int compute_dt0, int use_graph);

/* Final Godunov fluxes of the last advance through box `box` in direction
 * dir (0,1,2): raw fluxes F (per unit area and time, not scaled by a or
 * dt; reflux of Sec. 4.3 Step 8 scales them), components (rho, m_x, m_y,
 * m_z, rhoE, rhoe), each an (n_d+1) x (other extents) array, x fastest,
 * in out (device, 6 * (n_x+(d==0)) (n_y+(d==1)) (n_z+(d==2)) doubles).
 * Needs keep_fluxes = 1 in the plan's parameters. */
int nyx_hydro_fluxes(nyx_plan *plan, const nyx_level *level, int box, int dir, double *out);

/* End-to-end step with HOST buffers: copy host_state_in (a whole level
 * field of 6 components, layout as above, ghosts need not be filled) to
 * state[cur], advance one step (dt from *dt_inout when > 0, else the CFL
 * step of the input at a_old), copy the new state to host_state_out and the
 * next step's CFL dt to *dt_inout.  Gravity is level->grav, resident on
 * the device.  Synchronous.  Pinned host buffers give the full copy rate. */
int nyx_hydro_step_host(nyx_plan *plan, nyx_level *level, const double *host_state_in,
                        double *host_state_out, double a_old, double a_new, double *dt_inout);

/* The same end-to-end step with the level's VALID cells only on the host
 * (ghost cells are derived data, about 40 % of a field with 4-cell ghosts
 * on 32^3 boxes): host_in and host_out hold, box after box, the 6 components
 * of the box's n_x n_y n_z valid cells (component-major, x fastest; box b
 * starts at 6 times the number of valid cells of the boxes before it).  The
 * copies go through a device staging buffer of the same size, made on the
 * first call (NYX_ENOMEM if it cannot be); the scatter into and the gather
 * from the level's state run on the device.  On a persistent plan whose
 * level has enough work items, the boxes are cut into up to 32 groups: each
 * group's new cells are copied out while later groups advance, and, when
 * *dt_inout > 0, each group's cells are copied in while earlier groups
 * fill, flatten (flattening plans) and advance.  The library's own
 * streams for this wait on the plan's stream first.  The result is the same
 * either way.  The overlap needs pinned host buffers (pageable ones are
 * copied correctly, but each copy then holds the calling thread).  host_in
 * may equal host_out.  Synchronous: every copy has ended when the call
 * returns. */
int nyx_hydro_step_host_valid(nyx_plan *plan, nyx_level *level, const double *host_in,
                              double *host_out, double a_old, double a_new, double *dt_inout);

/* Tile shapes of the fused persistent kernel: shape index -> columns per
 * work item (tx, ty).  Shapes 0-2 are the column-owning form (FP64 and
 * mixed), 3-5 the task form (mixed only).  nyx_hydro_tile_shape returns
 * NYX_EINVAL for an index out of range; nyx_hydro_set_tile_shape fixes the
 * plan's shape (and turns its autotuner off; NYX_EINVAL if the shape does
 * not exist for the plan's precision); nyx_hydro_get_tile_shape reports the
 * shape in use. */
int nyx_hydro_tile_shape(int shape, int *tx, int *ty);
int nyx_hydro_set_tile_shape(nyx_plan *plan, int shape);
int nyx_hydro_get_tile_shape(const nyx_plan *plan, int *shape);

/* The autotuner of a persistent plan (params.autotune = 1; runs before the
 * first advance, outside any stream capture).  Analogue of the paper's
 * knapsack / space-filling-curve distribution of grids over processors
 * (Sec. 5.1), which balances work by box size: the level's boxes are grouped
 * into box-size classes (equal extents), and each class gets the tile shape
 * and resident CTAs per SM that run one full wave of its work items in the
 * least time per zone.  Classes with the same choice share one launch; the
 * advance makes one launch per distinct choice.  Choices are kept in a JSON
 * file keyed by GPU name, SM count, precision, scheme variant and box extent
 * -- $NYX_TUNE_CACHE if set (empty: no file), else _tune_cache.json beside
 * libnyxhydro.so -- and a class found there is not timed again.  After the
 * tuning, *classes receives the number of box-size classes, *trials the
 * trial launches it made (0: every class came from the file) and *launches
 * the fused launches of one advance.  Any output pointer may be NULL.
 * NYX_EINVAL for a null plan. */
int nyx_hydro_tune_info(const nyx_plan *plan, int *classes, int *trials, int *launches);

/* Work list of the fused persistent kernel for a level of nbox boxes with
 * interior extents n[3b], n[3b+1], n[3b+2] (x, y, z) and column tiles of
 * tx x ty, run on `slots` resident CTAs that take items from one queue.
 * Host only: it needs no GPU and no plan, and is the list a plan builds.
 * Each item is 7 ints (box, x0, y0, nx, ny, z0, nz): cells [x0, x0+nx) x
 * [y0, y0+ny) x [z0, z0+nz) of the box; the items tile every box once.
 * chunk = 0 keeps every column whole; chunk != 0 lets the list cut columns
 * along z into chunks when that evens out the CTAs' loads (the plans' lists,
 * for every tile shape, with z_chunks = 1).  Items come in queue order, the
 * largest first.  Writes min(cap, *count) items to `items` (caller-owned,
 * 7 * cap ints) and the full count to *count.  NYX_EINVAL for a negative
 * size, an empty box, tx, ty or slots below 1, or a null pointer. */
int nyx_task_items(int nbox, const int *n, int tx, int ty, int slots, int chunk, int *items,
                   int cap, int *count);

/* Counters of the plan: kernel launches it enqueued (graph replays count
 * the kernels of the graph), and, while profiling is on, the summed CUDA
 * event durations of its ghost fills and of its advance kernels (eager
 * calls only; graph replays are not split by kernel).  read synchronises
 * the stream; reset != 0 zeroes the counters after reading. */
typedef struct {
  long long launches;
  long long timed_fills, timed_advances;
  double fill_ms, advance_ms;
  long long timed_flattens;  /* shock-flattening passes (flattening plans) */
  double flatten_ms;
} nyx_hydro_counters;
int nyx_hydro_profile(nyx_plan *plan, int enable);
int nyx_hydro_counters_read(nyx_plan *plan, int reset, nyx_hydro_counters *out);

/* Synchronise the plan's stream, read and clear the device status word.
 * *flags (may be NULL) receives its bits (1 negative density, 2 non-finite,
 * 4 queue overrun, 8 timeout).  Returns NYX_OK, or the NYX_E* code of the
 * most severe raised bit. */
int nyx_hydro_status(nyx_plan *plan, int *flags);

/* Allocation-free CFL step (no counterpart in the paper: it serves callers,
 * not the method).  Same result as nyx_hydro_estdt of an FP64 plan, for a state
 * laid out as nyx_hydro_layout describes, but without a plan: it calls no cudaMalloc,
 * cudaFree or allocating library routine.  It is for callers that cannot
 * allocate device memory -- code running where a framework or application
 * owns every device allocation, or a latency-critical loop that must not
 * enter the allocator.
 *  - Scratch: one file-scope __device__ array of fixed size (box table for up
 *    to NYX_NOALLOC_MAX_BOXES boxes, cell offsets, the min accumulator and
 *    the scheme constants, about 0.4 MB), held by every GPU that loads the
 *    library until the process exits.  Levels with more boxes are rejected
 *    with NYX_EINVAL.
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *    Every call copies its tables from host memory, and a call whose stream
 *    is capturing is rejected with NYX_EINVAL.
 *  - Every call shares the array and leaves its contents behind; each call
 *    rewrites the tables and resets the accumulator before use.  Calls that
 *    overlap on the GPU (other streams, other host threads) race.
 *  - A non-finite or non-positive dx, gamma <= 1, or a non-finite gamma, cfl
 *    or small_pres is rejected with NYX_EINVAL, as nyx_hydro_plan does.
 *  - level, params: host descriptors as for nyx_hydro_plan (ng must be 4).
 *    state: device field of 6 components.  a_dev, dt_dev: device scalars.
 *    stream: a cudaStream_t (NULL = legacy default stream).  Asynchronous
 *    apart from the staging of the tables; errors as elsewhere. */
#define NYX_NOALLOC_MAX_BOXES 4096
int nyx_hydro_estdt_noalloc(const nyx_level_desc *level, const nyx_hydro_params *params,
                            const double *state, const double *a_dev, double *dt_dev,
                            void *stream);

/* Release the plan's device and host resources (not the caller's buffers). */
int nyx_plan_destroy(nyx_plan *plan);

/* Measured fused multiply-add throughput of the current device (no
 * counterpart in the paper: it gives the ALU denominators of the roofline
 * against which the advance is reported).  pipe 0: FP32, 1: FP64.  Runs
 * independent multiply-add chains on every SM for about `seconds` in total
 * (0 < seconds <= 10) on `stream`, synchronising with it, and stores the best
 * rate of five timed launches in *fma_per_s (lane operations per second; one
 * FMA is two floating-point operations).  Allocates nothing on the device.
 * NYX_EINVAL for a bad argument, NYX_ECUDA if a launch or event fails. */
int nyx_alu_peak(int pipe, double seconds, void *stream, double *fma_per_s);

/* ---------------------------------------------------------------- self-gravity
 * The Poisson equation of Sec. 3.4 on one level that tiles a single periodic
 * domain (even extents, equal cubic cells):
 *     L phi = four_pi_G / a (rho - mean rho),
 * L the 7-point Laplacian on cell centres, solved by geometric multigrid
 * (V-cycles with red-black Gauss-Seidel: red cells i+j+k even first; mean
 * restriction of the residual, piecewise-constant prolongation; coarsening
 * while every extent is a multiple of 4 and >= 2 min_size; coarse_sweeps
 * sweeps on the coarsest grid) until max|f - L phi| <= tol max|f|, then
 * g = -grad phi by centred differences between adjacent cell centres.  The
 * solve runs on the dense grid of the domain (gathered from the boxes); the
 * object keeps phi for a warm start.  rho is the gas density (component 0
 * of the state) plus the dark matter's dense density when one is given. */
typedef struct nyx_poisson nyx_poisson;
typedef struct {
  double tol;         /* relative max-norm residual (1e-12) */
  int max_cycles;     /* V-cycle cap (50) */
  int pre, post;      /* red-black sweeps before / after the coarse correction (2, 2) */
  int coarse_sweeps;  /* sweeps on the coarsest grid (40) */
  int min_size;       /* smallest coarse extent (2) */
  double four_pi_G;   /* 4 pi G in code units (1) */
  int precision;      /* NYX_FP64 (default): every operation in FP64.  NYX_MIXED:
                         iterative refinement, each cycle an FP64 residual, one
                         FP32 V-cycle on the correction equation from zero, and
                         an FP64 update of phi; the stopping test on that
                         FP64 residual, rounded to float */
} nyx_poisson_params;

void nyx_poisson_default_params(nyx_poisson_params *params);

/* Check the plan's level and allocate the grids (about 2.3 doubles per
 * cell).  NYX_EINVAL if the level cannot be solved this way. */
int nyx_poisson_create(nyx_plan *plan, const nyx_poisson_params *params, nyx_poisson **out);

/* Solve for the state (device field, 6 components, rho first) plus rho_dm
 * (dense device grid of the domain, x fastest; NULL = no dark matter) at
 * scale factor a (host scalar).  grav_out (may be NULL): device level field
 * of 3 components receiving g, ghosts filled by the plan's fill.
 * g_dense_out (may be NULL): 3 consecutive dense grids receiving g (for the
 * particles).  warm_start != 0 starts from the previous phi, else from
 * zero.  Synchronous: it reads the residual after every V-cycle.
 * *cycles_out, *resid_out (may be NULL): V-cycles taken and the final
 * relative residual.  NYX_ETIMEOUT if max_cycles did not reach the
 * tolerance (g is still written). */
int nyx_poisson_solve(nyx_poisson *ps, const double *state, const double *rho_dm, double a,
                      double *grav_out, double *g_dense_out, int warm_start, int *cycles_out,
                      double *resid_out);

/* Dark matter as particles (Sec. 3.3-3.6) on the dense periodic grid of a
 * nyx_poisson object (n cells of width dx per axis; positions in [0, n dx)).
 * Device SoA arrays: x[3 np] (comoving positions), u[3 np] (peculiar proper
 * velocities), m[np].  Cloud in cell: a particle is a cube of side dx; the
 * 8 cells it overlaps get its mass in proportion to the overlap / dx^3, and
 * the same weights interpolate g to it (no self-force with the centred g).
 *  - deposit: rho_dm (dense) = the particles' density (zeroed first;
 *    floating-point atomics, so the summation order is not fixed);
 *  - kick_drift (Step 3): u = (a_old u + dt/2 g^n(x)) / a_half, then
 *    x += dt u / a_half, wrapped into the domain (one period at most);
 *  - kick (Step 5): u = (a_half u + dt/2 g^{n+1}(x)) / a_new;
 *  - estdt (Sec. 3.5): *dt_dev = min(cfl_dm a dx / max |u_d|,
 *    sqrt(dx / max |g_d|)) over the particles (+inf if both maxima are 0);
 *  - kick_estdt: kick, then estdt of the kicked particles at a = a_new with
 *    the g^{n+1} the kick used (the next step's particle dt), in one pass.
 * The kernels multiply by reciprocals and use fused multiply-adds, so they
 * match a plain evaluation of these formulas to round-off.
 * Stream-ordered on the plan's stream; scalars are host doubles. */
int nyx_pm_deposit(nyx_poisson *ps, const double *x, const double *m, long long np,
                   double *rho_dm);
int nyx_pm_kick_drift(nyx_poisson *ps, double *x, double *u, long long np, const double *g_dense,
                      double a_old, double a_half, double dt);
int nyx_pm_kick(nyx_poisson *ps, const double *x, double *u, long long np, const double *g_dense,
                double a_half, double a_new, double dt);
int nyx_pm_estdt(nyx_poisson *ps, const double *x, const double *u, long long np,
                 const double *g_dense, double a, double cfl_dm, double *dt_dev);
int nyx_pm_kick_estdt(nyx_poisson *ps, const double *x, double *u, long long np,
                      const double *g_dense, double a_half, double a_new, double dt,
                      double cfl_dm, double *dt_dev);

/* Copy phi (dense, x fastest, domain extents) to a device buffer. */
int nyx_poisson_phi(nyx_poisson *ps, double *phi_out);

int nyx_poisson_destroy(nyx_poisson *ps);

/* ---------------------------------------------------------------- two levels
 * Coarse-fine coupling of Sec. 4.1-4.3 for a refinement ratio of 2 and no
 * subcycling (both levels take the same dt, Sec. 4.2).
 *  - Hierarchy: the fine plan's domain k refines the coarse plan's domain k
 *    (fine lo = 2 coarse lo, fine hi = 2 coarse hi + 1), every domain face
 *    periodic; fine boxes start and end on coarse cell boundaries (even lo,
 *    odd hi).  The coarse level must cover its domains (a plain plan), the
 *    fine plan is made with coarse_fine = 1; both with keep_fluxes = 1, the
 *    same precision and the same stream.
 *  - Interpolation (Sec. 4.1): in each coarse cell a linear profile with the
 *    MC-limited slope along each axis (from the two face neighbours), all
 *    three slopes scaled by one factor so that no fine value leaves the
 *    range of the coarse cell and its six face neighbours; the fine value is
 *    the profile at the fine cell centre (the 8 fine cells average to the
 *    coarse value).  Each component separately.
 *  - Reflux (Sec. 4.3 Steps 2 and 8): a coarse cell outside the fine level
 *    that shares a face with it has that face's coarse flux replaced by the
 *    mean of the 4 fine fluxes, with the update's coefficients (dt/a_h for
 *    rho, dt/a_new for m, a_h dt/a_new^2 for rhoE and rhoe).  The gravity
 *    corrector, pdV and dual-energy terms are not redone.
 *  - Average down (Sec. 4.3 Step 8): a coarse cell under the fine level
 *    takes the mean of its 8 fine cells (every component).
 * The amr object keeps both plans (which the caller still owns and must
 * destroy after it) and its own device tables. */
typedef struct nyx_amr nyx_amr;

#define NYX_AMR_GHOSTS 0   /* fine ghost cells that no fine box covers */
#define NYX_AMR_ALL 1      /* every cell of every fine box (initial data) */

/* Check the pair and build the interpolation, reflux and average-down
 * tables.  NYX_EINVAL if the plans do not form such a hierarchy. */
int nyx_amr_create(nyx_plan *coarse, nyx_plan *fine, nyx_amr **out);

/* Interpolate a coarse field (device, ncomp components, coarse layout, its
 * ghost cells filled) into a fine field (fine layout).  region
 * NYX_AMR_GHOSTS writes the fine ghost cells -- all of them; the fine
 * plan's nyx_hydro_fill (or its advance) then overwrites those another fine
 * box covers; NYX_AMR_ALL writes every cell of every fine box. */
int nyx_amr_interp(nyx_amr *amr, const double *coarse_field, double *fine_field, int ncomp,
                   int region);

/* Reflux the coarse state coarse_new (device, 6 components) with the
 * fluxes and step scalars of the last advance of each plan. */
int nyx_amr_reflux(nyx_amr *amr, double *coarse_new);

/* Average the fine field (ncomp components) down onto the coarse field. */
int nyx_amr_average_down(nyx_amr *amr, const double *fine_field, double *coarse_field,
                         int ncomp);

/* Shared CFL step of both levels: *dt_dev = min of nyx_hydro_estdt over the
 * coarse and the fine state[cur] at a. */
int nyx_amr_estdt(nyx_amr *amr, const nyx_level *coarse, const nyx_level *fine,
                  const double *a_dev, double *dt_dev);

/* One two-level step (Sec. 4.3 Advance(0) with no subcycling): advance the
 * coarse level (Steps 2 and 6, its own ghost fill first); interpolate the
 * fine ghost cells from the coarse state at t^n; advance the fine level (its
 * fine-fine ghost copies first); reflux and average down into the new
 * coarse state.  Both levels' cur flip.  Gravity: each level's grav (ghosts
 * filled; the fine one e.g. by nyx_amr_interp with NYX_AMR_ALL).
 * dt_next_dev (may be NULL) receives nyx_amr_estdt of the new states at
 * a_new.  Scalars are device pointers. */
int nyx_amr_step(nyx_amr *amr, nyx_level *coarse, nyx_level *fine, const double *a_old_dev,
                 const double *a_new_dev, const double *dt_dev, double *dt_next_dev);

/* nsteps two-level steps, like nyx_hydro_run (a_dev: nsteps+1 scale
 * factors; dt_dev: nsteps+1 scalars, dt_dev[0] computed here when
 * compute_dt0 != 0); use_graph != 0 captures them once into a CUDA graph. */
int nyx_amr_run(nyx_amr *amr, nyx_level *coarse, nyx_level *fine, const double *a_dev,
                double *dt_dev, int nsteps, int compute_dt0, int use_graph);

/* Release the amr object (not the plans or the caller's buffers). */
int nyx_amr_destroy(nyx_amr *amr);

/* Message of the last failing call on this thread ("" if none). */
const char *nyx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
