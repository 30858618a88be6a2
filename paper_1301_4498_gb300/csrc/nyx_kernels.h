// nyx_kernels.h -- host launchers of the kernels of libnyxhydro.so.
#pragma once
#include <cuda_runtime.h>

#include "nyx_internal.cuh"

namespace nyx {

// Set the message nyx_last_error() returns on this thread.
void record_error(const char *msg);

// Valid cells of a level field (6 components) to or from their packed form
// (box b at 6 cell_pref[b], component-major, x fastest); one block per plane
// of each box, plane_pref[b] the first block of box b.  Copies the nblocks
// box planes from block blk0 on (a range of whole boxes, or all of them).
void launch_valid_copy(double *field, double *packed, const BoxDev *boxes,
                       const long long *cell_pref, const int *plane_pref, int nbox, int nblocks,
                       int blk0, int to_field, cudaStream_t st);
int preload_copy_kernels();  // cudaError_t of loading the overlapped host step's copy kernels
void launch_fill(double *field, int ncomp, const BoxDev *boxes, const FillRect *rects,
                 const long long *rect_pref, int nrect, long long total, cudaStream_t st,
                 bool beside = false);

void launch_step_setup(const SchemeConsts *K, const double *a_old, const double *a_new,
                       const double *dt, StepConsts *SC, const BoxDev *boxes, int nbox,
                       BoxStep *BS, cudaStream_t st);

void launch_estdt(const BoxDev *boxes, const long long *cell_pref, int nbox, long long total,
                  const double *state, const SchemeConsts *K, const double *a_dev,
                  unsigned long long *dtacc, cudaStream_t st);

void launch_estdt_mixed(const BoxDev *boxes, const long long *cell_pref, int nbox, long long total,
                        const double *state, const SchemeConsts *K, const double *a_dev,
                        unsigned long long *dtacc, cudaStream_t st);

void launch_dt_finalize(const SchemeConsts *K, unsigned long long *dtacc, double *dt_out,
                        cudaStream_t st);

size_t staged_scratch_doubles(long long V);

void launch_staged_box(const BoxDev &b, const BoxDev *b_dev, const SchemeConsts *K,
                       const StepConsts *SC, const BoxStep *BSb, const double *Sbox,
                       const double *Gbox, const double *FLbox, double *Snbox, double *scratch,
                       long long V, unsigned long long *dtacc, unsigned *status,
                       double *flux_keep, int predict_only, cudaStream_t st);

// Arguments of one launch of the fused persistent advance.
struct FusedArgs {
  const BoxDev *boxes;
  const WorkItem *items;
  int nitems;
  int *queue;                     // work-queue counter (zeroed by the launcher)
  const SchemeConsts *K;
  const StepConsts *SC;
  const BoxStep *BS;
  const double *S;                // state field (6 comps), ghosts filled
  const double *G;                // gravity field (3 comps) or null
  double *Sn;                     // new state field
  unsigned long long *dtacc;      // CFL min accumulator, or null
  unsigned *status;
  double *flux_keep;              // final-flux store, or null
  const long long *flux_off;      // per-box offsets into flux_keep
  int predict_only;               // 1: Step 2 only (no corrector, no dual-energy sync, no dt)
  int variant;                    // scheme variant: bit 0 PLM, bit 1 linearised solver,
                                  // bit 2 shock flattening
  const void *flat;               // shock-flattening coefficients (double for FP64 plans,
                                  // float for mixed ones; one per cell, state layout) or null
  // TMA descriptors (CUtensorMap, one per box, in device memory) of S and G
  // for the tile shape being launched, or null: the kernels that stage
  // their plane inputs with tensor copies fall back to plain loads
  const void *tmS;
  const void *tmG;
};

// Tile shapes of the fused kernel (columns per CTA in x and y).
struct TileShape {
  int tx, ty;
  int task;  // the task form (streams any range of planes) rather than column-owning
};
int fused_num_shapes(int precision);
TileShape fused_shape(int idx);

// Launch the fused advance over all items with the given shape index.
// precision: NYX_FP64 or NYX_MIXED.  Returns a cudaError_t.
int launch_fused(int precision, int shape, const FusedArgs &a, int grid, cudaStream_t st);
int fused_max_grid(int precision, int shape);

int launch_fused_f64(int shape, const FusedArgs &a, int grid, cudaStream_t st);

// Step 6 alone over every valid cell of a level (FP64): the predictor in
// Sp (6 components) is corrected in place with the state at t^n in S, g^n in
// Go and g^{n+1} in Gn (either may be null: zero), then synchronised; the CFL
// minimum of the result goes to dtacc (may be null), formed in FP32 when
// f32_dt (mixed plans) and in FP64 otherwise.
void launch_correct(const BoxDev *boxes, const long long *cell_pref, int nbox, long long total,
                    const SchemeConsts *K, const StepConsts *SC, const double *S, double *Sp,
                    const double *Go, const double *Gn, unsigned long long *dtacc,
                    unsigned *status, bool f32_dt, cudaStream_t st);
int launch_fused_mixed(int shape, const FusedArgs &a, int grid, cudaStream_t st);
int max_grid_f64(int shape);
int max_grid_mixed(int shape);
int launch_flatten_f64(const BoxDev *boxes, const FlatTile *tiles, int ntiles, const double *S,
                       const SchemeConsts *K, void *fl, cudaStream_t st);
int launch_flatten_mixed(const BoxDev *boxes, const FlatTile *tiles, int ntiles, const double *S,
                         const SchemeConsts *K, void *fl, cudaStream_t st);
int flatten_init_f64();
int flatten_init_mixed();
int flat_ones_f64(void *fl, long long n, cudaStream_t st);
int flat_ones_mixed(void *fl, long long n, cudaStream_t st);

// Shock-flattening coefficients of the cells [-1, n]^3 of every box from the
// state S (ghosts filled), in the plan's arithmetic: fl is double for FP64
// plans, float for mixed ones.  tiles: the boxes' [-1, n]^2 columns cut into
// tiles of at most 34 x 17 (one block each).  Return a cudaError_t.
int launch_flatten(int precision, const BoxDev *boxes, const FlatTile *tiles, int ntiles,
                   const double *S, const SchemeConsts *K, void *fl, cudaStream_t st);
// Shared-memory attribute of the flattening kernel (once per process).
int flatten_init(int precision);
// Set the n coefficients of fl to 1.
int launch_flat_ones(int precision, void *fl, long long n, cudaStream_t st);

}  // namespace nyx
