// nyx_plan.h -- the plan object of libnyxhydro.so and the host helpers the
// translation units share (level advance, ghost fill, CFL reduction).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "nyx_hydro.h"
#include "nyx_internal.cuh"

namespace nyx {
namespace host {

struct FillPass {
  FillRect *d_rects = nullptr;
  long long *d_pref = nullptr;
  int n = 0;
  long long total = 0;
  std::vector<FillRect> h;  // host copy (regrouped for the pipelined host step)
};

using GraphKey = std::tuple<const void *, const void *, const void *, int, const void *, const void *,
                            int, int>;

// Set the thread's last error and return code.
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

}  // namespace host
}  // namespace nyx

#define CK(call)                                                       \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return nyx::host::cuda_fail(e_, #call);     \
  } while (0)

struct nyx_plan {
  int nbox = 0;
  std::vector<nyx_box> boxes;
  std::vector<nyx_domain> doms;
  nyx_hydro_params prm{};
  cudaStream_t stream = nullptr;
  std::vector<nyx::BoxDev> hbox;
  std::vector<long long> cell_pref;
  long long total_cells = 0;
  long long total_stride = 0;
  nyx::BoxDev *d_boxes = nullptr;
  long long *d_cell_pref = nullptr;
  nyx::SchemeConsts hK{};
  nyx::SchemeConsts *d_K = nullptr;
  nyx::StepConsts *d_SC = nullptr;
  nyx::BoxStep *d_BS = nullptr;
  unsigned long long *d_dtacc = nullptr;
  unsigned *d_status = nullptr;
  unsigned *d_status_tune = nullptr;  // status of autotuner launches (never reported)
  double *d_scal = nullptr;  // host-call scalars: a_old, a_new, dt, dt_next
  nyx::host::FillPass pass[4];
  // shock flattening: one coefficient per cell (double for FP64 plans, float
  // for mixed ones), set per advance on the boxes' [-1, n]^3 by one block
  // per tile of output columns
  void *d_flat = nullptr;
  nyx::FlatTile *d_flat_tiles = nullptr;
  int flat_ntiles = 0;
  std::vector<int> flat_tile_pref;  // first tile of each box (tiles come box by box), nbox + 1
  // packed valid cells of a state (nyx_hydro_step_host_valid), made on
  // first use: 6 doubles per valid cell, one copy block per box plane
  double *d_packed = nullptr;
  int *d_plane_pref = nullptr;
  std::vector<int> plane_pref;
  int plane_blocks = 0;
  // ... and its read-back overlapped with the advance: the fused form's
  // items regrouped by box ranges [grp_box[g], grp_box[g+1]) (each group in
  // queue order), one launch per group; a group's cells are gathered and
  // copied to the host on copy_stream while the next group advances
  int ngrp = 0;
  std::vector<int> grp_box;
  std::vector<int> grp_off[8];  // per shape: first item of each group, ngrp + 1 entries
  nyx::WorkItem *d_items_grp[8] = {nullptr};
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> ev_grp;
  // ... and its input overlapped too: each group's cells copied in and
  // scattered on h2d_stream (in in_order), each group's ghost fill (the
  // rects of pass p whose destination is in group g: d_rects_grp[p] from
  // rect_off[p][g]) launched once the groups it reads (grp_src[g], a bit
  // mask) are in
  cudaStream_t h2d_stream = nullptr;
  std::vector<cudaEvent_t> ev_in;
  cudaEvent_t ev_start = nullptr;
  // groups advance on the plan's stream and stream2 in turn (a group's
  // launch takes the SMs its predecessor's tail frees), each with its own
  // work-queue counter
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_setup = nullptr, ev_side = nullptr;
  int *d_queue_grp = nullptr;
  nyx::FillRect *d_rects_grp[4] = {nullptr};
  std::vector<int> rect_off[4];
  std::vector<unsigned> grp_src;
  std::vector<int> in_order;
  std::vector<int> proc_order;  // the order in which the groups advance
  // multi-step runs on the device (nyx_hydro_run): each group's ghost fill
  // of step s+1 runs on one of two fill streams as soon as the groups it
  // reads have advanced in step s, beside the other groups' advances
  cudaStream_t fill_stream[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> ev_gfill, ev_gadv;
  cudaEvent_t ev_fjoin[2] = {nullptr, nullptr};
  // per-box FP64 form
  double *d_scratch = nullptr;
  long long Vmax = 0;
  // final-flux store
  double *d_flux = nullptr;
  std::vector<long long> flux_off;
  long long *d_flux_off = nullptr;
  bool flux_valid = false;
  // fused persistent form.  parts: the autotuner's per-class choice when the
  // box-size classes settle on different (shape, grid) pairs, one launch per
  // part over the boxes of its classes; empty: one launch of `shape` over
  // the level-wide list d_items[shape]
  struct RunPart {
    int shape = 0, grid = 0;
    nyx::WorkItem *d_items = nullptr;
    int nitems = 0;
    std::vector<nyx::WorkItem> h_items;
    nyx::WorkItem *d_items_grp = nullptr;
    std::vector<int> grp_off;  // first item of each read-back group, ngrp + 1 entries
  };
  std::vector<RunPart> parts;
  // TMA descriptors of level fields for the shapes that stage with tensor
  // copies: one CUtensorMap per box, in device memory, keyed by (field
  // address, components, shape); null marks a field that cannot be mapped
  std::map<std::tuple<const void *, int, int>, void *> tmaps;
  int tune_trials = 0;       // trial launches of the last tuning (0: every class from the cache)
  int tune_classes = 0;      // box-size classes of the level
  nyx::WorkItem *d_items[8] = {nullptr};
  std::vector<nyx::WorkItem> h_items[8];
  int nitems[8] = {0};
  int *d_queue = nullptr;
  int shape = 0;
  bool tuned = false;
  int max_grid[8] = {0};
  std::map<nyx::host::GraphKey, std::pair<cudaGraphExec_t, long long>> graphs;  // graph, kernels in it
  // counters and profiling
  long long launches = 0;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_fill, ev_adv, ev_flat;
};


namespace nyx {
namespace host {

// Ghost fill of a level field, one advance, and the CFL reduction of one
// plan (all enqueued on the plan's stream; see nyx_api.cu).
int plan_fill(nyx_plan *P, double *field, int ncomp);
int plan_advance(nyx_plan *P, nyx_level *L, const double *a_old, const double *a_new,
                 const double *dt, const double *grav, double *dt_next);
// Fold the CFL minimum of a state into the plan's accumulator (no finalise).
void plan_estdt_accumulate(nyx_plan *P, const double *state, const double *a_dev,
                           unsigned long long *acc);
bool plan_capturing(nyx_plan *P);
// Time the tile shapes once (autotuning plans only) on state[cur] of L, its
// ghost cells filled here, with the step scalars a_dev[0], a_dev[1], *dt_dev.
int plan_tune(nyx_plan *P, nyx_level *L, const double *a_dev, const double *dt_dev);

}  // namespace host
}  // namespace nyx
