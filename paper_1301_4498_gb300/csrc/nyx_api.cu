// nyx_api.cu -- host side of libnyxhydro.so: level validation, the ghost-fill
// copy list, the batched work list (largest boxes first, as a knapsack-style
// balance of the paper's Sec. 5.1 distribution), CUDA-graph capture, status
// and the C ABI of include/nyx_hydro.h.
#include <cuda.h>  // CUtensorMap and its enums (the encoder comes through the runtime)
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <map>
#include <queue>
#include <string>
#include <tuple>
#include <vector>

#include "nyx_hydro.h"
#include "nyx_internal.cuh"
#include "nyx_kernels.h"
#include "nyx_plan.h"

using namespace nyx;

namespace {
thread_local std::string g_err;
}  // namespace

namespace nyx {
namespace host {

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(NYX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace host
}  // namespace nyx

using namespace nyx::host;

namespace {

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

bool intersect(const int alo[3], const int ahi[3], const int blo[3], const int bhi[3], int olo[3],
               int ohi[3]) {
  for (int d = 0; d < 3; ++d) {
    olo[d] = std::max(alo[d], blo[d]);
    ohi[d] = std::min(ahi[d], bhi[d]);
    if (olo[d] > ohi[d]) return false;
  }
  return true;
}

// Build the ghost-fill rectangles of every box: pass 0 = copies from boxes
// of the same domain (with periodic images), passes 1..3 = zero-gradient
// outflow along x, y, z.  Returns false (with g_err set) if the ghost cells
// of some box are not covered exactly once.
bool build_fill(const nyx_plan &P, std::vector<FillRect> out[4]) {
  const int ng = 4;
  const int nd = (int)P.doms.size();
  // boxes of each domain and a uniform bin grid per domain
  std::vector<std::vector<int>> dboxes(nd);
  for (int b = 0; b < P.nbox; ++b) dboxes[P.boxes[b].domain].push_back(b);
  struct Bins {
    int bs = 1, nb[3] = {1, 1, 1};
    std::vector<std::vector<int>> cell;
  };
  std::vector<Bins> bins(nd);
  for (int d = 0; d < nd; ++d) {
    const nyx_domain &D = P.doms[d];
    int bs = 1;
    for (int b : dboxes[d])
      for (int a = 0; a < 3; ++a) bs = std::max(bs, P.boxes[b].hi[a] - P.boxes[b].lo[a] + 1);
    Bins &B = bins[d];
    B.bs = bs;
    for (int a = 0; a < 3; ++a) B.nb[a] = (D.hi[a] - D.lo[a] + 1 + bs - 1) / bs;
    B.cell.assign((size_t)B.nb[0] * B.nb[1] * B.nb[2], {});
    for (int b : dboxes[d]) {
      int l[3], h[3];
      for (int a = 0; a < 3; ++a) {
        l[a] = (P.boxes[b].lo[a] - D.lo[a]) / bs;
        h[a] = (P.boxes[b].hi[a] - D.lo[a]) / bs;
      }
      for (int k = l[2]; k <= h[2]; ++k)
        for (int j = l[1]; j <= h[1]; ++j)
          for (int i = l[0]; i <= h[0]; ++i)
            B.cell[((size_t)k * B.nb[1] + j) * B.nb[0] + i].push_back(b);
    }
  }
  std::vector<int> stamp(P.nbox, -1);
  int stamp_id = 0;
  for (int b = 0; b < P.nbox; ++b) {
    const nyx_box &X = P.boxes[b];
    const nyx_domain &D = P.doms[X.domain];
    const Bins &B = bins[X.domain];
    int glo[3], ghi[3], L[3];
    long long ghost = 1, valid = 1;
    for (int a = 0; a < 3; ++a) {
      glo[a] = X.lo[a] - ng;
      ghi[a] = X.hi[a] + ng;
      L[a] = D.hi[a] - D.lo[a] + 1;
      ghost *= (ghi[a] - glo[a] + 1);
      valid *= (X.hi[a] - X.lo[a] + 1);
    }
    ghost -= valid;
    long long covered = 0;
    int smin[3], smax[3];
    for (int a = 0; a < 3; ++a) {
      bool per = D.bc[a] == NYX_BC_PERIODIC;
      smin[a] = per ? -1 : 0;
      smax[a] = per ? 1 : 0;
    }
    for (int sz = smin[2]; sz <= smax[2]; ++sz)
      for (int sy = smin[1]; sy <= smax[1]; ++sy)
        for (int sx = smin[0]; sx <= smax[0]; ++sx) {
          int sh[3] = {sx * L[0], sy * L[1], sz * L[2]};
          // candidate boxes: bins overlapping the grown box shifted back
          int ql[3], qh[3];
          bool any = true;
          for (int a = 0; a < 3; ++a) {
            int lo = std::max(glo[a] - sh[a], D.lo[a]);
            int hi = std::min(ghi[a] - sh[a], D.hi[a]);
            if (lo > hi) any = false;
            ql[a] = (lo - D.lo[a]) / B.bs;
            qh[a] = (hi - D.lo[a]) / B.bs;
          }
          if (!any) continue;
          ++stamp_id;
          for (int k = ql[2]; k <= qh[2]; ++k)
            for (int j = ql[1]; j <= qh[1]; ++j)
              for (int i = ql[0]; i <= qh[0]; ++i)
                for (int c : B.cell[((size_t)k * B.nb[1] + j) * B.nb[0] + i]) {
                  if (stamp[c] == stamp_id) continue;
                  stamp[c] = stamp_id;
                  if (c == b && sx == 0 && sy == 0 && sz == 0) continue;
                  const nyx_box &Y = P.boxes[c];
                  int rlo[3], rhi[3], olo[3], ohi[3];
                  for (int a = 0; a < 3; ++a) {
                    rlo[a] = Y.lo[a] + sh[a];
                    rhi[a] = Y.hi[a] + sh[a];
                  }
                  if (!intersect(glo, ghi, rlo, rhi, olo, ohi)) continue;
                  FillRect R;
                  R.dst_box = b;
                  R.src_box = c;
                  for (int a = 0; a < 3; ++a) {
                    R.dlo[a] = olo[a] - X.lo[a];
                    R.ext[a] = ohi[a] - olo[a] + 1;
                    R.slo[a] = olo[a] - sh[a] - Y.lo[a];
                    R.sstep[a] = 1;
                  }
                  // a copy into the box's own valid cells means overlapping boxes
                  int vlo[3], vhi[3];
                  int xl[3] = {X.lo[0], X.lo[1], X.lo[2]}, xh[3] = {X.hi[0], X.hi[1], X.hi[2]};
                  if (intersect(olo, ohi, xl, xh, vlo, vhi)) {
                    g_err = "boxes " + std::to_string(b) + " and " + std::to_string(c) +
                            " overlap (or a periodic domain is narrower than the ghost width)";
                    return false;
                  }
                  covered += (long long)R.ext[0] * R.ext[1] * R.ext[2];
                  out[0].push_back(R);
                }
        }
    // outflow passes: axis a, low and high sides touching the domain boundary
    for (int a = 0; a < 3; ++a) {
      for (int side = 0; side < 2; ++side) {
        int bc = D.bc[side ? 3 + a : a];
        bool touch = side ? (X.hi[a] == D.hi[a]) : (X.lo[a] == D.lo[a]);
        if (bc != NYX_BC_OUTFLOW || !touch) continue;
        FillRect R;
        R.dst_box = b;
        R.src_box = b;
        int n[3] = {X.hi[0] - X.lo[0] + 1, X.hi[1] - X.lo[1] + 1, X.hi[2] - X.lo[2] + 1};
        for (int e = 0; e < 3; ++e) {
          if (e == a) {
            R.dlo[e] = side ? n[e] : -ng;
            R.ext[e] = ng;
            R.slo[e] = side ? n[e] - 1 : 0;
            R.sstep[e] = 0;
          } else {
            // axes handled by a later pass stay inside the domain here
            int lo = -ng, hi = n[e] + ng - 1;
            if (e > a) {
              if (D.bc[e] == NYX_BC_OUTFLOW && X.lo[e] == D.lo[e]) lo = 0;
              if (D.bc[3 + e] == NYX_BC_OUTFLOW && X.hi[e] == D.hi[e]) hi = n[e] - 1;
            }
            R.dlo[e] = lo;
            R.ext[e] = hi - lo + 1;
            R.slo[e] = lo;
            R.sstep[e] = 1;
          }
        }
        covered += (long long)R.ext[0] * R.ext[1] * R.ext[2];
        out[1 + a].push_back(R);
      }
    }
    // the fine level of a coarse-fine pair may leave ghost cells to the
    // coarse interpolation; every other level covers each exactly once
    if (P.prm.coarse_fine ? covered > ghost : covered != ghost) {
      g_err = "ghost cells of box " + std::to_string(b) + " covered " + std::to_string(covered) +
              " times in total, expected " + std::to_string(ghost) +
              " (gap, overlap or unsupported boundary)";
      return false;
    }
  }
  return true;
}

int upload_pass(FillPass &p, const std::vector<FillRect> &rects) {
  p.n = (int)rects.size();
  if (!p.n) return NYX_OK;
  std::vector<long long> pref(p.n);
  long long acc = 0;
  for (int i = 0; i < p.n; ++i) {
    pref[i] = acc;
    acc += (long long)rects[i].ext[0] * rects[i].ext[1] * rects[i].ext[2];
  }
  p.total = acc;
  p.h = rects;
  CK(cudaMalloc(&p.d_rects, sizeof(FillRect) * p.n));
  CK(cudaMalloc(&p.d_pref, sizeof(long long) * p.n));
  CK(cudaMemcpy(p.d_rects, rects.data(), sizeof(FillRect) * p.n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p.d_pref, pref.data(), sizeof(long long) * p.n, cudaMemcpyHostToDevice));
  return NYX_OK;
}

// ---------------------------------------------------------------- work lists
// Relative cost of a work item: its columns times the plane steps it takes.
// An item of nz planes runs nz + 2 column steps (the first plane's traces
// and the last z face are extra) plus its ring prologue, about one more.
double item_cost(const WorkItem &w) { return double(w.nx + 2) * (w.ny + 2) * (w.nz + 3); }

void lpt_sort(std::vector<WorkItem> &it) {
  std::stable_sort(it.begin(), it.end(),
                   [](const WorkItem &a, const WorkItem &b) { return item_cost(a) > item_cost(b); });
}

// Finish time of the last of `slots` resident CTAs that each take the next
// item of the list when they are free (the work queue of the persistent
// kernels), with item_cost as the duration.
double queue_makespan(const std::vector<WorkItem> &it, int slots) {
  std::priority_queue<double, std::vector<double>, std::greater<double>> q;
  for (int i = 0; i < slots; ++i) q.push(0.0);
  double m = 0.0;
  for (const WorkItem &w : it) {
    const double t = q.top() + item_cost(w);
    q.pop();
    q.push(t);
    m = std::max(m, t);
  }
  return m;
}

constexpr int kWhole = 1 << 30;
constexpr int kRestChunk = 16;  // planes of the chunks a long column's rest is cut into

// Every box cut into tx x ty column tiles, every column of n planes cut by
// the rule (L, M): n > M gives a main chunk of M planes and the rest in
// chunks of at most kRestChunk; otherwise ceil(n / L) chunks as even as
// possible.  (kWhole, kWhole) keeps the columns whole.
std::vector<WorkItem> tile_items(const std::vector<std::array<int, 3>> &n, int tx, int ty, int L,
                                 int M) {
  std::vector<WorkItem> items;
  std::vector<std::pair<int, int>> cuts;
  for (int b = 0; b < (int)n.size(); ++b) {
    const int nz = n[b][2];
    cuts.clear();
    if (nz > M) {
      cuts.push_back({0, M});
      const int r = nz - M, k = (r + kRestChunk - 1) / kRestChunk;
      for (int i = 0; i < k; ++i) cuts.push_back({M + r * i / k, r * (i + 1) / k - r * i / k});
    } else {
      const int k = std::max(1, (int)(((long long)nz + L - 1) / L));
      for (int i = 0; i < k; ++i)
        cuts.push_back({(int)((long long)nz * i / k), (int)((long long)nz * (i + 1) / k - (long long)nz * i / k)});
    }
    for (const auto &c : cuts)
      for (int y0 = 0; y0 < n[b][1]; y0 += ty)
        for (int x0 = 0; x0 < n[b][0]; x0 += tx) {
          WorkItem w;
          w.box = b;
          w.x0 = x0;
          w.y0 = y0;
          w.nx = std::min(tx, n[b][0] - x0);
          w.ny = std::min(ty, n[b][1] - y0);
          w.z0 = c.first;
          w.nz = c.second;
          w.pad = 0;
          items.push_back(w);
        }
  }
  lpt_sort(items);
  return items;
}

// Work list of the fused kernel for one tile shape, in the order the queue
// hands it out (largest first).  Both forms stream any range of planes of a
// column (a chunk starts with its own ring prologue), so when whole columns leave
// the `slots` resident CTAs unevenly loaded (fewer tiles than CTAs, or a
// last partial wave), the columns are cut along z: among even cuts into
// chunks of at least 16 planes and cuts into one main chunk plus short
// rest chunks that fill the queue's tail, the one with the earliest
// simulated finish is taken, if it beats whole columns by 2 %.
std::vector<WorkItem> task_items(const std::vector<std::array<int, 3>> &n, int tx, int ty,
                                 int slots, bool chunk) {
  std::vector<WorkItem> best = tile_items(n, tx, ty, kWhole, kWhole);
  if (!chunk || slots < 1 || best.empty()) return best;
  const double whole = queue_makespan(best, slots);
  double total = 0.0;
  for (const WorkItem &w : best) total += item_cost(w);
  if (whole <= 1.02 * total / slots) return best;

  std::vector<std::pair<int, int>> rules;
  int nmax = 0;
  for (const auto &e : n) {
    nmax = std::max(nmax, e[2]);
    for (int k = 2; k <= e[2] / 16; ++k) rules.push_back({(e[2] + k - 1) / k, kWhole});
  }
  const double plane_lb = total / slots / ((tx + 2) * (ty + 2));
  for (int i = 0; i <= 24; ++i) {
    const int M = (int)std::floor(plane_lb * (1.0 + 0.01 * i)) - 3;
    if (M >= 16 && M < nmax) rules.push_back({kWhole, M});
  }
  std::sort(rules.begin(), rules.end());
  rules.erase(std::unique(rules.begin(), rules.end()), rules.end());

  const size_t cap = (size_t)64 * slots;
  double bm = 0.98 * whole;
  for (const auto &r : rules) {
    std::vector<WorkItem> it = tile_items(n, tx, ty, r.first, r.second);
    if (it.size() > std::max(cap, best.size())) continue;
    const double m = queue_makespan(it, slots);
    if (m < bm) {
      bm = m;
      best.swap(it);
    }
  }
  return best;
}

std::vector<WorkItem> build_items(const nyx_plan &P, int tx, int ty, int slots, bool chunk) {
  std::vector<std::array<int, 3>> n(P.nbox);
  for (int b = 0; b < P.nbox; ++b) n[b] = {P.hbox[b].n[0], P.hbox[b].n[1], P.hbox[b].n[2]};
  return task_items(n, tx, ty, slots, chunk);
}

void free_plan(nyx_plan *P) {
  if (!P) return;
  for (auto &kv : P->graphs) cudaGraphExecDestroy(kv.second.first);
  for (auto &e : P->ev_fill) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto &e : P->ev_adv) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto &e : P->ev_flat) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  cudaFree(P->d_boxes);
  cudaFree(P->d_cell_pref);
  cudaFree(P->d_K);
  cudaFree(P->d_SC);
  cudaFree(P->d_BS);
  cudaFree(P->d_dtacc);
  cudaFree(P->d_status);
  cudaFree(P->d_status_tune);
  cudaFree(P->d_scal);
  for (auto &p : P->pass) {
    cudaFree(p.d_rects);
    cudaFree(p.d_pref);
  }
  cudaFree(P->d_scratch);
  cudaFree(P->d_flat);
  cudaFree(P->d_flat_tiles);
  cudaFree(P->d_packed);
  cudaFree(P->d_plane_pref);
  cudaFree(P->d_flux);
  cudaFree(P->d_flux_off);
  for (auto &it : P->d_items) cudaFree(it);
  for (auto &it : P->d_items_grp) cudaFree(it);
  for (auto &pt : P->parts) {
    cudaFree(pt.d_items);
    cudaFree(pt.d_items_grp);
  }
  for (auto &e : P->ev_grp) cudaEventDestroy(e);
  for (auto &kv : P->tmaps) cudaFree(kv.second);
  if (P->copy_stream) cudaStreamDestroy(P->copy_stream);
  for (auto &r : P->d_rects_grp) cudaFree(r);
  for (auto &e : P->ev_in) cudaEventDestroy(e);
  if (P->ev_start) cudaEventDestroy(P->ev_start);
  if (P->h2d_stream) cudaStreamDestroy(P->h2d_stream);
  if (P->ev_setup) cudaEventDestroy(P->ev_setup);
  if (P->ev_side) cudaEventDestroy(P->ev_side);
  if (P->stream2) cudaStreamDestroy(P->stream2);
  for (int k = 0; k < 2; ++k) {
    if (P->fill_stream[k]) cudaStreamDestroy(P->fill_stream[k]);
    if (P->ev_fjoin[k]) cudaEventDestroy(P->ev_fjoin[k]);
  }
  for (auto &e : P->ev_gfill) cudaEventDestroy(e);
  for (auto &e : P->ev_gadv) cudaEventDestroy(e);
  cudaFree(P->d_queue_grp);
  cudaFree(P->d_queue);
  delete P;
}

bool capturing(nyx_plan *P) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(P->stream, &cs);
  return cs != cudaStreamCaptureStatusNone;
}

// Event pair around a span of launches when profiling an eager call.
struct Span {
  nyx_plan *P;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *list;
  cudaEvent_t e0 = nullptr;
  Span(nyx_plan *P_, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *l) : P(P_), list(l) {
    if (P->profiling && !capturing(P)) {
      cudaEventCreate(&e0);
      cudaEventRecord(e0, P->stream);
    }
  }
  ~Span() {
    if (e0) {
      cudaEvent_t e1;
      cudaEventCreate(&e1);
      cudaEventRecord(e1, P->stream);
      list->emplace_back(e0, e1);
    }
  }
};

int do_fill(nyx_plan *P, double *field, int ncomp) {
  Span sp(P, &P->ev_fill);
  for (int p = 0; p < 4; ++p) {
    launch_fill(field, ncomp, P->d_boxes, P->pass[p].d_rects, P->pass[p].d_pref, P->pass[p].n,
                P->pass[p].total, P->stream);
    if (P->pass[p].n > 0 && P->pass[p].total > 0) P->launches += 1;
  }
  return NYX_OK;
}

int do_estdt(nyx_plan *P, const double *state, const double *a_dev, double *dt_dev) {
  if (P->prm.precision == NYX_MIXED)
    launch_estdt_mixed(P->d_boxes, P->d_cell_pref, P->nbox, P->total_cells, state, P->d_K, a_dev,
                       P->d_dtacc, P->stream);
  else
    launch_estdt(P->d_boxes, P->d_cell_pref, P->nbox, P->total_cells, state, P->d_K, a_dev,
                 P->d_dtacc, P->stream);
  launch_dt_finalize(P->d_K, P->d_dtacc, dt_dev, P->stream);
  P->launches += 2;
  return NYX_OK;
}

int tune_shape(nyx_plan *P, const FusedArgs &base);

// Shock-flattening coefficients of state S (ghosts filled), when the plan
// flattens.
int do_flatten(nyx_plan *P, const double *S) {
  if (!P->d_flat) return NYX_OK;
  Span sp(P, &P->ev_flat);
  int e = launch_flatten(P->prm.precision, P->d_boxes, P->d_flat_tiles, P->flat_ntiles, S,
                         P->d_K, P->d_flat, P->stream);
  if (e) return cuda_fail((cudaError_t)e, "flattening launch");
  P->launches += 1;
  return NYX_OK;
}

int variant_bits(const nyx_plan *P) {
  return P->hK.plm | (P->hK.linear_rs << 1) | (P->hK.flat << 2);
}

int read_back_group(nyx_plan *P, const double *Sn, int g, double *host_out, cudaStream_t st);

FusedArgs fused_args(nyx_plan *P, const double *S, const double *G, double *Sn,
                     unsigned long long *acc, bool predict_only) {
  FusedArgs a;
  a.boxes = P->d_boxes;
  a.queue = P->d_queue;
  a.K = P->d_K;
  a.SC = P->d_SC;
  a.BS = P->d_BS;
  a.S = S;
  a.G = G;
  a.Sn = Sn;
  a.dtacc = acc;
  a.status = P->d_status;
  a.flux_keep = P->d_flux;
  a.flux_off = P->d_flux_off;
  a.predict_only = predict_only ? 1 : 0;
  a.variant = variant_bits(P);
  a.flat = P->d_flat;
  a.tmS = nullptr;
  a.tmG = nullptr;
  return a;
}

// ---------------------------------------------------------------- TMA descriptors
// The task form at 16 x 8 tiles stages each plane's state and gravity with
// tensor copies.  Its descriptors: per box, a 4-D tiled map over the box's
// component arrays (x, y, z with ghosts, component), box (tx + 4) x (ty + 2)
// x 1 x ncomp of FP64, out-of-range elements filled with zeros.  The encoder
// is the driver's cuTensorMapEncodeTiled, reached through the runtime; any
// failure leaves the plan on plain loads.
bool shape_stages_with_tma(const nyx_plan *P, int shape) {
  const TileShape ts = fused_shape(shape);
  return P->prm.precision == NYX_MIXED && ts.task && ts.tx == 16 && ts.ty == 8;
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
  }
  return fn;
}


// Descriptors of `field` (ncomp components) for `shape`, built on first use
// (not while the plan's stream is being captured: then null, plain loads).
const void *plan_tmaps(nyx_plan *P, const double *field, int ncomp, int shape) {
  if (!field || !shape_stages_with_tma(P, shape)) return nullptr;
  const auto key = std::make_tuple((const void *)field, ncomp, shape);
  auto it = P->tmaps.find(key);
  if (it != P->tmaps.end()) return it->second;
  if (capturing(P)) return nullptr;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  void *d = nullptr;
  if (enc) {
    const TileShape ts = fused_shape(shape);
    std::vector<CUtensorMap> h(P->nbox);
    bool ok = true;
    for (int b = 0; b < P->nbox && ok; ++b) {
      const BoxDev &X = P->hbox[b];
      void *base = const_cast<double *>(field) + (size_t)ncomp * X.pref;
      const cuuint64_t gdim[4] = {(cuuint64_t)X.N[0], (cuuint64_t)X.N[1], (cuuint64_t)X.N[2],
                                  (cuuint64_t)ncomp};
      const cuuint64_t gstr[3] = {8ull * X.N[0], 8ull * X.N[0] * X.N[1], 8ull * X.stride};
      const cuuint32_t box[4] = {(cuuint32_t)(ts.tx + 4), (cuuint32_t)(ts.ty + 2), 1u,
                                 (cuuint32_t)ncomp};
      const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
      ok = enc(&h[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base, gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (ok && cudaMalloc(&d, sizeof(CUtensorMap) * h.size()) == cudaSuccess) {
      if (cudaMemcpy(d, h.data(), sizeof(CUtensorMap) * h.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
        cudaFree(d);
        d = nullptr;
      }
    } else {
      d = nullptr;
    }
    cudaGetLastError();
  }
  P->tmaps[key] = d;
  return d;
}

// Descriptors of the level's state versions and gravity for the shapes in
// use (called before a graph capture, which cannot build them).
void prepare_tmaps(nyx_plan *P, const nyx_level *L) {
  std::vector<int> shapes;
  if (P->parts.empty())
    shapes.push_back(P->shape);
  else
    for (const auto &pt : P->parts) shapes.push_back(pt.shape);
  for (int s : shapes) {
    plan_tmaps(P, L->state[0], NCONS, s);
    plan_tmaps(P, L->state[1], NCONS, s);
    plan_tmaps(P, L->grav, NGRAV, s);
  }
}

void set_tmaps(nyx_plan *P, FusedArgs &a, int shape) {
  a.tmS = plan_tmaps(P, a.S, NCONS, shape);
  a.tmG = a.G ? plan_tmaps(P, a.G, NGRAV, shape) : nullptr;
  if (!a.tmS || (a.G && !a.tmG)) a.tmS = a.tmG = nullptr;
}

// The fused advance over the whole level (g < 0) or over read-back group g:
// one launch of the plan's shape, or one per part of the autotuner's
// per-class choice.
int launch_level(nyx_plan *P, FusedArgs a, int g, cudaStream_t st) {
  if (P->parts.empty()) {
    const int s = P->shape;
    if (g < 0) {
      a.items = P->d_items[s];
      a.nitems = P->nitems[s];
    } else {
      a.items = P->d_items_grp[s] + P->grp_off[s][g];
      a.nitems = P->grp_off[s][g + 1] - P->grp_off[s][g];
    }
    if (a.nitems > 0) {
      set_tmaps(P, a, s);
      int e = launch_fused(P->prm.precision, s, a, std::min(P->max_grid[s], a.nitems), st);
      if (e) return cuda_fail((cudaError_t)e, "fused advance launch");
      P->launches += 1;
    }
    return NYX_OK;
  }
  for (const auto &pt : P->parts) {
    if (g < 0) {
      a.items = pt.d_items;
      a.nitems = pt.nitems;
    } else {
      a.items = pt.d_items_grp + pt.grp_off[g];
      a.nitems = pt.grp_off[g + 1] - pt.grp_off[g];
    }
    if (a.nitems > 0) {
      set_tmaps(P, a, pt.shape);
      int e = launch_fused(P->prm.precision, pt.shape, a, std::min(pt.grid, a.nitems), st);
      if (e) return cuda_fail((cudaError_t)e, "fused advance launch");
      P->launches += 1;
    }
  }
  return NYX_OK;
}

// One advance of state[cur] into state[1-cur].  With host_out (a fused plan
// whose read-back groups are set up), the advance runs one launch per box
// group, each followed by the group's read-back into host_out.
int do_advance(nyx_plan *P, nyx_level *L, const double *a_old, const double *a_new,
               const double *dt, const double *grav, double *dt_next, bool predict_only = false,
               double *host_out = nullptr) {
  double *S = L->state[L->cur];
  double *Sn = L->state[1 - L->cur];
  const double *G = grav ? grav : L->grav;
  do_fill(P, S, NCONS);
  if (int rc = do_flatten(P, S)) return rc;
  launch_step_setup(P->d_K, a_old, a_new, dt, P->d_SC, P->d_boxes, P->nbox, P->d_BS, P->stream);
  P->launches += 1;
  unsigned long long *acc = dt_next ? P->d_dtacc : nullptr;
  {
  Span sp(P, &P->ev_adv);
  if (P->prm.batching == NYX_PER_BOX) {
    for (int b = 0; b < P->nbox; ++b) {
      const BoxDev &X = P->hbox[b];
      launch_staged_box(X, P->d_boxes + b, P->d_K, P->d_SC, P->d_BS + b, S + NCONS * X.pref,
                        G ? G + NGRAV * X.pref : nullptr,
                        P->d_flat ? static_cast<const double *>(P->d_flat) + X.pref : nullptr,
                        Sn + NCONS * X.pref, P->d_scratch,
                        P->Vmax, acc, P->d_status,
                        P->d_flux ? P->d_flux + P->flux_off[b] : nullptr, predict_only ? 1 : 0,
                        P->stream);
      P->launches += P->d_flux ? 29 : 26;
    }
  } else {
    FusedArgs a = fused_args(P, S, G, Sn, acc, predict_only);
    if (P->prm.autotune && !P->tuned) {
      int rc = tune_shape(P, a);
      if (rc) return rc;
    }
    // the TMA descriptors of both state versions at once (a level alternates
    // between them), so that no later step stops to build them
    prepare_tmaps(P, L);
    if (host_out && P->ngrp > 1) {
      for (int g = 0; g < P->ngrp; ++g) {
        if (int rc = launch_level(P, a, g, P->stream)) return rc;
        if (int rc = read_back_group(P, Sn, g, host_out, P->stream)) return rc;
      }
    } else {
      if (int rc = launch_level(P, a, -1, P->stream)) return rc;
    }
  }
  }
  if (dt_next) {
    launch_dt_finalize(P->d_K, P->d_dtacc, dt_next, P->stream);
    P->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "advance launch");
  P->flux_valid = P->d_flux != nullptr;
  if (!predict_only) L->cur = 1 - L->cur;
  return NYX_OK;
}

// A part's items regrouped by the read-back groups [gb[g], gb[g+1]) of boxes.
int part_groups(nyx_plan::RunPart &pt, const std::vector<int> &gb) {
  const int ng = (int)gb.size() - 1;
  std::vector<WorkItem> it;
  it.reserve(pt.h_items.size());
  pt.grp_off.assign(1, 0);
  for (int g = 0; g < ng; ++g) {
    for (const WorkItem &w : pt.h_items)
      if (w.box >= gb[g] && w.box < gb[g + 1]) it.push_back(w);
    pt.grp_off.push_back((int)it.size());
  }
  cudaFree(pt.d_items_grp);
  pt.d_items_grp = nullptr;
  CK(cudaMalloc(&pt.d_items_grp, sizeof(WorkItem) * std::max<size_t>(1, it.size())));
  CK(cudaMemcpy(pt.d_items_grp, it.data(), sizeof(WorkItem) * it.size(), cudaMemcpyHostToDevice));
  return NYX_OK;
}

// Box groups of a fused plan, used by nyx_hydro_step_host_valid (input,
// advance and read-back overlapped per group) and by nyx_hydro_run (each
// group's ghost fill beside the other groups' advances): up to 32 ranges of
// whole boxes with about equal cells (the groups' bit masks are 32 bits), as
// long as each group keeps 2 waves of items or more in the plan's tile shape.
// One group (no overlap) otherwise.  Every shape gets the same groups.  (On the 512^3 large level: 32 groups 1.74e9 zone-updates/s end
// to end, 16 groups 1.72e9, 8 groups 1.59e9.)
int setup_readback(nyx_plan *P) {
  const int nsh = fused_num_shapes(P->prm.precision);
  int waves = P->nitems[P->shape] / std::max(1, P->max_grid[P->shape]);
  if (!P->parts.empty()) {
    waves = 0;
    for (const auto &pt : P->parts) waves += pt.nitems / std::max(1, pt.grid);
  }
  const int G = std::min(std::min(32, P->nbox), waves / 2);
  std::vector<int> gb(1, 0);
  for (int g = 1; g < G; ++g) {
    const long long want = P->total_cells * g / G;
    int b = gb.back() + 1;
    while (b < P->nbox && P->cell_pref[b] < want) ++b;
    if (b >= P->nbox) break;
    gb.push_back(b);
  }
  gb.push_back(P->nbox);
  const int ng = (int)gb.size() - 1;
  // one group until every buffer below is in place: a set-up that fails
  // part way leaves the plan on the ungrouped path (free_plan releases what
  // was made)
  P->ngrp = 1;
  if (ng < 2) return NYX_OK;
  for (int s = 0; s < nsh; ++s) {
    std::vector<WorkItem> it;
    it.reserve(P->h_items[s].size());
    P->grp_off[s].assign(1, 0);
    for (int g = 0; g < ng; ++g) {
      for (const WorkItem &w : P->h_items[s])
        if (w.box >= gb[g] && w.box < gb[g + 1]) it.push_back(w);
      P->grp_off[s].push_back((int)it.size());
    }
    CK(cudaMalloc(&P->d_items_grp[s], sizeof(WorkItem) * it.size()));
    CK(cudaMemcpy(P->d_items_grp[s], it.data(), sizeof(WorkItem) * it.size(),
                  cudaMemcpyHostToDevice));
  }
  for (auto &pt : P->parts)
    if (int rc = part_groups(pt, gb)) return rc;
  // input side: each group's fill rects, the groups they read, and an
  // input order that brings in the groups the first advances need first
  std::vector<int> gof(P->nbox);
  for (int g = 0; g < ng; ++g)
    for (int b = gb[g]; b < gb[g + 1]; ++b) gof[b] = g;
  std::vector<unsigned> src(ng, 0u);
  for (int p = 0; p < 4; ++p) {
    std::vector<FillRect> r;
    r.reserve(P->pass[p].h.size());
    P->rect_off[p].assign(1, 0);
    for (int g = 0; g < ng; ++g) {
      for (const FillRect &R : P->pass[p].h) {
        if (gof[R.dst_box] != g) continue;
        r.push_back(R);
        src[g] |= 1u << gof[R.src_box];
      }
      P->rect_off[p].push_back((int)r.size());
    }
    if (!r.empty()) {
      CK(cudaMalloc(&P->d_rects_grp[p], sizeof(FillRect) * r.size()));
      CK(cudaMemcpy(P->d_rects_grp[p], r.data(), sizeof(FillRect) * r.size(),
                    cudaMemcpyHostToDevice));
    }
  }
  // groups advance in this order: first those whose fill reads only
  // themselves (independent boxes, which need no other group's input), then
  // the others in box order; the inputs come in the order these need them
  std::vector<int> proc;
  for (int g = 0; g < ng; ++g)
    if ((src[g] & ~(1u << g)) == 0u) proc.push_back(g);
  for (int g = 0; g < ng; ++g)
    if ((src[g] & ~(1u << g)) != 0u) proc.push_back(g);
  std::vector<int> order;
  std::vector<char> sent(ng, 0);
  for (int g : proc) {
    const unsigned need = src[g] | (1u << g);
    for (int q = 0; q < ng; ++q)
      if (((need >> q) & 1u) && !sent[q]) {
        sent[q] = 1;
        order.push_back(q);
      }
  }
  CK((cudaError_t)preload_copy_kernels());
  CK(cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&P->h2d_stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&P->stream2, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&P->ev_start, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_setup, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_side, cudaEventDisableTiming));
  CK(cudaMalloc(&P->d_queue_grp, sizeof(int) * ng));
  P->ev_grp.assign(ng, nullptr);
  for (auto &e : P->ev_grp) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  P->ev_in.assign(ng, nullptr);
  for (auto &e : P->ev_in) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (int k = 0; k < 2; ++k) {
    CK(cudaStreamCreateWithFlags(&P->fill_stream[k], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&P->ev_fjoin[k], cudaEventDisableTiming));
  }
  P->ev_gfill.assign(ng, nullptr);
  for (auto &e : P->ev_gfill) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  P->ev_gadv.assign(ng, nullptr);
  for (auto &e : P->ev_gadv) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  P->grp_src = src;
  P->in_order = order;
  P->proc_order = proc;
  P->grp_box = gb;
  P->ngrp = ng;
  return NYX_OK;
}

// nyx_hydro_step_host_valid with its input, advance and read-back overlapped
// per box group: the groups' valid cells are copied in and scattered on the
// input stream in in_order; group g's ghost fill and advance, on the plan's
// stream or stream2 in turn, wait only for the groups the fill reads; its
// new cells go back while later groups advance.  Needs the step scalars in
// d_scal[0..2] (dt given).
int step_pipelined(nyx_plan *P, nyx_level *L, const double *host_in, double *host_out) {
  double *S = L->state[L->cur];
  double *Sn = L->state[1 - L->cur];
  CK(cudaEventRecord(P->ev_start, P->stream));
  CK(cudaStreamWaitEvent(P->h2d_stream, P->ev_start, 0));
  for (int q : P->in_order) {
    const int b0 = P->grp_box[q], b1 = P->grp_box[q + 1];
    const long long c0 = P->cell_pref[b0], c1 = b1 < P->nbox ? P->cell_pref[b1] : P->total_cells;
    const int k0 = P->plane_pref[b0], k1 = b1 < P->nbox ? P->plane_pref[b1] : P->plane_blocks;
    CK(cudaMemcpyAsync(P->d_packed + NCONS * c0, host_in + NCONS * c0,
                       sizeof(double) * NCONS * (size_t)(c1 - c0), cudaMemcpyHostToDevice,
                       P->h2d_stream));
    launch_valid_copy(S, P->d_packed, P->d_boxes, P->d_cell_pref, P->d_plane_pref, P->nbox,
                      k1 - k0, k0, 1, P->h2d_stream);
    P->launches += 1;
    CK(cudaEventRecord(P->ev_in[q], P->h2d_stream));
  }
  launch_step_setup(P->d_K, P->d_scal, P->d_scal + 1, P->d_scal + 2, P->d_SC, P->d_boxes, P->nbox,
                    P->d_BS, P->stream);
  P->launches += 1;
  CK(cudaEventRecord(P->ev_setup, P->stream));
  CK(cudaStreamWaitEvent(P->stream2, P->ev_setup, 0));
  FusedArgs a = fused_args(P, S, L->grav, Sn, P->d_dtacc, false);
  const cudaStream_t cs[2] = {P->stream, P->stream2};
  unsigned waited[2] = {0u, 0u};
  for (int gi = 0; gi < P->ngrp; ++gi) {
    const int g = P->proc_order[gi];
    const cudaStream_t st = cs[gi & 1];
    const unsigned need = (P->grp_src[g] | (1u << g)) & ~waited[gi & 1];
    for (int q = 0; q < P->ngrp; ++q)
      if ((need >> q) & 1u) CK(cudaStreamWaitEvent(st, P->ev_in[q], 0));
    waited[gi & 1] |= need;
    for (int p = 0; p < 4; ++p) {
      const int r0 = P->rect_off[p][g], nr = P->rect_off[p][g + 1] - r0;
      if (nr > 0) {
        launch_fill(S, NCONS, P->d_boxes, P->d_rects_grp[p] + r0, nullptr, nr, P->pass[p].total,
                    st, true);
        P->launches += 1;
      }
    }
    if (P->d_flat) {
      // the group's flattening coefficients read only its own boxes, ghosts included
      const int t0 = P->flat_tile_pref[P->grp_box[g]], t1 = P->flat_tile_pref[P->grp_box[g + 1]];
      if (t1 > t0) {
        int e = launch_flatten(P->prm.precision, P->d_boxes, P->d_flat_tiles + t0, t1 - t0, S,
                               P->d_K, P->d_flat, st);
        if (e) return cuda_fail((cudaError_t)e, "flattening launch");
        P->launches += 1;
      }
    }
    a.queue = P->d_queue_grp + g;
    if (int rc = launch_level(P, a, g, st)) return rc;
    if (int rc = read_back_group(P, Sn, g, host_out, st)) return rc;
  }
  CK(cudaEventRecord(P->ev_side, P->stream2));
  CK(cudaStreamWaitEvent(P->stream, P->ev_side, 0));
  launch_dt_finalize(P->d_K, P->d_dtacc, P->d_scal + 3, P->stream);
  P->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pipelined step launch");
  P->flux_valid = P->d_flux != nullptr;
  L->cur = 1 - L->cur;
  return NYX_OK;
}

// The new valid cells of group g's boxes: gathered into the packed buffer
// on stream st (where the group advanced), then copied to host_out on the
// copy stream.
int read_back_group(nyx_plan *P, const double *Sn, int g, double *host_out, cudaStream_t st) {
  const int b0 = P->grp_box[g], b1 = P->grp_box[g + 1];
  const int k0 = P->plane_pref[b0], k1 = b1 < P->nbox ? P->plane_pref[b1] : P->plane_blocks;
  launch_valid_copy(const_cast<double *>(Sn), P->d_packed, P->d_boxes, P->d_cell_pref,
                    P->d_plane_pref, P->nbox, k1 - k0, k0, 0, st);
  P->launches += 1;
  const long long c0 = P->cell_pref[b0], c1 = b1 < P->nbox ? P->cell_pref[b1] : P->total_cells;
  CK(cudaEventRecord(P->ev_grp[g], st));
  CK(cudaStreamWaitEvent(P->copy_stream, P->ev_grp[g], 0));
  CK(cudaMemcpyAsync(host_out + NCONS * c0, P->d_packed + NCONS * c0,
                     sizeof(double) * NCONS * (size_t)(c1 - c0), cudaMemcpyDeviceToHost,
                     P->copy_stream));
  return NYX_OK;
}

// Step 6 alone: state[1-cur] (a predictor) corrected with g^n / g^{n+1},
// synchronised; cur flips.
int do_correct(nyx_plan *P, nyx_level *L, const double *a_old, const double *a_new,
               const double *dt, const double *g_old, const double *g_new, double *dt_next) {
  launch_step_setup(P->d_K, a_old, a_new, dt, P->d_SC, P->d_boxes, P->nbox, P->d_BS, P->stream);
  launch_correct(P->d_boxes, P->d_cell_pref, P->nbox, P->total_cells, P->d_K, P->d_SC,
                 L->state[L->cur], L->state[1 - L->cur], g_old, g_new,
                 dt_next ? P->d_dtacc : nullptr, P->d_status, P->prm.precision == NYX_MIXED,
                 P->stream);
  P->launches += 2;
  if (dt_next) {
    launch_dt_finalize(P->d_K, P->d_dtacc, dt_next, P->stream);
    P->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "corrector launch");
  L->cur = 1 - L->cur;
  return NYX_OK;
}

// ---------------------------------------------------------------- autotuner
// The level's boxes fall into box-size classes (boxes of equal extent), and
// each class is tuned on its own.  Every candidate -- a tile shape with a
// number of resident CTAs per SM (all that fit, or one) -- runs two waves of
// the class's work items (twice as many items as the candidate keeps
// resident; a class with fewer items has them repeated, so that the timing
// is of a full machine), and the candidate with the least time per zone wins.  Choices are
// kept in a JSON file keyed by GPU name, SM count, precision, scheme variant
// and box extent, so a later plan whose classes are all there makes no trial
// launch.  Classes that settle on the same candidate share one launch; the
// level's launch is one per distinct candidate (nyx_plan::parts), or the
// single level-wide list when every class agrees on a shape at full
// residency.  The staging depth of the kernels is fixed by their ring
// structure; the plane chunks of the task form come from the queue model of
// task_items, not from timing.

struct TuneChoice {
  int shape = -1, per_sm = 0;
  double ns_per_zone = 0.0;
};

std::string tune_cache_path() {
  if (const char *env = std::getenv("NYX_TUNE_CACHE")) return std::string(env);  // "": no cache
  Dl_info info;
  if (dladdr((void *)&tune_cache_path, &info) && info.dli_fname) {
    const std::string f = info.dli_fname;
    const size_t k = f.rfind('/');
    return (k == std::string::npos ? std::string(".") : f.substr(0, k)) + "/_tune_cache.json";
  }
  return "";
}

// One entry per line: "key": {"shape": S, "ctas_per_sm": K, "ns_per_zone": T}
std::map<std::string, TuneChoice> tune_cache_load(const std::string &path) {
  std::map<std::string, TuneChoice> m;
  if (path.empty()) return m;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    const size_t a = line.find('"');
    if (a == std::string::npos) continue;
    const size_t b = line.find('"', a + 1);
    if (b == std::string::npos) continue;
    TuneChoice c;
    if (std::sscanf(line.c_str() + b + 1, ": {\"shape\": %d, \"ctas_per_sm\": %d, \"ns_per_zone\": %lf",
                    &c.shape, &c.per_sm, &c.ns_per_zone) == 3 &&
        c.shape >= 0 && c.per_sm > 0)
      m[line.substr(a + 1, b - a - 1)] = c;
  }
  return m;
}

void tune_cache_save(const std::string &path, const std::map<std::string, TuneChoice> &m) {
  if (path.empty()) return;
  const std::string tmp = path + ".tmp" + std::to_string((long long)std::rand());
  {
    std::ofstream out(tmp);
    if (!out) return;
    out << "{\n";
    size_t n = 0;
    for (const auto &kv : m) {
      char buf[160];
      std::snprintf(buf, sizeof(buf), "{\"shape\": %d, \"ctas_per_sm\": %d, \"ns_per_zone\": %.6g}",
                    kv.second.shape, kv.second.per_sm, kv.second.ns_per_zone);
      out << " \"" << kv.first << "\": " << buf << (++n < m.size() ? ",\n" : "\n");
    }
    out << "}\n";
  }
  std::rename(tmp.c_str(), path.c_str());  // whole file or none: readers never see a partial one
}

// Items of the boxes `sel` (indices into the plan's box list) for one tile
// shape, with the box indices of the plan.
std::vector<WorkItem> subset_items(const nyx_plan &P, const std::vector<int> &sel, int tx, int ty,
                                   int slots, bool chunk) {
  std::vector<std::array<int, 3>> n(sel.size());
  for (size_t k = 0; k < sel.size(); ++k) {
    const BoxDev &X = P.hbox[sel[k]];
    n[k] = {X.n[0], X.n[1], X.n[2]};
  }
  std::vector<WorkItem> it = task_items(n, tx, ty, slots, chunk);
  for (WorkItem &w : it) w.box = sel[w.box];
  return it;
}

int tune_shape(nyx_plan *P, const FusedArgs &base) {
  P->tuned = true;
  cudaStreamCaptureStatus cs;
  CK(cudaStreamIsCapturing(P->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return NYX_OK;  // keep the current shape under capture
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  const int nsm = prop.multiProcessorCount;
  const int nsh = fused_num_shapes(P->prm.precision);
  // classes: boxes of equal extent, in order of first appearance
  std::map<std::array<int, 3>, int> cls_of;
  std::vector<std::array<int, 3>> cls_n;
  std::vector<std::vector<int>> cls_boxes;
  for (int b = 0; b < P->nbox; ++b) {
    const std::array<int, 3> e = {P->hbox[b].n[0], P->hbox[b].n[1], P->hbox[b].n[2]};
    auto f = cls_of.find(e);
    if (f == cls_of.end()) {
      f = cls_of.emplace(e, (int)cls_n.size()).first;
      cls_n.push_back(e);
      cls_boxes.emplace_back();
    }
    cls_boxes[f->second].push_back(b);
  }
  const int nc = (int)cls_n.size();
  P->tune_classes = nc;
  P->tune_trials = 0;
  const std::string path = tune_cache_path();
  std::map<std::string, TuneChoice> cache = tune_cache_load(path);
  const std::string prefix = std::string(prop.name) + "|sm" + std::to_string(nsm) + "|" +
                             (P->prm.precision == NYX_MIXED ? "mixed" : "fp64") + "|v" +
                             std::to_string(variant_bits(P)) + "|";
  std::vector<TuneChoice> pick(nc);
  bool fresh = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  WorkItem *d_wave = nullptr;
  size_t wave_cap = 0;
  int rc = NYX_OK;
  for (int c = 0; c < nc && rc == NYX_OK; ++c) {
    const std::string key = prefix + std::to_string(cls_n[c][0]) + "x" + std::to_string(cls_n[c][1]) +
                            "x" + std::to_string(cls_n[c][2]);
    auto hit = cache.find(key);
    if (hit != cache.end() && hit->second.shape < nsh &&
        hit->second.per_sm * nsm <= P->max_grid[hit->second.shape]) {
      pick[c] = hit->second;
      continue;
    }
    if (!e0) {
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
    }
    TuneChoice best;
    for (int sh = 0; sh < nsh && rc == NYX_OK; ++sh) {
      const TileShape ts = fused_shape(sh);
      const int full = std::max(1, P->max_grid[sh] / nsm);
      std::vector<WorkItem> all = subset_items(*P, cls_boxes[c], ts.tx, ts.ty, kWhole, false);
      std::vector<int> occ(1, full);  // resident CTAs per SM: all that fit, and one
      if (full > 1) occ.push_back(1);
      for (int per_sm : occ) {
        const int grid = per_sm * nsm;
        std::vector<WorkItem> wave(2 * grid);  // two waves: per-launch overhead weighs less
        double zones = 0.0;
        for (int k = 0; k < 2 * grid; ++k) {
          wave[k] = all[k % all.size()];
          zones += double(wave[k].nx) * wave[k].ny * wave[k].nz;
        }
        if (wave.size() > wave_cap) {
          cudaFree(d_wave);
          d_wave = nullptr;
          if (cudaMalloc(&d_wave, sizeof(WorkItem) * wave.size()) != cudaSuccess) {
            rc = fail(NYX_ENOMEM, "autotune item buffer");
            break;
          }
          wave_cap = wave.size();
        }
        CK(cudaMemcpy(d_wave, wave.data(), sizeof(WorkItem) * wave.size(), cudaMemcpyHostToDevice));
        FusedArgs a = base;
        a.items = d_wave;
        a.nitems = 2 * grid;
        a.dtacc = nullptr;
        a.flux_keep = nullptr;
        a.status = P->d_status_tune;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
          CK(cudaEventRecord(e0, P->stream));
          int e = launch_fused(P->prm.precision, sh, a, grid, P->stream);
          if (e) return cuda_fail((cudaError_t)e, "autotune launch");
          P->launches += 1;
          P->tune_trials += 1;
          CK(cudaEventRecord(e1, P->stream));
          CK(cudaEventSynchronize(e1));
          CK(cudaEventElapsedTime(&ms, e0, e1));
        }
        const double t = ms * 1e6 / zones;
        if (best.shape < 0 || t < best.ns_per_zone) {
          best.shape = sh;
          best.per_sm = per_sm;
          best.ns_per_zone = t;
        }
      }
    }
    pick[c] = best;
    cache[key] = best;
    fresh = true;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_wave);
  if (rc) return rc;
  if (fresh) tune_cache_save(path, cache);

  // one part per distinct choice, its classes' boxes together
  std::map<std::pair<int, int>, std::vector<int>> groups;
  std::map<std::pair<int, int>, long long> gcells;
  for (int c = 0; c < nc; ++c) {
    auto &v = groups[{pick[c].shape, pick[c].per_sm}];
    v.insert(v.end(), cls_boxes[c].begin(), cls_boxes[c].end());
    gcells[{pick[c].shape, pick[c].per_sm}] +=
        (long long)cls_boxes[c].size() * cls_n[c][0] * cls_n[c][1] * cls_n[c][2];
  }
  for (auto &pt : P->parts) {
    cudaFree(pt.d_items);
    cudaFree(pt.d_items_grp);
  }
  P->parts.clear();
  auto biggest = gcells.begin();
  for (auto it = gcells.begin(); it != gcells.end(); ++it)
    if (it->second > biggest->second) biggest = it;
  P->shape = biggest->first.first;
  if (groups.size() == 1 && biggest->first.second * nsm >= P->max_grid[P->shape]) return NYX_OK;
  for (auto &kv : groups) {
    nyx_plan::RunPart pt;
    pt.shape = kv.first.first;
    pt.grid = std::min(P->max_grid[pt.shape], kv.first.second * nsm);
    std::sort(kv.second.begin(), kv.second.end());
    const TileShape ts = fused_shape(pt.shape);
    pt.h_items = subset_items(*P, kv.second, ts.tx, ts.ty, pt.grid, P->prm.z_chunks != 0);
    pt.nitems = (int)pt.h_items.size();
    CK(cudaMalloc(&pt.d_items, sizeof(WorkItem) * std::max(1, pt.nitems)));
    CK(cudaMemcpy(pt.d_items, pt.h_items.data(), sizeof(WorkItem) * pt.nitems,
                  cudaMemcpyHostToDevice));
    P->parts.push_back(std::move(pt));
    if (P->ngrp > 1)
      if (int r2 = part_groups(P->parts.back(), P->grp_box)) return r2;
  }
  return NYX_OK;
}

// nsteps steps of a fused plan with box groups, the ghost fill overlapped
// with the advance.  Per step s, S = state[cur], Sn = state[1-cur]:
//   * group g's fill of S, on fill stream gi & 1, waits only for the
//     advances of step s-1 of the groups it reads
//     (itself included; at s = 0 for the start of the run), so it runs
//     beside the advances of the other groups.  It writes the ghost cells of
//     g's boxes in S, which no advance of step s-1 reads (they read the other
//     buffer) and none writes (advances write valid cells);
//   * a flattening plan's coefficient pass runs over the whole level on the
//     plan stream once every group is filled (it does not fit beside an
//     advance);
//   * the step set-up waits for step s-1's dt (plan stream); then group g
//     advances on the plan stream or stream2 in turn once its fill is done;
//   * the dt of step s+1 is finalised once every group has advanced.
// Every cell takes the same arithmetic as in the one-launch form, so the
// result is the same bit for bit.
int run_grouped(nyx_plan *P, nyx_level *L, const double *a_dev, double *dt_dev, int nsteps) {
  CK(cudaEventRecord(P->ev_start, P->stream));
  for (int k = 0; k < 2; ++k) CK(cudaStreamWaitEvent(P->fill_stream[k], P->ev_start, 0));
  const cudaStream_t cs[2] = {P->stream, P->stream2};
  for (int s = 0; s < nsteps; ++s) {
    double *S = L->state[L->cur];
    double *Sn = L->state[1 - L->cur];
    for (int gi = 0; gi < P->ngrp; ++gi) {
      const int g = P->proc_order[gi];
      const cudaStream_t fs = P->fill_stream[gi & 1];
      if (s > 0) {
        const unsigned need = P->grp_src[g] | (1u << g);
        for (int q = 0; q < P->ngrp; ++q)
          if ((need >> q) & 1u) CK(cudaStreamWaitEvent(fs, P->ev_gadv[q], 0));
      }
      for (int p = 0; p < 4; ++p) {
        const int r0 = P->rect_off[p][g], nr = P->rect_off[p][g + 1] - r0;
        if (nr > 0) {
          launch_fill(S, NCONS, P->d_boxes, P->d_rects_grp[p] + r0, nullptr, nr,
                      P->pass[p].total, fs, true);
          P->launches += 1;
        }
      }
      CK(cudaEventRecord(P->ev_gfill[g], fs));
    }
    if (P->d_flat) {
      // the coefficient pass (512 threads, 43 KB of shared memory per block)
      // does not fit beside the advance: it runs over the whole level once
      // every group is filled, before the step's advances
      for (int k = 0; k < 2; ++k) {
        CK(cudaEventRecord(P->ev_fjoin[k], P->fill_stream[k]));
        CK(cudaStreamWaitEvent(P->stream, P->ev_fjoin[k], 0));
      }
      if (int rc = do_flatten(P, S)) return rc;
    }
    launch_step_setup(P->d_K, a_dev + s, a_dev + s + 1, dt_dev + s, P->d_SC, P->d_boxes, P->nbox,
                      P->d_BS, P->stream);
    P->launches += 1;
    CK(cudaEventRecord(P->ev_setup, P->stream));
    CK(cudaStreamWaitEvent(P->stream2, P->ev_setup, 0));
    FusedArgs a = fused_args(P, S, L->grav, Sn, P->d_dtacc, false);
    for (int gi = 0; gi < P->ngrp; ++gi) {
      const int g = P->proc_order[gi];
      const cudaStream_t st = cs[gi & 1];
      CK(cudaStreamWaitEvent(st, P->ev_gfill[g], 0));
      a.queue = P->d_queue_grp + g;
      if (int rc = launch_level(P, a, g, st)) return rc;
      CK(cudaEventRecord(P->ev_gadv[g], st));
    }
    CK(cudaEventRecord(P->ev_side, P->stream2));
    CK(cudaStreamWaitEvent(P->stream, P->ev_side, 0));
    launch_dt_finalize(P->d_K, P->d_dtacc, dt_dev + s + 1, P->stream);
    P->launches += 1;
    L->cur = 1 - L->cur;
  }
  // every stream of the run ends joined to the plan stream
  for (int k = 0; k < 2; ++k) {
    CK(cudaEventRecord(P->ev_fjoin[k], P->fill_stream[k]));
    CK(cudaStreamWaitEvent(P->stream, P->ev_fjoin[k], 0));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "grouped run launch");
  P->flux_valid = P->d_flux != nullptr;
  return NYX_OK;
}

int enqueue_run(nyx_plan *P, nyx_level *L, const double *a_dev, double *dt_dev, int nsteps,
                int compute_dt0) {
  if (compute_dt0) do_estdt(P, L->state[L->cur], a_dev, dt_dev);
  // fused plans with box groups overlap each step's ghost fill with the
  // advance; profiled runs keep one fill and one advance launch per step so
  // that each is timed on its own
  if (P->prm.batching != NYX_PER_BOX && P->ngrp > 1 && !(P->prm.autotune && !P->tuned) &&
      !P->profiling && nsteps > 0) {
    prepare_tmaps(P, L);
    return run_grouped(P, L, a_dev, dt_dev, nsteps);
  }
  for (int s = 0; s < nsteps; ++s) {
    int rc = do_advance(P, L, a_dev + s, a_dev + s + 1, dt_dev + s, nullptr, dt_dev + s + 1);
    if (rc) return rc;
  }
  return NYX_OK;
}

}  // namespace

namespace nyx {
namespace host {

int plan_fill(nyx_plan *P, double *field, int ncomp) { return do_fill(P, field, ncomp); }

int plan_advance(nyx_plan *P, nyx_level *L, const double *a_old, const double *a_new,
                 const double *dt, const double *grav, double *dt_next) {
  return do_advance(P, L, a_old, a_new, dt, grav, dt_next);
}

void plan_estdt_accumulate(nyx_plan *P, const double *state, const double *a_dev,
                           unsigned long long *acc) {
  if (P->prm.precision == NYX_MIXED)
    launch_estdt_mixed(P->d_boxes, P->d_cell_pref, P->nbox, P->total_cells, state, P->d_K, a_dev,
                       acc, P->stream);
  else
    launch_estdt(P->d_boxes, P->d_cell_pref, P->nbox, P->total_cells, state, P->d_K, a_dev, acc,
                 P->stream);
  P->launches += 1;
}

bool plan_capturing(nyx_plan *P) { return capturing(P); }

int plan_tune(nyx_plan *P, nyx_level *L, const double *a_dev, const double *dt_dev) {
  if (!(P->prm.batching == NYX_PERSISTENT && P->prm.autotune && !P->tuned)) return NYX_OK;
  FusedArgs a{};
  a.boxes = P->d_boxes;
  a.queue = P->d_queue;
  a.K = P->d_K;
  a.SC = P->d_SC;
  a.BS = P->d_BS;
  a.S = L->state[L->cur];
  a.G = L->grav;
  a.Sn = L->state[1 - L->cur];
  a.status = P->d_status_tune;
  a.variant = variant_bits(P);
  a.flat = P->d_flat;
  do_fill(P, L->state[L->cur], NCONS);
  if (int rc = do_flatten(P, L->state[L->cur])) return rc;
  launch_step_setup(P->d_K, a_dev, a_dev + 1, dt_dev, P->d_SC, P->d_boxes, P->nbox, P->d_BS,
                    P->stream);
  return tune_shape(P, a);
}

}  // namespace host
}  // namespace nyx

// ====================================================================== fused dispatch
namespace nyx {

void record_error(const char *msg) { g_err = msg ? msg : ""; }

// 0-2: column-owning form (FP64 and mixed); 3-5: task form (mixed only)
static const TileShape kShapes[] = {{16, 16, 0}, {32, 8, 0}, {16, 8, 0},
                                    {16, 8, 1},  {8, 8, 1},  {32, 4, 1}};

int fused_num_shapes(int precision) { return precision == NYX_MIXED ? 6 : 3; }
TileShape fused_shape(int idx) { return kShapes[idx]; }

int launch_fused(int precision, int shape, const FusedArgs &a, int grid, cudaStream_t st) {
  if (grid < 1) grid = 1;
  return precision == NYX_MIXED ? launch_fused_mixed(shape, a, grid, st)
                                : launch_fused_f64(shape, a, grid, st);
}

int launch_flatten(int precision, const BoxDev *boxes, const FlatTile *tiles, int ntiles,
                   const double *S, const SchemeConsts *K, void *fl, cudaStream_t st) {
  return precision == NYX_MIXED ? launch_flatten_mixed(boxes, tiles, ntiles, S, K, fl, st)
                                : launch_flatten_f64(boxes, tiles, ntiles, S, K, fl, st);
}

int flatten_init(int precision) {
  return precision == NYX_MIXED ? flatten_init_mixed() : flatten_init_f64();
}

int launch_flat_ones(int precision, void *fl, long long n, cudaStream_t st) {
  return precision == NYX_MIXED ? flat_ones_mixed(fl, n, st) : flat_ones_f64(fl, n, st);
}

int fused_max_grid(int precision, int shape) {
  return precision == NYX_MIXED ? max_grid_mixed(shape) : max_grid_f64(shape);
}

}  // namespace nyx

// ====================================================================== C ABI
extern "C" {

void nyx_hydro_default_params(nyx_hydro_params *p) {
  if (!p) return;
  p->gamma = 5.0 / 3.0;
  p->cfl = 0.5;
  p->small_dens = 1e-10;
  p->small_pres = 1e-12;
  p->eta_de = 1e-4;
  p->riemann_max_iter = 12;
  p->riemann_tol = 1e-10;
  p->precision = NYX_FP64;
  p->grav_corrector = 1;
  p->batching = NYX_PERSISTENT;
  p->autotune = 0;
  p->keep_fluxes = 0;
  p->coarse_fine = 0;
  p->grav_energy = 0;
  p->reconstruction = NYX_PPM;
  p->riemann_solver = NYX_RS_TWO_SHOCK;
  p->flattening = 0;
  p->z_chunks = 1;
}

const char *nyx_last_error(void) { return g_err.c_str(); }

int nyx_hydro_plan(const nyx_level_desc *lev, const nyx_hydro_params *prm, void *stream,
                   nyx_plan **out) {
  g_err.clear();
  if (!lev || !prm || !out) return fail(NYX_EINVAL, "null argument");
  *out = nullptr;
  if (lev->nboxes <= 0 || !lev->boxes) return fail(NYX_EINVAL, "level has no boxes");
  if (lev->ndomains <= 0 || !lev->domains) return fail(NYX_EINVAL, "level has no domains");
  if (lev->ng != 4) return fail(NYX_EINVAL, "ghost width must be 4");
  if (!(prm->gamma > 1.0) || !(prm->cfl > 0.0 && prm->cfl <= 1.0) || !(prm->small_dens > 0.0) ||
      !(prm->small_pres > 0.0) || !(prm->eta_de >= 0.0) || prm->riemann_max_iter < 1 ||
      !(prm->riemann_tol > 0.0))
    return fail(NYX_EINVAL, "invalid scheme parameters");
  if (prm->precision != NYX_FP64 && prm->precision != NYX_MIXED)
    return fail(NYX_EINVAL, "precision must be NYX_FP64 or NYX_MIXED");
  if (prm->batching != NYX_PERSISTENT && prm->batching != NYX_PER_BOX)
    return fail(NYX_EINVAL, "batching must be NYX_PERSISTENT or NYX_PER_BOX");
  if (prm->batching == NYX_PER_BOX && prm->precision != NYX_FP64)
    return fail(NYX_EINVAL, "the per-box form is FP64 only");
  for (int d = 0; d < lev->ndomains; ++d) {
    const nyx_domain &D = lev->domains[d];
    for (int a = 0; a < 3; ++a) {
      if (D.hi[a] < D.lo[a]) return fail(NYX_EINVAL, "empty domain " + std::to_string(d));
      for (int s = 0; s < 2; ++s) {
        int bc = D.bc[s * 3 + a];
        if (bc != NYX_BC_PERIODIC && bc != NYX_BC_OUTFLOW)
          return fail(NYX_EINVAL, "unknown boundary kind in domain " + std::to_string(d));
      }
      if ((D.bc[a] == NYX_BC_PERIODIC) != (D.bc[3 + a] == NYX_BC_PERIODIC))
        return fail(NYX_EINVAL, "periodic boundaries must come in pairs");
      if (D.bc[a] == NYX_BC_PERIODIC && D.hi[a] - D.lo[a] + 1 < 4)
        return fail(NYX_EINVAL, "periodic domain narrower than the ghost width");
    }
  }
  for (int b = 0; b < lev->nboxes; ++b) {
    const nyx_box &X = lev->boxes[b];
    if (X.domain < 0 || X.domain >= lev->ndomains)
      return fail(NYX_EINVAL, "box " + std::to_string(b) + " has an invalid domain");
    const nyx_domain &D = lev->domains[X.domain];
    for (int a = 0; a < 3; ++a) {
      int n = X.hi[a] - X.lo[a] + 1;
      if (n <= 0 || (n & 1))
        return fail(NYX_EINVAL, "box " + std::to_string(b) + " extent must be even and positive");
      if (X.lo[a] < D.lo[a] || X.hi[a] > D.hi[a])
        return fail(NYX_EINVAL, "box " + std::to_string(b) + " lies outside its domain");
      if (!(X.dx[a] > 0.0) || !std::isfinite(X.dx[a]))
        return fail(NYX_EINVAL, "box " + std::to_string(b) + " has a non-positive dx");
    }
  }
  nyx_plan *P = new nyx_plan();
  P->nbox = lev->nboxes;
  P->boxes.assign(lev->boxes, lev->boxes + lev->nboxes);
  P->doms.assign(lev->domains, lev->domains + lev->ndomains);
  P->prm = *prm;
  P->stream = (cudaStream_t)stream;
  // layout
  long long pref = 0, cells = 0;
  P->hbox.resize(P->nbox);
  P->cell_pref.resize(P->nbox);
  for (int b = 0; b < P->nbox; ++b) {
    BoxDev &X = P->hbox[b];
    for (int a = 0; a < 3; ++a) {
      X.n[a] = P->boxes[b].hi[a] - P->boxes[b].lo[a] + 1;
      X.N[a] = X.n[a] + 8;
      X.dx[a] = P->boxes[b].dx[a];
      X.idx[a] = 1.0 / X.dx[a];
    }
    X.stride = round_up((long long)X.N[0] * X.N[1] * X.N[2], 32);
    X.pref = pref;
    pref += X.stride;
    P->cell_pref[b] = cells;
    cells += (long long)X.n[0] * X.n[1] * X.n[2];
    P->Vmax = std::max(P->Vmax, X.stride);
  }
  P->total_cells = cells;
  P->total_stride = pref;
  std::vector<FillRect> rects[4];
  if (!build_fill(*P, rects)) {
    std::string m = g_err;
    free_plan(P);
    return fail(NYX_EINVAL, m);
  }
  int rc = NYX_OK;
#define TRY(x)              \
  do {                      \
    rc = (x);               \
    if (rc) goto fail_out;  \
  } while (0)
#define TRYC(x)                                                  \
  do {                                                           \
    cudaError_t e_ = (x);                                        \
    if (e_ != cudaSuccess) {                                     \
      rc = (e_ == cudaErrorMemoryAllocation)                     \
               ? fail(NYX_ENOMEM, std::string("device allocation failed: ") + #x) \
               : cuda_fail(e_, #x);                              \
      goto fail_out;                                             \
    }                                                            \
  } while (0)
  {
    for (int p = 0; p < 4; ++p) TRY(upload_pass(P->pass[p], rects[p]));
    TRYC(cudaMalloc(&P->d_boxes, sizeof(BoxDev) * P->nbox));
    TRYC(cudaMemcpy(P->d_boxes, P->hbox.data(), sizeof(BoxDev) * P->nbox, cudaMemcpyHostToDevice));
    TRYC(cudaMalloc(&P->d_cell_pref, sizeof(long long) * P->nbox));
    TRYC(cudaMemcpy(P->d_cell_pref, P->cell_pref.data(), sizeof(long long) * P->nbox,
                    cudaMemcpyHostToDevice));
    SchemeConsts &K = P->hK;
    K.gamma = prm->gamma;
    K.gm1 = prm->gamma - 1.0;
    K.igm1 = 1.0 / K.gm1;
    K.kshock = (prm->gamma + 1.0) / (2.0 * prm->gamma);
    K.small_dens = prm->small_dens;
    K.small_pres = prm->small_pres;
    K.tol = prm->riemann_tol;
    K.tol_mixed = std::max(prm->riemann_tol, 1e-6);  // FP32 cannot resolve tighter
    K.eta_de = prm->eta_de;
    K.cfl = prm->cfl;
    K.kappa = 2.0 - 3.0 * K.gm1;
    K.efloor = prm->small_pres * K.igm1;
    K.max_iter = prm->riemann_max_iter;
    K.grav_corrector = prm->grav_corrector;
    K.grav_energy = prm->grav_energy;
    K.plm = prm->reconstruction == NYX_PLM;
    K.linear_rs = prm->riemann_solver == NYX_RS_LINEAR;
    K.flat = prm->flattening ? 1 : 0;
    TRYC(cudaMalloc(&P->d_K, sizeof(SchemeConsts)));
    TRYC(cudaMemcpy(P->d_K, &K, sizeof(SchemeConsts), cudaMemcpyHostToDevice));
    TRYC(cudaMalloc(&P->d_SC, sizeof(StepConsts)));
    TRYC(cudaMalloc(&P->d_BS, sizeof(BoxStep) * P->nbox));
    TRYC(cudaMalloc(&P->d_dtacc, sizeof(unsigned long long)));
    unsigned long long inf = 0x7ff0000000000000ULL;
    TRYC(cudaMemcpy(P->d_dtacc, &inf, sizeof(inf), cudaMemcpyHostToDevice));
    TRYC(cudaMalloc(&P->d_status, sizeof(unsigned)));
    TRYC(cudaMemset(P->d_status, 0, sizeof(unsigned)));
    TRYC(cudaMalloc(&P->d_status_tune, sizeof(unsigned)));
    TRYC(cudaMemset(P->d_status_tune, 0, sizeof(unsigned)));
    TRYC(cudaMalloc(&P->d_scal, 4 * sizeof(double)));
    if (K.flat) {
      const size_t esz = prm->precision == NYX_MIXED ? sizeof(float) : sizeof(double);
      TRYC(cudaMalloc(&P->d_flat, esz * (size_t)P->total_stride));
      // the [-1, n]^2 columns of each box in near-equal tiles of <= 34 x 17
      std::vector<FlatTile> ft;
      P->flat_tile_pref.assign(1, 0);
      for (int b = 0; b < P->nbox; ++b) {
        const int L0 = P->hbox[b].n[0] + 2, L1 = P->hbox[b].n[1] + 2;
        const int tx = (L0 + 33) / 34, ty = (L1 + 16) / 17;
        for (int v = 0; v < ty; ++v)
          for (int u = 0; u < tx; ++u) {
            FlatTile T;
            T.box = b;
            T.x0 = -1 + (int)((long long)L0 * u / tx);
            T.nx = -1 + (int)((long long)L0 * (u + 1) / tx) - T.x0;
            T.y0 = -1 + (int)((long long)L1 * v / ty);
            T.ny = -1 + (int)((long long)L1 * (v + 1) / ty) - T.y0;
            ft.push_back(T);
          }
        P->flat_tile_pref.push_back((int)ft.size());
      }
      P->flat_ntiles = (int)ft.size();
      TRYC(cudaMalloc(&P->d_flat_tiles, sizeof(FlatTile) * ft.size()));
      TRYC(cudaMemcpy(P->d_flat_tiles, ft.data(), sizeof(FlatTile) * ft.size(),
                      cudaMemcpyHostToDevice));
      TRYC((cudaError_t)flatten_init(prm->precision));
      TRYC((cudaError_t)launch_flat_ones(prm->precision, P->d_flat, P->total_stride, P->stream));
      TRYC(cudaStreamSynchronize(P->stream));
    }
    if (prm->batching == NYX_PER_BOX) {
      TRYC(cudaMalloc(&P->d_scratch, sizeof(double) * staged_scratch_doubles(P->Vmax)));
    } else {
      for (int sh = 0; sh < fused_num_shapes(prm->precision); ++sh) {
        P->max_grid[sh] = fused_max_grid(prm->precision, sh);
        if (P->max_grid[sh] < 1) {
          rc = fail(NYX_ECUDA, "tile shape " + std::to_string(sh) + " cannot be launched");
          goto fail_out;
        }
      }
      for (int s = 0; s < fused_num_shapes(prm->precision); ++s) {
        TileShape ts = fused_shape(s);
        std::vector<WorkItem> it = build_items(*P, ts.tx, ts.ty, P->max_grid[s], prm->z_chunks);
        P->nitems[s] = (int)it.size();
        TRYC(cudaMalloc(&P->d_items[s], sizeof(WorkItem) * it.size()));
        TRYC(cudaMemcpy(P->d_items[s], it.data(), sizeof(WorkItem) * it.size(),
                        cudaMemcpyHostToDevice));
        P->h_items[s] = std::move(it);
      }
      TRYC(cudaMalloc(&P->d_queue, sizeof(int)));
      TRYC(cudaMemset(P->d_queue, 0, sizeof(int)));
      TRYC(cudaGetLastError());
    }
    if (prm->keep_fluxes) {
      long long acc = 0;
      P->flux_off.resize(P->nbox);
      for (int b = 0; b < P->nbox; ++b) {
        P->flux_off[b] = acc;
        const BoxDev &X = P->hbox[b];
        for (int d = 0; d < 3; ++d)
          acc += 6LL * (X.n[0] + (d == 0)) * (X.n[1] + (d == 1)) * (X.n[2] + (d == 2));
      }
      TRYC(cudaMalloc(&P->d_flux, sizeof(double) * acc));
      TRYC(cudaMalloc(&P->d_flux_off, sizeof(long long) * P->nbox));
      TRYC(cudaMemcpy(P->d_flux_off, P->flux_off.data(), sizeof(long long) * P->nbox,
                      cudaMemcpyHostToDevice));
    }
  }
  *out = P;
  return NYX_OK;
fail_out:
  free_plan(P);
  return rc;
#undef TRY
#undef TRYC
}

int nyx_hydro_layout(const nyx_plan *P, int ncomp, size_t *off, size_t *stride) {
  if (!P || !off || ncomp <= 0) return fail(NYX_EINVAL, "null argument or ncomp <= 0");
  for (int b = 0; b < P->nbox; ++b) {
    off[b] = (size_t)ncomp * (size_t)P->hbox[b].pref;
    if (stride) stride[b] = (size_t)P->hbox[b].stride;
  }
  off[P->nbox] = (size_t)ncomp * (size_t)P->total_stride;
  return NYX_OK;
}

int nyx_hydro_fill(nyx_plan *P, double *field, int ncomp) {
  if (!P || !field || ncomp <= 0) return fail(NYX_EINVAL, "null argument or ncomp <= 0");
  do_fill(P, field, ncomp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ghost fill launch");
  return NYX_OK;
}

int nyx_hydro_estdt(nyx_plan *P, const nyx_level *L, const double *a_dev, double *dt_dev) {
  if (!P || !L || !a_dev || !dt_dev || !L->state[L->cur & 1])
    return fail(NYX_EINVAL, "null argument");
  do_estdt(P, L->state[L->cur & 1], a_dev, dt_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "estdt launch");
  return NYX_OK;
}

int nyx_hydro_advance(nyx_plan *P, nyx_level *L, const double *a_old, const double *a_new,
                      const double *dt, const double *grav, double *dt_next) {
  if (!P || !L || !a_old || !a_new || !dt) return fail(NYX_EINVAL, "null argument");
  if ((L->cur != 0 && L->cur != 1) || !L->state[0] || !L->state[1] || L->state[0] == L->state[1])
    return fail(NYX_EINVAL, "level needs two distinct state buffers and cur in {0,1}");
  return do_advance(P, L, a_old, a_new, dt, grav, dt_next);
}

int nyx_hydro_predict(nyx_plan *P, nyx_level *L, const double *a_old, const double *a_new,
                      const double *dt, const double *grav_old) {
  if (!P || !L || !a_old || !a_new || !dt) return fail(NYX_EINVAL, "null argument");
  if ((L->cur != 0 && L->cur != 1) || !L->state[0] || !L->state[1] || L->state[0] == L->state[1])
    return fail(NYX_EINVAL, "level needs two distinct state buffers and cur in {0,1}");
  return do_advance(P, L, a_old, a_new, dt, grav_old, nullptr, true);
}

int nyx_hydro_correct(nyx_plan *P, nyx_level *L, const double *a_old, const double *a_new,
                      const double *dt, const double *grav_old, const double *grav_new,
                      double *dt_next) {
  if (!P || !L || !a_old || !a_new || !dt) return fail(NYX_EINVAL, "null argument");
  if ((L->cur != 0 && L->cur != 1) || !L->state[0] || !L->state[1] || L->state[0] == L->state[1])
    return fail(NYX_EINVAL, "level needs two distinct state buffers and cur in {0,1}");
  return do_correct(P, L, a_old, a_new, dt, grav_old, grav_new, dt_next);
}

int nyx_hydro_run(nyx_plan *P, nyx_level *L, const double *a_dev, double *dt_dev, int nsteps,
                  int compute_dt0, int use_graph) {
  if (!P || !L || !a_dev || !dt_dev || nsteps < 0) return fail(NYX_EINVAL, "null argument");
  if ((L->cur != 0 && L->cur != 1) || !L->state[0] || !L->state[1] || L->state[0] == L->state[1])
    return fail(NYX_EINVAL, "level needs two distinct state buffers and cur in {0,1}");
  // box groups (made once, outside any capture): a run overlaps each group's
  // ghost fill with the other groups' advances
  if (P->prm.batching != NYX_PER_BOX && P->ngrp == 0)
    if (int rc = setup_readback(P)) return rc;
  if (!use_graph) return enqueue_run(P, L, a_dev, dt_dev, nsteps, compute_dt0);
  if (P->prm.batching == NYX_PERSISTENT && P->prm.autotune && !P->tuned) {
    // tune outside the capture: one eager step on scratch copies is not
    // possible without the caller's buffers, so tune on the real ones and
    // redo the work below (the tuning launches only write state[1-cur]).
    FusedArgs a{};
    a.boxes = P->d_boxes;
    a.queue = P->d_queue;
    a.K = P->d_K;
    a.SC = P->d_SC;
    a.BS = P->d_BS;
    a.S = L->state[L->cur];
    a.G = L->grav;
    a.Sn = L->state[1 - L->cur];
    a.status = P->d_status_tune;
    a.variant = variant_bits(P);
    a.flat = P->d_flat;
    // time the shapes on the first step as it will run: its own dt
    if (compute_dt0) do_estdt(P, L->state[L->cur], a_dev, dt_dev);
    do_fill(P, L->state[L->cur], NCONS);
    if (int rc = do_flatten(P, L->state[L->cur])) return rc;
    launch_step_setup(P->d_K, a_dev, a_dev + 1, dt_dev, P->d_SC, P->d_boxes, P->nbox, P->d_BS,
                      P->stream);
    int rc = tune_shape(P, a);
    if (rc) return rc;
  }
  if (P->prm.batching == NYX_PERSISTENT) prepare_tmaps(P, L);
  GraphKey key(L->state[0], L->state[1], L->grav, L->cur, a_dev, dt_dev, nsteps, compute_dt0);
  auto it = P->graphs.find(key);
  if (it == P->graphs.end()) {
    nyx_level tmp = *L;
    long long before = P->launches;
    CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_run(P, &tmp, a_dev, dt_dev, nsteps, compute_dt0);
    long long in_graph = P->launches - before;
    P->launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(P->stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    it = P->graphs.emplace(key, std::make_pair(ge, in_graph)).first;
  }
  CK(cudaGraphLaunch(it->second.first, P->stream));
  P->launches += it->second.second;
  L->cur = (L->cur + nsteps) & 1;
  P->flux_valid = P->d_flux != nullptr;
  return NYX_OK;
}

int nyx_hydro_fluxes(nyx_plan *P, const nyx_level *L, int box, int dir, double *out) {
  (void)L;
  if (!P || !out) return fail(NYX_EINVAL, "null argument");
  if (box < 0 || box >= P->nbox || dir < 0 || dir > 2) return fail(NYX_EINVAL, "box or dir out of range");
  if (!P->d_flux) return fail(NYX_EINVAL, "plan was made without keep_fluxes");
  if (!P->flux_valid) return fail(NYX_EINVAL, "no advance has run yet");
  const BoxDev &X = P->hbox[box];
  long long off = P->flux_off[box];
  for (int d = 0; d < dir; ++d)
    off += 6LL * (X.n[0] + (d == 0)) * (X.n[1] + (d == 1)) * (X.n[2] + (d == 2));
  long long n = 6LL * (X.n[0] + (dir == 0)) * (X.n[1] + (dir == 1)) * (X.n[2] + (dir == 2));
  CK(cudaMemcpyAsync(out, P->d_flux + off, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                     P->stream));
  return NYX_OK;
}

int nyx_hydro_step_host(nyx_plan *P, nyx_level *L, const double *host_in, double *host_out,
                        double a_old, double a_new, double *dt_inout) {
  if (!P || !L || !host_in || !host_out || !dt_inout) return fail(NYX_EINVAL, "null argument");
  if ((L->cur != 0 && L->cur != 1) || !L->state[0] || !L->state[1] || L->state[0] == L->state[1])
    return fail(NYX_EINVAL, "level needs two distinct state buffers and cur in {0,1}");
  size_t bytes = sizeof(double) * (size_t)NCONS * (size_t)P->total_stride;
  double h[3] = {a_old, a_new, *dt_inout};
  CK(cudaMemcpyAsync(L->state[L->cur], host_in, bytes, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->d_scal, h, 3 * sizeof(double), cudaMemcpyHostToDevice, P->stream));
  if (!(*dt_inout > 0.0)) do_estdt(P, L->state[L->cur], P->d_scal, P->d_scal + 2);
  int rc = do_advance(P, L, P->d_scal, P->d_scal + 1, P->d_scal + 2, nullptr, P->d_scal + 3);
  if (rc) return rc;
  CK(cudaMemcpyAsync(host_out, L->state[L->cur], bytes, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaMemcpyAsync(dt_inout, P->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return NYX_OK;
}

int nyx_hydro_step_host_valid(nyx_plan *P, nyx_level *L, const double *host_in, double *host_out,
                              double a_old, double a_new, double *dt_inout) {
  if (!P || !L || !host_in || !host_out || !dt_inout) return fail(NYX_EINVAL, "null argument");
  if ((L->cur != 0 && L->cur != 1) || !L->state[0] || !L->state[1] || L->state[0] == L->state[1])
    return fail(NYX_EINVAL, "level needs two distinct state buffers and cur in {0,1}");
  if (!P->d_packed) {
    std::vector<int> pp(P->nbox);
    long long nb = 0;
    for (int b = 0; b < P->nbox; ++b) {
      pp[b] = (int)nb;
      nb += P->hbox[b].n[2];
    }
    if (nb > 0x7fffffffLL) return fail(NYX_EINVAL, "too many box planes for one launch");
    cudaError_t e = cudaMalloc(&P->d_packed, sizeof(double) * NCONS * (size_t)P->total_cells);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_plane_pref, sizeof(int) * P->nbox);
    if (e == cudaSuccess)
      e = cudaMemcpy(P->d_plane_pref, pp.data(), sizeof(int) * P->nbox, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(P->d_packed);
      cudaFree(P->d_plane_pref);
      P->d_packed = nullptr;
      P->d_plane_pref = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(NYX_ENOMEM, "packed state allocation failed")
                                            : cuda_fail(e, "packed state set-up");
    }
    P->plane_blocks = (int)nb;
    P->plane_pref = pp;
  }
  if (P->prm.batching != NYX_PER_BOX && P->ngrp == 0)
    if (int rc = setup_readback(P)) return rc;
  if (P->prm.batching != NYX_PER_BOX && !(P->prm.autotune && !P->tuned)) prepare_tmaps(P, L);
  const size_t bytes = sizeof(double) * NCONS * (size_t)P->total_cells;
  double h[3] = {a_old, a_new, *dt_inout};
  CK(cudaMemcpyAsync(P->d_scal, h, 3 * sizeof(double), cudaMemcpyHostToDevice, P->stream));
  if (P->ngrp > 1 && *dt_inout > 0.0 && !(P->prm.autotune && !P->tuned)) {
    // input, advance and read-back overlapped per box group
    int rc = step_pipelined(P, L, host_in, host_out);
    if (rc) {
      cudaStreamSynchronize(P->h2d_stream);
      cudaStreamSynchronize(P->stream2);
      cudaStreamSynchronize(P->copy_stream);
      return rc;
    }
    CK(cudaMemcpyAsync(dt_inout, P->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost,
                       P->stream));
    CK(cudaStreamSynchronize(P->stream));
    CK(cudaStreamSynchronize(P->h2d_stream));
    CK(cudaStreamSynchronize(P->stream2));
    CK(cudaStreamSynchronize(P->copy_stream));
    return NYX_OK;
  }
  CK(cudaMemcpyAsync(P->d_packed, host_in, bytes, cudaMemcpyHostToDevice, P->stream));
  launch_valid_copy(L->state[L->cur], P->d_packed, P->d_boxes, P->d_cell_pref, P->d_plane_pref,
                    P->nbox, P->plane_blocks, 0, 1, P->stream);
  P->launches += 1;
  if (!(*dt_inout > 0.0)) do_estdt(P, L->state[L->cur], P->d_scal, P->d_scal + 2);
  if (P->ngrp > 1) {
    // the read-back of each box group overlaps the advance of the next ones
    int rc = do_advance(P, L, P->d_scal, P->d_scal + 1, P->d_scal + 2, nullptr, P->d_scal + 3,
                        false, host_out);
    if (rc) {
      cudaStreamSynchronize(P->copy_stream);
      return rc;
    }
    CK(cudaMemcpyAsync(dt_inout, P->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost,
                       P->stream));
    CK(cudaStreamSynchronize(P->stream));
    CK(cudaStreamSynchronize(P->copy_stream));
    return NYX_OK;
  }
  int rc = do_advance(P, L, P->d_scal, P->d_scal + 1, P->d_scal + 2, nullptr, P->d_scal + 3);
  if (rc) return rc;
  launch_valid_copy(L->state[L->cur], P->d_packed, P->d_boxes, P->d_cell_pref, P->d_plane_pref,
                    P->nbox, P->plane_blocks, 0, 0, P->stream);
  P->launches += 1;
  CK(cudaMemcpyAsync(host_out, P->d_packed, bytes, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaMemcpyAsync(dt_inout, P->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return NYX_OK;
}

int nyx_hydro_tile_shape(int shape, int *tx, int *ty) {
  if (shape < 0 || shape >= fused_num_shapes(NYX_MIXED)) return fail(NYX_EINVAL, "tile shape out of range");
  TileShape t = fused_shape(shape);
  if (tx) *tx = t.tx;
  if (ty) *ty = t.ty;
  return NYX_OK;
}

int nyx_task_items(int nbox, const int *n, int tx, int ty, int slots, int chunk, int *items,
                   int cap, int *count) {
  if (nbox < 0 || (nbox > 0 && !n) || tx < 1 || ty < 1 || slots < 1 || cap < 0 ||
      (cap > 0 && !items) || !count)
    return fail(NYX_EINVAL, "bad arguments to nyx_task_items");
  std::vector<std::array<int, 3>> e(nbox);
  for (int b = 0; b < nbox; ++b) {
    e[b] = {n[3 * b], n[3 * b + 1], n[3 * b + 2]};
    if (e[b][0] < 1 || e[b][1] < 1 || e[b][2] < 1) return fail(NYX_EINVAL, "empty box");
  }
  std::vector<WorkItem> it = task_items(e, tx, ty, slots, chunk != 0);
  *count = (int)it.size();
  for (int i = 0; i < std::min(cap, (int)it.size()); ++i) {
    const WorkItem &w = it[i];
    const int v[7] = {w.box, w.x0, w.y0, w.nx, w.ny, w.z0, w.nz};
    std::memcpy(items + 7 * i, v, sizeof v);
  }
  return NYX_OK;
}

int nyx_hydro_set_tile_shape(nyx_plan *P, int shape) {
  if (!P) return fail(NYX_EINVAL, "null plan");
  if (P->prm.batching != NYX_PERSISTENT) return fail(NYX_EINVAL, "plan is not persistent");
  if (shape < 0 || shape >= fused_num_shapes(P->prm.precision)) return fail(NYX_EINVAL, "tile shape out of range");
  for (auto &pt : P->parts) {
    cudaFree(pt.d_items);
    cudaFree(pt.d_items_grp);
  }
  P->parts.clear();
  P->shape = shape;
  P->tuned = true;
  return NYX_OK;
}

int nyx_hydro_tune_info(const nyx_plan *P, int *classes, int *trials, int *launches) {
  if (!P) return fail(NYX_EINVAL, "null plan");
  if (classes) *classes = P->tune_classes;
  if (trials) *trials = P->tune_trials;
  if (launches) *launches = P->parts.empty() ? 1 : (int)P->parts.size();
  return NYX_OK;
}

int nyx_hydro_get_tile_shape(const nyx_plan *P, int *shape) {
  if (!P || !shape) return fail(NYX_EINVAL, "null argument");
  *shape = P->shape;
  return NYX_OK;
}

int nyx_hydro_profile(nyx_plan *P, int enable) {
  if (!P) return fail(NYX_EINVAL, "null plan");
  P->profiling = enable != 0;
  return NYX_OK;
}

int nyx_hydro_counters_read(nyx_plan *P, int reset, nyx_hydro_counters *out) {
  if (!P || !out) return fail(NYX_EINVAL, "null argument");
  CK(cudaStreamSynchronize(P->stream));
  auto sum = [](std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v, double &ms, long long &n) {
    ms = 0.0;
    n = (long long)v.size();
    for (auto &e : v) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, e.first, e.second) == cudaSuccess) ms += t;
    }
  };
  sum(P->ev_fill, out->fill_ms, out->timed_fills);
  sum(P->ev_adv, out->advance_ms, out->timed_advances);
  sum(P->ev_flat, out->flatten_ms, out->timed_flattens);
  out->launches = P->launches;
  if (reset) {
    for (auto &e : P->ev_fill) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    for (auto &e : P->ev_adv) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    for (auto &e : P->ev_flat) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    P->ev_fill.clear();
    P->ev_adv.clear();
    P->ev_flat.clear();
    P->launches = 0;
  }
  return NYX_OK;
}

int nyx_hydro_status(nyx_plan *P, int *flags) {
  if (!P) return fail(NYX_EINVAL, "null plan");
  CK(cudaStreamSynchronize(P->stream));
  unsigned st = 0;
  CK(cudaMemcpy(&st, P->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CK(cudaMemset(P->d_status, 0, sizeof(unsigned)));
  if (flags) *flags = (int)st;
  if (st & ST_NONFINITE) return fail(NYX_ENONFINITE, "non-finite value in an updated state");
  if (st & ST_NEGATIVE) return fail(NYX_ENEGATIVE, "density <= 0 after an update");
  if (st & ST_TIMEOUT) return fail(NYX_ETIMEOUT, "a bounded device wait gave up");
  if (st & ST_OVERRUN) return fail(NYX_ECUDA, "work queue overrun");
  return NYX_OK;
}

int nyx_plan_destroy(nyx_plan *P) {
  if (!P) return fail(NYX_EINVAL, "null plan");
  cudaStreamSynchronize(P->stream);
  free_plan(P);
  return NYX_OK;
}

}  // extern "C"
