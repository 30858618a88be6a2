// nyx_fused2.cuh -- the mixed-precision fused advance, task form.
//
// Same algorithm as nyx_fused.cuh (see its header), with a different
// mapping onto the SM: every per-column value lives in shared memory
// (structure-of-arrays, [field][column]) and each stage is a list of
// independent tasks that the column threads take in order (three threads
// per column).  Per plane c the column threads run four stages:
//
//   S1 tracing at plane c, one direction per thread (x, y, z)
//   S2 normal solves: x, y faces of plane c, z face c-1/2
//   S3 intermediate solves, each task first correcting its face's two
//      states by the transverse normal fluxes (theta = 1/3): F^{x|y}, F^{y|x}
//      at c; F^{x|z}, F^{y|z} at c-1; F^{z|x}, F^{z|y} at face c-1/2
//   S4 final solves, each task first correcting its face's two states by
//      the intermediate fluxes (theta = 1/2): x, y faces of plane c-1, z
//      face c-1/2
//
// Each corrected state feeds exactly one face, so correcting it inside that
// face's task does the same arithmetic as a separate correction stage,
// without storing the states or a barrier between the two.  The z tasks
// also correct the high side of plane c, kept in a two-plane ring for the
// next plane's face.  S2-S4 take per-tile lists of the faces the tile needs.
//
// The FP64 update (stage 7) runs on its own warps, one output cell per
// thread, decoupled from the column threads' stage barriers: the column
// threads hand over the final fluxes of plane c-1 through named barriers
// (READY after they are stored, FREE before the buffer is overwritten), so
// the update of one plane, bound by the FP64 pipe and the state loads,
// overlaps all stages of the next plane instead of lengthening one of them.
// The update of plane p may run until the final fluxes of plane p+1 are
// stored, so the x/y flux buffer is single and the z-face buffer holds two
// faces.
//
// The update warps also load each plane's inputs, which the column threads
// used to load in a stage of their own (stage 0): primitive plane c+2 into
// the ring, plane c into the framed buffer with its 3-cell frame, and plane
// c's gravity and flattening rows.  Their FP64 update leaves the integer
// pipe, which does the conversions, idle.  Two more named barriers hand the
// inputs over: LOADED once they are written, CONSUMED once the column
// threads have traced plane c (the last read of ring plane c-2 and of the
// framed plane), before the update warps overwrite them.
//
// At 16 x 8 tiles (one CTA per SM) the update warps take each plane's state
// (at plane c+2, for the ring) and gravity (at plane c) from staging buffers
// that tensor copies (TMA, cp.async.bulk.tensor with per-box descriptors)
// fill one plane ahead: two buffers for alternate planes, the next plane's
// copies sent as soon as every update thread is past the plane that last
// read that buffer, each buffer completing on its own mbarrier whose wait is
// bounded.  The frame strips and the update's own reads stay plain loads.
//
// Rings over planes: slot = (plane + 2) & 1 for the two-plane rings, and
// (plane + 8) % 5 for the five-plane primitive ring.
#pragma once
#include <type_traits>

#include "nyx_fused.cuh"

namespace NYX_NS {

template <int TX, int TY, int XU>
struct G2 {
  static constexpr int W = TX + 2, H = TY + 2, NC = W * H;
  static constexpr int NCP = (NC + 31) / 32 * 32;  // task stride of one kind
  static constexpr int WE = TX + 6, HE = TY + 6, NE = WE * HE;
  static constexpr int NTC = 3 * NCP;                     // column-task threads
  // update threads: one per output cell, plus XU that only load inputs
  static constexpr int NU = (TX * TY + 31) / 32 * 32 + XU;
  static constexpr int NT = NTC + NU;
  // final fluxes of one plane, compact over the output cells: x faces
  // [(TX+1) x TY], then y faces [TX x (TY+1)]; z faces [TX x TY]
  static constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1), NUF = NXF + NYF, NZF = TX * TY;
  // shared layout, in floats
  static constexpr int PR = 0;                       // [5 planes][5 vars][NC] primitives ring
  static constexpr int PE = PR + 25 * NC;            // [5 vars][NE] plane c with its 3-cell frame
  static constexpr int QXY = PE + 5 * NE;            // [2 planes][2 dirs x,y][10][NC] traced x, y
  static constexpr int QZ = QXY + 40 * NC;           // [2 planes][10][NC] traced z
  static constexpr int FZ = QZ + 20 * NC;            // [2 faces][7][NC] normal z fluxes
  static constexpr int QZXP = FZ + 14 * NC;          // [2 planes][5][NC] q_{z|x} high side
  static constexpr int QZYP = QZXP + 10 * NC;        // [2][5][NC] q_{z|y} high side
  static constexpr int FZXY = QZYP + 10 * NC;        // [2 faces][2 kinds z|x, z|y][7][NC]
  static constexpr int QZFP = FZXY + 28 * NC;        // [2 planes][5][NC] final z, high side
  static constexpr int FN = QZFP + 10 * NC;          // [14][NC] normal x, y fluxes, plane c
  static constexpr int P1 = FN + 14 * NC;            // [28][NC] Fxy, Fyx (c) | Fxz, Fyz (c-1)
  static constexpr int GR = P1 + 28 * NC;            // [4][NC] gravity and flattening, plane c
  static constexpr int UF = GR + 4 * NC;             // [8][NUF] final x, y fluxes of plane c-1
  static constexpr int FFZ = UF + 8 * NUF;           // [2 faces][8][NZF] final z fluxes
  // task lists of stages S2-S4 for the full tile (ushort entries)
  static constexpr int T2 = (TX + 1) * H + W * (TY + 1) + NC;
  static constexpr int T3 = (TX + 1) * TY + TX * (TY + 1) + (TX + 1) * H + W * (TY + 1) + TX * H + W * TY;
  static constexpr int T4 = (TX + 1) * TY + TX * (TY + 1) + TX * TY;
  static constexpr int TT = T2 + T3 + T4;
  static constexpr int TAB = FFZ + 16 * NZF;         // [TT] ushort task lists
  static constexpr int TOTAL0 = TAB + (TT + 1) / 2;
  // TMA staging (16 x 8 tiles at one CTA per SM): one plane of the state
  // (6 components) and of gravity (3) over the tile's columns, x from x0 + 2
  // (an even coordinate: 16-byte aligned) for SX doubles, y from y0 + 3 for H
  // rows, as FP64, in two buffers for alternate planes, and the mbarriers the
  // copies complete on
  static constexpr bool TMA = (TX == 16 && TY == 8 && XU > 0);
  static constexpr int SX = TX + 4;
  static constexpr int STG = (TOTAL0 + 255) / 256 * 256;  // 1024-byte aligned
  // two buffers, used by alternate planes: [6][H][SX] + [3][H][SX] doubles each
  // one buffer, in floats, rounded up to 128 bytes (a tensor copy's
  // destination must be 128-byte aligned)
  static constexpr int STGB = (2 * 9 * H * SX + 31) / 32 * 32;
  static constexpr int STGS = STG;                        // state part of buffer 0
  static constexpr int STGG = STGS + 2 * 6 * H * SX;      // gravity part of buffer 0
  static constexpr int MBAR = STG + 2 * STGB;             // two 8-byte mbarriers
  static_assert((STGG - STGS) % 32 == 0, "gravity staging must start on a 128-byte boundary");
  static constexpr unsigned STG_BYTES_S = 8u * 6 * H * SX, STG_BYTES_G = 8u * 3 * H * SX;
  // + 32 floats: the staging area is aligned to 128 bytes at run time
  static constexpr int TOTAL = TMA ? MBAR + 4 + 32 : TOTAL0;
  static constexpr size_t SMEM = sizeof(float) * (size_t)TOTAL;
  static_assert(SMEM <= 227 * 1024, "task-form tile does not fit in shared memory");
};

// ---------------------------------------------------------------- TMA staging
// A CTA's tensor copies (cp.async.bulk.tensor) land in shared memory and
// complete on an mbarrier; waits are bounded and a wait that gives up raises
// ST_TIMEOUT and switches the CTA to plain loads.
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(void *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(void *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(void *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// bounded wait for phase `parity`; false if it gave up
__device__ __forceinline__ bool mbar_wait(void *bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 20); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_4d(void *dst, const void *tmap, int x, int y, int z, int c,
                                            void *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tmap_acquire(const void *tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Extra loading-only update threads: two warps when one CTA holds the SM
// (24 warps at 80 registers fit the per-scheduler register files), none
// when two CTAs share it.
#define XU_OF(MB) ((MB) == 1 ? 64 : 0)

// Named barriers: 0 is __syncthreads (all threads, item fetch and tile end);
// the column threads' stage barrier; the flux hand-over pair; the input
// hand-over pair.
constexpr int BAR_COL = 1, BAR_READY = 2, BAR_FREE = 3, BAR_LOADED = 4, BAR_CONSUMED = 5;
__device__ __forceinline__ void bar_sync_n(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ int par2(int plane) { return (plane + 2) & 1; }
__device__ __forceinline__ int ring5(int plane) { return (plane + 8) % 5; }

__device__ __forceinline__ void ld5(const float *b, int nc, int cell, float (&q)[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) q[k] = b[k * nc + cell];
}
__device__ __forceinline__ void st5(float *b, int nc, int cell, const float (&q)[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) b[k * nc + cell] = q[k];
}
__device__ __forceinline__ TFlux<float> ld7(const float *b, int nc, int cell) {
  TFlux<float> t;
#pragma unroll
  for (int k = 0; k < 7; ++k) t.f[k] = b[k * nc + cell];
  return t;
}
__device__ __forceinline__ void st7(float *b, int nc, int cell, const float (&F)[8]) {
  b[0 * nc + cell] = F[0];
  b[1 * nc + cell] = F[1];
  b[2 * nc + cell] = F[2];
  b[3 * nc + cell] = F[3];
  b[4 * nc + cell] = F[5];
  b[5 * nc + cell] = F[6];
  b[6 * nc + cell] = F[7];
}
__device__ __forceinline__ void st8(float *b, int nc, int cell, const float (&F)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) b[k * nc + cell] = F[k];
}
__device__ __forceinline__ void ld8(const float *b, int nc, int cell, float (&F)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) F[k] = b[k * nc + cell];
}

// Copy one cell's final fluxes (low faces, and the high faces on the box's
// last column/row/plane) into the flux store of its box: x block (6, nz, ny,
// nx+1), then y block (6, nz, ny+1, nx), then z block (6, nz+1, ny, nx).
__device__ __forceinline__ void keep_fluxes(double *fk, int nx, int ny, int nz, int gx, int gy,
                                            int p, const float (&Fxm)[8], const float (&Fxp)[8],
                                            const float (&Fym)[8], const float (&Fyp)[8],
                                            const float (&Fzm)[8], const float (&Fzp)[8]) {
  const long long fx = (long long)(nx + 1) * ny * nz;
  const long long ix = ((long long)p * ny + gy) * (nx + 1) + gx;
#pragma unroll
  for (int k = 0; k < 6; ++k) fk[k * fx + ix] = (double)Fxm[k];
  if (gx == nx - 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) fk[k * fx + ix + 1] = (double)Fxp[k];
  fk += 6 * fx;
  const long long fy = (long long)nx * (ny + 1) * nz;
  const long long iy = ((long long)p * (ny + 1) + gy) * nx + gx;
#pragma unroll
  for (int k = 0; k < 6; ++k) fk[k * fy + iy] = (double)Fym[k];
  if (gy == ny - 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) fk[k * fy + iy + nx] = (double)Fyp[k];
  fk += 6 * fy;
  const long long fz = (long long)nx * ny * (nz + 1);
  const long long iz = ((long long)p * ny + gy) * nx + gx;
#pragma unroll
  for (int k = 0; k < 6; ++k) fk[k * fz + iz] = (double)Fzm[k];
  if (p == nz - 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) fk[k * fz + iz + (long long)nx * ny] = (double)Fzp[k];
}

// Lab frame (rho, u_x, u_y, u_z, p) <-> the normal frame of face direction
// dir (rho, u_n, u_t1, u_t2, p), with dir warp-uniform: selects, no local
// memory.  Tangential axes in increasing order, as everywhere else.
__device__ __forceinline__ void to_normal(int dir, const float (&q)[5], float (&n)[5]) {
  n[0] = q[0];
  n[1] = (dir == 0) ? q[1] : ((dir == 1) ? q[2] : q[3]);
  n[2] = (dir == 0) ? q[2] : q[1];
  n[3] = (dir == 2) ? q[2] : q[3];
  n[4] = q[4];
}
__device__ __forceinline__ void to_lab(int dir, const float (&n)[5], float (&q)[5]) {
  q[0] = n[0];
  q[1] = (dir == 0) ? n[1] : n[2];
  q[2] = (dir == 0) ? n[2] : ((dir == 1) ? n[1] : n[3]);
  q[3] = (dir == 2) ? n[1] : n[3];
  q[4] = n[4];
}

// One Riemann problem on a direction-dir face; lab-frame states in and
// F = (F_rho, F_mx, F_my, F_mz, F_rhoE, F_rhoe, u_g, p_g) out.
__device__ __forceinline__ void face_flux_dir(const Eos<float> &E, int dir, const float (&ql)[5],
                                              const float (&qr)[5], float (&F)[8]) {
  float nl[5], nr[5], o[8];
  to_normal(dir, ql, nl);
  to_normal(dir, qr, nr);
  riemann_fast(E, nl, nr, o);
  F[0] = o[0];
  F[1] = (dir == 0) ? o[1] : o[2];
  F[2] = (dir == 0) ? o[2] : ((dir == 1) ? o[1] : o[3]);
  F[3] = (dir == 2) ? o[1] : o[3];
  F[4] = o[4];
  F[5] = o[5];
  F[6] = o[6];
  F[7] = o[7];
}

// Task lists of stages S2-S4.  Each kind of task covers a rectangle of the
// tile's columns (local i in [i0, nx-1+di1], j in [j0, ny-1+dj1]; -1 and n
// are the one-cell halo): the faces that the tile's corner-coupled fluxes
// need.  Kinds, in list order: S2 normal x, y, z faces; S3 F^{x|y}, F^{y|x},
// F^{x|z}, F^{y|z}, F^{z|x}, F^{z|y}; S4 final x, y, z faces.
struct KRect {
  int i0, di1, j0, dj1;
};
__device__ __forceinline__ KRect krect(int k) {
  switch (k) {
    case 0: return {0, 1, -1, 1};    // S2 x faces
    case 1: return {-1, 1, 0, 1};    // S2 y faces
    case 2: return {-1, 1, -1, 1};   // S2 z faces
    case 3: return {0, 1, 0, 0};     // S3 F^{x|y}
    case 4: return {0, 0, 0, 1};     // S3 F^{y|x}
    case 5: return {0, 1, -1, 1};    // S3 F^{x|z}
    case 6: return {-1, 1, 0, 1};    // S3 F^{y|z}
    case 7: return {0, 0, -1, 1};    // S3 F^{z|x}
    case 8: return {-1, 1, 0, 0};    // S3 F^{z|y}
    case 9: return {0, 1, 0, 0};     // S4 x faces
    case 10: return {0, 0, 0, 1};    // S4 y faces
    default: return {0, 0, 0, 0};    // S4 z faces
  }
}
__device__ __forceinline__ int kind0_of(int st) { return st == 0 ? 0 : (st == 1 ? 3 : 9); }
__device__ __forceinline__ int nkind_of(int st) { return st == 1 ? 6 : 3; }

// tn[0..2]: the number of tasks of S2..S4 for an nx x ny tile; tn[3], tn[4]:
// the list offsets of S3 and S4 (S2 starts at 0).
__device__ __forceinline__ void task_counts(int nx, int ny, int (&tn)[5]) {
  int off = 0;
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    int n = 0;
    for (int k = kind0_of(st); k < kind0_of(st) + nkind_of(st); ++k) {
      const KRect r = krect(k);
      n += (nx + r.di1 - r.i0) * (ny + r.dj1 - r.j0);
    }
    tn[st] = n;
    if (st > 0) tn[2 + st] = off;
    off += n;
  }
}

// Entries (kind within its stage << 12 | owned column) of every list, in
// kind order, written by threads [0, nthr).
template <int W>
__device__ void build_tasks(unsigned short *tab, int nx, int ny, const int (&tn)[5], int tid,
                            int nthr) {
  const int total = tn[0] + tn[1] + tn[2];
  for (int t = tid; t < total; t += nthr) {
    int st = 0, l = t;
    if (t >= tn[4]) { st = 2; l = t - tn[4]; }
    else if (t >= tn[3]) { st = 1; l = t - tn[3]; }
    const int k0 = kind0_of(st);
    unsigned short e = 0;
    for (int k = 0; k < nkind_of(st); ++k) {
      const KRect r = krect(k0 + k);
      const int w = nx + r.di1 - r.i0, h = ny + r.dj1 - r.j0;
      if (l < w * h) {
        const int i = r.i0 + l % w, j = r.j0 + l / w;
        e = (unsigned short)((k << 12) | ((j + 1) * W + (i + 1)));
        break;
      }
      l -= w * h;
    }
    tab[t] = e;
  }
}

template <int TX, int TY, int MB, int VAR>
__global__ void __launch_bounds__(G2<TX, TY, XU_OF(MB)>::NT, MB) k_fused2(nyx::FusedArgs a) {
  using G = G2<TX, TY, XU_OF(MB)>;
  constexpr int NC = G::NC, NCP = G::NCP, NE = G::NE, W = G::W, WE = G::WE, NT = G::NT;
  constexpr int NTC = G::NTC, NUF = G::NUF, NXF = G::NXF, NZF = G::NZF;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float *sm = reinterpret_cast<float *>(smem_raw);
  __shared__ int s_item;
  __shared__ int s_tma_fail;

  const nyx::SchemeConsts KK = *a.K;
  const nyx::StepConsts sc = *a.SC;
  Eos<float> E = make_eos<float>(KK, true);
  // VAR >= 0 fixes the scheme variant at compile time (bit 0 PLM, bit 1 the
  // linearised solver, bit 2 shock flattening), so the default instantiation
  // carries no variant code
  if constexpr (VAR >= 0) {
    E.plm = VAR & 1;
    E.linear = (VAR >> 1) & 1;
    E.flat = (VAR >> 2) & 1;
  }
  TraceSrc<float> src;
  src.hdtp = d2f_rn(sc.hdtp);
  src.src_u = d2f_rn(sc.src_u);
  src.src_p = d2f_rn(sc.src_p);
  const int tid = threadIdx.x;
  // Threads [0, NTC) take column tasks: every task of such a thread is on one
  // owned column, kind kq (and kq+3 in the six-kind stages) of column me.
  // Threads [NTC, NT) are the update warps: the FP64 update of one output
  // cell each, one plane behind the column threads.
  const bool colthr = tid < NTC;
  const int kq = colthr ? tid / NCP : 3;
  const int me = colthr ? tid - kq * NCP : NCP;
  const int mi = me % W - 1, mj = me / W - 1;
  const int mee = (mj + 3) * WE + (mi + 3);
  float dtmin = __int_as_float(0x7f800000);
  unsigned flags = 0;
  unsigned short *ttab = reinterpret_cast<unsigned short *>(sm + G::TAB);
  int tab_nx = -1, tab_ny = -1;  // the tile extent the lists were built for
  // TMA staging of the update warps' plane inputs (16 x 8 tiles with tensor
  // maps given): phase parity of the mbarrier, and whether copies are used
  // the staging area, moved up to the next 128-byte boundary (tensor copies
  // need a 128-byte aligned destination); offsets below are relative to it
  float *stg = sm + G::STG;
  if constexpr (G::TMA) stg += ((128u - (smem_addr(stg) & 127u)) & 127u) / 4u;
  // buffer k's mbarrier, and the phase parity each update thread waits for
  auto tbar = [&](int k) { return static_cast<void *>(stg + (G::MBAR - G::STG) + 2 * k); };
  unsigned tph0 = 0, tph1 = 0;
  bool use_tma = G::TMA && a.tmS != nullptr && (a.G == nullptr || a.tmG != nullptr);
  if constexpr (G::TMA) {
    if (tid == 0) {
      s_tma_fail = 0;
      mbar_init(tbar(0), 1);
      mbar_init(tbar(1), 1);
    }
  }

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= a.nitems) break;
    const nyx::WorkItem w = a.items[item];
    const nyx::BoxDev b = a.boxes[w.box];
    const int nxt = w.nx, nyt = w.ny, nz = b.n[2];
    const int zb = w.z0, ze = w.z0 + w.nz;  // this item's planes [zb, ze)
    const long long bs = b.stride;
    const long long ps = (long long)b.N[0] * b.N[1];
    const double *S = a.S + nyx::NCONS * b.pref;

    if (colthr) {
      const nyx::BoxStep bst = a.BS[w.box];
      const float dtdx0 = d2f_rn(bst.dtdx[0]), dtdx1 = d2f_rn(bst.dtdx[1]), dtdx2 = d2f_rn(bst.dtdx[2]);
      const float c30 = d2f_rn(bst.cdt3[0]), c31 = d2f_rn(bst.cdt3[1]), c32 = d2f_rn(bst.cdt3[2]);
      const float ch0 = d2f_rn(bst.chalf[0]), ch1 = d2f_rn(bst.chalf[1]), ch2 = d2f_rn(bst.chalf[2]);
      int tn[5];
      task_counts(nxt, nyt, tn);
      if (nxt != tab_nx || nyt != tab_ny) {
        // the previous item's lists are no longer read (item-end barrier)
        build_tasks<W>(ttab, nxt, nyt, tn, tid, NTC);
        tab_nx = nxt;
        tab_ny = nyt;
        bar_sync_n(BAR_COL, NTC);
      }
      // geometry of this thread's column for this tile
      const bool act = me < NC && mi <= nxt && mj <= nyt;
      const bool inX = mi >= 0 && mi < nxt, inY = mj >= 0 && mj < nyt;
      auto ring = [&](int plane) { return sm + G::PR + ring5(plane) * 5 * NC + me; };

      for (int c = zb - 1; c <= ze; ++c) {
        const int pc = par2(c), pm = par2(c - 1);
        const bool zc = c >= zb + 1;
        // ---------------------------------------------- S0: plane c's inputs (update warps)
        bar_sync_n(BAR_LOADED, NT);

        // ---------------------------------------------- S1: tracing at plane c
        // The direction is uniform over a warp (kq = tid / NCP), so each
        // direction runs its own instantiation: lab-frame stencil loads with
        // compile-time strides, no frame permutations.
        if (act) {
          const float *P0 = sm + G::PE;
          const float rho = P0[mee], p = P0[4 * NE + mee];
          const float cs2 = E.gamma * p / rho;
          const float cs = cs2 * rsqrtf(cs2);
          const float g3[3] = {sm[G::GR + me], sm[G::GR + NC + me], sm[G::GR + 2 * NC + me]};
          const float fl = E.flat ? sm[G::GR + 3 * NC + me] : 1.0f;
          auto trace_dir = [&](auto dirc) {
            constexpr int DIR = decltype(dirc)::value;
            float s5[5][5];
#pragma unroll
            for (int o = 0; o < 5; ++o) {
              const float *Po = (DIR == 2) ? ring(c - 2 + o)
                                           : P0 + ((DIR == 0) ? mee + (o - 2) : mee + (o - 2) * WE);
              constexpr int st = (DIR == 2) ? NC : NE;
#pragma unroll
              for (int v = 0; v < 5; ++v) s5[v][o] = Po[v * st];
            }
            const float dtdx = (DIR == 0) ? dtdx0 : ((DIR == 1) ? dtdx1 : dtdx2);
            float qm[5], qp[5];
            trace_cell<float, DIR>(E, s5, cs, g3, dtdx, src, fl, qm, qp);
            float *dst = (DIR == 2) ? sm + G::QZ + pc * 10 * NC : sm + G::QXY + (pc * 2 + DIR) * 10 * NC;
            st5(dst, NC, me, qm);
            st5(dst + 5 * NC, NC, me, qp);
          };
          if (kq == 0)
            trace_dir(std::integral_constant<int, 0>{});
          else if (kq == 1)
            trace_dir(std::integral_constant<int, 1>{});
          else
            trace_dir(std::integral_constant<int, 2>{});
        }
        bar_sync_n(BAR_COL, NTC);
        // ring plane c-2 and the framed plane c are no longer read
        if (c < ze) bar_arrive_n(BAR_CONSUMED, NT);

        // ---------------------------------------------- S2: normal solves
        // Stages S2-S4 run the tile's task lists (built for its extent when the
        // item starts): only the tasks whose faces the tile needs, in kind
        // order, dealt to the column threads in turn.
        for (int t = tid; t < tn[0]; t += NTC) {
          const int e = ttab[t], kind = e >> 12, cm = e & 0xfff;
          const float *L, *Rr;
          float *O;
          int lc;
          if (kind == 0) {
            L = sm + G::QXY + (pc * 2 + 0) * 10 * NC + 5 * NC; lc = cm - 1;
            Rr = sm + G::QXY + (pc * 2 + 0) * 10 * NC; O = sm + G::FN;
          } else if (kind == 1) {
            L = sm + G::QXY + (pc * 2 + 1) * 10 * NC + 5 * NC; lc = cm - W;
            Rr = sm + G::QXY + (pc * 2 + 1) * 10 * NC; O = sm + G::FN + 7 * NC;
          } else {
            L = sm + G::QZ + pm * 10 * NC + 5 * NC; lc = cm;
            Rr = sm + G::QZ + pc * 10 * NC; O = sm + G::FZ + pc * 7 * NC;
          }
          if (kind < 2 || c >= zb) {
            float l[5], r[5], F[8];
            ld5(L, NC, lc, l);
            ld5(Rr, NC, cm, r);
            face_flux_dir(E, kind, l, r, F);
            st7(O, NC, cm, F);
          }
        }
        bar_sync_n(BAR_COL, NTC);

        // ---------------------------------------------- S3: intermediate solves
        // Each task corrects its face's two states by the normal fluxes of the
        // transverse direction (theta = 1/3) and solves: F^{x|y}, F^{y|x} at
        // plane c; F^{x|z}, F^{y|z} at plane c-1; F^{z|x}, F^{z|y} at face
        // c-1/2, whose tasks also correct the high side of plane c for the
        // next plane's face (at plane zb-1 only that).
        for (int t = tid; t < tn[1]; t += NTC) {
          const int e = ttab[tn[3] + t], kind = e >> 12, cm = e & 0xfff;
          const float *Q, *Fmb, *Fpb;
          float *O;
          int foff, lstep, dir;
          float coef;
          switch (kind) {
            case 0:  // F^{x|y} at c: x states corrected by the y fluxes
              Q = sm + G::QXY + (pc * 2 + 0) * 10 * NC; Fmb = Fpb = sm + G::FN + 7 * NC;
              foff = W; coef = c31; lstep = 1; dir = 0; O = sm + G::P1;
              break;
            case 1:  // F^{y|x} at c
              Q = sm + G::QXY + (pc * 2 + 1) * 10 * NC; Fmb = Fpb = sm + G::FN;
              foff = 1; coef = c30; lstep = W; dir = 1; O = sm + G::P1 + 7 * NC;
              break;
            case 2:  // F^{x|z} at c-1: z fluxes of faces c-3/2 and c-1/2
              Q = sm + G::QXY + (pm * 2 + 0) * 10 * NC; Fmb = sm + G::FZ + pm * 7 * NC;
              Fpb = sm + G::FZ + pc * 7 * NC; foff = 0; coef = c32; lstep = 1; dir = 0;
              O = sm + G::P1 + 14 * NC;
              break;
            case 3:  // F^{y|z} at c-1
              Q = sm + G::QXY + (pm * 2 + 1) * 10 * NC; Fmb = sm + G::FZ + pm * 7 * NC;
              Fpb = sm + G::FZ + pc * 7 * NC; foff = 0; coef = c32; lstep = W; dir = 1;
              O = sm + G::P1 + 21 * NC;
              break;
            case 4:  // F^{z|x} at face c-1/2
              Q = sm + G::QZ + pc * 10 * NC; Fmb = Fpb = sm + G::FN;
              foff = 1; coef = c30; lstep = 0; dir = 2; O = sm + G::FZXY + (pc * 2 + 0) * 7 * NC;
              break;
            default:  // F^{z|y} at face c-1/2
              Q = sm + G::QZ + pc * 10 * NC; Fmb = Fpb = sm + G::FN + 7 * NC;
              foff = W; coef = c31; lstep = 0; dir = 2; O = sm + G::FZXY + (pc * 2 + 1) * 7 * NC;
              break;
          }
          float l[5], r[5];
          bool go;
          if (kind < 4) {
            go = kind < 2 || zc;
            if (go) {
              const int lcl = cm - lstep;  // the cell left of the face: its high side
              float q[5];
              ld5(Q + 5 * NC, NC, lcl, q);
              transverse1(E, q, coef, ld7(Fpb, NC, lcl + foff), ld7(Fmb, NC, lcl), l);
              ld5(Q, NC, cm, q);
              transverse1(E, q, coef, ld7(Fpb, NC, cm + foff), ld7(Fmb, NC, cm), r);
            }
          } else {
            // the cell of plane c: its high side for face c+1/2, its low side here
            float *ring_z = sm + ((kind == 4) ? G::QZXP : G::QZYP);
            const TFlux<float> Fm = ld7(Fmb, NC, cm), Fp = ld7(Fpb, NC, cm + foff);
            float q[5], h[5];
            ld5(Q + 5 * NC, NC, cm, q);
            transverse1(E, q, coef, Fp, Fm, h);
            st5(ring_z + pc * 5 * NC, NC, cm, h);
            go = c >= zb;
            if (go) {
              ld5(Q, NC, cm, q);
              transverse1(E, q, coef, Fp, Fm, r);
              ld5(ring_z + pm * 5 * NC, NC, cm, l);
            }
          }
          if (go) {
            float F[8];
            face_flux_dir(E, dir, l, r, F);
            st7(O, NC, cm, F);
          }
        }
        bar_sync_n(BAR_COL, NTC);

        // ---------------------------------------------- S4: final solves
        // Each task corrects its face's two states by the intermediate fluxes
        // of both transverse directions (theta = 1/2) and solves: x and y faces
        // of plane c-1, z face c-1/2 (whose tasks also correct the high side of
        // plane c for the next face).  The fluxes go to the update warps'
        // buffers, written once the update of plane c-2 has released them and
        // handed over after.  The list holds at most one task per column thread.
        {
          bool go = false;
          float F[8];
          int kind = 0, cm = 0;
          if (tid < tn[2]) {
            const int e = ttab[tn[4] + tid];
            kind = e >> 12;
            cm = e & 0xfff;
            float l[5], r[5], q[5];
            if (kind < 2) {
              go = zc;
              if (go) {
                // x: F^{y|z} in y, F^{z|y} in z; y: F^{x|z} in x, F^{z|x} in z
                const float *Q = sm + G::QXY + (pm * 2 + kind) * 10 * NC;
                const float *Ab = sm + G::P1 + (kind == 0 ? 21 : 14) * NC;
                const int aoff = (kind == 0) ? W : 1;
                const float k1c = (kind == 0) ? ch1 : ch0;
                const float *Bmb = sm + G::FZXY + (pm * 2 + (kind == 0 ? 1 : 0)) * 7 * NC;
                const float *Bpb = sm + G::FZXY + (pc * 2 + (kind == 0 ? 1 : 0)) * 7 * NC;
                const int lcl = cm - ((kind == 0) ? 1 : W);
                ld5(Q + 5 * NC, NC, lcl, q);
                transverse2(E, q, k1c, ld7(Ab, NC, lcl + aoff), ld7(Ab, NC, lcl), ch2,
                            ld7(Bpb, NC, lcl), ld7(Bmb, NC, lcl), l);
                ld5(Q, NC, cm, q);
                transverse2(E, q, k1c, ld7(Ab, NC, cm + aoff), ld7(Ab, NC, cm), ch2,
                            ld7(Bpb, NC, cm), ld7(Bmb, NC, cm), r);
              }
            } else {
              // z at plane c: F^{x|y} in x, F^{y|x} in y
              const float *Q = sm + G::QZ + pc * 10 * NC;
              const TFlux<float> Am = ld7(sm + G::P1, NC, cm), Ap = ld7(sm + G::P1, NC, cm + 1);
              const TFlux<float> Bm = ld7(sm + G::P1 + 7 * NC, NC, cm);
              const TFlux<float> Bp = ld7(sm + G::P1 + 7 * NC, NC, cm + W);
              float h[5];
              ld5(Q + 5 * NC, NC, cm, q);
              transverse2(E, q, ch0, Ap, Am, ch1, Bp, Bm, h);
              st5(sm + G::QZFP + pc * 5 * NC, NC, cm, h);
              go = c >= zb;
              if (go) {
                ld5(Q, NC, cm, q);
                transverse2(E, q, ch0, Ap, Am, ch1, Bp, Bm, r);
                ld5(sm + G::QZFP + pm * 5 * NC, NC, cm, l);
              }
            }
            if (go) face_flux_dir(E, kind, l, r, F);
          }
          if (c >= zb + 2) bar_sync_n(BAR_FREE, NT);
          if (go) {
            const int ci = cm % W - 1, cj = cm / W - 1;
            float *O = (kind == 0)   ? sm + G::UF + cj * (TX + 1) + ci
                       : (kind == 1) ? sm + G::UF + NXF + cj * TX + ci
                                     : sm + G::FFZ + (c & 1) * 8 * NZF + cj * TX + ci;
            st8(O, (kind == 2) ? NZF : NUF, 0, F);
          }
          if (c >= zb + 1) {
            __threadfence_block();
            bar_arrive_n(BAR_READY, NT);
          }
        }
        // no barrier here: the next plane's inputs touch nothing S2-S4 read or write
      }
    } else {
      // ------------------------------------------------ update warps (stage 7)
      const int nout = nxt * nyt;
      const int uthr = tid - NTC;
      const bool upd = uthr < nout;
      const int ui = upd ? uthr % nxt : 0, uj = upd ? uthr / nxt : 0;
      const long long ucol = (long long)(w.y0 + uj + 4) * b.N[0] + (w.x0 + ui + 4);
      const double *Gv = a.G ? a.G + nyx::NGRAV * b.pref : nullptr;
      double *Sn = a.Sn + nyx::NCONS * b.pref;
      const MixK mk = make_mixk(KK, sc, b);
      const int ux = uj * (TX + 1) + ui, uy = NXF + uj * TX + ui, uz = uj * TX + ui;
      const int nstrip = 4 * (nxt + 2) + 4 * (nyt + 2);

      auto load_prims = [&](long long id, float *dst, int stride) {
        float q[5];
        prims_of<float>(S, bs, id, E, q);
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * stride] = q[v];
      };
      auto ring_at = [&](int plane) { return sm + G::PR + ring5(plane) * 5 * NC; };
      // the tile's columns: e = (j+1) W + (i+1), i in [-1, nxt], j in [-1, nyt]
      auto column = [&](int e, long long &col) {
        const int ci = e % W - 1, cj = e / W - 1;
        col = (long long)(w.y0 + cj + 4) * b.N[0] + (w.x0 + ci + 4);
        return ci <= nxt && cj <= nyt;
      };
      // tensor copies of inputs(c)'s planes into the staging buffers: the
      // state at plane c+2 (the ring's new plane) and gravity at plane c,
      // over x in [x0+2, x0+2+SX), y in [y0+3, y0+3+H) of the box with ghosts
      // (the tile's columns and their halo; past the box edge the copy fills
      // zeros, which no column reads)
      if (s_tma_fail) use_tma = false;  // a wait gave up in an earlier item: plain loads
      const char *tmS_b = use_tma ? static_cast<const char *>(a.tmS) + 128 * (size_t)w.box : nullptr;
      const char *tmG_b = (use_tma && a.G) ? static_cast<const char *>(a.tmG) + 128 * (size_t)w.box
                                           : nullptr;
      if (G::TMA && use_tma && uthr == 0) {
        tmap_acquire(tmS_b);
        if (tmG_b) tmap_acquire(tmG_b);
      }
      // the copies of inputs(c) go to buffer c & 1
      auto issue = [&](int c) {
        if constexpr (G::TMA) {
          if (uthr == 0) {
            const int k = c & 1;
            float *buf = stg + k * G::STGB;
            fence_async_smem();  // earlier reads of the buffer precede the copies
            mbar_expect_tx(tbar(k), G::STG_BYTES_S + (tmG_b ? G::STG_BYTES_G : 0u));
            tma_load_4d(buf, tmS_b, w.x0 + 2, w.y0 + 3, c + 2 + 4, 0, tbar(k));
            if (tmG_b)
              tma_load_4d(buf + (G::STGG - G::STGS), tmG_b, w.x0 + 2, w.y0 + 3, c + 4, 0, tbar(k));
          }
        }
      };
      // inputs of plane c: ring plane c+2; plane c's gravity, flattening and
      // framed copy (its own columns from the ring, the frame strips loaded)
      auto inputs = [&](int c, bool staged) {
        const float *buf = stg + (c & 1) * G::STGB;
        if (G::TMA && staged) {
          unsigned &ph = (c & 1) ? tph1 : tph0;
          if (mbar_wait(tbar(c & 1), ph)) {
            ph ^= 1u;
          } else {  // gave up: flag it; the phase stays the one still owed
            flags |= nyx::ST_TIMEOUT;
            s_tma_fail = 1;
          }
        }
        for (int e = uthr; e < NC; e += G::NU) {
          long long col;
          if (!column(e, col)) continue;
          const long long id = col + (long long)(c + 4) * ps;
          float g0 = 0.f, g1 = 0.f, g2 = 0.f;
          if (G::TMA && staged) {
            // the column's values from the staging buffers
            const int sidx = (e / W) * G::SX + (e % W + 1);
            const double *stS = reinterpret_cast<const double *>(buf);
            float q[5];
            prims_of<float>(stS, G::H * G::SX, sidx, E, q);
            float *dst = ring_at(c + 2) + e;
#pragma unroll
            for (int v = 0; v < 5; ++v) dst[v * NC] = q[v];
            if (tmG_b) {
              const double *stG = reinterpret_cast<const double *>(buf + (G::STGG - G::STGS));
              g0 = d2f_rn(stG[sidx]);
              g1 = d2f_rn(stG[G::H * G::SX + sidx]);
              g2 = d2f_rn(stG[2 * G::H * G::SX + sidx]);
            }
          } else {
            load_prims(col + (long long)(c + 2 + 4) * ps, ring_at(c + 2) + e, NC);
            if (Gv) {
              g0 = d2f_rn(Gv[id]);
              g1 = d2f_rn(Gv[bs + id]);
              g2 = d2f_rn(Gv[2 * bs + id]);
            }
          }
          sm[G::GR + e] = g0;
          sm[G::GR + NC + e] = g1;
          sm[G::GR + 2 * NC + e] = g2;
          if (E.flat) sm[G::GR + 3 * NC + e] = static_cast<const float *>(a.flat)[b.pref + id];
          const float *rc = ring_at(c) + e;
          const int ee = (e / W + 2) * WE + (e % W + 2);
#pragma unroll
          for (int v = 0; v < 5; ++v) sm[G::PE + v * NE + ee] = rc[v * NC];
        }
        for (int u = uthr; u < nstrip; u += G::NU) {
          int x, y;
          if (u < 4 * (nyt + 2)) {
            const int r = u % (nyt + 2), s2 = u / (nyt + 2);
            y = r - 1;
            x = (s2 < 2) ? (-3 + s2) : (nxt + 1 + (s2 - 2));
          } else {
            const int v = u - 4 * (nyt + 2);
            const int r = v % (nxt + 2), s2 = v / (nxt + 2);
            x = r - 1;
            y = (s2 < 2) ? (-3 + s2) : (nyt + 1 + (s2 - 2));
          }
          const long long id =
              ((long long)(c + 4) * b.N[1] + (w.y0 + y + 4)) * b.N[0] + (w.x0 + x + 4);
          load_prims(id, sm + G::PE + (y + 3) * WE + (x + 3), NE);
        }
      };
      auto update_plane = [&](int p) {
        if (!upd) return;
        float Fxm[8], Fxp[8], Fym[8], Fyp[8], Fzm[8], Fzp[8];
        const float *U = sm + G::UF;
        const float *Zm = sm + G::FFZ + (p & 1) * 8 * NZF, *Zp = sm + G::FFZ + ((p + 1) & 1) * 8 * NZF;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          Fxm[k] = U[k * NUF + ux];
          Fxp[k] = U[k * NUF + ux + 1];
          Fym[k] = U[k * NUF + uy];
          Fyp[k] = U[k * NUF + uy + TX];
          Fzm[k] = Zm[k * NZF + uz];
          Fzp[k] = Zp[k * NZF + uz];
        }
        const long long id = ucol + (long long)(p + 4) * ps;
        update_cell_mixed(KK, sc, b, mk, S, Gv, Sn, id, Fxm, Fxp, Fym, Fyp, Fzm, Fzp, dtmin, flags,
                          a.dtacc != nullptr, !a.predict_only);
        if (a.flux_keep)
          keep_fluxes(a.flux_keep + a.flux_off[w.box], b.n[0], b.n[1], nz, w.x0 + ui, w.y0 + uj, p,
                      Fxm, Fxp, Fym, Fyp, Fzm, Fzp);
      };

      // prologue: ring planes -3 .. 0, then the inputs of plane -1
      for (int e = uthr; e < NC; e += G::NU) {
        long long col;
        if (!column(e, col)) continue;
#pragma unroll 1
        for (int k = zb - 3; k <= zb; ++k)
          load_prims(col + (long long)(k + 4) * ps, ring_at(k) + e, NC);
      }
      inputs(zb - 1, false);  // plain loads
      if (use_tma) issue(zb);
      __threadfence_block();
      bar_arrive_n(BAR_LOADED, NT);
      for (int c = zb; c <= ze; ++c) {
        // plane c-1 traced: its ring plane c-3 slot and the framed plane are
        // free, and every update thread is past inputs(c-1), so buffer
        // (c+1) & 1 is free for the copies of the next plane's inputs
        bar_sync_n(BAR_CONSUMED, NT);
        if (use_tma && c + 1 <= ze) issue(c + 1);
        inputs(c, use_tma);
        __threadfence_block();
        bar_arrive_n(BAR_LOADED, NT);
        if (c >= zb + 2) {
          // the final fluxes of plane c-2 (x, y faces; z faces c-5/2 and c-3/2)
          bar_sync_n(BAR_READY, NT);
          update_plane(c - 2);
          // plane c-2's buffers may be overwritten (by the fluxes of plane c-1)
          bar_arrive_n(BAR_FREE, NT);
        }
      }
      bar_sync_n(BAR_READY, NT);
      update_plane(ze - 1);
    }
    __syncthreads();
  }
  if constexpr (G::TMA) {
    // a wait that gave up may have left copies in flight: wait once more
    // (bounded) before the CTA's shared memory goes
    if (s_tma_fail && tid == NTC) {
      mbar_wait(tbar(0), tph0);
      mbar_wait(tbar(1), tph1);
    }
  }

  if (a.dtacc) {
    for (int o = 16; o > 0; o >>= 1) dtmin = fminf(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
    if ((tid & 31) == 0 && dtmin < __int_as_float(0x7f800000))
      nyx::atomic_min_pos(a.dtacc, (double)dtmin);
  }
  if (flags) atomicOr(a.status, flags);
}

template <int TX, int TY, int MB, int VAR>
int launch_two(const nyx::FusedArgs &a, int grid, cudaStream_t st) {
  using G = G2<TX, TY, XU_OF(MB)>;
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return (int)e;
  k_fused2<TX, TY, MB, VAR><<<grid, G::NT, G::SMEM, st>>>(a);
  return (int)cudaGetLastError();
}

template <int TX, int TY, int MB, int VAR>
int max_grid_two() {
  using G = G2<TX, TY, XU_OF(MB)>;
  cudaError_t e = cudaFuncSetAttribute(k_fused2<TX, TY, MB, VAR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused2<TX, TY, MB, VAR>, G::NT,
                                                G::SMEM);
  if (per_sm < 1) return 0;
  return per_sm * nsm;
}

}  // namespace NYX_NS
