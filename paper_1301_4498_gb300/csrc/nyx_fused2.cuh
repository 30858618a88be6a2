// nyx_fused2.cuh -- the mixed-precision fused advance, task form.
//
// Same algorithm and stage order as nyx_fused.cuh (see its header), with a
// different mapping onto the SM: every per-column value lives in shared
// memory (structure-of-arrays, [field][column]) and each stage is a list of
// independent tasks -- one trace direction of one column, one Riemann
// problem on one face, one corner-coupling correction, one update -- that
// the CTA's threads take in order.  Tasks of one kind are padded to a whole
// number of warps, so a warp runs one kind at a time.  With three threads per
// column a 16 x 8 tile runs 18 warps per SM at <= 113 registers per thread
// (the column-owning form runs 11 warps at 168 with spills), which is what
// the latency-bound Riemann and tracing arithmetic needs.  The FP64 update of
// plane c-1 (stage 7) has no barrier behind it, so it overlaps the loads of
// the next plane.
//
// Rings over planes: slot = (plane + 2) & 1 for the two-plane rings, and
// (plane + 8) % 5 for the five-plane primitive ring.
#pragma once
#include "nyx_fused.cuh"

namespace NYX_NS {

template <int TX, int TY>
struct G2 {
  static constexpr int W = TX + 2, H = TY + 2, NC = W * H;
  static constexpr int NCP = (NC + 31) / 32 * 32;  // task stride of one kind
  static constexpr int WE = TX + 6, HE = TY + 6, NE = WE * HE;
  static constexpr int NT = 3 * NCP;
  // shared layout, in floats
  static constexpr int PR = 0;                       // [5 planes][5 vars][NE] primitives
  static constexpr int QXY = PR + 25 * NE;           // [2 planes][2 dirs x,y][10][NC] traced x, y
  static constexpr int QZ = QXY + 40 * NC;           // [2 planes][10][NC] traced z
  static constexpr int FZ = QZ + 20 * NC;            // [2 faces][7][NC] normal z fluxes
  static constexpr int QZXM = FZ + 14 * NC;          // [5][NC] q_{z|x} low side, plane c
  static constexpr int QZXP = QZXM + 5 * NC;         // [2 planes][5][NC] q_{z|x} high side
  static constexpr int QZYM = QZXP + 10 * NC;        // [5][NC]
  static constexpr int QZYP = QZYM + 5 * NC;         // [2][5][NC]
  static constexpr int FZXY = QZYP + 10 * NC;        // [2 faces][2 kinds z|x, z|y][7][NC]
  static constexpr int QZFM = FZXY + 28 * NC;        // [5][NC] final z state, low side
  static constexpr int QZFP = QZFM + 5 * NC;         // [2 planes][5][NC] final z, high side
  static constexpr int FFZ = QZFP + 10 * NC;         // [2 faces][8][NC] final z fluxes
  static constexpr int P1 = FFZ + 16 * NC;           // [28][NC] pool: FX,FY | Fxy,Fyx,Fxz,Fyz | Ffx,Ffy
  static constexpr int P2 = P1 + 28 * NC;            // [40][NC] pool: qxy,qyx,qxz,qyz | qxf,qyf
  static constexpr int TOTAL = P2 + 40 * NC;
  static constexpr size_t SMEM = sizeof(float) * (size_t)TOTAL;
};

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

template <int TX, int TY, int MB>
__global__ void __launch_bounds__(G2<TX, TY>::NT, MB) k_fused2(nyx::FusedArgs a) {
  using G = G2<TX, TY>;
  constexpr int NC = G::NC, NCP = G::NCP, NE = G::NE, W = G::W, WE = G::WE, NT = G::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *sm = reinterpret_cast<float *>(smem_raw);
  __shared__ int s_item;

  const nyx::SchemeConsts KK = *a.K;
  const nyx::StepConsts sc = *a.SC;
  const Eos<float> E = make_eos<float>(KK, true);
  TraceSrc<float> src;
  src.hdtp = (float)sc.hdtp;
  src.src_u = (float)sc.src_u;
  src.src_p = (float)sc.src_p;
  const int tid = threadIdx.x;
  double dtmin = __longlong_as_double(0x7ff0000000000000LL);
  unsigned flags = 0;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= a.nitems) break;
    const nyx::WorkItem w = a.items[item];
    const nyx::BoxDev b = a.boxes[w.box];
    const nyx::BoxStep bst = a.BS[w.box];
    const int nxt = w.nx, nyt = w.ny, nz = b.n[2];
    const long long bs = b.stride;
    const long long ps = (long long)b.N[0] * b.N[1];
    const double *S = a.S + nyx::NCONS * b.pref;
    const double *Gv = a.G ? a.G + nyx::NGRAV * b.pref : nullptr;
    double *Sn = a.Sn + nyx::NCONS * b.pref;
    const float dtdx[3] = {(float)bst.dtdx[0], (float)bst.dtdx[1], (float)bst.dtdx[2]};
    const float c30 = (float)bst.cdt3[0], c31 = (float)bst.cdt3[1], c32 = (float)bst.cdt3[2];
    const float ch0 = (float)bst.chalf[0], ch1 = (float)bst.chalf[1], ch2 = (float)bst.chalf[2];
    const int nstrip = 4 * (nxt + 2) + 4 * (nyt + 2);
    // column geometry of owned column e
    auto col_i = [&](int e) { return e % W - 1; };
    auto col_j = [&](int e) { return e / W - 1; };
    auto active = [&](int e) { return e < NC && (e % W - 1) <= nxt && (e / W - 1) <= nyt; };
    auto gcol = [&](int i, int j) {
      return (long long)(w.y0 + j + 4) * b.N[0] + (w.x0 + i + 4);
    };
    auto load_prims = [&](long long id, int slot, int ecell) {
      float q[5];
      prims_of<float>(S, bs, id, E, q);
#pragma unroll
      for (int v = 0; v < 5; ++v) sm[G::PR + (slot * 5 + v) * NE + ecell] = q[v];
    };

    // prologue: planes -3 .. 0 of every owned column
    for (int t = tid; t < 4 * NCP; t += NT) {
      const int o = t / NCP, e = t - o * NCP;
      if (!active(e)) continue;
      const int i = col_i(e), j = col_j(e), p = o - 3;
      load_prims(gcol(i, j) + (long long)(p + 4) * ps, ring5(p), (j + 3) * WE + (i + 3));
    }

    for (int c = -1; c <= nz; ++c) {
      const int pc = par2(c), pm = par2(c - 1);
      const bool zc = c >= 1;
      // ------------------------------------------------ S0: primitives
      for (int t = tid; t < NCP + nstrip; t += NT) {
        if (t < NCP) {
          if (!active(t)) continue;
          const int i = col_i(t), j = col_j(t);
          load_prims(gcol(i, j) + (long long)(c + 2 + 4) * ps, ring5(c + 2), (j + 3) * WE + (i + 3));
        } else {
          const int u = t - NCP;
          int x, y;
          if (u < 4 * (nyt + 2)) {
            const int r = u % (nyt + 2), s = u / (nyt + 2);
            y = r - 1;
            x = (s < 2) ? (-3 + s) : (nxt + 1 + (s - 2));
          } else {
            const int v = u - 4 * (nyt + 2);
            const int r = v % (nxt + 2), s = v / (nxt + 2);
            x = r - 1;
            y = (s < 2) ? (-3 + s) : (nyt + 1 + (s - 2));
          }
          load_prims(gcol(x, y) + (long long)(c + 4) * ps, ring5(c), (y + 3) * WE + (x + 3));
        }
      }
      __syncthreads();

      // ------------------------------------------------ S1: tracing at plane c
      for (int t = tid; t < 3 * NCP; t += NT) {
        const int kind = t / NCP, e = t - kind * NCP;
        if (!active(e)) continue;
        const int i = col_i(e), j = col_j(e);
        const int ee = (j + 3) * WE + (i + 3);
        const float *P0 = sm + G::PR + ring5(c) * 5 * NE;
        const float rho = P0[ee], p = P0[4 * NE + ee];
        const float cs2 = E.gamma * p / rho;
        const float cs = cs2 * rsqrtf(cs2);
        float g3[3] = {0.f, 0.f, 0.f};
        if (Gv) {
          const long long id = gcol(i, j) + (long long)(c + 4) * ps;
          g3[0] = (float)Gv[id];
          g3[1] = (float)Gv[bs + id];
          g3[2] = (float)Gv[2 * bs + id];
        }
        float s[5][5], qm[5], qp[5];
        if (kind == 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int o = 0; o < 5; ++o) s[v][o] = P0[v * NE + ee + (o - 2)];
          trace_cell<float, 0>(E, s, cs, g3, dtdx[0], src, qm, qp);
          float *dst = sm + G::QXY + (pc * 2 + 0) * 10 * NC;
          st5(dst, NC, e, qm);
          st5(dst + 5 * NC, NC, e, qp);
        } else if (kind == 1) {
#pragma unroll
          for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int o = 0; o < 5; ++o) s[v][o] = P0[v * NE + ee + (o - 2) * WE];
          trace_cell<float, 1>(E, s, cs, g3, dtdx[1], src, qm, qp);
          float *dst = sm + G::QXY + (pc * 2 + 1) * 10 * NC;
          st5(dst, NC, e, qm);
          st5(dst + 5 * NC, NC, e, qp);
        } else {
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            const float *Po = sm + G::PR + ring5(c - 2 + o) * 5 * NE;
#pragma unroll
            for (int v = 0; v < 5; ++v) s[v][o] = Po[v * NE + ee];
          }
          trace_cell<float, 2>(E, s, cs, g3, dtdx[2], src, qm, qp);
          float *dst = sm + G::QZ + pc * 10 * NC;
          st5(dst, NC, e, qm);
          st5(dst + 5 * NC, NC, e, qp);
        }
      }
      __syncthreads();

      // ------------------------------------------------ S2: normal solves
      for (int t = tid; t < 3 * NCP; t += NT) {
        const int kind = t / NCP, e = t - kind * NCP;
        if (!active(e)) continue;
        const int i = col_i(e), j = col_j(e);
        float l[5], r[5], F[8];
        if (kind == 0) {
          if (i < 0) continue;
          const float *q = sm + G::QXY + (pc * 2 + 0) * 10 * NC;
          ld5(q + 5 * NC, NC, e - 1, l);
          ld5(q, NC, e, r);
          face_flux<float, 0>(E, l, r, F);
          st7(sm + G::P1, NC, e, F);
        } else if (kind == 1) {
          if (j < 0) continue;
          const float *q = sm + G::QXY + (pc * 2 + 1) * 10 * NC;
          ld5(q + 5 * NC, NC, e - W, l);
          ld5(q, NC, e, r);
          face_flux<float, 1>(E, l, r, F);
          st7(sm + G::P1 + 7 * NC, NC, e, F);
        } else {
          if (c < 0) continue;
          ld5(sm + G::QZ + pm * 10 * NC + 5 * NC, NC, e, l);
          ld5(sm + G::QZ + pc * 10 * NC, NC, e, r);
          face_flux<float, 2>(E, l, r, F);
          st7(sm + G::FZ + pc * 7 * NC, NC, e, F);
        }
      }
      __syncthreads();

      // ------------------------------------------------ S3: corner coupling, theta = 1/3
      for (int t = tid; t < 6 * NCP; t += NT) {
        const int kind = t / NCP, e = t - kind * NCP;
        if (!active(e)) continue;
        const int i = col_i(e), j = col_j(e);
        const bool inX = i >= 0 && i < nxt, inY = j >= 0 && j < nyt;
        float qa[5], qb[5], oa[5], ob[5];
        if (kind == 0 || kind == 3) {  // by normal y fluxes: q_{x|y} (0), q_{z|y} (3)
          if (!inY) continue;
          const TFlux<float> Fm = ld7(sm + G::P1 + 7 * NC, NC, e);
          const TFlux<float> Fp = ld7(sm + G::P1 + 7 * NC, NC, e + W);
          const float *q = (kind == 0) ? sm + G::QXY + (pc * 2 + 0) * 10 * NC : sm + G::QZ + pc * 10 * NC;
          ld5(q, NC, e, qa);
          ld5(q + 5 * NC, NC, e, qb);
          transverse1(E, qa, c31, Fp, Fm, oa);
          transverse1(E, qb, c31, Fp, Fm, ob);
          if (kind == 0) {
            st5(sm + G::P2, NC, e, oa);
            st5(sm + G::P2 + 5 * NC, NC, e, ob);
          } else {
            st5(sm + G::QZYM, NC, e, oa);
            st5(sm + G::QZYP + pc * 5 * NC, NC, e, ob);
          }
        } else if (kind == 1 || kind == 2) {  // by normal x fluxes: q_{y|x} (1), q_{z|x} (2)
          if (!inX) continue;
          const TFlux<float> Fm = ld7(sm + G::P1, NC, e);
          const TFlux<float> Fp = ld7(sm + G::P1, NC, e + 1);
          const float *q = (kind == 1) ? sm + G::QXY + (pc * 2 + 1) * 10 * NC : sm + G::QZ + pc * 10 * NC;
          ld5(q, NC, e, qa);
          ld5(q + 5 * NC, NC, e, qb);
          transverse1(E, qa, c30, Fp, Fm, oa);
          transverse1(E, qb, c30, Fp, Fm, ob);
          if (kind == 1) {
            st5(sm + G::P2 + 10 * NC, NC, e, oa);
            st5(sm + G::P2 + 15 * NC, NC, e, ob);
          } else {
            st5(sm + G::QZXM, NC, e, oa);
            st5(sm + G::QZXP + pc * 5 * NC, NC, e, ob);
          }
        } else {  // by normal z fluxes at plane c-1: q_{x|z} (4), q_{y|z} (5)
          if (!zc) continue;
          const TFlux<float> Fm = ld7(sm + G::FZ + pm * 7 * NC, NC, e);
          const TFlux<float> Fp = ld7(sm + G::FZ + pc * 7 * NC, NC, e);
          const float *q = sm + G::QXY + (pm * 2 + (kind - 4)) * 10 * NC;
          ld5(q, NC, e, qa);
          ld5(q + 5 * NC, NC, e, qb);
          transverse1(E, qa, c32, Fp, Fm, oa);
          transverse1(E, qb, c32, Fp, Fm, ob);
          float *dst = sm + G::P2 + (20 + 10 * (kind - 4)) * NC;
          st5(dst, NC, e, oa);
          st5(dst + 5 * NC, NC, e, ob);
        }
      }
      __syncthreads();

      // ------------------------------------------------ S4: intermediate solves
      for (int t = tid; t < 6 * NCP; t += NT) {
        const int kind = t / NCP, e = t - kind * NCP;
        if (!active(e)) continue;
        const int i = col_i(e), j = col_j(e);
        const bool inX = i >= 0 && i < nxt, inY = j >= 0 && j < nyt;
        float l[5], r[5], F[8];
        if (kind == 0) {  // F^{x|y} at plane c
          if (!(i >= 0 && inY)) continue;
          ld5(sm + G::P2 + 5 * NC, NC, e - 1, l);
          ld5(sm + G::P2, NC, e, r);
          face_flux<float, 0>(E, l, r, F);
          st7(sm + G::P1, NC, e, F);
        } else if (kind == 1) {  // F^{y|x} at plane c
          if (!(j >= 0 && inX)) continue;
          ld5(sm + G::P2 + 15 * NC, NC, e - W, l);
          ld5(sm + G::P2 + 10 * NC, NC, e, r);
          face_flux<float, 1>(E, l, r, F);
          st7(sm + G::P1 + 7 * NC, NC, e, F);
        } else if (kind == 2) {  // F^{x|z} at plane c-1
          if (!(zc && i >= 0)) continue;
          ld5(sm + G::P2 + 25 * NC, NC, e - 1, l);
          ld5(sm + G::P2 + 20 * NC, NC, e, r);
          face_flux<float, 0>(E, l, r, F);
          st7(sm + G::P1 + 14 * NC, NC, e, F);
        } else if (kind == 3) {  // F^{y|z} at plane c-1
          if (!(zc && j >= 0)) continue;
          ld5(sm + G::P2 + 35 * NC, NC, e - W, l);
          ld5(sm + G::P2 + 30 * NC, NC, e, r);
          face_flux<float, 1>(E, l, r, F);
          st7(sm + G::P1 + 21 * NC, NC, e, F);
        } else if (kind == 4) {  // F^{z|x} at face c-1/2
          if (!(c >= 0 && inX)) continue;
          ld5(sm + G::QZXP + pm * 5 * NC, NC, e, l);
          ld5(sm + G::QZXM, NC, e, r);
          face_flux<float, 2>(E, l, r, F);
          st7(sm + G::FZXY + (pc * 2 + 0) * 7 * NC, NC, e, F);
        } else {  // F^{z|y} at face c-1/2
          if (!(c >= 0 && inY)) continue;
          ld5(sm + G::QZYP + pm * 5 * NC, NC, e, l);
          ld5(sm + G::QZYM, NC, e, r);
          face_flux<float, 2>(E, l, r, F);
          st7(sm + G::FZXY + (pc * 2 + 1) * 7 * NC, NC, e, F);
        }
      }
      __syncthreads();

      // ------------------------------------------------ S5: final states, theta = 1/2
      for (int t = tid; t < 3 * NCP; t += NT) {
        const int kind = t / NCP, e = t - kind * NCP;
        if (!active(e)) continue;
        const int i = col_i(e), j = col_j(e);
        const bool inX = i >= 0 && i < nxt, inY = j >= 0 && j < nyt;
        float qa[5], qb[5], oa[5], ob[5];
        if (kind == 0) {  // z at plane c: by F^{x|y} in x, F^{y|x} in y
          if (!(inX && inY)) continue;
          const TFlux<float> Am = ld7(sm + G::P1, NC, e), Ap = ld7(sm + G::P1, NC, e + 1);
          const TFlux<float> Bm = ld7(sm + G::P1 + 7 * NC, NC, e), Bp = ld7(sm + G::P1 + 7 * NC, NC, e + W);
          const float *q = sm + G::QZ + pc * 10 * NC;
          ld5(q, NC, e, qa);
          ld5(q + 5 * NC, NC, e, qb);
          transverse2(E, qa, ch0, Ap, Am, ch1, Bp, Bm, oa);
          transverse2(E, qb, ch0, Ap, Am, ch1, Bp, Bm, ob);
          st5(sm + G::QZFM, NC, e, oa);
          st5(sm + G::QZFP + pc * 5 * NC, NC, e, ob);
        } else if (kind == 1) {  // x at plane c-1: by F^{y|z} in y, F^{z|y} in z
          if (!(zc && inY)) continue;
          const TFlux<float> Am = ld7(sm + G::P1 + 21 * NC, NC, e);
          const TFlux<float> Ap = ld7(sm + G::P1 + 21 * NC, NC, e + W);
          const TFlux<float> Bm = ld7(sm + G::FZXY + (pm * 2 + 1) * 7 * NC, NC, e);
          const TFlux<float> Bp = ld7(sm + G::FZXY + (pc * 2 + 1) * 7 * NC, NC, e);
          const float *q = sm + G::QXY + (pm * 2 + 0) * 10 * NC;
          ld5(q, NC, e, qa);
          ld5(q + 5 * NC, NC, e, qb);
          transverse2(E, qa, ch1, Ap, Am, ch2, Bp, Bm, oa);
          transverse2(E, qb, ch1, Ap, Am, ch2, Bp, Bm, ob);
          st5(sm + G::P2, NC, e, oa);
          st5(sm + G::P2 + 5 * NC, NC, e, ob);
        } else {  // y at plane c-1: by F^{x|z} in x, F^{z|x} in z
          if (!(zc && inX)) continue;
          const TFlux<float> Am = ld7(sm + G::P1 + 14 * NC, NC, e);
          const TFlux<float> Ap = ld7(sm + G::P1 + 14 * NC, NC, e + 1);
          const TFlux<float> Bm = ld7(sm + G::FZXY + (pm * 2 + 0) * 7 * NC, NC, e);
          const TFlux<float> Bp = ld7(sm + G::FZXY + (pc * 2 + 0) * 7 * NC, NC, e);
          const float *q = sm + G::QXY + (pm * 2 + 1) * 10 * NC;
          ld5(q, NC, e, qa);
          ld5(q + 5 * NC, NC, e, qb);
          transverse2(E, qa, ch0, Ap, Am, ch2, Bp, Bm, oa);
          transverse2(E, qb, ch0, Ap, Am, ch2, Bp, Bm, ob);
          st5(sm + G::P2 + 10 * NC, NC, e, oa);
          st5(sm + G::P2 + 15 * NC, NC, e, ob);
        }
      }
      __syncthreads();

      // ------------------------------------------------ S6: final solves
      for (int t = tid; t < 3 * NCP; t += NT) {
        const int kind = t / NCP, e = t - kind * NCP;
        if (!active(e)) continue;
        const int i = col_i(e), j = col_j(e);
        const bool inX = i >= 0 && i < nxt, inY = j >= 0 && j < nyt;
        float l[5], r[5], F[8];
        if (kind == 0) {
          if (!(zc && i >= 0 && inY)) continue;
          ld5(sm + G::P2 + 5 * NC, NC, e - 1, l);
          ld5(sm + G::P2, NC, e, r);
          face_flux<float, 0>(E, l, r, F);
          st8(sm + G::P1, NC, e, F);
        } else if (kind == 1) {
          if (!(zc && j >= 0 && inX)) continue;
          ld5(sm + G::P2 + 15 * NC, NC, e - W, l);
          ld5(sm + G::P2 + 10 * NC, NC, e, r);
          face_flux<float, 1>(E, l, r, F);
          st8(sm + G::P1 + 8 * NC, NC, e, F);
        } else {
          if (!(c >= 0 && inX && inY)) continue;
          ld5(sm + G::QZFP + pm * 5 * NC, NC, e, l);
          ld5(sm + G::QZFM, NC, e, r);
          face_flux<float, 2>(E, l, r, F);
          st8(sm + G::FFZ + pc * 8 * NC, NC, e, F);
        }
      }
      __syncthreads();

      // ------------------------------------------------ S7: update of plane c-1
      if (zc) {
        for (int t = tid; t < NCP; t += NT) {
          if (!active(t)) continue;
          const int i = col_i(t), j = col_j(t);
          if (!(i >= 0 && i < nxt && j >= 0 && j < nyt)) continue;
          float Fxm[8], Fxp[8], Fym[8], Fyp[8], Fzm[8], Fzp[8];
          ld8(sm + G::P1, NC, t, Fxm);
          ld8(sm + G::P1, NC, t + 1, Fxp);
          ld8(sm + G::P1 + 8 * NC, NC, t, Fym);
          ld8(sm + G::P1 + 8 * NC, NC, t + W, Fyp);
          ld8(sm + G::FFZ + pm * 8 * NC, NC, t, Fzm);
          ld8(sm + G::FFZ + pc * 8 * NC, NC, t, Fzp);
          const long long id = gcol(i, j) + (long long)(c - 1 + 4) * ps;
          update_cell_mixed(KK, sc, b, S, Gv, Sn, id, Fxm, Fxp, Fym, Fyp, Fzm, Fzp, dtmin, flags,
                            a.dtacc != nullptr);
          if (a.flux_keep) {
            double *fk = a.flux_keep + a.flux_off[w.box];
            const int nx = b.n[0], ny = b.n[1];
            const int gx = w.x0 + i, gy = w.y0 + j, p = c - 1;
            long long fx = (long long)(nx + 1) * ny * nz;
            long long ix = ((long long)p * ny + gy) * (nx + 1) + gx;
#pragma unroll
            for (int k = 0; k < 6; ++k) fk[k * fx + ix] = (double)Fxm[k];
            if (gx == nx - 1)
#pragma unroll
              for (int k = 0; k < 6; ++k) fk[k * fx + ix + 1] = (double)Fxp[k];
            fk += 6 * fx;
            long long fy = (long long)nx * (ny + 1) * nz;
            long long iy = ((long long)p * (ny + 1) + gy) * nx + gx;
#pragma unroll
            for (int k = 0; k < 6; ++k) fk[k * fy + iy] = (double)Fym[k];
            if (gy == ny - 1)
#pragma unroll
              for (int k = 0; k < 6; ++k) fk[k * fy + iy + nx] = (double)Fyp[k];
            fk += 6 * fy;
            long long fz = (long long)nx * ny * (nz + 1);
            long long iz = ((long long)p * ny + gy) * nx + gx;
#pragma unroll
            for (int k = 0; k < 6; ++k) fk[k * fz + iz] = (double)Fzm[k];
            if (p == nz - 1)
#pragma unroll
              for (int k = 0; k < 6; ++k) fk[k * fz + iz + (long long)nx * ny] = (double)Fzp[k];
          }
        }
      }
      // no barrier: the next plane's S0 writes only the primitive ring
    }
    __syncthreads();
  }

  if (a.dtacc) {
    for (int o = 16; o > 0; o >>= 1) {
      double v = __shfl_xor_sync(0xffffffffu, dtmin, o);
      if (v < dtmin) dtmin = v;
    }
    if ((tid & 31) == 0 && dtmin < __longlong_as_double(0x7ff0000000000000LL))
      nyx::atomic_min_pos(a.dtacc, dtmin);
  }
  if (flags) atomicOr(a.status, flags);
}

template <int TX, int TY, int MB>
int launch_two(const nyx::FusedArgs &a, int grid, cudaStream_t st) {
  using G = G2<TX, TY>;
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return (int)e;
  k_fused2<TX, TY, MB><<<grid, G::NT, G::SMEM, st>>>(a);
  return (int)cudaGetLastError();
}

template <int TX, int TY, int MB>
int max_grid_two() {
  using G = G2<TX, TY>;
  cudaError_t e = cudaFuncSetAttribute(k_fused2<TX, TY, MB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused2<TX, TY, MB>, G::NT, G::SMEM);
  if (per_sm < 1) return 0;
  return per_sm * nsm;
}

}  // namespace NYX_NS
