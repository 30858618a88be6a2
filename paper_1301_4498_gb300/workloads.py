"""Seeded synthetic inputs for the single-level comoving gas advance.

This module only *makes inputs*: box lists, domains and initial fields.  It
holds none of the advance's arithmetic, so both the CUDA path and the CPU
oracle can take their inputs from it.

Field recipe (the paper's Santa Barbara / cosmology initial conditions are
external data, so these stand in for them):

* code units: box length L = 1, mean density 1, specific internal energy
  e0 = 0.9 so that the mean sound speed sqrt(gamma (gamma-1) e0) = 1 for
  gamma = 5/3;
* G: unit-variance Gaussian random field with power spectrum P(k) ~ k^-2
  (k = 0 removed), drawn from numpy ``default_rng(seed)`` white noise and
  shaped with a real FFT;
* density: rho = exp(sigma G - sigma^2/2), divided by its sample mean
  (lognormal, mean 1);
* velocities: three more independent fields of the same spectrum, scaled so
  that rms |U| = 0.1 of the mean sound speed;
* gravity: a Gaussian potential phi of the same spectrum (own seed stream),
  g = minus the centred difference of phi (the cell-average rule of the
  paper's Sec. 3.4), scaled so that rms |g| = 0.1 c^2 / L;
* e uniform (temperature uniform), rho e = rho e0, rho E = rho e + rho U^2/2.

Every box array has shape (ncomp, nz+2ng, ny+2ng, nx+2ng), x fastest; ghost
cells are NaN on return, so a path that forgets to fill one shows it.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

NG = 4
BC_PERIODIC = 0
BC_OUTFLOW = 1
E0 = 0.9


@dataclass
class LevelSpec:
    """One AMR level: a union of boxes, each belonging to a domain.

    ``lo``/``hi`` are inclusive cell bounds in the domain's index space;
    ``dom_bc`` holds the boundary kind of the lo x,y,z and hi x,y,z faces.
    Boxes of one domain must not overlap.  The paper requires even cell
    counts per box (Sec. 4.1).
    """
    lo: np.ndarray
    hi: np.ndarray
    dom: np.ndarray
    dx: np.ndarray
    dom_lo: np.ndarray
    dom_hi: np.ndarray
    dom_bc: np.ndarray
    ng: int = NG
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nbox(self) -> int:
        return len(self.lo)

    def extent(self, b: int):
        """Valid cell counts (nx, ny, nz) of box b."""
        return tuple(int(x) for x in (self.hi[b] - self.lo[b] + 1))

    def shape(self, b: int, ncomp: int = 6):
        nx, ny, nz = self.extent(b)
        g = 2 * self.ng
        return (ncomp, nz + g, ny + g, nx + g)

    def valid_cells(self) -> int:
        return int(np.prod(self.hi - self.lo + 1, axis=1).sum())

    def subset(self, boxes) -> "LevelSpec":
        """Level made of some boxes only (their domains kept whole)."""
        boxes = np.asarray(boxes, dtype=np.int64)
        return LevelSpec(self.lo[boxes].copy(), self.hi[boxes].copy(), self.dom[boxes].copy(),
                         self.dx[boxes].copy(), self.dom_lo, self.dom_hi, self.dom_bc, self.ng,
                         self.name + "-subset", dict(self.meta))


def _mk(lo, hi, dom, dx, dom_lo, dom_hi, dom_bc, name, **meta) -> LevelSpec:
    return LevelSpec(np.asarray(lo, np.int32).reshape(-1, 3), np.asarray(hi, np.int32).reshape(-1, 3),
                     np.asarray(dom, np.int32).reshape(-1), np.asarray(dx, np.float64).reshape(-1, 3),
                     np.asarray(dom_lo, np.int32).reshape(-1, 3),
                     np.asarray(dom_hi, np.int32).reshape(-1, 3),
                     np.asarray(dom_bc, np.int32).reshape(-1, 6), NG, name, dict(meta))


def single_box_level(nx, ny, nz, dx, bc=(0, 0, 0, 0, 0, 0), name="box") -> LevelSpec:
    return _mk([0, 0, 0], [nx - 1, ny - 1, nz - 1], [0], [dx, dx, dx], [0, 0, 0],
               [nx - 1, ny - 1, nz - 1], list(bc), name)


def tiled_level(n, box, dx=None, name="tiled") -> LevelSpec:
    """A periodic n^3 domain cut into (n/box)^3 boxes of box^3 cells."""
    m = n // box
    assert m * box == n
    dx = 1.0 / n if dx is None else dx
    lo, hi = [], []
    for k in range(m):
        for j in range(m):
            for i in range(m):
                lo.append([i * box, j * box, k * box])
                hi.append([i * box + box - 1, j * box + box - 1, k * box + box - 1])
    nb = len(lo)
    return _mk(lo, hi, [0] * nb, [[dx] * 3] * nb, [0, 0, 0], [n - 1] * 3, [0] * 6, name)


def independent_boxes_level(extents, dx, name="independent") -> LevelSpec:
    """Each box its own periodic domain (extents: list of (nx, ny, nz))."""
    lo, hi, dlo, dhi = [], [], [], []
    for (nx, ny, nz) in extents:
        lo.append([0, 0, 0])
        hi.append([nx - 1, ny - 1, nz - 1])
        dlo.append([0, 0, 0])
        dhi.append([nx - 1, ny - 1, nz - 1])
    nb = len(lo)
    dxs = dx if np.ndim(dx) else [dx] * nb
    return _mk(lo, hi, list(range(nb)), [[d] * 3 for d in dxs], dlo, dhi, [[0] * 6] * nb, name)


def merge_levels(a: LevelSpec, b: LevelSpec, name="merged") -> LevelSpec:
    nd = len(a.dom_lo)
    return _mk(np.vstack([a.lo, b.lo]), np.vstack([a.hi, b.hi]),
               np.concatenate([a.dom, b.dom + nd]), np.vstack([a.dx, b.dx]),
               np.vstack([a.dom_lo, b.dom_lo]), np.vstack([a.dom_hi, b.dom_hi]),
               np.vstack([a.dom_bc, b.dom_bc]), name)


# ---------------------------------------------------------------------------
# random fields

def _fft_workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def gaussian_k2(shape_zyx, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance Gaussian field with P(k) ~ k^-2 on a periodic grid."""
    import scipy.fft as sfft
    nz, ny, nx = shape_zyx
    w = rng.standard_normal(shape_zyx)
    W = sfft.rfftn(w, workers=_fft_workers())
    del w
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    W *= 1.0 / np.sqrt(k2)
    W[0, 0, 0] = 0.0
    g = sfft.irfftn(W, s=shape_zyx, workers=_fft_workers())
    g -= g.mean()
    g /= g.std()
    return g


@dataclass
class Fields:
    """Valid-region fields of one periodic patch, shape (nz, ny, nx)."""
    rho: np.ndarray
    u: np.ndarray  # (3, nz, ny, nx)
    g: np.ndarray  # (3, nz, ny, nx)


def comoving_fields(shape_zyx, sigma, seed, dx) -> Fields:
    """The lognormal comoving field recipe above on one periodic patch."""
    rng = np.random.default_rng(seed)
    G = gaussian_k2(shape_zyx, rng)
    rho = np.exp(sigma * G - 0.5 * sigma * sigma)
    rho /= rho.mean()
    del G
    u = np.stack([gaussian_k2(shape_zyx, rng) for _ in range(3)])
    umag = np.sqrt((u * u).sum(axis=0).mean())
    u *= 0.1 / umag
    rng_phi = np.random.default_rng(seed + 7919)
    phi = gaussian_k2(shape_zyx, rng_phi)
    g = np.empty((3,) + tuple(shape_zyx))
    for d, ax in enumerate((2, 1, 0)):
        g[d] = -(np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)) / (2.0 * dx)
    gmag = np.sqrt((g * g).sum(axis=0).mean())
    g *= 0.1 / gmag
    return Fields(rho, u, g)


def conserved_from_primitive(rho, u, rhoe) -> np.ndarray:
    """(rho, m_x, m_y, m_z, rhoE, rhoe) from density, velocity, rho e."""
    m = rho[None] * u
    rhoE = rhoe + 0.5 * rho * (u * u).sum(axis=0)
    return np.concatenate([rho[None], m, rhoE[None], rhoe[None]])


def empty_box(lev: LevelSpec, b: int, ncomp: int) -> np.ndarray:
    return np.full(lev.shape(b, ncomp), np.nan)


def put_valid(arr: np.ndarray, valid: np.ndarray, ng: int = NG) -> None:
    arr[:, ng:arr.shape[1] - ng, ng:arr.shape[2] - ng, ng:arr.shape[3] - ng] = valid


def valid(arr: np.ndarray, ng: int = NG) -> np.ndarray:
    return arr[:, ng:arr.shape[1] - ng, ng:arr.shape[2] - ng, ng:arr.shape[3] - ng]


@dataclass
class Workload:
    """A level, its initial state and gravity (per box), the scale-factor
    schedule a_0..a_N and the run parameters."""
    name: str
    level: LevelSpec
    state: list
    grav: list | None
    a_sched: np.ndarray
    gamma: float
    cfl: float
    nsteps: int
    mixed: bool = False


def a_schedule(a0, aN, nsteps) -> np.ndarray:
    """Scale factor linear in step number from a0 to aN (reading)."""
    return a0 + (aN - a0) * np.arange(nsteps + 1) / nsteps


def _patch_state(lev, b, f: Fields):
    S = empty_box(lev, b, 6)
    put_valid(S, conserved_from_primitive(f.rho, f.u, f.rho * E0), lev.ng)
    G = empty_box(lev, b, 3)
    put_valid(G, f.g, lev.ng)
    return S, G


# ---------------------------------------------------------------------------
# the named workloads

def sod(n=128, ny=8, nz=8, axis=0, gamma=1.4, nsteps=20) -> Workload:
    """Sod shock tube along ``axis``: outflow along it, periodic across.
    Left (x < 0.5): rho = 1, p = 1; right: rho = 0.125, p = 0.1; at rest."""
    ext = [ny, nz]
    ext.insert(axis, n)
    bc = [0] * 6
    bc[axis] = BC_OUTFLOW
    bc[3 + axis] = BC_OUTFLOW
    lev = single_box_level(ext[0], ext[1], ext[2], 1.0 / n, bc, name=f"sod{n}")
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    rho1 = np.where(left, 1.0, 0.125)
    p1 = np.where(left, 1.0, 0.1)
    shp = (ext[2], ext[1], ext[0])
    bshape = [1, 1, 1]
    bshape[2 - axis] = n
    rho = np.broadcast_to(rho1.reshape(bshape), shp).copy()
    p = np.broadcast_to(p1.reshape(bshape), shp).copy()
    u = np.zeros((3,) + shp)
    S = empty_box(lev, 0, 6)
    put_valid(S, conserved_from_primitive(rho, u, p / (gamma - 1.0)))
    return Workload(f"sod {ext[0]}x{ext[1]}x{ext[2]}", lev, [S], None, np.ones(nsteps + 1), gamma,
                    0.5, nsteps)


def comoving_box(n=128, sigma=0.5, seed=1, nsteps=10, a0=1.0 / 51, aN=1.0 / 49,
                 mixed=False) -> Workload:
    """One periodic n^3 box of the lognormal comoving field."""
    dx = 1.0 / n
    lev = single_box_level(n, n, n, dx, name=f"comoving{n}")
    f = comoving_fields((n, n, n), sigma, seed, dx)
    S, G = _patch_state(lev, 0, f)
    return Workload(f"comoving {n}^3 sigma={sigma}", lev, [S], [G], a_schedule(a0, aN, nsteps),
                    5.0 / 3.0, 0.5, nsteps, mixed)


def uneven_boxes(nbox=512, seed=3, nsteps=10, sizes=(16, 24, 32, 48, 64), box_seed0=1000,
                 sigma=0.5, boxes=None) -> Workload:
    """``nbox`` independent periodic boxes with edges drawn uniformly from
    ``sizes`` per axis; box b filled with seed box_seed0 + b."""
    rng = np.random.default_rng(seed)
    ext = rng.choice(np.asarray(sizes), size=(nbox, 3))
    sel = range(nbox) if boxes is None else boxes
    ext_sel = [tuple(int(v) for v in ext[b]) for b in sel]
    dx = 1.0 / 128
    lev = independent_boxes_level(ext_sel, dx, name=f"uneven{nbox}")
    S, G = [], []
    for i, b in enumerate(sel):
        nx, ny, nz = ext_sel[i]
        f = comoving_fields((nz, ny, nx), sigma, box_seed0 + b, dx)
        s, g = _patch_state(lev, i, f)
        S.append(s)
        G.append(g)
    return Workload(f"{nbox} uneven boxes", lev, S, G, a_schedule(1.0 / 51, 1.0 / 49, nsteps),
                    5.0 / 3.0, 0.5, nsteps)


def tiled_box(n=64, box=32, sigma=0.5, seed=1, nsteps=2, a0=1.0 / 51, aN=1.0 / 49,
              mixed=False) -> Workload:
    """A periodic n^3 comoving field cut into box^3 boxes (neighbour fill)."""
    lev = tiled_level(n, box)
    f = comoving_fields((n, n, n), sigma, seed, 1.0 / n)
    S, G = [], []
    for b in range(lev.nbox):
        i0, j0, k0 = (int(v) for v in lev.lo[b])
        sl = (slice(k0, k0 + box), slice(j0, j0 + box), slice(i0, i0 + box))
        fb = Fields(f.rho[sl], f.u[(slice(None),) + sl], f.g[(slice(None),) + sl])
        s, g = _patch_state(lev, b, fb)
        S.append(s)
        G.append(g)
    return Workload(f"comoving {n}^3 as {lev.nbox} boxes of {box}^3", lev, S, G,
                    a_schedule(a0, aN, nsteps), 5.0 / 3.0, 0.5, nsteps, mixed)


def large_level(n=512, box=32, nfine=410, fine_n=64, sigma=1.0, seed=5, nsteps=100,
                fine_seed0=50000, fine_select=None, coarse_select=None,
                keep_fields=False) -> Workload:
    """A periodic n^3 level cut into (n/box)^3 boxes of box^3 plus ``nfine``
    independent periodic fine_n^3 boxes at half the cell width (a seeded 10%
    refined subset; no coarse-fine coupling).  a from 1/51 to 1/31.

    ``coarse_select`` / ``fine_select`` keep only some boxes (their fields are
    still cut from the same full-size draws)."""
    coarse = tiled_level(n, box, name="coarse")
    csel = range(coarse.nbox) if coarse_select is None else coarse_select
    f = comoving_fields((n, n, n), sigma, seed, 1.0 / n) if len(csel) else None
    fsel = range(nfine) if fine_select is None else fine_select
    S, G = [], []
    clev = coarse.subset(list(csel)) if coarse_select is not None else coarse
    for i, b in enumerate(csel):
        i0, j0, k0 = (int(v) for v in coarse.lo[b])
        sl = (slice(k0, k0 + box), slice(j0, j0 + box), slice(i0, i0 + box))
        fb = Fields(np.ascontiguousarray(f.rho[sl]), np.ascontiguousarray(f.u[(slice(None),) + sl]),
                    np.ascontiguousarray(f.g[(slice(None),) + sl]))
        s, g = _patch_state(clev, i, fb)
        S.append(s)
        G.append(g)
    coarse_fields = f if keep_fields else None
    del f
    fsel = list(fsel)
    fine = independent_boxes_level([(fine_n,) * 3] * len(fsel), 0.5 / n, name="fine")
    for i, b in enumerate(fsel):
        fb = comoving_fields((fine_n,) * 3, sigma, fine_seed0 + b, 0.5 / n)
        s, g = _patch_state(fine, i, fb)
        S.append(s)
        G.append(g)
    if not len(csel):
        lev = fine
    else:
        lev = merge_levels(clev, fine, name="large") if len(fsel) else clev
    w = Workload(f"{n}^3 level as {coarse.nbox} boxes of {box}^3 + {nfine} boxes of {fine_n}^3",
                 lev, S, G, a_schedule(1.0 / 51, 1.0 / 31, nsteps), 5.0 / 3.0, 0.5, nsteps, True)
    if keep_fields:
        w.level.meta["coarse_fields"] = coarse_fields
        w.level.meta["coarse_n"] = n
        w.level.meta["coarse_boxes"] = len(list(csel))
    return w


def ghosted_patch(fields: Fields, lo, hi, ng=NG):
    """State and gravity of the box [lo, hi] of a periodic patch with its
    ghost cells taken from the same patch (periodic wrap): the input a
    single box needs to be advanced one step on its own."""
    nz, ny, nx = fields.rho.shape
    idx = [np.arange(lo[d] - ng, hi[d] + ng + 1) % n for d, n in enumerate((nx, ny, nz))]
    sl = np.ix_(idx[2], idx[1], idx[0])
    rho = fields.rho[sl]
    u = np.stack([fields.u[c][sl] for c in range(3)])
    g = np.stack([fields.g[c][sl] for c in range(3)])
    return conserved_from_primitive(rho, u, rho * E0), g


def sound_wave(n, amp=1e-5, direction=(1, 0, 0), nz=8, gamma=5.0 / 3.0) -> Workload:
    """A right-moving linear acoustic wave of one wavelength across the
    periodic unit box (rho0 = 1, c0 = 1).  direction (1,0,0): n x 8 x 8 box;
    (1,1,0): n x n x nz box, wave along the diagonal with two wavelengths
    fitting the periodic box."""
    dirv = np.asarray(direction, float)
    if dirv[1] == 0:
        ext = (n, 8, 8)
    else:
        ext = (n, n, nz)
    dx = 1.0 / n
    lev = single_box_level(ext[0], ext[1], ext[2], dx, name="wave")
    p0 = 1.0 / gamma
    x = (np.arange(ext[0]) + 0.5) * dx
    y = (np.arange(ext[1]) + 0.5) * dx
    z = (np.arange(ext[2]) + 0.5) * dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    kvec = 2 * np.pi * dirv
    phase = kvec[0] * X + kvec[1] * Y
    khat = dirv / np.linalg.norm(dirv)
    # cell averages of sin over each cell (exact for the product of 1-D averages)
    fac = 1.0
    for kd in kvec[:2]:
        if kd != 0:
            fac *= np.sin(kd * dx / 2) / (kd * dx / 2)
    s = amp * np.sin(phase) * fac
    rho = 1.0 + s
    p = p0 + s  # c0^2 = 1
    un = s  # rho0 c0 = 1
    u = np.stack([khat[0] * un, khat[1] * un, khat[2] * un])
    S = empty_box(lev, 0, 6)
    put_valid(S, conserved_from_primitive(rho, u, p / (gamma - 1.0)))
    return Workload("sound wave", lev, [S], None, np.ones(2), gamma, 0.5, 1)


def uniform_level(state6, n=(16, 16, 16), dx=1.0 / 16, grav=None) -> Workload:
    """A periodic box holding one uniform conserved state (and gravity)."""
    lev = single_box_level(n[0], n[1], n[2], dx, name="uniform")
    S = empty_box(lev, 0, 6)
    put_valid(S, np.broadcast_to(np.asarray(state6, float)[:, None, None, None],
                                 (6, n[2], n[1], n[0])))
    G = None
    if grav is not None:
        g = empty_box(lev, 0, 3)
        put_valid(g, np.broadcast_to(np.asarray(grav, float)[:, None, None, None],
                                     (3, n[2], n[1], n[0])))
        G = [g]
    return Workload("uniform", lev, [S], G, np.ones(2), 5.0 / 3.0, 0.5, 1)


# ---------------------------------------------------------------------------
# two-level hierarchies (a fine level refining coarse regions by 2)

def refined_level(coarse: LevelSpec, regions, name="fine") -> LevelSpec:
    """The ratio-2 refinement of coarse regions.  Region (d, lo, hi), in
    coarse cells of domain d, becomes the fine box of fine cells
    2(lo - dom_lo) + dom_lo_f .. 2(hi - dom_lo) + 1 + dom_lo_f with half the
    cell width.  Fine domain k refines coarse domain k (dom_lo_f = 2 dom_lo,
    dom_hi_f = 2 dom_hi + 1) with the same boundary kinds."""
    dlo_f = 2 * coarse.dom_lo
    dhi_f = 2 * coarse.dom_hi + 1
    lo, hi, dom, dx = [], [], [], []
    for (d, rlo, rhi) in regions:
        rlo, rhi = np.asarray(rlo), np.asarray(rhi)
        lo.append(2 * (rlo - coarse.dom_lo[d]) + dlo_f[d])
        hi.append(2 * (rhi - coarse.dom_lo[d]) + 1 + dlo_f[d])
        dom.append(d)
        # cell width of the coarse box holding the region's first cell
        inside = np.all((coarse.lo <= rlo) & (rlo <= coarse.hi), axis=1) & (coarse.dom == d)
        dx.append(coarse.dx[int(np.argmax(inside))] / 2)
    return _mk(lo, hi, dom, dx, dlo_f, dhi_f, coarse.dom_bc, name)


def refine_boxes(coarse: LevelSpec, boxes, name="fine") -> LevelSpec:
    """The ratio-2 refinement of whole coarse boxes."""
    return refined_level(coarse, [(int(coarse.dom[b]), coarse.lo[b], coarse.hi[b]) for b in boxes],
                         name)


@dataclass
class AmrWorkload:
    """A coarse workload and a fine level refining part of it.  The fine
    initial data and gravity are not generated here: each path makes them by
    its own interpolation from the coarse level (Sec. 4.1: newly refined
    regions take interpolated coarse data)."""
    name: str
    coarse: Workload
    fine: LevelSpec
    refined: list


def amr_level(n=128, box=32, nfine=6, sigma=1.0, seed=5, select_seed=11, nsteps=10,
              a0=1.0 / 51, aN=1.0 / 49, refined=None) -> AmrWorkload:
    """A periodic n^3 comoving level cut into box^3 boxes, with ``nfine``
    seeded boxes refined by 2 (or the given coarse box indices)."""
    w = tiled_box(n=n, box=box, sigma=sigma, seed=seed, nsteps=nsteps, a0=a0, aN=aN)
    if refined is None:
        rng = np.random.default_rng(select_seed)
        refined = sorted(int(b) for b in rng.choice(w.level.nbox, size=nfine, replace=False))
    fine = refine_boxes(w.level, refined)
    w.name = f"{w.name}, {len(refined)} refined by 2"
    return AmrWorkload(w.name, w, fine, list(refined))


def amr_large(n=512, box=32, nfine=410, sigma=1.0, seed=5, select_seed=11, nsteps=100,
              coarse_only=False) -> AmrWorkload:
    """The large level's box structure with its refined 10% coupled: a
    periodic 512^3 level as 4096 boxes of 32^3, 410 seeded boxes refined by 2
    (64^3 fine boxes at half the cell width over them).  a from 1/51 to 1/31."""
    coarse = tiled_level(n, box, name="coarse")
    f = comoving_fields((n, n, n), sigma, seed, 1.0 / n)
    S, G = [], []
    for b in range(coarse.nbox):
        i0, j0, k0 = (int(v) for v in coarse.lo[b])
        sl = (slice(k0, k0 + box), slice(j0, j0 + box), slice(i0, i0 + box))
        fb = Fields(np.ascontiguousarray(f.rho[sl]), np.ascontiguousarray(f.u[(slice(None),) + sl]),
                    np.ascontiguousarray(f.g[(slice(None),) + sl]))
        s, g = _patch_state(coarse, b, fb)
        S.append(s)
        G.append(g)
    del f
    rng = np.random.default_rng(select_seed)
    refined = sorted(int(b) for b in rng.choice(coarse.nbox, size=nfine, replace=False))
    w = Workload(f"{n}^3 level as {coarse.nbox} boxes of {box}^3, {nfine} refined by 2",
                 coarse, S, G, a_schedule(1.0 / 51, 1.0 / 31, nsteps), 5.0 / 3.0, 0.5, nsteps, True)
    return AmrWorkload(w.name, w, refine_boxes(coarse, refined), refined)


def cell_factors(lev: LevelSpec, seed, amp) -> list:
    """Seeded per-cell factors 1 + amp N(0, 1) over the valid cells of every
    box (shape (nz, ny, nx) each).  Multiplying all six conserved components
    of a cell by its factor perturbs the density and keeps the velocity and
    the specific energies."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(lev.nbox):
        nx, ny, nz = lev.extent(b)
        out.append(1.0 + amp * rng.standard_normal((nz, ny, nx)))
    return out


def scale_valid(arrays, factors, ng: int = NG) -> list:
    """Copies of per-box arrays with every component of each valid cell
    multiplied by that cell's factor."""
    out = []
    for a, f in zip(arrays, factors):
        a = np.array(a, dtype=np.float64, copy=True)
        valid(a, ng)[...] *= f[None]
        out.append(a)
    return out


# ---------------------------------------------------------------------------
# dark-matter particles (seeded; positions in [0, n dx) per axis)

def dm_particles(n, dx, per_axis=None, seed=17, disp=0.3, vel_rms=0.05, mass_total=5.0):
    """Particles on a lattice of per_axis^3 points (default: one per cell)
    at the lattice cell centres, each displaced by a uniform random offset of
    up to disp lattice spacings per axis, with Gaussian velocities of rms
    vel_rms per component and equal masses summing to mass_total (times the
    domain volume).  Returns (x (3, np), u (3, np), m (np,))."""
    rng = np.random.default_rng(seed)
    n = np.asarray(n, dtype=np.int64)
    per = n if per_axis is None else np.asarray([per_axis] * 3, dtype=np.int64)
    L = n * dx
    sp = L / per
    grids = np.meshgrid(*(np.arange(int(per[d])) for d in range(3)), indexing="ij")
    base = np.stack([(grids[d].ravel() + 0.5) * sp[d] for d in range(3)])
    x = base + disp * sp[:, None] * rng.uniform(-1.0, 1.0, size=base.shape)
    x = np.mod(x, L[:, None])
    u = vel_rms * rng.standard_normal(size=x.shape)
    npart = x.shape[1]
    m = np.full(npart, mass_total * float(np.prod(L)) / npart)
    return np.ascontiguousarray(x), np.ascontiguousarray(u), m


def cosmo_level(n=512, box=32, sigma=1.0, seed=5, nsteps=100, part_seed=17, dm_mass=5.0,
                dm_vel_rms=0.1, a0=1.0 / 51, aN=1.0 / 31) -> Workload:
    """Gas on a periodic n^3 level cut into box^3 boxes (the comoving
    generator) plus one dark-matter particle per cell (dm_particles, total
    mass dm_mass times the mean gas mass), for the single-level algorithm
    with self-gravity.  The particles are in level.meta["dm"] = (x, u, m);
    the gravity field is left to the Poisson solve (grav = None)."""
    w = tiled_box(n=n, box=box, sigma=sigma, seed=seed, nsteps=nsteps, a0=a0, aN=aN)
    dx = 1.0 / n
    w.level.meta["dm"] = dm_particles((n, n, n), dx, seed=part_seed, vel_rms=dm_vel_rms,
                                      mass_total=dm_mass)
    w.grav = None
    w.name = f"{w.name} + {n}^3 dark-matter particles"
    w.mixed = True
    return w
