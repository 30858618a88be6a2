"""Plain FP64 CPU oracle for the single-level comoving gas advance.

TEST INFRASTRUCTURE, not product code.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It wraps ``nyx_oracle.c`` (built with gcc,
``-O2 -ffp-contract=off``, OpenMP) through ctypes and shares no code with
the CUDA path.

What it computes follows the Nyx paper (Almgren et al. 2013): Sec. 2.2
(comoving Euler + dual-energy equations, gamma-law EOS), Sec. 3.2 (unsplit
PPM Godunov with characteristic tracing, reference states, two-shock Riemann
solver, dual-energy switch, gravity predictor-corrector), Sec. 3.5 (CFL time
step), Sec. 3.6 Steps 2 and 6.

Arrays are per box, shape ``(ncomp, nz+2ng, ny+2ng, nx+2ng)`` float64, C
order (x fastest).  A level is any object with numpy attributes ``lo``,
``hi`` (nbox x 3, inclusive), ``dom`` (nbox), ``dx`` (nbox x 3), ``dom_lo``,
``dom_hi`` (ndom x 3), ``dom_bc`` (ndom x 6: lo x,y,z then hi x,y,z; 0
periodic, 1 outflow) and ``ng``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no FMA contraction)."""
    src = os.path.join(_HERE, "nyx_oracle.c")
    hdr = os.path.join(_HERE, "nyx_oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("small_dens", C.c_double),
                ("small_pres", C.c_double), ("eta_de", C.c_double),
                ("riemann_max_iter", C.c_int), ("riemann_tol", C.c_double),
                ("grav_corrector", C.c_int), ("dual_energy_sync", C.c_int),
                ("grav_energy", C.c_int), ("reconstruction", C.c_int),
                ("riemann_solver", C.c_int), ("flattening", C.c_int)]


class _Level(C.Structure):
    _fields_ = [("nbox", C.c_int), ("ng", C.c_int), ("lo", C.POINTER(C.c_int)),
                ("hi", C.POINTER(C.c_int)), ("dom", C.POINTER(C.c_int)),
                ("dx", C.POINTER(C.c_double)), ("ndom", C.c_int),
                ("dom_lo", C.POINTER(C.c_int)), ("dom_hi", C.POINTER(C.c_int)),
                ("dom_bc", C.POINTER(C.c_int))]


class _PoissonParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_cycles", C.c_int), ("pre", C.c_int), ("post", C.c_int),
                ("coarse_sweeps", C.c_int), ("min_size", C.c_int), ("four_pi_G", C.c_double)]


class _PoissonStats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("resid", C.c_double), ("rho_mean", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("floor_rho", C.c_longlong), ("floor_e", C.c_longlong),
                ("use_e", C.c_longlong), ("bad", C.c_longlong)]


@dataclass
class OracleParams:
    """Run-time parameters of the scheme (Sec. 3.2, 3.5, 3.6)."""
    gamma: float = 5.0 / 3.0
    cfl: float = 0.5
    small_dens: float = 1e-10
    small_pres: float = 1e-12
    eta_de: float = 1e-4
    riemann_max_iter: int = 12
    riemann_tol: float = 1e-10
    grav_corrector: int = 1
    dual_energy_sync: int = 1
    grav_energy: int = 0       # Sec. 3.2: 0 rho U . g in the energy; 1 the kinetic-energy change
    reconstruction: int = 0    # Sec. 3.2: 0 PPM, 1 PLM
    riemann_solver: int = 0    # Sec. 3.2: 0 two-shock (iterative), 1 linearised
    flattening: int = 0        # 1: Colella-Woodward shock flattening of the profiles

    def _c(self) -> _Params:
        return _Params(self.gamma, self.cfl, self.small_dens, self.small_pres, self.eta_de,
                       self.riemann_max_iter, self.riemann_tol, self.grav_corrector,
                       self.dual_energy_sync, self.grav_energy, self.reconstruction,
                       self.riemann_solver, self.flattening)


def load(path: str):
    """Load an oracle library file and declare its entry points."""
    L = C.CDLL(path)
    if True:
        dp = C.POINTER(C.c_double)
        L.orc_fill_ghosts.argtypes = [C.POINTER(_Level), C.c_int, C.POINTER(dp)]
        L.orc_fill_ghosts.restype = C.c_int
        L.orc_advance.argtypes = [C.POINTER(_Level), C.POINTER(_Params), C.POINTER(dp),
                                  C.POINTER(dp), C.POINTER(dp), C.c_double, C.c_double,
                                  C.c_double, C.c_int, C.POINTER(dp), C.POINTER(_Stats)]
        L.orc_advance.restype = C.c_int
        L.orc_estdt.argtypes = [C.POINTER(_Level), C.POINTER(_Params), C.POINTER(dp), C.c_double]
        L.orc_estdt.restype = C.c_double
        L.orc_ppm_line.argtypes = [C.c_int, dp, dp, dp, dp]
        L.orc_ppm_integrals.argtypes = [C.c_double] * 4 + [dp, dp]
        L.orc_riemann.argtypes = [C.POINTER(_Params), dp, dp, dp, dp, dp]
        L.orc_riemann_state.argtypes = [C.POINTER(_Params), dp, dp, dp]
        L.orc_riemann_counts.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.c_int]
        L.orc_riemann_counts.restype = None
        L.orc_trace_line.argtypes = [C.POINTER(_Params), C.c_int, dp, dp, dp, C.c_double,
                                     C.c_double, C.c_double, C.c_int, dp, dp, dp, dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = None
        L.orc_flatten_line.argtypes = [C.POINTER(_Params), C.c_int, dp, dp, dp]
        L.orc_flatten_line.restype = None
        L.orc_flatten_field.argtypes = [C.POINTER(_Level), C.POINTER(_Params), C.POINTER(dp),
                                        C.POINTER(dp)]
        L.orc_flatten_field.restype = C.c_int
        L.orc_correct.argtypes = [C.POINTER(_Level), C.POINTER(_Params), C.POINTER(dp),
                                  C.POINTER(dp), C.POINTER(dp), C.POINTER(dp), C.c_double,
                                  C.c_double, C.c_double, C.POINTER(_Stats)]
        L.orc_correct.restype = C.c_int
        L.orc_poisson_solve.argtypes = [C.POINTER(_Level), C.POINTER(_PoissonParams),
                                        C.POINTER(dp), dp, C.c_double, dp, C.POINTER(dp), dp,
                                        C.POINTER(_PoissonStats)]
        L.orc_poisson_solve.restype = C.c_int
        ip3 = C.POINTER(C.c_int)
        L.orc_pm_deposit.argtypes = [ip3, C.c_double, dp, dp, C.c_longlong, dp]
        L.orc_pm_deposit.restype = None
        L.orc_pm_interp.argtypes = [ip3, C.c_double, dp, dp, C.c_longlong, dp]
        L.orc_pm_interp.restype = None
        L.orc_pm_kick_drift.argtypes = [ip3, C.c_double, dp, dp, dp, C.c_longlong, C.c_double,
                                        C.c_double, C.c_double]
        L.orc_pm_kick_drift.restype = None
        L.orc_pm_kick.argtypes = [ip3, C.c_double, dp, dp, dp, C.c_longlong, C.c_double,
                                  C.c_double, C.c_double]
        L.orc_pm_kick.restype = None
        L.orc_pm_estdt.argtypes = [ip3, C.c_double, dp, dp, dp, C.c_longlong, C.c_double,
                                   C.c_double]
        L.orc_pm_estdt.restype = C.c_double
        L.orc_amr_check.argtypes = [C.POINTER(_Level), C.POINTER(_Level)]
        L.orc_amr_check.restype = C.c_int
        L.orc_amr_interp.argtypes = [C.POINTER(_Level), C.c_int, C.POINTER(dp), C.POINTER(_Level),
                                     C.POINTER(dp), C.c_int]
        L.orc_amr_interp.restype = C.c_int
        L.orc_amr_reflux.argtypes = [C.POINTER(_Level), C.POINTER(dp), C.POINTER(dp),
                                     C.POINTER(_Level), C.POINTER(dp), C.c_double, C.c_double,
                                     C.c_double]
        L.orc_amr_reflux.restype = C.c_int
        L.orc_amr_average_down.argtypes = [C.POINTER(_Level), C.c_int, C.POINTER(dp),
                                           C.POINTER(_Level), C.POINTER(dp)]
        L.orc_amr_average_down.restype = C.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of
    nyx_oracle.c (the mutation tests use it to plant mistakes)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptrs(arrs):
    arr = (C.POINTER(C.c_double) * len(arrs))()
    for i, a in enumerate(arrs):
        arr[i] = _dp(a)
    return arr


def _level(lev):
    keep = {}
    for name in ("lo", "hi", "dom", "dom_lo", "dom_hi", "dom_bc"):
        keep[name] = np.ascontiguousarray(getattr(lev, name), dtype=np.int32)
    keep["dx"] = np.ascontiguousarray(lev.dx, dtype=np.float64)
    ip = lambda n: keep[n].ctypes.data_as(C.POINTER(C.c_int))
    cl = _Level(len(keep["lo"]), int(lev.ng), ip("lo"), ip("hi"), ip("dom"),
                keep["dx"].ctypes.data_as(C.POINTER(C.c_double)), len(keep["dom_lo"]),
                ip("dom_lo"), ip("dom_hi"), ip("dom_bc"))
    return cl, keep


def fill_ghosts(lev, arrays) -> None:
    """Fill ghost cells of every box array in place (periodic / outflow / neighbour)."""
    cl, keep = _level(lev)
    ncomp = arrays[0].shape[0]
    rc = lib().orc_fill_ghosts(C.byref(cl), ncomp, _ptrs(arrays))
    if rc:
        raise ValueError("oracle ghost fill: a ghost cell maps to no box of its domain")


def advance(lev, params: OracleParams, states, grav=None, *, a_old=1.0, a_new=1.0, dt,
            fill_ghosts=True, want_flux=False):
    """One single-level advance (Steps 2 and 6).  Returns (new_states, stats, fluxes).

    ``states`` (and ``grav``) are copied; ghost cells of the copies are filled
    here unless ``fill_ghosts`` is False.  Fluxes (if asked) are per box a
    list of three arrays of shape (6, nz', ny', nx') with n' = n + 1 along the
    face direction: the raw final Godunov fluxes.
    """
    cl, keep = _level(lev)
    sin = [np.array(s, dtype=np.float64, order="C", copy=True) for s in states]
    sout = [s.copy() for s in sin]
    g = None if grav is None else [np.array(x, dtype=np.float64, order="C", copy=True) for x in grav]
    flux = None
    fptr = None
    if want_flux:
        flux = []
        flat = []
        for b in range(len(sin)):
            n = (lev.hi[b] - lev.lo[b] + 1).astype(int)
            per = []
            for d in range(3):
                e = [int(n[0]), int(n[1]), int(n[2])]
                e[d] += 1
                arr = np.zeros((6, e[2], e[1], e[0]))
                per.append(arr)
                flat.append(arr)
            flux.append(per)
        fptr = _ptrs(flat)
    st = _Stats()
    p = params._c()
    rc = lib().orc_advance(C.byref(cl), C.byref(p), _ptrs(sin), _ptrs(sout),
                           None if g is None else _ptrs(g), a_old, a_new, dt,
                           1 if fill_ghosts else 0, fptr, C.byref(st))
    stats = dict(floor_e=st.floor_e, use_e=st.use_e, bad=st.bad, rc=rc)
    if rc == -1:
        raise ValueError("oracle advance: invalid level or ghost fill failure")
    return sout, stats, flux


def predict(lev, params: OracleParams, states, grav=None, *, a_old, a_new, dt, fill_ghosts=True):
    """Step 2 alone: the advance without the gravity corrector and without
    the dual-energy sync (the predictor U^{n+1,*})."""
    import dataclasses
    p = dataclasses.replace(params, grav_corrector=0, dual_energy_sync=0)
    out, st, _ = advance(lev, p, states, grav, a_old=a_old, a_new=a_new, dt=dt,
                         fill_ghosts=fill_ghosts)
    return out, st


def correct(lev, params: OracleParams, old, pred, g_old=None, g_new=None, *, a_old, a_new, dt):
    """Step 6 alone (Sec. 3.6): gravity corrector with g^n and g^{n+1}, then
    the dual-energy sync (if params.dual_energy_sync), applied to a copy of
    the predictor.  Returns (new_states, stats)."""
    cl, keep = _level(lev)
    o = [np.ascontiguousarray(a, dtype=np.float64) for a in old]
    out = [np.array(a, dtype=np.float64, order="C", copy=True) for a in pred]
    go = None if g_old is None else [np.ascontiguousarray(a, dtype=np.float64) for a in g_old]
    gn = None if g_new is None else [np.ascontiguousarray(a, dtype=np.float64) for a in g_new]
    st = _Stats()
    p = params._c()
    rc = lib().orc_correct(C.byref(cl), C.byref(p), _ptrs(o), _ptrs(out),
                           None if go is None else _ptrs(go), None if gn is None else _ptrs(gn),
                           a_old, a_new, dt, C.byref(st))
    return out, dict(floor_e=st.floor_e, use_e=st.use_e, bad=st.bad, rc=rc)


def estdt(lev, params: OracleParams, states, a: float) -> float:
    """CFL time step (Sec. 3.5) over the valid cells of every box."""
    cl, keep = _level(lev)
    sin = [np.ascontiguousarray(s, dtype=np.float64) for s in states]
    p = params._c()
    return float(lib().orc_estdt(C.byref(cl), C.byref(p), _ptrs(sin), a))


def run(lev, params: OracleParams, states, grav=None, a_sched=None, nsteps=1):
    """Advance ``nsteps`` steps; dt of each step is the CFL step of its input
    state at a = a_sched[s] (a_sched defaults to a = 1).  Returns
    (states, dts, stats_list)."""
    if a_sched is None:
        a_sched = np.ones(nsteps + 1)
    cur = [np.array(s, dtype=np.float64, copy=True) for s in states]
    dts, stats = [], []
    for s in range(nsteps):
        dt = estdt(lev, params, cur, float(a_sched[s]))
        cur, st, _ = advance(lev, params, cur, grav, a_old=float(a_sched[s]),
                             a_new=float(a_sched[s + 1]), dt=dt)
        dts.append(dt)
        stats.append(st)
    return cur, dts, stats


def riemann_counts(reset: bool = True):
    """(two-shock solves, Newton iterations) since the last reset."""
    c, n = C.c_longlong(), C.c_longlong()
    lib().orc_riemann_counts(C.byref(c), C.byref(n), 1 if reset else 0)
    return c.value, n.value


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's loops (n <= 0: all host processors)."""
    lib().orc_set_threads(int(n))


def flatten_line(pr, u, params: OracleParams = None):
    """Shock-flattening coefficients along a line of pressures ``pr`` and
    velocities ``u`` along it: cells 3..n-4 (1 at the others)."""
    params = params or OracleParams()
    pr = np.ascontiguousarray(pr, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(len(pr))
    p = params._c()
    lib().orc_flatten_line(C.byref(p), len(pr), _dp(pr), _dp(u), _dp(out))
    return out


def flatten_field(lev, params: OracleParams, states):
    """Shock-flattening coefficient of every cell of every box (copies of
    ``states`` with their ghost cells filled): a list of (nz+2g, ny+2g,
    nx+2g) arrays, 1 outside [-1, n] in each direction."""
    S = [np.array(s, dtype=np.float64, copy=True) for s in states]
    fill_ghosts(lev, S)
    out = [np.zeros(s.shape[1:]) for s in S]
    cl, keep = _level(lev)
    p = params._c()
    lib().orc_flatten_field(C.byref(cl), C.byref(p), _ptrs(S), _ptrs(out))
    return out


def ppm_line(s: np.ndarray):
    """PPM edge values and curvature (sL, sR, s6) for cells 2..n-3 of a line."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = len(s)
    sL, sR, s6 = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_ppm_line(n, _dp(s), _dp(sL), _dp(sR), _dp(s6))
    return sL, sR, s6


def ppm_integrals(sL, sR, s6, sigma):
    ip, im = C.c_double(), C.c_double()
    lib().orc_ppm_integrals(sL, sR, s6, sigma, C.byref(ip), C.byref(im))
    return ip.value, im.value


def riemann(params: OracleParams, qL, qR):
    """Two-shock solve of one face problem; states (rho, u_n, u_t1, u_t2, p).
    Returns (flux8, pstar, ustar) with flux8 = (F_rho, F_mn, F_mt1, F_mt2,
    F_rhoE, F_rhoe, u_g, p_g)."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    out = np.zeros(8)
    ps, us = np.zeros(1), np.zeros(1)
    p = params._c()
    lib().orc_riemann(C.byref(p), _dp(qL), _dp(qR), _dp(out), _dp(ps), _dp(us))
    return out, float(ps[0]), float(us[0])


def riemann_state(params: OracleParams, qL, qR):
    """The Godunov state (rho, u_n, u_t1, u_t2, p) sampled at x/t = 0 by the
    two-shock solve (Sec. 3.2), from which ``riemann`` forms its fluxes."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    g = np.zeros(5)
    p = params._c()
    lib().orc_riemann_state(C.byref(p), _dp(qL), _dp(qR), _dp(g))
    return g


def trace_line(params: OracleParams, q5, g=None, *, dtp, dx, adot=0.0, direction=0, fl=None):
    """Trace a line of primitives (5 x n, rho,u_x,u_y,u_z,p) along
    ``direction``.  Returns (qm, qp, beta_m, beta_p) for cells 2..n-3: the
    low- and high-face edge states and the wave amplitudes (beta_-, beta_0,
    beta_+) of each side.  ``fl`` (n values, default 1) is each cell's
    shock-flattening coefficient."""
    q5 = np.ascontiguousarray(q5, dtype=np.float64)
    n = q5.shape[1]
    gl = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    fla = None if fl is None else np.ascontiguousarray(np.broadcast_to(fl, (n,)), dtype=np.float64)
    qm, qp = np.zeros((5, n)), np.zeros((5, n))
    bm, bp = np.zeros((3, n)), np.zeros((3, n))
    p = params._c()
    lib().orc_trace_line(C.byref(p), n, _dp(q5), None if gl is None else _dp(gl),
                         None if fla is None else _dp(fla), dtp, dx, adot,
                         direction, _dp(qm), _dp(qp), _dp(bm), _dp(bp))
    return qm, qp, bm, bp


# ---------------------------------------------------------------------------
# Coarse-fine coupling, refinement ratio 2, no subcycling (Sec. 4.1-4.3).
# A fine level refines the coarse level's domain k as its own domain k
# (lo_f = 2 lo_c, hi_f = 2 hi_c + 1, periodic); fine boxes start and end on
# coarse cell boundaries.

def amr_check(coarse, fine) -> bool:
    """True if ``fine`` refines ``coarse`` as the coupling functions require."""
    cc, kc = _level(coarse)
    cf, kf = _level(fine)
    return lib().orc_amr_check(C.byref(cc), C.byref(cf)) == 0


def amr_interp(coarse, cfield, fine, ffield, region: str = "ghosts"):
    """Conservative limited linear interpolation (Sec. 4.1) of the coarse
    field (ghosts filled) into a copy of the fine field.  region "all": every
    cell of every fine box; "ghosts": the fine ghost cells, a ghost cell in
    the valid region of a fine box taking that cell's value.  Returns the
    new fine arrays."""
    cc, kc = _level(coarse)
    cf, kf = _level(fine)
    src = [np.ascontiguousarray(a, dtype=np.float64) for a in cfield]
    out = [np.array(a, dtype=np.float64, order="C", copy=True) for a in ffield]
    rc = lib().orc_amr_interp(C.byref(cc), src[0].shape[0], _ptrs(src), C.byref(cf), _ptrs(out),
                              0 if region == "all" else 1)
    if rc:
        raise ValueError("oracle interpolation: not a ratio-2 hierarchy or a cell maps to no box")
    return out


def amr_reflux(coarse, cstate, cflux, fine, fflux, *, a_old, a_new, dt):
    """Reflux (Sec. 4.3, Steps 2 and 8) of a copy of the coarse state.
    ``cflux`` / ``fflux`` are the per-box flux lists returned by advance()."""
    cc, kc = _level(coarse)
    cf, kf = _level(fine)
    out = [np.array(a, dtype=np.float64, order="C", copy=True) for a in cstate]
    cfl = [np.ascontiguousarray(a) for per in cflux for a in per]
    ffl = [np.ascontiguousarray(a) for per in fflux for a in per]
    rc = lib().orc_amr_reflux(C.byref(cc), _ptrs(out), _ptrs(cfl), C.byref(cf), _ptrs(ffl),
                              a_old, a_new, dt)
    if rc:
        raise ValueError("oracle reflux: not a ratio-2 hierarchy")
    return out


def amr_average_down(coarse, cstate, fine, fstate):
    """Average down (Sec. 4.3, Step 8): a copy of the coarse field whose
    cells under the fine level hold the mean of their 8 fine cells."""
    cc, kc = _level(coarse)
    cf, kf = _level(fine)
    out = [np.array(a, dtype=np.float64, order="C", copy=True) for a in cstate]
    src = [np.ascontiguousarray(a, dtype=np.float64) for a in fstate]
    rc = lib().orc_amr_average_down(C.byref(cc), out[0].shape[0], _ptrs(out), C.byref(cf),
                                    _ptrs(src))
    if rc:
        raise ValueError("oracle average down: not a ratio-2 hierarchy")
    return out


def amr_estdt(coarse, fine, params: OracleParams, cstate, fstate, a: float) -> float:
    """Shared time step of both levels (no subcycling, Sec. 4.2-4.3)."""
    return min(estdt(coarse, params, cstate, a), estdt(fine, params, fstate, a))


def amr_step(coarse, fine, params: OracleParams, cstate, fstate, cgrav=None, fgrav=None, *,
             a_old, a_new, dt, reflux=True, average_down=True):
    """One two-level advance with no subcycling (Sec. 4.3 Advance(0) with
    l_a = l_finest): coarse ghost fill; fine ghost fill (fine neighbours,
    else interpolation from the coarse level); both levels advanced by dt
    (Steps 2 and 6); reflux of the coarse cells next to the fine level and
    average down (Step 8).  Gravity arrays must have their ghosts filled.
    Returns (coarse_new, fine_new, stats_coarse, stats_fine)."""
    cs = [np.array(a, dtype=np.float64, order="C", copy=True) for a in cstate]
    fill_ghosts(coarse, cs)
    fs = amr_interp(coarse, cs, fine, fstate, "ghosts")
    cn, stc, cfx = advance(coarse, params, cs, cgrav, a_old=a_old, a_new=a_new, dt=dt,
                           fill_ghosts=False, want_flux=True)
    fn, stf, ffx = advance(fine, params, fs, fgrav, a_old=a_old, a_new=a_new, dt=dt,
                           fill_ghosts=False, want_flux=True)
    if reflux:
        cn = amr_reflux(coarse, cn, cfx, fine, ffx, a_old=a_old, a_new=a_new, dt=dt)
    if average_down:
        cn = amr_average_down(coarse, cn, fine, fn)
    return cn, fn, stc, stf


# ---------------------------------------------------------------------------
# Self-gravity (Sec. 3.4): periodic 7-point Poisson equation by multigrid.

@dataclass
class PoissonParams:
    tol: float = 1e-12
    max_cycles: int = 50
    pre: int = 2
    post: int = 2
    coarse_sweeps: int = 40
    min_size: int = 2
    four_pi_G: float = 1.0

    def _c(self):
        return _PoissonParams(self.tol, self.max_cycles, self.pre, self.post, self.coarse_sweeps,
                              self.min_size, self.four_pi_G)


def poisson_solve(lev, params: PoissonParams, states, a: float, phi=None, rho_dm=None,
                  want_dense_g=False):
    """Solve L phi = four_pi_G / a (rho_b + rho_dm - mean) on the dense
    periodic grid of the level's single domain by V-cycles (red-black
    Gauss-Seidel), from the initial guess phi (dense, (nz, ny, nx); zero if
    None).  rho_dm: dense dark-matter density or None.  Returns (phi, grav,
    stats) -- grav per box (3 components, valid cells filled, ghosts zero),
    g = -grad phi by centred differences -- plus the dense g (3, nz, ny, nx)
    when want_dense_g."""
    cl, keep = _level(lev)
    n = (lev.dom_hi[0] - lev.dom_lo[0] + 1).astype(int)
    ph = np.zeros((n[2], n[1], n[0])) if phi is None else np.array(phi, dtype=np.float64,
                                                                     order="C", copy=True)
    sin = [np.ascontiguousarray(s, dtype=np.float64) for s in states]
    grav = [np.zeros(lev.shape(b, 3)) for b in range(lev.nbox)]
    rd = None if rho_dm is None else np.ascontiguousarray(rho_dm, dtype=np.float64)
    gd = np.zeros((3, n[2], n[1], n[0])) if want_dense_g else None
    st = _PoissonStats()
    p = params._c()
    rc = lib().orc_poisson_solve(C.byref(cl), C.byref(p), _ptrs(sin),
                                 None if rd is None else _dp(rd), a, _dp(ph), _ptrs(grav),
                                 None if gd is None else _dp(gd), C.byref(st))
    if rc == -1:
        raise ValueError("oracle Poisson: the level must tile one periodic domain with equal cells")
    out = (ph, grav, dict(cycles=st.cycles, resid=st.resid, rho_mean=st.rho_mean, rc=rc))
    return out + (gd,) if want_dense_g else out


# ---------------------------------------------------------------------------
# Dark matter (Sec. 3.3-3.6): particles on a dense periodic grid of n cells of
# width dx per axis (positions in [0, n dx)); x, u of shape (3, np), m (np,).

def _n3(n):
    return (C.c_int * 3)(int(n[0]), int(n[1]), int(n[2]))


def pm_deposit(n, dx, x, m):
    """Cloud-in-cell density (nz, ny, nx) of the particles (Sec. 3.4)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    rho = np.zeros((n[2], n[1], n[0]))
    lib().orc_pm_deposit(_n3(n), dx, _dp(x), _dp(m), m.shape[0], _dp(rho))
    return rho


def pm_interp(n, dx, g, x):
    """g (3, nz, ny, nx) at the particles by the cloud-in-cell weights."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros_like(x)
    lib().orc_pm_interp(_n3(n), dx, _dp(g), _dp(x), x.shape[1], _dp(out))
    return out


def pm_kick_drift(n, dx, g, x, u, *, a_old, a_half, dt):
    """Step 3 on copies: returns (x^{n+1}, u^{n+1/2})."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    lib().orc_pm_kick_drift(_n3(n), dx, _dp(g), _dp(x), _dp(u), x.shape[1], a_old, a_half, dt)
    return x, u


def pm_kick(n, dx, g, x, u, *, a_half, a_new, dt):
    """Step 5 on a copy: returns u^{n+1}."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    lib().orc_pm_kick(_n3(n), dx, _dp(g), _dp(x), _dp(u), x.shape[1], a_half, a_new, dt)
    return u


def pm_estdt(n, dx, g, x, u, a, cfl_dm=0.5):
    """Particle time step of Sec. 3.5."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return float(lib().orc_pm_estdt(_n3(n), dx, _dp(g), _dp(x), _dp(u), x.shape[1], a, cfl_dm))
