"""Thin ctypes binding of libnyxhydro.so (include/nyx_hydro.h).

Argument marshalling only: every step of the advance runs in the CUDA
library.  PyTorch provides device memory and the stream.  There is no CPU
fallback: if the library is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnyxhydro.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "nyx_hydro.h")

NYX_OK = 0
NYX_EINVAL = -1
NYX_ECUDA = -2
NYX_ENEGATIVE = -3
NYX_ENONFINITE = -4
NYX_ETIMEOUT = -5
NYX_ENOMEM = -6
NYX_FP64 = 0
NYX_MIXED = 1
NYX_PPM = 0
NYX_PLM = 1
NYX_RS_TWO_SHOCK = 0
NYX_RS_LINEAR = 1
NYX_PERSISTENT = 0
NYX_PER_BOX = 1
NOALLOC_MAX_BOXES = 4096  # NYX_NOALLOC_MAX_BOXES of include/nyx_hydro.h
NYX_AMR_GHOSTS = 0
NYX_AMR_ALL = 1

_lib = None


class NyxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nyx error {code}: {msg}")
        self.code = code


class NyxBox(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3), ("domain", C.c_int),
                ("dx", C.c_double * 3)]


class NyxDomain(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3), ("bc", C.c_int * 6)]


class NyxLevelDesc(C.Structure):
    _fields_ = [("nboxes", C.c_int), ("ng", C.c_int), ("boxes", C.POINTER(NyxBox)),
                ("ndomains", C.c_int), ("domains", C.POINTER(NyxDomain))]


class NyxParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("small_dens", C.c_double),
                ("small_pres", C.c_double), ("eta_de", C.c_double),
                ("riemann_max_iter", C.c_int), ("riemann_tol", C.c_double),
                ("precision", C.c_int), ("grav_corrector", C.c_int), ("batching", C.c_int),
                ("autotune", C.c_int), ("keep_fluxes", C.c_int), ("coarse_fine", C.c_int),
                ("grav_energy", C.c_int), ("reconstruction", C.c_int),
                ("riemann_solver", C.c_int), ("flattening", C.c_int),
                ("z_chunks", C.c_int)]


class NyxPoissonParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_cycles", C.c_int), ("pre", C.c_int), ("post", C.c_int),
                ("coarse_sweeps", C.c_int), ("min_size", C.c_int), ("four_pi_G", C.c_double),
                ("precision", C.c_int)]


class NyxLevel(C.Structure):
    _fields_ = [("state", C.c_void_p * 2), ("grav", C.c_void_p), ("cur", C.c_int)]


class NyxCounters(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("timed_fills", C.c_longlong),
                ("timed_advances", C.c_longlong), ("fill_ms", C.c_double),
                ("advance_ms", C.c_double), ("timed_flattens", C.c_longlong),
                ("flatten_ms", C.c_double)]


def header_functions():
    """Names of the functions include/nyx_hydro.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nyx_\w+)\s*\(", txt, flags=re.M)))


def load_library(path: str | None = None):
    """Load libnyxhydro.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise NyxError(NYX_ECUDA, f"{p} is not built; run __graft_entry__.build() first")
    L = C.CDLL(p)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    L.nyx_hydro_default_params.argtypes = [C.POINTER(NyxParams)]
    L.nyx_hydro_default_params.restype = None
    L.nyx_last_error.restype = C.c_char_p
    L.nyx_hydro_plan.argtypes = [C.POINTER(NyxLevelDesc), C.POINTER(NyxParams), vp, C.POINTER(vp)]
    L.nyx_hydro_layout.argtypes = [vp, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    L.nyx_hydro_fill.argtypes = [vp, vp, C.c_int]
    L.nyx_hydro_estdt.argtypes = [vp, C.POINTER(NyxLevel), vp, vp]
    L.nyx_hydro_advance.argtypes = [vp, C.POINTER(NyxLevel), vp, vp, vp, vp, vp]
    L.nyx_hydro_run.argtypes = [vp, C.POINTER(NyxLevel), vp, vp, C.c_int, C.c_int, C.c_int]
    L.nyx_hydro_predict.argtypes = [vp, C.POINTER(NyxLevel), vp, vp, vp, vp]
    L.nyx_hydro_correct.argtypes = [vp, C.POINTER(NyxLevel), vp, vp, vp, vp, vp, vp]
    L.nyx_hydro_fluxes.argtypes = [vp, C.POINTER(NyxLevel), C.c_int, C.c_int, vp]
    L.nyx_hydro_step_host.argtypes = [vp, C.POINTER(NyxLevel), vp, vp, C.c_double, C.c_double,
                                      dp]
    L.nyx_hydro_step_host_valid.argtypes = [vp, C.POINTER(NyxLevel), vp, vp, C.c_double,
                                            C.c_double, dp]
    L.nyx_hydro_status.argtypes = [vp, ip]
    L.nyx_plan_destroy.argtypes = [vp]
    L.nyx_hydro_tile_shape.argtypes = [C.c_int, ip, ip]
    L.nyx_task_items.argtypes = [C.c_int, ip, C.c_int, C.c_int, C.c_int, C.c_int, ip, C.c_int, ip]
    L.nyx_hydro_set_tile_shape.argtypes = [vp, C.c_int]
    L.nyx_hydro_tune_info.argtypes = [vp, ip, ip, ip]
    L.nyx_hydro_tune_info.restype = C.c_int
    L.nyx_hydro_get_tile_shape.argtypes = [vp, ip]
    L.nyx_hydro_profile.argtypes = [vp, C.c_int]
    L.nyx_hydro_counters_read.argtypes = [vp, C.c_int, C.POINTER(NyxCounters)]
    L.nyx_hydro_estdt_noalloc.argtypes = [C.POINTER(NyxLevelDesc), C.POINTER(NyxParams), vp, vp,
                                          vp, vp]
    L.nyx_alu_peak.argtypes = [C.c_int, C.c_double, vp, dp]
    L.nyx_alu_peak.restype = C.c_int
    L.nyx_poisson_default_params.argtypes = [C.POINTER(NyxPoissonParams)]
    L.nyx_poisson_default_params.restype = None
    L.nyx_poisson_create.argtypes = [vp, C.POINTER(NyxPoissonParams), C.POINTER(vp)]
    L.nyx_poisson_solve.argtypes = [vp, vp, vp, C.c_double, vp, vp, C.c_int, ip, dp]
    L.nyx_pm_deposit.argtypes = [vp, vp, vp, C.c_longlong, vp]
    L.nyx_pm_kick_drift.argtypes = [vp, vp, vp, C.c_longlong, vp, C.c_double, C.c_double,
                                    C.c_double]
    L.nyx_pm_kick.argtypes = [vp, vp, vp, C.c_longlong, vp, C.c_double, C.c_double, C.c_double]
    L.nyx_pm_estdt.argtypes = [vp, vp, vp, C.c_longlong, vp, C.c_double, C.c_double, vp]
    L.nyx_pm_kick_estdt.argtypes = [vp, vp, vp, C.c_longlong, vp, C.c_double, C.c_double,
                                    C.c_double, C.c_double, vp]
    for name in ("nyx_pm_deposit", "nyx_pm_kick_drift", "nyx_pm_kick", "nyx_pm_estdt",
                 "nyx_pm_kick_estdt"):
        getattr(L, name).restype = C.c_int
    L.nyx_poisson_phi.argtypes = [vp, vp]
    L.nyx_poisson_destroy.argtypes = [vp]
    for name in ("nyx_poisson_create", "nyx_poisson_solve", "nyx_poisson_phi",
                 "nyx_poisson_destroy"):
        getattr(L, name).restype = C.c_int
    L.nyx_amr_create.argtypes = [vp, vp, C.POINTER(vp)]
    L.nyx_amr_interp.argtypes = [vp, vp, vp, C.c_int, C.c_int]
    L.nyx_amr_reflux.argtypes = [vp, vp]
    L.nyx_amr_average_down.argtypes = [vp, vp, vp, C.c_int]
    L.nyx_amr_estdt.argtypes = [vp, C.POINTER(NyxLevel), C.POINTER(NyxLevel), vp, vp]
    L.nyx_amr_step.argtypes = [vp, C.POINTER(NyxLevel), C.POINTER(NyxLevel), vp, vp, vp, vp]
    L.nyx_amr_run.argtypes = [vp, C.POINTER(NyxLevel), C.POINTER(NyxLevel), vp, vp, C.c_int,
                              C.c_int, C.c_int]
    L.nyx_amr_destroy.argtypes = [vp]
    for name in ("nyx_amr_create", "nyx_amr_interp", "nyx_amr_reflux", "nyx_amr_average_down",
                 "nyx_amr_estdt", "nyx_amr_step", "nyx_amr_run", "nyx_amr_destroy"):
        getattr(L, name).restype = C.c_int
    for name in ("nyx_hydro_plan", "nyx_hydro_layout", "nyx_hydro_fill", "nyx_hydro_estdt",
                 "nyx_hydro_advance", "nyx_hydro_run", "nyx_hydro_fluxes", "nyx_hydro_step_host",
                 "nyx_hydro_step_host_valid",
                 "nyx_hydro_status", "nyx_plan_destroy", "nyx_hydro_tile_shape",
                 "nyx_hydro_set_tile_shape", "nyx_hydro_get_tile_shape", "nyx_hydro_profile",
                 "nyx_hydro_counters_read", "nyx_hydro_estdt_noalloc", "nyx_hydro_predict",
                 "nyx_hydro_correct"):
        getattr(L, name).restype = C.c_int
    if path is None:
        _lib = L
    return L


def _check(rc):
    if rc != NYX_OK:
        raise NyxError(rc, load_library().nyx_last_error().decode())
    return rc


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def level_desc(spec):
    """C level descriptor from a LevelSpec-like object (see workloads.LevelSpec)."""
    nb = len(spec.lo)
    boxes = (NyxBox * nb)()
    for b in range(nb):
        for a in range(3):
            boxes[b].lo[a] = int(spec.lo[b][a])
            boxes[b].hi[a] = int(spec.hi[b][a])
            boxes[b].dx[a] = float(spec.dx[b][a])
        boxes[b].domain = int(spec.dom[b])
    nd = len(spec.dom_lo)
    doms = (NyxDomain * nd)()
    for d in range(nd):
        for a in range(3):
            doms[d].lo[a] = int(spec.dom_lo[d][a])
            doms[d].hi[a] = int(spec.dom_hi[d][a])
        for a in range(6):
            doms[d].bc[a] = int(spec.dom_bc[d][a])
    desc = NyxLevelDesc(nb, int(spec.ng), boxes, nd, doms)
    return desc, (boxes, doms)


def make_params(**kw) -> NyxParams:
    p = NyxParams()
    load_library().nyx_hydro_default_params(C.byref(p))
    prec = kw.pop("precision", None)
    if prec is not None:
        p.precision = {"fp64": NYX_FP64, "mixed": NYX_MIXED}.get(prec, prec)
    rec = kw.pop("reconstruction", None)
    if rec is not None:
        p.reconstruction = {"ppm": NYX_PPM, "plm": NYX_PLM}.get(rec, rec)
    rs = kw.pop("riemann_solver", None)
    if rs is not None:
        p.riemann_solver = {"two_shock": NYX_RS_TWO_SHOCK, "linear": NYX_RS_LINEAR}.get(rs, rs)
    if "flattening" in kw:
        p.flattening = int(bool(kw.pop("flattening")))
    bat = kw.pop("batching", None)
    if bat is not None:
        p.batching = {"persistent": NYX_PERSISTENT, "per_box": NYX_PER_BOX}.get(bat, bat)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Level:
    """Two state fields, gravity and the current-version index of one level
    (caller-owned torch tensors)."""

    def __init__(self, state0, state1, grav=None, cur=0):
        self.state = [state0, state1]
        self.grav = grav
        self.cur = cur
        self._c = NyxLevel()

    def c(self):
        self._c.state[0] = self.state[0].data_ptr()
        self._c.state[1] = self.state[1].data_ptr()
        self._c.grav = None if self.grav is None else self.grav.data_ptr()
        self._c.cur = self.cur
        return self._c

    def sync_from_c(self):
        self.cur = self._c.cur

    @property
    def current(self):
        return self.state[self.cur]


class _Ordered:
    """Order library work after the caller's torch stream and torch work
    after the library's stream (the plan runs on its own non-default stream,
    which CUDA-graph capture requires)."""

    def __init__(self, plan):
        self.plan = plan

    def __enter__(self):
        import torch
        self.plan.torch_stream.wait_stream(torch.cuda.current_stream())
        return self

    def __exit__(self, *exc):
        import torch
        torch.cuda.current_stream().wait_stream(self.plan.torch_stream)
        return False


class Plan:
    """A plan of libnyxhydro.so over one level (see nyx_hydro_plan)."""

    def __init__(self, spec, stream=None, **params):
        import torch
        self.lib = load_library()
        self.spec = spec
        self.params = make_params(**params)
        desc, self._keep = level_desc(spec)
        if stream is None:
            stream = torch.cuda.Stream()
        self.torch_stream = stream
        self.stream = stream.cuda_stream
        h = C.c_void_p()
        _check(self.lib.nyx_hydro_plan(C.byref(desc), C.byref(self.params),
                                       C.c_void_p(self.stream), C.byref(h)))
        self.h = h
        self.nbox = len(spec.lo)

    def ordered(self):
        return _Ordered(self)

    # ---------------------------------------------------------- layout
    def layout(self, ncomp):
        off = (C.c_size_t * (self.nbox + 1))()
        st = (C.c_size_t * self.nbox)()
        _check(self.lib.nyx_hydro_layout(self.h, ncomp, off, st))
        return np.frombuffer(off, dtype=np.uint64).astype(np.int64), \
            np.frombuffer(st, dtype=np.uint64).astype(np.int64)

    def pack_host(self, arrays, ncomp, out=None):
        """Pack per-box arrays (ncomp, Nz, Ny, Nx) into one flat host array."""
        off, st = self.layout(ncomp)
        if out is None:
            out = np.zeros(int(off[-1]), dtype=np.float64)
        for b, a in enumerate(arrays):
            vol = a.shape[1] * a.shape[2] * a.shape[3]
            blk = out[off[b]:off[b + 1]].reshape(ncomp, st[b])
            blk[:, :vol] = a.reshape(ncomp, vol)
        return out

    def unpack_host(self, flat, ncomp):
        off, st = self.layout(ncomp)
        res = []
        for b in range(self.nbox):
            shp = self.spec.shape(b, ncomp)
            vol = shp[1] * shp[2] * shp[3]
            blk = flat[off[b]:off[b + 1]].reshape(ncomp, st[b])
            res.append(blk[:, :vol].reshape(shp).copy())
        return res

    def to_device(self, arrays, ncomp):
        import torch
        return torch.from_numpy(self.pack_host(arrays, ncomp)).cuda()

    def from_device(self, t, ncomp):
        return self.unpack_host(t.detach().cpu().numpy(), ncomp)

    def empty_field(self, ncomp):
        import torch
        off, _ = self.layout(ncomp)
        return torch.zeros(int(off[-1]), dtype=torch.float64, device="cuda")

    # ---------------------------------------------------------- calls
    def fill(self, field, ncomp):
        with self.ordered():
            _check(self.lib.nyx_hydro_fill(self.h, _ptr(field), ncomp))

    def estdt(self, level, a_dev, dt_dev):
        with self.ordered():
            _check(self.lib.nyx_hydro_estdt(self.h, C.byref(level.c()), _ptr(a_dev),
                                            _ptr(dt_dev)))

    def advance(self, level, a_old, a_new, dt, grav=None, dt_next=None):
        cl = level.c()
        with self.ordered():
            _check(self.lib.nyx_hydro_advance(self.h, C.byref(cl), _ptr(a_old), _ptr(a_new),
                                              _ptr(dt), _ptr(grav), _ptr(dt_next)))
        level.sync_from_c()

    def predict(self, level, a_old, a_new, dt, grav_old=None):
        """Step 2 alone: state[1-cur] = predictor (cur unchanged)."""
        cl = level.c()
        with self.ordered():
            _check(self.lib.nyx_hydro_predict(self.h, C.byref(cl), _ptr(a_old), _ptr(a_new),
                                              _ptr(dt), _ptr(grav_old)))
        level.sync_from_c()

    def correct(self, level, a_old, a_new, dt, grav_old=None, grav_new=None, dt_next=None):
        """Step 6 alone on the predictor in state[1-cur] (g^n, g^{n+1}); cur flips."""
        cl = level.c()
        with self.ordered():
            _check(self.lib.nyx_hydro_correct(self.h, C.byref(cl), _ptr(a_old), _ptr(a_new),
                                              _ptr(dt), _ptr(grav_old), _ptr(grav_new),
                                              _ptr(dt_next)))
        level.sync_from_c()

    def run(self, level, a_dev, dt_dev, nsteps, compute_dt0=True, use_graph=True):
        cl = level.c()
        with self.ordered():
            _check(self.lib.nyx_hydro_run(self.h, C.byref(cl), _ptr(a_dev), _ptr(dt_dev), nsteps,
                                          1 if compute_dt0 else 0, 1 if use_graph else 0))
        level.sync_from_c()

    def fluxes(self, level, box, direction):
        import torch
        n = list(self.spec.extent(box))
        n[direction] += 1
        out = torch.empty((6, n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
        with self.ordered():
            _check(self.lib.nyx_hydro_fluxes(self.h, C.byref(level.c()), box, direction,
                                             _ptr(out)))
        return out

    def set_tile_shape(self, shape):
        _check(self.lib.nyx_hydro_set_tile_shape(self.h, shape))

    def tile_shape(self):
        s = C.c_int()
        _check(self.lib.nyx_hydro_get_tile_shape(self.h, C.byref(s)))
        tx, ty = C.c_int(), C.c_int()
        _check(self.lib.nyx_hydro_tile_shape(s.value, C.byref(tx), C.byref(ty)))
        return s.value, (tx.value, ty.value)

    def tune_info(self):
        """(box-size classes, trial launches of the last tuning, fused launches
        per advance) of the plan's autotuner (nyx_hydro_tune_info)."""
        c, t, n = C.c_int(), C.c_int(), C.c_int()
        _check(self.lib.nyx_hydro_tune_info(self.h, C.byref(c), C.byref(t), C.byref(n)))
        return c.value, t.value, n.value

    def profile(self, enable=True):
        _check(self.lib.nyx_hydro_profile(self.h, 1 if enable else 0))

    def counters(self, reset=True):
        c = NyxCounters()
        _check(self.lib.nyx_hydro_counters_read(self.h, 1 if reset else 0, C.byref(c)))
        return dict(launches=c.launches, timed_fills=c.timed_fills,
                    timed_advances=c.timed_advances, fill_ms=c.fill_ms, advance_ms=c.advance_ms,
                    timed_flattens=c.timed_flattens, flatten_ms=c.flatten_ms)

    def step_host(self, level, host_in, host_out, a_old, a_new, dt=0.0):
        """End-to-end step through host buffers (torch CPU tensors, ideally
        pinned).  Returns the next step's CFL dt."""
        d = C.c_double(dt)
        cl = level.c()
        import torch
        self.torch_stream.wait_stream(torch.cuda.current_stream())
        _check(self.lib.nyx_hydro_step_host(self.h, C.byref(cl), C.c_void_p(host_in.data_ptr()),
                                            C.c_void_p(host_out.data_ptr()), a_old, a_new,
                                            C.byref(d)))
        level.sync_from_c()
        return d.value

    def step_host_valid(self, level, host_in, host_out, a_old, a_new, dt=0.0):
        """End-to-end step with only the valid cells on the host (pack_valid
        layout; torch CPU tensors, ideally pinned).  Returns the next step's
        CFL dt."""
        d = C.c_double(dt)
        cl = level.c()
        import torch
        self.torch_stream.wait_stream(torch.cuda.current_stream())
        _check(self.lib.nyx_hydro_step_host_valid(self.h, C.byref(cl),
                                                  C.c_void_p(host_in.data_ptr()),
                                                  C.c_void_p(host_out.data_ptr()), a_old, a_new,
                                                  C.byref(d)))
        level.sync_from_c()
        return d.value

    def pack_valid(self, arrays):
        """Valid cells of per-box state arrays (6, Nz, Ny, Nx) packed box by
        box, component-major, x fastest (the step_host_valid layout)."""
        g = self.spec.ng
        return np.concatenate([np.ascontiguousarray(a[:, g:-g, g:-g, g:-g]).ravel()
                               for a in arrays])

    def unpack_valid(self, flat):
        """Inverse of pack_valid: per-box arrays of the valid cells (6, nz, ny, nx)."""
        res, o = [], 0
        for b in range(self.nbox):
            n = self.spec.extent(b)
            v = 6 * n[0] * n[1] * n[2]
            res.append(np.asarray(flat[o:o + v]).reshape(6, n[2], n[1], n[0]).copy())
            o += v
        return res

    def status(self):
        f = C.c_int()
        rc = self.lib.nyx_hydro_status(self.h, C.byref(f))
        return rc, f.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.nyx_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tile_shape_of(shape):
    """Columns (tx, ty) of a tile shape of the fused kernel."""
    tx, ty = C.c_int(), C.c_int()
    _check(load_library().nyx_hydro_tile_shape(shape, C.byref(tx), C.byref(ty)))
    return tx.value, ty.value


def task_items(extents, tx, ty, slots, chunk=True):
    """The fused kernel's work list for boxes of interior extents [(nx, ny,
    nz), ...], tiles tx x ty on `slots` resident CTAs: an (items, 7) int
    array of (box, x0, y0, nx, ny, z0, nz) in queue order.  Host only."""
    lib = load_library()
    n = (C.c_int * max(1, 3 * len(extents)))(*[int(v) for e in extents for v in e])
    count = C.c_int()
    _check(lib.nyx_task_items(len(extents), n, tx, ty, slots, int(bool(chunk)), None, 0,
                              C.byref(count)))
    out = (C.c_int * max(1, 7 * count.value))()
    _check(lib.nyx_task_items(len(extents), n, tx, ty, slots, int(bool(chunk)), out, count.value,
                              C.byref(count)))
    return np.array(out[:7 * count.value], dtype=np.int64).reshape(count.value, 7)


def estdt_noalloc(spec, state, a_dev, dt_dev, stream=None, **params):
    """nyx_hydro_estdt_noalloc: the CFL step of a level field without a plan
    and without any device allocation (scratch in a fixed device array)."""
    import torch
    desc, keep = level_desc(spec)
    p = make_params(**params)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load_library().nyx_hydro_estdt_noalloc(C.byref(desc), C.byref(p), _ptr(state),
                                                   _ptr(a_dev), _ptr(dt_dev), C.c_void_p(stream)))


def alu_peak(pipe: str, seconds: float = 0.25, stream=None) -> float:
    """nyx_alu_peak: measured fused multiply-add rate of the current device
    (lane operations per second) on the FP32 (``"fp32"``) or FP64
    (``"fp64"``) pipe."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = C.c_double()
    _check(load_library().nyx_alu_peak({"fp32": 0, "fp64": 1}[pipe], seconds, C.c_void_p(stream),
                                       C.byref(out)))
    return out.value


class Poisson:
    """Self-gravity of a plan's level (nyx_poisson_*): periodic multigrid
    Poisson solve on the dense grid of its domain, g = -grad phi."""

    def __init__(self, plan: "Plan", **params):
        self.lib = load_library()
        self.plan = plan
        p = NyxPoissonParams()
        self.lib.nyx_poisson_default_params(C.byref(p))
        prec = params.pop("precision", None)
        if prec is not None:
            p.precision = {"fp64": NYX_FP64, "mixed": NYX_MIXED}.get(prec, prec)
        for k, v in params.items():
            setattr(p, k, v)
        self.params = p
        h = C.c_void_p()
        _check(self.lib.nyx_poisson_create(plan.h, C.byref(p), C.byref(h)))
        self.h = h
        n = plan.spec.dom_hi[0] - plan.spec.dom_lo[0] + 1
        self.shape = (int(n[2]), int(n[1]), int(n[0]))

    def solve(self, state, a, grav_out=None, warm_start=True, rho_dm=None, g_dense=None):
        """Returns (cycles, relative residual)."""
        cyc = C.c_int()
        res = C.c_double()
        with self.plan.ordered():
            _check(self.lib.nyx_poisson_solve(self.h, _ptr(state), _ptr(rho_dm), float(a),
                                              _ptr(grav_out), _ptr(g_dense),
                                              1 if warm_start else 0, C.byref(cyc),
                                              C.byref(res)))
        return cyc.value, res.value

    def dense(self, ncomp=1):
        import torch
        return torch.zeros((ncomp,) + self.shape, dtype=torch.float64, device="cuda")

    # dark matter: x, u (3, np), m (np,) device tensors; g a (3, nz, ny, nx) dense tensor
    def pm_deposit(self, x, m, rho_dm):
        with self.plan.ordered():
            _check(self.lib.nyx_pm_deposit(self.h, _ptr(x), _ptr(m), m.numel(), _ptr(rho_dm)))

    def pm_kick_drift(self, x, u, g, a_old, a_half, dt):
        with self.plan.ordered():
            _check(self.lib.nyx_pm_kick_drift(self.h, _ptr(x), _ptr(u), x.shape[1], _ptr(g),
                                              float(a_old), float(a_half), float(dt)))

    def pm_kick(self, x, u, g, a_half, a_new, dt):
        with self.plan.ordered():
            _check(self.lib.nyx_pm_kick(self.h, _ptr(x), _ptr(u), x.shape[1], _ptr(g),
                                        float(a_half), float(a_new), float(dt)))

    def pm_kick_estdt(self, x, u, g, a_half, a_new, dt, dt_dev, cfl_dm=0.5):
        """Kick (Step 5), then the particle dt of the kicked particles at a_new."""
        with self.plan.ordered():
            _check(self.lib.nyx_pm_kick_estdt(self.h, _ptr(x), _ptr(u), x.shape[1], _ptr(g),
                                              float(a_half), float(a_new), float(dt),
                                              float(cfl_dm), _ptr(dt_dev)))

    def pm_estdt(self, x, u, g, a, dt_dev, cfl_dm=0.5):
        with self.plan.ordered():
            _check(self.lib.nyx_pm_estdt(self.h, _ptr(x), _ptr(u), x.shape[1], _ptr(g), float(a),
                                         float(cfl_dm), _ptr(dt_dev)))

    def phi(self):
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        with self.plan.ordered():
            _check(self.lib.nyx_poisson_phi(self.h, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.nyx_poisson_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Amr:
    """A fine plan coupled to the coarse plan it refines by 2 (nyx_amr_*):
    fine ghost cells from the coarse level, reflux, average down, the
    shared CFL step and the two-level step.  Both plans must share a stream
    (pass the coarse plan's ``torch_stream`` to the fine Plan), keep fluxes,
    and the fine plan must be made with coarse_fine=1."""

    def __init__(self, coarse: "Plan", fine: "Plan"):
        self.lib = load_library()
        self.coarse, self.fine = coarse, fine
        h = C.c_void_p()
        _check(self.lib.nyx_amr_create(coarse.h, fine.h, C.byref(h)))
        self.h = h

    def ordered(self):
        return _Ordered(self.coarse)

    def interp(self, coarse_field, fine_field, ncomp, region="ghosts"):
        r = NYX_AMR_ALL if region == "all" else NYX_AMR_GHOSTS
        with self.ordered():
            _check(self.lib.nyx_amr_interp(self.h, _ptr(coarse_field), _ptr(fine_field), ncomp, r))

    def reflux(self, coarse_new):
        with self.ordered():
            _check(self.lib.nyx_amr_reflux(self.h, _ptr(coarse_new)))

    def average_down(self, fine_field, coarse_field, ncomp):
        with self.ordered():
            _check(self.lib.nyx_amr_average_down(self.h, _ptr(fine_field), _ptr(coarse_field),
                                                 ncomp))

    def estdt(self, coarse_level, fine_level, a_dev, dt_dev):
        with self.ordered():
            _check(self.lib.nyx_amr_estdt(self.h, C.byref(coarse_level.c()),
                                          C.byref(fine_level.c()), _ptr(a_dev), _ptr(dt_dev)))

    def step(self, coarse_level, fine_level, a_old, a_new, dt, dt_next=None):
        cc, cf = coarse_level.c(), fine_level.c()
        with self.ordered():
            _check(self.lib.nyx_amr_step(self.h, C.byref(cc), C.byref(cf), _ptr(a_old),
                                         _ptr(a_new), _ptr(dt), _ptr(dt_next)))
        coarse_level.sync_from_c()
        fine_level.sync_from_c()

    def run(self, coarse_level, fine_level, a_dev, dt_dev, nsteps, compute_dt0=True,
            use_graph=True):
        cc, cf = coarse_level.c(), fine_level.c()
        with self.ordered():
            _check(self.lib.nyx_amr_run(self.h, C.byref(cc), C.byref(cf), _ptr(a_dev),
                                        _ptr(dt_dev), nsteps, 1 if compute_dt0 else 0,
                                        1 if use_graph else 0))
        coarse_level.sync_from_c()
        fine_level.sync_from_c()

    def close(self):
        if getattr(self, "h", None):
            self.lib.nyx_amr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_level(plan, states, grav=None):
    """Device level from per-box host arrays (ghost cells need not be valid)."""
    s0 = plan.to_device(states, 6)
    s1 = plan.empty_field(6)
    g = None
    if grav is not None:
        g = plan.to_device(grav, 3)
        plan.fill(g, 3)
    return Level(s0, s1, g)
