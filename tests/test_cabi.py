"""The C-ABI library loads, exports every function include/nyx_hydro.h
declares, and rejects invalid levels and parameters on the host (no GPU
needed: validation runs before any CUDA call)."""
import ctypes as C
import os

import pytest

from paper_1301_4498_gb300 import build as B
from paper_1301_4498_gb300 import hydro as H
from paper_1301_4498_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(H.LIB_PATH):
        B.build()
    return H.load_library()


def test_exports_every_declared_symbol(lib):
    names = H.header_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params(lib):
    p = H.make_params()
    assert p.gamma == pytest.approx(5.0 / 3.0) and p.cfl == 0.5 and p.eta_de == 1e-4
    assert p.riemann_max_iter == 12 and p.precision == H.NYX_FP64
    assert p.batching == H.NYX_PERSISTENT


def _plan_rc(lib, spec, **kw):
    desc, keep = H.level_desc(spec)
    p = H.make_params(**kw)
    h = C.c_void_p()
    rc = lib.nyx_hydro_plan(C.byref(desc), C.byref(p), None, C.byref(h))
    return rc, lib.nyx_last_error().decode(), h


@pytest.mark.parametrize("case", ["odd", "ng", "overlap", "gap", "outside", "domain", "dx",
                                  "bc"])
def test_invalid_levels_rejected(lib, case):
    spec = W.tiled_level(32, 16)
    if case == "odd":
        spec.hi[0][0] = spec.lo[0][0] + 14  # 15 cells
    elif case == "ng":
        spec.ng = 3
    elif case == "overlap":
        spec.lo[1][0] -= 2  # box 1 now overlaps box 0
    elif case == "gap":
        spec = W.tiled_level(32, 16).subset([0, 1, 2, 3, 4, 5, 6])  # one box missing
    elif case == "outside":
        spec.hi[7][2] += 2
    elif case == "domain":
        spec.dom[3] = 5
    elif case == "dx":
        spec.dx[2][1] = 0.0
    elif case == "bc":
        spec.dom_bc[0][0] = 7
    rc, msg, h = _plan_rc(lib, spec)
    assert rc == H.NYX_EINVAL, (rc, msg)
    assert msg
    assert not h.value


@pytest.mark.parametrize("field,value", [("gamma", 1.0), ("cfl", 0.0), ("small_dens", 0.0),
                                         ("riemann_max_iter", 0), ("precision", 7),
                                         ("batching", 3)])
def test_invalid_params_rejected(lib, field, value):
    rc, msg, h = _plan_rc(lib, W.single_box_level(16, 16, 16, 1 / 16), **{field: value})
    assert rc == H.NYX_EINVAL and msg


def test_per_box_form_is_fp64_only(lib):
    rc, msg, _ = _plan_rc(lib, W.single_box_level(16, 16, 16, 1 / 16), precision="mixed",
                          batching="per_box")
    assert rc == H.NYX_EINVAL and "FP64" in msg


def test_null_arguments_rejected(lib):
    assert lib.nyx_hydro_plan(None, None, None, None) == H.NYX_EINVAL
    assert lib.nyx_hydro_status(None, None) == H.NYX_EINVAL
    assert lib.nyx_plan_destroy(None) == H.NYX_EINVAL
    assert lib.nyx_hydro_fill(None, None, 6) == H.NYX_EINVAL
