"""The C-ABI library loads, exports every function include/nyx_hydro.h
declares, and rejects invalid levels and parameters on the host (no GPU
needed: validation runs before any CUDA call)."""
import ctypes as C
import os

import numpy as np
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
                                  "bc", "empty"])
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
    elif case == "empty":
        spec = W.tiled_level(32, 16).subset([])  # a level with no boxes
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


# ------------------------------------------------------------ work lists
def _cost(it):
    """The scheduler's duration model: columns x (planes + 3)."""
    return ((it[:, 3] + 2) * (it[:, 4] + 2) * (it[:, 6] + 3)).astype(float)


def _queue_finish(it, slots):
    import heapq
    q = [0.0] * slots
    end = 0.0
    for c in _cost(it):
        t = heapq.heappop(q) + c
        heapq.heappush(q, t)
        end = max(end, t)
    return end


LEVELS = {"one128": [(128, 128, 128)], "one256": [(256, 256, 256)],
          "mix": [(32, 32, 32)] * 8 + [(64, 64, 64)] * 2,
          "ragged": [(40, 24, 50), (17, 9, 33), (5, 3, 1)]}


@pytest.mark.parametrize("level", sorted(LEVELS))
@pytest.mark.parametrize("tile", [(16, 8), (8, 8), (32, 4)])
@pytest.mark.parametrize("slots", [7, 152, 304])
@pytest.mark.parametrize("chunk", [False, True])
def test_task_items_tile_every_cell_once(lib, level, tile, slots, chunk):
    ext = LEVELS[level]
    it = H.task_items(ext, tile[0], tile[1], slots, chunk)
    seen = [np.zeros((n[2], n[1], n[0]), np.int32) for n in ext]
    for b, x0, y0, nx, ny, z0, nz in it:
        assert 1 <= nx <= tile[0] and 1 <= ny <= tile[1] and nz >= 1
        assert x0 % tile[0] == 0 and y0 % tile[1] == 0
        seen[b][z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] += 1
    assert all(np.all(s == 1) for s in seen)
    c = _cost(it)
    assert np.all(np.diff(c) <= 0)                  # queue order: largest first
    if not chunk:
        assert np.all(it[:, 5] == 0) and np.all(it[:, 6] == [ext[b][2] for b in it[:, 0]])


def test_task_items_even_out_a_single_box(lib):
    """128^3 in 16 x 8 tiles: 128 columns for 152 CTAs leave 24 idle with
    whole columns; the chunked list finishes within 6 % of the even share
    and 10 % before whole columns, in the duration model checked here."""
    ext = [(128, 128, 128)]
    whole = H.task_items(ext, 16, 8, 152, False)
    cut = H.task_items(ext, 16, 8, 152, True)
    lb = _cost(whole).sum() / 152
    assert len(whole) == 128 and _queue_finish(whole, 152) == pytest.approx(131 * 180)
    assert len(cut) > 152
    assert _queue_finish(cut, 152) <= 1.06 * lb
    assert _queue_finish(cut, 152) <= 0.9 * _queue_finish(whole, 152)


def test_task_items_keep_columns_of_a_many_box_level(lib):
    """A level with many more tiles than CTAs keeps whole columns."""
    ext = [(32, 32, 32)] * 64 + [(64, 64, 64)] * 6
    assert np.array_equal(H.task_items(ext, 16, 8, 152, True),
                          H.task_items(ext, 16, 8, 152, False))


@pytest.mark.parametrize("bad", [dict(ext=[(4, 4, 0)]), dict(slots=0), dict(tx=0)])
def test_task_items_reject_bad_arguments(lib, bad):
    kw = dict(ext=[(8, 8, 8)], tx=16, ty=8, slots=152)
    kw.update(bad)
    with pytest.raises(H.NyxError):
        H.task_items(kw["ext"], kw["tx"], kw["ty"], kw["slots"])


def test_task_items_count_query_and_short_buffer(lib):
    """cap = 0 only counts; a short buffer gets the first cap items of the
    same list and the full count."""
    ext = [(40, 24, 50), (17, 9, 33)]
    n = (C.c_int * 6)(*[v for e in ext for v in e])
    count = C.c_int()
    assert lib.nyx_task_items(2, n, 16, 8, 152, 1, None, 0, C.byref(count)) == H.NYX_OK
    full = H.task_items(ext, 16, 8, 152, True)
    assert count.value == len(full) > 5
    buf = (C.c_int * (7 * 6))(*([-7] * 42))
    assert lib.nyx_task_items(2, n, 16, 8, 152, 1, buf, 5, C.byref(count)) == H.NYX_OK
    assert count.value == len(full)
    got = np.array(buf[:], dtype=np.int64).reshape(6, 7)
    assert np.array_equal(got[:5], full[:5]) and np.all(got[5] == -7)


def test_alu_peak_rejects_bad_arguments(lib):
    out = C.c_double(-1.0)
    assert lib.nyx_alu_peak(2, 0.25, None, C.byref(out)) == H.NYX_EINVAL
    assert lib.nyx_alu_peak(0, 0.0, None, C.byref(out)) == H.NYX_EINVAL
    assert lib.nyx_alu_peak(1, 11.0, None, C.byref(out)) == H.NYX_EINVAL
    assert lib.nyx_alu_peak(0, 0.25, None, None) == H.NYX_EINVAL
    assert out.value == -1.0
