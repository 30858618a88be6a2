"""The per-class autotuner of persistent plans (nyx_hydro_tune_info): every
box-size class is timed once, its choice lands in the JSON cache, a second
plan of the same level makes no trial launch, and a level whose classes
choose different tile shapes (one launch per choice) gives the result of the
oracle within the mixed gates."""
import json
import os

import numpy as np
import pytest

import oracle
from gates import MIXED_GATES
from paper_1301_4498_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1301_4498_gb300 import hydro as H  # noqa: E402
from test_gpu_parity import field_errors  # noqa: E402


def _level():
    # the large level's box mix on a 64^3 domain: 8 boxes of 32^3 and 2
    # independent 64^3 boxes at half the cell width -- two classes
    return W.large_level(n=64, box=32, nfine=2, nsteps=100)


def _one_step(w, **kw):
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed", autotune=1, **kw)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(w.a_sched[:2], dtype=torch.float64, device="cuda")
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    plan.run(lev, a, dt, 1, compute_dt0=True, use_graph=False)
    torch.cuda.synchronize()
    rc, flags = plan.status()
    assert rc == H.NYX_OK, (rc, flags)
    return plan, plan.from_device(lev.current, 6)


def test_second_plan_takes_every_class_from_the_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("NYX_TUNE_CACHE", str(cache))
    w = _level()
    p1, s1 = _one_step(w)
    classes, trials, launches = p1.tune_info()
    assert classes == 2 and trials > 0 and launches >= 1
    entries = json.loads(cache.read_text())
    assert len(entries) == 2
    assert all(k.endswith(("32x32x32", "64x64x64")) and "|mixed|" in k for k in entries)
    p2, s2 = _one_step(w)
    assert p2.tune_info() == (2, 0, launches)
    assert p2.tile_shape()[0] == p1.tile_shape()[0]
    for x, y in zip(s1, s2):
        assert np.array_equal(W.valid(x), W.valid(y))


def test_classes_with_different_shapes_launch_separately(tmp_path, monkeypatch):
    props = torch.cuda.get_device_properties(0)
    prefix = f"{props.name}|sm{props.multi_processor_count}|mixed|v0|"
    cache = tmp_path / "tune.json"
    # 32^3 boxes in 16 x 8 tiles at one CTA per SM, 64^3 boxes in 8 x 8 tiles
    # at two: two launches per advance
    cache.write_text("{\n"
                     f' "{prefix}32x32x32": {{"shape": 3, "ctas_per_sm": 1, "ns_per_zone": 1}},\n'
                     f' "{prefix}64x64x64": {{"shape": 4, "ctas_per_sm": 2, "ns_per_zone": 1}}\n'
                     "}\n")
    monkeypatch.setenv("NYX_TUNE_CACHE", str(cache))
    w = _level()
    plan, got = _one_step(w)
    assert plan.tune_info() == (2, 0, 2)
    ref, _, _ = oracle.run(w.level, oracle.OracleParams(gamma=w.gamma, cfl=w.cfl), w.state,
                           w.grav, w.a_sched, 1)
    err = field_errors(got, ref)
    print("two-launch level, 1 step, mixed vs oracle:", err)
    for k, (linf, l1) in err.items():
        assert linf <= MIXED_GATES["linf"] and l1 <= MIXED_GATES["l1"], (k, err)
    # the end-to-end host step takes the same two launches
    host_in = torch.from_numpy(plan.pack_valid(w.state)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    plan.step_host_valid(H.make_level(plan, w.state, w.grav), host_in, host_out,
                         float(w.a_sched[0]), float(w.a_sched[1]), 0.0)
    torch.cuda.synchronize()
    assert plan.status()[0] == H.NYX_OK
    back = plan.unpack_valid(host_out.numpy())  # valid cells only
    for x, y in zip(back, got):
        assert np.array_equal(x, W.valid(y))


def test_no_cache_file_when_disabled(tmp_path, monkeypatch):
    monkeypatch.setenv("NYX_TUNE_CACHE", "")
    monkeypatch.chdir(tmp_path)
    w = _level()
    p, _ = _one_step(w)
    assert p.tune_info()[1] > 0
    assert not os.listdir(tmp_path)
