"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
identical seeded inputs.

Bar: the FP64 forms (per-box stage kernels and the fused persistent kernel)
match the oracle within 1e-12 normwise-relative L-infinity per conserved
field (both evaluate the same expression forms with IEEE-rounded FP64 and no
contraction, so they agree bit for bit in practice); the mixed-precision form
within the per-field gates of MIXED_GATES.
"""
import numpy as np
import pytest

import oracle
from gates import FP64_TOL, MIXED_GATES  # noqa: F401  (re-exported to the other GPU tests)
from paper_1301_4498_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1301_4498_gb300 import hydro as H  # noqa: E402

FIELDS = ("rho", "m_x", "m_y", "m_z", "rhoE", "rhoe")


def oracle_params(w, **kw):
    return oracle.OracleParams(gamma=w.gamma, cfl=w.cfl, **kw)


def gpu_run(w, nsteps, use_graph=False, **params):
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, **params)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(np.asarray(w.a_sched[:nsteps + 1], dtype=np.float64), device="cuda")
    dt = torch.zeros(nsteps + 1, dtype=torch.float64, device="cuda")
    plan.run(lev, a, dt, nsteps, compute_dt0=True, use_graph=use_graph)
    torch.cuda.synchronize()
    rc, flags = plan.status()
    assert rc == H.NYX_OK, (rc, flags)
    S = plan.from_device(lev.current, 6)
    out = (S, dt.cpu().numpy(), plan, lev)
    return out


def field_errors(got, ref):
    """Per field: normwise-relative L-inf and L1 over the valid cells of all boxes."""
    res = {}
    for c, name in enumerate(FIELDS):
        num_inf = max(np.abs(W.valid(g)[c] - W.valid(r)[c]).max() for g, r in zip(got, ref))
        den_inf = max(np.abs(W.valid(r)[c]).max() for r in ref)
        num_1 = sum(np.abs(W.valid(g)[c] - W.valid(r)[c]).sum() for g, r in zip(got, ref))
        den_1 = sum(np.abs(W.valid(r)[c]).sum() for r in ref)
        res[name] = (num_inf / den_inf if den_inf else num_inf, num_1 / den_1 if den_1 else num_1)
    return res


def assert_fp64(got, ref, tol=FP64_TOL):
    err = field_errors(got, ref)
    bad = {k: v for k, v in err.items() if not v[0] <= tol}
    assert not bad, err


# ------------------------------------------------------------------ ghost fill and dt

@pytest.mark.parametrize("make", [
    lambda: W.sod(),
    lambda: W.comoving_box(n=16, nsteps=1),
    lambda: W.tiled_box(n=64, box=32, nsteps=1),
    lambda: W.uneven_boxes(nbox=512, boxes=[0, 1, 2, 3, 4, 5], nsteps=1),
])
def test_ghost_fill_matches_oracle_bitwise(make):
    w = make()
    plan = H.Plan(w.level, gamma=w.gamma)
    d = plan.to_device(w.state, 6)
    plan.fill(d, 6)
    torch.cuda.synchronize()
    got = plan.from_device(d, 6)
    ref = [s.copy() for s in w.state]
    oracle.fill_ghosts(w.level, ref)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


def test_estdt_matches_oracle_bitwise():
    w = W.uneven_boxes(nbox=512, boxes=list(range(8)), nsteps=1)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor([1.0 / 51], dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.estdt(lev, a, dt)
    ref = oracle.estdt(w.level, oracle_params(w), w.state, 1.0 / 51)
    assert dt.item() == ref


# ------------------------------------------------------------------ FP64 parity

def _thin_slabs(nsteps=2):
    """A periodic 16 x 8 x 8 comoving field cut into four 16 x 8 x 2 slabs:
    every box has n_z = 2, so its z ghost cells come from boxes up to two
    slabs away, and the task form's plane pipeline (ring, input and flux
    hand-overs) runs at its shortest."""
    dx = 1.0 / 16
    lo = [[0, 0, 2 * k] for k in range(4)]
    hi = [[15, 7, 2 * k + 1] for k in range(4)]
    lev = W._mk(lo, hi, [0] * 4, [[dx] * 3] * 4, [0, 0, 0], [15, 7, 7], [0] * 6, "thin")
    f = W.comoving_fields((8, 8, 16), 0.5, 7, dx)
    S, G = [], []
    for b in range(4):
        sl = (slice(2 * b, 2 * b + 2), slice(0, 8), slice(0, 16))
        fb = W.Fields(f.rho[sl], f.u[(slice(None),) + sl], f.g[(slice(None),) + sl])
        s, g = W._patch_state(lev, b, fb)
        S.append(s)
        G.append(g)
    return W.Workload("thin slabs 16x8x2", lev, S, G, W.a_schedule(1 / 51, 1 / 49, nsteps),
                      5.0 / 3.0, 0.5, nsteps, False)


SMALL_CASES = {
    "sod": (lambda: W.sod(), 20),
    "comoving32": (lambda: W.comoving_box(n=32, nsteps=3), 3),
    "tiled64x8": (lambda: W.tiled_box(n=64, box=32, nsteps=2), 2),
    "uneven6": (lambda: W.uneven_boxes(nbox=512, boxes=[0, 1, 2, 3, 4, 5], nsteps=2), 2),
    "thin": (lambda: _thin_slabs(2), 2),
}


@pytest.fixture(scope="module")
def oracle_results():
    cache = {}

    def get(name):
        if name not in cache:
            make, n = SMALL_CASES[name]
            w = make()
            S, dts, _ = oracle.run(w.level, oracle_params(w), w.state, w.grav, w.a_sched, n)
            cache[name] = (w, S, dts, n)
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(SMALL_CASES))
def test_fp64_per_box_matches_oracle(oracle_results, name):
    w, ref, dts, n = oracle_results(name)
    S, dt, _, _ = gpu_run(w, n, batching="per_box")
    assert np.array_equal(dt[:n], np.asarray(dts))
    assert_fp64(S, ref)


@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("name", list(SMALL_CASES))
def test_fp64_fused_matches_oracle(oracle_results, name, shape):
    w, ref, dts, n = oracle_results(name)
    plan_kw = dict(batching="persistent")
    S, dt, plan, _ = gpu_run(w, n, **plan_kw) if shape == 0 else _run_shape(w, n, shape)
    assert_fp64(S, ref)


def _run_shape(w, n, shape):
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, batching="persistent")
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(np.asarray(w.a_sched[:n + 1], dtype=np.float64), device="cuda")
    dt = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    _set_shape(plan, shape)
    plan.run(lev, a, dt, n, compute_dt0=True, use_graph=False)
    torch.cuda.synchronize()
    rc, flags = plan.status()
    assert rc == H.NYX_OK
    return plan.from_device(lev.current, 6), dt.cpu().numpy(), plan, lev


def _set_shape(plan, shape):
    plan.set_tile_shape(shape)
    assert plan.tile_shape()[0] == shape


def test_fused_equals_per_box_bitwise():
    w = W.uneven_boxes(nbox=512, boxes=list(range(10, 22)), nsteps=2)
    S1, dt1, _, _ = gpu_run(w, 2, batching="per_box")
    S2, dt2, _, _ = gpu_run(w, 2, batching="persistent")
    assert np.array_equal(dt1, dt2)
    for a, b in zip(S1, S2):
        assert np.array_equal(W.valid(a), W.valid(b))


def test_graph_replay_equals_eager():
    w = W.tiled_box(n=64, box=32, nsteps=4)
    S1, dt1, _, _ = gpu_run(w, 4, use_graph=False, precision="mixed")
    S2, dt2, _, _ = gpu_run(w, 4, use_graph=True, precision="mixed")
    assert np.array_equal(dt1, dt2)
    for a, b in zip(S1, S2):
        assert np.array_equal(W.valid(a), W.valid(b))


def test_repeat_runs_bitwise_deterministic():
    w = W.comoving_box(n=32, nsteps=2)
    S1, _, _, _ = gpu_run(w, 2, precision="mixed")
    S2, _, _, _ = gpu_run(w, 2, precision="mixed")
    for a, b in zip(S1, S2):
        assert np.array_equal(W.valid(a), W.valid(b))


# ------------------------------------------------------------------ mixed precision

@pytest.mark.parametrize("name", ["comoving32", "tiled64x8", "uneven6"])
def test_mixed_within_gates(oracle_results, name):
    w, ref, dts, n = oracle_results(name)
    S, dt, _, _ = gpu_run(w, n, precision="mixed")
    err = field_errors(S, ref)
    for k, (linf, l1) in err.items():
        assert linf <= MIXED_GATES["linf"] and l1 <= MIXED_GATES["l1"], (k, err)


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("name", ["sod", "tiled64x8", "uneven6", "thin"])
def test_mixed_every_tile_shape_within_gates(oracle_results, name, shape):
    """Both forms of the mixed kernel (column-owning shapes 0-2, task form
    3-5), including ragged tiles of the uneven boxes."""
    w, ref, dts, n = oracle_results(name)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed")
    plan.set_tile_shape(shape)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(np.asarray(w.a_sched[:n + 1], dtype=np.float64), device="cuda")
    dt = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    plan.run(lev, a, dt, n, compute_dt0=True, use_graph=False)
    torch.cuda.synchronize()
    rc, flags = plan.status()
    assert rc == H.NYX_OK, (rc, flags)
    err = field_errors(plan.from_device(lev.current, 6), ref)
    for k, (linf, l1) in err.items():
        assert linf <= MIXED_GATES["linf"] and l1 <= MIXED_GATES["l1"], (shape, k, err)


def test_fp64_rejects_task_form_shapes():
    w = W.comoving_box(n=16, nsteps=1)
    plan = H.Plan(w.level, gamma=w.gamma, precision="fp64")
    with pytest.raises(H.NyxError):
        plan.set_tile_shape(3)


# ------------------------------------------------------------------ fluxes, host step, status

def test_flux_export_matches_oracle():
    w = W.uneven_boxes(nbox=512, boxes=[0, 1, 2], nsteps=1)
    P = oracle_params(w)
    dt = oracle.estdt(w.level, P, w.state, w.a_sched[0])
    _, _, flux = oracle.advance(w.level, P, w.state, w.grav, a_old=w.a_sched[0],
                                a_new=w.a_sched[1], dt=dt, want_flux=True)
    for batching in ("per_box", "persistent"):
        plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, batching=batching, keep_fluxes=1)
        if batching == "persistent":
            plan.set_tile_shape(2)  # ragged 16 x 8 tiles on these boxes
        lev = H.make_level(plan, w.state, w.grav)
        a = torch.tensor(w.a_sched[:2], dtype=torch.float64, device="cuda")
        d = torch.tensor([dt], dtype=torch.float64, device="cuda")
        plan.advance(lev, a[0:1], a[1:2], d)
        for b in range(3):
            for di in range(3):
                f = plan.fluxes(lev, b, di).cpu().numpy()
                r = flux[b][di]
                assert np.abs(f - r).max() <= FP64_TOL * np.abs(r).max(), (batching, b, di)


def test_step_host_matches_device_path():
    w = W.tiled_box(n=64, box=32, nsteps=1)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed")
    lev = H.make_level(plan, w.state, w.grav)
    host_in = torch.from_numpy(plan.pack_host(w.state, 6)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dt_next = plan.step_host(lev, host_in, host_out, float(w.a_sched[0]), float(w.a_sched[1]))
    S_host = plan.unpack_host(host_out.numpy(), 6)
    S_dev, dts, _, _ = gpu_run(w, 1, precision="mixed")
    for a, b in zip(S_host, S_dev):
        assert np.array_equal(W.valid(a), W.valid(b))
    assert dt_next == dts[1]


def test_negative_density_raises_status_without_fault():
    w = W.comoving_box(n=16, nsteps=1)
    w.state[0][0, 10, 10, 10] = -1.0  # an invalid input cell
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed")
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(w.a_sched[:2], dtype=torch.float64, device="cuda")
    dt = torch.tensor([1e-4], dtype=torch.float64, device="cuda")
    plan.advance(lev, a[0:1], a[1:2], dt)
    rc, flags = plan.status()
    assert rc in (H.NYX_ENEGATIVE, H.NYX_ENONFINITE) and flags != 0
    rc2, flags2 = plan.status()  # cleared
    assert rc2 == H.NYX_OK and flags2 == 0
    # the context is still usable
    x = torch.ones(4, device="cuda") * 2
    assert x.sum().item() == 8.0


@pytest.mark.parametrize("shape", [0, 3])
def test_mixed_flux_export_close_to_oracle(shape):
    """Flux export of the mixed path (both kernel forms) against the FP64
    oracle's fluxes: FP32 accuracy, normwise per component."""
    w = W.uneven_boxes(nbox=512, boxes=[0, 1], nsteps=1)
    P = oracle_params(w)
    dt = oracle.estdt(w.level, P, w.state, w.a_sched[0])
    _, _, flux = oracle.advance(w.level, P, w.state, w.grav, a_old=w.a_sched[0],
                                a_new=w.a_sched[1], dt=dt, want_flux=True)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed", keep_fluxes=1)
    plan.set_tile_shape(shape)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(w.a_sched[:2], dtype=torch.float64, device="cuda")
    d = torch.tensor([dt], dtype=torch.float64, device="cuda")
    plan.advance(lev, a[0:1], a[1:2], d)
    for b in range(2):
        for di in range(3):
            f = plan.fluxes(lev, b, di).cpu().numpy()
            r = flux[b][di]
            for c in range(6):
                scale = np.abs(r[c]).max()
                assert np.abs(f[c] - r[c]).max() <= 2e-3 * scale, (shape, b, di, c)


def test_autotuned_graph_run_reports_clean_status():
    """The autotuner times its shapes on the real first step before a graph
    capture; its timing launches must leave the plan's status clean and the
    result equal to an untuned eager run with the chosen shape."""
    w = W.tiled_box(n=64, box=32, nsteps=2)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed", autotune=1)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(w.a_sched[:3], dtype=torch.float64, device="cuda")
    dt = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan.run(lev, a, dt, 2, compute_dt0=True, use_graph=True)
    torch.cuda.synchronize()
    assert plan.status() == (H.NYX_OK, 0)
    shape = plan.tile_shape()[0]
    got = plan.from_device(lev.current, 6)
    plan2 = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed")
    plan2.set_tile_shape(shape)
    lev2 = H.make_level(plan2, w.state, w.grav)
    dt2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan2.run(lev2, a, dt2, 2, compute_dt0=True, use_graph=False)
    ref = plan2.from_device(lev2.current, 6)
    for x, y in zip(got, ref):
        assert np.array_equal(W.valid(x), W.valid(y))


def test_step_host_valid_matches_device_path():
    """nyx_hydro_step_host_valid: only the valid cells cross the host link;
    the step is the device path's, bitwise, and so is the next dt."""
    w = W.tiled_box(n=64, box=32, nsteps=1)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed")
    lev = H.make_level(plan, w.state, w.grav)
    host_in = torch.from_numpy(plan.pack_valid(w.state)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dt_next = plan.step_host_valid(lev, host_in, host_out, float(w.a_sched[0]),
                                   float(w.a_sched[1]))
    got = plan.unpack_valid(host_out.numpy())
    S_dev, dts, _, _ = gpu_run(w, 1, precision="mixed")
    for a, b in zip(got, S_dev):
        assert np.array_equal(a, W.valid(b))
    assert dt_next == dts[1]
    # a second call reuses the staging buffer and continues from host_out
    host_in.copy_(host_out)
    plan.step_host_valid(lev, host_in, host_out, float(w.a_sched[0]), float(w.a_sched[1]),
                         dt_next)
    assert np.isfinite(host_out.numpy()).all()
    plan.close()


@pytest.mark.parametrize("shape", [3, 5])
def test_step_host_valid_overlapped_read_back_matches_device_path(shape):
    """A level of 1000 boxes of 16^3 (13 or more waves of work items): the
    advance of nyx_hydro_step_host_valid runs one launch per group of boxes,
    and each group's new cells are copied to the host while the next groups
    advance.  The result and the next dt are the device path's, bit for bit;
    the plan's launch counter shows the groups (one advance launch and one
    gather per group, against one of each).  With dt given, the groups'
    input copies overlap the fills and advances of earlier groups as well,
    for the same result."""
    w = W.tiled_box(n=160, box=16, nsteps=1)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed")
    plan.set_tile_shape(shape)
    lev = H.make_level(plan, w.state, w.grav)
    host_in = torch.from_numpy(plan.pack_valid(w.state)).pin_memory()
    host_out = torch.full_like(host_in, float("nan")).pin_memory()
    plan.counters(reset=True)
    dt_next = plan.step_host_valid(lev, host_in, host_out, float(w.a_sched[0]),
                                   float(w.a_sched[1]))
    n_host = plan.counters(reset=True)["launches"]
    got = plan.unpack_valid(host_out.numpy())
    ref = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed")
    ref.set_tile_shape(shape)
    rlev = H.make_level(ref, w.state, w.grav)
    a = torch.tensor(np.asarray(w.a_sched[:2], dtype=np.float64), device="cuda")
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    ref.counters(reset=True)
    ref.estdt(rlev, a[0:1], dt[0:1])          # the one-launch device path: estdt, then
    ref.advance(rlev, a[0:1], a[1:2], dt[0:1], dt_next=dt[1:2])  # fill + one advance launch
    torch.cuda.synchronize()
    n_dev = ref.counters(reset=True)["launches"]
    assert ref.status()[0] == H.NYX_OK and plan.status()[0] == H.NYX_OK
    for x, y in zip(got, ref.from_device(rlev.current, 6)):
        assert np.array_equal(x, W.valid(y))
    assert dt_next == dt.cpu().numpy()[1]
    groups = (n_host - n_dev) // 2          # scatter + G gathers + G advances vs 1 advance
    assert n_host - n_dev == 2 * groups and groups >= 2, (n_host, n_dev)
    # with dt given, the input is pipelined too: each group's cells are
    # copied in and scattered while earlier groups fill and advance
    out2 = torch.full_like(host_in, float("nan")).pin_memory()
    dt0 = float(dt.cpu().numpy()[0])
    dt_next2 = plan.step_host_valid(lev, host_in, out2, float(w.a_sched[0]),
                                    float(w.a_sched[1]), dt0)
    assert plan.status()[0] == H.NYX_OK
    assert torch.equal(out2, host_out) and dt_next2 == dt_next
    plan.close()
    ref.close()


def test_step_host_valid_overlapped_with_flattening_matches_device_path():
    """The overlapped host step of a flattening plan (each group's
    coefficient pass after its own fill) equals the device path bit for bit,
    with dt given and with dt computed."""
    w = W.tiled_box(n=160, box=16, sigma=0.6, seed=3, nsteps=1)
    kw = dict(gamma=w.gamma, cfl=w.cfl, precision="mixed", flattening=True)
    ref = H.Plan(w.level, **kw)
    ref.set_tile_shape(3)
    rlev = H.make_level(ref, w.state, w.grav)
    a = torch.tensor(np.asarray(w.a_sched[:2], dtype=np.float64), device="cuda")
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    ref.estdt(rlev, a[0:1], dt[0:1])
    ref.advance(rlev, a[0:1], a[1:2], dt[0:1], dt_next=dt[1:2])
    torch.cuda.synchronize()
    assert ref.status()[0] == H.NYX_OK
    want = [W.valid(x) for x in ref.from_device(rlev.current, 6)]
    d = dt.cpu().numpy()
    plan = H.Plan(w.level, **kw)
    plan.set_tile_shape(3)
    lev = H.make_level(plan, w.state, w.grav)
    host_in = torch.from_numpy(plan.pack_valid(w.state)).pin_memory()
    for dt_in in (0.0, float(d[0])):
        out = torch.full_like(host_in, float("nan")).pin_memory()
        dt_next = plan.step_host_valid(lev, host_in, out, float(w.a_sched[0]),
                                       float(w.a_sched[1]), dt_in)
        assert plan.status()[0] == H.NYX_OK
        for x, y in zip(plan.unpack_valid(out.numpy()), want):
            assert np.array_equal(x, y), dt_in
        assert dt_next == d[1]
    plan.close()
    ref.close()


@pytest.mark.parametrize("precision,shape,flat", [("mixed", 3, False), ("mixed", 3, True),
                                                   ("fp64", 1, False)])
def test_grouped_run_equals_one_launch_steps(precision, shape, flat):
    """nyx_hydro_run on a level with box groups (1000 boxes of 16^3) runs
    each step as one launch per group, with each group's ghost fill (and
    flattening pass) on a fill stream beside the other groups' advances.
    Eager and graph-captured, the states and every dt equal, bit for bit,
    those of one fill and one advance launch per step (nyx_hydro_advance)."""
    n = 3
    w = W.tiled_box(n=160, box=16, nsteps=n)
    kw = dict(gamma=w.gamma, cfl=w.cfl, precision=precision, flattening=flat)
    a = torch.tensor(np.asarray(w.a_sched[:n + 1], dtype=np.float64), device="cuda")
    ref = H.Plan(w.level, **kw)
    ref.set_tile_shape(shape)
    rlev = H.make_level(ref, w.state, w.grav)
    dt_ref = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    ref.counters(reset=True)
    ref.estdt(rlev, a[0:1], dt_ref[0:1])
    for s in range(n):
        ref.advance(rlev, a[s:s + 1], a[s + 1:s + 2], dt_ref[s:s + 1], dt_next=dt_ref[s + 1:s + 2])
    torch.cuda.synchronize()
    n_ref = ref.counters(reset=True)["launches"]
    assert ref.status()[0] == H.NYX_OK
    want = [W.valid(x) for x in ref.from_device(rlev.current, 6)]
    for use_graph in (False, True):
        plan = H.Plan(w.level, **kw)
        plan.set_tile_shape(shape)
        lev = H.make_level(plan, w.state, w.grav)
        dt = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        plan.counters(reset=True)
        plan.run(lev, a, dt, n, compute_dt0=True, use_graph=use_graph)
        torch.cuda.synchronize()
        n_run = plan.counters(reset=True)["launches"]
        assert plan.status()[0] == H.NYX_OK
        assert torch.equal(dt, dt_ref), use_graph
        for x, y in zip(plan.from_device(lev.current, 6), want):
            assert np.array_equal(W.valid(x), y), use_graph
        assert n_run > n_ref + 2 * n, (n_run, n_ref)  # one advance launch per group and step
        plan.close()
    ref.close()


def _tall_box(nsteps=2):
    """A periodic 32 x 16 x 94 comoving box: 4 tiles of 16 x 8, far fewer
    than CTAs, over tall columns that the work list cuts into chunks of 18
    and 19 planes."""
    dx = 1.0 / 94
    lev = W.single_box_level(32, 16, 94, dx, name="tall")
    f = W.comoving_fields((94, 16, 32), 0.5, 5, dx)
    S, G = W._patch_state(lev, 0, f)
    return W.Workload("tall 32x16x94", lev, [S], [G], W.a_schedule(1 / 51, 1 / 49, nsteps),
                      5.0 / 3.0, 0.5, nsteps, False)


def _chunk_run(w, n, shape, z_chunks, precision="mixed", **kw):
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision=precision, z_chunks=z_chunks, **kw)
    plan.set_tile_shape(shape)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(np.asarray(w.a_sched[:n + 1], dtype=np.float64), device="cuda")
    dt = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    plan.run(lev, a, dt, n, compute_dt0=True, use_graph=False)
    torch.cuda.synchronize()
    assert plan.status()[0] == H.NYX_OK
    return plan, lev, dt.cpu().numpy()


@pytest.mark.parametrize("shape", [3, 4, 5])
@pytest.mark.parametrize("name", ["comoving32", "tiled64x8", "thin", "tall"])
def test_task_form_chunks_equal_whole_columns_bitwise(oracle_results, name, shape):
    """The task form with its columns cut into plane chunks (what the work
    list does where tiles are fewer than CTAs) gives the whole-column result
    bit for bit: each face flux comes from the same stencil in the same
    order, whichever item computes it.  Also with flattening and with the
    fluxes kept for reflux."""
    if name == "tall":
        w, n = _tall_box(2), 2
    else:
        w, _, _, n = oracle_results(name)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tx, ty = H.tile_shape_of(shape)
    ext = [w.level.extent(b) for b in range(w.level.nbox)]
    slots = sms * (2 if shape == 4 else 1)
    chunked = H.task_items(ext, tx, ty, slots, True)
    if name != "thin":       # the 2-plane slabs stay whole; the others are cut
        assert len(chunked) > len(H.task_items(ext, tx, ty, slots, False))
    for kw in (dict(), dict(flattening=True, keep_fluxes=1)):
        p1, l1, d1 = _chunk_run(w, n, shape, 1, **kw)
        p0, l0, d0 = _chunk_run(w, n, shape, 0, **kw)
        assert np.array_equal(d0, d1)
        for x, y in zip(p1.from_device(l1.current, 6), p0.from_device(l0.current, 6)):
            assert np.array_equal(W.valid(x), W.valid(y))
        if kw:
            for b in range(w.level.nbox):
                for di in range(3):
                    assert torch.equal(p1.fluxes(l1, b, di), p0.fluxes(l0, b, di)), (b, di)
        p1.close()
        p0.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("name", ["comoving32", "tall"])
def test_column_form_chunks_equal_whole_columns_bitwise(oracle_results, name, shape, precision):
    """The column-owning form (the FP64 path's fused kernel) with its columns
    cut into plane chunks gives the whole-column result bit for bit, and the
    chunked list is longer where a box has fewer tiles than the GPU has
    SMs."""
    if name == "tall":
        w, n = _tall_box(2), 2
    else:
        w, _, _, n = oracle_results(name)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tx, ty = H.tile_shape_of(shape)
    ext = [w.level.extent(b) for b in range(w.level.nbox)]
    assert len(H.task_items(ext, tx, ty, sms, True)) > len(H.task_items(ext, tx, ty, sms, False))
    p1, l1, d1 = _chunk_run(w, n, shape, 1, precision)
    p0, l0, d0 = _chunk_run(w, n, shape, 0, precision)
    assert np.array_equal(d0, d1)
    for x, y in zip(p1.from_device(l1.current, 6), p0.from_device(l0.current, 6)):
        assert np.array_equal(W.valid(x), W.valid(y))
    p1.close()
    p0.close()


# ------------------------------------------------------------------ degenerate input

def _uniform_moving(n=48, box=24, nsteps=2):
    """A uniform state moving obliquely under a uniform gravity, on a periodic
    n^3 level of box^3 boxes (24 = 16 + 8: ragged 16 x 8 tiles)."""
    lev = W.tiled_level(n, box)
    shape = (box, box, box)
    rho = np.full(shape, 1.3)
    u = np.stack([np.full(shape, v) for v in (0.2, -0.1, 0.05)])
    g = np.stack([np.full(shape, v) for v in (0.01, 0.02, -0.03)])
    S, G = [], []
    for b in range(lev.nbox):
        s, gg = W._patch_state(lev, b, W.Fields(rho, u, g))
        S.append(s)
        G.append(gg)
    return W.Workload("uniform", lev, S, G, W.a_schedule(1.0 / 51, 1.0 / 49, nsteps), 5.0 / 3.0,
                      0.5, nsteps)


@pytest.mark.parametrize("precision,shape", [("fp64", 1), ("mixed", 0), ("mixed", 3)])
def test_uniform_state_stays_uniform_and_matches_oracle(precision, shape):
    """Every face of a uniform state carries the same flux, so the flux
    divergence vanishes exactly and every cell of every box takes the same
    update: the result is uniform bit for bit, in both precisions and on
    ragged tiles; its value is the oracle's (FP64 tolerance, mixed gates)."""
    w = _uniform_moving()
    n = 2
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision=precision)
    plan.set_tile_shape(shape)
    lev = H.make_level(plan, w.state, w.grav)
    a = torch.tensor(np.asarray(w.a_sched[:n + 1], dtype=np.float64), device="cuda")
    dt = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    plan.run(lev, a, dt, n, compute_dt0=True, use_graph=False)
    torch.cuda.synchronize()
    assert plan.status()[0] == H.NYX_OK
    got = plan.from_device(lev.current, 6)
    first = W.valid(got[0])[:, :1, :1, :1]
    for g in got:
        assert np.array_equal(W.valid(g), np.broadcast_to(first, W.valid(g).shape))
    ref, _, _ = oracle.run(w.level, oracle_params(w), w.state, w.grav, w.a_sched, n)
    err = field_errors(got, ref)
    for k, (linf, l1) in err.items():
        if precision == "fp64":
            assert linf <= FP64_TOL, (k, err)
        else:
            assert linf <= MIXED_GATES["linf"] and l1 <= MIXED_GATES["l1"], (k, err)
