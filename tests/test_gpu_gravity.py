"""GPU parity of the gravity source variants against the oracle: energy
option (ii) in the fused advance, and Step 2 / Step 6 run separately with a
gravity field recomputed at t^{n+1} (nyx_hydro_predict, nyx_hydro_correct).
FP64 within 1e-12 normwise per field; mixed within the mixed gate."""
import numpy as np
import pytest

import oracle
from gates import MIXED_GATES
from paper_1301_4498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
H = pytest.importorskip("paper_1301_4498_gb300.hydro")
torch = pytest.importorskip("torch")


def _norm_rel(got, ref):
    worst = 0.0
    for c in range(ref[0].shape[0]):
        num = max(np.abs(W.valid(g)[c] - W.valid(r)[c]).max() for g, r in zip(got, ref))
        den = max(np.abs(W.valid(r)[c]).max() for r in ref)
        worst = max(worst, num / max(den, 1e-300))
    return worst


def _case():
    w = W.tiled_box(n=32, box=16, sigma=0.6, seed=7, nsteps=2)
    g_old = [g.copy() for g in w.grav]
    oracle.fill_ghosts(w.level, g_old)
    g_new = [1.3 * g for g in g_old]            # gravity recomputed at t^{n+1}
    return w, g_old, g_new


def _scalars(w, dt):
    a = torch.tensor([float(w.a_sched[0]), float(w.a_sched[1])], dtype=torch.float64,
                     device="cuda")
    d = torch.tensor([dt, 0.0], dtype=torch.float64, device="cuda")
    return a, d


@pytest.mark.parametrize("batching", ["persistent", "per_box"])
def test_fused_advance_with_energy_option_two(batching):
    w, g_old, _ = _case()
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl, grav_energy=1)
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dt = oracle.estdt(w.level, P, w.state, a0)
    ref, _, _ = oracle.advance(w.level, P, w.state, g_old, a_old=a0, a_new=a1, dt=dt)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64", batching=batching,
                  grav_energy=1)
    lev = H.make_level(plan, w.state, w.grav)
    a, d = _scalars(w, dt)
    plan.advance(lev, a[:1], a[1:], d[:1], dt_next=d[1:])
    torch.cuda.synchronize()
    assert plan.status() == (0, 0)
    assert _norm_rel(plan.from_device(lev.current, 6), ref) <= 1e-12
    plan.close()


@pytest.mark.parametrize("grav_energy", [0, 1])
@pytest.mark.parametrize("batching", ["persistent", "per_box"])
def test_predict_then_correct_with_new_gravity(grav_energy, batching):
    w, g_old, g_new = _case()
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl, grav_energy=grav_energy)
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dt = oracle.estdt(w.level, P, w.state, a0)
    pred, _ = oracle.predict(w.level, P, w.state, g_old, a_old=a0, a_new=a1, dt=dt)
    ref, _ = oracle.correct(w.level, P, w.state, pred, g_old, g_new, a_old=a0, a_new=a1, dt=dt)
    dt_next = oracle.estdt(w.level, P, ref, a1)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64", batching=batching,
                  grav_energy=grav_energy)
    lev = H.make_level(plan, w.state, w.grav)
    gn = plan.to_device(g_new, 3)
    a, d = _scalars(w, dt)
    plan.predict(lev, a[:1], a[1:], d[:1], lev.grav)
    torch.cuda.synchronize()
    assert _norm_rel(plan.from_device(lev.state[1 - lev.cur], 6), pred) <= 1e-12
    plan.correct(lev, a[:1], a[1:], d[:1], lev.grav, gn, dt_next=d[1:])
    torch.cuda.synchronize()
    assert plan.status() == (0, 0)
    assert _norm_rel(plan.from_device(lev.current, 6), ref) <= 1e-12
    assert abs(d[1].item() - dt_next) <= 1e-12 * dt_next
    plan.close()


def test_split_equals_fused_on_the_gpu():
    """With g^{n+1} = g^n, nyx_hydro_predict + nyx_hydro_correct reproduce
    nyx_hydro_advance bit for bit (FP64)."""
    w, g_old, _ = _case()
    res = []
    for split in (False, True):
        plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64")
        lev = H.make_level(plan, w.state, w.grav)
        a, d = _scalars(w, 0.0)
        plan.estdt(lev, a[:1], d[:1])
        if split:
            plan.predict(lev, a[:1], a[1:], d[:1], lev.grav)
            plan.correct(lev, a[:1], a[1:], d[:1], lev.grav, lev.grav, dt_next=d[1:])
        else:
            plan.advance(lev, a[:1], a[1:], d[:1], dt_next=d[1:])
        torch.cuda.synchronize()
        res.append((plan.from_device(lev.current, 6), d.cpu().numpy()))
        plan.close()
    for x, y in zip(res[0][0], res[1][0]):
        assert np.array_equal(W.valid(x), W.valid(y))
    assert np.array_equal(res[0][1], res[1][1])


def test_predict_then_correct_mixed_within_the_gate():
    w, g_old, g_new = _case()
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl, grav_energy=1)
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dt = 0.9 * oracle.estdt(w.level, P, w.state, a0)
    pred, _ = oracle.predict(w.level, P, w.state, g_old, a_old=a0, a_new=a1, dt=dt)
    ref, _ = oracle.correct(w.level, P, w.state, pred, g_old, g_new, a_old=a0, a_new=a1, dt=dt)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="mixed", grav_energy=1)
    lev = H.make_level(plan, w.state, w.grav)
    gn = plan.to_device(g_new, 3)
    a, d = _scalars(w, dt)
    plan.predict(lev, a[:1], a[1:], d[:1], lev.grav)
    plan.correct(lev, a[:1], a[1:], d[:1], lev.grav, gn)
    torch.cuda.synchronize()
    assert plan.status() == (0, 0)
    e_mixed = _norm_rel(plan.from_device(lev.current, 6), ref)
    print('mixed vs oracle, worst field L-inf:', e_mixed)
    assert e_mixed <= MIXED_GATES["linf"]
    plan.close()
