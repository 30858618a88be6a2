"""GPU parity of the dark-matter particle-mesh step (Sec. 3.3-3.6,
nyx_pm_*) against the oracle: cloud-in-cell deposit, the particle time
step, and one step of the full single-level algorithm with gas, dark
matter and self-gravity (Steps 1-6) in FP64.  The deposit sums with
floating-point atomics, so the comparisons allow round-off (1e-12)."""
import numpy as np
import pytest

import oracle
from paper_1301_4498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
H = pytest.importorskip("paper_1301_4498_gb300.hydro")
torch = pytest.importorskip("torch")

FOUR_PI_G = 1.5


def _case():
    w = W.tiled_box(n=32, box=16, sigma=0.8, seed=9, nsteps=2)
    n = (32, 32, 32)
    dx = 1.0 / 32
    x, u, m = W.dm_particles(n, dx, seed=4, vel_rms=0.1, mass_total=5.0)
    return w, n, dx, x, u, m


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_deposit_and_time_step_match_the_oracle():
    w, n, dx, x, u, m = _case()
    rho_ref = oracle.pm_deposit(n, dx, x, m)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64")
    lev = H.make_level(plan, w.state, None)
    ps = H.Poisson(plan, four_pi_G=FOUR_PI_G)
    xd = torch.tensor(x, device="cuda")
    ud = torch.tensor(u, device="cuda")
    md = torch.tensor(m, device="cuda")
    rho = ps.dense(1)[0]
    ps.pm_deposit(xd, md, rho)
    torch.cuda.synchronize()
    assert _rel(rho.cpu().numpy(), rho_ref) <= 1e-13
    assert float(rho.sum()) * dx ** 3 == pytest.approx(m.sum(), rel=1e-12)
    _, _, _, g_ref = oracle.poisson_solve(w.level, oracle.PoissonParams(four_pi_G=FOUR_PI_G),
                                          w.state, 0.5, rho_dm=rho_ref, want_dense_g=True)
    g = ps.dense(3)
    ps.solve(lev.current, 0.5, None, warm_start=False, rho_dm=rho, g_dense=g)
    torch.cuda.synchronize()
    assert _rel(g.cpu().numpy(), g_ref) <= 1e-12
    dt_ref = oracle.pm_estdt(n, dx, g_ref, x, u, 0.5)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps.pm_estdt(xd, ud, g, 0.5, dt)
    torch.cuda.synchronize()
    assert dt.item() == pytest.approx(dt_ref, rel=1e-12)
    ps.close()
    plan.close()


def test_cosmological_step_matches_the_oracle():
    """Steps 1-6 with gas, dark matter and self-gravity."""
    w, n, dx, x, u, m = _case()
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    ah = 0.5 * (a0 + a1)
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl)
    PP = oracle.PoissonParams(four_pi_G=FOUR_PI_G)
    # oracle
    rho0 = oracle.pm_deposit(n, dx, x, m)
    phi, gl0, _, gd0 = oracle.poisson_solve(w.level, PP, w.state, a0, rho_dm=rho0,
                                            want_dense_g=True)
    oracle.fill_ghosts(w.level, gl0)
    dt = min(oracle.estdt(w.level, P, w.state, a0), oracle.pm_estdt(n, dx, gd0, x, u, a0))
    pred, _ = oracle.predict(w.level, P, w.state, gl0, a_old=a0, a_new=a1, dt=dt)
    x1, uh = oracle.pm_kick_drift(n, dx, gd0, x, u, a_old=a0, a_half=ah, dt=dt)
    rho1 = oracle.pm_deposit(n, dx, x1, m)
    _, gl1, _, gd1 = oracle.poisson_solve(w.level, PP, pred, a1, phi, rho_dm=rho1,
                                          want_dense_g=True)
    oracle.fill_ghosts(w.level, gl1)
    u1 = oracle.pm_kick(n, dx, gd1, x1, uh, a_half=ah, a_new=a1, dt=dt)
    ref, _ = oracle.correct(w.level, P, w.state, pred, gl0, gl1, a_old=a0, a_new=a1, dt=dt)
    # GPU
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64")
    lev = H.make_level(plan, w.state, None)
    ps = H.Poisson(plan, four_pi_G=FOUR_PI_G)
    xd = torch.tensor(x, device="cuda")
    ud = torch.tensor(u, device="cuda")
    md = torch.tensor(m, device="cuda")
    rho = ps.dense(1)[0]
    gd = ps.dense(3)
    gn, gp = plan.empty_field(3), plan.empty_field(3)
    a = torch.tensor([a0, a1], dtype=torch.float64, device="cuda")
    d = torch.zeros(2, dtype=torch.float64, device="cuda")
    ps.pm_deposit(xd, md, rho)
    ps.solve(lev.current, a0, gn, warm_start=False, rho_dm=rho, g_dense=gd)
    plan.estdt(lev, a[:1], d[:1])
    dtp = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps.pm_estdt(xd, ud, gd, a0, dtp)
    torch.cuda.synchronize()
    dtv = min(d[0].item(), dtp.item())
    assert dtv == pytest.approx(dt, rel=1e-12)
    d[0] = dt                                       # the same step on both sides
    plan.predict(lev, a[:1], a[1:], d[:1], gn)
    ps.pm_kick_drift(xd, ud, gd, a0, ah, dt)
    ps.pm_deposit(xd, md, rho)
    ps.solve(lev.state[1 - lev.cur], a1, gp, warm_start=True, rho_dm=rho, g_dense=gd)
    ps.pm_kick(xd, ud, gd, ah, a1, dt)
    plan.correct(lev, a[:1], a[1:], d[:1], gn, gp)
    torch.cuda.synchronize()
    assert plan.status() == (0, 0)
    assert _rel(xd.cpu().numpy(), x1) <= 1e-13
    assert _rel(ud.cpu().numpy(), u1) <= 1e-11
    got = plan.from_device(lev.current, 6)
    for c in range(6):
        num = max(np.abs(W.valid(p)[c] - W.valid(q)[c]).max() for p, q in zip(got, ref))
        den = max(np.abs(W.valid(q)[c]).max() for q in ref)
        assert num <= 1e-12 * den, c
    ps.close()
    plan.close()


def test_fused_kick_and_time_step():
    """nyx_pm_kick_estdt: the kick of nyx_pm_kick and the particle dt that
    nyx_pm_estdt gives for the kicked particles, from one pass (bitwise)."""
    w, n, dx, x, u, m = _case()
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64")
    lev = H.make_level(plan, w.state, None)
    ps = H.Poisson(plan, four_pi_G=FOUR_PI_G)
    xd = torch.tensor(x, device="cuda")
    md = torch.tensor(m, device="cuda")
    rho = ps.dense(1)[0]
    g = ps.dense(3)
    ps.pm_deposit(xd, md, rho)
    ps.solve(lev.current, 0.5, None, warm_start=False, rho_dm=rho, g_dense=g)
    u1 = torch.tensor(u, device="cuda")
    u2 = u1.clone()
    d1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    d2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps.pm_kick(xd, u1, g, 0.45, 0.5, 0.01)
    ps.pm_estdt(xd, u1, g, 0.5, d1)
    ps.pm_kick_estdt(xd, u2, g, 0.45, 0.5, 0.01, d2)
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)
    assert d1.item() == d2.item() and 0.0 < d1.item() < float("inf")
    un = oracle.pm_kick(n, dx, g.cpu().numpy(), x, u, a_half=0.45, a_new=0.5, dt=0.01)
    assert _rel(u1.cpu().numpy(), un) <= 1e-13
    ps.close()
    plan.close()


def test_cosmological_step_mixed_poisson_and_particles():
    """Steps 1-6 with a mixed-precision Poisson object (refinement solves:
    phi and g within ~1e-10 of the FP64 solve's).  The particles and the
    gas see that g, so the gates are 1e-6 on velocities and the gas and
    1e-9 on positions (the drift moves a particle by far less than a cell)."""
    w, n, dx, x, u, m = _case()
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    ah = 0.5 * (a0 + a1)
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl)
    PP = oracle.PoissonParams(four_pi_G=FOUR_PI_G)
    rho0 = oracle.pm_deposit(n, dx, x, m)
    phi, gl0, _, gd0 = oracle.poisson_solve(w.level, PP, w.state, a0, rho_dm=rho0,
                                            want_dense_g=True)
    oracle.fill_ghosts(w.level, gl0)
    dt = min(oracle.estdt(w.level, P, w.state, a0), oracle.pm_estdt(n, dx, gd0, x, u, a0))
    pred, _ = oracle.predict(w.level, P, w.state, gl0, a_old=a0, a_new=a1, dt=dt)
    x1, uh = oracle.pm_kick_drift(n, dx, gd0, x, u, a_old=a0, a_half=ah, dt=dt)
    rho1 = oracle.pm_deposit(n, dx, x1, m)
    _, gl1, _, gd1 = oracle.poisson_solve(w.level, PP, pred, a1, phi, rho_dm=rho1,
                                          want_dense_g=True)
    oracle.fill_ghosts(w.level, gl1)
    u1 = oracle.pm_kick(n, dx, gd1, x1, uh, a_half=ah, a_new=a1, dt=dt)
    ref, _ = oracle.correct(w.level, P, w.state, pred, gl0, gl1, a_old=a0, a_new=a1, dt=dt)
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64")
    lev = H.make_level(plan, w.state, None)
    ps = H.Poisson(plan, four_pi_G=FOUR_PI_G, precision="mixed")
    xd = torch.tensor(x, device="cuda")
    ud = torch.tensor(u, device="cuda")
    md = torch.tensor(m, device="cuda")
    rho = ps.dense(1)[0]
    gd = ps.dense(3)
    gn, gp = plan.empty_field(3), plan.empty_field(3)
    a = torch.tensor([a0, a1], dtype=torch.float64, device="cuda")
    d = torch.zeros(2, dtype=torch.float64, device="cuda")
    ps.pm_deposit(xd, md, rho)
    ps.solve(lev.current, a0, gn, warm_start=False, rho_dm=rho, g_dense=gd)
    dtp = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps.pm_estdt(xd, ud, gd, a0, dtp)
    torch.cuda.synchronize()
    assert dtp.item() == pytest.approx(oracle.pm_estdt(n, dx, gd0, x, u, a0), rel=1e-6)
    d[0] = dt
    plan.predict(lev, a[:1], a[1:], d[:1], gn)
    ps.pm_kick_drift(xd, ud, gd, a0, ah, dt)
    ps.pm_deposit(xd, md, rho)
    ps.solve(lev.state[1 - lev.cur], a1, gp, warm_start=True, rho_dm=rho, g_dense=gd)
    ps.pm_kick(xd, ud, gd, ah, a1, dt)
    plan.correct(lev, a[:1], a[1:], d[:1], gn, gp)
    torch.cuda.synchronize()
    assert plan.status() == (0, 0)
    assert _rel(xd.cpu().numpy(), x1) <= 1e-9
    assert _rel(ud.cpu().numpy(), u1) <= 1e-6
    got = plan.from_device(lev.current, 6)
    for c in range(6):
        num = max(np.abs(W.valid(p)[c] - W.valid(q)[c]).max() for p, q in zip(got, ref))
        den = max(np.abs(W.valid(q)[c]).max() for q in ref)
        assert num <= 1e-6 * den, c
    ps.close()
    plan.close()
