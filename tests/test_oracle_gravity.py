"""Pins of the gravity source variants (Sec. 3.2 and Sec. 3.6 Steps 2, 4, 6):
the two discretisations of rho U . g in the total energy, and Step 6 run on
its own with a gravity field recomputed at t^{n+1}.

* With g^{n+1} = g^n, predictor then corrector is the fused advance, bit for
  bit, for both energy options.
* A uniform gas at rest, a = 1, uniform g^n != g^{n+1}: closed forms.  The
  momentum is rho dt (g^n + g^{n+1})/2; option (i) adds rho dt^2 g^n.g^{n+1}/2
  to rho E and so changes e by -rho dt^2 |g^n - g^{n+1}|^2 / 8; option (ii)
  adds exactly the new kinetic energy and leaves e unchanged (Sec. 3.2).
* Option (ii) leaves e to the hydro update on a uniform moving gas, and on a
  general flow its corrector changes rho E by exactly the kinetic-energy
  change of its momentum update."""
import numpy as np
import pytest

import oracle
from paper_1301_4498_gb300 import workloads as W

G53 = 5.0 / 3.0


def _comoving(seed=4):
    w = W.tiled_box(n=32, box=16, sigma=0.6, seed=seed, nsteps=2)
    return w


@pytest.mark.parametrize("grav_energy", [0, 1])
def test_split_equals_fused_when_gravity_is_unchanged(grav_energy):
    w = _comoving()
    P = oracle.OracleParams(gamma=w.gamma, grav_energy=grav_energy)
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dt = oracle.estdt(w.level, P, w.state, a0)
    g = [x.copy() for x in w.grav]
    oracle.fill_ghosts(w.level, g)
    fused, _, _ = oracle.advance(w.level, P, w.state, g, a_old=a0, a_new=a1, dt=dt)
    pred, _ = oracle.predict(w.level, P, w.state, g, a_old=a0, a_new=a1, dt=dt)
    split, _ = oracle.correct(w.level, P, w.state, pred, g, g, a_old=a0, a_new=a1, dt=dt)
    for x, y in zip(fused, split):
        assert np.array_equal(W.valid(x), W.valid(y))


def _rest(go, gn, grav_energy, rho=0.8, e=0.9, dt=0.01):
    S0 = np.array([rho, 0, 0, 0, rho * e, rho * e])
    w = W.uniform_level(S0, n=(8, 8, 8), dx=1 / 8, grav=go)
    wn = W.uniform_level(S0, n=(8, 8, 8), dx=1 / 8, grav=gn)
    P = oracle.OracleParams(gamma=G53, grav_energy=grav_energy)
    pred, _ = oracle.predict(w.level, P, w.state, w.grav, a_old=1.0, a_new=1.0, dt=dt)
    out, _ = oracle.correct(w.level, P, w.state, pred, w.grav, wn.grav, a_old=1.0, a_new=1.0,
                            dt=dt)
    return W.valid(out[0]), S0


@pytest.mark.parametrize("grav_energy", [0, 1])
def test_uniform_gas_at_rest_with_new_gravity(grav_energy):
    go = np.array([0.3, -0.2, 0.1])
    gn = np.array([0.25, -0.1, 0.3])
    rho, dt = 0.8, 0.01
    v, S0 = _rest(go, gn, grav_energy, rho=rho, dt=dt)
    m = 0.5 * rho * dt * (go + gn)
    for c in range(3):
        assert np.allclose(v[1 + c], m[c], rtol=1e-13, atol=0)
    ke = 0.5 * (m @ m) / rho
    if grav_energy == 0:
        rE = S0[4] + 0.5 * rho * dt * dt * (go @ gn)
        re = S0[5] - rho * dt * dt * ((go - gn) @ (go - gn)) / 8
    else:
        rE = S0[4] + ke
        re = S0[5]
    assert np.allclose(v[4], rE, rtol=1e-14, atol=0)
    assert np.allclose(v[5], re, rtol=1e-13, atol=0)
    assert np.allclose(v[4] - v[5], ke, rtol=1e-9, atol=0)


def test_option_two_leaves_internal_energy_to_the_hydro():
    """Uniform moving gas, uniform g, expansion: the fluxes do not depend on g
    (no divergence), so with option (ii) E - |m|^2/(2 rho) after the step is
    exactly the separately evolved rho e (the switch has nothing to do).
    (Option (i) agrees here: its corrector restores the dt^2 |g|^2 term when
    g^{n+1} = g^n and the density is unchanged.)"""
    grav_energy = 1
    rho, e = 1.1, 0.9
    u = np.array([0.1, -0.05, 0.02])
    m = rho * u
    S0 = np.array([rho, *m, rho * e + 0.5 * rho * (u @ u), rho * e])
    g = np.array([0.3, -0.2, 0.1])
    w = W.uniform_level(S0, n=(8, 8, 8), dx=1 / 8, grav=g)
    P = oracle.OracleParams(gamma=G53, grav_energy=grav_energy, dual_energy_sync=0)
    out, _, _ = oracle.advance(w.level, P, w.state, w.grav, a_old=1 / 51, a_new=1 / 50, dt=1e-3)
    v = W.valid(out[0])
    eint = v[4] - 0.5 * (v[1] ** 2 + v[2] ** 2 + v[3] ** 2) / v[0]
    gap = np.max(np.abs(eint - v[5])) / np.max(np.abs(v[5]))
    assert gap <= 1e-13


@pytest.mark.parametrize("grav_energy", [1, 0])
def test_option_two_corrector_adds_the_kinetic_energy_change(grav_energy):
    """General flow, g^{n+1} != g^n, switch off: with option (ii) the
    corrector changes rho E by exactly the kinetic-energy change of its
    momentum update; option (i) does not (a control)."""
    w = _comoving(seed=7)
    P = oracle.OracleParams(gamma=w.gamma, grav_energy=grav_energy, dual_energy_sync=0)
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dt = oracle.estdt(w.level, P, w.state, a0)
    go = [x.copy() for x in w.grav]
    oracle.fill_ghosts(w.level, go)
    gn = [1.3 * x for x in go]
    pred, _ = oracle.predict(w.level, P, w.state, go, a_old=a0, a_new=a1, dt=dt)
    out, _ = oracle.correct(w.level, P, w.state, pred, go, gn, a_old=a0, a_new=a1, dt=dt)
    worst = 0.0
    for x, y in zip(out, pred):
        x, y = W.valid(x), W.valid(y)
        dke = 0.5 * ((x[1:4] ** 2).sum(0) - (y[1:4] ** 2).sum(0)) / x[0]
        worst = max(worst, np.max(np.abs((x[4] - y[4]) - dke)) / np.max(np.abs(y[4])))
    if grav_energy == 1:
        assert worst <= 1e-14
    else:
        assert worst > 1e-9
