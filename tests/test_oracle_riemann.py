"""Pins of the oracle's two-shock Riemann solver (Sec. 3.2, Colella & Glaz
1985) and of the exact solver used to check it."""
import math
import os

import numpy as np
import pytest

import exact_riemann as ER
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _params(gamma=1.4, tol=1e-14, iters=60):
    return oracle.OracleParams(gamma=gamma, riemann_tol=tol, riemann_max_iter=iters)


# ---------------------------------------------------------------- exact solver pins

def test_exact_solver_matches_textbook_sod():
    ref = _golden("sod_star_state.txt")
    p, u = ER.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    rl, rr = ER.star_densities(1.0, 1.0, 0.125, 0.1, p, 1.4)
    assert p == pytest.approx(ref["p_star"], abs=1e-5)
    assert u == pytest.approx(ref["u_star"], abs=1e-5)
    assert rl == pytest.approx(ref["rho_star_left"], abs=1e-5)
    assert rr == pytest.approx(ref["rho_star_right"], abs=1e-5)


def test_exact_solver_jump_conditions():
    """Rankine-Hugoniot across the shock and isentropic invariants across
    the rarefaction, for the Sod data."""
    g = 1.4
    rl, ul, pl, rr, ur, pr = 1.0, 0.0, 1.0, 0.125, 0.0, 0.1
    p, u = ER.star_state(rl, ul, pl, rr, ur, pr, g)
    rsl, rsr = ER.star_densities(rl, pl, rr, pr, p, g)
    # right shock: mass, momentum, energy flux continuity in the shock frame
    S = ur + math.sqrt(g * pr / rr) * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
    m1, m2 = rr * (ur - S), rsr * (u - S)
    assert m1 == pytest.approx(m2, rel=1e-12)
    assert rr * (ur - S) ** 2 + pr == pytest.approx(rsr * (u - S) ** 2 + p, rel=1e-12)
    h1 = g / (g - 1) * pr / rr + 0.5 * (ur - S) ** 2
    h2 = g / (g - 1) * p / rsr + 0.5 * (u - S) ** 2
    assert h1 == pytest.approx(h2, rel=1e-12)
    # left rarefaction: entropy and the left-going Riemann invariant
    assert pl / rl ** g == pytest.approx(p / rsl ** g, rel=1e-12)
    cl, csl = math.sqrt(g * pl / rl), math.sqrt(g * p / rsl)
    assert ul + 2 * cl / (g - 1) == pytest.approx(u + 2 * csl / (g - 1), rel=1e-12)


# ---------------------------------------------------------------- two-shock solver

def test_contact_only():
    P = _params()
    qL = [2.0, 0.3, 0.1, -0.2, 0.7]
    qR = [0.5, 0.3, -0.4, 0.6, 0.7]
    F, ps, us = oracle.riemann(P, qL, qR)
    assert ps == pytest.approx(0.7, rel=4e-16)
    assert us == pytest.approx(0.3, rel=4e-16)
    # upwind (left) density and tangential velocities are carried
    assert F[0] == pytest.approx(2.0 * 0.3, rel=1e-15)
    assert F[2] == pytest.approx(2.0 * 0.3 * 0.1, rel=1e-15)
    assert F[3] == pytest.approx(2.0 * 0.3 * -0.2, rel=1e-15)
    assert F[6] == pytest.approx(0.3, rel=1e-15) and F[7] == pytest.approx(0.7, rel=1e-15)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
@pytest.mark.parametrize("U", [0.1, 1.0, 5.0])
def test_symmetric_collision_closed_form(gamma, U):
    """u_L = -u_R = U: two shocks, u* = 0 and p* is the root of
    (p - p0) = U W(p), W = C sqrt(1 + K (p - p0)/p0): a quadratic."""
    rho, p0 = 1.3, 0.8
    P = _params(gamma)
    F, ps, us = oracle.riemann(P, [rho, U, 0, 0, p0], [rho, -U, 0, 0, p0])
    C = rho * math.sqrt(gamma * p0 / rho)
    K = (gamma + 1) / (2 * gamma)
    b = U * U * C * C * K / p0
    x = 0.5 * (b + math.sqrt(b * b + 4 * U * U * C * C))
    assert us == 0.0
    assert ps == pytest.approx(p0 + x, rel=1e-13)
    # the same problem is two exact shocks, so the exact solver agrees
    pe, ue = ER.star_state(rho, U, p0, rho, -U, p0, gamma)
    assert ps == pytest.approx(pe, rel=1e-12)


def test_weak_waves_agree_with_exact_solver_to_third_order():
    P = _params(5.0 / 3.0)
    rng = np.random.default_rng(3)
    for eps in (1e-2, 1e-3):
        for _ in range(10):
            rl, rr = 1 + eps * rng.normal(size=2)
            pl, pr = 0.6 * (1 + eps * rng.normal(size=2))
            ul, ur = eps * rng.normal(size=2)
            _, ps, us = oracle.riemann(P, [rl, ul, 0, 0, pl], [rr, ur, 0, 0, pr])
            pe, ue = ER.star_state(rl, ul, pl, rr, ur, pr, 5.0 / 3.0)
            assert abs(ps - pe) / pe < 30 * eps ** 3
            assert abs(us - ue) < 30 * eps ** 3


def test_sod_two_shock_close_to_exact():
    P = _params(1.4)
    _, ps, us = oracle.riemann(P, [1.0, 0.0, 0, 0, 1.0], [0.125, 0.0, 0, 0, 0.1])
    pe, ue = ER.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert abs(ps - pe) / pe < 0.02
    assert abs(us - ue) / ue < 0.02


def test_galilean_shift_and_mirror():
    P = _params(5.0 / 3.0)
    rng = np.random.default_rng(4)
    for _ in range(20):
        qL = [rng.uniform(0.2, 3), rng.normal(), rng.normal(), rng.normal(), rng.uniform(0.1, 2)]
        qR = [rng.uniform(0.2, 3), rng.normal(), rng.normal(), rng.normal(), rng.uniform(0.1, 2)]
        F, ps, us = oracle.riemann(P, qL, qR)
        V = rng.normal()
        _, ps2, us2 = oracle.riemann(P, [qL[0], qL[1] + V] + qL[2:], [qR[0], qR[1] + V] + qR[2:])
        assert ps2 == pytest.approx(ps, rel=1e-11)
        assert us2 == pytest.approx(us + V, rel=1e-11, abs=1e-11)
        # mirror: swap sides and negate normal velocities
        Fm, psm, usm = oracle.riemann(P, [qR[0], -qR[1]] + qR[2:], [qL[0], -qL[1]] + qL[2:])
        assert psm == pytest.approx(ps, rel=1e-11)
        assert usm == pytest.approx(-us, rel=1e-11, abs=1e-11)
        assert Fm[0] == pytest.approx(-F[0], rel=1e-11, abs=1e-12)
        assert Fm[1] == pytest.approx(F[1], rel=1e-11, abs=1e-12)
        assert Fm[4] == pytest.approx(-F[4], rel=1e-11, abs=1e-12)


def _euler_flux(q, g):
    r, u, t1, t2, p = q
    re = p / (g - 1)
    return [r * u, r * u * u + p, r * u * t1, r * u * t2,
            u * (re + 0.5 * r * (u * u + t1 * t1 + t2 * t2) + p), u * re]


def test_supersonic_upwinding():
    g = 5.0 / 3.0
    P = _params(g)
    qL = [1.0, 3.0, 0.2, -0.1, 0.5]
    qR = [0.8, 2.9, 0.4, 0.3, 0.45]
    F, _, _ = oracle.riemann(P, qL, qR)
    assert np.allclose(F[:6], _euler_flux(qL, g), rtol=1e-13)
    qL2 = [1.0, -3.0, 0.2, -0.1, 0.5]
    qR2 = [0.8, -2.9, 0.4, 0.3, 0.45]
    F, _, _ = oracle.riemann(P, qL2, qR2)
    assert np.allclose(F[:6], _euler_flux(qR2, g), rtol=1e-13)


def test_sod_face_state_close_to_exact_sample():
    """Godunov state at x/t = 0 for Sod: the exact one lies in the left star
    region.  The two-shock solver gets u*, p* within 2%; its star density on
    the rarefaction side comes from the shock curve instead of the isentrope,
    which puts the mass flux about 5% off."""
    g = 1.4
    P = _params(g)
    F, _, _ = oracle.riemann(P, [1.0, 0.0, 0, 0, 1.0], [0.125, 0.0, 0, 0, 0.1])
    r, u, p = ER.sample(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g, [0.0])
    assert F[6] == pytest.approx(u[0], rel=0.02)
    assert F[7] == pytest.approx(p[0], rel=0.02)
    assert F[0] == pytest.approx(r[0] * u[0], rel=0.06)


def test_rarefaction_fan_interpolation_brackets():
    """Inside a transonic fan the sampled state lies between the side state
    and the star state (linear fan)."""
    g = 1.4
    P = _params(g)
    qL = [1.0, 0.75, 0, 0, 1.0]
    qR = [0.125, 0.0, 0, 0, 0.1]
    F, ps, us = oracle.riemann(P, qL, qR)
    ug, pg = F[6], F[7]
    assert min(qL[1], us) - 1e-14 <= ug <= max(qL[1], us) + 1e-14
    assert min(qL[4], ps) - 1e-14 <= pg <= max(qL[4], ps) + 1e-14
