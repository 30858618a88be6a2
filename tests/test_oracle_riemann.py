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


def _fan_scan(P, qL, qR, xi):
    """Godunov state at x/t = xi of the problem (qL, qR): the problem seen
    from a frame moving at xi (both normal velocities shifted by -xi),
    sampled at x/t = 0, with the frame velocity added back."""
    out = []
    for x in xi:
        g = oracle.riemann_state(P, [qL[0], qL[1] - x] + list(qL[2:]), [qR[0], qR[1] - x] + list(qR[2:]))
        out.append([g[0], g[1] + x, g[4]])
    return np.array(out)


def test_transonic_rarefaction_fan_is_continuous_and_linear():
    """Sec. 3.2's two-shock solver samples a rarefaction with a linear fan
    (Colella & Glaz 1985): between the head (speed u_o - c_o) and the tail
    (u* - c*) the sampled state is linear in x/t, and it meets the side state
    at the head and the star state at the tail, so the whole self-similar
    profile is continuous across both edges of the fan.  Scanning the
    profile through Galilean shifts tests exactly that; a weight measured
    from the wrong edge (w <-> 1 - w) puts a jump of the whole wave strength
    at both edges."""
    g = 1.4
    P = _params(g)
    qL = [1.0, 0.0, 0.0, 0.0, 1.0]
    qR = [0.125, 0.0, 0.0, 0.0, 0.1]
    _, ps, us = oracle.riemann(P, qL, qR)
    cL = math.sqrt(g * qL[4] / qL[0])
    head = qL[1] - cL
    # from left of the head to just left of the contact (left side sampled)
    d = 2.0 ** -12
    xi = head - 0.25 + d * np.arange(int((us - 0.05 - (head - 0.25)) / d))
    prof = _fan_scan(P, qL, qR, xi)
    # the left state before the head, the star state (p*, u*) before the contact
    assert np.all(prof[xi < head - d] == np.array([qL[0], qL[1], qL[4]]))
    assert prof[-1][2] == pytest.approx(ps, rel=1e-14)
    assert prof[-1][1] == pytest.approx(us, rel=1e-14)
    # continuity: no step larger than the fan's slope allows
    span = np.abs(prof[-1] - prof[0])
    assert np.all(np.abs(np.diff(prof, axis=0)) <= 2e-3 * span)
    # inside the fan (strictly between both edge states, with both neighbours)
    # the profile is linear in x/t: vanishing second differences
    tail = float(xi[np.argmax(np.all(np.abs(prof - prof[-1]) <= 1e-13 * span, axis=1))])
    assert head < tail < us
    inner = (xi > head + 2 * d) & (xi < tail - 2 * d)
    assert inner.sum() > 100
    dd = np.abs(prof[2:] - 2 * prof[1:-1] + prof[:-2])[inner[1:-1]]
    assert np.all(dd <= 1e-12 * span)
    # the slopes are the wave strengths over the fan's width (tail - head)
    slope = (prof[-1] - prof[0]) / (tail - head)
    mid = np.flatnonzero(inner)[len(np.flatnonzero(inner)) // 2]
    assert (prof[mid + 1] - prof[mid]) / d == pytest.approx(slope, rel=2e-2)


def test_stationary_contact_face_takes_the_mean_of_both_sides():
    """u* = 0 exactly (a contact at rest, equal pressures, different
    densities and tangential velocities): the face sits on the contact, and
    the reading of Sec. 3.2's solver takes the arithmetic mean of the two
    sides' samples.  Every value here is exact in binary.  The choice enters
    no flux, because each flux but F_mn = p* carries a factor u_g = 0."""
    P = _params(5.0 / 3.0)
    qL = [2.0, 0.0, 0.25, -0.5, 1.0]
    qR = [0.5, 0.0, 0.75, 0.5, 1.0]
    F, ps, us = oracle.riemann(P, qL, qR)
    assert us == 0.0 and ps == 1.0
    g = oracle.riemann_state(P, qL, qR)
    assert list(g) == [1.25, 0.0, 0.5, 0.0, 1.0]
    assert list(F) == [0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]
    # mirrored problem: the same mean
    gm = oracle.riemann_state(P, [qR[0], -0.0] + qR[2:], [qL[0], -0.0] + qL[2:])
    assert list(gm) == [1.25, 0.0, 0.5, 0.0, 1.0]
