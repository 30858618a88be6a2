"""Pins of the scheme variants Sec. 3.2 names besides PPM and the two-shock
solver: unsplit PLM with the same reference-state tracing, and the
linearised approximate Riemann solver.

* PLM: the profile is linear with the MC-limited slope d of the cell, so on
  a monotone quadratic s_i = alpha + beta i + gamma i^2 (limiter inactive,
  d = beta + 2 gamma i) the density advected to the high face by a uniform
  flow u > 0 is s_i + (1 - sigma_0) d / 2 with sigma_0 = u dt/dx, and the
  low-face state is the reference s_i - (1 - sigma_-) d / 2 (the only wave
  toward it is the reference wave u - c).  PPM differs there by the
  curvature.  The scheme stays second order on a smooth sound wave.
* Linearised solver: exact for a lone contact; p* = p + rho c du for a
  symmetric collision; its error against the exact solver is second order
  in the wave strength; supersonic upwinding; a Sod run within a measured
  gate of the exact solution."""
import math

import numpy as np
import pytest

import exact_riemann as ER
import oracle
from paper_1301_4498_gb300 import workloads as W


def _trace_quadratic(reconstruction, u=0.3, dtdx=0.8):
    n = 12
    i = np.arange(n, dtype=np.float64)
    alpha, beta, gamma_ = 1.0, 0.05, 0.001
    rho = alpha + beta * i + gamma_ * i * i
    q5 = np.zeros((5, n))
    q5[0] = rho
    q5[1] = u
    q5[4] = 1.0                              # uniform pressure
    P = oracle.OracleParams(gamma=5.0 / 3.0, reconstruction=reconstruction)
    qm, qp, _, _ = oracle.trace_line(P, q5, None, dtp=dtdx, dx=1.0, direction=0)
    return i, rho, beta, gamma_, qm, qp, q5


def test_plm_traced_density_closed_form():
    u, dtdx = 0.3, 0.8
    i, rho, beta, gamma_, qm, qp, q5 = _trace_quadratic(1, u=u, dtdx=dtdx)
    gam = 5.0 / 3.0
    for k in range(2, len(i) - 2):
        d = beta + 2 * gamma_ * i[k]
        c = math.sqrt(gam * q5[4, k] / rho[k])
        sig0 = u * dtdx
        sigm = abs(u - c) * dtdx
        assert qp[0, k] == pytest.approx(rho[k] + 0.5 * (1 - sig0) * d, rel=1e-14)
        assert qm[0, k] == pytest.approx(rho[k] - 0.5 * (1 - sigm) * d, rel=1e-14)
        assert qp[1, k] == pytest.approx(u, rel=1e-14) and qm[1, k] == pytest.approx(u, rel=1e-14)


def test_ppm_differs_from_plm_by_the_curvature():
    _, _, _, _, _, qp_plm, _ = _trace_quadratic(1)
    _, _, _, _, _, qp_ppm, _ = _trace_quadratic(0)
    d = np.abs(qp_ppm[0, 2:-2] - qp_plm[0, 2:-2])
    assert d.min() > 1e-6


def _wave_error(n, reconstruction, riemann_solver=0):
    w = W.sound_wave(n, direction=(1, 0, 0))
    P = oracle.OracleParams(gamma=5.0 / 3.0, cfl=0.4, reconstruction=reconstruction,
                            riemann_solver=riemann_solver)
    dt0 = oracle.estdt(w.level, P, w.state, 1.0)
    nsteps = int(math.ceil(1.0 / dt0))
    dt = 1.0 / nsteps
    S = w.state
    for _ in range(nsteps):
        S, _, _ = oracle.advance(w.level, P, S, None, dt=dt)
    return np.abs(W.valid(S[0])[0] - W.valid(w.state[0])[0]).mean() / 1e-5


@pytest.mark.slow
@pytest.mark.parametrize("reconstruction,riemann_solver", [(1, 0), (0, 1), (1, 1)])
def test_variants_are_second_order(reconstruction, riemann_solver):
    errs = [_wave_error(n, reconstruction, riemann_solver) for n in (32, 64, 128)]
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert rates[-1] >= 1.8, (errs, rates)


def _lin(gamma=1.4):
    return oracle.OracleParams(gamma=gamma, riemann_solver=1)


def test_linearised_contact_is_exact():
    qL = np.array([1.3, 0.2, 0.1, -0.3, 0.7])
    qR = np.array([0.4, 0.2, -0.5, 0.2, 0.7])
    f, ps, us = oracle.riemann(_lin(), qL, qR)
    assert ps == pytest.approx(0.7, rel=1e-15) and us == pytest.approx(0.2, rel=1e-15)
    assert f[0] == pytest.approx(1.3 * 0.2, rel=1e-15)   # upwind (left) density


def test_linearised_symmetric_collision_closed_form():
    rho, p, du, g = 1.0, 1.0, 0.05, 1.4
    c = math.sqrt(g * p / rho)
    f, ps, us = oracle.riemann(_lin(g), np.array([rho, du, 0, 0, p]),
                               np.array([rho, -du, 0, 0, p]))
    assert ps == pytest.approx(p + rho * c * du, rel=1e-15)
    assert us == 0.0


def test_linearised_error_is_second_order_in_wave_strength():
    rho, p, g = 1.0, 1.0, 1.4
    errs = []
    for du in (0.04, 0.02, 0.01):
        _, ps, _ = oracle.riemann(_lin(g), np.array([rho, du, 0, 0, p]),
                                  np.array([rho, -du, 0, 0, p]))
        pe, _ = ER.star_state(rho, du, p, rho, -du, p, g)
        errs.append(abs(ps - pe))
    for k in range(2):
        assert 3.5 < errs[k] / errs[k + 1] < 4.5, errs


def test_linearised_supersonic_upwinding():
    qL = np.array([1.0, 3.0, 0.1, 0.2, 1.0])        # Mach ~2.5 to the right
    qR = np.array([0.8, 2.9, -0.1, 0.0, 0.9])
    f, _, _ = oracle.riemann(_lin(), qL, qR)
    r, u, t1, t2, p = qL
    assert f[0] == pytest.approx(r * u, rel=1e-14)
    assert f[1] == pytest.approx(r * u * u + p, rel=1e-14)
    assert f[2] == pytest.approx(r * u * t1, rel=1e-14)
    assert f[4] == pytest.approx(u * (p / 0.4 + 0.5 * r * (u * u + t1 * t1 + t2 * t2) + p), rel=1e-14)


def test_sod_with_the_linearised_solver():
    """Config 1 with the linearised solver and with PLM: L1(rho) per unit
    length against the exact solution within the gate (the two-shock PPM run
    measures 1.3e-3)."""
    w = W.sod()
    edges = np.arange(129) / 128.0
    for P in (oracle.OracleParams(gamma=1.4, riemann_solver=1),
              oracle.OracleParams(gamma=1.4, reconstruction=1)):
        S, dts, _ = oracle.run(w.level, P, w.state, None, None, w.nsteps)
        rho = W.valid(S[0])[0]
        re, _, _ = ER.cell_average(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, edges, 0.5, sum(dts))
        l1 = np.abs(rho[0, 0] - re).sum() / 128.0
        assert l1 <= 4e-3, (P, l1)
