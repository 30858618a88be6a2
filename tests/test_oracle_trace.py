"""Pins of the oracle's characteristic tracing with reference states
(Sec. 3.2) and of its half-step comoving sources (Sec. 2.2)."""
import numpy as np
import pytest

import oracle

G53 = 5.0 / 3.0


def _line(n, rho, u, p, direction=0):
    q = np.zeros((5, n))
    q[0] = rho
    q[1 + direction] = u
    q[4] = p
    return q


def test_uniform_state_edges_equal_cell_state():
    P = oracle.OracleParams(gamma=G53)
    for d in range(3):
        q = np.zeros((5, 12))
        q[:] = np.array([1.3, 0.2, -0.3, 0.1, 0.7])[:, None]
        qm, qp, _, _ = oracle.trace_line(P, q, dtp=0.01, dx=0.05, direction=d)
        for c in range(2, 10):
            assert np.allclose(qm[:, c], q[:, c], rtol=1e-15, atol=1e-16)
            assert np.allclose(qp[:, c], q[:, c], rtol=1e-15, atol=1e-16)


def test_gravity_shifts_edge_velocity_by_half_step():
    P = oracle.OracleParams(gamma=G53)
    q = np.zeros((5, 12))
    q[:] = np.array([1.3, 0.2, -0.3, 0.1, 0.7])[:, None]
    g = np.zeros((3, 12))
    g[:] = np.array([0.5, -1.0, 2.0])[:, None]
    dtp = 0.01
    qm, qp, _, _ = oracle.trace_line(P, q, g, dtp=dtp, dx=0.05, direction=0)
    for c in range(2, 10):
        for k in range(3):
            assert qm[1 + k, c] == pytest.approx(q[1 + k, c] + 0.5 * dtp * g[k, c], rel=1e-15)
            assert qp[1 + k, c] == pytest.approx(q[1 + k, c] + 0.5 * dtp * g[k, c], rel=1e-15)
        assert qm[0, c] == q[0, c] and qm[4, c] == q[4, c]


def test_expansion_sources_on_uniform_state():
    """Over half a step the primitive comoving equations give
    dU = -(adot/a) U dt/2 and dp = -3 (gamma-1)(adot/a) p dt/2."""
    P = oracle.OracleParams(gamma=1.4)
    q = np.zeros((5, 10))
    q[:] = np.array([0.9, 0.4, -0.2, 0.3, 1.1])[:, None]
    adot = 0.004
    qm, qp, _, _ = oracle.trace_line(P, q, dtp=0.01, dx=0.05, adot=adot, direction=1)
    for c in range(2, 8):
        for s in (qm, qp):
            for k in range(3):
                assert s[1 + k, c] == pytest.approx(q[1 + k, c] * (1 - 0.5 * adot), rel=1e-14)
            assert s[4, c] == pytest.approx(q[4, c] * (1 - 1.5 * 0.4 * adot), rel=1e-14)


def test_reference_wave_amplitude_vanishes():
    """The reference state is the fastest wave's own domain-of-dependence
    average, so that wave's amplitude is identically zero (Sec. 3.2)."""
    P = oracle.OracleParams(gamma=G53)
    rng = np.random.default_rng(5)
    n = 30
    for trial in range(20):
        q = np.zeros((5, n))
        q[0] = 1 + 0.3 * rng.random(n)
        q[1] = rng.normal(scale=0.5, size=n)
        q[2] = rng.normal(size=n)
        q[3] = rng.normal(size=n)
        q[4] = 0.6 + 0.3 * rng.random(n)
        qm, qp, bm, bp = oracle.trace_line(P, q, dtp=0.01, dx=0.02, direction=0)
        c = np.sqrt(G53 * q[4] / q[0])
        for i in range(2, n - 2):
            if q[1, i] + c[i] > 0:
                assert bp[2, i] == 0.0   # beta_+ on the high face
            if q[1, i] - c[i] < 0:
                assert bm[0, i] == 0.0   # beta_- on the low face


def test_entropy_wave_traced_to_exact_advected_value():
    """Linear density profile, uniform u > 0 and p: only the entropy wave
    carries the jump, so the high-face density is the exact upstream value
    rho(x_{i+1/2} - u dt'/2)."""
    P = oracle.OracleParams(gamma=G53)
    n = 16
    x = np.arange(n, dtype=float)
    u, dtp, dx = 0.3, 0.2, 1.0
    q = _line(n, 1.0 + 0.01 * x, u, 0.6)
    qm, qp, _, _ = oracle.trace_line(P, q, dtp=dtp, dx=dx, direction=0)
    for i in range(3, n - 3):
        assert qp[0, i] == pytest.approx(1.0 + 0.01 * (i + 0.5 - u * dtp / dx / 2), rel=1e-14)
        assert qp[1, i] == pytest.approx(u, rel=1e-14) and qp[4, i] == pytest.approx(0.6, rel=1e-14)


def test_acoustic_simple_wave_linear_limit():
    """Small right-moving acoustic wave (rho, u, p) = (1, 0, p0) + eps (1, c, c^2) f(x)
    with linear f: each edge state equals f at the upstream foot of the
    u+c characteristic, to O(eps^2)."""
    P = oracle.OracleParams(gamma=G53)
    n = 16
    eps = 1e-6
    x = np.arange(n, dtype=float)
    p0 = 1.0 / G53
    f = eps * (x - 8.0)
    q = np.zeros((5, n))
    q[0] = 1.0 + f
    q[1] = f
    q[4] = p0 + f
    dtp, dx = 0.2, 1.0
    qm, qp, _, _ = oracle.trace_line(P, q, dtp=dtp, dx=dx, direction=0)
    for i in range(3, n - 3):
        foot = eps * (i + 0.5 - dtp / dx / 2 - 8.0)
        assert qp[0, i] - 1.0 == pytest.approx(foot, abs=1e-11)
        assert qp[1, i] == pytest.approx(foot, abs=1e-11)
        assert qp[4, i] - p0 == pytest.approx(foot, abs=1e-11)


def test_acoustic_wave_in_supersonic_flow():
    """Supersonic flow (u = 3c) carrying a small u-c acoustic wave: both
    acoustic families move toward the high face, the u+c one is the
    reference and the u-c one is projected with the eigenvectors, so the
    high-face state is the wave at the foot of the u-c characteristic."""
    P = oracle.OracleParams(gamma=G53)
    n = 16
    eps = 1e-6
    x = np.arange(n, dtype=float)
    p0, c, U = 1.0 / G53, 1.0, 3.0
    f = eps * (x - 8.0)
    q = np.zeros((5, n))
    q[0] = 1.0 - f      # (rho, u, p) = (1, U, p0) - f (1, -c, c^2): the u-c family
    q[1] = U + f
    q[4] = p0 - f
    dtp, dx = 0.1, 1.0
    qm, qp, _, _ = oracle.trace_line(P, q, dtp=dtp, dx=dx, direction=0)
    for i in range(3, n - 3):
        foot = eps * (i + 0.5 - (U - c) * dtp / dx / 2 - 8.0)
        assert qp[0, i] - 1.0 == pytest.approx(-foot, abs=1e-11)
        assert qp[1, i] - U == pytest.approx(foot, abs=1e-11)
        assert qp[4, i] - p0 == pytest.approx(-foot, abs=1e-11)
