"""Pins of the oracle's dark-matter particle-mesh step (Sec. 3.3-3.6):
cloud-in-cell deposit and interpolation, the kick-drift-kick update with the
scale-factor weights, periodic wrap, and the particle time step.

* Deposit conserves mass exactly; a particle at a cell centre lands in that
  cell, one at a cell corner splits evenly over 8 cells.
* Interpolation reproduces linear fields.
* With centred-difference g and the same weights for deposit and
  interpolation, a particle exerts no force on itself and a pair of
  particles pull on each other with opposite momenta (Sec. 3.4).
* KDK: closed forms for a uniform field at a = 1 and for free streaming
  under expansion.
* dt_dm in closed form (Sec. 3.5)."""
import math

import numpy as np
import pytest

import oracle
from paper_1301_4498_gb300 import workloads as W


def test_deposit_conserves_mass():
    n, dx = (16, 12, 20), 1.0 / 16
    x, u, m = W.dm_particles(n, dx, seed=3)
    rho = oracle.pm_deposit(n, dx, x, m)
    assert rho.sum() * dx ** 3 == pytest.approx(m.sum(), rel=1e-13)


def test_deposit_centre_and_corner():
    n, dx = (8, 8, 8), 0.5
    x = np.array([[2.5 * dx], [3.5 * dx], [4.5 * dx]])     # centre of cell (2, 3, 4)
    rho = oracle.pm_deposit(n, dx, x, np.array([2.0]))
    assert rho[4, 3, 2] == pytest.approx(2.0 / dx ** 3, rel=1e-15)
    assert np.count_nonzero(rho) == 1
    x = np.array([[3 * dx], [0.0], [5 * dx]])              # a corner, periodic in y
    rho = oracle.pm_deposit(n, dx, x, np.array([8.0]))
    nz = np.argwhere(rho > 0)
    assert len(nz) == 8
    assert np.allclose(rho[rho > 0], 1.0 / dx ** 3, rtol=1e-15)
    assert set(nz[:, 1]) == {0, 7}                          # y cells 7 and 0


def test_interpolation_reproduces_linear_fields():
    n, dx = (16, 16, 16), 0.25
    z, y, xg = np.meshgrid(*(np.arange(16) for _ in range(3)), indexing="ij")
    cx, cy, cz = (xg + 0.5) * dx, (y + 0.5) * dx, (z + 0.5) * dx
    coef = np.array([[0.3, 1.0, -2.0, 0.5], [1.0, 0.0, 0.7, -1.1], [-0.4, 0.2, 0.3, 0.9]])
    g = np.stack([c[0] + c[1] * cx + c[2] * cy + c[3] * cz for c in coef])
    rng = np.random.default_rng(1)
    x = rng.uniform(1.0 * dx, 14.5 * dx, size=(3, 50))      # away from the periodic wrap
    gp = oracle.pm_interp(n, dx, g, x)
    for c in range(3):
        exact = coef[c, 0] + coef[c, 1] * x[0] + coef[c, 2] * x[1] + coef[c, 3] * x[2]
        assert np.allclose(gp[c], exact, rtol=1e-13, atol=1e-13)


def _dm_only_g(n, dx, x, m, four_pi_G=1.0):
    lev = W.single_box_level(n[0], n[1], n[2], dx)
    gas = [np.zeros(lev.shape(0, 6))]
    rho = oracle.pm_deposit(n, dx, x, m)
    P = oracle.PoissonParams(four_pi_G=four_pi_G, tol=1e-13)
    _, _, st, g = oracle.poisson_solve(lev, P, gas, 1.0, rho_dm=rho, want_dense_g=True)
    assert st["rc"] == 0
    return g


def test_no_self_force_and_opposite_pair_forces():
    n, dx = (32, 32, 32), 1.0 / 32
    one = np.array([[0.3137], [0.5521], [0.6872]])
    g = _dm_only_g(n, dx, one, np.array([1.0]))
    self_g = oracle.pm_interp(n, dx, g, one)[:, 0]
    near = oracle.pm_interp(n, dx, g, one + np.array([[2 * dx], [0], [0]]))[:, 0]
    assert np.abs(self_g).max() <= 1e-9 * np.abs(near).max()
    two = np.array([[0.21, 0.47], [0.33, 0.61], [0.72, 0.58]])
    m = np.array([1.0, 2.5])
    g = _dm_only_g(n, dx, two, m)
    gp = oracle.pm_interp(n, dx, g, two)
    total = gp[:, 0] * m[0] + gp[:, 1] * m[1]
    assert np.abs(total).max() <= 1e-9 * np.abs(gp[:, 0] * m[0]).max()


def test_kdk_uniform_field_at_unit_scale_factor():
    n, dx, dt = (8, 8, 8), 1.0, 0.3
    gv = np.array([0.2, -0.1, 0.05])
    g = np.broadcast_to(gv[:, None, None, None], (3, 8, 8, 8)).copy()
    x0 = np.array([[1.2, 4.4], [2.7, 5.1], [3.3, 6.6]])
    u0 = np.array([[0.5, -0.2], [0.1, 0.3], [-0.4, 0.0]])
    x1, uh = oracle.pm_kick_drift(n, dx, g, x0, u0, a_old=1.0, a_half=1.0, dt=dt)
    u1 = oracle.pm_kick(n, dx, g, x1, uh, a_half=1.0, a_new=1.0, dt=dt)
    assert np.allclose(x1, x0 + u0 * dt + 0.5 * gv[:, None] * dt * dt, rtol=1e-14)
    assert np.allclose(u1, u0 + gv[:, None] * dt, rtol=1e-14, atol=1e-16)


def test_free_streaming_under_expansion_and_periodic_wrap():
    n, dx, dt = (8, 8, 8), 1.0, 0.5
    g = np.zeros((3, 8, 8, 8))
    a0, ah, a1 = 1 / 51, 1 / 50.5, 1 / 50
    x0 = np.array([[7.9], [0.05], [4.0]])
    u0 = np.array([[0.008], [-0.012], [0.0]])          # moves +0.2 and -0.3 cells: both wrap
    x1, uh = oracle.pm_kick_drift(n, dx, g, x0, u0, a_old=a0, a_half=ah, dt=dt)
    u1 = oracle.pm_kick(n, dx, g, x1, uh, a_half=ah, a_new=a1, dt=dt)
    assert np.allclose(uh, a0 * u0 / ah, rtol=1e-15)
    assert np.allclose(u1, a0 * u0 / a1, rtol=1e-14)
    free = x0 + dt / ah * (a0 * u0 / ah)
    assert np.allclose(x1, np.mod(free, 8.0), rtol=1e-14)
    assert 0.0 <= x1.min() and x1.max() < 8.0


def test_particle_time_step_closed_form():
    n, dx = (8, 8, 8), 0.5
    x = np.array([[1.0, 2.0], [1.0, 2.0], [1.0, 2.0]])
    u = np.array([[0.3, -0.9], [0.1, 0.2], [0.0, 0.4]])
    g = np.zeros((3, 8, 8, 8))
    a = 0.1
    assert oracle.pm_estdt(n, dx, g, x, u, a, 0.5) == pytest.approx(0.5 * a * dx / 0.9, rel=1e-15)
    g[1] = 4.0                                   # resting particles: only g limits dt
    dt = oracle.pm_estdt(n, dx, g, x, np.zeros_like(u), a, 0.5)
    assert dt == pytest.approx(math.sqrt(dx / 4.0), rel=1e-15)
