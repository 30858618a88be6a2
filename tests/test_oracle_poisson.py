"""Pins of the oracle's self-gravity solve (Sec. 3.4): the periodic 7-point
Poisson equation L phi = 4 pi G / a (rho - mean rho) by multigrid V-cycles
with red-black Gauss-Seidel, and g = -grad phi by centred differences.

* A single Fourier mode is an eigenvector of the discrete Laplacian with
  eigenvalue -(4/dx^2) sum_d sin^2(pi k_d / n_d): phi and g in closed form.
* The solve stops at the stated relative residual; a warm start from the
  solution takes no cycle; V-cycles converge by a large factor each.
* The result does not depend on how the level is cut into boxes."""
import math

import numpy as np
import pytest

import oracle
from paper_1301_4498_gb300 import workloads as W


def _mode_level(n=(32, 16, 24), k=(2, 1, 3), box=None, amp=0.1):
    nx, ny, nz = n
    dx = 1.0 / nx
    if box is None:
        lev = W.single_box_level(nx, ny, nz, dx)
    else:
        lev = W.tiled_level(n[0], box, dx=dx)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    theta = 2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz)
    rho = 1.0 + amp * np.sin(theta)
    states = []
    for b in range(lev.nbox):
        arr = np.zeros(lev.shape(b, 6))
        lo, hi = lev.lo[b], lev.hi[b]
        W.valid(arr)[0] = rho[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        states.append(arr)
    return lev, states, rho, theta, dx


def test_single_mode_closed_form():
    n, k = (32, 16, 24), (2, 1, 3)
    lev, states, rho, theta, dx = _mode_level(n, k)
    a, four_pi_G = 0.5, 3.0
    P = oracle.PoissonParams(four_pi_G=four_pi_G, tol=1e-13)
    phi, grav, st = oracle.poisson_solve(lev, P, states, a)
    assert st["rc"] == 0 and st["resid"] <= 1e-13
    lam = -(4 / dx ** 2) * sum(math.sin(math.pi * k[d] / n[d]) ** 2 for d in range(3))
    f = four_pi_G / a * 0.1 * np.sin(theta)
    exact = f / lam
    phi0 = phi - phi.mean()
    assert np.abs(phi0 - exact).max() <= 1e-10 * np.abs(exact).max()
    # g_d = -(phi(+1) - phi(-1)) / (2 dx) of B sin(theta): -B cos(theta) sin(2 pi k_d / n_d) / dx
    B = four_pi_G / a * 0.1 / lam
    g = W.valid(grav[0])
    for d in range(3):
        gd = -B * np.cos(theta) * math.sin(2 * math.pi * k[d] / n[d]) / dx
        assert np.abs(g[d] - gd).max() <= 1e-9 * np.abs(gd).max()


def test_residual_tolerance_warm_start_and_convergence_rate():
    w = W.tiled_box(n=64, box=32, sigma=1.0, seed=5, nsteps=1)
    P = oracle.PoissonParams(tol=1e-12)
    phi, _, st = oracle.poisson_solve(w.level, P, w.state, 1 / 51)
    assert st["rc"] == 0 and st["resid"] <= 1e-12
    assert st["cycles"] <= 15
    factor = st["resid"] ** (1.0 / st["cycles"])
    assert factor < 0.2
    _, _, st2 = oracle.poisson_solve(w.level, P, w.state, 1 / 51, phi)
    assert st2["cycles"] == 0


def test_independent_of_the_box_decomposition():
    lev1, s1, _, _, _ = _mode_level(n=(32, 32, 32), k=(1, 2, 1), amp=0.3)
    lev8, s8, _, _, _ = _mode_level(n=(32, 32, 32), k=(1, 2, 1), box=16, amp=0.3)
    P = oracle.PoissonParams()
    phi1, g1, _ = oracle.poisson_solve(lev1, P, s1, 1.0)
    phi8, g8, _ = oracle.poisson_solve(lev8, P, s8, 1.0)
    assert np.array_equal(phi1, phi8)
    for b in range(lev8.nbox):
        lo, hi = lev8.lo[b], lev8.hi[b]
        ref = W.valid(g1[0])[:, lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        assert np.array_equal(W.valid(g8[b]), ref)


def test_rejects_levels_it_cannot_solve():
    lev, s, _, _, _ = _mode_level(n=(16, 16, 16), k=(1, 1, 1))
    P = oracle.PoissonParams()
    out = W.single_box_level(16, 16, 16, 1 / 16, bc=(1, 0, 0, 1, 0, 0))
    with pytest.raises(ValueError):
        oracle.poisson_solve(out, P, s, 1.0)
    part = W.tiled_level(32, 16, dx=1 / 32).subset([0, 1])     # does not tile the domain
    with pytest.raises(ValueError):
        oracle.poisson_solve(part, P, [np.zeros(part.shape(b, 6)) for b in range(2)], 1.0)
