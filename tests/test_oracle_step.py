"""Whole-step pins of the oracle: closed forms, conservation, symmetry, the
exact Sod solution, second-order convergence, the CFL step, ghost fill and
box decomposition (Sec. 2.2, 3.2, 3.5, 3.6, 4.1)."""
import math

import numpy as np
import pytest

import exact_riemann as ER
import oracle
from paper_1301_4498_gb300 import workloads as W

G53 = 5.0 / 3.0


def _one_step(w, P, dt, a_old=1.0, a_new=1.0, **kw):
    S, st, fl = oracle.advance(w.level, P, w.state, w.grav, a_old=a_old, a_new=a_new, dt=dt, **kw)
    return S, st, fl


def test_uniform_state_under_expansion():
    """gamma = 5/3: rho unchanged, m scales by a_old/a_new, rho e and rho E by
    (a_old/a_new)^2 (Sec. 2.2 with a uniform state)."""
    rho, u, e = 1.2, np.array([0.1, -0.05, 0.02]), 0.9
    S0 = W.conserved_from_primitive(np.array([[[rho]]]), u[:, None, None, None],
                                    np.array([[[rho * e]]]))[:, 0, 0, 0]
    w = W.uniform_level(S0, n=(8, 8, 8), dx=1 / 8)
    P = oracle.OracleParams(gamma=G53)
    a0, a1 = 1 / 51, 1 / 50
    S, st, _ = _one_step(w, P, dt=1e-3, a_old=a0, a_new=a1)
    v = W.valid(S[0])
    r = a0 / a1
    assert np.allclose(v[0], rho, rtol=1e-14)
    for c in range(3):
        assert np.allclose(v[1 + c], S0[1 + c] * r, rtol=1e-13)
    assert np.allclose(v[4], S0[4] * r * r, rtol=1e-13)
    assert np.allclose(v[5], S0[5] * r * r, rtol=1e-13)


def test_uniform_gravity_at_rest():
    """a = 1, uniform g: m = rho g dt, rho E gains rho |g|^2 dt^2 / 2, rho e
    unchanged (energy option (i) with the corrector, Sec. 3.2 / Step 6)."""
    rho, e = 0.8, 0.9
    g = np.array([0.3, -0.2, 0.1])
    S0 = np.array([rho, 0, 0, 0, rho * e, rho * e])
    w = W.uniform_level(S0, n=(8, 8, 8), dx=1 / 8, grav=g)
    P = oracle.OracleParams(gamma=G53)
    dt = 0.01
    S, st, _ = _one_step(w, P, dt=dt)
    v = W.valid(S[0])
    assert np.allclose(v[0], rho, rtol=1e-14)
    for c in range(3):
        assert np.allclose(v[1 + c], rho * g[c] * dt, rtol=1e-12)
    assert np.allclose(v[4], rho * e + 0.5 * rho * (g @ g) * dt * dt, rtol=1e-14)
    assert np.allclose(v[5], rho * e, rtol=1e-12)


def test_expansion_cooling_term_kappa():
    """gamma = 1.4 (kappa = 2 - 3(gamma-1) = 0.8 != 0): on a uniform state at
    rest a^2 rho e grows like a^kappa, so rho e ~ a^{-3(gamma-1)}; one step
    reproduces this to O((da/a)^2)."""
    rho, e = 1.0, 2.0
    S0 = np.array([rho, 0, 0, 0, rho * e, rho * e])
    w = W.uniform_level(S0, n=(8, 8, 8), dx=1 / 8)
    w.gamma = 1.4
    P = oracle.OracleParams(gamma=1.4)
    a0 = 0.5
    for eps in (1e-2, 1e-3):
        a1 = a0 * (1 + eps)
        S, _, _ = _one_step(w, P, dt=1e-3, a_old=a0, a_new=a1)
        got = W.valid(S[0])[5].mean() / (rho * e)
        exact = (a0 / a1) ** (3 * 0.4)
        assert abs(got - exact) < 1.0 * eps * eps
        # without the term the error would be first order
        assert abs((a0 / a1) ** 2 - exact) > 0.5 * eps


def test_conservation_periodic():
    """a constant, g = 0, no sync: sums of rho, m, rho E are conserved to
    round-off (the flux form telescopes over a periodic box)."""
    w = W.comoving_box(n=16, sigma=0.5, seed=11, nsteps=3, a0=1.0, aN=1.0)
    P = oracle.OracleParams(gamma=G53, dual_energy_sync=0)
    S = w.state
    s0 = W.valid(S[0])[:5].reshape(5, -1).sum(axis=1)
    for _ in range(3):
        dt = oracle.estdt(w.level, P, S, 1.0)
        S, st, _ = oracle.advance(w.level, P, S, None, dt=dt)
    s1 = W.valid(S[0])[:5].reshape(5, -1).sum(axis=1)
    scale = np.abs(W.valid(w.state[0])[:5]).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale)


def test_conservation_with_expansion():
    """g = 0 with a varying: sum rho and sum a m are conserved (Sec. 2.2
    continuity and momentum equations in flux form)."""
    w = W.comoving_box(n=16, sigma=0.5, seed=12, nsteps=2)
    P = oracle.OracleParams(gamma=G53)
    S = w.state
    a = w.a_sched
    m0 = a[0] * W.valid(S[0])[1:4].reshape(3, -1).sum(axis=1)
    r0 = W.valid(S[0])[0].sum()
    for s in range(2):
        dt = oracle.estdt(w.level, P, S, a[s])
        S, _, _ = oracle.advance(w.level, P, S, None, a_old=a[s], a_new=a[s + 1], dt=dt)
    m1 = a[2] * W.valid(S[0])[1:4].reshape(3, -1).sum(axis=1)
    mscale = a[0] * np.abs(W.valid(w.state[0])[1:4]).reshape(3, -1).sum(axis=1)
    assert np.all(np.abs(m1 - m0) <= 1e-13 * mscale)
    assert abs(W.valid(S[0])[0].sum() - r0) <= 1e-13 * r0


def _mirror_x(arr, signs):
    out = arr[:, :, :, ::-1].copy()
    for c, s in enumerate(signs):
        out[c] *= s
    return out


def test_mirror_symmetry_x():
    w = W.comoving_box(n=16, sigma=0.5, seed=13, nsteps=1)
    P = oracle.OracleParams(gamma=G53)
    a = w.a_sched
    dt = oracle.estdt(w.level, P, w.state, a[0])
    S, _, _ = oracle.advance(w.level, P, w.state, w.grav, a_old=a[0], a_new=a[1], dt=dt)
    sgn = [1, -1, 1, 1, 1, 1]
    Sm_in = [_mirror_x(w.state[0], sgn)]
    Gm = [_mirror_x(w.grav[0], [-1, 1, 1])]
    Sm, _, _ = oracle.advance(w.level, P, Sm_in, Gm, a_old=a[0], a_new=a[1], dt=dt)
    ref = W.valid(_mirror_x(S[0], sgn))
    got = W.valid(Sm[0])
    for c in range(6):
        scale = np.abs(ref[c]).max()
        assert np.abs(got[c] - ref[c]).max() <= 1e-13 * scale


def test_sod_axis_permutation():
    P = oracle.OracleParams(gamma=1.4)
    res = []
    for axis in range(3):
        w = W.sod(n=64, ny=8, nz=8, axis=axis, nsteps=5)
        S, _, _ = oracle.run(w.level, P, w.state, None, None, 5)
        v = W.valid(S[0])
        # bring the Sod axis to x and its momentum to component 1
        perm_axes = {0: (0, 1, 2, 3), 1: (0, 1, 3, 2), 2: (0, 3, 2, 1)}[axis]
        v = np.transpose(v, perm_axes)
        comp = [0, 1 + axis, 4, 5]
        res.append(v[comp])
    for r in res[1:]:
        assert np.abs(r - res[0]).max() <= 1e-13 * np.abs(res[0]).max()


def test_sod_against_exact_solution():
    """Config 1: 128 x 8 x 8, 20 steps; L1(rho) per unit length against the
    exact solution (cell averages) <= 4e-3 (measured 1.3e-3); columns
    identical, m_y = m_z = 0."""
    w = W.sod()
    P = oracle.OracleParams(gamma=1.4)
    S, dts, st = oracle.run(w.level, P, w.state, None, None, w.nsteps)
    v = W.valid(S[0])
    t = sum(dts)
    rho = v[0]
    assert np.all(rho == rho[:1, :1, :])
    assert np.all(v[2] == 0.0) and np.all(v[3] == 0.0)
    edges = np.arange(129) / 128.0
    re, ue, pe = ER.cell_average(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, edges, 0.5, t)
    l1 = np.abs(rho[0, 0] - re).sum() / 128.0
    assert l1 <= 4e-3, l1
    # mass conserved exactly up to the outflow fluxes, which are zero (no wave reaches x = 0, 1)
    assert rho[0, 0].sum() == pytest.approx(w.state[0][0, 4, 4, 4:-4].sum(), rel=1e-14)


@pytest.mark.slow
def test_sod_to_t_0p2_plateaus():
    """Oracle-only longer run: at t = 0.2 the star plateaus match the exact
    values to within 2%, the shock position within two cells."""
    w = W.sod(nsteps=1)
    P = oracle.OracleParams(gamma=1.4)
    S = w.state
    t = 0.0
    while t < 0.2 - 1e-12:
        dt = min(oracle.estdt(w.level, P, S, 1.0), 0.2 - t)
        S, _, _ = oracle.advance(w.level, P, S, None, dt=dt)
        t += dt
    v = W.valid(S[0])
    rho = v[0, 0, 0]
    x = (np.arange(128) + 0.5) / 128
    ps, us = ER.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    rsl, rsr = ER.star_densities(1.0, 1.0, 0.125, 0.1, ps, 1.4)
    xc = 0.5 + us * 0.2
    plateau_l = (x > xc - 0.08) & (x < xc - 0.03)
    assert np.allclose(rho[plateau_l], rsl, rtol=0.02)
    u = v[1, 0, 0] / rho
    mid = (x > xc - 0.05) & (x < xc + 0.05)
    assert np.allclose(u[mid], us, rtol=0.02)
    S_sh = 0.5 + 1.75216 * 0.2
    jump = x[np.argmax(-np.diff(rho) * (x[:-1] > xc + 0.02))]
    assert abs(jump - S_sh) < 2.0 / 128


def _wave_error(n, direction):
    w = W.sound_wave(n, direction=direction)
    P = oracle.OracleParams(gamma=G53, cfl=0.4)
    T = 1.0 / np.linalg.norm(direction)
    dt0 = oracle.estdt(w.level, P, w.state, 1.0)
    nsteps = int(math.ceil(T / dt0))
    dt = T / nsteps
    S = w.state
    for _ in range(nsteps):
        S, _, _ = oracle.advance(w.level, P, S, None, dt=dt)
    d = W.valid(S[0])[0] - W.valid(w.state[0])[0]
    return np.abs(d).mean() / 1e-5


@pytest.mark.slow
@pytest.mark.parametrize("direction", [(1, 0, 0), (1, 1, 0)])
def test_second_order_convergence_sound_wave(direction):
    ns = (16, 32, 64) if direction[1] else (32, 64, 128)
    errs = [_wave_error(n, direction) for n in ns]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] >= 1.8, (errs, rates)


def test_dt_closed_form_uniform():
    u = np.array([0.3, -0.7, 0.1])
    rho, e = 1.1, 0.9
    S0 = W.conserved_from_primitive(np.array([[[rho]]]), u[:, None, None, None],
                                    np.array([[[rho * e]]]))[:, 0, 0, 0]
    w = W.uniform_level(S0, n=(8, 8, 8), dx=0.125)
    P = oracle.OracleParams(gamma=G53, cfl=0.5)
    a = 0.03
    c = math.sqrt(G53 * (G53 - 1) * e)
    expected = 0.5 * a * 0.125 / (np.abs(u).max() + c)
    assert oracle.estdt(w.level, P, w.state, a) == pytest.approx(expected, rel=1e-14)


def test_ghost_fill_periodic_outflow_and_tiles():
    rng = np.random.default_rng(7)
    # periodic single box == wrap padding
    lev = W.single_box_level(8, 6, 10, 0.1)
    arr = W.empty_box(lev, 0, 2)
    val = rng.normal(size=(2, 10, 6, 8))
    W.put_valid(arr, val)
    oracle.fill_ghosts(lev, [arr])
    assert np.array_equal(arr, np.pad(val, ((0, 0), (4, 4), (4, 4), (4, 4)), mode="wrap"))
    # outflow in x, periodic in y/z == edge padding in x after wrap in y/z
    lev = W.single_box_level(8, 6, 10, 0.1, bc=(1, 0, 0, 1, 0, 0))
    arr = W.empty_box(lev, 0, 1)
    val = rng.normal(size=(1, 10, 6, 8))
    W.put_valid(arr, val)
    oracle.fill_ghosts(lev, [arr])
    ref = np.pad(val, ((0, 0), (4, 4), (4, 4), (0, 0)), mode="wrap")
    ref = np.pad(ref, ((0, 0), (0, 0), (0, 0), (4, 4)), mode="edge")
    assert np.array_equal(arr, ref)
    # tiled periodic domain == wrap padding of the assembled domain
    lev = W.tiled_level(16, 8)
    full = rng.normal(size=(1, 16, 16, 16))
    arrs = []
    for b in range(lev.nbox):
        i0, j0, k0 = lev.lo[b]
        a = W.empty_box(lev, b, 1)
        W.put_valid(a, full[:, k0:k0 + 8, j0:j0 + 8, i0:i0 + 8])
        arrs.append(a)
    oracle.fill_ghosts(lev, arrs)
    padded = np.pad(full, ((0, 0), (4, 4), (4, 4), (4, 4)), mode="wrap")
    for b in range(lev.nbox):
        i0, j0, k0 = lev.lo[b]
        assert np.array_equal(arrs[b], padded[:, k0:k0 + 16, j0:j0 + 16, i0:i0 + 16])


def test_box_decomposition_is_exact():
    """A periodic 32^3 field advanced as one box or as 8 boxes of 16^3 with
    neighbour ghost fill gives bitwise identical valid cells."""
    w1 = W.comoving_box(n=32, sigma=0.5, seed=21, nsteps=1)
    w8 = W.tiled_box(n=32, box=16, sigma=0.5, seed=21, nsteps=1)
    P = oracle.OracleParams(gamma=G53)
    a = w1.a_sched
    dt = oracle.estdt(w1.level, P, w1.state, a[0])
    assert oracle.estdt(w8.level, P, w8.state, a[0]) == dt
    S1, _, _ = oracle.advance(w1.level, P, w1.state, w1.grav, a_old=a[0], a_new=a[1], dt=dt)
    S8, _, _ = oracle.advance(w8.level, P, w8.state, w8.grav, a_old=a[0], a_new=a[1], dt=dt)
    full = W.valid(S1[0])
    for b in range(w8.level.nbox):
        i0, j0, k0 = w8.level.lo[b]
        assert np.array_equal(W.valid(S8[b]), full[:, k0:k0 + 16, j0:j0 + 16, i0:i0 + 16])


def test_flux_export_reproduces_density_update():
    w = W.comoving_box(n=16, sigma=0.5, seed=31, nsteps=1)
    P = oracle.OracleParams(gamma=G53)
    a = w.a_sched
    dt = oracle.estdt(w.level, P, w.state, a[0])
    S, _, fl = oracle.advance(w.level, P, w.state, w.grav, a_old=a[0], a_new=a[1], dt=dt,
                              want_flux=True)
    F = fl[0]
    div = ((F[0][0][:, :, 1:] - F[0][0][:, :, :-1]) * 16 + (F[1][0][:, 1:, :] - F[1][0][:, :-1, :]) * 16
           + (F[2][0][1:] - F[2][0][:-1]) * 16)
    dtp = dt / (0.5 * (a[0] + a[1]))
    rho0 = W.valid(w.state[0])[0]
    assert np.allclose(W.valid(S[0])[0], rho0 - dtp * div, rtol=1e-13)
    # periodic: the flux on the last face equals the one on the first
    assert np.array_equal(F[0][0][:, :, 0], F[0][0][:, :, -1])


def test_internal_energy_tracks_total_minus_kinetic():
    """Sync off, a = 1, smooth compressive flow: the separately evolved rho e
    (with its -p div U term, Sec. 2.2) stays within truncation error of
    rho E - rho U^2/2; without the p div U term it would drift by
    O(dt p div U) per step."""
    w = W.comoving_box(n=32, sigma=0.3, seed=41, nsteps=4, a0=1.0, aN=1.0)
    # a strong converging velocity field makes p div U large
    v = W.valid(w.state[0])
    rho = v[0]
    x = (np.arange(32) + 0.5) / 32
    ux = -0.5 * np.sin(2 * np.pi * x)[None, None, :] * np.ones_like(rho)
    rhoe = v[5]
    v[:] = W.conserved_from_primitive(rho, np.stack([ux, 0 * ux, 0 * ux]), rhoe)
    P = oracle.OracleParams(gamma=G53, dual_energy_sync=0)
    S = w.state
    for _ in range(4):
        dt = oracle.estdt(w.level, P, S, 1.0)
        S, _, _ = oracle.advance(w.level, P, S, None, dt=dt)
    vv = W.valid(S[0])
    ke = 0.5 * (vv[1] ** 2 + vv[2] ** 2 + vv[3] ** 2) / vv[0]
    e_from_E = vv[4] - ke
    drift = np.abs(vv[5] - e_from_E).max() / np.abs(e_from_E).max()
    change = np.abs(vv[5] - rhoe).max() / np.abs(rhoe).max()
    # measured: rho e changes by ~66% while the drift stays ~2%; with the
    # p div U term removed from the rho e update the drift is ~53%
    assert change > 0.2
    assert drift < 0.05


@pytest.mark.parametrize("frac,keeps_e", [(5e-5, True), (0.5, False)])
def test_dual_energy_switch_direction(frac, keeps_e):
    """Step 6 sync on a uniform moving state (no fluxes act): where
    rhoE - KE > 1e-4 rhoE the internal energy is re-derived from E, else E is
    re-derived from the evolved e.  rho e is deliberately inconsistent with
    rho E - KE on input, so the branch taken shows in the output."""
    rho, u = 1.0, np.array([2.0, 0.0, 0.0])
    ke = 0.5 * rho * (u @ u)
    rhoE = ke / (1.0 - frac)          # (rhoE - KE)/rhoE = frac
    rhoe = 0.3 * (rhoE - ke)          # evolved e, not equal to E - KE
    S0 = np.array([rho, rho * u[0], 0.0, 0.0, rhoE, rhoe])
    w = W.uniform_level(S0, n=(8, 8, 8), dx=1 / 8)
    P = oracle.OracleParams(gamma=G53)
    S, st, _ = _one_step(w, P, dt=1e-3)
    v = W.valid(S[0])
    if keeps_e:
        assert np.allclose(v[5], rhoe, rtol=1e-12)
        assert np.allclose(v[4], rhoe + ke, rtol=1e-12)
    else:
        assert np.allclose(v[4], rhoE, rtol=1e-12)
        assert np.allclose(v[5], rhoE - ke, rtol=1e-9)


def test_trilinear_advection_exact():
    """Uniform velocity and pressure: the Euler equations reduce to linear
    advection of rho.  For a trilinear density field the fully corner-coupled
    scheme (theta = 1/3 for the singly corrected states, 1/2 for the final
    ones) transports it exactly: cells beyond the stencil's reach of the
    outflow boundary match rho(x - U dt) to round-off."""
    n = 16
    lev = W.single_box_level(n, n, n, 1.0 / n, bc=(1, 1, 1, 1, 1, 1))
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    U = np.array([0.3, 0.2, 0.1])
    p0 = 1.0

    def rho_of(X, Y, Z):
        return 1.0 + 0.5 * (X - 0.5) * (Y - 0.5) * (Z - 0.5) + 0.1 * (X - 0.5) - 0.05 * (Y - 0.5)

    rho = rho_of(X, Y, Z)
    u = np.stack([np.full_like(rho, U[0]), np.full_like(rho, U[1]), np.full_like(rho, U[2])])
    S = W.empty_box(lev, 0, 6)
    W.put_valid(S, W.conserved_from_primitive(rho, u, np.full_like(rho, p0 / (G53 - 1))))
    P = oracle.OracleParams(gamma=G53)
    dt = 0.5 * (1.0 / n) / (U.max() + np.sqrt(G53 * p0 / rho.min()))
    out, _, _ = oracle.advance(lev, P, [S], None, dt=dt)
    got = W.valid(out[0])[0]
    exact = rho_of(X - U[0] * dt, Y - U[1] * dt, Z - U[2] * dt)
    inner = (slice(4, n - 4),) * 3
    assert np.abs(got[inner] - exact[inner]).max() <= 1e-13
