"""Pins of the oracle's coarse-fine coupling (refinement ratio 2, no
subcycling): conservative limited interpolation (Sec. 4.1), fine ghost cells
from fine neighbours or the coarse level (Sec. 4.3 Step 2), reflux and
average down (Sec. 4.3 Step 8).

What pins them: closed forms (constant and linear data are reproduced
exactly), the defining properties (the 8 fine cells average to the coarse
cell; no new extrema; average down undoes interpolation; a two-level step
conserves mass, momentum and energy only with the reflux), and the reduction
to a single level when the fine level covers the whole domain."""
import numpy as np
import pytest

import oracle
from paper_1301_4498_gb300 import workloads as W

NG = 4


def _hierarchy(n=32, box=16, seed=2):
    """A periodic n^3 comoving level as (n/box)^3 boxes and five fine boxes:
    one inside a coarse box, one across a coarse box boundary, one sharing a
    face with the first, one at the periodic corner, and two separated by a
    single coarse cell."""
    w = W.tiled_box(n=n, box=box, sigma=0.6, seed=seed, nsteps=2)
    regions = [(0, (4, 4, 4), (11, 11, 11)),
               (0, (12, 20, 8), (19, 27, 15)),
               (0, (4, 12, 4), (11, 15, 11)),
               (0, (28, 0, 28), (31, 3, 31)),
               (0, (20, 4, 20), (23, 7, 23)),
               (0, (25, 4, 20), (28, 7, 23))]
    fine = W.refined_level(w.level, regions)
    return w, fine


def _filled(lev, arrays):
    out = [a.copy() for a in arrays]
    oracle.fill_ghosts(lev, out)
    return out


def _fine_empty(fine, ncomp):
    return [np.zeros(fine.shape(b, ncomp)) for b in range(fine.nbox)]


def _coarse_value(w, ci, comp):
    """Coarse value at coarse global cell ci (wrapped)."""
    lev = w.level
    n = lev.dom_hi[0] - lev.dom_lo[0] + 1
    ci = [int(ci[a]) % int(n[a]) for a in range(3)]
    for b in range(lev.nbox):
        if all(lev.lo[b][a] <= ci[a] <= lev.hi[b][a] for a in range(3)):
            return w._filled[b][comp, ci[2] - lev.lo[b][2] + NG, ci[1] - lev.lo[b][1] + NG,
                                ci[0] - lev.lo[b][0] + NG]
    raise KeyError(ci)


def test_check_rejects_bad_hierarchies():
    w, fine = _hierarchy()
    assert oracle.amr_check(w.level, fine)
    odd = W.refined_level(w.level, [(0, (4, 4, 4), (11, 11, 11))])
    odd.lo[0, 0] += 1                     # starts inside a coarse cell
    assert not oracle.amr_check(w.level, odd)
    wide = W.refined_level(w.level, [(0, (4, 4, 4), (11, 11, 11))])
    wide.dom_hi = wide.dom_hi + 2         # not twice the coarse domain
    assert not oracle.amr_check(w.level, wide)
    outflow = W.refined_level(w.level, [(0, (4, 4, 4), (11, 11, 11))])
    outflow.dom_bc = outflow.dom_bc.copy()
    outflow.dom_bc[0, 0] = 1
    assert not oracle.amr_check(w.level, outflow)


def test_interp_reproduces_constants():
    w, fine = _hierarchy()
    vals = np.array([1.3, -0.2, 0.05, 0.0, 2.5, 1.1])
    cs = [np.broadcast_to(vals[:, None, None, None], s.shape).copy() for s in w.state]
    out = oracle.amr_interp(w.level, cs, fine, _fine_empty(fine, 6), "all")
    for b, f in enumerate(out):
        assert np.array_equal(f, np.broadcast_to(vals[:, None, None, None], f.shape))


def test_interp_reproduces_linear_data():
    """u = a + b x + c y + d z (coarse cell units) away from the periodic
    wrap: MC slopes are exact, the limiter inactive, so every fine value is
    the linear function at the fine cell centre x_f = f/2 - 1/4."""
    w, fine = _hierarchy()
    lev = w.level
    coef = np.array([0.7, 0.013, -0.021, 0.008])
    cs = []
    for b in range(lev.nbox):
        shp = lev.shape(b, 1)
        z, y, x = np.meshgrid(*(np.arange(shp[a]) - NG + lev.lo[b][2 - (a - 1)] for a in (1, 2, 3)),
                              indexing="ij")
        cs.append((coef[0] + coef[1] * x + coef[2] * y + coef[3] * z)[None].astype(np.float64))
    # box 0 of the fine level (coarse cells 4..11) and its ghosts need coarse
    # cells 1..14: no wrap, so the linear data are consistent there
    out = oracle.amr_interp(lev, cs, fine, _fine_empty(fine, 1), "all")
    f0 = out[0][0]
    flo = fine.lo[0]
    kk, jj, ii = np.meshgrid(*(np.arange(f0.shape[a]) - NG + flo[2 - a] for a in range(3)),
                             indexing="ij")
    xf, yf, zf = ii / 2 - 0.25, jj / 2 - 0.25, kk / 2 - 0.25
    exact = coef[0] + coef[1] * xf + coef[2] * yf + coef[3] * zf
    assert np.max(np.abs(f0 - exact)) <= 1e-14


def _coarse_cells_of_fine_box(fine, b):
    lo = (fine.lo[b] - fine.dom_lo[0]) // 2
    hi = (fine.hi[b] + 1 - fine.dom_lo[0]) // 2 - 1
    return lo, hi


def test_interp_is_conservative_and_makes_no_new_extrema():
    w, fine = _hierarchy()
    lev = w.level
    cs = _filled(lev, w.state)
    w._filled = cs
    out = oracle.amr_interp(lev, cs, fine, _fine_empty(fine, 6), "all")
    worst_mean, worst_ext = 0.0, 0.0
    for b in range(fine.nbox):
        f = W.valid(out[b])
        lo, hi = _coarse_cells_of_fine_box(fine, b)
        for K in range(hi[2] - lo[2] + 1):
            for J in range(hi[1] - lo[1] + 1):
                for I in range(0, hi[0] - lo[0] + 1, 3):
                    blk = f[:, 2 * K:2 * K + 2, 2 * J:2 * J + 2, 2 * I:2 * I + 2].reshape(6, 8)
                    ci = (lo[0] + I, lo[1] + J, lo[2] + K)
                    for c in range(6):
                        uc = _coarse_value(w, ci, c)
                        nb = [uc] + [_coarse_value(w, tuple(ci[a] + (s if a == d else 0)
                                                            for a in range(3)), c)
                                     for d in range(3) for s in (-1, 1)]
                        lo_v, hi_v = min(nb), max(nb)
                        span = max(hi_v - lo_v, 1e-300)
                        # rounding of uc + alpha (...) is relative to |uc| + the slopes
                        scale = abs(uc) + span
                        worst_mean = max(worst_mean, abs(blk[c].mean() - uc) / scale)
                        ext = max(lo_v - blk[c].min(), blk[c].max() - hi_v, 0.0) / span
                        worst_ext = max(worst_ext, ext)
    assert worst_mean <= 1e-15
    assert worst_ext <= 1e-14


def test_average_down_undoes_interpolation():
    w, fine = _hierarchy()
    lev = w.level
    cs = _filled(lev, w.state)
    fs = oracle.amr_interp(lev, cs, fine, _fine_empty(fine, 6), "all")
    back = oracle.amr_average_down(lev, cs, fine, fs)
    covered = 0
    for b in range(lev.nbox):
        d = np.abs(W.valid(back[b]) - W.valid(cs[b]))
        scale = np.abs(W.valid(cs[b])).max(axis=(1, 2, 3))[:, None, None, None]
        assert np.all(d <= 1e-15 * scale)
        covered += int(np.count_nonzero(np.any(W.valid(back[b]) != W.valid(cs[b]), axis=0)))
    # uncovered coarse cells are untouched: only cells under the fine level may differ
    nfine_coarse = sum(int(np.prod((fine.hi[b] - fine.lo[b] + 1) // 2)) for b in range(fine.nbox))
    assert covered <= nfine_coarse


def test_fine_ghosts_take_fine_neighbours_first():
    """Ghost cells inside another fine box copy its valid cell exactly; the
    others are the coarse interpolation."""
    w, fine = _hierarchy()
    lev = w.level
    cs = _filled(lev, w.state)
    base = oracle.amr_interp(lev, cs, fine, _fine_empty(fine, 6), "all")
    rng = np.random.default_rng(4)
    pert = []
    for b in range(fine.nbox):                       # fine data != interpolation
        a = base[b].copy()
        W.valid(a)[...] *= 1.0 + 0.01 * rng.standard_normal(W.valid(a).shape)
        pert.append(a)
    got = oracle.amr_interp(lev, cs, fine, pert, "ghosts")
    # box 0 is coarse 4..11 (fine 8..23); box 2 is coarse y 12..15 (fine y 24..31)
    g0 = got[0]
    nx = fine.hi[0][0] - fine.lo[0][0] + 1
    # ghost layer y = 16..19 (fine global y 24..27) lies in box 2's valid cells
    ghost = g0[:, NG:NG + nx, NG + 16:NG + 20, NG:NG + nx]
    src = pert[2][:, NG:NG + nx, NG:NG + 4, NG:NG + nx]
    assert np.array_equal(ghost, src)
    # ghost layer y = -4..-1 is uncovered: interpolated
    assert np.array_equal(g0[:, :, 0:NG, :], base[0][:, :, 0:NG, :])
    # valid cells are left alone
    assert np.array_equal(W.valid(got[0]), W.valid(pert[0]))


def _two_level_state(w, fine, pert=0.02, seed=9):
    """Coarse state of the workload, fine state interpolated from it and
    perturbed cell by cell (seeded factors), coarse cells under the fine
    level averaged down: a composite state whose coarse level holds its
    totals."""
    lev = w.level
    cs = _filled(lev, w.state)
    fs = oracle.amr_interp(lev, cs, fine, _fine_empty(fine, 6), "all")
    fs = W.scale_valid(fs, W.cell_factors(fine, seed, pert))
    cs = oracle.amr_average_down(lev, cs, fine, fs)
    return cs, fs


def _totals(lev, states):
    vol = np.prod(lev.dx, axis=1)
    return np.array([sum(W.valid(s)[c].sum() * vol[b] for b, s in enumerate(states))
                     for c in range(5)])


@pytest.mark.parametrize("reflux", [True, False])
def test_two_level_step_conserves_only_with_reflux(reflux):
    """Periodic, a constant, g = 0, no dual-energy switch: after reflux and
    average down the coarse level holds the composite solution, whose
    totals of rho, m and rho E are conserved to round-off (Sec. 4.3 Step 8).
    Without the reflux the mass is not conserved."""
    w, fine = _hierarchy()
    P = oracle.OracleParams(gamma=5.0 / 3.0, dual_energy_sync=0)
    cs, fs = _two_level_state(w, fine)
    before = _totals(w.level, cs)
    dt = 0.5 * oracle.amr_estdt(w.level, fine, P, cs, fs, 1.0)
    cn, fn, _, _ = oracle.amr_step(w.level, fine, P, cs, fs, a_old=1.0, a_new=1.0, dt=dt,
                                   reflux=reflux)
    after = _totals(w.level, cn)
    scale = np.array([before[0], 1.0, 1.0, 1.0, before[4]]) * 1.0
    scale[1:4] = np.abs(before[0]) * 0.1         # momentum: rms |U| = 0.1 c
    rel = np.abs(after - before) / scale
    if reflux:
        assert np.all(rel <= 2e-14), rel
    else:
        assert rel[0] > 1e-9, rel


def test_reflux_is_zero_for_uniform_flow():
    w, fine = _hierarchy()
    P = oracle.OracleParams(gamma=5.0 / 3.0)
    S0 = np.array([1.1, 0.11, -0.055, 0.033, 0.0, 1.0])
    S0[4] = S0[5] + 0.5 * (S0[1] ** 2 + S0[2] ** 2 + S0[3] ** 2) / S0[0]
    cs = [np.broadcast_to(S0[:, None, None, None], s.shape).copy() for s in w.state]
    fs = oracle.amr_interp(w.level, cs, fine, _fine_empty(fine, 6), "all")
    dt = 1e-3
    a, _, _, _ = oracle.amr_step(w.level, fine, P, cs, fs, a_old=1.0, a_new=1.0, dt=dt)
    b, _, _, _ = oracle.amr_step(w.level, fine, P, cs, fs, a_old=1.0, a_new=1.0, dt=dt,
                                 reflux=False)
    for x, y in zip(a, b):
        assert np.allclose(W.valid(x), W.valid(y), rtol=1e-14, atol=0)
        assert np.allclose(W.valid(x), S0[:, None, None, None], rtol=1e-13, atol=1e-16)


def test_full_refinement_reduces_to_the_fine_level():
    """A fine level covering the whole domain: its step is exactly the
    single-level advance of that level, and the coarse level becomes its
    average."""
    w = W.tiled_box(n=16, box=8, sigma=0.5, seed=6, nsteps=1)
    fine = W.refine_boxes(w.level, range(w.level.nbox))
    P = oracle.OracleParams(gamma=5.0 / 3.0)
    cs, fs = _two_level_state(w, fine, pert=0.01)
    a0, a1 = 1 / 51, 1 / 50
    dt = oracle.amr_estdt(w.level, fine, P, cs, fs, a0)
    cn, fn, _, _ = oracle.amr_step(w.level, fine, P, cs, fs, a_old=a0, a_new=a1, dt=dt)
    ref, _, _ = oracle.advance(fine, P, fs, None, a_old=a0, a_new=a1, dt=dt)
    for x, y in zip(fn, ref):
        assert np.array_equal(W.valid(x), W.valid(y))
    avg = oracle.amr_average_down(w.level, cn, fine, ref)
    for x, y in zip(cn, avg):
        assert np.array_equal(W.valid(x), W.valid(y))
