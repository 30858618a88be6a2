"""GPU parity of the coarse-fine coupling (nyx_amr_*) against the oracle:
interpolation, average down, the two-level step (fine ghosts, both advances,
reflux, average down), the graph-captured run and conservation.  FP64 plans
must match the oracle to 1e-12 (normwise, per field); mixed plans within the
mixed gates."""
import numpy as np
import pytest

import oracle
from gates import MIXED_GATES
from paper_1301_4498_gb300 import workloads as W

import test_oracle_amr as TA

pytestmark = pytest.mark.gpu
H = pytest.importorskip("paper_1301_4498_gb300.hydro")
torch = pytest.importorskip("torch")

NG = 4


def _norm_rel(got, ref):
    """max over fields of ||got - ref||_inf / ||ref||_inf over the valid cells."""
    worst = 0.0
    for c in range(ref[0].shape[0]):
        num = max(np.abs(W.valid(g)[c] - W.valid(r)[c]).max() for g, r in zip(got, ref))
        den = max(np.abs(W.valid(r)[c]).max() for r in ref)
        worst = max(worst, num / max(den, 1e-300))
    return worst


def _plans(w, fine, precision="fp64", **kw):
    cp = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision=precision, keep_fluxes=1, **kw)
    fp = H.Plan(fine, stream=cp.torch_stream, gamma=w.gamma, cfl=w.cfl, precision=precision,
                keep_fluxes=1, coarse_fine=1, **kw)
    return cp, fp, H.Amr(cp, fp)


def _setup(w, fine, precision="fp64", grav=True, pert=0.02, seed=9, **kw):
    """GPU two-level state made by the library alone: coarse state of the
    workload, fine state by interpolation, perturbed by the seeded cell
    factors, coarse cells under the fine level averaged down; fine gravity
    by interpolation."""
    cp, fp, amr = _plans(w, fine, precision, **kw)
    lc = H.make_level(cp, w.state, w.grav if grav else None)
    cp.fill(lc.current, 6)
    fs = fp.empty_field(6)
    amr.interp(lc.current, fs, 6, "all")
    torch.cuda.synchronize()
    if pert:
        host = W.scale_valid(fp.from_device(fs, 6), W.cell_factors(fine, seed, pert))
        fs = fp.to_device(host, 6)
        amr.average_down(fs, lc.current, 6)
    fg = None
    if grav:
        fg = fp.empty_field(3)
        amr.interp(lc.grav, fg, 3, "all")
    lf = H.Level(fs, fp.empty_field(6), fg)
    return cp, fp, amr, lc, lf


def _oracle_setup(w, fine, grav=True, pert=0.02, seed=9):
    cs = TA._filled(w.level, w.state)
    fs = oracle.amr_interp(w.level, cs, fine, TA._fine_empty(fine, 6), "all")
    if pert:
        fs = W.scale_valid(fs, W.cell_factors(fine, seed, pert))
        cs = oracle.amr_average_down(w.level, cs, fine, fs)
    cg = fg = None
    if grav:
        cg = TA._filled(w.level, w.grav)
        fg = oracle.amr_interp(w.level, cg, fine, TA._fine_empty(fine, 3), "all")
    return cs, fs, cg, fg


def test_interp_and_average_down_match_the_oracle_bitwise():
    w, fine = TA._hierarchy()
    cp, fp, amr, lc, lf = _setup(w, fine, pert=0)
    cs, fs, cg, fg = _oracle_setup(w, fine, pert=0)
    torch.cuda.synchronize()
    got = fp.from_device(lf.current, 6)
    for g, r in zip(got, fs):
        assert np.array_equal(g, r)          # every cell, ghosts included
    gotg = fp.from_device(lf.grav, 3)
    for g, r in zip(gotg, fg):
        assert np.array_equal(g, r)
    # ghost region only, on perturbed fine data
    pert = W.scale_valid(fs, W.cell_factors(fine, 3, 0.01))
    ref = oracle.amr_interp(w.level, cs, fine, pert, "ghosts")
    dev = fp.to_device(pert, 6)
    amr.interp(lc.current, dev, 6, "ghosts")
    fp.fill(dev, 6)
    torch.cuda.synchronize()
    for g, r in zip(fp.from_device(dev, 6), ref):
        assert np.array_equal(g, r)
    # average down of the perturbed fine data
    cref = oracle.amr_average_down(w.level, cs, fine, pert)
    cdev = cp.to_device(cs, 6)
    amr.average_down(dev, cdev, 6)
    torch.cuda.synchronize()
    for g, r in zip(cp.from_device(cdev, 6), cref):
        assert np.array_equal(W.valid(g), W.valid(r))
    amr.close(); fp.close(); cp.close()


@pytest.mark.parametrize("grav", [True, False])
def test_two_level_step_fp64_matches_the_oracle(grav):
    w, fine = TA._hierarchy()
    cp, fp, amr, lc, lf = _setup(w, fine, grav=grav)
    cs, fs, cg, fg = _oracle_setup(w, fine, grav=grav)
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl)
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dt_ref = oracle.amr_estdt(w.level, fine, P, cs, fs, a0)
    a = torch.tensor([a0, a1], dtype=torch.float64, device="cuda")
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    amr.estdt(lc, lf, a[:1], dt[:1])
    torch.cuda.synchronize()
    assert abs(dt[0].item() - dt_ref) <= 1e-15 * dt_ref
    amr.step(lc, lf, a[:1], a[1:], dt[:1], dt[1:])
    torch.cuda.synchronize()
    assert cp.status() == (0, 0) and fp.status() == (0, 0)
    cn, fn, _, _ = oracle.amr_step(w.level, fine, P, cs, fs, cg, fg, a_old=a0, a_new=a1,
                                   dt=dt[0].item())
    assert _norm_rel(cp.from_device(lc.current, 6), cn) <= 1e-12
    assert _norm_rel(fp.from_device(lf.current, 6), fn) <= 1e-12
    dt_next = oracle.amr_estdt(w.level, fine, P, cn, fn, a1)
    assert abs(dt[1].item() - dt_next) <= 1e-12 * dt_next
    amr.close(); fp.close(); cp.close()


def test_two_level_step_mixed_within_the_mixed_gates():
    w, fine = TA._hierarchy()
    cp, fp, amr, lc, lf = _setup(w, fine, precision="mixed")
    cs, fs, cg, fg = _oracle_setup(w, fine)
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl)
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dtv = 0.9 * oracle.amr_estdt(w.level, fine, P, cs, fs, a0)
    a = torch.tensor([a0, a1], dtype=torch.float64, device="cuda")
    dt = torch.tensor([dtv], dtype=torch.float64, device="cuda")
    amr.step(lc, lf, a[:1], a[1:], dt)
    torch.cuda.synchronize()
    assert cp.status() == (0, 0) and fp.status() == (0, 0)
    cn, fn, _, _ = oracle.amr_step(w.level, fine, P, cs, fs, cg, fg, a_old=a0, a_new=a1, dt=dtv)
    e_mixed = _norm_rel(cp.from_device(lc.current, 6), cn)
    print('mixed vs oracle, worst field L-inf:', e_mixed)
    assert e_mixed <= MIXED_GATES["linf"]
    e_mixed = _norm_rel(fp.from_device(lf.current, 6), fn)
    print('mixed vs oracle, worst field L-inf:', e_mixed)
    assert e_mixed <= MIXED_GATES["linf"]
    amr.close(); fp.close(); cp.close()


def test_graph_run_equals_eager_steps():
    """Three steps through nyx_amr_run with and without graph capture give
    the same bits."""
    w, fine = TA._hierarchy()
    res = []
    for use_graph in (False, True):
        cp, fp, amr, lc, lf = _setup(w, fine)
        a = torch.tensor(w.a_sched[:1].tolist() * 4, dtype=torch.float64, device="cuda")
        a += torch.arange(4, dtype=torch.float64, device="cuda") * 1e-5
        dt = torch.zeros(4, dtype=torch.float64, device="cuda")
        amr.run(lc, lf, a, dt, 3, compute_dt0=True, use_graph=use_graph)
        torch.cuda.synchronize()
        assert cp.status() == (0, 0) and fp.status() == (0, 0)
        res.append((cp.from_device(lc.current, 6), fp.from_device(lf.current, 6),
                    dt.cpu().numpy()))
        amr.close(); fp.close(); cp.close()
    for x, y in zip(res[0][0] + res[0][1], res[1][0] + res[1][1]):
        assert np.array_equal(W.valid(x), W.valid(y))
    assert np.array_equal(res[0][2], res[1][2])


def test_conservation_on_the_gpu():
    """a constant, g = 0: after the step the coarse level (reflux, average
    down) holds the composite totals of rho and m, conserved to round-off.
    (rho E also changes through the dual-energy switch, so it is not
    checked here.)"""
    w, fine = TA._hierarchy()
    cp, fp, amr, lc, lf = _setup(w, fine, grav=False)
    torch.cuda.synchronize()
    before = TA._totals(w.level, cp.from_device(lc.current, 6))
    a = torch.ones(2, dtype=torch.float64, device="cuda")
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    amr.estdt(lc, lf, a[:1], dt[:1])
    amr.step(lc, lf, a[:1], a[1:], dt[:1])
    torch.cuda.synchronize()
    after = TA._totals(w.level, cp.from_device(lc.current, 6))
    scale = np.array([before[0], 0.1 * before[0], 0.1 * before[0], 0.1 * before[0]])
    assert np.all(np.abs(after[:4] - before[:4]) / scale <= 2e-14)
    amr.close(); fp.close(); cp.close()


def test_create_rejects_bad_pairs():
    w, fine = TA._hierarchy()
    cp = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64", keep_fluxes=1)
    fp_nokeep = H.Plan(fine, stream=cp.torch_stream, precision="fp64", coarse_fine=1)
    with pytest.raises(H.NyxError):
        H.Amr(cp, fp_nokeep)
    fp_other_stream = H.Plan(fine, precision="fp64", keep_fluxes=1, coarse_fine=1)
    with pytest.raises(H.NyxError):
        H.Amr(cp, fp_other_stream)
    with pytest.raises(H.NyxError):
        H.Plan(fine, precision="fp64", keep_fluxes=1)      # holes without coarse_fine
    fp_nokeep.close(); fp_other_stream.close(); cp.close()


def test_two_level_step_with_flattening_fp64():
    """The two-level step with shock flattening on both levels (the fine
    level's coefficients see its interpolated ghost cells) against the
    oracle's, FP64, within 1e-12."""
    w, fine = TA._hierarchy()
    cp, fp, amr, lc, lf = _setup(w, fine, flattening=True)
    cs, fs, cg, fg = _oracle_setup(w, fine)
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl, flattening=1)
    f = oracle.flatten_field(w.level, P, cs)
    assert min(float(x.min()) for x in f) < 1.0
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    dtv = oracle.amr_estdt(w.level, fine, P, cs, fs, a0)
    a = torch.tensor([a0, a1], dtype=torch.float64, device="cuda")
    dt = torch.tensor([dtv], dtype=torch.float64, device="cuda")
    amr.step(lc, lf, a[:1], a[1:], dt)
    torch.cuda.synchronize()
    assert cp.status() == (0, 0) and fp.status() == (0, 0)
    cn, fn, _, _ = oracle.amr_step(w.level, fine, P, cs, fs, cg, fg, a_old=a0, a_new=a1, dt=dtv)
    assert _norm_rel(cp.from_device(lc.current, 6), cn) <= 1e-12
    assert _norm_rel(fp.from_device(lf.current, 6), fn) <= 1e-12
    amr.close(); fp.close(); cp.close()
