"""The seeded synthetic inputs follow their stated recipe: a unit-variance
Gaussian field with a k^-2 spectrum; a lognormal density of mean 1 whose
logarithm has standard deviation sigma; velocities and gravity scaled to an
rms magnitude of 0.1; gravity the centred difference of a potential (so its
periodic mean and its discrete curl vanish); conserved variables from the
primitives with e = 0.9; NaN ghost cells; per-box seeds that do not depend on
which boxes are drawn; the tiled level covering its periodic domain once."""
import numpy as np
import pytest

from paper_1301_4498_gb300 import workloads as W


def _shell_power(g):
    """Shell-averaged |FFT|^2 of a periodic cube against integer |k|."""
    n = g.shape[0]
    P = np.abs(np.fft.fftn(g)) ** 2
    k = np.fft.fftfreq(n) * n
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    shell = np.rint(kk).astype(int)
    return np.bincount(shell.ravel(), P.ravel()) / np.maximum(np.bincount(shell.ravel()), 1)


def test_gaussian_field_unit_variance_and_k2_spectrum():
    g = W.gaussian_k2((48, 48, 48), np.random.default_rng(4))
    assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(1.0, rel=1e-12)
    p = _shell_power(g)
    ks = np.arange(3, 17)
    slope = np.polyfit(np.log(ks), np.log(p[ks]), 1)[0]
    assert slope == pytest.approx(-2.0, abs=0.15)
    # white noise would be flat: the spectrum is not an artefact of the fit
    flat = _shell_power(np.random.default_rng(4).standard_normal((48, 48, 48)))
    assert abs(np.polyfit(np.log(ks), np.log(flat[ks]), 1)[0]) < 0.15


def test_gaussian_field_is_seeded():
    a = W.gaussian_k2((8, 12, 16), np.random.default_rng(9))
    b = W.gaussian_k2((8, 12, 16), np.random.default_rng(9))
    c = W.gaussian_k2((8, 12, 16), np.random.default_rng(10))
    assert np.array_equal(a, b) and not np.allclose(a, c)


@pytest.mark.parametrize("sigma", [0.5, 1.0])
def test_comoving_fields_recipe(sigma):
    shape = (16, 24, 32)                       # (z, y, x), not a cube
    dx = 1.0 / 32
    f = W.comoving_fields(shape, sigma, 7, dx)
    assert f.rho.shape == shape and f.u.shape == (3,) + shape and f.g.shape == (3,) + shape
    assert np.all(f.rho > 0) and f.rho.mean() == pytest.approx(1.0, rel=1e-13)
    assert np.log(f.rho).std() == pytest.approx(sigma, rel=1e-12)
    assert np.sqrt((f.u ** 2).sum(axis=0).mean()) == pytest.approx(0.1, rel=1e-12)
    assert np.sqrt((f.g ** 2).sum(axis=0).mean()) == pytest.approx(0.1, rel=1e-12)
    # g = -grad(phi) by centred differences: zero periodic mean, zero discrete curl
    assert np.abs(f.g.mean(axis=(1, 2, 3))).max() < 1e-15
    d = lambda a, ax: (np.roll(a, -1, axis=ax) - np.roll(a, 1, axis=ax)) / (2 * dx)
    gx, gy, gz = f.g
    for curl in (d(gy, 2) - d(gx, 1), d(gz, 1) - d(gy, 0), d(gx, 0) - d(gz, 2)):
        assert np.abs(curl).max() <= 1e-12 * np.abs(d(gx, 2)).max()
    # the velocity components are independent draws, not copies
    assert abs(np.corrcoef(f.u[0].ravel(), f.u[1].ravel())[0, 1]) < 0.2


def test_patched_state_is_conserved_form_with_nan_ghosts():
    lev = W.single_box_level(8, 8, 8, 1.0 / 8)
    f = W.comoving_fields((8, 8, 8), 0.5, 3, 1.0 / 8)
    S, G = W._patch_state(lev, 0, f)
    v = W.valid(S)
    assert np.array_equal(v[0], f.rho)
    assert np.array_equal(v[1:4], f.rho[None] * f.u)
    assert np.array_equal(v[5], f.rho * W.E0)
    assert np.allclose(v[4], v[5] + 0.5 * f.rho * (f.u ** 2).sum(axis=0), rtol=1e-15)
    assert W.E0 == 0.9
    ghosts = np.ones(S.shape[1:], bool)
    ghosts[4:-4, 4:-4, 4:-4] = False
    assert np.isnan(S[:, ghosts]).all() and np.isnan(G[:, ghosts]).all()
    assert np.isfinite(v).all() and np.array_equal(W.valid(G), f.g)


def test_uneven_boxes_draw_per_box():
    sizes = (16, 24, 32, 48, 64)
    a = W.uneven_boxes(nbox=512, boxes=[3, 7], nsteps=1)
    b = W.uneven_boxes(nbox=512, boxes=[7], nsteps=1)
    assert a.level.extent(1) == b.level.extent(0)
    assert all(v in sizes for e in (a.level.extent(0), a.level.extent(1)) for v in e)
    assert np.array_equal(a.state[1], b.state[0], equal_nan=True)


def test_tiled_level_covers_its_periodic_domain_once():
    lev = W.tiled_level(512, 32)
    assert lev.nbox == 4096
    assert all(lev.extent(b) == (32, 32, 32) for b in (0, 1, 4095))
    assert lev.valid_cells() == 512 ** 3
    lo = np.asarray(lev.lo)
    assert len({tuple(x) for x in lo}) == 4096 and lo.min() == 0 and np.asarray(lev.hi).max() == 511
    assert np.all(lo % 32 == 0)


def test_scale_factor_schedule_is_linear():
    a = W.a_schedule(1.0 / 51, 1.0 / 31, 100)
    assert len(a) == 101 and a[0] == 1.0 / 51 and a[-1] == pytest.approx(1.0 / 31, rel=1e-15)
    assert np.allclose(np.diff(a), (1.0 / 31 - 1.0 / 51) / 100, rtol=1e-10)
