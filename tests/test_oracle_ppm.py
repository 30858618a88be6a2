"""Pins of the oracle's PPM reconstruction (Sec. 3.2, Colella & Woodward 1984)
against closed forms and invariants of the method."""
import numpy as np
import pytest

import oracle


def test_linear_profile_reproduced_exactly():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.normal(), rng.normal() * 3
        i = np.arange(16.0)
        s = a + b * i
        sL, sR, s6 = oracle.ppm_line(s)
        for c in range(2, 14):
            assert sL[c] == pytest.approx(a + b * (c - 0.5), rel=1e-14, abs=1e-14)
            assert sR[c] == pytest.approx(a + b * (c + 0.5), rel=1e-14, abs=1e-14)
            assert abs(s6[c]) <= 1e-13 * (abs(a) + abs(b) * 16)
            for sig in (0.0, 0.1, 0.5, 0.9):
                ip, im = oracle.ppm_integrals(sL[c], sR[c], s6[c], sig)
                # exact averages of the line over [c+1/2-sig, c+1/2] and [c-1/2, c-1/2+sig]
                assert ip == pytest.approx(a + b * (c + 0.5 - 0.5 * sig), rel=1e-13, abs=1e-13)
                assert im == pytest.approx(a + b * (c - 0.5 + 0.5 * sig), rel=1e-13, abs=1e-13)


def _cubic_avg(coef, xl, xr):
    # exact average of c0 + c1 x + c2 x^2 + c3 x^3 over [xl, xr]
    P = lambda x: sum(c * x ** (k + 1) / (k + 1) for k, c in enumerate(coef))
    return (P(xr) - P(xl)) / (xr - xl)


def test_unlimited_interface_exact_for_cubic_averages():
    """For smooth monotone data the limiters are inactive and the interface
    value is the fourth-order formula, exact for cell averages of a cubic."""
    coef = (0.3, 1.0, 0.02, 0.001)
    i = np.arange(20.0)
    s = np.array([_cubic_avg(coef, c - 0.5, c + 0.5) for c in i])
    sL, sR, s6 = oracle.ppm_line(s)
    f = lambda x: sum(c * x ** k for k, c in enumerate(coef))
    for c in range(3, 16):
        assert sR[c] == pytest.approx(f(c + 0.5), rel=1e-13)
        assert sL[c] == pytest.approx(f(c - 0.5), rel=1e-13)


def test_local_extremum_is_flattened():
    sL, sR, s6 = oracle.ppm_line(np.array([0.0, 1.0, 3.0, 1.0, 0.0]))
    assert sL[2] == 3.0 and sR[2] == 3.0 and s6[2] == 0.0
    sL, sR, s6 = oracle.ppm_line(np.array([2.0, 1.0, -1.0, 1.5, 2.0]))
    assert sL[2] == -1.0 and sR[2] == -1.0 and s6[2] == 0.0


def test_interface_values_bounded_and_parabolas_monotone():
    """Invariants of CW84 limiting on random data: every interface value lies
    between its two neighbouring cell values, and every limited parabola is
    monotone inside its cell and takes the cell value as its average."""
    rng = np.random.default_rng(1)
    for trial in range(200):
        s = rng.normal(size=40) * rng.uniform(0.1, 10) + np.cumsum(rng.normal(size=40))
        sL, sR, s6 = oracle.ppm_line(s)
        for c in range(2, 38):
            # the parabola  a(xi) = sL + xi (dS + s6 (1 - xi)),  xi in [0, 1]
            dS = sR[c] - sL[c]
            d0 = dS + s6[c]      # derivative at xi = 0
            d1 = dS - s6[c]      # derivative at xi = 1
            assert d0 * d1 >= -1e-12 * (1 + abs(dS) + abs(s6[c])) ** 2
            # average of the parabola equals the cell value
            avg = sL[c] + 0.5 * dS + s6[c] / 6.0
            assert avg == pytest.approx(s[c], rel=1e-12, abs=1e-12)
            lo = min(s[c - 1], s[c], s[c + 1])
            hi = max(s[c - 1], s[c], s[c + 1])
            tol = 1e-12 * (1 + abs(lo) + abs(hi))
            assert lo - tol <= sL[c] <= hi + tol
            assert lo - tol <= sR[c] <= hi + tol


def test_integrals_are_averages_of_the_parabola():
    """I+(sigma) and I-(sigma) equal the numerically integrated parabola."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        sL, sR, s6 = rng.normal(size=3)
        for sig in (0.05, 0.3, 0.77, 1.0):
            ip, im = oracle.ppm_integrals(sL, sR, s6, sig)
            xi = np.linspace(1 - sig, 1, 20001)
            par = sL + xi * ((sR - sL) + s6 * (1 - xi))
            assert ip == pytest.approx(np.trapezoid(par, xi) / sig, rel=1e-8, abs=1e-8)
            xi = np.linspace(0, sig, 20001)
            par = sL + xi * ((sR - sL) + s6 * (1 - xi))
            assert im == pytest.approx(np.trapezoid(par, xi) / sig, rel=1e-8, abs=1e-8)
