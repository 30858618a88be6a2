"""Exact Riemann solver for the 1-D Euler equations with a gamma-law gas.

Test infrastructure: an independent pin for the oracle's two-shock solver
and its whole-step Sod run.  It follows the published exact method (Toro,
"Riemann Solvers and Numerical Methods for Fluid Dynamics", 3rd ed., 2009,
ch. 4): Newton iteration on the exact pressure function built from the
Rankine-Hugoniot shock curve and the isentropic rarefaction curve, then
self-similar sampling.  Written here from those relations; it shares
nothing with the oracle.
"""
from __future__ import annotations

import math

import numpy as np


def _fK(p, rho, pk, c, g):
    """Velocity change across the K wave at star pressure p, and its derivative."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        sq = math.sqrt(A / (p + B))
        f = (p - pk) * sq
        df = sq * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction
        f = 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * c) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, g, tol=1e-15, max_iter=200):
    """Exact (p*, u*) of the Riemann problem."""
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    # two-rarefaction initial guess
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-14)
    for _ in range(max_iter):
        fl, dfl = _fK(p, rl, pl, cl, g)
        fr, dfr = _fK(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, cl, g)
    fr, _ = _fK(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def star_densities(rl, pl, rr, pr, pstar, g):
    def rho_star(rk, pk):
        if pstar > pk:
            r = pstar / pk
            q = (g - 1.0) / (g + 1.0)
            return rk * (r + q) / (q * r + 1.0)
        return rk * (pstar / pk) ** (1.0 / g)
    return rho_star(rl, pl), rho_star(rr, pr)


def sample(rl, ul, pl, rr, ur, pr, g, xi):
    """Exact (rho, u, p) at similarity coordinate xi = x/t (array)."""
    xi = np.asarray(xi, dtype=float)
    ps, us = star_state(rl, ul, pl, rr, ur, pr, g)
    rsl, rsr = star_densities(rl, pl, rr, pr, ps, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for n, s in enumerate(xi.ravel()):
        if s <= us:  # left of contact
            if ps > pl:
                S = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                st = (rl, ul, pl) if s <= S else (rsl, us, ps)
            else:
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                head, tail = ul - cl, us - csl
                if s <= head:
                    st = (rl, ul, pl)
                elif s >= tail:
                    st = (rsl, us, ps)
                else:
                    uu = 2.0 / (g + 1) * (cl + 0.5 * (g - 1) * ul + s)
                    cc = 2.0 / (g + 1) * (cl + 0.5 * (g - 1) * (ul - s))
                    rr_ = rl * (cc / cl) ** (2.0 / (g - 1))
                    st = (rr_, uu, pl * (cc / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                S = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                st = (rr, ur, pr) if s >= S else (rsr, us, ps)
            else:
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                head, tail = ur + cr, us + csr
                if s >= head:
                    st = (rr, ur, pr)
                elif s <= tail:
                    st = (rsr, us, ps)
                else:
                    uu = 2.0 / (g + 1) * (-cr + 0.5 * (g - 1) * ur + s)
                    cc = 2.0 / (g + 1) * (cr - 0.5 * (g - 1) * (ur - s))
                    rr_ = rr * (cc / cr) ** (2.0 / (g - 1))
                    st = (rr_, uu, pr * (cc / cr) ** (2 * g / (g - 1)))
        rho.flat[n], u.flat[n], p.flat[n] = st
    return rho, u, p


def cell_average(rl, ul, pl, rr, ur, pr, g, x_edges, x0, t, sub=64):
    """Cell averages of (rho, u, p) over cells with the given edges at time t."""
    x_edges = np.asarray(x_edges, float)
    n = len(x_edges) - 1
    frac = (np.arange(sub) + 0.5) / sub
    xs = x_edges[:-1, None] + (x_edges[1:] - x_edges[:-1])[:, None] * frac[None, :]
    r, u, p = sample(rl, ul, pl, rr, ur, pr, g, (xs - x0) / t)
    return r.reshape(n, sub).mean(1), u.reshape(n, sub).mean(1), p.reshape(n, sub).mean(1)
