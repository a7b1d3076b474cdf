"""Exact solution of the 1D Euler Riemann problem for an ideal gas.

Textbook construction (e.g. Toro, "Riemann Solvers and Numerical Methods for
Fluid Dynamics", ch. 4): Newton iteration on the star pressure p* from the
shock (Rankine-Hugoniot) and rarefaction (isentropic) relations, then sampling
of the self-similar solution.  Used by the tests as an independent pin for the
shock-tube runs of the oracle; it shares nothing with the scheme.
"""
from __future__ import annotations

import math

import numpy as np


def _f(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    r = (p / pk) ** ((gamma - 1.0) / (2.0 * gamma))
    return 2.0 * a / (gamma - 1.0) * (r - 1.0), 1.0 / (rho * a) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))


def star_state(left, right, gamma=1.4, tol=1e-14):
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(tol, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _f(p, rl, pl, gamma)
        fr, dr = _f(p, rr, pr, gamma)
        g = fl + fr + (ur - ul)
        pn = max(tol, p - g / (dl + dr))
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, gamma)
    fr, _ = _f(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, gamma=1.4):
    """Primitive (rho, u, p) of the self-similar solution at x/t = xi (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    g = gamma
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi); u = np.empty_like(xi); p = np.empty_like(xi)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                S = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                st = (rl, ul, pl) if s <= S else (rs, us, ps)
            else:
                rs = rl * (ps / pl) ** (1 / g)
                asl = al * (ps / pl) ** ((g - 1) / (2 * g))
                head, tail = ul - al, us - asl
                if s <= head:
                    st = (rl, ul, pl)
                elif s >= tail:
                    st = (rs, us, ps)
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
                    st = (rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + s), pl * c ** (2 * g / (g - 1)))
        else:
            if ps > pr:  # right shock
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                S = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                st = (rr, ur, pr) if s >= S else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1 / g)
                asr = ar * (ps / pr) ** ((g - 1) / (2 * g))
                head, tail = ur + ar, us + asr
                if s >= head:
                    st = (rr, ur, pr)
                elif s <= tail:
                    st = (rs, us, ps)
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
                    st = (rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s), pr * c ** (2 * g / (g - 1)))
        rho[idx], u[idx], p[idx] = st
    return rho, u, p


def cell_averages(left, right, x0, t, edges, gamma=1.4, sub=64):
    """Exact cell averages of the conservative variables (Gauss sub-sampling)."""
    gx, gw = np.polynomial.legendre.leggauss(sub)
    n = len(edges) - 1
    W = np.zeros((3, n))
    for i in range(n):
        a, b = edges[i], edges[i + 1]
        xs = 0.5 * (a + b) + 0.5 * (b - a) * gx
        r, u, p = sample(left, right, (xs - x0) / t, gamma)
        cons = np.stack([r, r * u, p / (gamma - 1) + 0.5 * r * u * u])
        W[:, i] = (cons * (0.5 * gw)).sum(axis=1)
    return W
