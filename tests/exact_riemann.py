"""Exact solution of the Riemann problem for a gamma-law gas.

Independent reference for the shock-tube pins: the standard textbook
construction (E. F. Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4).  The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0,
where each f_K is the shock (Rankine-Hugoniot) or rarefaction (isentropic)
velocity jump across the K wave; the solution is then sampled along x/t.
Shares nothing with the oracle or the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, gamma):
    c = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma):
    (rl, ul, pl), (rr, ur, pr) = left, right
    g = lambda p: _f(p, rl, pl, gamma) + _f(p, rr, pr, gamma) + (ur - ul)
    lo, hi = 1e-12, 10.0 * max(pl, pr)
    while g(hi) < 0:
        hi *= 2.0
    ps = brentq(g, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_f(ps, rr, pr, gamma) - _f(ps, rl, pl, gamma))
    return ps, us


def sample(left, right, gamma, xi):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t (array)."""
    (rl, ul, pl), (rr, ur, pr) = left, right
    ps, us = star_state(left, right, gamma)
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    gm = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, xi.size))
    for n, s in enumerate(np.asarray(xi).ravel()):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                rsl = rl * ((ps / pl + gm) / (gm * ps / pl + 1.0))
                S = ul - cl * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pl + (gamma - 1.0) / (2 * gamma))
                st = (rl, ul, pl) if s < S else (rsl, us, ps)
            else:  # left rarefaction
                rsl = rl * (ps / pl) ** (1.0 / gamma)
                csl = cl * (ps / pl) ** ((gamma - 1.0) / (2 * gamma))
                head, tail = ul - cl, us - csl
                if s < head:
                    st = (rl, ul, pl)
                elif s > tail:
                    st = (rsl, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) * (cl + (gamma - 1.0) / 2.0 * (ul - s))
                    u = 2.0 / (gamma + 1.0) * (cl + (gamma - 1.0) / 2.0 * ul + s)
                    r = rl * (c / cl) ** (2.0 / (gamma - 1.0))
                    st = (r, u, pl * (c / cl) ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of contact
            if ps > pr:  # right shock
                rsr = rr * ((ps / pr + gm) / (gm * ps / pr + 1.0))
                S = ur + cr * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pr + (gamma - 1.0) / (2 * gamma))
                st = (rsr, us, ps) if s < S else (rr, ur, pr)
            else:  # right rarefaction
                rsr = rr * (ps / pr) ** (1.0 / gamma)
                csr = cr * (ps / pr) ** ((gamma - 1.0) / (2 * gamma))
                head, tail = ur + cr, us + csr
                if s > head:
                    st = (rr, ur, pr)
                elif s < tail:
                    st = (rsr, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) * (cr - (gamma - 1.0) / 2.0 * (ur - s))
                    u = 2.0 / (gamma + 1.0) * (-cr + (gamma - 1.0) / 2.0 * ur + s)
                    r = rr * (c / cr) ** (2.0 / (gamma - 1.0))
                    st = (r, u, pr * (c / cr) ** (2.0 * gamma / (gamma - 1.0)))
        out[:, n] = st
    return out


def cell_averages(left, right, gamma, x0, t, edges, nsub=16):
    """Cell averages of (rho, u, p) over cells with the given edges at time t
    (midpoint rule on nsub sub-points per cell)."""
    n = len(edges) - 1
    xs = []
    for i in range(n):
        a, b = edges[i], edges[i + 1]
        xs.append(a + (np.arange(nsub) + 0.5) * (b - a) / nsub)
    xs = np.concatenate(xs)
    w = sample(left, right, gamma, (xs - x0) / t)
    return w.reshape(3, n, nsub).mean(axis=2)
