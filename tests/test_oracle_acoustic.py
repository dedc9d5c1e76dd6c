"""CPU pins of the oracle's acoustic parts: the two-shock Riemann update and
the u-c / u+c characteristic tracing.

* Riemann solver: two weak two-shock problems (colliding flows) started from
  piecewise-constant data.  The detector marks the cells at the jump, whose
  parabolas the constraints make flat, so after one pass the face flux at
  the jump follows from the change of the two cells beside it and the exact
  Euler flux of the undisturbed states (the faces beside are between equal
  states).  That flux is checked against the exact Godunov flux (Toro's
  exact solver, tests/exact_riemann.py): the acoustic guess alone misses
  p* - p by about 6% at these strengths, one two-shock update of the
  impedances brings it within a fraction of a percent, so a dropped or
  mis-weighted update, or a wrong shock-impedance factor (gamma+1)/(2 gamma),
  fails.
* Tracing: a linear sound wave (rho = 1 + e sin 2 pi x, u = U + c e sin 2 pi x
  for the u+c family, p = 1 + gamma e sin 2 pi x, e = 1e-8) crosses a
  periodic box once; its L1 error against the start falls with the grid at
  third order (measured 3.0-3.6).  In subsonic flow only the reference
  domains of the tracing act on it; the u-c and u+c corrections of the
  characteristic tracing act only where a second acoustic family reaches
  the same edge, i.e. in supersonic flow, so a u-c wave on a Mach-2 flow to
  the right and a u+c wave on a Mach-2 flow to the left pin them: a wrong
  sign or factor in a correction, or the wrong domain of dependence, costs
  the order.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from exact_riemann import sample, star_state

GAMMA = 1.4


def _tube_problem(n):
    p = workloads.tube("sod", n=n, axis=0, ntrans=4, gamma=GAMMA)
    return p


def _euler_flux(rho, u, p):
    E = p / (GAMMA - 1.0) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, u * (E + p)])


def _face_flux_after_one_pass(left, right, n=32):
    """Flux the oracle's Riemann solver puts at the jump face, read from the
    change of the cells on both sides of it."""
    p = _tube_problem(n)
    q = workloads.build(p)
    nz, ny, nx = q[0].shape
    j = nx // 2                      # jump between cells j-1 and j
    (rl, ul, pl), (rr, ur, pr) = left, right
    for a in q:
        a[...] = 0.0
    for sl, (rho, u, pp) in ((slice(0, j), left), (slice(j, nx), right)):
        q[0][:, :, sl] = rho
        q[1][:, :, sl] = rho * u
        q[4][:, :, sl] = pp / (GAMMA - 1.0) + 0.5 * rho * u * u
    q0 = [a.copy() for a in q]
    c = max(math.sqrt(GAMMA * pl / rl) + abs(ul), math.sqrt(GAMMA * pr / rr) + abs(ur))
    dt = 0.4 * p.dx / c
    oracle.Oracle(p).sweep(q, 0, dt, 0)
    dq = lambda i: np.array([q[0][0, 0, i] - q0[0][0, 0, i], q[1][0, 0, i] - q0[1][0, 0, i],
                             q[4][0, 0, i] - q0[4][0, 0, i]])
    # cells two away from the jump see equal states on both faces (to the
    # 1e-9 floor of the continuous detector weight, which leaves the
    # parabolas beside the jump flat only to about 1e-10)
    big = np.abs(dq(j - 1)).max()
    assert np.abs(dq(j - 3)).max() <= 1e-8 * big and np.abs(dq(j + 2)).max() <= 1e-8 * big
    lam = dt / p.dx
    F_from_left = _euler_flux(*left) - dq(j - 1) / lam      # cell j-1: F(j-1/2) - F_L = -dq/lam
    F_from_right = _euler_flux(*right) + dq(j) / lam        # cell j:   F_R - F(j-1/2) = -dq/lam
    return F_from_left, F_from_right


def _exact_godunov_flux(left, right):
    r, u, pp = sample(left, right, GAMMA, np.array([0.0]))[:, 0]
    return _euler_flux(r, u, pp)


CASES = {
    # symmetric collision at Mach 0.1: u* = 0, both waves shocks
    "symmetric": ((1.0, 0.1 * math.sqrt(GAMMA), 1.0), (1.0, -0.1 * math.sqrt(GAMMA), 1.0)),
    # unequal states, both waves shocks, u* > 0 (left star state at x/t = 0)
    "asymmetric": ((1.0, 0.25, 1.0), (0.5, -0.05, 0.8)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_riemann_flux_matches_exact_for_weak_two_shock_problems(case):
    left, right = CASES[case]
    ps, us = star_state(left, right, GAMMA)
    assert ps > left[2] and ps > right[2]          # both waves are shocks
    F1, F2 = _face_flux_after_one_pass(left, right)
    # the two cells beside the jump give the same face flux
    np.testing.assert_allclose(F1, F2, rtol=1e-8, atol=1e-9)
    Fx = _exact_godunov_flux(left, right)
    # momentum flux carries p*: compare p* - p to its exact value
    pl = left[2]
    if case == "symmetric":
        assert abs(F1[0]) <= 1e-9 and abs(F1[2]) <= 1e-9      # u* = 0 by symmetry
        dp_num, dp_ex = F1[1] - pl, ps - pl
        assert abs(dp_num - dp_ex) <= 1.5e-2 * dp_ex, (dp_num, dp_ex)
    else:
        scale = np.abs(Fx) + np.array([0.0, ps - min(left[2], right[2]), 0.0])
        err = np.abs(F1 - Fx) / scale
        assert err.max() <= 1e-2, (F1, Fx, err)


def _sound_wave(n, family, U, eps=1e-8):
    """Linear acoustic mode of the family u + family*c on a uniform
    background flow U (rho0 = 1, p0 = 1): cell averages of
    rho = 1 + e sin, u = U + family c e sin, p = 1 + gamma e sin."""
    p = workloads.wave(n=n, axis=0, kind="density", u=0.0, gamma=GAMMA)
    x_l = np.arange(n) * p.dx
    x_r = x_l + p.dx
    k = 2.0 * math.pi
    s_avg = (np.cos(k * x_l) - np.cos(k * x_r)) / (k * p.dx)       # cell average of sin(kx)
    c0 = math.sqrt(GAMMA)
    rho = 1.0 + eps * s_avg
    mom = U + U * eps * s_avg + family * eps * c0 * s_avg
    pr = 1.0 + GAMMA * eps * s_avg
    q = workloads.build(p)
    for a in q:
        a[...] = 0.0
    q[0][...] = rho[None, None, :]
    q[1][...] = mom[None, None, :]
    q[4][...] = (pr / (GAMMA - 1.0) + 0.5 * mom * mom / rho)[None, None, :]
    return p, q, c0


def _sound_wave_error(n, family, mach, cfl=0.5, eps=1e-8):
    """Largest L1 error of rho, rho u and E (each relative to its
    perturbation amplitude) after the wave has crossed the periodic box once."""
    c0 = math.sqrt(GAMMA)
    U = mach * c0
    p, q, _ = _sound_wave(n, family, U, eps)
    start = [q[v][0, 0].copy() for v in (0, 1, 4)]
    T = 1.0 / abs(U + family * c0)
    smax = abs(U) + c0
    nsteps = int(math.ceil(T / (2.0 * cfl * p.dx / smax)))
    dt = T / (2.0 * nsteps)
    o = oracle.Oracle(p)
    for _ in range(nsteps):
        o.double_step(q, dt)
    # rho, rho u and E, each relative to its own perturbation amplitude
    amp = (eps, eps * (abs(U) + c0), eps * (GAMMA / (GAMMA - 1.0) + abs(U) * c0 + 0.5 * U * U))
    return max(np.abs(q[v][0, 0] - s0).mean() / a for v, s0, a in zip((0, 1, 4), start, amp))


@pytest.mark.parametrize("family,mach", [(1, 0.0), (-1, 2.0), (1, -2.0)])
def test_sound_wave_converges_at_third_order(family, mach):
    """family, background Mach number: (+1, 0) the u+c wave at rest (only the
    reference domains of the tracing); (-1, 2) the u-c wave in a supersonic
    flow to the right, where every family reaches the right edge and the u-c
    correction of that edge carries the wave; (+1, -2) the mirror case, the
    u+c correction of the left edge."""
    ns = [16, 32, 64, 128]
    errs = [_sound_wave_error(n, family, mach) for n in ns]
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(ns) - 1)]
    assert errs[-1] < 1e-2, errs
    assert min(orders) >= 2.7, (errs, orders)
