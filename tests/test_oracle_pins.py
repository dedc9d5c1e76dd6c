"""CPU pins of the FP64 oracle against what the mathematics fixes.

The paper prints no worked values for the sweep (Woodward et al. give the
ingredients in Sec. 1 and Sec. 4 but no formulas), so the oracle is pinned by
exact solutions, exact invariants and measured convergence, each chosen so a
plausible slip (a dropped term, a wrong sign or index, a transposed operand)
fails one of them:

* shock tubes (Sod, Lax) along every axis against the exact Riemann solution,
  itself pinned by the published Sod star state (tests/golden/sod_star.txt);
* uniform states and hydrostatic states (plane layer and sphere) preserved
  bit for bit;
* conservation of mass, momentum, energy and rho*FV in a periodic box;
* axis-permutation symmetry (bit for bit);
* 0 <= FV <= 1 after every pass;
* measured convergence order on smooth advection (density wave, FV bump);
* exact transport of a quadratic FV profile and of the FV first moment at
  constant velocity;
* diagnostics against library sums.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from exact_riemann import cell_averages, star_state

HERE = os.path.dirname(os.path.abspath(__file__))


def _copy(q):
    return [a.copy() for a in q]


def _run(o, q, steps, cfl=None):
    for _ in range(steps):
        o.double_step(q, o.cfl_dt(q, cfl))


# --------------------------------------------------------------------------
def test_exact_solver_matches_published_sod_star():
    vals = np.loadtxt(os.path.join(HERE, "golden", "sod_star.txt"))
    ps, us = star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    g = 1.4
    gm = (g - 1) / (g + 1)
    rl = (ps / 1.0) ** (1 / g)
    rr = 0.125 * ((ps / 0.1 + gm) / (gm * ps / 0.1 + 1))
    np.testing.assert_allclose([ps, us, rl, rr], vals, rtol=2e-5)


def _tube_error(kind, n, axis, length):
    p = workloads.tube(kind, n=n, axis=axis, length=length)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    L, R, T = workloads.TUBE_STATES[kind]
    t = 0.0
    while t < T - 1e-14:
        dt = min(o.cfl_dt(q, 0.6), 0.5 * (T - t))
        o.double_step(q, dt)
        t += 2 * dt
    sl = [0, 0, 0]
    sl[2 - axis] = slice(None)
    N = p.shape[axis]
    edges = p.origin[axis] + np.arange(N + 1) * p.dx
    ex = cell_averages(L, R, 1.4, 0.5, T, edges)
    win = (edges[:-1] >= -1e-12) & (edges[1:] <= 1 + 1e-12)
    # transverse uniformity: the 1-D problem stays 1-D
    for v in (0, 4):
        a = q[v]
        assert np.array_equal(a, np.broadcast_to(a[tuple(sl)].reshape(
            [N if d == 2 - axis else 1 for d in range(3)]), a.shape))
    return np.abs(q[0][tuple(sl)] - ex[0])[win].mean()


@pytest.mark.parametrize("kind,length", [("sod", 1.0), ("lax", 2.0)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shock_tube_converges(kind, length, axis):
    errs = [_tube_error(kind, n, axis, length) for n in (100, 200, 400)]
    order = math.log2(errs[0] / errs[2]) / 2.0
    assert errs[2] < (2e-3 if kind == "sod" else 6e-3), errs
    assert order >= 0.8, (errs, order)


def test_shock_tube_identical_along_axes():
    res = []
    for axis in range(3):
        p = workloads.tube("sod", n=64, axis=axis)
        q = workloads.build(p)
        o = oracle.Oracle(p)
        _run(o, q, 10, 0.6)
        sl = [0, 0, 0]
        sl[2 - axis] = slice(None)
        res.append(np.stack([q[0][tuple(sl)], q[1 + axis][tuple(sl)], q[4][tuple(sl)]]))
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


# --------------------------------------------------------------------------
def _uniform_problem(shape, rho, vel, p, fv, base=(1.0, 1.0), gamma=5.0 / 3.0):
    prob = workloads.periodic_box(shape=shape, gamma=gamma)
    prob.tables = workloads._uniform_tables(*base)
    nz_ny_nx = (shape[2], shape[1], shape[0])
    q = [np.zeros(nz_ny_nx) for _ in range(9)]
    q[0][:] = rho
    for d in range(3):
        q[1 + d][:] = rho * vel[d]
    q[4][:] = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    q[5][:] = fv
    return prob, q


@pytest.mark.parametrize("rho,vel,p,fv,base", [
    (1.0, (0.25, -0.125, 0.375), 0.75, 1.0, (1.0, 1.0)),
    (1.75, (-0.3, 0.2, 0.1), 1.25, 0.0, (1.5, 1.0)),
])
def test_uniform_state_preserved_bitwise(rho, vel, p, fv, base):
    prob, q = _uniform_problem((8, 12, 16), rho, vel, p, fv, base)
    q0 = _copy(q)
    o = oracle.Oracle(prob)
    _run(o, q, 20)
    for a, b in zip(q, q0):
        assert np.array_equal(a, b)


def _hydrostatic_strat():
    p = workloads.strat_box(shape=(8, 6, 24), noise=0.0)
    p.tables.heat = None
    p.tables.damp = None
    return p


def _hydrostatic_sphere():
    p = workloads.sphere(n=20, mach=0.0)
    p.tables.heat = None
    p.tables.damp = None
    return p


@pytest.mark.parametrize("maker", [_hydrostatic_strat, _hydrostatic_sphere])
def test_hydrostatic_state_preserved_bitwise(maker):
    p = maker()
    q = workloads.build(p)
    for d in range(3):
        assert not q[1 + d].any()
    q0 = _copy(q)
    o = oracle.Oracle(p)
    oracle.Oracle.reset_counters()
    _run(o, q, 20)
    for v, (a, b) in enumerate(zip(q, q0)):
        assert np.array_equal(a, b), v


# --------------------------------------------------------------------------
def test_conservation_periodic_box():
    p = workloads.periodic_box(32)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    t0, _, _ = o.diagnostics(q)
    pscale = sum(np.abs(q[1 + d]).sum() for d in range(3)) * p.dx ** 3
    _run(o, q, 20)
    t1, _, _ = o.diagnostics(q)
    for m in (0, 4, 5):
        assert abs(t1[m] - t0[m]) <= 1e-12 * abs(t0[m]), (m, t0[m], t1[m])
    for m in (1, 2, 3):
        assert abs(t1[m] - t0[m]) <= 1e-12 * pscale, (m, t0[m], t1[m])


def _permute(q, perm):
    """Relabel axes: new axis d is old axis perm[d]; arrays are (z, y, x)."""
    # numpy axes (z,y,x) = (2,1,0) in physical numbering
    np_axes = [2 - perm[2 - ax] for ax in range(3)]
    out = [None] * 9
    for v in (0, 4, 5):
        out[v] = np.ascontiguousarray(np.transpose(q[v], np_axes))
    for d in range(3):
        out[1 + d] = np.ascontiguousarray(np.transpose(q[1 + perm[d]], np_axes))
        out[6 + d] = np.ascontiguousarray(np.transpose(q[6 + perm[d]], np_axes))
    return out


@pytest.mark.parametrize("perm", [(1, 2, 0), (1, 0, 2), (2, 1, 0)])
def test_axis_permutation_symmetry(perm):
    shape = (8, 12, 16)
    p = workloads.periodic_box(shape=shape)
    p.dx = 1.0 / 16
    q = workloads.build(p)
    pshape = tuple(shape[perm[d]] for d in range(3))
    pp = workloads.periodic_box(shape=pshape)
    pp.dx = p.dx
    qp = _permute(q, perm)
    o, op = oracle.Oracle(p), oracle.Oracle(pp)
    dt = o.cfl_dt(q)
    inv = [perm.index(d) for d in range(3)]
    for axis in (0, 1, 2, 2, 1, 0):
        o.sweep(q, axis, dt)
        op.sweep(qp, inv[axis], dt)
    back = _permute(qp, inv)
    for v in range(9):
        assert np.array_equal(back[v], q[v]), v


# --------------------------------------------------------------------------
def test_fv_bounds_every_pass():
    p = workloads.periodic_box(24)
    q = workloads.build(p)
    # add a strong compressive/expansive velocity so FV is squeezed
    x = (np.arange(24) + 0.5) / 24
    for d in range(3):
        sh = [1, 1, 1]
        sh[2 - d] = -1
        q[1 + d] += 0.4 * np.sin(2 * np.pi * x).reshape(sh)
    q[4] += 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2)
    o = oracle.Oracle(p)
    for _ in range(6):
        dt = o.cfl_dt(q)
        for axis in (0, 1, 2, 2, 1, 0):
            o.sweep(q, axis, dt)
            assert q[5].min() >= 0.0 and q[5].max() <= 1.0
            assert np.isfinite(q[0]).all()


# --------------------------------------------------------------------------
def _advect_wave(n, kind, T=1.0):
    p = workloads.wave(n=n, axis=0, kind=kind, u=1.0)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    nst = int(math.ceil(T / (2 * o.cfl_dt(q, 0.5))))
    dt = T / (2 * nst)
    oracle.Oracle.reset_counters()
    for _ in range(nst):
        o.double_step(q, dt)
    xs = torch.tensor((np.arange(n) + 0.5) / n - T)
    if kind == "density":
        ex = workloads.wave_density_average(xs, 1.0 / n).numpy()
        return np.abs(q[0][0, 0, :] - ex).mean(), oracle.Oracle.counters()
    ex, _ = workloads.wave_fv_cell(xs, 1.0 / n)
    return np.abs(q[5][0, 0, :] - ex.numpy()).mean(), oracle.Oracle.counters()


def test_density_wave_third_order_and_unconstrained():
    res = [_advect_wave(n, "density") for n in (16, 32, 64)]
    errs = [r[0] for r in res]
    order = math.log2(errs[0] / errs[2]) / 2.0
    assert order >= 2.7, (errs, order)
    for _, c in res:
        assert c["nonsmooth"] == 0 and c["flattened"] == 0


def test_fv_bump_converges_unlimited():
    res = [_advect_wave(n, "fv") for n in (16, 32, 64)]
    errs = [r[0] for r in res]
    order = math.log2(errs[0] / errs[2]) / 2.0
    assert order >= 2.0, (errs, order)
    for _, c in res:
        assert c["theta_limited"] == 0 and c["fct_limited"] == 0 and c["moment_clamped"] == 0


def _quadratic_fv_problem(n, u):
    p = workloads.tube("sod", n=n, axis=0)  # reflecting x walls, uniform base
    p.extra = {}
    q = [np.zeros((4, 4, n)) for _ in range(9)]
    q[0][:] = 1.0
    q[1][:] = u
    q[4][:] = 1.0 / (p.gamma - 1.0) + 0.5 * u * u
    return p, q


def _quad_cell(a, b, c, xl, xr):
    """Average and normalised first moment of a + b x + c x^2 on [xl, xr]."""
    h = xr - xl
    xc = 0.5 * (xl + xr)
    I0 = a * h + b * (xr ** 2 - xl ** 2) / 2 + c * (xr ** 3 - xl ** 3) / 3
    I1 = (a * (xr ** 2 - xl ** 2) / 2 + b * (xr ** 3 - xl ** 3) / 3 + c * (xr ** 4 - xl ** 4) / 4)
    avg = I0 / h
    mom = 12.0 * (I1 / h - xc * avg) / h
    return avg, mom


@pytest.mark.parametrize("u", [0.3, -0.45])
def test_quadratic_fv_profile_advects_exactly(u):
    n = 32
    p, q = _quadratic_fv_problem(n, u)
    a, b, c = 0.2, 0.9, -0.6        # stays inside (0.2, 0.5) on [0, 1]
    x = np.arange(n + 1) / n
    avg, mom = _quad_cell(a, b, c, x[:-1], x[1:])
    q[5][:] = avg
    q[6][:] = mom
    o = oracle.Oracle(p)
    dt = 0.3 / n / (abs(u) + 1.2)
    oracle.Oracle.reset_counters()
    o.sweep(q, 0, dt)
    s = u * dt
    ex_avg, ex_mom = _quad_cell(a, b, c, x[:-1] - s, x[1:] - s)
    inner = slice(6, n - 6)
    np.testing.assert_allclose(q[5][0, 0, inner], ex_avg[inner], rtol=0, atol=2e-14)
    np.testing.assert_allclose(q[6][0, 0, inner], ex_mom[inner], rtol=0, atol=1e-12)
    c_ = oracle.Oracle.counters()
    assert c_["fct_limited"] == 0


def test_first_moment_shifts_by_u_dt():
    """At constant rho and u every piece of FV content moves by u dt, whatever
    the profile limiter did, so sum(x FV + dx m/12) dx grows by u t sum(FV dx)
    (minus L per unit of content that wrapped through the periodic boundary)."""
    n, u = 48, 0.5
    p = workloads.wave(n=n, axis=0, kind="fv", u=u)
    q = workloads.build(p)
    xc = (np.arange(n) + 0.5) / n
    # compact bump on a uniform floor
    floor = 0.003
    f = floor + np.where(np.abs(xc - 0.45) < 0.2, 0.9 * (1 - ((xc - 0.45) / 0.2) ** 2) ** 2, 0.0)
    q[5][:] = f
    q[6][:] = 0.0
    o = oracle.Oracle(p)
    dt = 0.2 / n
    dx = 1.0 / n

    def first_moment(q):
        fv, m = q[5][0, 0, :], q[6][0, 0, :]
        return np.sum(xc * fv + dx * m / 12.0) * dx, np.sum(fv) * dx

    M0, S0 = first_moment(q)
    oracle.Oracle.reset_counters()
    for _ in range(10):
        o.sweep(q, 0, dt)
    M1, S1 = first_moment(q)
    c = oracle.Oracle.counters()
    assert c["moment_clamped"] == 0 and c["fct_limited"] == 0
    t = 10 * dt
    assert abs(S1 - S0) <= 1e-14
    assert abs((M1 - M0) - (u * t * S0 - 1.0 * floor * u * t)) <= 1e-13


# --------------------------------------------------------------------------
def test_pencil_entry_point_matches_grid_pass():
    p = workloads.sphere(n=16)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    dt = o.cfl_dt(q)
    for axis in range(3):
        qa = _copy(q)
        o.sweep(qa, axis, dt, sources=True)
        ja, jb = 5, 11
        idx = [None] * 3
        idx[axis] = slice(None)
        idx[(axis + 1) % 3] = ja
        idx[(axis + 2) % 3] = jb
        npidx = (idx[2], idx[1], idx[0])
        out = o.sweep_pencil([a[npidx] for a in q], axis, ja, jb, dt, sources=True)
        for v in range(9):
            assert np.array_equal(out[v], qa[v][npidx]), (axis, v)


def test_diagnostics_match_library_sums():
    p = workloads.sphere(n=16)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    tot, prof, mm = o.diagnostics(q, nbins=8, rmax=1.0)
    dV = p.dx ** 3
    ref = [q[0].sum(), q[1].sum(), q[2].sum(), q[3].sum(), q[4].sum(),
           (q[0] * q[5]).sum(), q[5].sum()]
    np.testing.assert_allclose(tot, np.array(ref) * dV, rtol=1e-13, atol=1e-16)
    # shell average of density by numpy bincount
    c = (np.arange(16) + 0.5) * p.dx - 1.0
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    b = np.floor(r / 1.0 * 8).astype(int)
    m = b < 8
    cnt = np.bincount(b[m], minlength=8)
    rs = np.bincount(b[m], weights=q[0][m], minlength=8)
    np.testing.assert_allclose(prof[:, 0], np.where(cnt > 0, rs / np.maximum(cnt, 1), 0), rtol=1e-13)
    assert 0.0 < mm < 1.0


def test_cfl_dt_definition():
    p = workloads.periodic_box(16)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    g = p.gamma
    rho = q[0]
    u = [q[1 + d] / rho for d in range(3)]
    pr = (g - 1) * (q[4] - 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    c = np.sqrt(g * pr / rho)
    s = np.maximum(np.maximum(np.abs(u[0]), np.abs(u[1])), np.abs(u[2])) + c
    assert abs(o.cfl_dt(q, 0.7) - 0.7 * p.dx / s.max()) <= 1e-14


def test_flop_census_is_plausible():
    p = workloads.periodic_box(shape=(64, 4, 4))
    q = workloads.build(p)
    o = oracle.Oracle(p)
    fl, sel = o.count_flops(q, 0, o.cfl_dt(q))
    assert 200 < fl < 3000 and sel > 0


def test_roundoff_sized_perturbations_stay_small():
    """A 1e-7 relative perturbation of the inputs (the size of FP32 storage
    rounding) must not be amplified by switching constraints on and off: the
    smoothness judgment is continuous, so after 20 double steps of the
    periodic box the momentum moves by less than 1e-5 of its maximum and FV
    by less than 1e-7 on average."""
    p = workloads.periodic_box(32)
    q = workloads.build(p)
    rng = np.random.default_rng(0)
    qa = [a.copy() for a in q]
    qb = [a * (1 + 1e-7 * rng.standard_normal(a.shape)) for a in q]
    qb[5] = np.clip(qb[5], 0.0, 1.0)
    o = oracle.Oracle(p)
    for _ in range(20):
        dt = o.cfl_dt(qa)
        o.double_step(qa, dt)
        o.double_step(qb, dt)
    for d in range(3):
        assert np.abs(qa[1 + d] - qb[1 + d]).max() <= 1e-5 * np.abs(qa[1 + d]).max()
    assert np.abs(qa[5] - qb[5]).mean() <= 1e-7
