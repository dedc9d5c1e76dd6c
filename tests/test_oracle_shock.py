"""CPU pins of the 3-D shock dissipation in the FP64 oracle.

Sec. 1: in flows with shocks the method adds a fully 3-D dissipation inside
shocks, against multi-dimensional grid imprint (details in a reference not
available here).  Reading: in every pass, momentum and E' diffuse across a
face with nu = K max(0, -div(u) dx - 0.05 c), div(u) the 3-D velocity
divergence (central differences) of the pass's input state averaged to the
face; mass is not diffused.

Pins: the divergence operator is exact for linear velocity fields; states at
rest (uniform, hydrostatic) and a Mach-0.03 flow are bit-identical with and
without the dissipation (it never switches on there); mass, momentum and
energy are conserved to round-off in a periodic box with forming shocks
while it is active; shock tubes still converge to the exact solution and
give identical results along every axis; it acts only at the shock.
"""
import copy

import numpy as np
import pytest

import oracle
import workloads
from exact_riemann import cell_averages


def _with_k(p, k=0.1):
    p = copy.copy(p)
    p.shock_k = k
    return p


def test_divergence_exact_for_linear_velocity():
    p = workloads.tube("sod", n=16, axis=0)
    p.shape = (16, 12, 10)
    p.bc = (1,) * 6
    q = [np.zeros((10, 12, 16)) for _ in range(9)]
    a, b, c = 0.3, -0.7, 0.45
    h = p.dx
    x = (np.arange(16) + 0.5) * h
    y = (np.arange(12) + 0.5) * h
    z = (np.arange(10) + 0.5) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    rho = 1.0 + 0.2 * np.sin(3 * X + 2 * Y + Z)
    q[0][:] = rho
    q[1][:] = rho * a * (X - 0.3)
    q[2][:] = rho * b * (Y - 0.2)
    q[3][:] = rho * c * (Z - 0.1)
    q[4][:] = 2.5
    D = oracle.Oracle(_with_k(p)).divergence(q)
    np.testing.assert_allclose(D[1:-1, 1:-1, 1:-1], a + b + c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("maker", ["uniform", "hydro_strat", "hydro_sphere", "mach003"])
def test_no_effect_where_there_is_no_shock(maker):
    if maker == "uniform":
        p = workloads.periodic_box(shape=(8, 8, 8), mach=0.0)
    elif maker == "hydro_strat":
        p = workloads.strat_box(shape=(8, 6, 24), noise=0.0)
        p.tables.heat = p.tables.damp = None
    elif maker == "hydro_sphere":
        p = workloads.sphere(n=16, mach=0.0)
        p.tables.heat = p.tables.damp = None
    else:
        p = workloads.periodic_box(shape=(16, 16, 16))
    q = workloads.build(p)
    qa, qb = [a.copy() for a in q], [a.copy() for a in q]
    o, ok = oracle.Oracle(p), oracle.Oracle(_with_k(p))
    oracle.Oracle.reset_counters()
    for _ in range(5):
        dt = o.cfl_dt(qa)
        o.double_step(qa, dt)
        ok.double_step(qb, dt)
    assert oracle.Oracle.counters()["dissipative_faces"] == 0
    for v in range(9):
        assert np.array_equal(qa[v], qb[v]), v


def test_conservation_with_forming_shocks():
    p = _with_k(workloads.periodic_box(shape=(16, 16, 16), mach=0.0))
    q = workloads.build(p)
    x = (np.arange(16) + 0.5) / 16
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    q[1] += 0.9 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    q[2] += 0.9 * np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * Z)
    q[3] += 0.9 * np.sin(2 * np.pi * Z)
    q[4] += 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0]
    o = oracle.Oracle(p)
    t0, _, _ = o.diagnostics(q)
    oracle.Oracle.reset_counters()
    for _ in range(8):
        o.double_step(q, o.cfl_dt(q, 0.5))
    t1, _, _ = o.diagnostics(q)
    assert oracle.Oracle.counters()["dissipative_faces"] > 0
    assert abs(t1[0] - t0[0]) <= 1e-12 * abs(t0[0])
    assert abs(t1[4] - t0[4]) <= 1e-12 * abs(t0[4])
    pscale = np.abs(q[1]).sum() * p.dx ** 3
    for m in (1, 2, 3):
        assert abs(t1[m] - t0[m]) <= 1e-12 * pscale, m


def _tube_error(kind, n, axis):
    length = 2.0 if kind == "lax" else 1.0
    p = _with_k(workloads.tube(kind, n=n, axis=axis, length=length))
    q = workloads.build(p)
    o = oracle.Oracle(p)
    L, R, T = workloads.TUBE_STATES[kind]
    t = 0.0
    oracle.Oracle.reset_counters()
    steps = 0
    while t < T - 1e-14:
        dt = min(o.cfl_dt(q, 0.6), 0.5 * (T - t))
        o.double_step(q, dt)
        t += 2 * dt
        steps += 1
    c = oracle.Oracle.counters()
    sl = [0, 0, 0]
    sl[2 - axis] = slice(None)
    N = p.shape[axis]
    edges = p.origin[axis] + np.arange(N + 1) * p.dx
    ex = cell_averages(L, R, 1.4, 0.5, T, edges)
    win = (edges[:-1] >= -1e-12) & (edges[1:] <= 1 + 1e-12)
    rho = q[0][tuple(sl)]
    return np.abs(rho - ex[0])[win].mean(), c, rho, steps


@pytest.mark.parametrize("kind", ["sod", "lax"])
def test_shock_tubes_converge_with_dissipation(kind):
    e1, c1, _, steps = _tube_error(kind, 100, 0)
    e2, _, _, _ = _tube_error(kind, 400, 0)
    assert c1["dissipative_faces"] > 0
    assert np.log(e1 / e2) / np.log(4.0) >= 0.8, (e1, e2)
    # it acts at the shock only: a few faces of each 100-cell pencil
    assert c1["dissipative_faces"] <= 0.06 * c1["cells"], c1


def test_shock_tube_identical_along_axes():
    ref = _tube_error("sod", 100, 0)[2]
    for axis in (1, 2):
        assert np.array_equal(_tube_error("sod", 100, axis)[2], ref), axis
