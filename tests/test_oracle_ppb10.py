"""CPU pins of the ten-value PPB in the FP64 oracle (FV, 3 first moments, 3
second moments, 3 mixed moments: the paper's production representation,
Sec. 1 and Sec. 4; each 1-D pass then has a purely local parabola).

Pins: a quadratic profile along the pass and a bilinear profile across it
(first, second and mixed moments) are transported exactly at constant
velocity; a state at rest with arbitrary valid moments stays bit for bit;
rho*FV is conserved to round-off and 0 <= FV <= 1 holds in a compressive
flow; axis permutations give the transposed result bit for bit; a smooth
wave converges at fourth order (measured 4.0 for n = 16..128); the single-pencil entry point agrees with the
grid pass.
"""
import copy

import numpy as np
import pytest

import oracle
import workloads


def _ten(p):
    p = copy.copy(p)
    p.nmom = 9
    return p


def _walls_x_problem(nx, ny, u):
    """Uniform gas moving at u along x between walls, ny periodic rows."""
    p = workloads.tube("sod", n=nx, axis=0, ntrans=4)
    p.shape = (nx, ny, 4)
    p.extra = {}
    p = _ten(p)
    q = [np.zeros((4, ny, nx)) for _ in range(15)]
    q[0][:] = 1.0
    q[1][:] = u
    q[4][:] = 1.0 / (p.gamma - 1.0) + 0.5 * u * u
    return p, q


def _poly_cells(coef, xc, yc, h):
    """Exact cell values of f = a + b x + c y + d x y + e x^2 on cells of size
    h centred at (xc, yc): (FV, m_x, m_y, q_x, c_xy)."""
    a, b, c, d, e = coef
    A = a + b * xc + c * yc + d * xc * yc + e * xc * xc
    B = (b + d * yc + 2.0 * e * xc) * h
    C = (c + d * xc) * h
    D = d * h * h
    E = e * h * h
    return A + E / 12.0, B, C, E, D


@pytest.mark.parametrize("u", [0.3, -0.45])
@pytest.mark.parametrize("coef", [(0.2, 0.9, 0.0, 0.0, -0.6), (0.35, 0.2, 0.15, -0.25, 0.0)])
def test_polynomial_profiles_transport_exactly(u, coef):
    nx, ny = 32, 8
    p, q = _walls_x_problem(nx, ny, u)
    h = 1.0 / nx
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h + 0.1
    X, Y = np.meshgrid(xc, yc)                     # (ny, nx)
    f, mx, my, qx, cxy = _poly_cells(coef, X, Y, h)
    assert f.min() > 0.05 and f.max() < 0.95
    q[5][:] = f
    q[6][:] = mx
    q[7][:] = my
    q[9][:] = qx
    q[14][:] = cxy
    o = oracle.Oracle(p)
    dt = 0.3 / nx / (abs(u) + 1.2)
    oracle.Oracle.reset_counters()
    o.sweep(q, 0, dt)
    s = u * dt
    ef, emx, emy, eqx, ecxy = _poly_cells(coef, X - s, Y, h)
    inner = (slice(None), slice(None), slice(6, nx - 6))
    tol = 1e-13
    np.testing.assert_allclose(q[5][inner], np.broadcast_to(ef, q[5].shape)[inner], rtol=0, atol=tol)
    np.testing.assert_allclose(q[6][inner], np.broadcast_to(emx, q[6].shape)[inner], rtol=0, atol=tol)
    np.testing.assert_allclose(q[7][inner], np.broadcast_to(emy, q[7].shape)[inner], rtol=0, atol=tol)
    np.testing.assert_allclose(q[9][inner], np.broadcast_to(eqx, q[9].shape)[inner], rtol=0, atol=tol)
    np.testing.assert_allclose(q[14][inner], np.broadcast_to(ecxy, q[14].shape)[inner], rtol=0, atol=tol)
    for v in (8, 10, 11, 12, 13):
        assert np.abs(q[v][inner]).max() <= tol, v
    c_ = oracle.Oracle.counters()
    assert c_["fct_limited"] == 0 and c_["theta_limited"] == 0 and c_["moment_clamped"] == 0


def _random_moments(fv, rng, scale=0.3):
    g = fv * (1 - fv)
    out = []
    for d in range(3):
        out.append(scale * 6 * g * rng.uniform(-1, 1, fv.shape))
    for d in range(3):
        out.append(scale * 15 * g * rng.uniform(-1, 1, fv.shape))
    for d in range(3):
        out.append(scale * 36 * g * rng.uniform(-1, 1, fv.shape))
    return out


def _ten_state(p, q, seed=7):
    rng = np.random.default_rng(seed)
    fv = rng.uniform(0.1, 0.9, q[0].shape)
    mom = _random_moments(fv, rng)
    return q[:5] + [fv] + mom


def test_rest_state_with_moments_stays_bitwise():
    p = _ten(workloads.periodic_box(shape=(8, 8, 8), mach=0.0))
    q = _ten_state(p, workloads.build(workloads.periodic_box(shape=(8, 8, 8), mach=0.0)))
    q0 = [a.copy() for a in q]
    o = oracle.Oracle(p)
    for _ in range(10):
        o.double_step(q, o.cfl_dt(q))
    for v in range(15):
        assert np.array_equal(q[v], q0[v]), v


def test_conservation_and_bounds_periodic_box():
    base = workloads.periodic_box(shape=(16, 16, 16), mach=0.3)
    p = _ten(base)
    q = _ten_state(p, workloads.build(base), seed=3)
    o = oracle.Oracle(p)
    tot0 = (q[0] * q[5]).sum()
    for _ in range(5):
        dt = o.cfl_dt(q)
        for axis in (0, 1, 2, 2, 1, 0):
            o.sweep(q, axis, dt)
            assert q[5].min() >= 0.0 and q[5].max() <= 1.0
            g = q[5] * (1 - q[5])
            for d in range(3):
                assert np.all(np.abs(q[6 + d]) <= 6 * g + 1e-15)
                assert np.all(q[9 + d] <= 15 * g * (2 - q[5]) + 1e-15)
                assert np.all(q[9 + d] >= -15 * g * (1 + q[5]) - 1e-15)
                assert np.all(np.abs(q[12 + d]) <= 36 * g + 1e-15)
    tot1 = (q[0] * q[5]).sum()
    assert abs(tot1 - tot0) <= 1e-12 * tot0


def _permute(q, perm):
    np_axes = [2 - perm[2 - ax] for ax in range(3)]
    out = [None] * 15
    for v in (0, 4, 5):
        out[v] = np.ascontiguousarray(np.transpose(q[v], np_axes))
    for d in range(3):
        for base in (1, 6, 9, 12):
            out[base + d] = np.ascontiguousarray(np.transpose(q[base + perm[d]], np_axes))
    return out


@pytest.mark.parametrize("perm", [(1, 2, 0), (2, 1, 0)])
def test_axis_permutation_symmetry(perm):
    shape = (8, 8, 8)
    base = workloads.periodic_box(shape=shape)
    p = _ten(base)
    q = _ten_state(p, workloads.build(base), seed=11)
    qp = _permute(q, perm)
    o = oracle.Oracle(p)
    dt = o.cfl_dt(q)
    inv = [perm.index(d) for d in range(3)]
    for axis in (0, 1, 2, 2, 1, 0):
        o.sweep(q, axis, dt)
        o.sweep(qp, inv[axis], dt)
    back = _permute(qp, inv)
    for v in range(15):
        assert np.array_equal(back[v], q[v]), v


def _gl_cells(f, n, npt=8):
    """(FV, m, q) of f on the n cells of [0, 1) by Gauss-Legendre quadrature."""
    xg, wg = np.polynomial.legendre.leggauss(npt)
    xg, wg = 0.5 * xg, 0.5 * wg
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    F = sum(w * f(xc + x * h) for x, w in zip(xg, wg))
    M = 12 * sum(w * x * f(xc + x * h) for x, w in zip(xg, wg))
    Q = 180 * sum(w * (x * x - 1.0 / 12) * f(xc + x * h) for x, w in zip(xg, wg))
    return F, M, Q


def _wave_error(n):
    base = workloads.wave(n=n, axis=0, kind="fv", u=1.0)
    p = _ten(base)
    q = workloads.build(base) + [np.zeros((4, 4, n)) for _ in range(6)]
    f = lambda x: 0.5 + 0.3 * np.sin(2 * np.pi * x)
    F, M, Q = _gl_cells(f, n)
    q[5][:] = F
    q[6][:] = M
    q[9][:] = Q
    o = oracle.Oracle(p)
    T, t = 0.5, 0.0
    dt = 0.4 / n
    while t < T - 1e-14:
        step = min(dt, T - t)
        o.sweep(q, 0, step)
        t += step
    Fe, _, _ = _gl_cells(lambda x: f(x - T), n)
    return np.abs(q[5][0, 0] - Fe).mean()


def test_smooth_wave_converges_at_fourth_order():
    e = [_wave_error(n) for n in (16, 32, 64)]
    orders = [np.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) >= 3.7, (e, orders)


def test_pencil_entry_point_matches_grid_pass():
    base = workloads.periodic_box(shape=(12, 10, 8))
    p = _ten(base)
    q = _ten_state(p, workloads.build(base), seed=5)
    o = oracle.Oracle(p)
    dt = o.cfl_dt(q)
    for axis in range(3):
        qa = [a.copy() for a in q]
        o.sweep(qa, axis, dt)
        ja, jb = 3, 5
        idx = [None] * 3
        idx[axis] = slice(None)
        idx[(axis + 1) % 3] = ja
        idx[(axis + 2) % 3] = jb
        npidx = (idx[2], idx[1], idx[0])
        out = o.sweep_pencil([a[npidx] for a in q], axis, ja, jb, dt)
        for v in range(15):
            assert np.array_equal(out[v], qa[v][npidx]), (axis, v)
