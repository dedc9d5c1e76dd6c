"""CPU pins of the confining sphere in the FP64 oracle.

Sec. 3: the star is enclosed in an impenetrable, immovable sphere inscribed
in the cubical grid, and gravity drops to zero a few cells before the sphere
so that a simple boundary condition suffices there.  Reading: a cell is
fluid when its centre lies strictly inside the sphere; the fluid cells of a
pencil form one run, which the pass treats as a pencil with reflecting walls
at both ends; solid cells are never updated and never read.

Pins: solid cells are neither changed nor read (two states that differ only
in their solid cells give bit-identical fluid cells and the same dt); the
run of every pencil is the brute-force set of cells inside the sphere; a
hydrostatic star at rest under the tapered gravity stays at rest bit for
bit; mass and rho*FV are conserved to round-off; without gravity the result
is symmetric under axis permutations bit for bit; the single-pencil entry
point agrees with the grid pass.
"""
import copy

import numpy as np
import pytest

import oracle
import workloads


def _copy(q):
    return [a.copy() for a in q]


def _confined(n=20, mach=0.03, sources=True):
    p = workloads.sphere(n=n, mach=mach, confine=True)
    if not sources:
        p.tables.heat = None
        p.tables.damp = None
    return p


def _solid(p):
    """Brute-force solid mask (z, y, x): centre not strictly inside radius."""
    nx, ny, nz = p.shape
    x = p.origin[0] + (np.arange(nx) + 0.5) * p.dx
    y = p.origin[1] + (np.arange(ny) + 0.5) * p.dx
    z = p.origin[2] + (np.arange(nz) + 0.5) * p.dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return ~(X * X + Y * Y + Z * Z < p.confine_r * p.confine_r)


def test_solid_cells_are_never_changed_nor_read():
    p = _confined(20)
    q = workloads.build(p)
    solid = _solid(p)
    assert solid.any() and (~solid).any()
    qa, qb = _copy(q), _copy(q)
    junk = [7.0, 0.3, -0.2, 0.1, 50.0, 0.5, 0.4, -0.4, 0.2]
    for v in range(9):
        qb[v][solid] = junk[v]
    o = oracle.Oracle(p)
    for _ in range(3):
        dta, dtb = o.cfl_dt(qa), o.cfl_dt(qb)
        assert dta == dtb
        o.double_step(qa, dta)
        o.double_step(qb, dtb)
    for v in range(9):
        assert np.array_equal(qa[v][~solid], qb[v][~solid]), v
        assert np.array_equal(qa[v][solid], q[v][solid]), v
        assert np.all(qb[v][solid] == junk[v]), v
    assert not np.array_equal(qa[1][~solid], q[1][~solid])


def test_every_pencil_run_is_the_set_of_cells_inside():
    """One pass with NaN in every solid cell: the fluid cells stay finite and
    change, the solid ones stay NaN (so the runs are exactly the inside)."""
    p = _confined(16, sources=False)
    q = workloads.build(p)
    solid = _solid(p)
    for v in range(9):
        q[v][solid] = np.nan
    o = oracle.Oracle(p)
    dt = o.cfl_dt(q)
    assert np.isfinite(dt) and dt > 0
    for axis in range(3):
        o.sweep(q, axis, 0.5 * dt)
        for v in range(9):
            assert np.isfinite(q[v][~solid]).all(), (axis, v)
            assert np.isnan(q[v][solid]).all(), (axis, v)


def test_confined_hydrostatic_star_stays_at_rest_bitwise():
    p = _confined(20, mach=0.0, sources=False)
    g = p.tables.g
    assert g[-1] == 0.0 and np.abs(g).max() > 0.0  # gravity tapered to zero
    q = workloads.build(p)
    q0 = _copy(q)
    o = oracle.Oracle(p)
    for _ in range(10):
        o.double_step(q, o.cfl_dt(q))
    for v in range(9):
        assert np.array_equal(q[v], q0[v]), v


def test_confined_sphere_conserves_mass_and_fv_content():
    p = _confined(20, sources=False)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    t0, _, _ = o.diagnostics(q)
    for _ in range(10):
        o.double_step(q, o.cfl_dt(q))
    t1, _, _ = o.diagnostics(q)
    for m in (0, 5):
        assert abs(t1[m] - t0[m]) <= 1e-12 * abs(t0[m]), (m, t0[m], t1[m])


def _permute(q, perm):
    np_axes = [2 - perm[2 - ax] for ax in range(3)]
    out = [None] * 9
    for v in (0, 4, 5):
        out[v] = np.ascontiguousarray(np.transpose(q[v], np_axes))
    for d in range(3):
        out[1 + d] = np.ascontiguousarray(np.transpose(q[1 + perm[d]], np_axes))
        out[6 + d] = np.ascontiguousarray(np.transpose(q[6 + perm[d]], np_axes))
    return out


@pytest.mark.parametrize("perm", [(1, 2, 0), (2, 1, 0)])
def test_confined_axis_permutation_symmetry(perm):
    p = _confined(16, sources=False)
    q = workloads.build(p)
    # same state, uniform base and no gravity: the staircase sphere and the
    # pass are then symmetric under relabelling the axes
    pu = copy.copy(p)
    pu.grav = workloads.GRAV_NONE
    pu.tables = workloads._uniform_tables(1.0, 1.0)
    qp = _permute(q, perm)
    o = oracle.Oracle(pu)
    dt = o.cfl_dt(q)
    inv = [perm.index(d) for d in range(3)]
    for axis in (0, 1, 2, 2, 1, 0):
        o.sweep(q, axis, dt)
        o.sweep(qp, inv[axis], dt)
    back = _permute(qp, inv)
    for v in range(9):
        assert np.array_equal(back[v], q[v]), v


def test_confined_pencil_entry_point_matches_grid_pass():
    p = _confined(16)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    dt = o.cfl_dt(q)
    for axis in range(3):
        qa = _copy(q)
        o.sweep(qa, axis, dt, sources=True)
        for ja, jb in ((8, 8), (3, 9), (1, 1)):
            idx = [None] * 3
            idx[axis] = slice(None)
            idx[(axis + 1) % 3] = ja
            idx[(axis + 2) % 3] = jb
            npidx = (idx[2], idx[1], idx[0])
            out = o.sweep_pencil([a[npidx] for a in q], axis, ja, jb, dt, sources=True)
            for v in range(9):
                assert np.array_equal(out[v], qa[v][npidx]), (axis, ja, jb, v)


# --------------------------------------------------------------------------
# Rotation ramp (Sec. 3): a solid-body flow added gradually, once per double
# step, after the last X pass, to the fluid cells.
def test_rotation_increment_closed_form():
    """With dt = 0 the passes change nothing, so one double step adds exactly
    the increment: m += rho*domega*(-y, x, 0), E += m.du + rho|du|^2/2, and
    solid cells keep their values."""
    p = _confined(16, sources=False)
    q = workloads.build(p)
    q0 = _copy(q)
    o = oracle.Oracle(p)
    w = 0.037
    o.set_rotation(w)
    o.double_step(q, 0.0)
    nx, ny, nz = p.shape
    x = p.origin[0] + (np.arange(nx) + 0.5) * p.dx
    y = p.origin[1] + (np.arange(ny) + 0.5) * p.dx
    Z, Y, X = np.meshgrid(np.zeros(nz), y, x, indexing="ij")
    fluid = ~_solid(p)
    rho = q0[0]
    dux, duy = -w * Y, w * X
    ex_mx = q0[1] + rho * dux
    ex_my = q0[2] + rho * duy
    ex_E = q0[4] + (q0[1] * dux + q0[2] * duy) + 0.5 * rho * (dux * dux + duy * duy)
    scale = np.abs(rho * w).max()
    assert np.abs(q[1] - np.where(fluid, ex_mx, q0[1])).max() <= 1e-14 * scale
    assert np.abs(q[2] - np.where(fluid, ex_my, q0[2])).max() <= 1e-14 * scale
    assert np.abs(q[4] - np.where(fluid, ex_E, q0[4])).max() <= 1e-14 * np.abs(q0[4]).max()
    for v in (0, 3, 5, 6, 7, 8):
        assert np.array_equal(q[v], q0[v]), v
    # angular momentum about z grows by domega * sum rho (x^2 + y^2)
    Lz = lambda s: (X * s[2] - Y * s[1])[fluid].sum()
    dL = Lz(q) - Lz(q0)
    assert abs(dL - w * (rho * (X * X + Y * Y))[fluid].sum()) <= 1e-12 * abs(dL)


def test_rotation_only_in_the_last_x_pass():
    """Single passes apply the increment only when asked (sources bit 1)."""
    p = _confined(16, sources=False)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    o.set_rotation(0.02)
    dt = o.cfl_dt(q)
    qa, qb = _copy(q), _copy(q)
    o.sweep(qa, 0, dt, sources=0)
    o.set_rotation(0.0)
    o.sweep(qb, 0, dt, sources=2)
    for v in range(9):
        assert np.array_equal(qa[v], qb[v]), v
