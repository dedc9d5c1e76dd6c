"""CPU pins of the oracle's gravity terms against what the mechanics fixes.

The perturbation form (Sec. 1: the hydrostatic initial state is removed from
the scheme) carries gravity in three places: half a step of the buoyancy
acceleration (rho'/rho) g added to the traced normal velocity, the momentum
source dt g rho' (rho' time-centred) and the energy source dt g times the
time-centred face mass flux.  A state at rest in the base state makes all
three vanish, so the rest-state pins cannot see them.  These pins can:

* impulse: a slab of heavier gas (rho' = eps rho0, p' = 0) at rest in a
  polytropic layer under constant g.  After one z pass of length dt its
  interior carries the momentum rho' g dt (Newton's second law; the pressure
  is still uniform there), so the sign and the factor of the momentum source
  are fixed;
* the mass flux of the accelerating slab: the interior velocity grows as
  a t with a = (rho'/rho) g, so over the pass the gas moves by a dt^2 / 2 and
  the interior density changes by -(1/2) eps g dt^2 d(rho0)/dz (continuity
  with a uniform velocity).  The displacement is carried by the half-step
  buoyancy alone (the velocity is zero at the start of the pass), so its sign
  and its factor one half are fixed;
* energy: with constant g and walls, total energy plus gravitational
  potential energy is conserved, sum E - g sum z rho = const (g signed along
  +z), for any state, pass by pass.  In the scheme this holds only when the
  energy source has the sign and the time-centred mass flux it has.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def _layer(shape):
    """n = 1.5 polytropic layer, gravity -1.25 z_hat, no light fluid, no
    heating or damping; periodic x, y and reflecting z walls."""
    p = workloads.strat_box(shape=shape, mu_ratio=1.0, heat_rate=0.0, noise=0.0)
    p.tables.heat = None
    p.tables.damp = None
    return p


def _base_at(p, z):
    t = p.tables
    s = (z - t.s0) / t.ds
    i = np.clip(np.floor(s).astype(int), 0, t.n - 2)
    w = s - i
    return (t.rho0[i] + w * (t.rho0[i + 1] - t.rho0[i]), t.p0[i] + w * (t.p0[i + 1] - t.p0[i]))


def _slab_state(p, eps, ka, kb):
    nx, ny, nz = p.shape
    z = p.origin[2] + (np.arange(nz) + 0.5) * p.dx
    rho0, p0 = _base_at(p, z)
    rho = np.repeat(rho0[:, None, None], ny, 1).repeat(nx, 2)
    rho[ka:kb] *= (1.0 + eps)
    q = [np.zeros((nz, ny, nx)) for _ in range(9)]
    q[0] = rho.copy()
    q[4] = np.repeat((p0 / (p.gamma - 1.0))[:, None, None], ny, 1).repeat(nx, 2)
    return q, z, rho0


def _one_pass(eps):
    p = _layer((4, 4, 96))
    ka, kb = 24, 72
    q, z, rho0 = _slab_state(p, eps, ka, kb)
    q0 = [a.copy() for a in q]
    c = np.sqrt(p.gamma * _base_at(p, z)[1] / rho0).max()
    dt = 0.5 * p.dx / c
    oracle.Oracle(p).sweep(q, 2, dt, 0)
    g = float(p.tables.g[0])
    inner = slice(ka + 6, kb - 6)
    return p, q0, q, z, rho0, dt, g, inner


@pytest.mark.parametrize("eps", [1e-4, -1e-4])
def test_impulse_of_a_buoyant_slab(eps):
    """Momentum after one z pass equals rho' g dt (to O(dt^2, eps))."""
    p, q0, q, z, rho0, dt, g, inner = _one_pass(eps)
    rho_p = (q0[0] - rho0[:, None, None])[inner]
    expect = rho_p * g * dt
    got = q[3][inner]
    assert np.all(np.sign(got) == np.sign(expect))
    np.testing.assert_allclose(got, expect, rtol=2e-3)
    # nothing moves sideways
    assert np.abs(q[1]).max() == 0.0 and np.abs(q[2]).max() == 0.0


@pytest.mark.parametrize("eps", [1e-4, -1e-4])
def test_half_step_buoyancy_moves_the_slab(eps):
    """Interior density change after one z pass equals -(1/2) eps g dt^2
    d(rho0)/dz, the centred difference of rho0 across the cell taken from
    the table at the faces."""
    p, q0, q, z, rho0, dt, g, inner = _one_pass(eps)
    rlo, _ = _base_at(p, z - 0.5 * p.dx)
    rhi, _ = _base_at(p, z + 0.5 * p.dx)
    drho0 = ((rhi - rlo) / p.dx)[:, None, None]
    expect = (-0.5 * eps * g * dt * dt * drho0 * np.ones_like(q[0]))[inner]
    got = (q[0] - q0[0])[inner]
    assert np.abs(expect).min() > 1e-12
    np.testing.assert_allclose(got, expect, rtol=1e-2)


def _rough_layer_state(p, seed):
    g = np.random.default_rng(seed)
    nx, ny, nz = p.shape
    z = p.origin[2] + (np.arange(nz) + 0.5) * p.dx
    rho0, p0 = _base_at(p, z)
    shp = (nz, ny, nx)
    rho = rho0[:, None, None] * (1.0 + 0.05 * g.uniform(-1, 1, shp))
    c = np.sqrt(p.gamma * p0 / rho0)[:, None, None]
    u = [0.1 * c * g.uniform(-1, 1, shp) for _ in range(3)]
    u[2][0] = u[2][-1] = 0.0
    pr = p0[:, None, None] * (1.0 + 0.01 * g.uniform(-1, 1, shp))
    q = [np.zeros(shp) for _ in range(9)]
    q[0] = rho
    for d in range(3):
        q[1 + d] = rho * u[d]
    q[4] = pr / (p.gamma - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    q[5] = np.full(shp, 0.3)
    return q, z


@pytest.mark.parametrize("axis_order", ["z", "double"])
def test_energy_plus_potential_energy_conserved(axis_order):
    """sum(E) - g sum(z rho) is unchanged by every pass of a closed layer
    under constant gravity: after single z passes and after double steps."""
    p = _layer((8, 8, 32))
    q, z = _rough_layer_state(p, 11)
    o = oracle.Oracle(p)
    g = float(p.tables.g[0])
    zz = z[:, None, None]
    E0, Z0 = q[4].sum(), (zz * q[0]).sum()
    for _ in range(6):
        dt = o.cfl_dt(q, 0.5)
        if axis_order == "z":
            o.sweep(q, 2, dt, 0)
        else:
            o.double_step(q, dt)
    dE, dZ = q[4].sum() - E0, (zz * q[0]).sum() - Z0
    # the state is far from rest: both changes are well above rounding
    assert abs(dE) > 1e-6 * abs(E0)
    assert abs(dE - g * dZ) <= 1e-9 * abs(dE)


def _isothermal_layer(nx, nz, lx=2.0, lz=1.0, gamma=5.0 / 3.0):
    """Isothermal layer rho0 = p0 = exp(-z) under g = -1 (scale height 1),
    periodic in x and y, rigid lids at z = 0 and z = lz."""
    dz = lz / nz
    ds = dz / 16.0
    s = np.arange(-8 * 16, (nz + 8) * 16 + 1) * ds
    tab = workloads.Tables(s0=float(s[0]), ds=ds, rho0=np.exp(-s), p0=np.exp(-s), g=-np.ones_like(s))
    return workloads.Problem("isothermal_layer", (nx, 4, nz), (0.0, 0.0, 0.0), dz, gamma,
                             (0, 0, 0, 0, 1, 1), workloads.GRAV_PLANE_Z, tab, cfl=0.7)


def test_internal_gravity_wave_frequency():
    """A standing internal gravity wave (k_x = pi over x in [0, 2], the
    first vertical mode between the lids) oscillates at the gravity branch of
    the exact dispersion relation of an isothermal atmosphere,
    w^4 - w^2 c^2 (k^2 + 1/(4 H^2)) + N^2 c^2 k_x^2 = 0, with N^2 = (g/H)(1 - 1/gamma):
    w = 0.4457 here (measured 0.4452 from the zero crossings of the mode's
    momentum; bound 1%).
    Without the buoyancy (or with its sign reversed) there is no such
    oscillation; a wrong factor shifts the frequency."""
    nx, nz = 64, 32
    p = _isothermal_layer(nx, nz)
    gam, g0, H = p.gamma, 1.0, 1.0
    kx, kz = math.pi, math.pi
    c2 = gam * g0 * H
    N2 = (g0 / H) * (1.0 - 1.0 / gam)
    bq = c2 * (kx * kx + kz * kz + 0.25 / H ** 2)
    w_exact = math.sqrt(0.5 * (bq - math.sqrt(bq * bq - 4.0 * N2 * c2 * kx * kx)))
    # the gravity mode's velocity (anelastic form of its eigenvector), rho' = p' = 0
    x = (np.arange(nx) + 0.5) * p.dx
    z = (np.arange(nz) + 0.5) * p.dx
    Z, X = np.meshgrid(z, x, indexing="ij")
    rho0 = np.exp(-Z)
    amp = 1e-4
    mw = amp * np.exp(-0.5 * Z) * np.sin(kz * Z) * np.cos(kx * X)                  # rho0 w
    mu = -amp / kx * np.sin(kx * X) * np.exp(-0.5 * Z) * (kz * np.cos(kz * Z) - 0.5 * np.sin(kz * Z))
    q = [np.zeros((nz, 4, nx)) for _ in range(9)]
    q[0][:] = rho0[:, None, :]
    q[1][:] = mu[:, None, :]
    q[3][:] = mw[:, None, :]
    q[4][:] = (np.exp(-Z) / (gam - 1.0) + 0.5 * (mu ** 2 + mw ** 2) / rho0)[:, None, :]
    shape_w = (np.sin(kz * Z) * np.cos(kx * X) * np.exp(-0.5 * Z))[:, None, :]
    o = oracle.Oracle(p)
    dt = 0.5 * o.cfl_dt(q, 0.7)
    t, ts, P = 0.0, [0.0], [float((q[3] * shape_w).sum())]
    while t < 1.7 * math.pi / w_exact:
        o.double_step(q, dt)
        t += 2.0 * dt
        ts.append(t)
        P.append(float((q[3] * shape_w).sum()))
    ts, P = np.array(ts), np.array(P)
    # the sound waves the start also excites are fast (period ~1) and small:
    # smooth over one of their periods, then take the zero crossings
    k = max(1, int(round(2.0 * math.pi / math.sqrt(bq) / (2.0 * dt))))
    Ps = np.convolve(P, np.ones(k) / k, mode="valid")
    tsm = np.convolve(ts, np.ones(k) / k, mode="valid")
    sgn = np.sign(Ps)
    idx = np.where(sgn[1:] * sgn[:-1] < 0)[0]
    assert len(idx) >= 2, "no oscillation"
    tz = [tsm[i] - Ps[i] * (tsm[i + 1] - tsm[i]) / (Ps[i + 1] - Ps[i]) for i in idx[:2]]
    w_meas = math.pi / (tz[1] - tz[0])
    assert abs(w_meas - w_exact) <= 0.01 * w_exact, (w_meas, w_exact)
    # and it stays a small oscillation (no growth)
    assert np.abs(P).max() <= 1.5 * abs(P[0])
