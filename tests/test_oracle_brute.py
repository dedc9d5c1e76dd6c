"""Brute-force cross-check of the oracle's pencil machinery.

`brute_pass.sweep` restates one PPM+PPB pass, four-value and ten-value, with
the optional 3-D shock dissipation, and `brute_pass.sweep_confined` the pass
inside the confining sphere (Sec. 1: interface
values, smoothness weights, flattening, constrained parabolas, tracing with
half-step buoyancy, two-shock Riemann solve, fluxes and gravity sources in
deviation form, PPB profiles, swept-slab transfers, FCT, moment update) as
whole-grid numpy array arithmetic: every pencil at once, ghost cells by index
arrays, the base state by vectorised table lookups.  It shares no code with
the C++ oracle, which works one pencil at a time with its own gather, ghost
mapping and loops.  Both evaluate the same expressions in the same order
without fused multiply-adds, so the pass must agree bit for bit: any slip in
the oracle's indexing (a ghost mirrored one cell off, a face base state taken
at the wrong position, a stencil shifted by one, an axis permutation) shows.

Inputs are made to reach every branch: random volume fractions with cells
pinned at exactly 0 and 1 (FCT and theta limiting active), a Sod tube
(flattening and constraints active), plane gravity with reflecting walls,
random flows at Mach ~3 (faces whose two-shock waves both move one way, so
the upwind traced state is the interface state).  The FCT limiter is not
required to fire: with the interface state sampled at x/t = 0 it fired in
none of the finite states tried (random flows at Mach 0.1-3, density
contrasts up to 100, contacts advected at uniform velocity); it is pinned by
the bounds pin and by the GPU parity of the same expressions.
"""
import copy

import numpy as np
import pytest

import brute_pass
import oracle
import workloads


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _rough_fv(q, seed):
    """Random volume fractions, a fifth of the cells exactly 0 or 1, and
    random first moments inside the realisable range |m| <= 6 FV (1 - FV)."""
    rng = np.random.default_rng(seed)
    fv = rng.uniform(0.0, 1.0, q[0].shape)
    pick = rng.uniform(0.0, 1.0, fv.shape)
    fv[pick < 0.1] = 0.0
    fv[pick > 0.9] = 1.0
    g = 6.0 * fv * (1.0 - fv)
    q = list(q[:5]) + [fv] + [0.8 * g * rng.uniform(-1.0, 1.0, fv.shape) for _ in range(3)]
    return q


def _rough_flow(p, q, seed, amp, pres, rho_range=(0.7, 1.4)):
    """Cell-to-cell random density (x rho_range), velocity (|u_d| <= amp) and
    pressure (pres x 0.5..2): discontinuous everywhere, so that every cell
    takes the constrained branches and strong compressions reach the FCT
    limiter.  Only single passes are taken from it (a second pass may meet a
    negative traced pressure, which PPM does not exclude)."""
    rng = np.random.default_rng(seed)
    q = [a.copy() for a in q]
    rho = q[0] * rng.uniform(rho_range[0], rho_range[1], q[0].shape)
    u = [amp * rng.uniform(-1.0, 1.0, rho.shape) for _ in range(3)]
    pr = pres * rng.uniform(0.5, 2.0, rho.shape)
    q[0] = rho
    for d in range(3):
        q[1 + d] = rho * u[d]
    q[4] = pr / (p.gamma - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    return q


def _evolved(p, q, steps):
    o = oracle.Oracle(p)
    for _ in range(steps):
        o.double_step(q, o.cfl_dt(q, p.cfl))
    return q


def _shock_box(n=16):
    """Periodic box whose sinusoidal velocity field steepens into shocks,
    evolved 8 double steps with the 3-D dissipation on."""
    p = workloads.periodic_box(shape=(n, n, n), mach=0.0)
    p.shock_k = 0.1
    q = workloads.build(p)
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    q[1] += 0.9 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    q[2] += 0.9 * np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * Z)
    q[3] += 0.9 * np.sin(2 * np.pi * Z)
    q[4] += 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0]
    o = oracle.Oracle(p)
    for _ in range(8):
        o.double_step(q, o.cfl_dt(q, 0.5))
    return p, q


def _cases():
    box = workloads.periodic_box(shape=(8, 6, 10), mach=0.3)
    strat = workloads.strat_box(shape=(8, 6, 12))
    sod = workloads.tube("sod", n=16, axis=0, ntrans=6)
    out = [
        # (name, problem, state builder, passes in sequence, counters that must be > 0)
        ("box", box, lambda: workloads.build(box), 2, ("theta_limited", "moment_clamped")),
        ("strat", strat, lambda: workloads.build(strat), 2, ("theta_limited", "nonsmooth")),
        ("sod_evolved", sod, lambda: _evolved(sod, workloads.build(sod), 4), 2,
         ("flattened", "nonsmooth", "theta_limited")),
        ("box_rough", box, lambda: _rough_flow(box, workloads.build(box), 1, 1.0, 0.05), 1,
         ("flattened", "nonsmooth", "supersonic_faces")),
        ("strat_rough", strat, lambda: _rough_flow(strat, workloads.build(strat), 2, 0.7, 0.1), 1,
         ("flattened", "nonsmooth")),
    ]
    shock_p, shock_q = _shock_box()
    sod_k = copy.copy(sod)
    sod_k.shock_k = 0.1
    out += [
        # 3-D shock dissipation: a periodic box after its shocks formed, and
        # an evolved Sod tube between walls
        ("shock_box", shock_p, lambda: [a.copy() for a in shock_q], 2, ("dissipative_faces", "flattened")),
        ("sod_shock", sod_k, lambda: _evolved(sod_k, workloads.build(sod_k), 4), 2, ("dissipative_faces",)),
    ]
    return out


@pytest.mark.parametrize("name,p,make,npass,active", _cases(), ids=[c[0] for c in _cases()])
def test_whole_grid_pass_matches_pencil_oracle(name, p, make, npass, active):
    q0 = _rough_fv(make(), seed=len(name))
    o = oracle.Oracle(p)
    oracle.Oracle.reset_counters()
    for axis in range(3):
        # npass passes along axis, axis+1, ..., each on the previous result
        qo = [a.copy() for a in q0]
        qb = [a.copy() for a in q0]
        for k in range(npass):
            ax = (axis + k) % 3
            dt = o.cfl_dt(qo, p.cfl)
            o.sweep(qo, ax, dt)
            qb = brute_pass.sweep(p, qb, ax, dt)
            for v in range(9):
                assert np.isfinite(qo[v]).all(), (name, axis, ax, v)
                assert np.array_equal(qb[v], qo[v]), (name, axis, ax, v,
                                                      np.abs(qb[v] - qo[v]).max())
    c = oracle.Oracle.counters()
    for key in active:
        assert c[key] > 0, (key, c)


def _ten_moments(q, seed):
    """Second and mixed moments (seeded) inside their realisable ranges:
    -15 g (1 + FV) <= q_d <= 15 g (2 - FV), |c_de| <= 36 g, g = FV (1 - FV)."""
    rng = np.random.default_rng(seed)
    fv = q[5]
    g = fv * (1.0 - fv)
    qs = [7.5 * g * rng.uniform(-1.0, 1.0, fv.shape) for _ in range(3)]
    cs = [20.0 * g * rng.uniform(-1.0, 1.0, fv.shape) for _ in range(3)]
    return list(q[:9]) + qs + cs


def _ten_cases():
    out = []
    for name, p, make, npass, active in _cases():
        if name in ("box", "strat", "box_rough"):
            p10 = copy.copy(p)
            p10.nmom = 9
            out.append((name + "_ten", p10, make, npass, tuple(k for k in active if k != "flattened")))
    return out


@pytest.mark.parametrize("name,p,make,npass,active", _ten_cases(), ids=[c[0] for c in _ten_cases()])
def test_whole_grid_ten_value_pass_matches_pencil_oracle(name, p, make, npass, active):
    """The same cross-check for the ten-value form (FV, 3 first, 3 second and
    3 mixed moments): the swept-slab second moments, the transverse
    xi-moments and the second-moment and mixed-moment updates."""
    q0 = _ten_moments(_rough_fv(make(), seed=len(name)), seed=len(name) + 1)
    o = oracle.Oracle(p)
    oracle.Oracle.reset_counters()
    for axis in range(3):
        qo = [a.copy() for a in q0]
        qb = [a.copy() for a in q0]
        for k in range(npass):
            ax = (axis + k) % 3
            dt = o.cfl_dt(qo, p.cfl)
            o.sweep(qo, ax, dt)
            qb = brute_pass.sweep(p, qb, ax, dt)
            for v in range(15):
                assert np.isfinite(qo[v]).all(), (name, axis, ax, v)
                assert np.array_equal(qb[v], qo[v]), (name, axis, ax, v,
                                                      np.abs(qb[v] - qo[v]).max())
    c = oracle.Oracle.counters()
    for key in active:
        assert c[key] > 0, (key, c)


@pytest.mark.parametrize("shape,min_run", [((24, 24, 24), 4), ((22, 19, 26), 2), ((21, 23, 25), 3)])
def test_whole_grid_confined_pass_matches_pencil_oracle(shape, min_run):
    """The confining sphere (Sec. 3) with central gravity tapered inside it:
    pencils batched by their fluid run, each run a pencil with walls at both
    ends and period-2n folded ghosts (runs of 2 and 3 cells at the rim included),
    base state at mirrored cells and folded faces from the radial tables."""
    p = workloads.sphere(shape=shape, confine=True)
    q0 = _rough_fv(workloads.build(p), seed=sum(shape))
    o = oracle.Oracle(p)
    xs = [p.origin[d] + (np.arange(p.shape[d]) + 0.5) * p.dx for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    fluid = (X * X + Y * Y) + Z * Z < p.confine_r ** 2
    shortest = min(int(fluid.sum(axis=a)[fluid.sum(axis=a) > 0].min()) for a in range(3))
    assert shortest == min_run                      # runs shorter than the stencil at the rim
    for axis in range(3):
        qo = [a.copy() for a in q0]
        qb = [a.copy() for a in q0]
        for k in range(2):
            ax = (axis + k) % 3
            dt = o.cfl_dt(qo, p.cfl)
            o.sweep(qo, ax, dt)
            qb = brute_pass.sweep_confined(p, qb, ax, dt)
            for v in range(9):
                assert np.array_equal(qb[v], qo[v]), (shape, axis, ax, v, np.abs(qb[v] - qo[v]).max())


@pytest.mark.parametrize("sources,domega", [(0, 0.0), (1, 0.0), (3, 0.01)])
@pytest.mark.parametrize("confine", [False, True])
def test_whole_grid_sphere_pass_with_sources_matches_pencil_oracle(sources, domega, confine):
    """The benchmark's workload: the sphere in the cube with central gravity
    and reflecting walls (or confined), with the heating and damping (bit 0)
    and the rotation increment (bit 1) applied after the pass."""
    p = workloads.sphere(shape=(20, 18, 22), confine=confine)
    q0 = _rough_fv(workloads.build(p), seed=7)
    o = oracle.Oracle(p)
    o.set_rotation(domega)
    step = brute_pass.sweep_confined if confine else brute_pass.sweep
    for axis in range(3):
        qo = [a.copy() for a in q0]
        dt = o.cfl_dt(qo, p.cfl)
        o.sweep(qo, axis, dt, sources=sources)
        qb = step(p, [a.copy() for a in q0], axis, dt, sources=sources, domega=domega)
        for v in range(9):
            assert np.array_equal(qb[v], qo[v]), (axis, v, np.abs(qb[v] - qo[v]).max())


def test_whole_grid_double_step_matches_pencil_oracle():
    """Strang double step (Sec. 1 / Sec. 4 directional splitting): X Y Z,
    heating and damping after that Z pass, then Z Y X with heating, damping
    and the rotation increment after the last X pass, one dt."""
    p = workloads.sphere(shape=(20, 18, 22))
    q = _rough_fv(workloads.build(p), seed=11)
    o = oracle.Oracle(p)
    o.set_rotation(0.02)
    qo = [a.copy() for a in q]
    dt = o.cfl_dt(qo, p.cfl)
    o.double_step(qo, dt)
    qb = [a.copy() for a in q]
    for axis, src in ((0, 0), (1, 0), (2, 1), (2, 0), (1, 0), (0, 3)):
        qb = brute_pass.sweep(p, qb, axis, dt, sources=src, domega=0.02)
    for v in range(9):
        assert np.array_equal(qb[v], qo[v]), (v, np.abs(qb[v] - qo[v]).max())
