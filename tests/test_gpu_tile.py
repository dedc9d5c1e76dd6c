"""GPU parity of the tile form of the FP32 pass (PPM_PASS_TILE: cell-parallel
8 x 32 tiles, stages joined by shared-memory rings, TMA copies) against the
FP64 oracle, at the FP32 tolerances, on the same seeded inputs as the
register-window form: periodic box, ragged gravity problems (several tiles
and a partial last tile in x, chunks with a ragged tail along every pass),
the 128^3 stratified box at full size, smallest grids with walls and
periodic faces, supersonic faces; plus the exact states (uniform flow,
hydrostatic layer and sphere) bit for bit, the graph step against six single
passes bit for bit, the CFL maximum fused into the last pass, and the
contexts the tile form does not apply to.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1810_13416_gb300 as ppm
import workloads
from parity_f32 import assert_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ppm.build()
    oracle.build()


def _tile_ctx(p):
    ctx = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    assert ctx.tile_available
    ctx.set_pass_design(ppm.PASS_TILE)
    assert ctx.pass_design == ppm.PASS_TILE
    return ctx


def _run_pair(p, steps, q0=None):
    q = workloads.build(p) if q0 is None else [a.copy() for a in q0]
    qo = [a.copy() for a in q]
    o = oracle.Oracle(p)
    with _tile_ctx(p) as ctx:
        ctx.set_state(q)
        for _ in range(steps):
            dt = o.cfl_dt(qo, p.cfl)
            o.double_step(qo, dt)
            ctx.step(dt)
        qg = ctx.get_state()
    return qg, qo


def test_periodic_box_20_steps():
    p = workloads.periodic_box(32)
    qg, qo = _run_pair(p, 20)
    assert_f32(qg, qo, "tile periodic 32")


@pytest.mark.parametrize("make", [lambda: workloads.strat_box(shape=(148, 20, 36)),
                                  lambda: workloads.sphere(shape=(44, 36, 40)),
                                  lambda: workloads.strat_box(shape=(36, 70, 33))],
                         ids=["strat148", "sphere44", "strat36x70x33"])
def test_gravity_problems(make):
    p = make()
    qg, qo = _run_pair(p, 8)
    assert_f32(qg, qo, "tile gravity")


def test_stratified_box_128_full_size_20_steps():
    p = workloads.strat_box(shape=(128, 128, 128))
    qg, qo = _run_pair(p, 20)
    assert_f32(qg, qo, "tile strat 128")


@pytest.mark.parametrize("shape", [(4, 4, 4), (8, 8, 8), (4, 9, 5), (12, 33, 40)])
@pytest.mark.parametrize("bc", ["periodic", "walls"])
def test_smallest_and_ragged_grids(shape, bc):
    if bc == "periodic":
        p = workloads.periodic_box(shape=shape)
    else:
        p = workloads.strat_box(shape=shape)
    qg, qo = _run_pair(p, 4)
    assert_f32(qg, qo, f"tile {bc} {shape}")


def test_uniform_state_preserved_bitwise():
    p = workloads.periodic_box(shape=(8, 12, 16))
    q = [np.zeros((16, 12, 8)) for _ in range(9)]
    q[0][:] = 1.0
    vel = (0.25, -0.125, 0.375)
    for d in range(3):
        q[1 + d][:] = vel[d]
    q[4][:] = 0.75 / (p.gamma - 1.0) + 0.5 * sum(v * v for v in vel)
    q[5][:] = 1.0
    with _tile_ctx(p) as ctx:
        ctx.set_state(q)
        q_in = ctx.get_state()
        for _ in range(10):
            ctx.step(ctx.cfl_dt(0.7))
        q_out = ctx.get_state()
    for v in range(9):
        assert np.array_equal(q_in[v], q_out[v]), v


@pytest.mark.parametrize("which", ["strat", "sphere"])
def test_hydrostatic_state_preserved_bitwise(which):
    if which == "strat":
        p = workloads.strat_box(shape=(8, 6, 24), noise=0.0)
    else:
        p = workloads.sphere(n=20, mach=0.0)
    p.tables.heat = None
    p.tables.damp = None
    q = workloads.build(p)
    with _tile_ctx(p) as ctx:
        ctx.set_state(q)
        q_in = ctx.get_state()
        for _ in range(10):
            ctx.step(ctx.cfl_dt(0.7))
        q_out = ctx.get_state()
    for v in range(9):
        assert np.array_equal(q_in[v], q_out[v]), v


def test_graph_step_equals_six_passes():
    p = workloads.sphere(shape=(24, 20, 28))
    q = workloads.build(p)
    with _tile_ctx(p) as a, _tile_ctx(p) as b:
        a.set_state(q)
        b.set_state(q)
        dt = a.cfl_dt(0.7)
        a.step(dt)
        for axis, src in ((0, 0), (1, 0), (2, 1), (2, 0), (1, 0), (0, 1)):
            b.sweep(axis, dt, sources=bool(src))
        qa, qb = a.get_state(), b.get_state()
    for v in range(9):
        assert np.array_equal(qa[v], qb[v]), v


def test_cfl_after_step_matches_a_fresh_maximum():
    p = workloads.sphere(shape=(32, 26, 34))
    q = workloads.build(p)
    with _tile_ctx(p) as ctx:
        ctx.set_state(q)
        for _ in range(2):
            ctx.step(ctx.cfl_dt(p.cfl))
        dt_fused = ctx.cfl_dt(p.cfl)
        qs = ctx.get_state()
        ctx.set_state(qs)
        dt_fresh = ctx.cfl_dt(p.cfl)
    dt_orc = oracle.Oracle(p).cfl_dt(qs, p.cfl)
    assert abs(dt_fused - dt_fresh) <= 1e-6 * dt_fresh
    assert abs(dt_fused - dt_orc) <= 1e-6 * dt_orc


def test_tile_agrees_with_register_window_form():
    """Both FP32 forms on the same state for 10 double steps: the same
    arithmetic in a different order (contractions), so they agree at the
    FP32 tolerances, not bit for bit."""
    p = workloads.sphere(shape=(40, 36, 44))
    q = workloads.build(p)
    with _tile_ctx(p) as a, ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION) as b:
        a.set_state(q)
        b.set_state(q)
        for _ in range(10):
            dt = b.cfl_dt(0.7)
            a.step(dt)
            b.step(dt)
        assert_f32(a.get_state(), b.get_state(), "tile vs march")


def test_tile_not_available_is_refused():
    for p, prec in ((workloads.strat_box(shape=(30, 8, 8)), ppm.FP32_DEVIATION),      # nx % 4 != 0
                    (workloads.periodic_box(shape=(8, 8, 8)), ppm.FP64_PLAIN),
                    (workloads.sphere(shape=(24, 24, 24), confine=True), ppm.FP32_DEVIATION)):
        with ppm.Context.from_problem(p, precision=prec) as ctx:
            assert not ctx.tile_available
            with pytest.raises(ppm.PpmError):
                ctx.set_pass_design(ppm.PASS_TILE)
            assert ctx.pass_design == ppm.PASS_MARCH


def test_tuner_keeps_the_state_and_uses_its_cache(tmp_path):
    """ppm_tune times both designs per axis on the live state, leaves the
    state bit for bit as it was, picks a valid design per axis, writes the
    cache, and a second context takes the same choice from the cache."""
    p = workloads.sphere(shape=(44, 36, 40))
    q = workloads.build(p)
    cache = str(tmp_path / "tune.txt")
    with ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION) as ctx:
        ctx.set_state(q)
        ctx.step(ctx.cfl_dt(0.7))
        before = ctx.get_state()
        assert ctx.tune(cache) is False
        after = ctx.get_state()
        for v in range(9):
            assert np.array_equal(before[v], after[v]), v
        chosen = ctx.pass_designs
        assert all(d in (ppm.PASS_MARCH, ppm.PASS_TILE) for d in chosen)
        ctx.step(ctx.cfl_dt(0.7))          # steps after tuning run
    with ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION) as ctx:
        ctx.set_state(q)
        assert ctx.tune(cache) is True
        assert ctx.pass_designs == chosen
    # one design only: nothing to tune
    with ppm.Context.from_problem(p, precision=ppm.FP64_PLAIN) as ctx:
        ctx.set_state(q)
        assert ctx.tune(cache) is False
        assert ctx.pass_designs == (ppm.PASS_MARCH,) * 3
