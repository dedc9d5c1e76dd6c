"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Same seeded inputs on both sides, the same explicit dt sequence (taken from
the oracle), element by element:
  * FP64 plain form: relative L-inf <= 1e-10 per variable after 20 double
    steps (relative to the variable's largest magnitude);
  * FP32 deviation form: relative L1 <= 1e-5 on rho and E, mean |dFV| <= 1e-7;
  * exact states (uniform, hydrostatic) preserved bit for bit;
  * full-size sampled parity: single passes of the 1024^3 sphere checked
    pencil by pencil against the oracle's single-pencil pass.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1810_13416_gb300 as ppm
import workloads
from parity_f32 import assert_f32

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-10
TOL_F32_L1 = 1e-5
TOL_F32_FV = 1e-7


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ppm.build()
    oracle.build()


def _relinf(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _run_pair(p, precision, steps, q0=None):
    q = workloads.build(p) if q0 is None else [a.copy() for a in q0]
    qo = [a.copy() for a in q]
    o = oracle.Oracle(p)
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(q)
    for _ in range(steps):
        dt = o.cfl_dt(qo, p.cfl)
        o.double_step(qo, dt)
        ctx.step(dt)
    qg = ctx.get_state()
    ctx.close()
    return qg, qo


def _assert_f64(qg, qo):
    for v in range(9):
        assert _relinf(qg[v], qo[v]) <= TOL_F64, (v, _relinf(qg[v], qo[v]))


def _assert_f32(qg, qo, tag=""):
    # rho, E, the momenta, FV (mean and L-inf) and the first moments
    assert_f32(qg, qo, tag)


def test_periodic_box_fp64_20_steps():
    p = workloads.periodic_box(32)
    qg, qo = _run_pair(p, ppm.FP64_PLAIN, 20)
    _assert_f64(qg, qo)


def test_periodic_box_fp32_20_steps():
    p = workloads.periodic_box(32)
    qg, qo = _run_pair(p, ppm.FP32_DEVIATION, 20)
    _assert_f32(qg, qo)


def _strat_ragged():
    # not a multiple of the 128-thread tile, several tiles along x
    return workloads.strat_box(shape=(150, 20, 36))


def _sphere_ragged():
    return workloads.sphere(shape=(44, 36, 40))


@pytest.mark.parametrize("maker", [_strat_ragged, _sphere_ragged])
def test_gravity_problems_fp64(maker):
    p = maker()
    qg, qo = _run_pair(p, ppm.FP64_PLAIN, 8)
    _assert_f64(qg, qo)


@pytest.mark.parametrize("maker", [_strat_ragged, _sphere_ragged])
def test_gravity_problems_fp32(maker):
    p = maker()
    qg, qo = _run_pair(p, ppm.FP32_DEVIATION, 8)
    _assert_f32(qg, qo)


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_stratified_box_128_full_size_20_steps(precision):
    """The stratified convection box at its full 128^3 size (plane gravity,
    reflecting z walls, heating, the light-fluid layer): 20 double steps,
    whole grid against the oracle (FP64 1e-10 relative L-inf; FP32 1e-5
    relative L1 on rho and E, 1e-7 mean on FV)."""
    p = workloads.strat_box(shape=(128, 128, 128))
    qg, qo = _run_pair(p, precision, 20)
    if precision == ppm.FP64_PLAIN:
        _assert_f64(qg, qo)
    else:
        _assert_f32(qg, qo)


@pytest.mark.parametrize("kind", ["sod", "lax"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shock_tubes_fp64(kind, axis):
    p = workloads.tube(kind, n=64, axis=axis, length=1.0 if kind == "sod" else 2.0)
    p.cfl = 0.6
    qg, qo = _run_pair(p, ppm.FP64_PLAIN, 15)
    _assert_f64(qg, qo)


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_uniform_state_preserved_bitwise(precision):
    p = workloads.periodic_box(shape=(8, 12, 16))
    nz, ny, nx = 16, 12, 8
    q = [np.zeros((nz, ny, nx)) for _ in range(9)]
    q[0][:] = 1.0
    vel = (0.25, -0.125, 0.375)
    for d in range(3):
        q[1 + d][:] = vel[d]
    q[4][:] = 0.75 / (p.gamma - 1.0) + 0.5 * sum(v * v for v in vel)
    q[5][:] = 1.0
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(q)
    q_in = ctx.get_state()
    for _ in range(10):
        ctx.step(ctx.cfl_dt(0.7))
    q_out = ctx.get_state()
    for v in range(9):
        assert np.array_equal(q_in[v], q_out[v]), v


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
@pytest.mark.parametrize("which", ["strat", "sphere"])
def test_hydrostatic_state_preserved_bitwise(precision, which):
    if which == "strat":
        p = workloads.strat_box(shape=(8, 6, 24), noise=0.0)
    else:
        p = workloads.sphere(n=20, mach=0.0)
    p.tables.heat = None
    p.tables.damp = None
    q = workloads.build(p)
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(q)
    q_in = ctx.get_state()
    for _ in range(10):
        ctx.step(ctx.cfl_dt(0.7))
    q_out = ctx.get_state()
    for v in range(9):
        assert np.array_equal(q_in[v], q_out[v]), v
    if precision == ppm.FP64_PLAIN:
        for v in range(9):
            assert np.array_equal(q_out[v], q[v]), v


def test_graph_step_equals_six_passes():
    p = workloads.sphere(shape=(24, 20, 28))
    q = workloads.build(p)
    a = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    b = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    a.set_state(q)
    b.set_state(q)
    dt = a.cfl_dt(0.7)
    a.step(dt)
    for axis, src in ((0, 0), (1, 0), (2, 1), (2, 0), (1, 0), (0, 1)):
        b.sweep(axis, dt, sources=bool(src))
    qa, qb = a.get_state(), b.get_state()
    for v in range(9):
        assert np.array_equal(qa[v], qb[v]), v


def test_device_dt_path_matches_explicit_dt():
    p = workloads.periodic_box(16)
    q = workloads.build(p)
    a = ppm.Context.from_problem(p, precision=ppm.FP64_PLAIN)
    b = ppm.Context.from_problem(p, precision=ppm.FP64_PLAIN)
    a.set_state(q)
    b.set_state(q)
    a.cfl_dt(0.7, fetch=False)
    for _ in range(3):
        a.step(0.0)                      # dt from the fused CFL maximum on the device
        b.step(b.cfl_dt(0.7))            # dt fetched and passed back explicitly
    qa, qb = a.get_state(), b.get_state()
    for v in range(9):
        assert _relinf(qa[v], qb[v]) <= 1e-14, v


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
@pytest.mark.parametrize("confine", [False, True])
def test_cfl_after_step_matches_a_fresh_maximum(precision, confine):
    """After a double step the time step comes from the maximum the last
    pass took (no pass over the grid); it equals the maximum taken afresh
    from the stored state (after a re-upload) and the oracle's."""
    p = workloads.sphere(shape=(30, 26, 34), confine=confine)
    q = workloads.build(p)
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(q)
    o = oracle.Oracle(p)
    for _ in range(2):
        ctx.step(ctx.cfl_dt(p.cfl))
    n0 = ctx.launch_count
    dt_fused = ctx.cfl_dt(p.cfl)
    assert ctx.launch_count - n0 == 1          # the cfl scalar only
    qs = ctx.get_state()
    ctx.set_state(qs)
    n0 = ctx.launch_count
    dt_fresh = ctx.cfl_dt(p.cfl)
    assert ctx.launch_count - n0 == 2          # the cfl scalar and the grid pass
    dt_orc = o.cfl_dt(qs, p.cfl)
    tol = 1e-13 if precision == ppm.FP64_PLAIN else 1e-6
    assert abs(dt_fused - dt_fresh) <= tol * dt_fresh
    assert abs(dt_fused - dt_orc) <= tol * dt_orc
    ctx.close()


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_cfl_and_diagnostics_match_oracle(precision):
    p = workloads.sphere(shape=(32, 28, 36))
    q = workloads.build(p)
    o = oracle.Oracle(p)
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(q)
    qs = ctx.get_state()                 # what the GPU holds (FP32-rounded for FP32)
    dt_o = o.cfl_dt(qs, 0.7)
    dt_g = ctx.cfl_dt(0.7)
    tol = 1e-13 if precision == ppm.FP64_PLAIN else 1e-6
    assert abs(dt_g - dt_o) <= tol * dt_o
    tg, pg, mg = ctx.diagnostics(16, 1.0)
    to, po, mo = o.diagnostics(qs, 16, 1.0)
    np.testing.assert_allclose(tg, to, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pg, po, rtol=(1e-12 if precision == ppm.FP64_PLAIN else 1e-5), atol=1e-12)
    assert abs(mg - mo) <= (1e-12 if precision == ppm.FP64_PLAIN else 1e-5) * mo


@pytest.mark.parametrize("make", [lambda: workloads.sphere(shape=(40, 36, 44)),
                                  lambda: workloads.strat_box(shape=(24, 20, 32))],
                         ids=["sphere", "strat"])
def test_fp32_diagnostics_totals_after_steps(make):
    """FP32 form after a few steps (folded FV near 1, moving gas): totals to
    1e-12 of the FP64 sums of the downloaded state, with and without shell
    bins, on the first call (which builds the cached base state) and on later
    calls."""
    p = make()
    q = workloads.build(p)
    ctx = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    ctx.set_state(q)
    o = oracle.Oracle(p)
    for it in range(3):
        dt = ctx.cfl_dt(p.cfl)
        ctx.step(dt)
        qs = ctx.get_state()
        for nb in ((0, 8) if it != 1 else (8, 0)):
            tg, pg, mg = ctx.diagnostics(nb, 1.0)
            to, po, mo = o.diagnostics(qs, nb, 1.0)
            np.testing.assert_allclose(tg, to, rtol=1e-12, atol=1e-14 * np.abs(to).max())
            if nb:
                np.testing.assert_allclose(pg, po, rtol=1e-5, atol=1e-12)
            assert abs(mg - mo) <= 1e-5 * mo
    assert (qs[5] > 0.5).any() and (qs[5] < 0.5).any()
    ctx.close()


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_state_larger_than_the_device_is_refused(precision):
    """A grid whose state cannot be allocated (4096^3: 2.4 TB in FP32) is
    refused with PPM_ENOMEM and leaves nothing behind: a context of a usable
    size then works as before."""
    p = workloads.periodic_box(shape=(4096, 4096, 4096))
    with pytest.raises(ppm.PpmError) as e:
        ppm.Context.from_problem(p, precision=precision)
    assert e.value.code == -2
    q_p = workloads.periodic_box(shape=(16, 16, 16))
    qg, qo = _run_pair(q_p, precision, 2)
    if precision == ppm.FP64_PLAIN:
        _assert_f64(qg, qo)
    else:
        _assert_f32(qg, qo)


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
@pytest.mark.parametrize("var", [0, 1, 4])
def test_nan_in_host_input_is_reported(precision, var):
    """A NaN planted in the host state (density, a momentum, the energy)
    makes the next pass report PPM_ENONPHYS; a clean upload afterwards runs
    normally and matches the oracle."""
    p = workloads.periodic_box(16)
    q = workloads.build(p)
    bad = [a.copy() for a in q]
    bad[var][5, 6, 7] = np.nan
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(bad)
    ctx.sweep(0, 1e-4)
    with pytest.raises(ppm.PpmError) as e:
        ctx.sync()
    assert e.value.code == -4
    ctx.set_state(q)
    o = oracle.Oracle(p)
    qo = [a.copy() for a in q]
    for _ in range(2):
        dt = o.cfl_dt(qo, p.cfl)
        o.double_step(qo, dt)
        ctx.step(dt)
    qg = ctx.get_state()
    ctx.close()
    if precision == ppm.FP64_PLAIN:
        _assert_f64(qg, qo)
    else:
        _assert_f32(qg, qo)


def test_nonphysical_state_is_reported():
    p = workloads.periodic_box(16)
    q = workloads.build(p)
    q[4][3, 4, 5] = -1.0                 # negative energy -> negative pressure
    ctx = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    ctx.set_state(q)
    ctx.sweep(0, 1e-4)
    with pytest.raises(ppm.PpmError) as e:
        ctx.sync()
    assert e.value.code == -4
    ctx.sync()                           # flag cleared after the report


def test_region_roundtrip_host_and_device():
    p = workloads.sphere(shape=(20, 18, 22))
    q = workloads.build(p)
    ctx = ppm.Context.from_problem(p, precision=ppm.FP64_PLAIN)
    ctx.set_state(q)
    lo, hi = (3, 2, 5), (17, 11, 20)
    sub = ctx.get_region(lo, hi)
    for v in range(9):
        assert np.array_equal(sub[v], q[v][lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]])
    dev = [torch.tensor(s, device="cuda") for s in sub]
    for t in dev:
        t.mul_(1.0)
    ctx.set_region(lo, hi, dev, device=True)
    out = [torch.empty_like(t) for t in dev]
    ctx.get_region(lo, hi, out, device=True)
    torch.cuda.synchronize()
    for v in range(9):
        assert np.array_equal(out[v].cpu().numpy(), sub[v])


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_pinned_host_transfers_match_pageable(precision):
    """Page-locked host arrays are read and written in place over the host
    link, pageable ones go through the staging buffers: identical results,
    for the whole state, a sub-box, and a pinned array of which only a part
    holds the region (a pinned view in the middle of a larger pinned buffer,
    whose other parts stay untouched)."""
    p = workloads.sphere(shape=(20, 18, 22))
    q = workloads.build(p)
    pin = [torch.from_numpy(a.copy()).pin_memory() for a in q]
    a = ppm.Context.from_problem(p, precision=precision)
    b = ppm.Context.from_problem(p, precision=precision)
    a.set_state(q)
    b.set_state([t.numpy() for t in pin])
    qa = a.get_state()
    qb = [torch.empty(t.shape, dtype=torch.float64).pin_memory() for t in pin]
    b.get_state_into([t.numpy() for t in qb])
    for v in range(9):
        assert np.array_equal(qb[v].numpy(), qa[v]), v
    lo, hi = (3, 2, 5), (17, 11, 20)
    n = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    big = [torch.zeros(3 * n, dtype=torch.float64).pin_memory() for _ in range(9)]
    mid = [t[n:2 * n].view(hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]) for t in big]
    b.get_region(lo, hi, [m.numpy() for m in mid])
    sub = a.get_region(lo, hi)
    for v in range(9):
        assert np.array_equal(mid[v].numpy(), sub[v]), v
        assert not big[v][:n].any() and not big[v][2 * n:].any(), v
    for m in mid:
        m.mul_(1.0 + 1e-3)
    a.set_region(lo, hi, [m.numpy().copy() for m in mid])
    b.set_region(lo, hi, [m.numpy() for m in mid])
    qa, qb2 = a.get_state(), b.get_state()
    for v in range(9):
        assert np.array_equal(qa[v], qb2[v]), v
    a.close()
    b.close()


def test_pinned_host_transfers_in_several_slabs():
    """A state of 512 x 512 x 300 cells (2^26 cells and more): in-place host
    transfers run in slabs of 256 planes; pinned and pageable uploads and
    downloads agree bit for bit."""
    p = workloads.periodic_box(shape=(512, 512, 300))
    rng = np.random.default_rng(7)
    shape = (300, 512, 512)
    q = [1.0 + 0.1 * rng.random(shape)] + [0.05 * rng.standard_normal(shape) for _ in range(3)]
    q += [2.0 + 0.1 * rng.random(shape), rng.random(shape)] + [np.zeros(shape) for _ in range(3)]
    pin = [torch.from_numpy(a).pin_memory() for a in q]
    a = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    b = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    a.set_state(q)                              # staging
    b.set_state([t.numpy() for t in pin])       # in place, two slabs
    qa = a.get_state()                          # staging
    for t in pin:                               # reuse the pinned buffers for b's download
        t.zero_()
    b.get_state_into([t.numpy() for t in pin])  # in place, two slabs
    for v in range(9):
        assert np.array_equal(pin[v].numpy(), qa[v]), v
    a.close()
    b.close()


# --------------------------------------------------------------------------
# Full size (the 1024^3 sphere in FP32, launch configuration of the benchmark):
# single passes checked pencil by pencil against the oracle.
# --------------------------------------------------------------------------
def _upload_sphere(ctx, p, slab=64):
    nz = p.shape[2]
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        qs = [t.contiguous() for t in workloads.initial_state(p, device="cuda", z_lo=z0, z_hi=z1)]
        qs += [torch.zeros_like(qs[0]) for _ in range(ctx.nvar - len(qs))]   # ten-value moments
        ctx.set_region((0, 0, z0), (p.shape[0], p.shape[1], z1), qs, device=True)
        del qs
    torch.cuda.synchronize()


def _pencil_box(p, axis, ja, jb):
    lo, hi = [0, 0, 0], [0, 0, 0]
    lo[axis], hi[axis] = 0, p.shape[axis]
    for d, j in (((axis + 1) % 3, ja), ((axis + 2) % 3, jb)):
        lo[d], hi[d] = j, j + 1
    return lo, hi


@pytest.mark.parametrize("variant", ["plain", "confined", "ten"])
def test_full_size_sphere_sampled_pencils_fp32(variant):
    """The 1024^3 benchmark grid (plain, with the confining sphere, with the
    ten-value PPB) in the launch configuration the benchmark times: single
    passes along each axis checked pencil by pencil against the oracle's
    single-pencil pass on the same inputs."""
    n = 1024
    free, _ = torch.cuda.mem_get_info()
    if free < (80e9 if variant == "ten" else 60e9):
        pytest.skip("needs 60-80 GB of device memory")
    p = workloads.sphere(n=n, confine=(variant == "confined"))
    if variant == "ten":
        p.nmom = 9
    o = oracle.Oracle(p)
    ctx = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
    _upload_sphere(ctx, p)
    dt = ctx.cfl_dt(0.7)
    rng = np.random.default_rng(1810)
    for axis in (0, 1, 2):
        picks = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(6)]
        picks.append((n // 2, n // 2))     # through the centre of the star
        ins = []
        for ja, jb in picks:
            lo, hi = _pencil_box(p, axis, ja, jb)
            ins.append([a.reshape(-1).copy() for a in ctx.get_region(lo, hi)])
        ctx.sweep(axis, dt, sources=(axis == 2))
        for (ja, jb), pin in zip(picks, ins):
            lo, hi = _pencil_box(p, axis, ja, jb)
            got = [a.reshape(-1) for a in ctx.get_region(lo, hi)]
            ref = o.sweep_pencil(pin, axis, ja, jb, dt, sources=(axis == 2))
            for v in (0, 4):
                err = np.abs(got[v] - ref[v]).max() / np.abs(ref[v]).max()
                assert err <= 1e-6, (axis, ja, jb, v, err)
            for v in (1, 2, 3):
                scale = max(np.abs(ref[v]).max(), 1e-30)
                assert np.abs(got[v] - ref[v]).max() <= 1e-4 * scale + 1e-7 * np.abs(ref[0]).max(), (axis, v)
            assert np.abs(got[5] - ref[5]).max() <= 1e-5, (axis, ja, jb)
            for v in range(6, len(ref)):
                assert np.abs(got[v] - ref[v]).max() <= 1e-4, (axis, ja, jb, v)
    tot, _, mm = ctx.diagnostics()
    assert np.isfinite(tot).all() and 0 < mm < 1
    ctx.close()


@pytest.mark.parametrize("shape,bc", [((4, 4, 4), 0), ((8, 4, 5), 1), ((16, 4, 4), 0), ((8, 8, 8), 1)])
@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_smallest_grids(shape, bc, precision):
    """Extents at the minimum (4, the stencil reach) and the smallest 16-byte
    x path (8): ghosts reach the far end of the pencil, periodic or walls."""
    p = workloads.periodic_box(shape=shape)
    p.dx = 1.0 / max(shape)
    p.bc = (bc,) * 6
    qg, qo = _run_pair(p, precision, 5)
    if precision == ppm.FP64_PLAIN:
        _assert_f64(qg, qo)
    else:
        _assert_f32(qg, qo)


@pytest.mark.parametrize("which", ["strat128", "sphere96"])
@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_gravity_configs_20_steps(which, precision):
    """The stratified box at its configured 128^3 and the sphere recipe at
    96^3, 20 double steps: FP64 within 1e-10 relative L-inf, FP32 within
    1e-5 relative L1 on rho and E and 1e-7 on FV."""
    if which == "strat128":
        p = workloads.strat_box(shape=(128, 128, 128))
    else:
        p = workloads.sphere(n=96)
    qg, qo = _run_pair(p, precision, 20)
    if precision == ppm.FP64_PLAIN:
        _assert_f64(qg, qo)
    else:
        _assert_f32(qg, qo)


@pytest.mark.parametrize("design", [ppm.PASS_MARCH, ppm.PASS_TILE])
def test_pass_times_inside_the_step(design):
    """ppm_pass_times: ESTATE before any step; afterwards six positive pass
    durations that add up to no more than the step itself (timed around it
    with CUDA events on the context's stream)."""
    p = workloads.sphere(shape=(64, 64, 64))
    q = workloads.build(p)
    stream = torch.cuda.Stream()
    with ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION, stream=stream) as ctx:
        ctx.set_pass_design(design)
        with pytest.raises(ppm.PpmError):
            ctx.pass_times()
        ctx.set_state(q)
        ctx.cfl_dt(p.cfl, fetch=False)
        ctx.step(0.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(0.0)
        e1.record(stream)
        pt = ctx.pass_times()
        e1.synchronize()
        step_ms = e0.elapsed_time(e1)
    assert pt.shape == (6,) and (pt > 0).all()
    assert pt.sum() <= step_ms * 1.001 + 0.01
