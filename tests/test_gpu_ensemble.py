"""Batched ensembles (one launch per pass for many uneven boxes) on the GPU.

* Every box of an ensemble evolves exactly (bit for bit) as the same box in
  its own single-grid context, under every tile configuration the autotuner
  can choose (64/128-thread blocks, persistent or one block per item, x-pass
  vector path on or off), including a box whose x extent is not a multiple
  of 8 and a box with periodic x/y.
* Boxes agree with the oracle within the FP32 (and FP64) tolerances.
* The autotuner leaves the states unchanged and reuses its cache.
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


def _boxes():
    shapes = [(48, 32, 40), (52, 36, 44), (64, 48, 32), (40, 40, 56), (32, 24, 24)]
    rates = [1e-4, 3e-3, 1e-2, 5e-4, 2e-3]
    return [workloads.strat_box(shape=s, seed=7000 + i, heat_rate=r) for i, (s, r) in enumerate(zip(shapes, rates))]


CONFIGS = [
    [(128, 1, 1), (128, 1, 1), (128, 1, 1)],
    [(64, 0, 0), (64, 0, 0), (64, 0, 0)],
    [(128, 0, 1), (64, 1, 0), (128, 0, 0)],
    [(64, 1, 0), (128, 0, 0), (64, 1, 0)],
    # 32-pencil blocks, and the x-pass vector path in 32- and 64-pencil blocks
    [(32, 0, 1), (32, 1, 0), (32, 0, 0)],
    [(64, 1, 1), (32, 0, 0), (64, 0, 0)],
    [(32, 1, 0), (128, 1, 0), (32, 1, 0)],
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_ensemble_equals_single_contexts_bitwise(cfg):
    probs = _boxes()
    qs = [workloads.build(p) for p in probs]
    ens = ppm.Ensemble(probs, precision=ppm.FP32_DEVIATION)
    for axis, (nb, pers, vec) in enumerate(cfg):
        ens.set_config(axis, nb, pers, vec)
    for b, q in enumerate(qs):
        ens.set_state(b, q)
    ens.cfl_dt(0.7, fetch=False)
    for _ in range(4):
        ens.step(0.0)
    ens.sync()
    for b, (p, q) in enumerate(zip(probs, qs)):
        with ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION) as ctx:
            ctx.set_state(q)
            ctx.cfl_dt(0.7, fetch=False)
            for _ in range(4):
                ctx.step(0.0)
            ref = ctx.get_state()
        got = ens.get_state(b)
        for v in range(9):
            assert np.array_equal(got[v], ref[v]), (b, v)
    ens.close()


@pytest.mark.parametrize("precision,tol", [(ppm.FP32_DEVIATION, 1e-5), (ppm.FP64_PLAIN, 1e-10)])
def test_ensemble_matches_oracle(precision, tol):
    probs = _boxes()[:3]
    qs = [workloads.build(p) for p in probs]
    qo = [[a.copy() for a in q] for q in qs]
    ens = ppm.Ensemble(probs, precision=precision)
    for b, q in enumerate(qs):
        ens.set_state(b, q)
    os_ = [oracle.Oracle(p) for p in probs]
    for _ in range(4):
        dt = min(o.cfl_dt(q, 0.7) for o, q in zip(os_, qo))
        for o, q in zip(os_, qo):
            o.double_step(q, dt)
        ens.step(dt)
    for b in range(len(probs)):
        got = ens.get_state(b)
        ref = qo[b]
        if precision == ppm.FP64_PLAIN:
            for v in range(9):
                s = np.abs(ref[v]).max()
                assert np.abs(got[v] - ref[v]).max() <= tol * (s if s > 0 else 1.0), (b, v)
        else:
            assert_f32(got, ref, f"ensemble box {b}")
    ens.close()


def test_tuner_keeps_states_and_uses_cache(tmp_path):
    probs = _boxes()
    qs = [workloads.build(p) for p in probs]
    cache = str(tmp_path / "tune.txt")
    ens = ppm.Ensemble(probs, precision=ppm.FP32_DEVIATION)
    for b, q in enumerate(qs):
        ens.set_state(b, q)
    before = [ens.get_state(b) for b in range(len(probs))]
    assert ens.tune(cache) is False
    cfg = ens.config()
    after = [ens.get_state(b) for b in range(len(probs))]
    for b in range(len(probs)):
        for v in range(9):
            assert np.array_equal(before[b][v], after[b][v])
    for ax in "xyz":
        assert cfg[ax][0] in (32, 64, 128)
    ens.cfl_dt(0.7, fetch=False)
    ens.step(0.0)
    ens.sync()
    ens.close()
    ens2 = ppm.Ensemble(probs, precision=ppm.FP32_DEVIATION)
    for b, q in enumerate(qs):
        ens2.set_state(b, q)
    assert ens2.tune(cache) is True
    assert ens2.config() == cfg
    ens2.close()


def test_ensemble_step_needs_dt():
    probs = _boxes()[:2]
    ens = ppm.Ensemble(probs, precision=ppm.FP32_DEVIATION)
    for b, p in enumerate(probs):
        ens.set_state(b, workloads.build(p))
    with pytest.raises(ppm.PpmError) as e:
        ens.step(0.0)
    assert e.value.code == -7
    ens.close()


def _uneven_boxes():
    # uneven extents (one with nx not a multiple of 8) and periodic x / y
    shapes = [(48, 32, 40), (52, 36, 44), (64, 48, 32), (40, 40, 56), (32, 24, 24), (96, 64, 48)]
    return [workloads.strat_box(shape=s, seed=7100 + i, heat_rate=1e-3 * (i + 1)) for i, s in enumerate(shapes)]


@pytest.mark.parametrize("precision", [ppm.FP32_DEVIATION, ppm.FP64_PLAIN])
def test_one_launch_step_equals_per_pass_bitwise(precision):
    """The whole double step in one launch (items of all passes from one
    counter, each pass of a box waiting for its previous pass) gives the
    per-pass ensemble's result bit for bit, over 4 double steps with device
    time steps, in two launches per step (dt kernel + the step)."""
    probs = _uneven_boxes()
    qs = [workloads.build(p) for p in probs]
    out = {}
    for mode in (ppm.ENS_PER_PASS, ppm.ENS_ONE_LAUNCH):
        ens = ppm.Ensemble(probs, precision=precision)
        ens.set_launch_mode(mode)
        assert ens.launch_mode == mode
        for b, q in enumerate(qs):
            ens.set_state(b, q)
        ens.cfl_dt(0.7, fetch=False)
        l0 = ens.launch_count
        for _ in range(4):
            ens.step(0.0)
        ens.sync()
        if mode == ppm.ENS_ONE_LAUNCH:
            assert (ens.launch_count - l0) == 2 * 4
        out[mode] = [ens.get_state(b) for b in range(len(probs))]
        ens.close()
    for b in range(len(probs)):
        for v in range(9):
            assert np.array_equal(out[ppm.ENS_PER_PASS][b][v], out[ppm.ENS_ONE_LAUNCH][b][v]), (b, v)


def test_one_launch_wait_that_runs_out_is_reported():
    """Every bounded wait of the step made to run out (the test option: the
    first item of each block waits for a count that never comes): the step
    ends with PPM_ETIMEOUT instead of hanging, and the ensemble stays usable:
    after a fresh upload a normal step matches the per-pass result."""
    probs = _uneven_boxes()[:3]
    qs = [workloads.build(p) for p in probs]
    ens = ppm.Ensemble(probs, precision=ppm.FP32_DEVIATION)
    ens.set_launch_mode(ppm.ENS_ONE_LAUNCH)
    for b, q in enumerate(qs):
        ens.set_state(b, q)
    dt = ens.cfl_dt(0.7)
    ens.set_wait_test(True)
    ens.step(float(np.min(dt)))
    with pytest.raises(ppm.PpmError) as ei:
        ens.sync()
    assert "PPM_ETIMEOUT" in str(ei.value)
    ens.set_wait_test(False)
    for b, q in enumerate(qs):
        ens.set_state(b, q)
    ens.step(float(np.min(dt)))
    ens.sync()
    got = [ens.get_state(b) for b in range(len(probs))]
    ens.close()
    ref = ppm.Ensemble(probs, precision=ppm.FP32_DEVIATION)
    for b, q in enumerate(qs):
        ref.set_state(b, q)
    ref.step(float(np.min(dt)))
    ref.sync()
    for b in range(len(probs)):
        r = ref.get_state(b)
        for v in range(9):
            assert np.array_equal(got[b][v], r[v]), (b, v)
    ref.close()
