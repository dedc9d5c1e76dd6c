"""GPU parity of the ten-value PPB (FV with first, second and mixed moments;
Sec. 1 and Sec. 4) against the FP64 oracle, through the C ABI:
  * FP64 plain form: relative L-inf <= 1e-10 on all 15 stored values after
    10 double steps;
  * FP32 deviation form: relative L1 <= 1e-5 on rho and E, mean |dFV| <=
    1e-7, and the moments within 1e-4 of their scale (mean absolute);
  * a periodic box with arbitrary valid moments, the sphere with gravity and
    sources, and a ragged grid;
  * a state at rest with moments stays bit for bit.
"""
import copy

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


def _ten(p):
    p = copy.copy(p)
    p.nmom = 9
    return p


def _moments(q, seed, scale=0.3):
    """The 9-value state plus valid random second and mixed moments (first
    moments and FV as given)."""
    rng = np.random.default_rng(seed)
    fv = q[5]
    g = fv * (1 - fv)
    extra = [scale * 15 * g * rng.uniform(-1, 1, fv.shape) for _ in range(3)]
    extra += [scale * 36 * g * rng.uniform(-1, 1, fv.shape) for _ in range(3)]
    return list(q) + extra


def _relinf(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _run_pair(p, q0, precision, steps):
    qo = [a.copy() for a in q0]
    o = oracle.Oracle(p)
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(q0)
    for _ in range(steps):
        dt = o.cfl_dt(qo, p.cfl)
        o.double_step(qo, dt)
        ctx.step(dt)
    qg = ctx.get_state()
    ctx.close()
    return qg, qo


def _cases():
    box = workloads.periodic_box(shape=(24, 20, 16))
    sph = workloads.sphere(shape=(22, 19, 26))
    return [("box", _ten(box), box), ("sphere", _ten(sph), sph)]


@pytest.mark.parametrize("case", [0, 1])
def test_ten_value_fp64_matches_oracle(case):
    name, p, base = _cases()[case]
    q0 = _moments(workloads.build(base), seed=case)
    qg, qo = _run_pair(p, q0, ppm.FP64_PLAIN, 10)
    for v in range(15):
        assert _relinf(qg[v], qo[v]) <= 1e-10, (name, v, _relinf(qg[v], qo[v]))


@pytest.mark.parametrize("case", [0, 1])
def test_ten_value_fp32_matches_oracle(case):
    name, p, base = _cases()[case]
    q0 = _moments(workloads.build(base), seed=case)
    qg, qo = _run_pair(p, q0, ppm.FP32_DEVIATION, 10)
    assert_f32(qg[:9], qo[:9], f"ten-value {name}")
    for v in range(6, 15):
        err = np.abs(qg[v] - qo[v]).mean() / max(np.abs(qo[v]).mean(), 1e-3)
        assert err <= 1e-4, (name, v, err)


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
def test_ten_value_rest_state_bitwise(precision):
    base = workloads.periodic_box(shape=(16, 16, 16), mach=0.0)
    p = _ten(base)
    q0 = _moments(workloads.build(base), seed=9)
    ctx = ppm.Context.from_problem(p, precision=precision)
    ctx.set_state(q0)
    qs = ctx.get_state()
    dt = ctx.cfl_dt(p.cfl)
    for _ in range(10):
        ctx.step(dt)
    q1 = ctx.get_state()
    ctx.close()
    for v in range(15):
        assert np.array_equal(q1[v], qs[v]), v


def test_ten_value_rejects_confinement():
    p = _ten(workloads.sphere(n=16, confine=True))
    with pytest.raises(ppm.PpmError):
        ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION)
