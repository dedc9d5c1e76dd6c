"""The FP32 deviation form against the FP64 oracle: one set of checks for
every FP32 parity test.

  * rho and E: relative L1 <= 1e-5 (the stated FP32 target);
  * the three momenta: relative L1 <= TOL_MOM over sum |rho u_d|;
  * FV: mean |dFV| <= 1e-7 (the stated FV target), and 0 <= FV <= 1;
    the FV L-inf is reported beside it and bounded by TOL_FV_INF;
  * the first moments m_x, m_y, m_z: mean |dm| <= TOL_MOM1 and L-inf <= TOL_MOM1_INF.

The bounds beyond the stated ones sit about ten times above the largest
values measured over every FP32 parity case on a GB300 (momenta 1.1e-6
relative L1; FV L-inf 8.3e-7; moments 3.2e-8 mean, 1.9e-6 L-inf): FP32
rounding of the O(1) fractions and moments (ulp 6e-8) accumulated over the
120 passes of 20 double steps, and for the momenta FP32 rounding of the
pressure-sized flux terms relative to Mach-0.03 momenta.

With PPM_PARITY_LOG set, every comparison appends one JSON line with the
measured figures to that file (the tolerances are checked all the same).
"""
import json
import os

import numpy as np

TOL_L1 = 1e-5
TOL_FV = 1e-7
TOL_MOM = 1e-5
TOL_FV_INF = 1e-5
TOL_MOM1 = 3e-7
TOL_MOM1_INF = 2e-5


def f32_errors(qg, qo):
    e = {}
    for v, name in ((0, "rho"), (4, "E"), (1, "mx"), (2, "my"), (3, "mz")):
        den = np.abs(qo[v]).sum()
        e[name] = float(np.abs(qg[v] - qo[v]).sum() / (den if den > 0 else 1.0))
    d = np.abs(qg[5] - qo[5])
    e["fv_mean"] = float(d.mean())
    e["fv_inf"] = float(d.max())
    for v, name in ((6, "m1x"), (7, "m1y"), (8, "m1z")):
        d = np.abs(qg[v] - qo[v])
        e[name + "_mean"] = float(d.mean())
        e[name + "_inf"] = float(d.max())
    return e


def assert_f32(qg, qo, tag=""):
    e = f32_errors(qg, qo)
    log = os.environ.get("PPM_PARITY_LOG")
    if log:
        with open(log, "a") as f:
            f.write(json.dumps({"tag": tag, **e}) + "\n")
    for k in ("rho", "E"):
        assert e[k] <= TOL_L1, (tag, k, e[k])
    for k in ("mx", "my", "mz"):
        assert e[k] <= TOL_MOM, (tag, k, e[k])
    assert e["fv_mean"] <= TOL_FV, (tag, "fv_mean", e["fv_mean"])
    assert e["fv_inf"] <= TOL_FV_INF, (tag, "fv_inf", e["fv_inf"])
    for k in ("m1x", "m1y", "m1z"):
        assert e[k + "_mean"] <= TOL_MOM1, (tag, k + "_mean", e[k + "_mean"])
        assert e[k + "_inf"] <= TOL_MOM1_INF, (tag, k + "_inf", e[k + "_inf"])
    assert qg[5].min() >= 0.0 and qg[5].max() <= 1.0
    return e
