"""Zalesak's slotted disk carried once round by a solid-body rotation, as the
qualitative check of the PPB transport (the paper shows this test, Fig. 3).

The gas has uniform density and a rotation u = omega (-y, x) inside r < 0.7
(tapered to rest at r = 0.9) held by the pressure of cyclostrophic balance,
so the flow is steady up to the splitting error.  After one turn the FV
field is compared with its start: it stays in [0, 1], the disk keeps its
content, and the ten-value form (own second moments) is closer to the start
than the four-value form.
"""
import copy
import math

import numpy as np

import oracle
import workloads


def _setup(n, nmom):
    p = workloads.periodic_box(shape=(n, n, 4), mach=0.0)
    p = copy.copy(p)
    p.origin = (-1.0, -1.0, 0.0)
    p.dx = 2.0 / n
    p.bc = (1, 1, 1, 1, 0, 0)
    p.nmom = nmom
    h = p.dx
    c = -1.0 + (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(c, c)                      # (y, x)
    r = np.hypot(X, Y)
    w = 1.0
    taper = np.clip((0.9 - r) / 0.2, 0.0, 1.0)
    taper = taper * taper * (3 - 2 * taper)
    ut = w * r * taper                            # azimuthal speed
    # cyclostrophic pressure: dp/dr = rho ut^2 / r, p(0) = 10
    rr = np.linspace(0.0, 1.5, 3001)
    tr = np.clip((0.9 - rr) / 0.2, 0.0, 1.0)
    tr = tr * tr * (3 - 2 * tr)
    f = (w * rr * tr) ** 2 / np.maximum(rr, 1e-12)
    pr = 10.0 + np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(rr))])
    P = np.interp(r, rr, pr)
    U = -ut * np.where(r > 0, Y / np.maximum(r, 1e-300), 0.0)
    V = ut * np.where(r > 0, X / np.maximum(r, 1e-300), 0.0)
    # slotted disk: centre (0, 0.35), radius 0.3, slot 0.1 wide, 0.35 deep
    sub = 8
    s = (np.arange(sub) + 0.5) / sub - 0.5
    F = np.zeros((n, n)); MX = np.zeros((n, n)); MY = np.zeros((n, n))
    QX = np.zeros((n, n)); QY = np.zeros((n, n)); CXY = np.zeros((n, n))
    for a in s:
        for b in s:
            x = X + a * h
            y = Y + b * h
            inside = (np.hypot(x, y - 0.35) < 0.3) & ~((np.abs(x) < 0.05) & (y < 0.35 + 0.05))
            g = inside.astype(float) / sub ** 2
            F += g
            MX += 12 * a * g
            MY += 12 * b * g
            QX += 180 * (a * a - 1.0 / 12) * g
            QY += 180 * (b * b - 1.0 / 12) * g
            CXY += 144 * a * b * g
    def vol(a2):
        return np.broadcast_to(a2, (4, n, n)).copy()
    gm1 = p.gamma - 1.0
    q = [vol(np.ones((n, n))), vol(U), vol(V), vol(np.zeros((n, n))),
         vol(P / gm1 + 0.5 * (U * U + V * V)), vol(F)]
    g = F * (1 - F)
    q += [vol(np.clip(MX, -6 * g, 6 * g)), vol(np.clip(MY, -6 * g, 6 * g)), vol(np.zeros((n, n)))]
    if nmom == 9:
        qlo, qhi = -15 * g * (1 + F), 15 * g * (2 - F)
        q += [vol(np.clip(QX, qlo, qhi)), vol(np.clip(QY, qlo, qhi)), vol(np.zeros((n, n))),
              vol(np.zeros((n, n))), vol(np.zeros((n, n))), vol(np.clip(CXY, -36 * g, 36 * g))]
    return p, q, 2 * math.pi / w


def _one_turn(nmom, n=64):
    p, q, T = _setup(n, nmom)
    f0 = q[5].copy()
    c0 = (q[0] * q[5]).sum()
    o = oracle.Oracle(p)
    t = 0.0
    while t < T - 1e-12:
        dt = min(o.cfl_dt(q, 0.6), 0.5 * (T - t))
        o.double_step(q, dt)
        t += 2 * dt
        assert q[5].min() >= 0.0 and q[5].max() <= 1.0
    assert abs((q[0] * q[5]).sum() - c0) <= 1e-12 * c0       # rho*FV content
    assert np.abs(q[0] - 1.0).max() < 0.05                    # the flow stayed nearly steady
    return f0, q[5]


def test_slotted_disk_one_turn():
    f0, f4 = _one_turn(3)
    _, f10 = _one_turn(9)
    area0 = f0.sum()
    e4 = np.abs(f4 - f0).sum() / area0
    e10 = np.abs(f10 - f0).sum() / area0
    assert e10 < e4, (e4, e10)
    assert e10 < 0.45, e10          # measured 0.43 (0.47 four-value); 0.30 at 96^2
