"""A second, separately written statement of one pass of the PPM+PPB method
(four-value and ten-value forms): whole-grid, array-at-a-time numpy (every
pencil of the grid at once, the pass axis last), against which the
pencil-by-pencil C++ oracle is checked.  Same readings of the paper,
independent code: boundary ghosts by index arrays, base state by vectorised
table lookups, every step as shifted-array arithmetic.  Plane-parallel or no
gravity; no sources.
"""
import numpy as np

G = 4
C_SMOOTH, EPS_SMOOTH = 0.5, 1e-9
EPS_SHOCK, OMEGA1, OMEGA2 = 0.33, 0.75, 10.0
P_FLOOR = 1e-10


def _lerp(tab, s0, ds, s):
    u = (s - s0) / ds
    i = np.clip(np.floor(u), 0, len(tab) - 2).astype(int)
    w = u - i
    return tab[i] + w * (tab[i + 1] - tab[i])


def _ghost_index(n, periodic):
    """Source cell and mirror flag of the n + 2G cells of a pencil."""
    i = np.arange(-G, n + G)
    if periodic:
        return np.mod(i, n), np.zeros(i.shape, bool)
    src = np.where(i < 0, -1 - i, np.where(i >= n, 2 * n - 1 - i, i))
    return src, (i < 0) | (i >= n)


def _face_pos(n, periodic):
    """Position (cells from the low end) of faces j + 1/2, j in [-G, n+G)."""
    P = np.arange(-G, n + G) + 1
    if periodic:
        return np.where((P >= n) | (P < 0), np.mod(P, n), P)
    return np.where(P < 0, -P, np.where(P > n, 2 * n - P, P))


def divergence(p, q):
    """Cell velocity divergence (central differences of u_d = m_d / rho,
    summed x, y, z), ghosts by the boundary conditions: periodic wrap, or at
    a wall the mirror cell with its normal velocity reversed."""
    diffs = []
    for d in range(3):
        npd = 2 - d
        assert p.bc[2 * d] == p.bc[2 * d + 1]
        u = np.moveaxis(q[1 + d] / q[0], npd, -1)
        if p.bc[2 * d] == 0:
            up = np.concatenate([u[..., 1:], u[..., :1]], axis=-1)
            dn = np.concatenate([u[..., -1:], u[..., :-1]], axis=-1)
        else:
            up = np.concatenate([u[..., 1:], -u[..., -1:]], axis=-1)
            dn = np.concatenate([-u[..., :1], u[..., :-1]], axis=-1)
        diffs.append(np.moveaxis(up - dn, -1, npd))
    return ((diffs[0] + diffs[1]) + diffs[2]) * (0.5 / p.dx)


def sweep(p, q, axis, dt, sources=0, domega=0.0):
    """One pass along `axis` of the full-variable arrays q (z, y, x);
    sources: bit 0 heating / damping, bit 1 the rotation increment domega."""
    t = p.tables
    gam, gm1 = p.gamma, p.gamma - 1.0
    n = p.shape[axis]
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    assert p.bc[2 * axis] == p.bc[2 * axis + 1] and p.shape[axis] > G
    periodic = p.bc[2 * axis] == 0
    npax = 2 - axis
    mv = lambda a: np.moveaxis(a, npax, -1)           # pass axis last
    src, flip = _ghost_index(n, periodic)
    sg = np.where(flip, -1.0, 1.0)
    take = lambda a: np.take(mv(a), src, axis=-1)
    rho_full = take(q[0])
    mn = take(q[1 + axis]) * sg
    m1 = take(q[1 + t1])
    m2 = take(q[1 + t2])
    E = take(q[4])
    fv = take(q[5])
    on = take(q[6 + axis]) * sg
    o1 = take(q[6 + t1])
    o2 = take(q[6 + t2])
    kshock = float(getattr(p, "shock_k", 0.0) or 0.0)
    if kshock > 0.0:
        dv = take(divergence(p, q))          # even under a mirror
    ten = len(q) == 15
    if ten:
        # second moments along (n, t1, t2); mixed moments: c12 of the two
        # transverse axes, c_n1 / c_n2 of the normal with t1 / t2 (odd in n)
        qn, q1, q2 = take(q[9 + axis]), take(q[9 + t1]), take(q[9 + t2])
        c12 = take(q[12 + axis])
        cn1, cn2 = take(q[12 + t2]) * sg, take(q[12 + t1]) * sg
    # cell positions along every axis (for the base state: plane gravity in z)
    shape = mv(q[0]).shape[:-1] + (n + 2 * G,)
    coord = [p.origin[d] + (np.arange(p.shape[d]) + 0.5) * p.dx for d in range(3)]
    if p.grav == 0:
        rho0c = np.full(shape, t.rho0[0])
        p0c = np.full(shape, t.p0[0])
        gc = np.zeros(shape)
        rho0f = np.full(shape, t.rho0[0])
        p0f = np.full(shape, t.p0[0])
    elif p.grav == 2:
        # central gravity: tables in r at the mirrored cells' own positions
        # and at the folded faces (transverse coordinates of the pencil)
        Z3, Y3, X3 = np.meshgrid(coord[2], coord[1], coord[0], indexing="ij")
        XYZ = [mv(X3), mv(Y3), mv(Z3)]
        pos = [np.take(c, src, axis=-1) for c in XYZ]
        rho0c, p0c, gor = _central_base(p, pos[0], pos[1], pos[2])
        gc = (gor * pos[axis]) * sg
        fpos = [np.broadcast_to(c[..., :1], shape) for c in XYZ]
        fpos[axis] = np.broadcast_to(p.origin[axis] + _face_pos(n, periodic) * p.dx, shape)
        rho0f, p0f, _ = _central_base(p, fpos[0], fpos[1], fpos[2])
    else:
        assert p.grav == 1
        if axis == 2:
            z = coord[2][src]
            zf = p.origin[2] + _face_pos(n, periodic) * p.dx
        else:
            # an x or y pass: z is the leading array axis, constant along the pencil
            z = np.broadcast_to(coord[2][:, None, None], shape)
            zf = z
        rho0c = np.broadcast_to(_lerp(t.rho0, t.s0, t.ds, z), shape)
        p0c = np.broadcast_to(_lerp(t.p0, t.s0, t.ds, z), shape)
        gz = np.broadcast_to(_lerp(t.g, t.s0, t.ds, z), shape)
        gc = gz * sg if axis == 2 else np.zeros(shape)
        rho0f = np.broadcast_to(_lerp(t.rho0, t.s0, t.ds, zf), shape)
        p0f = np.broadcast_to(_lerp(t.p0, t.s0, t.ds, zf), shape)
    rd = rho_full - rho0c
    ed = E - p0c / gm1
    g = dict(rd=rd, mn=mn, m1=m1, m2=m2, ed=ed, fv=fv, on=on, o1=o1, o2=o2, rho0c=rho0c, p0c=p0c, gc=gc,
             rho0f=rho0f, p0f=p0f)
    if kshock > 0.0:
        g["dv"] = dv
    if ten:
        g.update(qn=qn, q1=q1, q2=q2, c12=c12, cn1=cn1, cn2=cn2)
    src_info = None
    if sources:
        Z3, Y3, X3 = np.meshgrid(coord[2], coord[1], coord[0], indexing="ij")
        src_info = dict(flags=sources, domega=domega, pos=[mv(X3), mv(Y3), mv(Z3)])
    out = _core(p, axis, dt, n, not periodic, g, src_info)
    return [np.ascontiguousarray(np.moveaxis(a, -1, npax)) for a in out]


def _sources(p, axis, dt, rho, mn, m1, m2, ed, info):
    """Heating / damping (bit 0) then the rotation increment (bit 1) on the
    new values of the updated cells, in the pass frame."""
    t = p.tables
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    x, y, z = info["pos"]
    if (info["flags"] & 1) and (t.heat is not None or t.damp is not None):
        sv = z if p.grav == 1 else np.sqrt((x * x + y * y) + z * z)
        if t.heat is not None:
            ed = ed + dt * _lerp(t.heat, t.s0, t.ds, sv)
        if t.damp is not None:
            kd = _lerp(t.damp, t.s0, t.ds, sv)
            f = np.maximum(0.0, 1.0 - dt * kd)
            ke = 0.5 * (mn * mn + (m1 * m1 + m2 * m2)) / rho
            mn, m1, m2 = mn * f, m1 * f, m2 * f
            ed = ed - (1.0 - f * f) * ke
    if (info["flags"] & 2) and info["domega"] != 0.0:
        w = info["domega"]
        du = [-(w * y), w * x, np.zeros_like(x)]
        dn, d1, d2 = du[axis], du[t1], du[t2]
        dE = (mn * dn + (m1 * d1 + m2 * d2)) + 0.5 * rho * (dn * dn + (d1 * d1 + d2 * d2))
        mn, m1, m2 = mn + rho * dn, m1 + rho * d1, m2 + rho * d2
        ed = ed + dE
    return mn, m1, m2, ed


def _core(p, axis, dt, n, walls, g, src_info=None):
    """Steps a1 (primitives) to a9 on pencil-batched arrays (pass axis
    last, n cells plus G ghosts on each side), walls at both ends or not.
    Returns the new full variables of the n cells, in the pass frame's
    storage order (index = stored variable)."""
    t = p.tables
    gam, gm1 = p.gamma, p.gamma - 1.0
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    kshock = float(getattr(p, "shock_k", 0.0) or 0.0)
    ten = "qn" in g
    rd, mn, m1, m2, ed = g["rd"], g["mn"], g["m1"], g["m2"], g["ed"]
    fv, on, o1, o2 = g["fv"], g["on"], g["o1"], g["o2"]
    rho0c, p0c, gc, rho0f, p0f = g["rho0c"], g["p0c"], g["gc"], g["rho0f"], g["p0f"]
    if kshock > 0.0:
        dv = g["dv"]
    if ten:
        qn, q1, q2, c12, cn1, cn2 = g["qn"], g["q1"], g["q2"], g["c12"], g["cn1"], g["cn2"]
    # primitives
    rho = rho0c + rd
    u, v, w = mn / rho, m1 / rho, m2 / rho
    pd = gm1 * (ed - 0.5 * (mn * u + (m1 * v + m2 * w)))
    pf = p0c + pd
    c2 = gam * pf / rho
    cs = np.sqrt(c2)
    W = [rd, u, v, w, pd]
    def at(a, k, lo, hi):
        """a[i + k] for i in [lo, hi) (pencil indices, ghosts negative)."""
        return a[..., G + lo + k:G + hi + k]
    # interface values of faces j + 1/2, j in [-3, n+2)
    jl, jh = -3, n + 2
    af = [(7.0 * (at(a, 0, jl, jh) + at(a, 1, jl, jh)) - (at(a, -1, jl, jh) + at(a, 2, jl, jh))) * (1.0 / 12.0)
          for a in W]
    # smoothness weights, flattening, parabolas of cells i in [-2, n+2)
    il, ih = -2, n + 2
    scales = [at(rho, 0, il, ih), at(cs, 0, il, ih), at(cs, 0, il, ih), at(cs, 0, il, ih), at(pf, 0, il, ih)]
    wgt = []
    for a, sc in zip(W, scales):
        d1m2 = at(a, -1, il, ih) - at(a, -2, il, ih)
        d1m1 = at(a, 0, il, ih) - at(a, -1, il, ih)
        d10 = at(a, 1, il, ih) - at(a, 0, il, ih)
        d1p1 = at(a, 2, il, ih) - at(a, 1, il, ih)
        d2m, d20, d2p = d1m1 - d1m2, d10 - d1m1, d1p1 - d10
        T = np.maximum(np.abs(d20 - d2m), np.abs(d2p - d20))
        S = np.maximum(np.maximum(np.abs(d1m1), np.abs(d10)),
                       np.maximum(np.maximum(np.abs(d2m), np.abs(d20)), np.abs(d2p)))
        fl = EPS_SMOOTH * sc
        x = T - C_SMOOTH * S - fl
        with np.errstate(divide="ignore", invalid="ignore"):
            wgt.append(np.where(x > 0, np.minimum(1.0, x / ((1 - C_SMOOTH) * S + fl)), 0.0))
    dp1 = at(pd, 1, il, ih) - at(pd, -1, il, ih)
    dp2 = at(pd, 2, il, ih) - at(pd, -2, il, ih)
    pmin = np.minimum(at(pf, 1, il, ih), at(pf, -1, il, ih))
    shock = (np.abs(dp1) > EPS_SHOCK * pmin) & (at(u, -1, il, ih) - at(u, 1, il, ih) > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(dp2 != 0, dp1 / dp2, 1.0)
    flat = np.where(shock, np.clip(OMEGA2 * (r - OMEGA1), 0.0, 1.0), 0.0)
    PL, PR, PD, P6 = [], [], [], []
    for a, afv, wv in zip(W, af, wgt):
        ac = at(a, 0, il, ih)
        aL = afv[..., (il - 1) - jl:(ih - 1) - jl]
        aR = afv[..., il - jl:ih - jl]
        aL = np.where(flat > 0, aL + flat * (ac - aL), aL)
        aR = np.where(flat > 0, aR + flat * (ac - aR), aR)
        am, ap = at(a, -1, il, ih), at(a, 1, il, ih)
        cL = np.clip(aL, np.minimum(am, ac), np.maximum(am, ac))
        cR = np.clip(aR, np.minimum(ac, ap), np.maximum(ac, ap))
        ext = (cR - ac) * (ac - cL) <= 0
        da = cR - cL
        dm = ac - 0.5 * (cL + cR)
        d6 = da * da * (1.0 / 6.0)
        fixL = da * dm > d6
        fixR = ~fixL & (-d6 > da * dm)
        nL = np.where(ext, ac, np.where(fixL, 3.0 * ac - 2.0 * cR, cL))
        nR = np.where(ext, ac, np.where(fixR, 3.0 * ac - 2.0 * cL, cR))
        aL = np.where(wv > 0, aL + wv * (nL - aL), aL)
        aR = np.where(wv > 0, aR + wv * (nR - aR), aR)
        PL.append(aL)
        PR.append(aR)
        PD.append(aR - aL)
        P6.append(6.0 * (ac - 0.5 * (aL + aR)))
    fR = lambda k, s: PR[k] - 0.5 * s * (PD[k] - (1.0 - (2.0 / 3.0) * s) * P6[k])
    fL = lambda k, s: PL[k] + 0.5 * s * (PD[k] + (1.0 - (2.0 / 3.0) * s) * P6[k])
    dtdx = dt / p.dx
    uc, cc, c2c, rc = at(u, 0, il, ih), at(cs, 0, il, ih), at(c2, 0, il, ih), at(rho, 0, il, ih)
    C = rc * cc
    lm, l0, lp = uc - cc, uc, uc + cc
    hg = 0.5 * dt * ((at(rd, 0, il, ih) / rc) * at(gc, 0, il, ih))
    # right edges (left states of faces i + 1/2)
    sp = np.maximum(lp, 0.0) * dtdx
    WLs = [fR(k, sp) for k in range(5)]
    ref = list(WLs)
    s0 = l0 * dtdx
    on0 = l0 > 0
    WLs[0] = np.where(on0, WLs[0] - ((ref[0] - fR(0, s0)) - (ref[4] - fR(4, s0)) / c2c), WLs[0])
    WLs[2] = np.where(on0, WLs[2] - (ref[2] - fR(2, s0)), WLs[2])
    WLs[3] = np.where(on0, WLs[3] - (ref[3] - fR(3, s0)), WLs[3])
    sm = lm * dtdx
    onm = lm > 0
    Am = 0.5 * ((ref[4] - fR(4, sm)) - C * (ref[1] - fR(1, sm)))
    WLs[0] = np.where(onm, WLs[0] - Am / c2c, WLs[0])
    WLs[1] = np.where(onm, WLs[1] + Am / C, WLs[1])
    WLs[4] = np.where(onm, WLs[4] - Am, WLs[4])
    WLs[1] = WLs[1] + hg
    # left edges (right states of faces i - 1/2)
    smm = np.maximum(-lm, 0.0) * dtdx
    WRs = [fL(k, smm) for k in range(5)]
    ref = list(WRs)
    s0 = -l0 * dtdx
    on0 = l0 < 0
    WRs[0] = np.where(on0, WRs[0] - ((ref[0] - fL(0, s0)) - (ref[4] - fL(4, s0)) / c2c), WRs[0])
    WRs[2] = np.where(on0, WRs[2] - (ref[2] - fL(2, s0)), WRs[2])
    WRs[3] = np.where(on0, WRs[3] - (ref[3] - fL(3, s0)), WRs[3])
    s1 = -lp * dtdx
    onp = lp < 0
    Ap_ = 0.5 * ((ref[4] - fL(4, s1)) + C * (ref[1] - fL(1, s1)))
    WRs[0] = np.where(onp, WRs[0] - Ap_ / c2c, WRs[0])
    WRs[1] = np.where(onp, WRs[1] - Ap_ / C, WRs[1])
    WRs[4] = np.where(onp, WRs[4] - Ap_, WRs[4])
    WRs[1] = WRs[1] + hg
    # faces j + 1/2, j in [-2, n+1): left state from cell j, right from cell j+1
    fl_, fh_ = -2, n + 1
    L = [a[..., fl_ - il:fh_ - il] for a in WLs]
    Rt = [a[..., fl_ + 1 - il:fh_ + 1 - il] for a in WRs]
    r0 = at(rho0f, 0, fl_, fh_)
    p0 = at(p0f, 0, fl_, fh_)
    rdL, uL, pdL = L[0], L[1], L[4]
    rdR, uR, pdR = Rt[0], Rt[1], Rt[4]
    rL, pL, rR, pR = r0 + rdL, p0 + pdL, r0 + rdR, p0 + pdR
    CL, CR = np.sqrt(gam * pL * rL), np.sqrt(gam * pR * rR)
    pfl = P_FLOOR * np.minimum(pL, pR)
    den = CL + CR
    pst = pdL + CL * (CR * (uL - uR) + (pdR - pdL)) / den
    pst = np.where(p0 + pst < pfl, pfl - p0, pst)
    kk = (gam + 1.0) / (2.0 * gam)
    WLi = CL * np.sqrt(1.0 + kk * (pst - pdL) / pL)
    WRi = CR * np.sqrt(1.0 + kk * (pst - pdR) / pR)
    den = WLi + WRi
    pst = pdL + WLi * (WRi * (uL - uR) + (pdR - pdL)) / den
    ust = uL + (WRi * (uR - uL) + (pdL - pdR)) / den
    pst = np.where(p0 + pst < pfl, pfl - p0, pst)
    wall = np.zeros(fh_ - fl_, dtype=bool)
    if walls:
        jj = np.arange(fl_, fh_)
        wall = (jj == -1) | (jj == n - 1)
        ust = np.where(wall, 0.0, ust)
    left = ust >= 0
    rds, pds = np.where(left, rdL, rdR), np.where(left, pdL, pdR)
    rs, pss = np.where(left, rL, rR), np.where(left, pL, pR)
    vst, wst = np.where(left, L[2], Rt[2]), np.where(left, L[3], Rt[3])
    dps = pst - pds
    rdst = rds + rs * dps / (gam * pss + 0.5 * gm1 * dps)
    # both two-shock waves on one side of the face (supersonic flow through
    # it): the solution at x/t = 0 is the upwind traced state
    sup_l = ~wall & (uL - WLi / rL >= 0.0)
    sup_r = ~wall & ~sup_l & (uR + WRi / rR <= 0.0)
    for msk, (ru, rp, rr_, rv, rw) in ((sup_l, (uL, pdL, rdL, L[2], L[3])), (sup_r, (uR, pdR, rdR, Rt[2], Rt[3]))):
        ust = np.where(msk, ru, ust)
        pst = np.where(msk, rp, pst)
        rdst = np.where(msk, rr_, rdst)
        vst = np.where(msk, rv, vst)
        wst = np.where(msk, rw, wst)
    Fr = (r0 + rdst) * ust
    gg1 = gam / gm1
    Fn = Fr * ust + pst
    Ft1, Ft2 = Fr * vst, Fr * wst
    FE = ust * (gg1 * pst + gg1 * p0) + 0.5 * (ust * ust + (vst * vst + wst * wst)) * Fr
    if kshock > 0.0:
        # dissipation across faces where the face divergence marks a shock
        dface = 0.5 * (at(dv, 0, fl_, fh_) + at(dv, 1, fl_, fh_))
        cface = 0.5 * (CL / rL + CR / rR)
        nu = kshock * np.maximum(0.0, -(dface * p.dx) - 0.05 * cface)
        on_ = nu > 0.0
        jump = lambda a: at(a, 1, fl_, fh_) - at(a, 0, fl_, fh_)
        Fn = np.where(on_, Fn - nu * jump(mn), Fn)
        Ft1 = np.where(on_, Ft1 - nu * jump(m1), Ft1)
        Ft2 = np.where(on_, Ft2 - nu * jump(m2), Ft2)
        FE = np.where(on_, FE - nu * jump(ed), FE)
    # cells i in [-1, n+1): faces i - 1/2 (index i-1) and i + 1/2 (index i)
    cl_, ch_ = -1, n + 1
    f_m = lambda F: F[..., (cl_ - 1) - fl_:(ch_ - 1) - fl_]
    f_p = lambda F: F[..., cl_ - fl_:ch_ - fl_]
    gcell = at(gc, 0, cl_, ch_)
    rd0 = at(rd, 0, cl_, ch_)
    rdn = rd0 - dtdx * (f_p(Fr) - f_m(Fr))
    mnn = at(mn, 0, cl_, ch_) - dtdx * (f_p(Fn) - f_m(Fn)) + dt * gcell * (0.5 * (rd0 + rdn))
    m1n = at(m1, 0, cl_, ch_) - dtdx * (f_p(Ft1) - f_m(Ft1))
    m2n = at(m2, 0, cl_, ch_) - dtdx * (f_p(Ft2) - f_m(Ft2))
    edn = at(ed, 0, cl_, ch_) - dtdx * (f_p(FE) - f_m(FE)) + dt * gcell * (0.5 * (f_m(Fr) + f_p(Fr)))
    # PPB profiles of cells [-2, n+2): own FV and slope, curvature from neighbours
    F = at(fv, 0, il, ih)
    mm = at(on, 0, il, ih)
    a2 = at(qn, 0, il, ih) if ten else 0.25 * (at(on, 1, il, ih) - at(on, -1, il, ih))
    ep = 0.5 * mm + a2 * (1.0 / 6.0)
    em = a2 * (1.0 / 6.0) - 0.5 * mm
    gmax, gmin = np.maximum(ep, em), np.minimum(ep, em)
    with np.errstate(divide="ignore", invalid="ignore"):
        xv = np.where(a2 != 0, -mm / (2.0 * a2), 1.0)
        gv = mm * xv + a2 * (xv * xv - 1.0 / 12.0)
        inside = (a2 != 0) & (np.abs(xv) < 0.5)
        gmax = np.where(inside, np.maximum(gmax, gv), gmax)
        gmin = np.where(inside, np.minimum(gmin, gv), gmin)
        th = np.ones_like(F)
        th = np.where(F + gmax > 1.0, np.minimum(th, (1.0 - F) / gmax), th)
        th = np.where(F + gmin < 0.0, np.minimum(th, F / (-gmin)), th)
    me, ae = th * mm, th * a2
    # transfers across faces [-2, n+1): donor = upwind cell (index j or j+1)
    sig = ust * dtdx
    phi = dtdx * Fr
    fromleft = sig >= 0
    s = np.abs(sig)
    M1 = 0.5 - 0.5 * s
    M2 = 0.25 - 0.5 * s + s * s * (1.0 / 3.0)
    M3 = 0.125 - 0.375 * s + 0.5 * s * s - 0.25 * s * s * s
    M1 = np.where(fromleft, M1, -M1)
    M3 = np.where(fromleft, M3, -M3)
    donor = lambda a: np.where(fromleft, a[..., fl_ - il:fh_ - il], a[..., fl_ + 1 - il:fh_ + 1 - il])
    Fd, med, aed = donor(F), donor(me), donor(ae)
    o1d, o2d = donor(at(o1, 0, il, ih)), donor(at(o2, 0, il, ih))
    phibar = Fd + med * M1 + aed * (M2 - 1.0 / 12.0)
    psibar = Fd * M1 + med * M2 + aed * (M3 - M1 * (1.0 / 12.0))
    GL, GH = phi * Fd, phi * phibar
    KL, KH = phi * Fd * M1, phi * psibar
    PHI, KM = phi, phi * M1
    if ten:
        M4 = 0.0625 - 0.25 * s + 0.5 * s * s - 0.5 * s * s * s + 0.2 * s * s * s * s
        chibar = Fd * M2 + med * M3 + aed * (M4 - M2 * (1.0 / 12.0))
        K2L, K2H, KM2 = phi * Fd * M2, phi * chibar, phi * M2
        cn1d, cn2d = donor(at(cn1, 0, il, ih)), donor(at(cn2, 0, il, ih))
        T1, T2 = phi * (o1d + cn1d * M1), phi * (o2d + cn2d * M1)
        U1, U2 = phi * (o1d * M1 + cn1d * M2), phi * (o2d * M1 + cn2d * M2)
        Q1, Q2 = phi * donor(at(q1, 0, il, ih)), phi * donor(at(q2, 0, il, ih))
        C12 = phi * donor(at(c12, 0, il, ih))
    else:
        T1, T2 = phi * o1d, phi * o2d
    # FCT factors of cells [-1, n+1)
    rold = at(rho0c, 0, cl_, ch_) + rd0
    rnew = at(rho0c, 0, cl_, ch_) + rdn
    fvc = at(fv, 0, cl_, ch_)
    cLo = rold * fvc - (f_p(GL) - f_m(GL))
    FVL = cLo / rnew
    Apl, Amn = f_p(GH) - f_p(GL), f_m(GH) - f_m(GL)
    Pp = np.maximum(0.0, Amn) - np.minimum(0.0, Apl)
    Pm = np.maximum(0.0, Apl) - np.minimum(0.0, Amn)
    with np.errstate(divide="ignore", invalid="ignore"):
        Rp = np.where(Pp > 0, np.clip((1.0 - FVL) * rnew / Pp, 0.0, 1.0), 0.0)
        Rm = np.where(Pm > 0, np.clip(FVL * rnew / Pm, 0.0, 1.0), 0.0)
    # limited transfers of faces [-1, n): cells j (index j+1 in [-1, n+1)) and j+1
    ff = slice(-1 - fl_, n - fl_)
    A = GH[..., ff] - GL[..., ff]
    Rp_j, Rm_j = Rp[..., 0:n + 1], Rm[..., 0:n + 1]
    Rp_j1, Rm_j1 = Rp[..., 1:n + 2], Rm[..., 1:n + 2]
    Cf = np.where(A >= 0, np.minimum(Rp_j1, Rm_j), np.minimum(Rp_j, Rm_j1))
    Gf = GL[..., ff] + Cf * A
    Kf = KL[..., ff] + Cf * (KH[..., ff] - KL[..., ff])
    if ten:
        K2f = K2L[..., ff] + Cf * (K2H[..., ff] - K2L[..., ff])
    T1f, T2f, PHIf, KMf = T1[..., ff], T2[..., ff], PHI[..., ff], KM[..., ff]
    sgf = sig[..., ff]
    # update of cells [0, n): faces i - 1/2 (index i in [-1,n) -> i) and i + 1/2 (i+1)
    q_ = lambda a: a[..., 0:n]        # face i - 1/2
    p_ = lambda a: a[..., 1:n + 1]    # face i + 1/2
    ro = rold[..., 1:n + 1]
    rn = rnew[..., 1:n + 1]
    fc = fvc[..., 1:n + 1]
    smv, spv = q_(sgf), p_(sgf)
    cold = ro * fc
    outp = spv >= 0
    inm = smv >= 0
    shp, shm = spv + 1.0, smv - 1.0
    c_out = np.where(outp, p_(Gf), 0.0) + np.where(inm, 0.0, -q_(Gf))
    z_out = np.where(outp, p_(Kf), 0.0) + np.where(inm, 0.0, -q_(Kf))
    m_out = np.where(outp, p_(PHIf), 0.0) + np.where(inm, 0.0, -q_(PHIf))
    zr_out = np.where(outp, p_(KMf), 0.0) + np.where(inm, 0.0, -q_(KMf))
    z_in = np.where(outp, 0.0, -p_(Kf) - p_(Gf) * shp) + np.where(inm, q_(Kf) + q_(Gf) * shm, 0.0)
    zr_in = np.where(outp, 0.0, -p_(KMf) - p_(PHIf) * shp) + np.where(inm, q_(KMf) + q_(PHIf) * shm, 0.0)
    sbar = 0.5 * (smv + spv)
    dZc = (cold - c_out) * sbar + z_in - z_out
    Zr = (ro - m_out) * sbar + zr_in - zr_out
    dPhi = p_(PHIf) - q_(PHIf)
    dG = p_(Gf) - q_(Gf)
    fvn = np.clip(fc + (fc * dPhi - dG) / rn, 0.0, 1.0)
    onc, o1c, o2c = on[..., G:G + n], o1[..., G:G + n], o2[..., G:G + n]
    onn = onc + (onc * dPhi + 12.0 * (dZc - fvn * Zr)) / rn
    o1n = o1c + (o1c * dPhi - (p_(T1f) - q_(T1f))) / rn
    o2n = o2c + (o2c * dPhi - (p_(T2f) - q_(T2f))) / rn
    bnd = 6.0 * fvn * (1.0 - fvn)
    if ten:
        sel = lambda cond, a: np.where(cond, a, 0.0)
        KM2f = KM2[..., ff]
        U1f, U2f = U1[..., ff], U2[..., ff]
        z2_out = sel(outp, p_(K2f)) - sel(~inm, q_(K2f))
        zr2_out = sel(outp, p_(KM2f)) - sel(~inm, q_(KM2f))
        t1_out = sel(outp, p_(T1f)) - sel(~inm, q_(T1f))
        t2_out = sel(outp, p_(T2f)) - sel(~inm, q_(T2f))
        u1_out = sel(outp, p_(U1f)) - sel(~inm, q_(U1f))
        u2_out = sel(outp, p_(U2f)) - sel(~inm, q_(U2f))
        z2_in = (-sel(~outp, p_(K2f) + 2.0 * shp * p_(Kf) + shp * shp * p_(Gf))
                 + sel(inm, q_(K2f) + 2.0 * shm * q_(Kf) + shm * shm * q_(Gf)))
        zr2_in = (-sel(~outp, p_(KM2f) + 2.0 * shp * p_(KMf) + shp * shp * p_(PHIf))
                  + sel(inm, q_(KM2f) + 2.0 * shm * q_(KMf) + shm * shm * q_(PHIf)))
        u1_in = -sel(~outp, p_(U1f) + p_(T1f) * shp) + sel(inm, q_(U1f) + q_(T1f) * shm)
        u2_in = -sel(~outp, p_(U2f) + p_(T2f) * shp) + sel(inm, q_(U2f) + q_(T2f) * shm)
        S0 = cold - c_out
        S1 = ro * onc * (1.0 / 12.0) - z_out
        dZc2 = 2.0 * sbar * S1 + sbar * sbar * S0 + z2_in - z2_out
        Zr2 = -2.0 * sbar * zr_out + sbar * sbar * (ro - m_out) + zr2_in - zr2_out + (ro - rn) * (1.0 / 12.0)
        dC2p = dZc2 + dG * (1.0 / 12.0)
        qnc, q1c, q2c = qn[..., G:G + n], q1[..., G:G + n], q2[..., G:G + n]
        cn1c, cn2c, c12c = cn1[..., G:G + n], cn2[..., G:G + n], c12[..., G:G + n]
        qnn = qnc + (qnc * dPhi + 180.0 * (dC2p - fvn * Zr2) - 12.0 * onn * Zr) / rn
        dY1 = (ro * o1c - t1_out) * sbar + u1_in - u1_out
        dY2 = (ro * o2c - t2_out) * sbar + u2_in - u2_out
        cn1n = cn1c + (cn1c * dPhi + 12.0 * (dY1 - o1n * Zr)) / rn
        cn2n = cn2c + (cn2c * dPhi + 12.0 * (dY2 - o2n * Zr)) / rn
        Q1f, Q2f, C12f = Q1[..., ff], Q2[..., ff], C12[..., ff]
        q1n = q1c + (q1c * dPhi - (p_(Q1f) - q_(Q1f))) / rn
        q2n = q2c + (q2c * dPhi - (p_(Q2f) - q_(Q2f))) / rn
        c12n = c12c + (c12c * dPhi - (p_(C12f) - q_(C12f))) / rn
        g_ = fvn * (1.0 - fvn)
        bm, bcn = 6.0 * g_, 36.0 * g_
        qlo, qhi = -15.0 * g_ * (1.0 + fvn), 15.0 * g_ * (2.0 - fvn)
        qnn, q1n, q2n = (np.clip(a, qlo, qhi) for a in (qnn, q1n, q2n))
        cn1n, cn2n, c12n = (np.clip(a, -bcn, bcn) for a in (cn1n, cn2n, c12n))
        bnd = bm
    onn, o1n, o2n = (np.clip(a, -bnd, bnd) for a in (onn, o1n, o2n))
    # back to full variables, physical frame
    inner = lambda a: a[..., 1:n + 1]
    out = [None] * (15 if ten else 9)
    r0c = rho0c[..., G:G + n]
    p0cc = p0c[..., G:G + n]
    mni, m1i, m2i, edi = inner(mnn), inner(m1n), inner(m2n), inner(edn)
    if src_info is not None:
        mni, m1i, m2i, edi = _sources(p, axis, dt, r0c + inner(rdn), mni, m1i, m2i, edi, src_info)
    out[0] = r0c + inner(rdn)
    out[1 + axis] = mni
    out[1 + t1] = m1i
    out[1 + t2] = m2i
    out[4] = p0cc / gm1 + edi
    out[5] = fvn
    out[6 + axis] = onn
    out[6 + t1] = o1n
    out[6 + t2] = o2n
    if ten:
        out[9 + axis], out[9 + t1], out[9 + t2] = qnn, q1n, q2n
        out[12 + axis], out[12 + t2], out[12 + t1] = c12n, cn1n, cn2n
    return out


def _fold(i, n):
    """Source cell and mirror flag of pencil index i for a run of n cells
    with walls at both ends: the run and its mirror images repeat with
    period 2n."""
    k = np.mod(i, 2 * n)
    inside = (i >= 0) & (i < n)
    src = np.where(inside, i, np.where(k < n, k, 2 * n - 1 - k))
    flip = ~inside & (k >= n)
    return src, flip


def _fold_face(j, n):
    """Position (cells from the run's low end) of face j + 1/2, walls at
    both ends, same images as _fold."""
    P = j + 1
    k = np.mod(P, 2 * n)
    return np.where((P >= 0) & (P <= n), P, np.where(k <= n, k, 2 * n - k))


def _central_base(p, x, y, z):
    """rho0, p0 and g/r at points (x, y, z): tables in r about the origin."""
    t = p.tables
    r = np.sqrt((x * x + y * y) + z * z)
    rho0 = _lerp(t.rho0, t.s0, t.ds, r)
    p0 = _lerp(t.p0, t.s0, t.ds, r)
    with np.errstate(divide="ignore", invalid="ignore"):
        gor = np.where(r > 0.0, _lerp(t.g, t.s0, t.ds, r) / r, 0.0)
    return rho0, p0, gor


def sweep_confined(p, q, axis, dt, sources=0, domega=0.0):
    """One pass along `axis` with a confining sphere (central gravity, four
    values): every pencil's run of fluid cells is updated as a pencil with
    walls at both ends; pencils are batched by their run (start, length)."""
    assert p.grav == 2 and p.confine_r > 0.0 and len(q) == 9
    gm1 = p.gamma - 1.0
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    npax = 2 - axis
    mv = lambda a: np.moveaxis(a, npax, -1)
    coord = [p.origin[d] + (np.arange(p.shape[d]) + 0.5) * p.dx for d in range(3)]
    Z, Y, X = np.meshgrid(coord[2], coord[1], coord[0], indexing="ij")
    fluid = mv((X * X + Y * Y) + Z * Z < p.confine_r * p.confine_r)
    XYZ = [mv(X), mv(Y), mv(Z)]
    qm = [mv(a) for a in q]
    out = [a.copy() for a in qm]
    groups = {}
    for lead in np.ndindex(fluid.shape[:-1]):
        f = fluid[lead]
        idx = np.nonzero(f)[0]
        if idx.size == 0:
            continue
        i0, n = int(idx[0]), int(idx.size)
        assert idx[-1] - idx[0] + 1 == n
        groups.setdefault((i0, n), []).append(lead)
    for (i0, n), leads in groups.items():
        l1 = np.array([a for a, _ in leads])
        l2 = np.array([b for _, b in leads])
        i = np.arange(-G, n + G)
        src, flip = _fold(i, n)
        cells = i0 + src
        sg = np.where(flip, -1.0, 1.0)
        take = lambda a: a[l1, l2][:, cells]
        pos = [take(c) for c in XYZ]
        rho0c, p0c, gor = _central_base(p, pos[0], pos[1], pos[2])
        gc = (gor * pos[axis]) * sg
        # faces: along-axis position from the folded face index, transverse
        # coordinates those of the pencil
        fpos = [np.broadcast_to(c[l1, l2][:, :1], (len(leads), n + 2 * G)) for c in XYZ]
        fpos[axis] = p.origin[axis] + (i0 + _fold_face(i, n)) * p.dx
        fpos[axis] = np.broadcast_to(fpos[axis], (len(leads), n + 2 * G))
        rho0f, p0f, _ = _central_base(p, fpos[0], fpos[1], fpos[2])
        g = dict(rd=take(qm[0]) - rho0c, mn=take(qm[1 + axis]) * sg, m1=take(qm[1 + t1]),
                 m2=take(qm[1 + t2]), ed=take(qm[4]) - p0c / gm1, fv=take(qm[5]),
                 on=take(qm[6 + axis]) * sg, o1=take(qm[6 + t1]), o2=take(qm[6 + t2]),
                 rho0c=rho0c, p0c=p0c, gc=gc, rho0f=rho0f, p0f=p0f)
        run = np.arange(i0, i0 + n)
        info = None
        if sources:
            info = dict(flags=sources, domega=domega, pos=[c[l1, l2][:, run] for c in XYZ])
        res = _core(p, axis, dt, n, True, g, info)
        for v in range(9):
            o = out[v]
            o[l1[:, None], l2[:, None], run[None, :]] = res[v]
    return [np.ascontiguousarray(np.moveaxis(a, -1, npax)) for a in out]
