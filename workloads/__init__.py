"""Seeded synthetic inputs for the PPM+PPB sweeps.

This module builds initial states, base-state tables and source tables for the
problems the sweeps are tested and measured on.  It is the ONE module that both
sides of the parity check use (the CPU oracle under ``oracle/`` and the CUDA
library ``paper_1810_13416_gb300``); it holds none of the method's arithmetic
(no interpolation, limiter, Riemann solve or update) -- only problem set-up:
random numbers, Fourier velocity modes, polytropic base states, tanh
interfaces and their cell moments.

Every array is float64.  Generation runs through torch so that the small cases
are built on the host for the oracle and the 1024^3 case can be built slab by
slab on the device for the throughput run; the same code serves both.

Problems (the paper's stellar models are not available, so these synthetic
stand-ins follow the setting the paper describes: low-Mach convection with a
multifluid interface, Sec. 1-3):

* ``periodic_box``   periodic cube, uniform base, random solenoidal modes at
                     rms Mach 0.03, tanh FV layer (the 32^3 plain-method case).
* ``strat_box``      plane-parallel n=1.5 polytropic layer under constant
                     gravity, reflecting z walls, heating near the bottom,
                     light fluid above z=0.7, seeded density noise.
* ``sphere``         sphere-in-cube: n=3 polytrope under central gravity,
                     heating shell, damping near the centre and the outer
                     shell, light-fluid layer at r=0.6R, velocity modes in the
                     convection zone.
* ``tube``           Sod / Lax shock tubes along one axis.
* ``wave``           smooth advected density wave and FV bump (order tests).

State layout: 9 arrays in the order (rho, rho*u, rho*v, rho*w, E, FV, m_x,
m_y, m_z), each shaped (nz, ny, nx) with x fastest; rho and E are the full
(not base-subtracted) values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

NVAR = 9
VAR_NAMES = ("rho", "mx", "my", "mz", "E", "fv", "mom_x", "mom_y", "mom_z")

BC_PERIODIC = 0
BC_REFLECT = 1
GRAV_NONE = 0
GRAV_PLANE_Z = 1
GRAV_CENTRAL = 2


# --------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014): the published 64-bit mixing generator.
# --------------------------------------------------------------------------
_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def splitmix_field(seed: int, shape, offset: int = 0, device="cpu") -> torch.Tensor:
    """Counter-based uniform [0,1) field: value at flat index n is the
    SplitMix64 output for state seed + (n+offset+1)*golden (vectorised)."""
    n = int(np.prod(shape))
    idx = torch.arange(offset + 1, offset + n + 1, dtype=torch.int64, device=device)
    # emulate uint64 arithmetic in int64 (two's complement wrap is identical)
    golden = torch.tensor(0x9E3779B97F4A7C15 - (1 << 64), dtype=torch.int64)
    z = idx * golden.to(device) + torch.tensor(_to_i64(seed), dtype=torch.int64, device=device)
    z = _mix(z)
    u = _srl(z, 11).to(torch.float64) * (1.0 / (1 << 53))
    return u.reshape(shape)


def _to_i64(v: int) -> int:
    v &= _M64
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 viewed as uint64."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    c1 = torch.tensor(_to_i64(0xBF58476D1CE4E5B9), dtype=torch.int64, device=z.device)
    c2 = torch.tensor(_to_i64(0x94D049BB133111EB), dtype=torch.int64, device=z.device)
    z = (z ^ _srl(z, 30)) * c1
    z = (z ^ _srl(z, 27)) * c2
    return z ^ _srl(z, 31)


# --------------------------------------------------------------------------
# Problem description shared by both sides
# --------------------------------------------------------------------------
@dataclass
class Tables:
    """Radial (or height) profiles on a uniform coordinate grid s_i = s0 + i*ds.

    rho0, p0: hydrostatic base state; g: signed acceleration along +s
    (negative = towards s=0 for the sphere, downwards for the layer);
    heat: energy added per unit volume and time; damp: velocity damping rate.
    """
    s0: float
    ds: float
    rho0: np.ndarray
    p0: np.ndarray
    g: np.ndarray
    heat: Optional[np.ndarray] = None
    damp: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.rho0.shape[0])


@dataclass
class Problem:
    name: str
    shape: tuple            # (nx, ny, nz)
    origin: tuple           # (x0, y0, z0): low corner of the grid
    dx: float
    gamma: float
    bc: tuple               # 6 faces: -x,+x,-y,+y,-z,+z
    grav: int
    tables: Tables
    cfl: float = 0.7
    steps: int = 20
    seed: int = 0
    extra: dict = field(default_factory=dict)
    confine_r: float = 0.0  # > 0: confining sphere of this radius about the origin

    @property
    def ncell(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


def _cell_coords(p: Problem, device, z_lo=0, z_hi=None):
    nx, ny, nz = p.shape
    if z_hi is None:
        z_hi = nz
    x = p.origin[0] + (torch.arange(nx, dtype=torch.float64, device=device) + 0.5) * p.dx
    y = p.origin[1] + (torch.arange(ny, dtype=torch.float64, device=device) + 0.5) * p.dx
    z = p.origin[2] + (torch.arange(z_lo, z_hi, dtype=torch.float64, device=device) + 0.5) * p.dx
    return x, y, z


def _lerp_table(tab: np.ndarray, s0: float, ds: float, s: torch.Tensor) -> torch.Tensor:
    """Evaluate a tabulated profile at coordinates s (set-up only)."""
    t = torch.as_tensor(tab, dtype=torch.float64, device=s.device)
    u = (s - s0) / ds
    i = torch.clamp(torch.floor(u), 0, t.numel() - 2).to(torch.int64)
    w = u - i.to(torch.float64)
    return t[i] + w * (t[i + 1] - t[i])


# Gauss-Legendre nodes/weights on [-1/2, 1/2] (3 points), for cell averages
# and cell moments of the analytic interface profiles.
_GL3_X = (-0.5 * math.sqrt(3.0 / 5.0), 0.0, 0.5 * math.sqrt(3.0 / 5.0))
_GL3_W = (5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0)
_GL8 = np.polynomial.legendre.leggauss(8)
_GL8_X = tuple(0.5 * _GL8[0])
_GL8_W = tuple(0.5 * _GL8[1])


def _sqrt(t: torch.Tensor) -> torch.Tensor:
    """Correctly rounded square root (torch's vectorised CPU sqrt is not
    always; CUDA's float64 sqrt is)."""
    if t.device.type == "cpu":
        return torch.from_numpy(np.sqrt(t.numpy()))
    return torch.sqrt(t)


def _valid_fv(fv: torch.Tensor, moms):
    """Make (FV, moments) a realisable sub-cell representation: 0<=FV<=1 and
    |m_d| <= 6 FV (1-FV) (quadrature round-off can step outside by an ulp)."""
    fv = torch.clamp(fv, 0.0, 1.0)
    b = 6.0 * fv * (1.0 - fv)
    return fv, [torch.maximum(torch.minimum(m, b), -b) for m in moms]


def _tanh_profile(s, s_c, width):
    return 0.5 * (1.0 + torch.tanh((s - s_c) / width))


# --------------------------------------------------------------------------
# Velocity modes
# --------------------------------------------------------------------------
def _fourier_modes(rng: SplitMix64, nmodes: int, kmax: int):
    """nmodes integer wave vectors 0<|k|<=kmax, unit amplitudes perpendicular
    to k (solenoidal), uniform random phases."""
    modes = []
    while len(modes) < nmodes:
        k = [int(math.floor(rng.uniform() * (2 * kmax + 1))) - kmax for _ in range(3)]
        kk = math.sqrt(k[0] ** 2 + k[1] ** 2 + k[2] ** 2)
        if kk == 0.0 or kk > kmax:
            continue
        # random direction, projected perpendicular to k
        a = [2.0 * rng.uniform() - 1.0 for _ in range(3)]
        dot = sum(a[i] * k[i] for i in range(3)) / (kk * kk)
        a = [a[i] - dot * k[i] for i in range(3)]
        an = math.sqrt(sum(v * v for v in a))
        if an < 1e-3:
            continue
        a = [v / an for v in a]
        phase = 2.0 * math.pi * rng.uniform()
        modes.append((k, a, phase))
    return modes


def _velocity_from_modes(modes, x, y, z, length):
    """Sum of modes sin(2 pi k.x/L + phase) * a, broadcast over (z, y, x)."""
    X = x.view(1, 1, -1)
    Y = y.view(1, -1, 1)
    Z = z.view(-1, 1, 1)
    shape = (z.numel(), y.numel(), x.numel())
    u = [torch.zeros(shape, dtype=torch.float64, device=x.device) for _ in range(3)]
    for k, a, ph in modes:
        arg = (2.0 * math.pi / length) * (k[0] * X + k[1] * Y + k[2] * Z) + ph
        s = torch.sin(arg)
        for d in range(3):
            if a[d] != 0.0:
                u[d] += a[d] * s
    return u


def _modes_rms(modes) -> float:
    # each mode a*sin(...) with |a|=1 has mean square 1/2; distinct k are orthogonal
    # except k and -k which may interfere: measured on the grid instead when needed.
    return math.sqrt(0.5 * len(modes))


# --------------------------------------------------------------------------
# Lane-Emden polytropes (RK4, FP64)
# --------------------------------------------------------------------------
def lane_emden(n: float, xi_max: float, h: float = 1e-4):
    """Solve theta'' + 2 theta'/xi + theta^n = 0, theta(0)=1, theta'(0)=0.

    Returns arrays (xi, theta, dtheta) on a uniform grid of step h, starting
    from the series theta = 1 - xi^2/6 + n xi^4/120 at xi=h.  Stops at xi_max
    (which must lie inside the first zero)."""
    npts = int(round(xi_max / h)) + 1
    xi = np.zeros(npts)
    th = np.zeros(npts)
    dth = np.zeros(npts)
    th[0], dth[0] = 1.0, 0.0
    x0 = h
    t = 1.0 - x0 * x0 / 6.0 + n * x0 ** 4 / 120.0
    dt = -x0 / 3.0 + n * x0 ** 3 / 30.0
    xi[1], th[1], dth[1] = x0, t, dt

    def f(x, y, yp):
        return yp, -2.0 * yp / x - (max(y, 0.0)) ** n

    for i in range(1, npts - 1):
        x = xi[i]
        y, yp = th[i], dth[i]
        k1 = f(x, y, yp)
        k2 = f(x + h / 2, y + h / 2 * k1[0], yp + h / 2 * k1[1])
        k3 = f(x + h / 2, y + h / 2 * k2[0], yp + h / 2 * k2[1])
        k4 = f(x + h, y + h * k3[0], yp + h * k3[1])
        xi[i + 1] = x + h
        th[i + 1] = y + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        dth[i + 1] = yp + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return xi, th, dth


def _integrate_pressure(s, rho, g, p_start):
    """p(s) = p_start + int_0^s rho g ds' by the trapezoid rule on a fine grid."""
    f = rho * g
    p = np.empty_like(s)
    p[0] = p_start
    p[1:] = p_start + np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(s))
    return p


# --------------------------------------------------------------------------
# Problem builders
# --------------------------------------------------------------------------
def _uniform_tables(rho0=1.0, p0=1.0) -> Tables:
    one = np.ones(2)
    return Tables(s0=0.0, ds=1.0, rho0=rho0 * one, p0=p0 * one, g=0.0 * one)


def periodic_box(n: int = 32, seed: int = 1810, nmodes: int = 8, kmax: int = 4,
                 mach: float = 0.03, gamma: float = 5.0 / 3.0, shape=None) -> Problem:
    """Periodic unit cube, rho=1, p=1, no gravity, random solenoidal modes."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    dx = 1.0 / shape[0]
    p = Problem("periodic_box", shape, (0.0, 0.0, 0.0), dx, gamma,
                (BC_PERIODIC,) * 6, GRAV_NONE, _uniform_tables(), cfl=0.7, steps=20,
                seed=seed, extra=dict(nmodes=nmodes, kmax=kmax, mach=mach))
    return p


def strat_box(shape=(128, 128, 128), seed: int = 2810, g0: float = 1.25,
              heat_rate: float = 2e-3, noise: float = 1e-3, mu_ratio: float = 1.0 / 1.3,
              z_if: float = 0.7, width: float = 0.01, gamma: float = 5.0 / 3.0) -> Problem:
    """n=1.5 polytropic layer on [0,Lx]x[0,Ly]x[0,1], gravity -g0 z_hat,
    rho0=(1-z/2)^1.5 s(z), p0 re-integrated so that dp0/dz = -g0 rho0 where
    s(z) = 1 - FV0 + FV0*mu_ratio accounts for the light fluid above z_if."""
    nx, ny, nz = shape
    dx = 1.0 / nz
    ds = dx / 16.0
    s = np.arange(-8 * 16, (nz + 8) * 16 + 1) * ds
    fv0 = 0.5 * (1.0 + np.tanh((s - z_if) / width))
    scale = 1.0 - fv0 + fv0 * mu_ratio
    rho_poly = np.maximum(1.0 - s / 2.0, 1e-6) ** 1.5
    rho0 = rho_poly * scale
    g = -g0 * np.ones_like(s)
    # integrate from s=0 upward and downward (ghost region below 0)
    i0 = 8 * 16
    p_up = _integrate_pressure(s[i0:], rho0[i0:], g[i0:], 1.0)
    p_dn = _integrate_pressure(s[i0::-1], rho0[i0::-1], g[i0::-1], 1.0)[::-1]
    p0 = np.concatenate([p_dn[:-1], p_up])
    heat = heat_rate * 0.5 * (1.0 - np.tanh((s - 0.1) / 0.01))
    damp = np.zeros_like(s)
    tab = Tables(s0=float(s[0]), ds=ds, rho0=rho0, p0=p0, g=g, heat=heat, damp=damp)
    return Problem("strat_box", tuple(shape), (0.0, 0.0, 0.0), dx, gamma,
                   (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_REFLECT, BC_REFLECT),
                   GRAV_PLANE_Z, tab, cfl=0.7, steps=200, seed=seed,
                   extra=dict(noise=noise, z_if=z_if, width=width, mu_ratio=mu_ratio))


def sphere(n: int = 1024, seed: int = 5810, xi_R: float = 3.0, gamma: float = 5.0 / 3.0,
           mach: float = 0.03, heat_rate: float = 1e-3, tau_damp: float = 2.0,
           mu_ratio: float = 1.0 / 1.3, r_if: float = 0.6, width: float = 0.01,
           nmodes: int = 8, kmax: int = 6, shape=None, confine: bool = False,
           taper_cells=(6.0, 2.0)) -> Problem:
    """Sphere-in-cube on [-1,1]^3 (R=1): n=3 polytrope with xi(R)=xi_R so the
    cube corners (r=sqrt 3) stay inside the star; rho0=theta^3 s(r),
    g = 4 theta'(xi)/alpha (alpha=R/xi_R), p0 re-integrated from the centre.

    confine=True: the star is enclosed in the sphere of radius 1 inscribed in
    the cube, and gravity falls smoothly to zero between taper_cells[0] and
    taper_cells[1] cells inside that sphere (cubic smoothstep in r), with p0
    integrated against the tapered gravity so the base stays hydrostatic."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    nx, ny, nz = shape
    L = 2.0
    dx = L / nz
    alpha = 1.0 / xi_R
    r_max = math.sqrt(3.0) * 1.02
    h = (r_max / alpha) / 8192.0
    xi, th, dth = lane_emden(3.0, r_max / alpha + 2 * h, h)
    r = xi * alpha
    # table on uniform r grid with spacing alpha*h
    fv0 = 0.5 * (1.0 + np.tanh((r - r_if) / width))
    scale = 1.0 - fv0 + fv0 * mu_ratio
    rho0 = th ** 3 * scale
    g = 4.0 * dth / alpha
    if confine:
        r_in, r_out = 1.0 - taper_cells[0] * dx, 1.0 - taper_cells[1] * dx
        t = np.clip((r_out - r) / (r_out - r_in), 0.0, 1.0)
        g = g * (t * t * (3.0 - 2.0 * t))
    p0 = _integrate_pressure(r, rho0, g, 1.0)
    heat = heat_rate * 0.25 * (1.0 + np.tanh((r - 0.25) / 0.01)) * (1.0 - np.tanh((r - 0.3) / 0.01))
    damp = (1.0 / tau_damp) * (0.5 * (1.0 - np.tanh((r - 0.2) / 0.01))
                               + 0.5 * (1.0 + np.tanh((r - 0.95) / 0.01)))
    tab = Tables(s0=0.0, ds=alpha * h, rho0=rho0, p0=p0, g=g, heat=heat, damp=damp)
    return Problem("sphere", shape, (-1.0, -1.0, -1.0), dx, gamma, (BC_REFLECT,) * 6,
                   GRAV_CENTRAL, tab, cfl=0.7, steps=100, seed=seed,
                   extra=dict(mach=mach, r_if=r_if, width=width, mu_ratio=mu_ratio,
                              nmodes=nmodes, kmax=kmax), confine_r=1.0 if confine else 0.0)


def ensemble_boxes(nbox: int = 24, seed: int = 3810, sizes=tuple(range(48, 193, 16))) -> List[Problem]:
    """Batched-ensemble workload: nbox stratified boxes whose three extents are
    drawn independently from `sizes` (48..192 in steps of 16, so shapes such
    as 64x128x96 occur), each with its own heating rate (log-uniform in
    [1e-4, 1e-2]) and its own noise seed."""
    rng = SplitMix64(seed)
    out = []
    for b in range(nbox):
        shape = tuple(sizes[int(rng.uniform() * len(sizes))] for _ in range(3))
        rate = 10.0 ** (-4.0 + 2.0 * rng.uniform())
        p = strat_box(shape=shape, seed=seed * 1000 + b, heat_rate=rate)
        p.name = "strat_box"
        p.extra["box"] = b
        p.extra["heat_rate"] = rate
        out.append(p)
    return out


def tube(kind: str = "sod", n: int = 100, axis: int = 0, ntrans: int = 4,
         gamma: float = 1.4, length: float = 1.0) -> Problem:
    """Sod or Lax shock tube along `axis` on [0.5-L/2, 0.5+L/2] with n cells
    per unit length, interface at x=0.5, reflecting ends, `ntrans` periodic
    cells across.  L > 1 keeps waves launched at the walls out of [0,1]."""
    shape = [ntrans, ntrans, ntrans]
    shape[axis] = int(round(n * length))
    bc = [BC_PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = BC_REFLECT
    origin = [0.0, 0.0, 0.0]
    origin[axis] = 0.5 - 0.5 * length
    return Problem(f"tube_{kind}", tuple(shape), tuple(origin), 1.0 / n, gamma,
                   tuple(bc), GRAV_NONE, _uniform_tables(1.0, 1.0), cfl=0.6, steps=0,
                   extra=dict(kind=kind, axis=axis, length=length))


TUBE_STATES = {
    # (rho, u, p) left | right, interface x=0.5
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.2),
    "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.13),
}


def wave(n: int = 32, axis: int = 0, kind: str = "density", u: float = 1.0,
         ntrans: int = 4, gamma: float = 1.4) -> Problem:
    """Periodic 1-D smooth advection along `axis`: 'density' is
    rho = 1 + 0.2 sin(2 pi x), u, p = 1; 'fv' is a smooth FV bump."""
    shape = [ntrans, ntrans, ntrans]
    shape[axis] = n
    return Problem(f"wave_{kind}", tuple(shape), (0.0, 0.0, 0.0), 1.0 / n, gamma,
                   (BC_PERIODIC,) * 6, GRAV_NONE, _uniform_tables(1.0, 1.0), cfl=0.5,
                   steps=0, extra=dict(kind=kind, axis=axis, u=u))


# --------------------------------------------------------------------------
# Initial states
# --------------------------------------------------------------------------
def _empty_state(shape_zyx, device):
    return [torch.zeros(shape_zyx, dtype=torch.float64, device=device) for _ in range(NVAR)]


def _fv_cell_1d(s_c: torch.Tensor, ds: float, s_if: float, width: float):
    """Cell average and normalised first moment 12*int xi f dxi of the tanh
    profile along one coordinate, by 8-point Gauss-Legendre quadrature."""
    avg = torch.zeros_like(s_c)
    mom = torch.zeros_like(s_c)
    for xg, wg in zip(_GL8_X, _GL8_W):
        f = _tanh_profile(s_c + xg * ds, s_if, width)
        avg += wg * f
        mom += wg * xg * f
    return avg, 12.0 * mom


def initial_state(p: Problem, device="cpu", z_lo: int = 0, z_hi: Optional[int] = None):
    """Initial state (full variables) for z-planes [z_lo, z_hi)."""
    nx, ny, nz = p.shape
    if z_hi is None:
        z_hi = nz
    x, y, z = _cell_coords(p, device, z_lo, z_hi)
    shp = (z_hi - z_lo, ny, nx)
    q = _empty_state(shp, device)
    gm1 = p.gamma - 1.0
    if p.name == "periodic_box":
        rng = SplitMix64(p.seed)
        modes = _fourier_modes(rng, p.extra["nmodes"], p.extra["kmax"])
        u = _velocity_from_modes(modes, x, y, z, 1.0)
        # normalise to rms Mach using the mode amplitudes (exact mean square of
        # the sum over the periodic grid is computed on a full grid once)
        scale = p.extra["mach"] * math.sqrt(p.gamma) / _grid_rms_modes(modes, p, device)
        rho = torch.ones(shp, dtype=torch.float64, device=device)
        q[0] = rho
        for d in range(3):
            q[1 + d] = rho * (scale * u[d])
        ke = 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / rho
        q[4] = 1.0 / gm1 + ke
        fv, mz = _fv_cell_1d(z, p.dx, 0.5, 0.05)
        fv, (mz,) = _valid_fv(fv, [mz])
        q[5] = fv.view(-1, 1, 1).expand(shp).clone()
        q[8] = mz.view(-1, 1, 1).expand(shp).clone()
        return q
    if p.name == "strat_box":
        t = p.tables
        rho0 = _lerp_table(t.rho0, t.s0, t.ds, z).view(-1, 1, 1)
        p0 = _lerp_table(t.p0, t.s0, t.ds, z).view(-1, 1, 1)
        noise = splitmix_field(p.seed, shp, offset=z_lo * nx * ny, device=device)
        rho = rho0 * (1.0 + p.extra["noise"] * (2.0 * noise - 1.0))
        q[0] = rho
        q[4] = (p0 / gm1).expand(shp).clone()
        fv, mz = _fv_cell_1d(z, p.dx, p.extra["z_if"], p.extra["width"])
        fv, (mz,) = _valid_fv(fv, [mz])
        q[5] = fv.view(-1, 1, 1).expand(shp).clone()
        q[8] = mz.view(-1, 1, 1).expand(shp).clone()
        return q
    if p.name == "sphere":
        t = p.tables
        X = x.view(1, 1, -1)
        Y = y.view(1, -1, 1)
        Z = z.view(-1, 1, 1)
        r = _sqrt(X * X + Y * Y + Z * Z)
        rho0 = _lerp_table(t.rho0, t.s0, t.ds, r)
        p0 = _lerp_table(t.p0, t.s0, t.ds, r)
        rng = SplitMix64(p.seed)
        modes = _fourier_modes(rng, p.extra["nmodes"], p.extra["kmax"])
        u = _velocity_from_modes(modes, x, y, z, 2.0)
        # window: convection zone 0.25<r<0.6 with smooth edges
        win = 0.25 * (1.0 + torch.tanh((r - 0.25) / 0.02)) * (1.0 - torch.tanh((r - 0.6) / 0.02))
        c = _sqrt(p.gamma * p0 / rho0)
        amp = p.extra["mach"] / _modes_rms(modes)
        q[0] = rho0
        for d in range(3):
            q[1 + d] = rho0 * (amp * win * c * u[d])
        ke = 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / rho0
        q[4] = p0 / gm1 + ke
        # FV cell average and moments: 3-point Gauss-Legendre tensor quadrature
        r_if, w_if = p.extra["r_if"], p.extra["width"]
        fv = torch.zeros(shp, dtype=torch.float64, device=device)
        mx = torch.zeros_like(fv)
        my = torch.zeros_like(fv)
        mz = torch.zeros_like(fv)
        for a, wa in zip(_GL3_X, _GL3_W):
            for b, wb in zip(_GL3_X, _GL3_W):
                for cc, wc in zip(_GL3_X, _GL3_W):
                    rr = _sqrt((X + a * p.dx) ** 2 + (Y + b * p.dx) ** 2 + (Z + cc * p.dx) ** 2)
                    f = _tanh_profile(rr, r_if, w_if) * (wa * wb * wc)
                    fv += f
                    mx += a * f
                    my += b * f
                    mz += cc * f
        fv, (mx, my, mz) = _valid_fv(fv, [12.0 * mx, 12.0 * my, 12.0 * mz])
        q[5], q[6], q[7], q[8] = fv, mx, my, mz
        return q
    if p.name.startswith("tube_"):
        (rl, ul, pl), (rr_, ur, pr), _ = TUBE_STATES[p.extra["kind"]]
        axis = p.extra["axis"]
        coord = (x, y, z)[axis]
        left = (coord < 0.5)
        view = [1, 1, 1]
        view[2 - axis] = -1
        left = left.view(view).expand(shp)
        rho = torch.where(left, torch.tensor(rl, dtype=torch.float64), torch.tensor(rr_, dtype=torch.float64))
        vel = torch.where(left, torch.tensor(ul, dtype=torch.float64), torch.tensor(ur, dtype=torch.float64))
        pr_ = torch.where(left, torch.tensor(pl, dtype=torch.float64), torch.tensor(pr, dtype=torch.float64))
        q[0] = rho
        q[1 + axis] = rho * vel
        q[4] = pr_ / gm1 + 0.5 * rho * vel * vel
        return q
    if p.name.startswith("wave_"):
        axis = p.extra["axis"]
        coord = (x, y, z)[axis]
        view = [1, 1, 1]
        view[2 - axis] = -1
        uu = p.extra["u"]
        if p.extra["kind"] == "density":
            rho = wave_density_average(coord, p.dx).view(view).expand(shp)
            fv = torch.zeros_like(rho)
            mom = torch.zeros_like(rho)
        else:
            rho = torch.ones(shp, dtype=torch.float64, device=device)
            f_avg, f_mom = wave_fv_cell(coord, p.dx)
            fv = f_avg.view(view).expand(shp)
            mom = f_mom.view(view).expand(shp)
        q[0] = rho.clone()
        q[1 + axis] = rho * uu
        q[4] = 1.0 / gm1 + 0.5 * rho * uu * uu
        q[5] = fv.clone()
        q[6 + axis] = mom.clone()
        return q
    raise ValueError(p.name)


def wave_density_average(x_c: torch.Tensor, dx: float) -> torch.Tensor:
    """Exact cell average of 1 + 0.2 sin(2 pi x) over [x_c-dx/2, x_c+dx/2]."""
    k = 2.0 * math.pi
    return 1.0 + 0.2 * torch.sin(k * x_c) * (math.sin(k * dx / 2) / (k * dx / 2))


def wave_fv_profile(x: torch.Tensor) -> torch.Tensor:
    """Smooth periodic FV bump 0.5 + 0.4 sin(2 pi x) (stays inside [0.1,0.9])."""
    return 0.5 + 0.4 * torch.sin(2.0 * math.pi * x)


def wave_fv_cell(x_c: torch.Tensor, dx: float):
    avg = torch.zeros_like(x_c)
    mom = torch.zeros_like(x_c)
    for xg, wg in zip(_GL8_X, _GL8_W):
        f = wave_fv_profile(x_c + xg * dx)
        avg += wg * f
        mom += wg * xg * f
    return avg, 12.0 * mom


def _grid_rms_modes(modes, p: Problem, device) -> float:
    x, y, z = _cell_coords(p, "cpu")
    u = _velocity_from_modes(modes, x, y, z, 1.0)
    ms = sum(float((ud ** 2).mean()) for ud in u)
    return math.sqrt(ms)


def state_numpy(q: Sequence[torch.Tensor]) -> List[np.ndarray]:
    return [np.ascontiguousarray(t.detach().cpu().numpy()) for t in q]


def build(p: Problem, device="cpu"):
    """Initial state as a list of 9 contiguous float64 numpy arrays (z, y, x)."""
    return state_numpy(initial_state(p, device))
