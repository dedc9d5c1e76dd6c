"""ctypes binding to the FP64 CPU oracle (``liboracle.so``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it.  The CUDA library never imports it.

``build()`` compiles ``ppm_oracle.cpp`` with g++ (-O2 -fopenmp
-ffp-contract=off) into this directory; ``Oracle(problem)`` wraps one problem
description from :mod:`workloads` and offers sweep / double step / CFL /
single-pencil / diagnostics / flop-census calls on float64 numpy state lists.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppm_oracle.cpp")
_HDR = os.path.join(_HERE, "ppm_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_DP = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
        ("dx", C.c_double), ("gamma", C.c_double),
        ("bc", C.c_int * 6),
        ("grav", C.c_int),
        ("ntab", C.c_int),
        ("s0", C.c_double), ("ds", C.c_double),
        ("rho0", _DP), ("p0", _DP), ("g", _DP), ("heat", _DP), ("damp", _DP),
        ("confine_r", C.c_double), ("domega", C.c_double), ("nmom", C.c_int),
        ("shock_k", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or older than its sources."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                   "-shared", "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.POINTER(_Problem)
        Q = C.POINTER(_DP)
        lib.oracle_sweep.argtypes = [P, Q, C.c_int, C.c_double, C.c_int]
        lib.oracle_double_step.argtypes = [P, Q, C.c_double]
        lib.oracle_cfl_dt.argtypes = [P, Q, C.c_double]
        lib.oracle_cfl_dt.restype = C.c_double
        lib.oracle_sweep_pencil.argtypes = [P, C.c_int, C.c_int, C.c_int, Q, Q, C.c_double, C.c_int]
        lib.oracle_diagnostics.argtypes = [P, Q, _DP, C.c_int, C.c_double, _DP, _DP]
        lib.oracle_sweep_z_slab.argtypes = [P, Q, C.c_int, C.c_int, C.c_double, C.c_int]
        lib.oracle_counters.argtypes = [C.POINTER(C.c_longlong)]
        lib.oracle_divergence.argtypes = [P, Q, _DP]
        lib.oracle_reset_counters.argtypes = []
        lib.oracle_count_flops.argtypes = [P, Q, C.c_int, C.c_double, _DP]
        lib.oracle_set_threads.argtypes = [C.c_int]
        lib.oracle_get_threads.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


class Oracle:
    """One problem (grid, gas, boundaries, base-state and source tables)."""

    def __init__(self, problem):
        self.lib = _load()
        p = problem
        t = p.tables
        self._keep = []

        def arr(x):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
            self._keep.append(a)
            return a

        rho0, p0, g = arr(t.rho0), arr(t.p0), arr(t.g)
        heat, damp = arr(t.heat), arr(t.damp)
        s = _Problem()
        s.nx, s.ny, s.nz = p.shape
        s.x0, s.y0, s.z0 = p.origin
        s.dx = p.dx
        s.gamma = p.gamma
        for i in range(6):
            s.bc[i] = int(p.bc[i])
        s.grav = int(p.grav)
        s.ntab = int(rho0.shape[0])
        s.s0, s.ds = float(t.s0), float(t.ds)
        s.rho0, s.p0, s.g = _ptr(rho0), _ptr(p0), _ptr(g)
        s.heat = _ptr(heat) if heat is not None else None
        s.damp = _ptr(damp) if damp is not None else None
        s.confine_r = float(getattr(p, "confine_r", 0.0) or 0.0)
        s.domega = 0.0
        s.nmom = int(getattr(p, "nmom", 3) or 3)
        if s.nmom not in (3, 9):
            raise ValueError("nmom must be 3 or 9")
        self.nvar = 15 if s.nmom == 9 else 9
        s.shock_k = float(getattr(p, "shock_k", 0.0) or 0.0)
        if s.shock_k > 0.0 and s.confine_r > 0.0:
            raise ValueError("shock dissipation is not combined with a confining sphere")
        self.s = s
        self.problem = p

    def _q(self, q: Sequence[np.ndarray]):
        assert len(q) == self.nvar, (len(q), self.nvar)
        n = self.problem.ncell
        for a in q:
            assert a.size == n, (a.shape, n)
        return (_DP * 15)(*[_ptr(a) for a in q])

    def set_rotation(self, domega: float):
        """Rotation increment added once per double step (0 = none)."""
        self.s.domega = float(domega)

    def sweep(self, q, axis: int, dt: float, sources: int = 0):
        """sources: 1 (or True) heating/damping, 2 rotation increment, 3 both."""
        self.lib.oracle_sweep(C.byref(self.s), self._q(q), axis, dt, int(sources))

    def double_step(self, q, dt: float):
        self.lib.oracle_double_step(C.byref(self.s), self._q(q), dt)

    def cfl_dt(self, q, cfl: Optional[float] = None) -> float:
        c = self.problem.cfl if cfl is None else cfl
        return self.lib.oracle_cfl_dt(C.byref(self.s), self._q(q), c)

    def sweep_pencil(self, pencil_in: Sequence[np.ndarray], axis: int, ja: int, jb: int,
                     dt: float, sources: bool = False) -> List[np.ndarray]:
        """One pass of one pencil (the 3-D shock dissipation needs the whole
        grid and is not applied here)."""
        n = self.problem.shape[axis]
        pin = [np.ascontiguousarray(a, dtype=np.float64) for a in pencil_in]
        assert len(pin) == self.nvar
        for a in pin:
            assert a.size == n
        out = [np.zeros(n) for _ in range(self.nvar)]
        self.lib.oracle_sweep_pencil(C.byref(self.s), axis, ja, jb,
                                     (_DP * 15)(*[_ptr(a) for a in pin]),
                                     (_DP * 15)(*[_ptr(a) for a in out]), dt, int(sources))
        return out

    def sweep_z_slab(self, qloc, k0: int, nzl: int, dt: float, sources: bool = False):
        """z pass of global planes [k0, k0+nzl) given with 4 halo planes on
        each side (qloc: 9 arrays of shape (nzl+8, ny, nx))."""
        nx, ny, _ = self.problem.shape
        if self.s.confine_r > 0.0 or self.s.nmom == 9 or self.s.shock_k > 0.0:
            raise ValueError("sweep_z_slab: no confining sphere, first moments only, no shock dissipation")
        for a in qloc:
            assert a.shape == (nzl + 8, ny, nx) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        self.lib.oracle_sweep_z_slab(C.byref(self.s), (_DP * 9)(*[_ptr(a) for a in qloc]), int(k0), int(nzl),
                                     dt, int(sources))

    def diagnostics(self, q, nbins: int = 0, rmax: float = 1.0):
        tot = np.zeros(7)
        prof = np.zeros(max(nbins, 1) * 5)
        mm = np.zeros(1)
        self.lib.oracle_diagnostics(C.byref(self.s), self._q(q), _ptr(tot), nbins, rmax,
                                    _ptr(prof), _ptr(mm))
        return tot, prof[: nbins * 5].reshape(nbins, 5), float(mm[0])

    def divergence(self, q) -> np.ndarray:
        """Cell velocity divergence used by the shock dissipation."""
        out = np.zeros(self.problem.ncell)
        self.lib.oracle_divergence(C.byref(self.s), self._q(q), _ptr(out))
        nx, ny, nz = self.problem.shape
        return out.reshape(nz, ny, nx)

    def count_flops(self, q, axis: int, dt: float):
        out = np.zeros(2)
        self.lib.oracle_count_flops(C.byref(self.s), self._q(q), axis, dt, _ptr(out))
        return float(out[0]), float(out[1])

    @staticmethod
    def counters():
        lib = _load()
        out = (C.c_longlong * 8)()
        lib.oracle_counters(out)
        keys = ("nonsmooth", "flattened", "theta_limited", "fct_limited", "moment_clamped", "cells",
                "dissipative_faces", "supersonic_faces")
        return dict(zip(keys, list(out)))

    @staticmethod
    def reset_counters():
        _load().oracle_reset_counters()

    @staticmethod
    def set_threads(n: int):
        _load().oracle_set_threads(int(n))

    @staticmethod
    def threads() -> int:
        return int(_load().oracle_get_threads())


def run(problem, q, steps: int, cfl: Optional[float] = None):
    """Advance `steps` double steps, recomputing dt before each; returns dts."""
    o = Oracle(problem)
    dts = []
    for _ in range(steps):
        dt = o.cfl_dt(q, cfl)
        o.double_step(q, dt)
        dts.append(dt)
    return dts
