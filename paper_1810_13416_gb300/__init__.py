"""GB300-native PPM + PPB multifluid sweeps: Python binding of libppm.so.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libppm.so`` (built from ``csrc/`` by :func:`build`).  The calls have the
names of the C ABI in ``include/ppm.h``:

    ctx = Context(shape, gamma, bc, grav_kind, tables, origin, dx, precision)
    ctx.set_state(q)          # 9 float64 arrays, full variables, (nz, ny, nx)
    dt = ctx.cfl_dt(0.7)
    ctx.step(dt)              # one Strang double step X Y Z [src] Z Y X [src]
    q = ctx.get_state()
    totals, profiles, max_mach = ctx.diagnostics(nbins, rmax)

PyTorch is only used, where a caller wants it, for device buffers and
streams (``set_region(..., device tensors)``, ``stream=torch stream``).
There is no CPU fallback: if the library is missing the import of a
Context fails.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build_mod

__all__ = ["Context", "Ensemble", "PpmError", "build", "library_path", "FP64_PLAIN", "FP32_DEVIATION",
           "BC_PERIODIC", "BC_REFLECT", "GRAV_NONE", "GRAV_PLANE_Z", "GRAV_CENTRAL"]

FP64_PLAIN = 0
FP32_DEVIATION = 1
PASS_MARCH = 0      # one thread per pencil, register window
PASS_TILE = 1       # cell-parallel tiles of 8 pencils x 32 cells, TMA staging
ENS_PER_PASS = 0    # ensemble: one launch per pass
ENS_ONE_LAUNCH = 1  # ensemble: the whole double step in one launch
BC_PERIODIC = 0
BC_REFLECT = 1
GRAV_NONE = 0
GRAV_PLANE_Z = 1
GRAV_CENTRAL = 2
MEM_HOST = 0
MEM_DEVICE = 1

STATUS = {0: "PPM_OK", -1: "PPM_EINVAL", -2: "PPM_ENOMEM", -3: "PPM_ECUDA", -4: "PPM_ENONPHYS",
          -5: "PPM_ECFL", -6: "PPM_ETIMEOUT", -7: "PPM_ESTATE"}

_DP = C.POINTER(C.c_double)
_lib = None


class PpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Gravity(C.Structure):
    _fields_ = [("kind", C.c_int), ("ntab", C.c_int), ("s0", C.c_double), ("ds", C.c_double),
                ("rho0", _DP), ("p0", _DP), ("g", _DP)]


class _Options(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double), ("dx", C.c_double),
                ("precision", C.c_int), ("heat", _DP), ("damp", _DP), ("stream", C.c_void_p),
                ("device", C.c_int), ("confine_r", C.c_double), ("nmom", C.c_int),
                ("shock_k", C.c_double), ("halo_z", C.c_int), ("z_index0", C.c_int)]


class _Box(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("bc", C.c_int * 6), ("grav", _Gravity), ("x0", C.c_double),
                ("y0", C.c_double), ("z0", C.c_double), ("dx", C.c_double), ("heat", _DP), ("damp", _DP)]


def build(force: bool = False, verbose: bool = False) -> str:
    return _build_mod.build(force=force, verbose=verbose)


def library_path() -> str:
    return _build_mod.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build_mod.LIB
    if not os.path.exists(path):
        raise ImportError(f"libppm.so is not built ({path}); run paper_1810_13416_gb300.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    Q = C.POINTER(_DP)   # 6 + nmom array pointers
    I3 = C.c_int * 3
    lib.ppm_create.argtypes = [C.POINTER(P), C.c_int, C.c_int, C.c_int, C.c_double, C.c_int * 6,
                               C.POINTER(_Gravity), C.POINTER(_Options)]
    lib.ppm_set_state.argtypes = [P, Q]
    lib.ppm_get_state.argtypes = [P, Q]
    lib.ppm_set_region.argtypes = [P, I3, I3, Q, C.c_int]
    lib.ppm_get_region.argtypes = [P, I3, I3, Q, C.c_int]
    lib.ppm_cfl_dt.argtypes = [P, C.c_double, _DP]
    lib.ppm_step.argtypes = [P, C.c_double]
    lib.ppm_sweep.argtypes = [P, C.c_int, C.c_double, C.c_int]
    lib.ppm_set_rotation.argtypes = [P, C.c_double]
    lib.ppm_set_pass_design.argtypes = [P, C.c_int]
    lib.ppm_get_pass_design.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.ppm_set_pass_designs.argtypes = [P, C.POINTER(C.c_int)]
    lib.ppm_tune.argtypes = [P, C.c_char_p, C.POINTER(C.c_int)]
    lib.ppm_pass_times.argtypes = [P, _DP]
    lib.ppm_slab_halo.argtypes = [P, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]
    lib.ppm_slab_pack.argtypes = [P, C.c_int, C.c_void_p]
    lib.ppm_diagnostics.argtypes = [P, _DP, C.c_int, C.c_double, _DP, _DP]
    lib.ppm_sync.argtypes = [P]
    lib.ppm_launch_count.argtypes = [P]
    lib.ppm_launch_count.restype = C.c_longlong
    lib.ppm_last_error.argtypes = [P]
    lib.ppm_last_error.restype = C.c_char_p
    lib.ppm_destroy.argtypes = [P]
    lib.ppm_destroy.restype = None
    lib.ppm_ensemble_create.argtypes = [C.POINTER(P), C.c_int, C.POINTER(_Box), C.c_double, C.c_int, C.c_void_p,
                                        C.c_int]
    lib.ppm_ensemble_set_state.argtypes = [P, C.c_int, Q]
    lib.ppm_ensemble_set_region.argtypes = [P, C.c_int, I3, I3, Q, C.c_int]
    lib.ppm_ensemble_get_state.argtypes = [P, C.c_int, Q]
    lib.ppm_ensemble_cfl_dt.argtypes = [P, C.c_double, _DP]
    lib.ppm_ensemble_step.argtypes = [P, C.c_double]
    lib.ppm_ensemble_diagnostics.argtypes = [P, C.c_int, _DP, _DP]
    lib.ppm_ensemble_sync.argtypes = [P]
    lib.ppm_ensemble_set_config.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.ppm_ensemble_get_config.argtypes = [P, C.POINTER(C.c_int)]
    lib.ppm_ensemble_tune.argtypes = [P, C.c_char_p, C.POINTER(C.c_int)]
    lib.ppm_ensemble_set_launch_mode.argtypes = [P, C.c_int]
    lib.ppm_ensemble_get_launch_mode.argtypes = [P]
    lib.ppm_ensemble_set_wait_test.argtypes = [P, C.c_int]
    lib.ppm_ensemble_launch_count.argtypes = [P]
    lib.ppm_ensemble_launch_count.restype = C.c_longlong
    lib.ppm_ensemble_last_error.argtypes = [P]
    lib.ppm_ensemble_last_error.restype = C.c_char_p
    lib.ppm_ensemble_destroy.argtypes = [P]
    lib.ppm_ensemble_destroy.restype = None
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptrs(arrs) -> "C.Array":
    return (_DP * len(arrs))(*[a.ctypes.data_as(_DP) for a in arrs])


class Context:
    """One grid on one GPU (a ``ppm_ctx``)."""

    def __init__(self, shape, gamma: float, bc: Sequence[int], grav_kind: int, s0: float, ds: float,
                 rho0, p0, g, origin=(0.0, 0.0, 0.0), dx: float = 1.0, precision: int = FP32_DEVIATION,
                 heat=None, damp=None, stream=None, device: int = 0, confine_r: float = 0.0,
                 nmom: int = 3, shock_k: float = 0.0, halo_z: int = 0, z_index0: int = 0):
        self.lib = _load()
        self.shape = tuple(int(v) for v in shape)
        self._keep = [_f64(rho0), _f64(p0), _f64(g)]
        gr = _Gravity(int(grav_kind), int(self._keep[0].size), float(s0), float(ds),
                      self._keep[0].ctypes.data_as(_DP), self._keep[1].ctypes.data_as(_DP),
                      self._keep[2].ctypes.data_as(_DP))
        hp = dp = None
        if heat is not None:
            self._keep.append(_f64(heat))
            hp = self._keep[-1].ctypes.data_as(_DP)
        if damp is not None:
            self._keep.append(_f64(damp))
            dp = self._keep[-1].ctypes.data_as(_DP)
        sptr = None
        if stream is not None:
            sptr = int(getattr(stream, "cuda_stream", stream))
        opt = _Options(float(origin[0]), float(origin[1]), float(origin[2]), float(dx), int(precision),
                       hp, dp, sptr, int(device), float(confine_r), int(nmom), float(shock_k), int(halo_z),
                       int(z_index0))
        h = C.c_void_p()
        rc = self.lib.ppm_create(C.byref(h), self.shape[0], self.shape[1], self.shape[2], float(gamma),
                                 (C.c_int * 6)(*[int(b) for b in bc]), C.byref(gr), C.byref(opt))
        if rc != 0:
            raise PpmError(rc, self.lib.ppm_last_error(None).decode())
        self.h = h
        self.precision = precision
        self.nvar = 15 if int(nmom) == 9 else 9
        self.ncell = self.shape[0] * self.shape[1] * self.shape[2]

    @classmethod
    def slab(cls, p, k0: int, nzl: int, halo_z: int, precision: int = FP32_DEVIATION, stream=None,
             device: int = 0):
        """The z slab of planes [k0, k0 + nzl) of problem p, as its own
        context: the whole grid's origin with the slab's global z index k0
        (so positions are computed exactly as on the whole grid); halo_z
        bit 0 / bit 1 = its low / high z face takes halo planes (ppm_slab_halo)."""
        t = p.tables
        shape = (p.shape[0], p.shape[1], int(nzl))
        return cls(shape, p.gamma, p.bc, p.grav, t.s0, t.ds, t.rho0, t.p0, t.g, origin=p.origin,
                   dx=p.dx, precision=precision, heat=getattr(t, "heat", None),
                   damp=getattr(t, "damp", None), stream=stream, device=device, halo_z=int(halo_z),
                   z_index0=int(k0))

    def slab_halo(self, side: int):
        """(device address, bytes) of the low (0) or high (1) halo planes."""
        ptr, n = C.c_void_p(), C.c_size_t()
        self._check(self.lib.ppm_slab_halo(self.h, int(side), C.byref(ptr), C.byref(n)))
        return int(ptr.value), int(n.value)

    def slab_pack(self, side: int, dst: int):
        """Copy this context's 4 boundary planes of `side` to device address dst."""
        self._check(self.lib.ppm_slab_pack(self.h, int(side), C.c_void_p(int(dst))))

    @classmethod
    def from_problem(cls, p, precision: int = FP32_DEVIATION, stream=None, device: int = 0):
        """Build from any object with the fields of a problem description
        (shape, gamma, bc, grav, tables(s0, ds, rho0, p0, g, heat, damp),
        origin, dx, optional confine_r)."""
        t = p.tables
        return cls(p.shape, p.gamma, p.bc, p.grav, t.s0, t.ds, t.rho0, t.p0, t.g, origin=p.origin,
                   dx=p.dx, precision=precision, heat=getattr(t, "heat", None),
                   damp=getattr(t, "damp", None), stream=stream, device=device,
                   confine_r=float(getattr(p, "confine_r", 0.0) or 0.0),
                   nmom=int(getattr(p, "nmom", 3) or 3),
                   shock_k=float(getattr(p, "shock_k", 0.0) or 0.0))

    # ------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise PpmError(rc, self.lib.ppm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.ppm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------
    def set_state(self, q: Sequence[np.ndarray]):
        arrs = [_f64(a) for a in q]
        assert len(arrs) == self.nvar and all(a.size == self.ncell for a in arrs)
        self._check(self.lib.ppm_set_state(self.h, _ptrs(arrs)))

    def get_state(self) -> List[np.ndarray]:
        nx, ny, nz = self.shape
        out = [np.empty((nz, ny, nx)) for _ in range(self.nvar)]
        self._check(self.lib.ppm_get_state(self.h, _ptrs(out)))
        return out

    def get_state_into(self, out: Sequence[np.ndarray]):
        assert len(out) == self.nvar and all(
            a.dtype == np.float64 and a.size == self.ncell and a.flags.c_contiguous for a in out)
        self._check(self.lib.ppm_get_state(self.h, _ptrs(out)))

    @staticmethod
    def _sync_torch():
        # device tensors may still be in production on torch's streams, which
        # the library's stream does not wait for
        import torch
        torch.cuda.synchronize()

    def set_region(self, lo, hi, q, device: bool = False):
        """q: 6 + nmom host float64 arrays, or CUDA float64 tensors when device=True."""
        assert len(q) == self.nvar
        nb = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        if device:
            import torch
            assert all(t.dtype == torch.float64 and t.numel() == nb and t.is_contiguous() for t in q)
            self._sync_torch()
            ptrs = (_DP * len(q))(*[C.cast(C.c_void_p(int(t.data_ptr())), _DP) for t in q])
        else:
            q = [_f64(a) for a in q]
            assert all(a.size == nb for a in q)
            ptrs = _ptrs(q)
        self._check(self.lib.ppm_set_region(self.h, (C.c_int * 3)(*lo), (C.c_int * 3)(*hi), ptrs,
                                            MEM_DEVICE if device else MEM_HOST))

    def get_region(self, lo, hi, out=None, device: bool = False):
        b = [hi[d] - lo[d] for d in range(3)]
        if out is None:
            out = [np.empty((b[2], b[1], b[0])) for _ in range(self.nvar)]
        assert len(out) == self.nvar
        nb = b[0] * b[1] * b[2]
        if device:
            import torch
            assert all(t.dtype == torch.float64 and t.numel() == nb and t.is_contiguous() for t in out)
            self._sync_torch()
            ptrs = (_DP * len(out))(*[C.cast(C.c_void_p(int(t.data_ptr())), _DP) for t in out])
        else:
            assert all(a.dtype == np.float64 and a.size == nb and a.flags.c_contiguous for a in out)
            ptrs = _ptrs(out)
        self._check(self.lib.ppm_get_region(self.h, (C.c_int * 3)(*lo), (C.c_int * 3)(*hi), ptrs,
                                            MEM_DEVICE if device else MEM_HOST))
        return out

    def cfl_dt(self, cfl: float, fetch: bool = True) -> Optional[float]:
        if fetch:
            v = C.c_double()
            self._check(self.lib.ppm_cfl_dt(self.h, float(cfl), C.byref(v)))
            return v.value
        self._check(self.lib.ppm_cfl_dt(self.h, float(cfl), None))
        return None

    def step(self, dt: float = 0.0):
        self._check(self.lib.ppm_step(self.h, float(dt)))

    def sweep(self, axis: int, dt: float, sources: int = 0):
        """sources: 1 (or True) heating/damping, 2 rotation increment, 3 both."""
        self._check(self.lib.ppm_sweep(self.h, int(axis), float(dt), int(sources)))

    def set_rotation(self, domega: float):
        """Rotation increment added by each following double step (0 ends the ramp)."""
        self._check(self.lib.ppm_set_rotation(self.h, float(domega)))

    def pass_times(self) -> np.ndarray:
        """Device ms of the six passes of the last double step (waits for it)."""
        out = np.zeros(6)
        self._check(self.lib.ppm_pass_times(self.h, out.ctypes.data_as(_DP)))
        return out

    def set_pass_design(self, design):
        """PASS_MARCH or PASS_TILE for every axis, or a sequence of three
        (x, y, z); PASS_TILE needs the FP32 four-value form and nx % 4 == 0."""
        if isinstance(design, (list, tuple)):
            d = (C.c_int * 3)(*[int(x) for x in design])
            self._check(self.lib.ppm_set_pass_designs(self.h, d))
        else:
            self._check(self.lib.ppm_set_pass_design(self.h, int(design)))

    def _designs(self):
        d, a = (C.c_int * 3)(), C.c_int()
        self._check(self.lib.ppm_get_pass_design(self.h, d, C.byref(a)))
        return tuple(d), bool(a.value)

    @property
    def pass_design(self):
        """The design of every axis when they agree, else the (x, y, z) tuple."""
        d, _ = self._designs()
        return d[0] if d[0] == d[1] == d[2] else d

    @property
    def pass_designs(self) -> tuple:
        return self._designs()[0]

    @property
    def tile_available(self) -> bool:
        return self._designs()[1]

    def tune(self, cache_path: Optional[str] = None) -> bool:
        """Autotune the pass design per axis; True when taken from the cache."""
        fc = C.c_int()
        self._check(self.lib.ppm_tune(self.h, cache_path.encode() if cache_path else None, C.byref(fc)))
        return bool(fc.value)

    def diagnostics(self, nbins: int = 0, rmax: float = 1.0):
        tot = np.zeros(7)
        prof = np.zeros(max(nbins, 1) * 5)
        mm = C.c_double()
        self._check(self.lib.ppm_diagnostics(self.h, tot.ctypes.data_as(_DP), int(nbins), float(rmax),
                                             prof.ctypes.data_as(_DP), C.byref(mm)))
        return tot, prof[: nbins * 5].reshape(nbins, 5), mm.value

    def sync(self):
        self._check(self.lib.ppm_sync(self.h))

    @property
    def launch_count(self) -> int:
        return int(self.lib.ppm_launch_count(self.h))


class Ensemble:
    """Independent boxes advanced together (a ``ppm_ens``): one launch per
    pass for all boxes, one graph per double step, tile configuration chosen
    by the library's autotuner."""

    def __init__(self, problems, precision: int = FP32_DEVIATION, stream=None, device: int = 0):
        self.lib = _load()
        self._keep = []
        boxes = (_Box * len(problems))()
        gammas = {float(p.gamma) for p in problems}
        if len(gammas) != 1:
            raise ValueError("all boxes of an ensemble share gamma")
        for i, p in enumerate(problems):
            t = p.tables
            arrs = [_f64(t.rho0), _f64(t.p0), _f64(t.g)]
            self._keep.extend(arrs)
            b = boxes[i]
            for d in range(3):
                b.n[d] = int(p.shape[d])
            for f in range(6):
                b.bc[f] = int(p.bc[f])
            b.grav = _Gravity(int(p.grav), int(arrs[0].size), float(t.s0), float(t.ds),
                              arrs[0].ctypes.data_as(_DP), arrs[1].ctypes.data_as(_DP), arrs[2].ctypes.data_as(_DP))
            b.x0, b.y0, b.z0 = (float(v) for v in p.origin)
            b.dx = float(p.dx)
            for name in ("heat", "damp"):
                a = getattr(t, name, None)
                if a is not None:
                    a = _f64(a)
                    self._keep.append(a)
                    setattr(b, name, a.ctypes.data_as(_DP))
        sptr = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        h = C.c_void_p()
        rc = self.lib.ppm_ensemble_create(C.byref(h), len(problems), boxes, gammas.pop(), int(precision), sptr,
                                          int(device))
        if rc != 0:
            raise PpmError(rc, self.lib.ppm_ensemble_last_error(None).decode())
        self.h = h
        self.nbox = len(problems)
        self.shapes = [tuple(int(v) for v in p.shape) for p in problems]

    def _check(self, rc: int):
        if rc != 0:
            raise PpmError(rc, self.lib.ppm_ensemble_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.ppm_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, box: int, q):
        arrs = [_f64(a) for a in q]
        nx, ny, nz = self.shapes[box]
        assert len(arrs) == 9 and all(a.size == nx * ny * nz for a in arrs)
        self._check(self.lib.ppm_ensemble_set_state(self.h, int(box), _ptrs(arrs)))

    def set_region(self, box: int, lo, hi, q, device: bool = False):
        assert len(q) == 9
        nb = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        if device:
            import torch
            assert all(t.dtype == torch.float64 and t.numel() == nb and t.is_contiguous() for t in q)
            Context._sync_torch()
            ptrs = (_DP * len(q))(*[C.cast(C.c_void_p(int(t.data_ptr())), _DP) for t in q])
        else:
            q = [_f64(a) for a in q]
            assert all(a.size == nb for a in q)
            ptrs = _ptrs(q)
        self._check(self.lib.ppm_ensemble_set_region(self.h, int(box), (C.c_int * 3)(*lo), (C.c_int * 3)(*hi),
                                                     ptrs, MEM_DEVICE if device else MEM_HOST))

    def get_state(self, box: int):
        nx, ny, nz = self.shapes[box]
        out = [np.empty((nz, ny, nx)) for _ in range(9)]
        self._check(self.lib.ppm_ensemble_get_state(self.h, int(box), _ptrs(out)))
        return out

    def cfl_dt(self, cfl: float, fetch: bool = True):
        if fetch:
            out = np.zeros(self.nbox)
            self._check(self.lib.ppm_ensemble_cfl_dt(self.h, float(cfl), out.ctypes.data_as(_DP)))
            return out
        self._check(self.lib.ppm_ensemble_cfl_dt(self.h, float(cfl), None))
        return None

    def step(self, dt: float = 0.0):
        self._check(self.lib.ppm_ensemble_step(self.h, float(dt)))

    def diagnostics(self, box: int):
        tot = np.zeros(7)
        mm = C.c_double()
        self._check(self.lib.ppm_ensemble_diagnostics(self.h, int(box), tot.ctypes.data_as(_DP), C.byref(mm)))
        return tot, mm.value

    def sync(self):
        self._check(self.lib.ppm_ensemble_sync(self.h))

    def set_config(self, axis: int, block: int, persistent: bool, vec: bool = True):
        self._check(self.lib.ppm_ensemble_set_config(self.h, int(axis), int(block), int(bool(persistent)),
                                                     int(bool(vec))))

    def config(self):
        c = (C.c_int * 7)()
        self._check(self.lib.ppm_ensemble_get_config(self.h, c))
        v = list(c)
        return {"x": (v[0], bool(v[1])), "y": (v[2], bool(v[3])), "z": (v[4], bool(v[5])), "vec_x": bool(v[6])}

    def tune(self, cache_path: Optional[str] = None) -> bool:
        """Run the autotuner; returns True when the configuration came from
        the cache file."""
        fc = C.c_int(0)
        path = cache_path.encode() if cache_path else None
        self._check(self.lib.ppm_ensemble_tune(self.h, path, C.byref(fc)))
        return bool(fc.value)

    def set_launch_mode(self, mode: int):
        """ENS_PER_PASS (one launch per pass) or ENS_ONE_LAUNCH (the double
        step of every box in one launch)."""
        self._check(self.lib.ppm_ensemble_set_launch_mode(self.h, int(mode)))

    @property
    def launch_mode(self) -> int:
        return int(self.lib.ppm_ensemble_get_launch_mode(self.h))

    def set_wait_test(self, on: bool):
        """Tests of the failure path only: every bounded wait of the next
        one-launch step runs out (the step ends with PPM_ETIMEOUT)."""
        self._check(self.lib.ppm_ensemble_set_wait_test(self.h, 1 if on else 0))

    @property
    def launch_count(self) -> int:
        return int(self.lib.ppm_ensemble_launch_count(self.h))
