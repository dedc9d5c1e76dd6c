"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/ppm.h declares, and
rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

import paper_1810_13416_gb300 as ppm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ppm.h")).read()
    return sorted(set(re.findall(r"\b(ppm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    ppm.build()
    return ppm._load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "ppm_create" in names and "ppm_step" in names
    for n in names:
        assert hasattr(lib, n), n


def _create(lib, **kw):
    args = dict(nx=8, ny=8, nz=8, gamma=1.4, bc=[0] * 6, kind=0, ntab=2, ds=1.0, dx=0.1,
                precision=1)
    args.update(kw)
    one = (C.c_double * 2)(1.0, 1.0)
    zero = (C.c_double * 2)(0.0, 0.0)
    dp = C.cast(one, C.POINTER(C.c_double))
    gr = ppm._Gravity(args["kind"], args["ntab"], 0.0, args["ds"], dp, dp,
                      C.cast(zero, C.POINTER(C.c_double)))
    opt = ppm._Options(0.0, 0.0, 0.0, args["dx"], args["precision"], None, None, None, 0,
                       args.get("confine_r", 0.0), args.get("nmom", 3), args.get("shock_k", 0.0))
    h = C.c_void_p()
    rc = lib.ppm_create(C.byref(h), args["nx"], args["ny"], args["nz"], args["gamma"],
                        (C.c_int * 6)(*args["bc"]), C.byref(gr), C.byref(opt))
    return rc, h


@pytest.mark.parametrize("kw,frag", [
    (dict(nx=3), "extent"),
    (dict(gamma=1.0), "gamma"),
    (dict(bc=[0, 1, 0, 0, 0, 0]), "pairs"),
    (dict(bc=[0, 0, 0, 0, 0, 7]), "boundary"),
    (dict(kind=5), "gravity"),
    (dict(ntab=1), "ntab"),
    (dict(ds=0.0), "ntab"),
    (dict(precision=3), "precision"),
    (dict(dx=-1.0), "dx"),
    (dict(confine_r=-1.0), "confine_r"),
    (dict(confine_r=0.5), "six faces"),
    (dict(nmom=5), "nmom"),
    (dict(shock_k=-0.1), "shock_k"),
    (dict(shock_k=0.1, nmom=9), "shock dissipation"),
])
def test_create_rejects_bad_arguments(lib, kw, frag):
    rc, h = _create(lib, **kw)
    assert rc == -1 and not h.value
    assert frag in lib.ppm_last_error(None).decode()


def test_null_context_calls_are_rejected(lib):
    assert lib.ppm_step(None, 1.0) == -1
    assert lib.ppm_sync(None) == -1
    assert lib.ppm_launch_count(None) == 0
    lib.ppm_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ppm._build_mod, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(ppm, "_lib", None)
    with pytest.raises(ImportError):
        ppm._load()


def test_ensemble_create_rejects_bad_arguments(lib):
    h = C.c_void_p()
    boxes = (ppm._Box * 1)()
    assert lib.ppm_ensemble_create(C.byref(h), 0, boxes, 1.4, 1, None, 0) == -1
    assert "nbox" in lib.ppm_ensemble_last_error(None).decode()
    assert lib.ppm_ensemble_create(C.byref(h), 1, boxes, 1.4, 7, None, 0) == -1
    assert lib.ppm_ensemble_step(None, 1.0) == -1
    assert lib.ppm_ensemble_launch_count(None) == 0
    lib.ppm_ensemble_destroy(None)
