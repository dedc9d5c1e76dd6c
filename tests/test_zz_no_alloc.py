"""ppm_totals_noalloc: conserved totals without any device allocation.

This entry point is for callers that cannot let a library call cudaMalloc
(their own allocator owns the device memory, or their step loop cannot take
the synchronisation an allocation may bring).  The test calls it through the
C ABI on a state held in caller-owned device buffers, twice in a row, and
checks both results against the totals of the existing ppm_diagnostics call
on the same state, within the tolerance the diagnostics tests use.  Kept in a
file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1810_13416_gb300 as ppm
import workloads

pytestmark = pytest.mark.gpu

_DP = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ppm.build()
    lib = ppm._load()
    lib.ppm_totals_noalloc.argtypes = [_DP * 9, C.c_int, C.c_int, C.c_int, C.c_double, _DP, C.c_void_p]
    lib.ppm_totals_noalloc.restype = C.c_int
    return lib


def _dptr(t):
    return C.cast(C.c_void_p(int(t.data_ptr())), _DP)


def test_noalloc_totals_match_diagnostics_twice(lib):
    p = workloads.sphere(shape=(40, 36, 44))
    q = workloads.build(p)
    nx, ny, nz = p.shape
    # existing entry point: a context holding the same state
    with ppm.Context.from_problem(p, precision=ppm.FP64_PLAIN) as ctx:
        ctx.set_state(q)
        ref, _, _ = ctx.diagnostics()
    # caller-owned device buffers; the library allocates nothing for this call
    dev = [torch.tensor(a, device="cuda") for a in q]
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    ptrs = (_DP * 9)(*[_dptr(t) for t in dev])
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for _ in range(2):
        out.fill_(-1.0)
        rc = lib.ppm_totals_noalloc(ptrs, nx, ny, nz, p.dx, _dptr(out), C.c_void_p(stream))
        assert rc == 0, lib.ppm_last_error(None).decode()
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    for r in results:
        np.testing.assert_allclose(r, ref, rtol=1e-12, atol=1e-14)
    assert np.array_equal(results[0], results[1])


def test_noalloc_rejects_too_many_planes(lib):
    dev = [torch.zeros(4, dtype=torch.float64, device="cuda") for _ in range(9)]
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    ptrs = (_DP * 9)(*[_dptr(t) for t in dev])
    rc = lib.ppm_totals_noalloc(ptrs, 1, 1, 8193, 1.0, _dptr(out), None)
    assert rc == -1
    assert "8192" in lib.ppm_last_error(None).decode()


def test_noalloc_last_scratch_row_and_sub_warp_planes(lib):
    """nz equal to the scratch limit (its last row is used) and planes of 6
    cells, smaller than a warp, so most lanes add zeros in the shuffle
    reduction; checked against numpy sums of the same arrays times dx^3."""
    nx, ny, nz, dx = 3, 2, 8192, 0.125
    g = np.random.default_rng(7)
    q = [g.uniform(0.5, 2.0, nx * ny * nz) for _ in range(9)]
    q[5] = g.uniform(0.0, 1.0, nx * ny * nz)
    dev = [torch.tensor(a, device="cuda") for a in q]
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    ptrs = (_DP * 9)(*[_dptr(t) for t in dev])
    for _ in range(2):
        out.fill_(-1.0)
        rc = lib.ppm_totals_noalloc(ptrs, nx, ny, nz, dx, _dptr(out), None)
        assert rc == 0, lib.ppm_last_error(None).decode()
        torch.cuda.synchronize()
        r = out.cpu().numpy()
        ref = np.array([q[0].sum(), q[1].sum(), q[2].sum(), q[3].sum(), q[4].sum(),
                        (q[0] * q[5]).sum(), q[5].sum()]) * dx ** 3
        np.testing.assert_allclose(r, ref, rtol=1e-12, atol=0.0)
