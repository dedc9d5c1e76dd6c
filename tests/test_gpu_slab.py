"""GPU side of the z-slab decomposition (Sec. 4/5: a grid brick is updated
from its neighbours' boundary planes): one box split into two slab contexts
on one GPU.  Before each z pass each slab's boundary planes are copied into
the other's halo buffer (ppm_slab_pack / ppm_slab_halo, device-to-device,
the exchange step a multi-GPU run would do with send/receive); the x and y
passes need no exchange.  After 3 double steps the gathered slabs equal the
unsplit context bit for bit, FP64 and FP32, for a stratified layer with walls,
gravity and heating and for a periodic box (wrapped exchange)."""
import numpy as np
import pytest
import torch

import paper_1810_13416_gb300 as ppm
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ppm.build()


ORDER = ((0, 0), (1, 0), (2, 1), (2, 0), (1, 0), (0, 1))   # X Y Z[src] Z Y X[src]


def _split_run(p, q, cut, precision, dts, periodic):
    stream = torch.cuda.Stream()
    nz = p.shape[2]
    halo_a = 3 if periodic else 2
    halo_b = 3 if periodic else 1
    a = ppm.Context.slab(p, 0, cut, halo_a, precision=precision, stream=stream)
    b = ppm.Context.slab(p, cut, nz - cut, halo_b, precision=precision, stream=stream)
    a.set_state([x[:cut] for x in q])
    b.set_state([x[cut:] for x in q])

    def exchange():
        b.slab_pack(0, a.slab_halo(1)[0])      # B's lowest planes above A
        a.slab_pack(1, b.slab_halo(0)[0])      # A's highest planes below B
        if periodic:
            b.slab_pack(1, a.slab_halo(0)[0])  # wrapped: B's top below A
            a.slab_pack(0, b.slab_halo(1)[0])  # A's bottom above B

    for dt in dts:
        for axis, src in ORDER:
            if axis == 2:
                exchange()
            a.sweep(axis, dt, src)
            b.sweep(axis, dt, src)
    qa, qb = a.get_state(), b.get_state()
    a.close()
    b.close()
    return [np.concatenate([x, y], axis=0) for x, y in zip(qa, qb)]


@pytest.mark.parametrize("precision", [ppm.FP64_PLAIN, ppm.FP32_DEVIATION])
@pytest.mark.parametrize("which", ["strat_walls", "periodic"])
def test_two_slabs_equal_the_unsplit_box_bitwise(precision, which):
    if which == "strat_walls":
        p = workloads.strat_box(shape=(32, 24, 40))
        cut, periodic = 17, False
    else:
        p = workloads.periodic_box(shape=(24, 20, 36))
        cut, periodic = 20, True
    q = workloads.build(p)
    with ppm.Context.from_problem(p, precision=precision) as full:
        full.set_state(q)
        dts = []
        for _ in range(3):
            dt = full.cfl_dt(0.6)
            dts.append(dt)
            full.step(dt)
        ref = full.get_state()
    got = _split_run(p, q, cut, precision, dts, periodic)
    for v in range(9):
        assert np.array_equal(got[v], ref[v]), (v, np.abs(got[v] - ref[v]).max())


def test_slab_options_are_checked():
    p = workloads.strat_box(shape=(16, 16, 16))
    with pytest.raises(ppm.PpmError):   # the face without halo planes is periodic
        ppm.Context.slab(workloads.periodic_box(shape=(16, 16, 16)), 0, 8, 2)
    with ppm.Context.slab(p, 0, 8, 2) as c:
        with pytest.raises(ppm.PpmError):
            c.slab_halo(0)                 # the low face has no halo planes
        ptr, n = c.slab_halo(1)
        assert ptr != 0 and n == 9 * 4 * 16 * 16 * 4
        assert not c.tile_available
