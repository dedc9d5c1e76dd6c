"""Domain decomposition of a single box over ranks, on CPU (gloo).

The multi-GPU plan for one large box splits it into z slabs; each pass along
x or y is local to a slab, each pass along z first exchanges 4 halo planes
with the neighbouring slabs (4 = the stencil reach, Sec. 4), and dt is a
max-reduction of the signal speed over ranks.  Here the ranks are CPU
processes running the FP64 oracle; the result after several double steps
must equal the unsplit run bit for bit, for a periodic box and for a
stratified box with reflecting walls, gravity and sources.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads

G = 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _make(kind):
    if kind == "periodic":
        return workloads.periodic_box(shape=(12, 10, 24))
    p = workloads.strat_box(shape=(10, 8, 24))
    p.tables.damp = 0.5 * np.ones_like(p.tables.rho0)
    return p


def _slab_problem(p, k0, nzl):
    import copy
    q = copy.copy(p)
    q.shape = (p.shape[0], p.shape[1], nzl)
    q.origin = (p.origin[0], p.origin[1], p.origin[2] + k0 * p.dx)
    return q


def _exchange(qloc, nzl, rank, world, bc_lo, bc_hi):
    """Fill the 4 halo planes on each side from the neighbours (or from the
    global boundary: wrapped planes when periodic, mirrored planes when
    reflecting; normal components are flipped by the pass itself)."""
    mine = ([a[G:2 * G].copy() for a in qloc], [a[nzl:nzl + G].copy() for a in qloc])
    allp = [None] * world
    dist.all_gather_object(allp, mine)
    below = rank - 1 if rank > 0 else (world - 1 if bc_lo == 0 else None)
    above = rank + 1 if rank < world - 1 else (0 if bc_hi == 0 else None)
    for v, a in enumerate(qloc):
        if below is not None:
            a[0:G] = allp[below][1][v]
        else:
            a[0:G] = a[G:2 * G][::-1]
        if above is not None:
            a[nzl + G:nzl + 2 * G] = allp[above][0][v]
        else:
            a[nzl + G:nzl + 2 * G] = a[nzl:nzl + G][::-1]


def _worker(rank, world, port, kind, steps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.Oracle.set_threads(1)
        p = _make(kind)
        nx, ny, nz = p.shape
        q = workloads.build(p)
        nzl = nz // world
        k0 = rank * nzl
        sub = _slab_problem(p, k0, nzl)
        o_slab = oracle.Oracle(sub)
        o_full = oracle.Oracle(p)
        qloc = [np.zeros((nzl + 2 * G, ny, nx)) for _ in range(9)]
        for v in range(9):
            qloc[v][G:G + nzl] = q[v][k0:k0 + nzl]
        inner = [a[G:G + nzl] for a in qloc]
        src = p.tables.heat is not None or p.tables.damp is not None
        bc_lo, bc_hi = p.bc[4], p.bc[5]
        for _ in range(steps):
            dt_local = o_slab.cfl_dt(inner, p.cfl)
            t = torch.tensor([dt_local], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MIN)            # = cfl dx / global max speed
            dt = float(t.item())
            o_slab.sweep(inner, 0, dt)
            o_slab.sweep(inner, 1, dt)
            _exchange(qloc, nzl, rank, world, bc_lo, bc_hi)
            o_full.sweep_z_slab(qloc, k0, nzl, dt, sources=src)
            _exchange(qloc, nzl, rank, world, bc_lo, bc_hi)
            o_full.sweep_z_slab(qloc, k0, nzl, dt, sources=False)
            o_slab.sweep(inner, 1, dt)
            o_slab.sweep(inner, 0, dt, sources=src)
        parts = [None] * world
        dist.all_gather_object(parts, [a.copy() for a in inner])
        if rank == 0:
            out["split"] = [np.concatenate([parts[r][v] for r in range(world)], axis=0) for v in range(9)]
            qf = [a.copy() for a in q]
            for _ in range(steps):
                o_full.double_step(qf, o_full.cfl_dt(qf, p.cfl))
            out["full"] = qf
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind,world", [("periodic", 2), ("strat", 3)])
def test_z_slab_decomposition_equals_unsplit_run(kind, world):
    oracle.build()
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, kind, 4, out), nprocs=world, start_method="spawn", join=True)
    split, full = out["split"], out["full"]
    for v in range(9):
        assert np.array_equal(split[v], full[v]), v
