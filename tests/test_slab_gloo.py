"""The x-slab partition of the IB-LBM step (the multi-GPU design) on CPU
ranks: two and four gloo ranks on 127.0.0.1, each holding an x-slab of the
oracle's state, exchanging a two-plane (rho, u*) ghost layer, the crossing
populations and one all-reduce of the owned markers' interpolations per
step.  After 20 steps of the small wing pair the gathered populations and
every body's C_L / C_T / C_D history equal the undivided oracle's bitwise."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W

STEPS = 20


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    return W.clap_fling_3d(nx=48, ny=40, nz=40, chord=6.0, Re=5.0, J=0.1, period=1200.0, precision="fp64",
                           faces="periodic")


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    from oracle.slab import SlabSimulation
    cfg = _case()
    sim = SlabSimulation(cfg["lattice"], cfg["grid"], cfg["tau"], dist, rank, world)
    sim.init_fluid(np.asarray(cfg["u0"]))
    for b in cfg["bodies"]:
        sim.add_body(b)
    r = cfg["reference"]
    sim.set_reference(r["U_ref"], r["L"], r["rho_ref"])
    sim.step(STEPS)
    f = sim.gather_populations()
    out[rank] = (f, [np.array(h) for h in sim.history])
    dist.destroy_process_group()


def _undivided(_, out):
    """The undivided oracle, in a process of its own with the ranks' BLAS
    thread count (the dense LU's rounding depends on it)."""
    from tests.parity import oracle_from_workload
    sim = oracle_from_workload(_case())
    sim.step(STEPS)
    out["ref"] = (sim.f, [np.array(h) for h in sim.history])


@pytest.mark.parametrize("world", [2, 4])   # 4: slabs of 12, the wing (x 10.5..15.5) spans two owners
def test_slab_partition_equals_the_undivided_oracle(world):
    port = _free_port()
    # one BLAS thread per rank: the spawned ranks inherit this environment
    # before they import numpy
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    try:
        with mp.Manager() as m:
            out = m.dict()
            mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
            mp.spawn(_undivided, args=(out,), nprocs=1, join=True)
            res = dict(out)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    f_ref, hist_ref = res["ref"]
    f0, hist0 = res[0]
    assert np.array_equal(f0, f_ref)
    for r in range(world):
        for h, href in zip(res[r][1], hist_ref):
            assert np.array_equal(h, href)
