"""Sharded fmo_run over two processes with a gloo exchange, both on GPU 0
(their kernels never wait on each other: the ranks meet only in the host-side
exchange between launches).  Every rank must end with the unsharded results,
bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _systems():
    from paper_2606_28022_b300.inputs import geometry as G
    water12 = G.water_cluster(64, 1).subsystem(range(12))
    pc, _ = G.pentacene_cluster(660, 4)
    pent4 = pc.subsystem([0, 2, 93, 1])
    return [("water12-fmo2-mixed", water12, dict(precision="mixed")),
            ("water12-fmo2-fp64", water12, dict(precision="fp64")),
            ("pentacene4-fmo3-mixed", pent4, dict(level=3, precision="mixed"))]


def _results(g):
    d = g.dimers()
    t = g.trimers()
    m = g.monomers()
    return (g.energies(), m.energy.copy(), m.shell_dq.copy(), d.dE.copy(), t.dE3.copy(), t.corr.copy())


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_28022_b300 import fmo, shard
    from paper_2606_28022_b300.inputs.params import synthetic_gfn1_table
    g = fmo.FMO(synthetic_gfn1_table(), 0)
    g.set_exchange(shard.allreduce_exchange())
    res = {}
    for name, s, kw in _systems():
        g.set_system(s)
        g.run(fmo.options(shard_rank=rank, shard_world=world, **kw))
        res[name] = _results(g)
        if rank == 0:                                   # the unsharded run, same process
            g.run(fmo.options(**kw))
            res[name + "/ref"] = _results(g)
    g.close()
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_one_gpu_equal_the_unsharded_run():
    out = mp.get_context("spawn").Manager().dict()   # no fork of a process that holds a CUDA context
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    ref = out[0]
    for name, _, _ in _systems():
        want = ref[name + "/ref"]
        for r in range(2):
            got = out[r][name]
            # FMO totals (NaN above the run's level) and every array, bit for bit
            assert np.array_equal(np.array(got[0]), np.array(want[0]), equal_nan=True), (name, r)
            for a, b in zip(got[1:], want[1:]):
                assert np.array_equal(a, b, equal_nan=True), (name, r)


def test_sharded_run_needs_an_exchange(params):
    from paper_2606_28022_b300 import build, fmo
    from paper_2606_28022_b300.inputs import geometry as G
    build.build()
    g = fmo.FMO(params, 0)
    g.set_system(G.water_cluster(64, 1).subsystem(range(3)))
    with pytest.raises(fmo.FMOError) as e:
        g.run(fmo.options(shard_rank=0, shard_world=2))
    assert e.value.status == 7                                # FMO_ERR_STATE
    with pytest.raises(fmo.FMOError) as e:
        g.run(fmo.options(shard_rank=2, shard_world=2))
    assert e.value.status == 1                                # FMO_ERR_ARG

    def failing(buf):
        raise RuntimeError("peer gone")
    g.set_exchange(failing)
    with pytest.raises(fmo.FMOError) as e:
        g.run(fmo.options(shard_rank=0, shard_world=2))
    assert e.value.status == 9                                # FMO_ERR_EXCHANGE
    g.set_exchange(None)
    g.run(fmo.options())                                      # unsharded still fine
    g.close()
