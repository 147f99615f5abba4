"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their timed
seconds (max) and solve counts (sum) into the whole-job rate, and every rank
> 0 times its own jittered frame of the same workload (weak scaling)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, solves = [2.0, 3.0][rank], [100, 140][rank]
    out[rank] = bench.job_rate(t, solves)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_job_rate():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        rate, tmax, solves = out[r]
        assert tmax == 3.0 and solves == 240.0
        assert abs(rate - 240.0 / 3.0) < 1e-12


def test_single_process_rate_and_rank_workloads():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(2.0, 50) == (25.0, 2.0, 50.0)
    s0, _ = bench.workload(0, n_mol=8)
    s1, _ = bench.workload(1, n_mol=8)
    s2, _ = bench.workload(2, n_mol=8)
    assert np.array_equal(s0.Z, s1.Z) and np.array_equal(s0.frag, s1.frag)
    assert not np.allclose(s0.xyz, s1.xyz) and not np.allclose(s1.xyz, s2.xyz)
    assert np.max(np.abs(s1.xyz - s0.xyz)) < 0.5            # a jitter, not a new geometry


def test_pass_rates_from_run_stats():
    sys.path.insert(0, ROOT)
    import bench
    st = {"n_monomer_solves": 128, "ms_monomer": 16.0, "n_dimer_scc": 511, "ms_dimer": 28.0,
          "n_trimer_scc": 0, "ms_trimer": 0.001}
    r = bench.pass_rates([st, st])
    assert set(r) == {"monomer", "dimer"}                      # no trimers ran
    assert r["monomer"]["solves"] == 256 and abs(r["monomer"]["per_s"] - 256 / 0.032) < 1e-6
    assert abs(r["dimer"]["per_s"] - 1022 / 0.056) < 1e-6
