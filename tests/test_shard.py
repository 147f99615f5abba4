"""Sharding over processes on the CPU: the library's LPT partition against
its definition and Graham's bound, and the sharded FMO2 protocol of fmo_run
(owned monomer steps + an exact sum of their outputs per step, a replicated
Broyden step, owned dimers + an exact sum, totals on every rank) run by two
gloo ranks with the oracle as the engine: bit-identical to one rank and to
the oracle's own FMO2."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fmo_mod():
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo


def _lpt_reference(cost, world):
    # the rule written out: units by decreasing cost (ties: lower index) onto
    # the least loaded rank (ties: lower rank)
    order = sorted(range(len(cost)), key=lambda i: (-cost[i], i))
    load = [0.0] * world
    owner = [0] * len(cost)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += cost[i]
    return owner


def test_lpt_partition_follows_its_rule(fmo_mod):
    rng = np.random.default_rng(5)
    for n, world in ((0, 3), (1, 4), (7, 2), (50, 3), (400, 8)):
        cost = np.round(rng.uniform(1, 100, n)) ** 3        # ties occur
        own = fmo_mod.lpt_partition(cost, world)
        assert own.tolist() == _lpt_reference(cost.tolist(), world)
        assert ((own >= 0) & (own < world)).all()


def test_lpt_partition_within_graham_bound(fmo_mod):
    rng = np.random.default_rng(11)
    for trial in range(20):
        n, world = int(rng.integers(3, 9)), int(rng.integers(2, 4))
        cost = rng.uniform(0.5, 10.0, n)
        own = fmo_mod.lpt_partition(cost, world)
        span = max(cost[own == r].sum() for r in range(world))
        best = min(max(sum(cost[i] for i in range(n) if a[i] == r) for r in range(world))
                   for a in itertools.product(range(world), repeat=n))
        assert span <= (4.0 / 3.0 - 1.0 / (3 * world)) * best + 1e-12


def test_lpt_partition_rejects_bad_input(fmo_mod):
    lib = fmo_mod.load_library()
    own = np.zeros(2, dtype=np.int32)
    bad = [np.array([1.0, -1.0]), np.array([1.0, np.nan])]
    for c in bad:
        assert lib.fmo_lpt_partition(fmo_mod._dp(c), 2, 2, fmo_mod._ip(own)) == 1
    c = np.ones(2)
    assert lib.fmo_lpt_partition(fmo_mod._dp(c), 2, 0, fmo_mod._ip(own)) == 1


# ---------------------------------------------------------------------------
# the sharded protocol with the oracle as the engine

def _sharded_fmo2(system, params, rank, world, exchange, max_outer=200):
    from oracle import fmo as ofmo
    from oracle import xtb
    from paper_2606_28022_b300 import fmo
    opts = ofmo.FMOOptions()
    fr = ofmo._Frags(system, params)
    nf = system.n_frag
    nao = [xtb.make_basis(system.Z[fr.atoms[f]], params).n_ao for f in range(nf)]
    own_m = fmo.lpt_partition([float(a) ** 3 for a in nao], world)
    probs = [fr.problem((I,)) for I in range(nf)]
    bounds = np.concatenate([[0], np.cumsum(fr.n_sh)])
    nsh = int(bounds[-1])
    split = lambda x: [x[bounds[I]:bounds[I + 1]] for I in range(nf)]
    x = np.zeros(nsh)
    mixer = xtb.Broyden()
    e_prev = None
    for outer in range(1, max_outer + 1):
        parts = split(x)
        buf = np.zeros(nsh + nf)
        for I in range(nf):
            if own_m[I] != rank:
                continue
            o = probs[I].step(parts[I], esp=fr.esp((I,), parts))
            buf[bounds[I]:bounds[I + 1]] = o["dq_out"]
            buf[nsh + I] = o["e_el"] + probs[I].e_rep
        exchange(buf)                                      # every rank: all outputs
        x_out, e_mono = buf[:nsh].copy(), buf[nsh:].copy()
        diff = float(np.max(np.abs(x_out - x)))
        e1 = float(np.sum(e_mono))
        if e_prev is not None and diff < opts.outer_tol and abs(e1 - e_prev) < opts.e_tol:
            break
        e_prev = e1
        x = mixer.step(x, x_out)
    dq_mono = [p.copy() for p in split(x_out)]
    pairs = [(I, J) for I in range(nf) for J in range(I + 1, nf)]
    scc = [fr.closest(I, J) < opts.dimer_cut for I, J in pairs]
    k_scc = [k for k in range(len(pairs)) if scc[k]]
    own_d = fmo.lpt_partition([float(nao[pairs[k][0]] + nao[pairs[k][1]]) ** 3 for k in k_scc], world)
    buf = np.zeros(len(pairs))
    for k, r in zip(k_scc, own_d):
        if r != rank:
            continue
        I, J = pairs[k]
        mask = fr.shell_mask((I, J))
        res = fr.solve((I, J), fr.esp_full((I, J), dq_mono)[mask],
                       np.concatenate([dq_mono[I], dq_mono[J]])[mask], opts)
        dev = ofmo._embedding_correction(fr, (I, J), res.dq, dq_mono)
        buf[k] = res.energy - e_mono[I] - e_mono[J] + dev
    exchange(buf)
    dE = buf
    for k, (I, J) in enumerate(pairs):
        if not scc[k]:
            dE[k] = float(dq_mono[I] @ fr.gamma(I, J) @ dq_mono[J])    # ES-DIM, every rank
    e1 = float(np.sum(e_mono))
    return e1, e1 + float(np.sum(dE)), dE, np.array(own_m), np.array(own_d)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_28022_b300 import shard
    from paper_2606_28022_b300.inputs.geometry import water_cluster
    from paper_2606_28022_b300.inputs.params import synthetic_gfn1_table
    s = water_cluster(64, 1).subsystem(range(6))
    out[rank] = _sharded_fmo2(s, synthetic_gfn1_table(), rank, world, shard.allreduce_exchange())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_one_rank_and_the_oracle(fmo_mod, params, water64):
    from oracle import fmo as ofmo
    s = water64.subsystem(range(6))
    one = _sharded_fmo2(s, params, 0, 1, lambda buf: None)
    ref = ofmo.fmo(s, params, ofmo.FMOOptions())
    assert one[1] == ref.e_fmo2 and one[0] == ref.e_fmo1
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        e1, e2, dE, own_m, own_d = out[r]
        assert e1 == one[0] and e2 == one[1]                 # bit for bit
        assert np.array_equal(dE, one[2])
        assert set(own_m.tolist()) == {0, 1}                 # both ranks did monomer work
        assert set(own_d.tolist()) == {0, 1} or len(own_d) < 2
