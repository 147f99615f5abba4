"""Host side of sharded FMO runs: one process per GPU.

fmo_run (options shard_rank / shard_world) splits every pass with the
library's LPT partition (cost n^3 of each n-mer's basis) and, through an
exchange callback, sums over the ranks the output charges and energies of
each monomer-loop step (Sec. 2.3: one SCC step of every monomer, then one
Broyden step on all monomer charges together, taken identically on every
rank) and the per-n-mer results of the dimer and trimer passes (Eqs. 12-19).
Each summed entry is non-zero on its owner only, so every rank ends with the
unsharded results, bit for bit, and forms the FMO totals in the same order.

allreduce_exchange builds that callback on torch.distributed.  The buffer is
a host array: use a gloo process group (with an NCCL default group, pass
torch.distributed.new_group(backend="gloo")).
"""
import numpy as np


def allreduce_exchange(group=None):
    """Exchange callback for FMO.set_exchange: all_reduce(SUM) of the buffer
    over `group` (default: the world group)."""
    import torch
    import torch.distributed as dist

    def fn(buf: np.ndarray) -> None:
        t = torch.from_numpy(buf)          # shares memory with the library's buffer
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return fn


def sharded_options(opts, rank: int, world: int):
    """Copy of an fmo_options structure with the shard fields set."""
    import ctypes
    o = type(opts)()
    ctypes.pointer(o)[0] = opts
    o.shard_rank, o.shard_world = int(rank), int(world)
    return o
