"""Benchmark of the batched FMO-xTB SCC path on B300.

Workload (default): FMO2 energy of 128 anthracene molecules on a seeded
herringbone lattice (3072 atoms, 76 basis functions per fragment); pairs with a
closest-atom distance below 4.0 A get an SCC dimer (152 basis functions), the
others the electrostatic dimer approximation.  One step = one complete FMO2
run: coordination numbers, integrals, the monomer loop in the ESP, pair
selection, all SCC dimers, ES-DIM pairs and the FMO sums.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

Prints one JSON line (rank 0).  value = fragment-SCC solves per second over
all ranks (a solve = one n-mer SCC run to convergence: every monomer solve of
every outer iteration, every SCC dimer).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMO2/3 energy wall time & fragment-SCC/s vs plain FP64 GPU at |dE|<=1e-6 Eh"
UNIT = "fragment-SCC/s"
# peaks for the ALU-bound SCC kernel (148 SMs; clocks from the profiling recipe)
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12      # FP32 FMA lanes x 2 flops x max SM clock
FP64_PEAK_TFLOPS = 1.25                                 # nominal B300 FP64 rate
# DRAM bytes (read + write) of the dimer-pass SCC launch of this workload, from
# one ncu capture of the current kernel; None whenever the kernel has changed
# since that capture
DIMER_SCC_DRAM_BYTES = 531186944 + 527815168


def workload(rank: int, n_mol: int = 128):
    from paper_2606_28022_b300.inputs import geometry as G
    system, info = G.anthracene_cluster(128, seed=2)
    if n_mol < 128:                   # a smaller case (profiling): the first n_mol molecules
        system = system.subsystem(range(n_mol))
    if rank > 0:                      # weak scaling: every rank its own jittered frame
        system = G.jittered(system, 0.02, 5000 + rank)
    return system, info


def job_rate(t_total: float, solves: float, dev=None):
    """Whole-job throughput over all ranks: the solves of every rank divided by
    the slowest rank's timed seconds.  Returns (rate, t_max, solves_all)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(solves) / t_total, t_total, float(solves)
    t = torch.tensor([t_total, float(solves)], dtype=torch.float64, device=dev)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t[1]) / float(tmax[0]), float(tmax[0]), float(t[1])


def pass_rates(stats: list) -> dict:
    """Fragment-SCC solves per second of each pass (size class) over the timed
    steps: monomer solves over the monomer stage (setup excluded), SCC dimers
    over the dimer stage, SCC trimers over the trimer stage."""
    out = {}
    for name, n_key, ms_key in (("monomer", "n_monomer_solves", "ms_monomer"),
                                ("dimer", "n_dimer_scc", "ms_dimer"),
                                ("trimer", "n_trimer_scc", "ms_trimer")):
        n = sum(s[n_key] for s in stats)
        ms = sum(s[ms_key] for s in stats)
        if n > 0 and ms > 0:
            out[name] = {"solves": int(n), "stage_ms": float(ms), "per_s": float(n / (ms / 1e3))}
    return out


def clocks_sampler(dev_index: int):
    """Sample nvidia-smi clocks / throttle reasons in the background."""
    cmd = ["nvidia-smi", "-i", str(dev_index),
           "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None, []
    rows = []

    def reader():
        for line in proc.stdout:
            rows.append([x.strip() for x in line.split(",")])
    th = threading.Thread(target=reader, daemon=True)
    th.start()
    return proc, rows


def summarize_clocks(rows):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        try:
            sm.append(float(r[0]))
            mx.append(float(r[1]))
            for nm, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        except (ValueError, IndexError):
            continue
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def cpu_oracle_sample(system, params, n_mono=24, n_dim=10):
    """The FP64 oracle as it stands on a bounded sample of the workload's
    n-mers: monomer and SCC-dimer solves (in zero ESP; the cost of a solve does
    not depend on the ESP values).  Returns (solves/s, seconds, solves)."""
    from oracle import xtb
    from paper_2606_28022_b300.inputs.params import ANGSTROM
    nf = system.n_frag
    xyz = system.xyz.reshape(nf, -1, 3)
    pairs = []
    for I in range(nf):
        d = np.sqrt(((xyz[I][:, None, None, :] - xyz[None, :, :, :]) ** 2).sum(-1)).min(axis=(0, 2))
        for J in range(I + 1, nf):
            if d[J] < 4.0 * ANGSTROM:
                pairs.append((I, J))
        if len(pairs) >= n_dim:
            break
    cn = xtb.coordination_numbers(system.Z, system.xyz, params)
    t0 = time.perf_counter()
    solves = 0
    for I in range(n_mono):
        idx = np.nonzero(system.frag == I)[0]
        xtb.scc(system.Z[idx], system.xyz[idx], params, cn[idx])
        solves += 1
    for (I, J) in pairs[:n_dim]:
        idx = np.concatenate([np.nonzero(system.frag == I)[0], np.nonzero(system.frag == J)[0]])
        xtb.scc(system.Z[idx], system.xyz[idx], params, cn[idx])
        solves += 1
    dt = time.perf_counter() - t0
    return solves / dt, dt, solves


def cores_used():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    from paper_2606_28022_b300.inputs.params import synthetic_gfn1_table
    params = synthetic_gfn1_table()
    system, _ = workload(0)
    for _ in range(args.warmup):
        cpu_oracle_sample(system, params, n_mono=2, n_dim=1)
    rates, secs = [], []
    for _ in range(args.steps):
        r, dt, n = cpu_oracle_sample(system, params, n_mono=6, n_dim=3)
        rates.append(r)
        secs.append(dt)
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "anthracene128-FMO2 (C14H10 x 128, herringbone, 4.0 A SCC-dimer cut)",
                       "sample": "6 monomer + 3 SCC-dimer solves per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                             "sample": "6 monomer + 3 SCC-dimer oracle solves per step, zero ESP"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-mol", type=int, default=128,
                    help="anthracenes in the workload (128 = the benchmark; fewer for profiling)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2606_28022_b300 import build, fmo
    from paper_2606_28022_b300.inputs.params import synthetic_gfn1_table

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    params = synthetic_gfn1_table()
    system, geo = workload(rank, args.n_mol)
    g = fmo.FMO(params, dev.index)
    g.set_system(system)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    opts = fmo.options(precision=args.precision)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (126 MB)

    def step_once():
        return g.run(opts, stream=sptr)

    for _ in range(max(args.warmup, 3) if args.warmup > 0 else 0):
        step_once()
    torch.cuda.synchronize(dev)

    proc, rows = clocks_sampler(dev.index) if rank == 0 else (None, [])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()                                  # L2 flush between timed steps
        ev[k][0].record(stream)
        step_once()
        ev[k][1].record(stream)
        stats.append(g.stats())
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    if proc is not None:
        proc.terminate()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1e3
    solves = sum(s["n_monomer_solves"] + s["n_dimer_scc"] + s["n_trimer_scc"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    value, t_total_max, solves_all = job_rate(t_total, solves, dev)

    e1, e2, _ = g.energies()
    s0 = stats[-1]

    # e2e through the public API with host buffers: coordinates in, energies out
    e2e = None
    xyz_host = np.ascontiguousarray(system.xyz, dtype=np.float64)
    t0 = time.perf_counter()
    e2e_steps = max(1, min(3, args.steps))
    h2d = d2h = 0
    for _ in range(e2e_steps):
        g.set_coordinates(xyz_host)
        g.run(opts, stream=sptr)
        g.energies()
        m = g.monomers()
        d = g.dimers()
        st = g.stats()
        h2d += st["h2d_bytes"]
        d2h += st["d2h_bytes"]
    torch.cuda.synchronize(dev)
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": (s0["n_monomer_solves"] + s0["n_dimer_scc"]) / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(h2d / e2e_steps),
           "d2h_bytes_per_step": int(d2h / e2e_steps) + 8 * (len(m.energy) + len(m.shell_dq)) + 34 * len(d.dE)}

    # plain FP64 GPU form of the same workload, for the metric's comparison
    fp64 = None
    if rank == 0 and args.precision == "mixed" and not args.no_fp64_compare:
        o64 = fmo.options(precision="fp64")
        g.run(o64, stream=sptr)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        g.run(o64, stream=sptr)
        b.record(stream)
        torch.cuda.synchronize(dev)
        f1, f2, _ = g.energies()
        s64 = g.stats()
        fp64 = {"ms_per_step": a.elapsed_time(b), "e_fmo2": f2,
                "fragment_scc_per_s": (s64["n_monomer_solves"] + s64["n_dimer_scc"]) / (a.elapsed_time(b) / 1e3),
                "abs_dE_total_mixed_vs_fp64": abs(e2 - f2)}

    # roofline of the dominant kernel: the SCC kernel of the dimer pass
    ms_scc = [np.mean([s["ms_scc"][p] for s in stats]) for p in range(3)]
    f32 = np.mean([s["flops_fp32"][1] for s in stats])
    f64 = np.mean([s["flops_fp64"][1] for s in stats])
    t_meas = ms_scc[1] / 1e3
    t_min = f32 / (FP32_PEAK_TFLOPS * 1e12) + f64 / (FP64_PEAK_TFLOPS * 1e12)
    achieved = (f32 + f64) / t_meas / 1e12 if t_meas > 0 else 0.0
    peak = (f32 + f64) / t_min / 1e12 if t_min > 0 else 0.0
    roofline = {"bound": "alu", "kernel": "scc_kernel (dimer pass)", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak if peak else 0.0,
                "traffic": DIMER_SCC_DRAM_BYTES if args.n_mol == 128 else None,
                "peak_basis": f"FP32 {FP32_PEAK_TFLOPS:.1f} TF/s (148 SM x 128 lanes x 2 x 2.032 GHz) and "
                              f"FP64 {FP64_PEAK_TFLOPS} TF/s nominal, weighted by the kernel's FP32/FP64 flops",
                "flops_fp32": f32, "flops_fp64": f64, "kernel_ms": ms_scc[1],
                "kernel_share_of_step": ms_scc[1] / np.mean(step_ms)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, dt, n = cpu_oracle_sample(system, params)
        cpu = {"value": rate, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
               "sample": f"{n} oracle n-mer SCC solves of this workload (24 monomers + 10 SCC dimers, zero ESP), "
                         f"{dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": f"anthracene{system.n_frag}-FMO2: {system.n_frag} C14H10 ({system.n_atoms} atoms), seeded herringbone "
                                       "a=8.56 b=6.04 c=11.16 A beta=124.7, 0.05 A jitter; SCC dimer iff "
                                       "closest atom < 4.0 A, else ES-DIM",
                           "precision": args.precision, "n_frag": system.n_frag,
                           "n_dimer_scc": s0["n_dimer_scc"], "n_dimer_esdim": s0["n_dimer_esdim"],
                           "outer_iterations": s0["outer_iterations"],
                           "n_monomer_solves": s0["n_monomer_solves"],
                           "l2": "256 MB buffer written between timed steps (L2 flush)",
                           "parallelism": f"replicas x{world} (independent frames)", "geometry": geo},
                "e_fmo1": e1, "e_fmo2": e2, "fp64_form": fp64,
                "stage_ms": {k: s0[k] for k in ("ms_setup", "ms_monomer", "ms_select", "ms_dimer", "ms_reduce")},
                "per_pass": pass_rates(stats),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": summarize_clocks(rows)}
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
