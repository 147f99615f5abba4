"""Benchmark of the batched FMO-xTB SCC path on B300.

Workload (default, --workload pentacene660): FMO3 energy of 660 pentacene
molecules (23,760 atoms, 116 basis functions per fragment) cut from a seeded
triclinic herringbone crystal with 0.05 A jitter; pairs with a closest-atom
distance below 4.0 A get an SCC dimer (232 basis functions), the others the
electrostatic dimer approximation, and every triangle of three such pairs an
SCC trimer (348 basis functions).  One step = one complete fmo_run:
coordination numbers, integrals, the monomer loop in the ESP, n-mer
selection, all SCC dimers and trimers, ES-DIM pairs and the FMO sums.
--workload anthracene128: FMO2 of the 128-anthracene aggregate.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload W] [--precision mixed|fp64]
    python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

Prints one JSON line (rank 0).  value = fragment-SCC solves per second over
all ranks (a solve = one n-mer SCC run to convergence: every monomer of the
monomer loop, every SCC dimer and trimer).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
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
WORKLOADS = {
    "water64": dict(level=2, opts=dict(all_dimers_scc=1),
                    desc="water64-FMO2: 64 rigid waters (O-H 0.957 A, 104.5 deg), seeded centres uniform in a "
                         "1.0 g/cm3 sphere with O-O >= 2.6 A, random orientations; all 2016 dimers with full SCC"),
    "pentacene660": dict(level=3, desc="pentacene660-FMO3: 660 C22H14 (23,760 atoms), seeded triclinic herringbone "
                                       "a=6.27 b=7.78 c=14.53 A (76.5/87.7/84.7 deg), 0.05 A jitter; SCC dimer iff "
                                       "closest atom < 4.0 A, else ES-DIM; SCC trimer iff all three pairs < 4.0 A"),
    "anthracene128": dict(level=2, desc="anthracene128-FMO2: 128 C14H10 (3072 atoms), seeded herringbone a=8.56 "
                                        "b=6.04 c=11.16 A beta=124.7, 0.05 A jitter; SCC dimer iff closest atom "
                                        "< 4.0 A, else ES-DIM"),
}
# profiles/traffic.json: DRAM bytes per launch of the dominant SCC launch from
# an ncu capture, with the hash of the kernel sources it was taken on; used
# only while those sources are unchanged
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = ["paper_2606_28022_b300/csrc/kernels.cu", "paper_2606_28022_b300/csrc/fmo_device.cuh",
                  "paper_2606_28022_b300/csrc/tridiag.cuh"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, pass_name: str):
    """(bytes per launch, note) from profiles/traffic.json if it was taken on
    the current kernel sources, else (None, reason)."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None, "no capture"
    e = d.get(workload, {}).get(pass_name)
    if not e:
        return None, "no capture of this launch"
    if e.get("source_sha16") != kernel_source_hash():
        return None, "kernel changed since the capture"
    return float(e["dram_bytes_per_launch"]), e.get("note", "")


def workload(rank: int, name: str = "pentacene660", n_mol: int | None = None):
    """The seeded system of a workload; rank > 0: its own jittered frame (weak
    scaling); n_mol: the first n_mol molecules (a smaller case)."""
    from paper_2606_28022_b300.inputs import geometry as G
    if name == "pentacene660":
        system, info = G.pentacene_cluster(660, seed=4)
    elif name == "water64":
        system, info = G.water_cluster(64, 1), {}
    else:
        system, info = G.anthracene_cluster(128, seed=2)
    if n_mol is not None and n_mol < system.n_frag:
        system = system.subsystem(range(n_mol))
    if rank > 0:
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


def nmer_lists(system, level: int, cut_bohr: float):
    """SCC dimers (closest-atom distance < cut) and trimers (all three pairs
    < cut) of a system, by the same rule as the library, in NumPy (to draw the
    CPU baseline's sample of n-mers when no GPU run supplies the lists)."""
    nf = system.n_frag
    atoms = [np.nonzero(system.frag == f)[0] for f in range(nf)]
    cen = np.array([system.xyz[a].mean(0) for a in atoms])
    rad = np.array([np.linalg.norm(system.xyz[a] - cen[f], axis=1).max() for f, a in enumerate(atoms)])
    near = {f: set() for f in range(nf)}
    dimers = []
    for I in range(nf):
        d = np.linalg.norm(cen[I + 1:] - cen[I], axis=1) - rad[I + 1:] - rad[I]
        for J in (np.nonzero(d < cut_bohr)[0] + I + 1):
            r = np.sqrt(((system.xyz[atoms[I]][:, None, :] - system.xyz[atoms[J]][None, :, :]) ** 2).sum(-1)).min()
            if r < cut_bohr:
                dimers.append((I, int(J)))
                near[I].add(int(J))
    trimers = []
    if level >= 3:
        for I, J in dimers:
            for K in sorted(near[I] & near[J]):
                if K > J:
                    trimers.append((I, J, K))
    return dimers, trimers


def _oracle_solve(job):
    """One oracle n-mer SCC solve (zero ESP: the cost of a solve does not
    depend on the ESP values); returns seconds."""
    from oracle import xtb
    Z, xyz = job
    t0 = time.perf_counter()
    cn = xtb.coordination_numbers(Z, xyz, _oracle_solve.params)
    xtb.scc(Z, xyz, _oracle_solve.params, cn)
    return time.perf_counter() - t0


def _pool_init():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    from paper_2606_28022_b300.inputs.params import synthetic_gfn1_table
    _oracle_solve.params = synthetic_gfn1_table()


def cpu_workers() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def cpu_oracle_sample(system, n_mono: int, dimers, trimers, n_solves: int, seed: int = 7, workers: int | None = None):
    """The FP64 oracle as it stands, timed on the host cores (a spawn pool of
    one-BLAS-thread workers) over a seeded sample of the workload's n-mer
    solves in the workload's proportions (monomer-loop solves, SCC dimers,
    SCC trimers).  Returns (solves/s, seconds, sample counts, workers)."""
    workers = cpu_workers() if workers is None else workers
    rng = np.random.default_rng(seed)
    tot = n_mono + len(dimers) + len(trimers)
    k_t = int(round(n_solves * len(trimers) / tot))
    k_d = int(round(n_solves * len(dimers) / tot))
    k_m = max(1, n_solves - k_t - k_d)
    jobs = []
    for I in rng.choice(system.n_frag, size=min(k_m, system.n_frag), replace=False):
        idx = np.nonzero(system.frag == I)[0]
        jobs.append((system.Z[idx], system.xyz[idx]))
    for lst, k in ((dimers, k_d), (trimers, k_t)):
        for q in rng.choice(len(lst), size=min(k, len(lst)), replace=False) if len(lst) else []:
            idx = np.concatenate([np.nonzero(system.frag == f)[0] for f in lst[q]])
            jobs.append((system.Z[idx], system.xyz[idx]))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_pool_init) as pool:
        pool.map(_oracle_solve, jobs[:workers], chunksize=1)       # workers started and warm
        t0 = time.perf_counter()
        pool.map(_oracle_solve, jobs, chunksize=1)
        dt = time.perf_counter() - t0
    counts = {"monomers": min(k_m, system.n_frag), "dimers": min(k_d, len(dimers)), "trimers": min(k_t, len(trimers))}
    return len(jobs) / dt, dt, counts, workers


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, timed on the host cores,
    each step a bounded seeded sample of the workload's n-mer solves."""
    if rank != 0:
        return
    from paper_2606_28022_b300.inputs.params import ANGSTROM
    wl = WORKLOADS[args.workload]
    system, _ = workload(0, args.workload, args.n_mol)
    cut = float("inf") if wl.get("opts", {}).get("all_dimers_scc") else 4.0 * ANGSTROM
    dimers, trimers = nmer_lists(system, wl["level"], cut)
    workers = cpu_workers()
    per_step = max(8, 2 * workers)
    for k in range(args.warmup):
        cpu_oracle_sample(system, system.n_frag, dimers, trimers, max(2, workers // 2), seed=100 + k, workers=workers)
    rates, secs = [], []
    counts = None
    for k in range(args.steps):
        r, dt, counts, _ = cpu_oracle_sample(system, system.n_frag, dimers, trimers, per_step, seed=k, workers=workers)
        rates.append(r)
        secs.append(dt)
    value = float(np.mean(rates))
    sample = (f"{per_step} oracle n-mer SCC solves per step ({counts}), in the workload's proportions of monomer, "
              f"SCC-dimer and SCC-trimer solves, zero ESP, {workers} worker processes")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "of measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "of fallback"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="pentacene660", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-repeats", type=int, default=1,
                    help="timed runs of the plain FP64 GPU form (median); 0 = not run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gradient", action="store_true")
    ap.add_argument("--n-mol", type=int, default=None, help="the first n molecules only (a smaller case)")
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
    from paper_2606_28022_b300.inputs.params import ANGSTROM, synthetic_gfn1_table

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    wl = WORKLOADS[args.workload]
    params = synthetic_gfn1_table()
    system, geo = workload(rank, args.workload, args.n_mol)
    g = fmo.FMO(params, dev.index)
    g.set_system(system)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    # the dimer/trimer schedule cached by the autotuner for this size class
    # (the built-in rule when none is cached)
    from paper_2606_28022_b300 import autotune
    opts = autotune.options(system, wl["level"], args.precision, dev.index, **wl.get("opts", {}))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (126 MB)
    e_key = wl["level"] - 1

    for _ in range(max(args.warmup, 3)):
        g.run(opts, stream=sptr)
    torch.cuda.synchronize(dev)

    proc, rows = clocks_sampler(dev.index) if rank == 0 else (None, [])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()                                  # L2 flush between timed steps
        ev[k][0].record(stream)
        g.run(opts, stream=sptr)
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
    energies = g.energies()
    s0 = stats[-1]
    solves_step = s0["n_monomer_solves"] + s0["n_dimer_scc"] + s0["n_trimer_scc"]

    # e2e through the public API with host buffers: coordinates in, results out
    xyz_host = np.ascontiguousarray(system.xyz, dtype=np.float64)
    e2e_steps = max(1, min(3, args.steps))
    h2d = d2h = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_coordinates(xyz_host)
        g.run(opts, stream=sptr)
        g.energies()
        g.monomers()
        g.dimers()
        g.trimers()
        st = g.stats()
        h2d += st["h2d_bytes"]
        d2h += st["d2h_bytes"]
    torch.cuda.synchronize(dev)
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": solves_step / t_e2e, "unit": UNIT, "ms_per_step": 1e3 * t_e2e,
           "h2d_bytes_per_step": int(h2d / e2e_steps), "d2h_bytes_per_step": int(d2h / e2e_steps)}
    dims = g.dimers()
    tris = g.trimers()

    # plain FP64 GPU form of the same workload (the metric's comparison)
    fp64 = None
    if rank == 0 and args.precision == "mixed" and args.fp64_repeats > 0:
        o64 = fmo.options(level=wl["level"], precision="fp64", **wl.get("opts", {}))
        ms64 = []
        for _ in range(args.fp64_repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            g.run(o64, stream=sptr)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ms64.append(a.elapsed_time(b))
        e64 = g.energies()
        s64 = g.stats()
        med = float(statistics.median(ms64))
        fp64 = {"ms_per_step_median": med, "runs": len(ms64), "ms_runs": ms64, "energies": e64,
                "fragment_scc_per_s": (s64["n_monomer_solves"] + s64["n_dimer_scc"] + s64["n_trimer_scc"]) / (med / 1e3),
                "abs_dE_total_mixed_vs_fp64": abs(energies[e_key] - e64[e_key]),
                "speedup_mixed_over_fp64": med / float(np.median(step_ms)),
                "note": "the first FP64 run of the process (its buffers allocated inside the timed run)"
                        if args.fp64_repeats == 1 else "median"}

    # analytic gradient of the same workload (energy run with want_gradient,
    # then fmo_get_gradient), once
    grad = None
    if rank == 0 and not args.no_gradient:
        og = fmo.options(level=wl["level"], precision=args.precision, want_gradient=1, **wl.get("opts", {}))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.run(og, stream=sptr)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms_run = a.elapsed_time(b)
        eg = g.energies()
        t0 = time.perf_counter()
        gr = g.gradient()
        t_grad = time.perf_counter() - t0
        sg = g.stats()
        grad = {"ms_energy_run_want_gradient": ms_run, "ms_gradient": sg["ms_gradient"],
                "wall_s_gradient_call": t_grad, "zvector_gmres_iterations": sg["zvector_iterations"],
                "zvector_rel_residual": sg["zvector_residual"], "max_abs_grad": float(np.abs(gr).max()),
                "max_abs_sum_of_forces": float(np.abs(gr.sum(axis=0)).max()),
                "abs_dE_vs_timed_run": abs(eg[e_key] - energies[e_key])}

    # roofline of the dominant kernel: the SCC launch of the longest pass
    peaks, peak_src = measured_peaks()
    p32 = fmo.fma_peak("fp32", dev.index)
    p64 = fmo.fma_peak("fp64", dev.index)
    ptf32 = peaks["bf16_tflops"] / 2.0                # TF32 dense = half the BF16 rate (nominal ratio)
    ms_scc = [float(np.mean([s["ms_scc"][p] for s in stats])) for p in range(3)]
    dom = int(np.argmax(ms_scc))
    pass_name = ["monomer", "dimer", "trimer"][dom]
    f32 = float(np.mean([s["flops_fp32"][dom] for s in stats]))
    f64 = float(np.mean([s["flops_fp64"][dom] for s in stats]))
    t_meas = ms_scc[dom] / 1e3
    # 15 n^3 per SCC iteration: 6 n^3 GEMM-shaped (transform, C = X C', P =
    # C n C^T) at the TF32 tensor rate, 9 n^3 eigensolve at the FP32 FMA rate;
    # the FP64 work (FP64 iterations, the FP64 energy finish) at the FP64 rate
    t_min = 0.4 * f32 / (ptf32 * 1e12) + 0.6 * f32 / (p32 * 1e12) + f64 / (p64 * 1e12)
    achieved = (f32 + f64) / t_meas / 1e12 if t_meas > 0 else 0.0
    peak = (f32 + f64) / t_min / 1e12 if t_min > 0 else 0.0
    traffic, tnote = measured_traffic(args.workload, pass_name)
    roofline = {"bound": "alu", "kernel": f"scc_kernel ({pass_name} pass)", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak if peak else 0.0, "traffic": traffic,
                "traffic_note": tnote,
                "peak_basis": f"T_min = 6n^3/it at TF32 {ptf32:.0f} TF/s (bf16_tflops/2, {peak_src}) + 9n^3/it at "
                              f"FP32 {p32:.1f} TF/s + FP64 work at {p64:.2f} TF/s (FP32/FP64 FMA-loop peaks "
                              "measured in this run by fmo_fma_peak); peak = flops / T_min",
                "fp32_fma_tflops_measured": p32, "fp64_fma_tflops_measured": p64, "tf32_tensor_tflops": ptf32,
                "flops_fp32": f32, "flops_fp64": f64, "kernel_ms": ms_scc[dom],
                "kernel_share_of_step": ms_scc[dom] / float(np.mean(step_ms))}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dl = [tuple(x) for x in dims.ij[dims.scc]]
        tl = [tuple(x) for x in tris.ijk]
        workers = cpu_workers()
        rate, dt, counts, workers = cpu_oracle_sample(system, s0["n_monomer_solves"], dl, tl, max(8, 15 * workers),
                                                      workers=workers)
        cpu = {"value": rate, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{sum(counts.values())} oracle n-mer SCC solves of this workload {counts} in the workload's "
                         f"proportions, zero ESP, {workers} one-thread worker processes, {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)),
                "ms_per_step_median": float(np.median(step_ms)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": wl["desc"], "precision": args.precision, "level": wl["level"],
                           "schedule": {**{f: int(getattr(opts, f)) for f in autotune.FIELDS},
                                        "source": "autotuner cache" if any(getattr(opts, f) for f in
                                                                           autotune.FIELDS) else "rule"},
                           "n_frag": system.n_frag, "n_atoms": system.n_atoms,
                           "n_dimer_scc": s0["n_dimer_scc"], "n_dimer_esdim": s0["n_dimer_esdim"],
                           "n_trimer_scc": s0["n_trimer_scc"], "outer_iterations": s0["outer_iterations"],
                           "fragment_scc_solves_per_step": solves_step,
                           "l2": "256 MB buffer written between timed steps (L2 flush)",
                           "parallelism": f"replicas x{world} (independent frames)", "geometry": geo},
                "energies": {"e_fmo1": energies[0], "e_fmo2": energies[1], "e_fmo3": energies[2]},
                "fp64_form": fp64, "gradient": grad,
                "stage_ms": {k: s0[k] for k in ("ms_setup", "ms_monomer", "ms_select", "ms_dimer", "ms_trimer",
                                                 "ms_reduce")},
                "per_pass": pass_rates(stats),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": summarize_clocks(rows)}
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
