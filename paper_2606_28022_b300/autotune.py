"""Schedule autotuner of the SCC passes (monomers, dimers, trimers).

Knobs of fmo_options that change how fast the passes run, not what they
compute: nmer_ctas_per_sm / monomer_ctas_per_sm (one CTA per SM with 255
registers per thread, or two with 128 registers and half an SM of shared
memory each) and nmer_matrix_smem / monomer_matrix_smem (the n x n
eigen-solve matrix of every n-mer in shared memory where it fits, in global
memory, or for monomers only its FP32 copy in shared memory).  tune() times
every combination of the dimer/trimer knobs on the device for one system (the
passes' own CUDA-event stage times, best of `repeats` runs), then the monomer
knobs with that choice, keeps the fastest in a JSON cache keyed by the
workload's size class, and reports it beside the built-in rule; options()
returns fmo_options with the cached choice, or the rule when nothing is
cached.

    python -m paper_2606_28022_b300.autotune --workload pentacene660 --precision mixed
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

from . import fmo

KNOBS = [(c, m) for c in (1, 2) for m in (1, 2)]
MONO_KNOBS = [(1, 1), (2, 1), (2, 2), (2, 3)]
FIELDS = ("nmer_ctas_per_sm", "nmer_matrix_smem", "monomer_ctas_per_sm", "monomer_matrix_smem")
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedules.json")


def size_class(system, level: int, precision: str, device_name: str) -> str:
    """Cache key: FMO level, precision, the number of fragments rounded up to a
    power of two, the largest fragment (atoms), and the device."""
    nat = np.bincount(np.asarray(system.frag))
    nf = 1 << max(0, math.ceil(math.log2(max(1, system.n_frag))))
    return f"L{level}-{precision}-nfrag{nf}-maxat{int(nat.max())}-{device_name}"


def _device_name(device: int) -> str:
    import torch
    return torch.cuda.get_device_name(device).replace(" ", "_")


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def options(system, level: int, precision: str, device: int = 0, path: str = DEFAULT_CACHE,
            device_name: str | None = None, **kw):
    """fmo_options for this system with the cached schedule (the built-in rule
    when the cache has no entry for its size class)."""
    name = device_name if device_name is not None else _device_name(device)
    e = load(path).get(size_class(system, level, precision, name))
    knobs = {} if e is None else {f: int(e[f]) for f in FIELDS if f in e}
    return fmo.options(level=level, precision=precision, **knobs, **kw)


def tune(g: "fmo.FMO", system, level: int, precision: str, device: int = 0, repeats: int = 2,
         path: str = DEFAULT_CACHE, **kw) -> dict:
    """Time the built-in rule and every knob combination on `system` (the
    dimer and trimer stages for their knobs, then the monomer stage for its
    knobs, best of `repeats` each); cache and return the fastest choice with
    all timings."""
    g.set_system(system)

    def timed(knobs, stage):
        o = fmo.options(level=level, precision=precision, **knobs, **kw)
        best, energies = math.inf, None
        for _ in range(repeats):
            g.run(o, allow_unconverged=True)
            st = g.stats()
            best = min(best, sum(st[x] for x in stage))
            energies = g.energies()
        return best, list(energies)

    rows = []
    for c, m in [(0, 0)] + KNOBS:
        t, e = timed({"nmer_ctas_per_sm": c, "nmer_matrix_smem": m}, ("ms_dimer", "ms_trimer"))
        rows.append({"nmer_ctas_per_sm": c, "nmer_matrix_smem": m, "ms": t, "energies": e})
    choice = min(rows[1:], key=lambda r: r["ms"])
    nk = {"nmer_ctas_per_sm": choice["nmer_ctas_per_sm"], "nmer_matrix_smem": choice["nmer_matrix_smem"]}
    mrows = []
    for c, m in [(0, 0)] + MONO_KNOBS:
        t, e = timed({**nk, "monomer_ctas_per_sm": c, "monomer_matrix_smem": m}, ("ms_monomer",))
        mrows.append({"monomer_ctas_per_sm": c, "monomer_matrix_smem": m, "ms": t, "energies": e})
    mchoice = min(mrows[1:], key=lambda r: r["ms"])
    key = size_class(system, level, precision, _device_name(device))
    entry = {**nk, "ms": choice["ms"], "rule_ms": rows[0]["ms"], "timings": rows,
             "monomer_ctas_per_sm": mchoice["monomer_ctas_per_sm"],
             "monomer_matrix_smem": mchoice["monomer_matrix_smem"], "monomer_ms": mchoice["ms"],
             "monomer_rule_ms": mrows[0]["ms"], "monomer_timings": mrows}
    cache = load(path)
    cache[key] = entry
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
        fh.write("\n")
    os.replace(tmp, path)
    return {"key": key, **entry}


def _system(name: str):
    from .inputs import geometry as G
    if name == "pentacene660":
        return G.pentacene_cluster(660, seed=4)[0], 3
    if name == "anthracene128":
        return G.anthracene_cluster(128, seed=2)[0], 2
    if name == "ala300":
        return G.polyalanine_helix(300, seed=11), 2
    if name == "water64":
        return G.water_cluster(64, 1), 2
    raise ValueError(name)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="pentacene660", choices=["pentacene660", "anthracene128", "ala300", "water64"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--cache", default=DEFAULT_CACHE)
    args = ap.parse_args(argv)
    from . import build
    from .inputs.params import synthetic_gfn1_table
    build.build()
    system, level = _system(args.workload)
    g = fmo.FMO(synthetic_gfn1_table(), 0)
    r = tune(g, system, level, args.precision, repeats=args.repeats, path=args.cache)
    g.close()
    print(json.dumps({"workload": args.workload, **r}))


if __name__ == "__main__":
    main()
