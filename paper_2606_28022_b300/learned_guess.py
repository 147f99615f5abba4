"""Train and evaluate the learned initial-charge model on jittered frames of
the 128-anthracene aggregate (the learned-guess workload).

    python -m paper_2606_28022_b300.learned_guess [--train 2000] [--test 200] [--epochs 20]

1. Frames: the seeded anthracene aggregate with every atom displaced by a
   Gaussian of 0.1 A (a different seed per frame); the first --train frames
   train the model, the next --test frames evaluate it.
2. Targets: the converged monomer shell charges of each training frame
   (fmo_run at FMO1, monomers converged in FP64 to the usual 1e-10).
3. Training on the GPU (fmo_mlp_train): Adam over shuffled batches.
4. Evaluation: FMO2 (mixed precision) of every test frame from the neutral
   guess and from the learned guess: monomer-loop iterations (one SCC
   iteration of every monomer each), monomer-stage and total time, and the
   largest |dE_FMO2| between the two (both converge to the same tolerances).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--sigma", type=float, default=0.1, help="frame jitter (angstrom)")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)

    from . import build, fmo
    from .inputs import geometry as G
    from .inputs.params import synthetic_gfn1_table

    build.build()
    params = synthetic_gfn1_table()
    base, _ = G.anthracene_cluster(128, seed=2)
    g = fmo.FMO(params, 0)
    g.set_system(base)
    frame = lambda k: G.jittered(base, args.sigma, 10_000 + args.seed * 100_000 + k).xyz

    t0 = time.perf_counter()
    xyz, dq = [], []
    skipped = 0
    o1 = fmo.options(level=1, precision="mixed")
    for k in range(args.train):
        x = frame(k)
        g.set_coordinates(x)
        if g.run(o1, allow_unconverged=True) != fmo.FMO_OK:
            skipped += 1                       # monomer loop not converged: no target
            continue
        xyz.append(x)
        dq.append(g.monomers().shell_dq)
    t_data = time.perf_counter() - t0

    t0 = time.perf_counter()
    g.mlp_init(args.seed)
    loss = g.mlp_train(np.stack(xyz), np.stack(dq), epochs=args.epochs, batch_frames=args.batch, lr=args.lr,
                       seed=args.seed)
    t_train = time.perf_counter() - t0
    del xyz, dq

    rows = []
    unconverged = 0
    o0 = fmo.options(level=2, precision="mixed")
    o1 = fmo.options(level=2, precision="mixed", guess=1)
    for k in range(args.train, args.train + args.test):
        x = frame(k)
        g.set_coordinates(x)
        ref = g.mlp_predict()
        res = {}
        for name, o in (("neutral", o0), ("learned", o1)):
            ok = g.run(o, allow_unconverged=True) == fmo.FMO_OK
            st = g.stats()
            res[name] = (g.energies()[1], st["outer_iterations"], st["ms_monomer"],
                         st["ms_setup"] + st["ms_monomer"] + st["ms_select"] + st["ms_dimer"] + st["ms_reduce"], ok)
        if not (res["neutral"][4] and res["learned"][4]):
            unconverged += 1
            continue
        g.run(fmo.options(level=1, precision="mixed"), allow_unconverged=True)
        err = float(np.sqrt(np.mean((ref - g.monomers().shell_dq) ** 2)))
        rows.append((res["neutral"], res["learned"], err))
    n_it = np.array([r[0][1] for r in rows], dtype=float)
    l_it = np.array([r[1][1] for r in rows], dtype=float)
    out = {
        "workload": f"anthracene128 frames, {args.sigma} A Gaussian jitter; train {args.train}, test {args.test}",
        "epochs": args.epochs, "batch_frames": args.batch, "lr": args.lr,
        "loss_first_last": [float(loss[0]), float(loss[-1])],
        "seconds": {"targets": round(t_data, 2), "training": round(t_train, 2)},
        "training_frames_used": args.train - skipped, "training_frames_unconverged": skipped,
        "test_frames_compared": len(rows), "test_frames_unconverged": unconverged,
        "test_rms_dq_error": float(np.mean([r[2] for r in rows])),
        "monomer_iterations": {"neutral": float(n_it.mean()), "learned": float(l_it.mean()),
                               "saved": float((n_it - l_it).mean())},
        "monomer_ms": {"neutral": float(np.mean([r[0][2] for r in rows])),
                       "learned": float(np.mean([r[1][2] for r in rows]))},
        "fmo2_ms": {"neutral": float(np.mean([r[0][3] for r in rows])),
                    "learned": float(np.mean([r[1][3] for r in rows]))},
        "max_abs_dE_fmo2": float(max(abs(r[0][0] - r[1][0]) for r in rows)),
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
