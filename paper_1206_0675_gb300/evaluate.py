"""Wall time and iterations to a threshold: plain FP64 FA-SD against the
mixed FP32 -> FP64 mode with and without the learned multiplier.

    python -m paper_1206_0675_gb300.evaluate --lattice 32 --eps 0.7 --seeds 100-107 [--tol 1e-15]

Prints one JSON line per configuration and a summary line.
"""

from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import fields, lgf
from .preconditioner import DEFAULT_WEIGHTS

MODES = {
    "fp64": dict(precision="fp64"),
    "fp64_learned": dict(precision="fp64", learned=True),
    "mixed": dict(precision="mixed", store12=True),
    "mixed_learned": dict(precision="mixed", store12=True, learned=True),
}


def run_mode(mode, ext, U, tol, max_iter, weights):
    import torch
    kw = MODES[mode]
    with lgf.Lattice(ext, **kw) as lat:
        if kw.get("learned"):
            lat.load_preconditioner(weights)
        lat.set_links(U)
        lat.fix(tol, 1, 0.08)   # builds the loop graphs
        lat.set_links(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, F, th, conv = lat.fix(tol, max_iter, 0.08)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        nf = lat.fallbacks() if kw.get("learned") else 0
    return {"seconds": dt, "iters": it, "F": F, "theta": th, "converged": conv, "fallbacks": nf}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", type=int, default=32)
    ap.add_argument("--eps", type=float, default=0.7)
    ap.add_argument("--seeds", default="100-107")
    ap.add_argument("--tol", type=float, default=1e-15)
    ap.add_argument("--max-iter", type=int, default=30000)
    ap.add_argument("--modes", default="fp64,mixed,mixed_learned")
    ap.add_argument("--weights", default=DEFAULT_WEIGHTS)
    args = ap.parse_args()
    a, b = (int(v) for v in args.seeds.split("-")) if "-" in args.seeds else (int(args.seeds),) * 2
    ext = (args.lattice,) * 4
    weights = np.load(args.weights)
    modes = args.modes.split(",")
    tot = {m: [0.0, 0] for m in modes}
    for seed in range(a, b + 1):
        U = fields.random_links(ext, args.eps, seed)
        row = {"lattice": args.lattice, "eps": args.eps, "seed": seed}
        for m in modes:
            r = run_mode(m, ext, U, args.tol, args.max_iter, weights)
            row[m] = r
            tot[m][0] += r["seconds"]
            tot[m][1] += r["iters"]
        print(json.dumps(row), flush=True)
    summary = {m: {"seconds": v[0], "iters": v[1]} for m, v in tot.items()}
    if "fp64" in tot:
        for m in modes:
            summary[m]["speedup_vs_fp64"] = tot["fp64"][0] / tot[m][0]
    print(json.dumps({"summary": summary, "lattice": args.lattice, "eps": args.eps, "seeds": args.seeds,
                      "tol": args.tol}), flush=True)


if __name__ == "__main__":
    main()
