"""Wall time and iterations to a threshold: plain FP64 FA-SD against the
mixed FP32 -> FP64 mode with and without the learned multiplier, the
exact-exponential and plain-SD variants, and scans over alpha.

    python -m paper_1206_0675_gb300.evaluate --lattice 32 --eps 0.7 --seeds 100-107 [--tol 1e-15]
    python -m paper_1206_0675_gb300.evaluate --lattice 16 --eps 1.0 --seeds 100-101 \
        --modes fp64,fp64_exp,fp64_sd --alphas 0.04,0.06,0.08,0.1,0.12 --tol 1e-12
    python -m paper_1206_0675_gb300.evaluate --run-steps 3 --lattice 32 --eps 1.0 --seeds 0 \
        --modes fp32 --store12 --decomps 2d2d     # a few steps of one lattice (profiling case)
    python -m paper_1206_0675_gb300.evaluate --lattice 32 --eps 1.0 --seeds 0-3 \
        --modes fp64,fp64_or,mixed_or --omega 1.7  # overrelaxation against FA-SD (sweeps under "iters")

Prints one JSON line per configuration and a summary line.
"""

from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import accounting, fields, lgf
from .preconditioner import DEFAULT_WEIGHTS

STORAGES = {"fp64_18": ("fp64", False, 8, 3, 3), "fp64_12": ("fp64", True, 8, 2, 3),
            "fp32_12": ("fp32", True, 4, 2, 2), "fp32_18": ("fp32", False, 4, 3, 3)}

MODES = {
    "fp64": dict(precision="fp64"),
    "fp64_learned": dict(precision="fp64", learned=True),
    "mixed": dict(precision="mixed", store12=True),
    "mixed_learned": dict(precision="mixed", store12=True, learned=True),
    "fp64_exp": dict(precision="fp64", exact_exp=True),
    "mixed_exp": dict(precision="mixed", store12=True, exact_exp=True),
    "fp64_sd": dict(precision="fp64", plain_sd=True),
    # overrelaxation (omega = --omega, theta measured every OR_CHECK sweeps)
    "fp64_or": dict(precision="fp64"),
    "fp32_or": dict(precision="fp32", store12=True),
    "mixed_or": dict(precision="mixed", store12=True),
}
OR_CHECK = 10


def run_or(mode, ext, U, tol, max_sweeps, omega, switch=None):
    """Overrelaxation to tol: seconds, sweeps, final F and theta."""
    import torch
    kw = MODES[mode]
    with lgf.Lattice(ext, **kw) as lat:
        if switch is not None and kw["precision"] == "mixed":
            lat.set_switch_theta(switch)
        lat.set_links(U)
        lat.or_fix(tol, 1, omega, OR_CHECK)   # builds the loop graph
        lat.set_links(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n, F, th, conv = lat.or_fix(tol, max_sweeps, omega, OR_CHECK)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    return {"seconds": dt, "iters": n, "F": F, "theta": th, "converged": conv, "omega": omega}


def run_mode(mode, ext, U, tol, max_iter, weights, switch=None, alpha=0.08, omega=1.7, learned_theta=None):
    import torch
    if mode.endswith("_or"):
        return run_or(mode, ext, U, tol, max_iter, omega, switch)
    kw = MODES[mode]
    with lgf.Lattice(ext, **kw) as lat:
        if kw.get("learned"):
            lat.load_preconditioner(weights)
            if learned_theta is not None:
                lat.set_learned_theta(learned_theta)
        if switch is not None and kw["precision"] == "mixed":
            lat.set_switch_theta(switch)
        lat.set_links(U)
        lat.fix(tol, 1, alpha)   # builds the loop graphs
        lat.set_links(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            it, F, th, conv = lat.fix(tol, max_iter, alpha)
        except lgf.LgfError as e:  # a diverging step size: reported, not fatal to a scan
            torch.cuda.synchronize()
            return {"seconds": time.perf_counter() - t0, "iters": max_iter, "F": None, "theta": None,
                    "converged": False, "fallbacks": 0, "error": str(e)}
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        nf = lat.fallbacks() if kw.get("learned") else 0
    return {"seconds": dt, "iters": it, "F": F, "theta": th, "converged": conv, "fallbacks": nf}


def time_steps(lat, steps, warmup):
    """Wall seconds per lgf_step and the mean per-kernel CUDA-event times."""
    import torch
    for _ in range(warmup):
        lat.step(0.08)
    lat.set_timing(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        lat.step(0.08)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    ms, _ = lat.get_timing()
    return dt, ms


def kernel_table(ext, U, steps=20, warmup=5, peak_gbs=None, decomps=("2d2d",), unfused=False):
    """Per-kernel CUDA-event times and compulsory-traffic GB/s of every precision/storage.

    With several decompositions of the 4D transform, every storage is timed
    with each of them; pass A / B / C then read "forward passes", "the pass
    with the filter" and "inverse passes + g" (the GB/s of the 2D + 2D passes
    are left out for the others, whose traffic differs).  FP32 storages run
    the fused update + measurement (reported under "update"); with unfused
    they are also timed with the two kernels apart ("<storage>/unfused")."""
    V = int(np.prod(ext))
    out = {}
    for name, (prec, s12, rb, rows, grows) in STORAGES.items():
        byt = accounting.bytes_per_site(rb, rows, grows, k_bytes=rb)
        variants = [(dec, True) for dec in decomps]
        if unfused and prec == "fp32":
            variants.append(("2d2d", False))
        for dec, fused in variants:
            key = name if dec == "2d2d" else f"{name}/{dec}"
            if not fused:
                key = f"{name}/unfused"
            fused_here = fused and prec == "fp32"
            with lgf.Lattice(ext, prec, store12=s12) as lat:
                try:
                    lat.set_fft_decomposition(dec)
                except lgf.LgfError as e:
                    out[key] = {"unsupported": str(e)}
                    continue
                if prec == "fp32":
                    lat.set_fused_update(fused)
                lat.set_links(U)
                dt, ms = time_steps(lat, steps, warmup)
            row = {"iters_per_s": 1.0 / dt, "ms_per_step": dt * 1e3, "fused_update_measure": fused_here,
                   "kernels": {}}
            for k, t in zip(accounting.KERNELS, ms):
                own = dec == "2d2d" or k in ("update", "measure")
                b = byt[k]
                if fused_here and k == "update":
                    b = accounting.fused_update_measure_bytes(rb, rows, grows)
                gbs = b * V / (t * 1e-3) / 1e9 if (t > 0 and own) else None
                row["kernels"][k] = {"ms": t, "gbs": gbs, "hbm_frac": gbs / peak_gbs if (gbs and peak_gbs) else None}
            out[key] = row
    return out


def run_steps(ext, eps, seed, mode, store12, decomp, steps, weights, omega=1.7):
    """A few lgf_step calls (modes fp64_or / fp32_or: overrelaxation sweeps) on
    one lattice with a fixed plan: the small case a profiler captures one
    kernel of."""
    import torch
    if mode.endswith("_or"):
        U = fields.random_links(ext, eps, seed)
        with lgf.Lattice(ext, mode[:4], store12=store12) as lat:
            lat.set_links(U)
            lat.or_sweep(omega, steps)
            torch.cuda.synchronize()
            F, th = lat.measure()
        print(json.dumps({"extents": ext, "mode": mode, "store12": store12, "sweeps": steps, "omega": omega,
                          "F": F, "theta": th}), flush=True)
        return
    prec = {"fp64": "fp64", "fp32": "fp32", "mixed": "mixed", "fp32_learned": "fp32", "fp64_learned": "fp64"}[mode]
    learned = mode.endswith("_learned")
    U = fields.random_links(ext, eps, seed)
    with lgf.Lattice(ext, prec, store12=store12, learned=learned) as lat:
        if learned:
            lat.load_preconditioner(weights)
        lat.set_fft_decomposition(decomp)
        lat.set_links(U)
        for _ in range(steps):
            lat.step(0.08)
        torch.cuda.synchronize()
        F, th = lat.measure()
    print(json.dumps({"extents": ext, "mode": mode, "store12": store12, "decomposition": decomp, "steps": steps,
                      "F": F, "theta": th}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", type=int, default=32)
    ap.add_argument("--eps", type=float, default=0.7)
    ap.add_argument("--seeds", default="100-107")
    ap.add_argument("--tol", type=float, default=1e-15)
    ap.add_argument("--max-iter", type=int, default=30000)
    ap.add_argument("--modes", default="fp64,mixed,mixed_learned")
    ap.add_argument("--weights", default=DEFAULT_WEIGHTS)
    ap.add_argument("--extents", default=None, help="Lx,Ly,Lz,Lt (overrides --lattice)")
    ap.add_argument("--kernels", action="store_true", help="per-kernel table of every precision/storage")
    ap.add_argument("--unfused", action="store_true",
                    help="with --kernels: also time the FP32 storages with the update and measurement apart")
    ap.add_argument("--decomps", default="2d2d",
                    help="decompositions of the 4D transform for --kernels (2d2d,1d4,3d1d)")
    ap.add_argument("--switch", type=float, default=None, help="switch level of the mixed modes")
    ap.add_argument("--alphas", default="0.08", help="comma-separated step sizes alpha (a scan if several)")
    ap.add_argument("--run-steps", type=int, default=0,
                    help="only run this many steps of one lattice (first seed, first mode of fp64, fp32, mixed, "
                         "fp32_learned, fp64_learned; first of --decomps) and print F and theta")
    ap.add_argument("--store12", action="store_true", help="with --run-steps: 12-real link storage")
    ap.add_argument("--omega", type=float, default=1.7, help="overrelaxation parameter of the *_or modes")
    ap.add_argument("--learned-theta", default=None,
                    help="comma-separated levels below which the learned modes apply the table (a scan if several)")
    args = ap.parse_args()
    a, b = (int(v) for v in args.seeds.split("-")) if "-" in args.seeds else (int(args.seeds),) * 2
    ext = tuple(int(v) for v in args.extents.split(",")) if args.extents else (args.lattice,) * 4
    if args.run_steps:
        run_steps(ext, args.eps, a, args.modes.split(",")[0], args.store12, args.decomps.split(",")[0], args.run_steps,
                  np.load(args.weights), args.omega)
        return
    if args.kernels:
        peak = None
        try:
            with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                   "MEASURED_PEAKS.json")) as f:
                peak = float(json.load(f)["hbm_gbs"])
        except Exception:
            pass
        U = fields.random_links(ext, args.eps, a)
        print(json.dumps({"extents": ext, "eps": args.eps, "seed": a, "peak_gbs": peak,
                          "table": kernel_table(ext, U, peak_gbs=peak, decomps=args.decomps.split(","),
                                                unfused=args.unfused)}),
              flush=True)
        return
    weights = np.load(args.weights)
    alphas = [float(v) for v in args.alphas.split(",")]
    scan = len(alphas) > 1
    levels = [None] if args.learned_theta is None else [float(v) for v in args.learned_theta.split(",")]
    runs = [(m, al, lv, (f"{m}@{al:g}" if scan else m) + (f"<{lv:g}" if lv is not None and "learned" in m else ""))
            for al in alphas for m in args.modes.split(",") for lv in (levels if "learned" in m else [None])]
    tot = {key: [0.0, 0, 0] for _, _, _, key in runs}
    for seed in range(a, b + 1):
        U = fields.random_links(ext, args.eps, seed)
        row = {"lattice": list(ext), "eps": args.eps, "seed": seed}
        for m, al, lv, key in runs:
            r = run_mode(m, ext, U, args.tol, args.max_iter, weights, args.switch, al, args.omega, lv)
            row[key] = r
            tot[key][0] += r["seconds"]
            tot[key][1] += r["iters"]
            tot[key][2] += int(not r["converged"])
        print(json.dumps(row), flush=True)
    summary = {k: {"seconds": v[0], "iters": v[1], "not_converged": v[2]} for k, v in tot.items()}
    for m, al, _, key in runs:
        base = f"fp64@{al:g}" if scan else "fp64"
        if base in tot:
            summary[key]["speedup_vs_fp64"] = tot[base][0] / tot[key][0]
    print(json.dumps({"summary": summary, "lattice": list(ext), "eps": args.eps, "seeds": args.seeds,
                      "tol": args.tol, "switch": args.switch, "alphas": alphas}), flush=True)


if __name__ == "__main__":
    main()
