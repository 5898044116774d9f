"""Writes the stored oracle trajectories under tests/golden/.

Every value in the fixtures comes from the FP64 CPU oracle (oracle/, which
follows Sec. 2 and Algorithm 1 of arXiv:1206.0675) on the seeded synthetic
fields of paper_1206_0675_gb300/fields.py; nothing here calls the CUDA path.
The fixtures guard the oracle against unintended changes and give the GPU
tests stored expectations that need no oracle run.

    python tests/golden/make_golden.py              # the small fa_*.json cases
    python tests/golden/make_golden.py --headline   # the 32^4 cases (minutes per case)
    python tests/golden/make_golden.py --headline-spread   # then their rounding spread

The 32^4 cases are the 32^4 workload of the benchmark: U_mu(x) = h(x)
exp(i eps sum_a c_a lambda_a/2) h^dag(x+mu) with eps = 1.0, seed 0 (a 50-step
trajectory) and eps = 0.5, seeds 0-3 (fixed to theta < 1e-15), alpha = 0.08.
They run as separate processes (multiprocessing, spawn), one per case.
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lgf_oracle as O  # noqa: E402
from paper_1206_0675_gb300 import fields  # noqa: E402

CASES = [
    # name, extents (Lx, Ly, Lz, Lt), eps, seed, alpha, iterations, exact_exp
    ("fa_4x6x4x8_eps0.8_seed5", (4, 6, 4, 8), 0.8, 5, 0.08, 25, False),
    ("fa_exp_6x4x4x6_eps1.0_seed2", (6, 4, 4, 6), 1.0, 2, 0.08, 25, True),
    ("fa_3x4x6x9_eps0.5_seed0", (3, 4, 6, 9), 0.5, 0, 0.1, 25, False),
]
SAMPLE_SITES = [(0, 0, 0, 0), (1, 2, 3, 1), (3, 1, 0, 2)]  # (x, y, z, t), wrapped into the lattice

HEADLINE_EXT = (32, 32, 32, 32)
HEADLINE_CASES = [
    # name, eps, seed, tol, max_iter: tol = 0 runs exactly max_iter steps
    ("headline_32x4_eps1.0_seed0_50steps", 1.0, 0, 0.0, 50),
    ("headline_32x4_eps0.5_seed0_tol1e-15", 0.5, 0, 1e-15, 3000),
    ("headline_32x4_eps0.5_seed1_tol1e-15", 0.5, 1, 1e-15, 3000),
    ("headline_32x4_eps0.5_seed2_tol1e-15", 0.5, 2, 1e-15, 3000),
    ("headline_32x4_eps0.5_seed3_tol1e-15", 0.5, 3, 1e-15, 3000),
]
HEADLINE_SITES = [(0, 0, 0, 0), (5, 17, 30, 11), (31, 31, 31, 31), (16, 2, 9, 27)]


def make(name, ext, eps, seed, alpha, n, exact_exp):
    U = fields.random_links(ext, eps, seed)
    res = O.fix(U, alpha=alpha, tol=0.0, max_iter=n, track_G=True, exact_exp=exact_exp)
    lx, ly, lz, lt = ext
    G = res["G"]
    samples = []
    for (x, y, z, t) in SAMPLE_SITES:
        x, y, z, t = x % lx, y % ly, z % lz, t % lt
        samples.append({"site": [x, y, z, t], "G_re": G[t, z, y, x].real.tolist(), "G_im": G[t, z, y, x].imag.tolist()})
    return {
        "source": "FP64 CPU oracle, Algorithm 1 of arXiv:1206.0675 (oracle/lgf_oracle.py fix); fields from "
                  "paper_1206_0675_gb300/fields.py random_links",
        "extents": list(ext), "eps": eps, "seed": seed, "alpha": alpha, "exact_exp": exact_exp,
        "iterations": n, "F": res["F"].tolist(), "theta": res["theta"].tolist(),
        "plaquette": O.plaquette(U), "G_samples": samples,
    }


def make_headline(case):
    name, eps, seed, tol, max_iter = case
    U = fields.random_links(HEADLINE_EXT, eps, seed)
    res = O.fix(U, alpha=0.08, tol=tol, max_iter=max_iter, track_G=True)
    G = res["G"]
    samples = [{"site": [x, y, z, t], "G_re": G[t, z, y, x].real.tolist(), "G_im": G[t, z, y, x].imag.tolist()}
               for (x, y, z, t) in HEADLINE_SITES]
    out = {
        "source": "FP64 CPU oracle, Algorithm 1 of arXiv:1206.0675 (oracle/lgf_oracle.py fix); fields from "
                  "paper_1206_0675_gb300/fields.py random_links",
        "extents": list(HEADLINE_EXT), "eps": eps, "seed": seed, "alpha": 0.08, "exact_exp": False,
        "tol": tol, "max_iter": max_iter, "iterations": int(res["iters"]), "converged": bool(res["converged"]),
        "F": res["F"].tolist(), "theta": res["theta"].tolist(), "plaquette": O.plaquette(U),
        "G_samples": samples,
    }
    path = os.path.join(HERE, name + ".json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return path


SPREAD_DELTA = 2.0 ** -52  # one unit in the last place of an entry of size 1


def rounding_spread(case):
    """A second oracle trajectory of a headline fixture whose links are moved,
    after every step, by a random rounding-level amount: U <- U + i delta H U
    with H Hermitian, entries N(0, 1), delta = 2^-52.  Its relative distance
    from the fixture's F and theta, step by step, is the spread that
    different but equally valid FP64 rounding orders produce along that
    trajectory; it is stored beside the trajectory."""
    name, eps, seed, tol, max_iter = case
    path = os.path.join(HERE, name + ".json")
    with open(path) as f:
        g = json.load(f)
    rng = np.random.Generator(np.random.Philox(key=991 + seed))
    U = fields.random_links(HEADLINE_EXT, eps, seed)
    K = O.fa_filter(HEADLINE_EXT, 0.08)

    def nudge(U):
        A = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
        H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
        return U + 1j * SPREAD_DELTA * (H @ U)

    U = nudge(U)
    F, th, D = O.measure(U)
    dF, dT = [abs(F / g["F"][0] - 1)], [abs(th / g["theta"][0] - 1)]
    for k in range(1, g["iterations"] + 1):
        U, _ = O.fa_step(U, 0.08, K, D)
        U = nudge(U)
        F, th, D = O.measure(U)
        dF.append(abs(F / g["F"][k] - 1))
        dT.append(abs(th / g["theta"][k] - 1))
    g["spread"] = {"delta": SPREAD_DELTA, "F_rel": dF, "theta_rel": dT,
                   "how": "oracle rerun with U <- U + i delta H U (H Hermitian, N(0,1) entries) after every step"}
    with open(path, "w") as f:
        json.dump(g, f, indent=1)
    return path


def main():
    if "--headline-spread" in sys.argv[1:]:
        import multiprocessing as mp
        cases = [c for c in HEADLINE_CASES if c[3] > 0]
        with mp.get_context("spawn").Pool(len(cases)) as pool:
            for path in pool.imap_unordered(rounding_spread, cases):
                print("wrote spread into", path, flush=True)
        return
    if "--headline" in sys.argv[1:]:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(len(HEADLINE_CASES)) as pool:
            for path in pool.imap_unordered(make_headline, HEADLINE_CASES):
                print("wrote", path, flush=True)
        return
    for name, *args in CASES:
        path = os.path.join(HERE, name + ".json")
        with open(path, "w") as f:
            json.dump(make(name, *args), f, indent=1)
        print("wrote", path)


if __name__ == "__main__":
    main()
