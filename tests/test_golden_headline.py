"""The stored 32^4 oracle values (tests/golden/headline_32x4_*.json) against
the oracle itself and against Algorithm 1's stop rule.

Re-running whole 32^4 trajectories takes minutes of CPU time, so this checks
the first measurement and the first step of the 50-step trajectory, plus the
structure every fixture must have (strict stop test theta < tol, one F and
theta per measurement)."""

import glob
import json
import os

import numpy as np
import pytest

from oracle import lgf_oracle as O
from paper_1206_0675_gb300 import fields

HERE = os.path.dirname(os.path.abspath(__file__))
PATHS = sorted(glob.glob(os.path.join(HERE, "golden", "headline_32x4_*.json")))


def load(path):
    with open(path) as f:
        return json.load(f)


def test_five_fixtures():
    assert len(PATHS) == 5


@pytest.mark.parametrize("path", PATHS, ids=[os.path.basename(p) for p in PATHS])
def test_fixture_structure(path):
    g = load(path)
    n = g["iterations"]
    assert len(g["F"]) == len(g["theta"]) == n + 1
    th = np.array(g["theta"])
    if g["tol"] > 0:
        # Algorithm 1 iterates while theta >= tol: only the last entry is below it
        assert g["converged"] and th[-1] < g["tol"] and np.all(th[:-1] >= g["tol"])
    else:
        assert n == g["max_iter"]
    # F of every fixture rises monotonically along these trajectories (alpha = 0.08)
    assert np.all(np.diff(g["F"]) > -1e-15)
    for s in g["G_samples"]:
        G = np.array(s["G_re"]) + 1j * np.array(s["G_im"])
        assert np.max(np.abs(G @ G.conj().T - np.eye(3))) < 1e-12
    if g["tol"] > 0:
        # the oracle's rounding spread along the fix: one entry per measurement,
        # at the level of FP64 rounding (written by make_golden.py --headline-spread)
        sp = g["spread"]
        assert len(sp["theta_rel"]) == len(sp["F_rel"]) == n + 1
        assert 0 <= min(sp["theta_rel"]) and max(sp["theta_rel"]) < 1e-9 and max(sp["F_rel"]) < 1e-13


def test_first_step_of_the_50_step_trajectory_reproduces():
    g = load(os.path.join(HERE, "golden", "headline_32x4_eps1.0_seed0_50steps.json"))
    U = fields.random_links(tuple(g["extents"]), g["eps"], g["seed"])
    F0, th0, D = O.measure(U)
    assert abs(F0 - g["F"][0]) < 1e-14 * abs(g["F"][0]) + 1e-16
    assert abs(th0 - g["theta"][0]) < 1e-13 * g["theta"][0]
    U1, _ = O.fa_step(U, g["alpha"], D=D)
    del U
    F1, th1, _ = O.measure(U1)
    assert abs(F1 - g["F"][1]) < 1e-13 * abs(g["F"][1])
    assert abs(th1 - g["theta"][1]) < 1e-12 * g["theta"][1]
