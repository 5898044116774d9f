"""The oracle against its stored trajectories (tests/golden/, written by
tests/golden/make_golden.py from the oracle itself): a regression guard
that any change to the oracle's arithmetic shows up here."""

import glob
import json
import os

import numpy as np
import pytest

from oracle import lgf_oracle as O
from paper_1206_0675_gb300 import fields

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "fa_*.json")))


def load(path):
    with open(path) as f:
        return json.load(f)


def test_fixtures_present():
    assert len(GOLDEN) >= 3


@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p) for p in GOLDEN])
def test_oracle_reproduces_stored_trajectory(path):
    g = load(path)
    U = fields.random_links(tuple(g["extents"]), g["eps"], g["seed"])
    res = O.fix(U, alpha=g["alpha"], tol=0.0, max_iter=g["iterations"], track_G=True, exact_exp=g["exact_exp"])
    assert np.allclose(res["F"], g["F"], rtol=1e-12, atol=1e-14)
    assert np.allclose(res["theta"], g["theta"], rtol=1e-11, atol=0)
    assert abs(O.plaquette(U) - g["plaquette"]) < 1e-14
    for s in g["G_samples"]:
        x, y, z, t = s["site"]
        want = np.array(s["G_re"]) + 1j * np.array(s["G_im"])
        assert np.max(np.abs(res["G"][t, z, y, x] - want)) < 1e-11
