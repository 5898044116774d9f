"""The GPU path against the stored oracle trajectories of tests/golden/
(per-iteration F and theta, sampled entries of the accumulated transform G)."""

import glob
import json
import os

import numpy as np
import pytest

from paper_1206_0675_gb300 import fields
from paper_1206_0675_gb300 import lgf

pytestmark = pytest.mark.gpu

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "fa_*.json")))


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lgf.load_library()


@pytest.mark.parametrize("decomp", ["2d2d", "1d4"])
@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p) for p in GOLDEN])
def test_gpu_reproduces_stored_trajectory(path, decomp):
    with open(path) as f:
        g = json.load(f)
    ext = tuple(g["extents"])
    U = fields.random_links(ext, g["eps"], g["seed"])
    n = g["iterations"]
    with lgf.Lattice(ext, "fp64", track_G=True, exact_exp=g["exact_exp"]) as lat:
        lat.set_fft_decomposition(decomp)
        lat.set_links(U)
        Fh, Th = lat.set_trace(n + 1)
        it, F, th, conv = lat.fix(0.0, n, g["alpha"])
        G = lat.get_transform()
    assert it == n
    assert np.allclose(Fh, g["F"], rtol=1e-11, atol=1e-13)
    assert np.allclose(Th, g["theta"], rtol=1e-11, atol=0)
    for s in g["G_samples"]:
        x, y, z, t = s["site"]
        want = np.array(s["G_re"]) + 1j * np.array(s["G_im"])
        assert np.max(np.abs(G[t, z, y, x] - want)) < 1e-10
