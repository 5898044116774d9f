"""Determinism and resume.

The reductions of F and theta use per-CTA partials summed in a fixed order
(no floating-point atomics), so two runs of the same input are bit-identical.
A fix can be split at any iteration: its state is only the links (and the
accumulated transform), so taking the links out with lgf_get_links and
starting a new handle from them continues the same trajectory bit for bit.
"""

import numpy as np
import pytest

from oracle import lgf_oracle as O
from paper_1206_0675_gb300 import fields
from paper_1206_0675_gb300 import lgf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lgf.load_library()


def trajectory(ext, U, prec, n, store12=False):
    with lgf.Lattice(ext, prec, store12=store12, track_G=True) as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(n + 1)
        lat.fix(0.0, n, 0.08)
        return Fh.copy(), Th.copy(), lat.get_links(), lat.get_transform()


@pytest.mark.parametrize("prec,store12", [("fp64", False), ("fp64", True), ("fp32", True), ("fp32", False)])
def test_two_runs_are_bit_identical(prec, store12):
    ext = (8, 6, 12, 8)
    U = fields.random_links(ext, eps=0.9, seed=12)
    a = trajectory(ext, U, prec, 40, store12)
    b = trajectory(ext, U, prec, 40, store12)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_resume_from_links_continues_bit_for_bit():
    ext = (8, 8, 6, 6)
    U = fields.random_links(ext, eps=1.0, seed=13)
    F_all, T_all, U_all, G_all = trajectory(ext, U, "fp64", 50)
    F_a, T_a, U_mid, G_a = trajectory(ext, U, "fp64", 30)
    F_b, T_b, U_end, G_b = trajectory(ext, U_mid, "fp64", 20)
    assert np.array_equal(F_a, F_all[:31]) and np.array_equal(T_a, T_all[:31])
    assert np.array_equal(F_b, F_all[30:]) and np.array_equal(T_b, T_all[30:])
    assert np.array_equal(U_end, U_all)
    # the transforms compose: G_total = G_second G_first
    assert np.max(np.abs(G_b @ G_a - G_all)) < 1e-13
    assert np.max(np.abs(O.apply_gauge(U, G_b @ G_a) - U_end)) < 1e-12
