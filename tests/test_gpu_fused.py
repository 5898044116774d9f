"""The fused update + measurement of FP32 lanes (lgf_set_fused_update).

The fused kernel recomputes the updated backward links with the same
arithmetic as the update kernel, so a fused run must be bit-identical to an
unfused run: the same F and theta after every step and the same links.  It is
also checked against the FP64 CPU oracle like every FP32 path.
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


def run(ext, U, store12, fused, n, switch_after=None):
    with lgf.Lattice(ext, "fp32", store12=store12) as lat:
        lat.set_fused_update(fused)
        lat.set_links(U)
        Fh, Th = [], []
        for k in range(n):
            if switch_after is not None and k == switch_after:
                lat.set_fused_update(not fused)
            lat.step(0.08)
            F, th = lat.measure()
            Fh.append(F)
            Th.append(th)
        return np.array(Fh), np.array(Th), lat.get_links(), lat.get_divergence()


@pytest.mark.parametrize("store12", [True, False])
@pytest.mark.parametrize("ext", [(8, 8, 8, 8), (3, 4, 6, 9), (12, 6, 4, 8)])
def test_fused_is_bit_identical_to_unfused(ext, store12):
    U = fields.random_links(ext, eps=0.9, seed=5)
    a = run(ext, U, store12, True, 7)
    b = run(ext, U, store12, False, 7)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_switching_fusion_mid_run_keeps_the_links():
    """Turning fusion off after an odd number of fused steps moves the links
    out of the second buffer; the run continues exactly as an unfused one."""
    ext = (8, 4, 6, 8)
    U = fields.random_links(ext, eps=0.8, seed=6)
    a = run(ext, U, True, True, 8, switch_after=3)
    b = run(ext, U, True, False, 8)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    c = run(ext, U, True, False, 8, switch_after=5)   # unfused, then fused
    for x, y in zip(c, b):
        assert np.array_equal(x, y)


def test_fused_fix_against_oracle_and_mixed():
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=0)
    ref = O.fix(U, tol=0.0, max_iter=50, track_G=False)
    with lgf.Lattice(ext, "fp32", store12=True, track_G=True) as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(51)
        it, F, th, conv = lat.fix(0.0, 50, 0.08)       # 50 steps: the links end in the first buffer
        U50 = lat.get_links()
        lat.step(0.08)                                   # one more: they end in the second
        U51 = lat.get_links()
        G = lat.get_transform()
    assert it == 50
    for k in range(51):
        assert abs(Fh[k] - ref["F"][k]) < 1e-5 * abs(ref["F"][k]) + 1e-6
        assert abs(Th[k] - ref["theta"][k]) < 1e-5 * ref["theta"][k]
    assert np.max(np.abs(U50 - ref["U"])) < 2e-4
    assert np.max(np.abs(O.apply_gauge(U, G) - U51)) < 1e-4
    ref2 = O.fix(U, tol=1e-15, max_iter=6000, track_G=False)
    with lgf.Lattice(ext, "mixed", store12=True, track_G=True) as lat:
        lat.set_links(U)
        it, F, th, conv = lat.fix(1e-15, 6000, 0.08)
        U1 = lat.get_links()
    assert conv and abs(F - ref2["F"][-1]) < 1e-10
    assert abs(it - ref2["iters"]) <= max(1, 0.02 * ref2["iters"])
    assert abs(O.plaquette(U1) - O.plaquette(U)) < 1e-12


def test_learned_handles_fuse_bit_identically():
    """A learned FP32 handle runs the fused update + measure: with a constant
    multiplier of 2 and alpha scaled by 1.6 steps are rejected, undone on the
    current link buffer and redone, and the run equals the unfused one bit
    for bit (histories, fallbacks, links, transform)."""
    from oracle import lgf_mlp_oracle as M
    p = np.zeros(M.NPARAM)
    p[M.OFF_B4] = 3.0
    bits = (M.bf16_round(p).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    ext = (6, 4, 8, 4)
    U = fields.random_links(ext, eps=0.9, seed=21)
    out = []
    for fused in (True, False):
        with lgf.Lattice(ext, "fp32", store12=True, track_G=True, learned=True) as lat:
            lat.set_fused_update(fused)
            lat.load_preconditioner(bits)
            lat.set_links(U)
            Fh, Th, Fl, Dh = lat.set_trace(31, flags=True)
            it, F, th, conv = lat.fix(0.0, 30, 0.128)
            out.append((it, lat.fallbacks(), Fh.copy(), Th.copy(), Fl.copy(), lat.get_links(), lat.get_transform()))
    a, b = out
    assert a[0] == b[0] == 30 and a[1] == b[1] and a[1] > 0
    for x, y in zip(a[2:], b[2:]):
        assert np.array_equal(x, y)
    assert np.count_nonzero(a[4] & lgf.LGF_TRACE_REDO) == a[1]
