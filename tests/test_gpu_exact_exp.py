"""The exact-exponential variant (LGF_EXACT_EXP, g = reunitarize(exp(Delta')))
against the FP64 CPU oracle's ``exact_exp`` path.

The GPU evaluates the exponential by the Cayley-Hamilton form with scaling
and squaring; the oracle by an eigendecomposition.  Both agree to rounding
for the exponent norms met here (|Delta'|_F up to ~10 with the large alpha
of the robustness case), so the tolerances are those of the first-order
parity tests.
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


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("ext", [(2, 2, 2, 2), (4, 4, 4, 4), (8, 8, 8, 8), (3, 4, 6, 9), (12, 6, 4, 8)])
@pytest.mark.parametrize("store12", [False, True])
def test_one_step_parity_fp64(ext, store12):
    U = fields.random_links(ext, eps=0.8, seed=7)
    with lgf.Lattice(ext, "fp64", store12=store12, exact_exp=True) as lat:
        lat.set_links(U)
        lat.step(0.08)
        F, th = lat.measure()
        g = lat.get_gauge()
        U1 = lat.get_links()
    Uo, go = O.fa_step(U, 0.08, exact_exp=True)
    Fo, tho, _ = O.measure(Uo)
    assert np.max(np.abs(g - go)) < 1e-12
    assert np.max(np.abs(U1 - Uo)) < 1e-12
    assert rel(F, Fo) < 1e-13
    assert rel(th, tho) < 1e-11
    # and it is not the first-order step
    _, g1 = O.fa_step(U, 0.08)
    assert np.max(np.abs(g - g1)) > 1e-3


@pytest.mark.parametrize("alpha", [0.3, 0.8])
def test_large_exponents_use_squaring(alpha):
    """Large alpha gives |Delta'|_F of several units, so the scaling-and-squaring
    branch (s > 0) runs on most sites."""
    ext = (4, 6, 4, 8)
    U = fields.random_links(ext, eps=1.0, seed=9)
    D = O.divergence(U)
    Dp = O.ifft4(O.fft4(D) * O.fa_filter(ext, alpha)[..., None, None])
    assert np.max(np.linalg.norm(Dp, axis=(-2, -1))) > 2.0
    with lgf.Lattice(ext, "fp64", exact_exp=True) as lat:
        lat.set_links(U)
        lat.step(alpha)
        g = lat.get_gauge()
    _, go = O.fa_step(U, alpha, exact_exp=True)
    assert np.max(np.abs(g - go)) < 2e-13 * max(1.0, alpha * 10)


def test_abelian_field_closed_form():
    """Diagonal links: g = diag(exp(i d)) exactly, d the diagonal of Delta'/i."""
    ext = (4, 6, 4, 4)
    rng = np.random.default_rng(3)
    lx, ly, lz, lt = ext
    ph = rng.uniform(-0.8, 0.8, size=(4, lt, lz, ly, lx, 2))
    U = np.zeros((4, lt, lz, ly, lx, 3, 3), complex)
    U[..., 0, 0] = np.exp(1j * ph[..., 0])
    U[..., 1, 1] = np.exp(1j * ph[..., 1])
    U[..., 2, 2] = np.exp(-1j * (ph[..., 0] + ph[..., 1]))
    D = O.divergence(U)
    Dp = O.ifft4(O.fft4(D) * O.fa_filter(ext, 0.08)[..., None, None])
    want = np.zeros((lt, lz, ly, lx, 3, 3), complex)
    for i in range(3):
        want[..., i, i] = np.exp(1j * Dp[..., i, i].imag)
    with lgf.Lattice(ext, "fp64", exact_exp=True) as lat:
        lat.set_links(U)
        lat.step(0.08)
        g = lat.get_gauge()
    assert np.max(np.abs(g - want)) < 1e-13


def test_trajectory_50_fp64():
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=0)
    ref = O.fix(U, tol=0.0, max_iter=50, track_G=False, exact_exp=True)
    with lgf.Lattice(ext, "fp64", exact_exp=True) as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(51)
        it, F, th, conv = lat.fix(0.0, 50, 0.08)
    assert it == 50
    for k in range(51):
        assert rel(Fh[k], ref["F"][k]) < 1e-11, k
        assert rel(Th[k], ref["theta"][k]) < 1e-11, k


@pytest.mark.parametrize("alpha", [0.08, 0.1])
def test_iterations_to_threshold_and_transform(alpha):
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=2)
    ref = O.fix(U, alpha=alpha, tol=1e-12, max_iter=3000, track_G=False, exact_exp=True)
    with lgf.Lattice(ext, "fp64", track_G=True, exact_exp=True) as lat:
        lat.set_links(U)
        it, F, th, conv = lat.fix(1e-12, 3000, alpha)
        G = lat.get_transform()
        U1 = lat.get_links()
    assert conv == ref["converged"] and conv
    assert abs(it - ref["iters"]) <= max(1, 0.02 * ref["iters"])
    assert abs(F - ref["F"][-1]) < 1e-10
    assert np.max(np.abs(O.apply_gauge(U, G) - U1)) < 1e-11
    assert abs(O.plaquette(U1) - O.plaquette(U)) < 1e-12


def test_fp32_step_and_mixed_to_1e15():
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=1)
    Uo, go = O.fa_step(U, 0.08, exact_exp=True)
    with lgf.Lattice(ext, "fp32", store12=True, exact_exp=True) as lat:
        lat.set_links(U)
        lat.step(0.08)
        g = lat.get_gauge()
        U1 = lat.get_links()
    assert np.max(np.abs(g - go)) < 2e-5
    assert np.max(np.abs(U1 - Uo)) < 2e-5
    ref = O.fix(U, tol=1e-15, max_iter=6000, track_G=False, exact_exp=True)
    with lgf.Lattice(ext, "mixed", store12=True, track_G=True, exact_exp=True) as lat:
        lat.set_links(U)
        it, F, th, conv = lat.fix(1e-15, 6000, 0.08)
        U1 = lat.get_links()
        G = lat.get_transform()
    assert conv and th < 1e-15
    assert abs(F - ref["F"][-1]) < 1e-10
    assert abs(it - ref["iters"]) <= max(1, 0.02 * ref["iters"])
    assert np.max(np.abs(O.apply_gauge(U, G) - U1)) < 1e-11
