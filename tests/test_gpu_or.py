"""Overrelaxation gauge fixing on the GPU (liblgf.so through its C-ABI)
against the overrelaxation oracle (oracle/lgf_or_oracle.py).

Both sides run on the same seeded synthetic fields.  Tolerances, as for the
Fourier-accelerated path:

* FP64, one sweep from identical links: links to 1e-12, F and theta to 1e-12
  relative (the kernel forms rows 1-2 of each product and rebuilds row 3,
  the oracle multiplies full matrices: the two differ by rounding).
* FP64 trajectories: F and theta within 1e-11 relative per sweep over the
  first 50 sweeps; sweeps to threshold within 2%; final F within 1e-10.
* FP32: F and theta within 1e-5 relative over the first 50 sweeps.
"""

import numpy as np
import pytest

from oracle import lgf_oracle as O
from oracle import lgf_or_oracle as R
from paper_1206_0675_gb300 import fields
from paper_1206_0675_gb300 import lgf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lgf.load_library()  # fails loudly when liblgf.so is missing


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


EXTENTS_EVEN = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (6, 4, 8, 2), (8, 8, 8, 8)]


# ---------------------------------------------------------------------------
# one sweep
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ext", EXTENTS_EVEN)
@pytest.mark.parametrize("store12", [False, True])
@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_one_sweep_parity_fp64(ext, store12, omega):
    U = fields.random_links(ext, eps=0.8, seed=4)
    with lgf.Lattice(ext, "fp64", store12=store12) as lat:
        lat.set_links(U)
        lat.or_sweep(omega, 1)
        F, th = lat.measure()
        U1 = lat.get_links()
    Uo, _ = R.or_sweep(U, omega)
    Fo, tho, _ = O.measure(Uo)
    assert np.max(np.abs(U1 - Uo)) < 1e-12
    assert rel(F, Fo) < 1e-12
    assert rel(th, tho) < 1e-12


@pytest.mark.parametrize("ext", [(4, 4, 4, 4), (4, 6, 2, 8)])
@pytest.mark.parametrize("store12", [False, True])
def test_one_sweep_parity_fp32(ext, store12):
    U = fields.random_links(ext, eps=0.8, seed=5)
    with lgf.Lattice(ext, "fp32", store12=store12) as lat:
        lat.set_links(U)
        lat.or_sweep(1.7, 1)
        F, th = lat.measure()
        U1 = lat.get_links()
    Uo, _ = R.or_sweep(U, 1.7)
    Fo, tho, _ = O.measure(Uo)
    assert np.max(np.abs(U1 - Uo)) < 3e-6
    assert abs(F - Fo) < 1e-6
    assert rel(th, tho) < 1e-5


def test_half_sweeps_touch_one_colour_each():
    """After the even colour only, the odd sites' local maximisation is untouched:
    one lgf_or_sweep equals the oracle's even half followed by its odd half, and
    two single sweeps equal one call with nsweeps = 2."""
    ext = (4, 4, 6, 2)
    U = fields.random_links(ext, eps=1.0, seed=6)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        lat.or_sweep(1.5, 1)
        lat.or_sweep(1.5, 1)
        Ua = lat.get_links()
        lat.set_links(U)
        lat.or_sweep(1.5, 2)
        Ub = lat.get_links()
    Uo = U
    for parity in (0, 1, 0, 1):
        Uo, _ = R.or_half_sweep(Uo, parity, 1.5)
    assert np.array_equal(Ua, Ub)
    assert np.max(np.abs(Ua - Uo)) < 1e-12


# ---------------------------------------------------------------------------
# trajectories and the loop
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("store12", [False, True])
def test_50_sweep_trajectory_fp64(store12):
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=3)
    ref = R.or_fix(U, omega=1.7, tol=0.0, max_sweeps=50, check_every=1, track_G=True)
    with lgf.Lattice(ext, "fp64", store12=store12, track_G=True) as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(51)
        n, F, th, conv = lat.or_fix(0.0, 50, 1.7, 1)
        G = lat.get_transform()
    assert n == 50 and not conv
    for k in range(51):
        assert rel(Fh[k], ref["F"][k]) < 1e-11, k
        assert rel(Th[k], ref["theta"][k]) < 1e-11, k
    assert np.max(np.abs(G - ref["G"])) < 1e-10


@pytest.mark.parametrize("store12", [False, True])
def test_50_sweep_trajectory_fp32(store12):
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=3)
    ref = R.or_fix(U, omega=1.7, tol=0.0, max_sweeps=50, check_every=1, track_G=False)
    with lgf.Lattice(ext, "fp32", store12=store12) as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(51)
        n, F, th, conv = lat.or_fix(0.0, 50, 1.7, 1)
    assert n == 50
    for k in range(51):
        assert rel(Fh[k], ref["F"][k]) < 1e-5, k
        assert rel(Th[k], ref["theta"][k]) < 1e-5, k


@pytest.fixture(scope="module")
def oracle_fix_8x4():
    U = fields.random_links((8, 8, 8, 8), eps=0.5, seed=0)
    return U, R.or_fix(U, omega=1.7, tol=1e-12, max_sweeps=3000, check_every=1, track_G=False)


def test_sweeps_to_threshold_fp64(oracle_fix_8x4):
    U, ref = oracle_fix_8x4
    with lgf.Lattice((8, 8, 8, 8), "fp64") as lat:
        lat.set_links(U)
        n, F, th, conv = lat.or_fix(1e-12, 3000, 1.7, 1)
    assert conv and th < 1e-12
    assert abs(n - ref["sweeps"]) <= 0.02 * ref["sweeps"]
    assert abs(F - ref["F"][-1]) < 1e-10


def test_check_every_counts_whole_groups(oracle_fix_8x4):
    """Measuring every 5 sweeps stops at the first multiple of 5 at or past the
    oracle's stopping sweep (the same trajectory, measured less often)."""
    U, ref = oracle_fix_8x4
    with lgf.Lattice((8, 8, 8, 8), "fp64") as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(3001)
        n, F, th, conv = lat.or_fix(1e-12, 3000, 1.7, 5)
    assert conv and n % 5 == 0
    expect = 5 * -(-ref["sweeps"] // 5)
    assert abs(n - expect) <= max(5, 0.02 * expect)
    # the trace holds the measured counts only: entry 5 k after 5 k sweeps
    for k in range(5, min(n, 50) + 1, 5):
        assert rel(Th[k], ref["theta"][k]) < 1e-11


def test_mixed_precision_reaches_threshold_and_keeps_invariants(oracle_fix_8x4):
    U, ref = oracle_fix_8x4
    with lgf.Lattice((8, 8, 8, 8), "mixed") as lat:
        lat.set_links(U)
        n, F, th, conv = lat.or_fix(1e-12, 3000, 1.7, 1)
        assert lat.phase == 64  # finished in FP64
        U1 = lat.get_links()
    assert conv and th < 1e-12
    assert abs(n - ref["sweeps"]) <= max(2, 0.02 * ref["sweeps"])
    assert abs(F - ref["F"][-1]) < 1e-10
    assert abs(O.plaquette(U1) - O.plaquette(U)) < 1e-12
    assert np.max(np.abs(O.polyakov_loops(U1) - O.polyakov_loops(U))) < 1e-12
    assert O.unitarity_defect(U1) < 1e-13


def test_pure_gauge_field_goes_to_F_equal_one():
    ext = (4, 4, 4, 4)
    U = fields.pure_gauge_links(ext, seed=7)
    with lgf.Lattice(ext, "fp64", track_G=True) as lat:
        lat.set_links(U)
        n, F, th, conv = lat.or_fix(1e-24, 2000, 1.7, 2)
        U1 = lat.get_links()
    assert conv
    assert abs(F - 1.0) < 1e-13
    # every link is the identity up to one global rotation C U C^dag = 1
    assert np.max(np.abs(U1 - np.eye(3))) < 1e-10


def test_transform_reproduces_the_links():
    ext = (4, 6, 2, 8)
    U = fields.random_links(ext, eps=0.9, seed=8)
    with lgf.Lattice(ext, "fp64", track_G=True) as lat:
        lat.set_links(U)
        lat.or_sweep(1.7, 20)
        U1 = lat.get_links()
        G = lat.get_transform()
    assert np.max(np.abs(O.apply_gauge(U, G) - U1)) < 1e-12


def test_fa_and_or_share_the_handle():
    """A Fourier-accelerated step, then overrelaxation sweeps, then a step,
    all on one handle: the same as the oracle's sequence."""
    ext = (4, 4, 4, 4)
    U = fields.random_links(ext, eps=0.8, seed=9)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        lat.step(0.08)
        lat.or_sweep(1.7, 3)
        with pytest.raises(lgf.LgfError):
            lat.get_gauge()  # no single g describes the sweeps
        lat.step(0.08)
        F, th = lat.measure()
        U1 = lat.get_links()
    Uo, _ = O.fa_step(U, 0.08)
    for _ in range(3):
        Uo, _ = R.or_sweep(Uo, 1.7)
    Uo, _ = O.fa_step(Uo, 0.08)
    Fo, tho, _ = O.measure(Uo)
    assert np.max(np.abs(U1 - Uo)) < 1e-12
    assert rel(F, Fo) < 1e-12 and rel(th, tho) < 1e-11


# ---------------------------------------------------------------------------
# the 32^4 workload (whole lattice, one sweep; the launch shape the bench times)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def sweep_32x4():
    U = fields.random_links((32, 32, 32, 32), eps=1.0, seed=0)
    Uo, _ = R.or_sweep(U, 1.7)
    Fo, tho, _ = O.measure(Uo)
    return U, Uo, Fo, tho


def test_full_size_32x4_one_sweep_fp64(sweep_32x4):
    U, Uo, Fo, tho = sweep_32x4
    with lgf.Lattice((32, 32, 32, 32), "fp64") as lat:
        lat.set_links(U)
        lat.or_sweep(1.7, 1)
        F, th = lat.measure()
        U1 = lat.get_links()
    assert rel(F, Fo) < 1e-12
    assert rel(th, tho) < 1e-12
    assert np.max(np.abs(U1 - Uo)) < 1e-12


def test_full_size_32x4_one_sweep_fp32_12real(sweep_32x4):
    U, Uo, Fo, tho = sweep_32x4
    with lgf.Lattice((32, 32, 32, 32), "fp32", store12=True) as lat:
        lat.set_links(U)
        lat.or_sweep(1.7, 1)
        F, th = lat.measure()
        U1 = lat.get_links()
    assert abs(F - Fo) < 1e-6
    assert rel(th, tho) < 1e-5
    # The SU(2) maximiser r = b~/|b| passes the FP32 rounding of the local
    # field on amplified by |w|/|b|, large where a subgroup block is small: over
    # the 4 x 2^20 links of this field the largest entry error is 6.3e-6, about
    # a hundred FP32 units; bounded by the 1e-5 relative FP32 tolerance of the FP32 paths.
    assert np.max(np.abs(U1 - Uo)) < 1e-5


# ---------------------------------------------------------------------------
# arguments the library refuses
# ---------------------------------------------------------------------------

def test_refusals():
    U = fields.random_links((4, 4, 4, 4), eps=0.5, seed=1)
    with lgf.Lattice((4, 4, 4, 4), "fp64") as lat:
        lat.set_links(U)
        for omega in (0.99, 2.0, float("nan")):
            with pytest.raises(lgf.LgfError) as e:
                lat.or_sweep(omega, 1)
            assert e.value.status == lgf.LGF_E_ARG
        with pytest.raises(lgf.LgfError) as e:
            lat.or_fix(1e-12, 10, 1.7, 0)
        assert e.value.status == lgf.LGF_E_ARG
    ext = (4, 3, 4, 4)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(fields.random_links(ext, eps=0.5, seed=1))
        with pytest.raises(lgf.LgfError) as e:
            lat.or_sweep(1.7, 1)
        assert e.value.status == lgf.LGF_E_UNSUPPORTED
    with lgf.Lattice((4, 4, 4, 4), "fp64", learned=True) as lat:
        lat.set_links(U)
        with pytest.raises(lgf.LgfError) as e:
            lat.or_fix(1e-12, 10, 1.7, 1)
        assert e.value.status == lgf.LGF_E_UNSUPPORTED
