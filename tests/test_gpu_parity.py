"""GPU path (liblgf.so through its C-ABI) against the FP64 CPU oracle.

Every comparison runs both sides on the same seeded synthetic field
(``paper_1206_0675_gb300.fields``).  Tolerances:

* FP64, one step from identical links: F, theta, Delta, g and U to ~1e-12.
* FP64 trajectories: per-iteration F and theta within 1e-11 relative over
  the first 50 iterations; iterations to threshold within 2%; final F within
  1e-10.
* FP32 trajectories: per-iteration F and theta within 1e-5 relative over the
  first 50 iterations.
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
    lgf.load_library()  # fails loudly when liblgf.so is missing


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def oracle_trajectory(U, n, alpha=0.08, K=None):
    return O.fix(U, alpha=alpha, tol=0.0, max_iter=n, K=K, track_G=False)


EXTENTS_SMALL = [(2, 2, 2, 2), (4, 4, 4, 4), (8, 8, 8, 8), (3, 4, 6, 9), (2, 3, 4, 6), (12, 6, 4, 8), (6, 12, 9, 3)]


# ---------------------------------------------------------------------------
# measurement (kernel k2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ext", EXTENTS_SMALL)
@pytest.mark.parametrize("store12", [False, True])
def test_measure_parity_fp64(ext, store12):
    U = fields.random_links(ext, eps=0.7, seed=1)
    with lgf.Lattice(ext, "fp64", store12=store12) as lat:
        lat.set_links(U)
        F, th = lat.measure()
        D = lat.get_divergence()
    Fo, tho, Do = O.measure(U)
    assert rel(F, Fo) < 1e-14
    assert rel(th, tho) < 1e-13
    assert np.max(np.abs(D - Do)) < 1e-13


@pytest.mark.parametrize("ext", [(4, 4, 4, 4), (3, 4, 6, 9)])
@pytest.mark.parametrize("store12", [False, True])
def test_measure_parity_fp32(ext, store12):
    U = fields.random_links(ext, eps=0.7, seed=2)
    with lgf.Lattice(ext, "fp32", store12=store12) as lat:
        lat.set_links(U)
        F, th = lat.measure()
        D = lat.get_divergence()
    Fo, tho, Do = O.measure(U)
    # F is a mean of O(1) traces (here close to 0 for a gauge-rotated field),
    # so its FP32 error is absolute
    assert abs(F - Fo) < 1e-6
    assert rel(th, tho) < 1e-5
    assert np.max(np.abs(D - Do)) < 2e-6


# ---------------------------------------------------------------------------
# 4D DFT passes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ext", EXTENTS_SMALL + [(16, 16, 16, 16), (32, 8, 16, 4), (24, 18, 12, 27)])
def test_fft4_against_numpy_and_inverse(ext):
    lx, ly, lz, lt = ext
    rng = np.random.default_rng(3)
    f = rng.standard_normal((4, lt, lz, ly, lx)) + 1j * rng.standard_normal((4, lt, lz, ly, lx))
    ref = np.fft.fftn(f, axes=(1, 2, 3, 4))
    with lgf.Lattice(ext, "fp64") as lat:
        fh = lat.fft4(f, -1)
        back = lat.fft4(fh, +1)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(fh - ref)) < 1e-14 * scale * np.log2(f[0].size + 1)
    V = f[0].size
    assert np.max(np.abs(back / V - f)) < 1e-13


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_fft4_against_cufft_32x4(prec, tol):
    """Cross-check at the full 32^4 size against cuFFT (through torch.fft on
    the device): the library's own passes must give the same 4D DFT."""
    import torch
    ext = (32, 32, 32, 32)
    rng = np.random.default_rng(31)
    f = rng.standard_normal((4, 32, 32, 32, 32)) + 1j * rng.standard_normal((4, 32, 32, 32, 32))
    with lgf.Lattice(ext, prec) as lat:
        ours = lat.fft4(f, -1)
    ref = torch.fft.fftn(torch.from_numpy(f).cuda(), dim=(1, 2, 3, 4)).cpu().numpy()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(ours - ref)) < tol * scale


def test_fft4_defining_sum_tiny():
    """Against the defining sum, written out for a 2x3x2x3 lattice."""
    ext = (2, 3, 2, 3)
    lx, ly, lz, lt = ext
    rng = np.random.default_rng(4)
    f = rng.standard_normal((4, lt, lz, ly, lx)) + 1j * rng.standard_normal((4, lt, lz, ly, lx))
    ref = np.zeros_like(f)
    for kt in range(lt):
        for kz in range(lz):
            for ky in range(ly):
                for kx in range(lx):
                    t, z, y, x = np.meshgrid(range(lt), range(lz), range(ly), range(lx), indexing="ij")
                    ph = np.exp(-2j * np.pi * (kx * x / lx + ky * y / ly + kz * z / lz + kt * t / lt))
                    ref[:, kt, kz, ky, kx] = np.sum(f * ph, axis=(1, 2, 3, 4))
    with lgf.Lattice(ext, "fp64") as lat:
        fh = lat.fft4(f, -1)
    assert np.max(np.abs(fh - ref)) < 1e-13


def test_fft4_fp32():
    ext = (8, 12, 6, 16)
    lx, ly, lz, lt = ext
    rng = np.random.default_rng(5)
    f = rng.standard_normal((4, lt, lz, ly, lx)) + 1j * rng.standard_normal((4, lt, lz, ly, lx))
    ref = np.fft.fftn(f, axes=(1, 2, 3, 4))
    with lgf.Lattice(ext, "fp32") as lat:
        fh = lat.fft4(f, -1)
    assert np.max(np.abs(fh - ref)) < 2e-6 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# one Algorithm-1 step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ext", EXTENTS_SMALL)
@pytest.mark.parametrize("store12", [False, True])
def test_one_step_parity_fp64(ext, store12):
    U = fields.random_links(ext, eps=0.8, seed=7)
    with lgf.Lattice(ext, "fp64", store12=store12) as lat:
        lat.set_links(U)
        lat.step(0.08)
        F, th = lat.measure()
        g = lat.get_gauge()
        U1 = lat.get_links()
    Uo, go = O.fa_step(U, 0.08)
    Fo, tho, _ = O.measure(Uo)
    assert np.max(np.abs(g - go)) < 1e-12
    assert np.max(np.abs(U1 - Uo)) < 1e-12
    assert rel(F, Fo) < 1e-13
    assert rel(th, tho) < 1e-11
    # the FP64 reunitarisation leaves g unitary to rounding
    assert O.unitarity_defect(g) < 4e-15


@pytest.mark.parametrize("ext", [(96, 2, 3, 2), (2, 2, 2, 128), (4, 3, 128, 2), (96, 96, 2, 2)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_extreme_extents_one_step(ext, prec, tol):
    """The largest accepted extents: 96 along x and y, 128 along z and t.  A
    96 x 96 (x,y) plane holds one field in shared memory but not four, so
    that lattice takes the unfused inverse pass and the separate g kernel."""
    U = fields.random_links(ext, eps=0.8, seed=17)
    with lgf.Lattice(ext, prec) as lat:
        lat.set_links(U)
        lat.step(0.08)
        g = lat.get_gauge()
        U1 = lat.get_links()
    Uo, go = O.fa_step(U, 0.08)
    assert np.max(np.abs(g - go)) < tol
    assert np.max(np.abs(U1 - Uo)) < tol


def test_one_step_plain_sd_fp64():
    ext = (4, 6, 4, 8)
    U = fields.random_links(ext, eps=0.8, seed=8)
    with lgf.Lattice(ext, "fp64", plain_sd=True) as lat:
        lat.set_links(U)
        lat.step(0.05)
        U1 = lat.get_links()
    Uo, _ = O.fa_step(U, 0.05, K=O.sd_filter(ext, 0.05))
    assert np.max(np.abs(U1 - Uo)) < 1e-12


# ---------------------------------------------------------------------------
# trajectories and iterations to threshold
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ext,eps,seed", [((8, 8, 8, 8), 1.0, 0), ((6, 4, 12, 9), 0.9, 3)])
def test_trajectory_50_fp64(ext, eps, seed):
    U = fields.random_links(ext, eps=eps, seed=seed)
    ref = oracle_trajectory(U, 50)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(51)
        it, F, th, conv = lat.fix(0.0, 50, 0.08)
    assert it == 50
    for k in range(51):
        assert rel(Fh[k], ref["F"][k]) < 1e-11, k
        assert rel(Th[k], ref["theta"][k]) < 1e-11, k


@pytest.mark.parametrize("store12", [False, True])
def test_trajectory_50_fp32(store12):
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=0)
    ref = oracle_trajectory(U, 50)
    with lgf.Lattice(ext, "fp32", store12=store12) as lat:
        lat.set_links(U)
        Fh, Th = lat.set_trace(51)
        it, F, th, conv = lat.fix(0.0, 50, 0.08)
    assert it == 50
    for k in range(51):
        assert rel(Fh[k], ref["F"][k]) < 1e-5, k
        assert rel(Th[k], ref["theta"][k]) < 1e-5, k


@pytest.mark.parametrize("eps", [0.5, 1.0])
def test_iterations_to_threshold_fp64_8x4(eps):
    """The 8^4, alpha = 0.08 workload, stopped at theta < 1e-12 or 3000 iterations."""
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=eps, seed=0)
    ref = O.fix(U, tol=1e-12, max_iter=3000, track_G=False)
    with lgf.Lattice(ext, "fp64", track_G=True) as lat:
        lat.set_links(U)
        it, F, th, conv = lat.fix(1e-12, 3000, 0.08)
        G = lat.get_transform()
        U1 = lat.get_links()
    assert conv == ref["converged"]
    assert abs(it - ref["iters"]) <= max(1, 0.02 * ref["iters"])
    assert abs(F - ref["F"][-1]) < 1e-10
    # the transform reproduces the final links and gauge invariants are kept
    assert np.max(np.abs(O.apply_gauge(U, G) - U1)) < 1e-11
    assert abs(O.plaquette(U1) - O.plaquette(U)) < 1e-12
    # No step of Algorithm 1 reunitarises the links, so rounding drift
    # accumulates over ~1000 updates: the oracle itself ends this run at a
    # defect of 9.5e-13; the GPU path (row 3 rebuilt from rows 1-2) at 1.1e-13.
    assert O.unitarity_defect(U1) < 5e-13


def test_fix_to_1e15_fp64_and_transform():
    ext = (4, 6, 8, 6)
    U = fields.random_links(ext, eps=0.8, seed=5)
    ref = O.fix(U, tol=1e-15, max_iter=5000, track_G=True)
    with lgf.Lattice(ext, "fp64", track_G=True) as lat:
        lat.set_links(U)
        it, F, th, conv = lat.fix(1e-15, 5000, 0.08)
        G = lat.get_transform()
    assert conv and th < 1e-15
    assert abs(it - ref["iters"]) <= max(1, 0.02 * ref["iters"])
    assert abs(F - ref["F"][-1]) < 1e-10
    assert np.max(np.abs(G - ref["G"])) < 1e-9


# ---------------------------------------------------------------------------
# mixed precision
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("store12,switch", [(True, None), (False, None), (True, 1e-10)])
def test_mixed_reaches_1e15_and_keeps_gauge_invariants(store12, switch):
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=1)
    ref = O.fix(U, tol=1e-15, max_iter=6000, track_G=False)
    with lgf.Lattice(ext, "mixed", store12=store12, track_G=True) as lat:
        if switch is not None:
            lat.set_switch_theta(switch)
        lat.set_links(U)
        assert lat.phase == 32
        Fh, Th = lat.set_trace(6001)
        it, F, th, conv = lat.fix(1e-15, 6000, 0.08)
        assert lat.phase == 64
        U1 = lat.get_links()
        G = lat.get_transform()
    assert conv and th < 1e-15
    assert abs(F - ref["F"][-1]) < 1e-10
    assert abs(it - ref["iters"]) <= max(1, 0.02 * ref["iters"])
    assert abs(O.plaquette(U1) - O.plaquette(U)) < 1e-12
    assert np.max(np.abs(O.polyakov_loops(U1) - O.polyakov_loops(U))) < 1e-12
    assert np.max(np.abs(O.apply_gauge(U, G) - U1)) < 1e-11
    assert O.unitarity_defect(U1) < 5e-13
    Fo, tho, _ = O.measure(U1)
    assert rel(F, Fo) < 1e-13 and tho < 1e-15


def test_mixed_steps_switch_like_fix():
    """lgf_step on a mixed handle: a step taken from links whose theta is below
    the switch level runs in FP64, so stepping by hand gives the same result,
    bit for bit, as lgf_fix over the same number of updates."""
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=0.5, seed=0)
    n, switched_at = 0, None
    with lgf.Lattice(ext, "mixed", store12=True) as lat:
        lat.set_links(U)
        while n < 80:
            F, th = lat.measure()
            if th < 1e-13:
                break
            lat.step(0.08)
            n += 1
            assert lat.phase == (64 if th < 1e-9 else 32), (n, th)
            if lat.phase == 64 and switched_at is None:
                switched_at = n
        Fs, ths = lat.measure()
    assert switched_at is not None and switched_at < n
    with lgf.Lattice(ext, "mixed", store12=True) as lat:
        lat.set_links(U)
        it, F, th, conv = lat.fix(0.0, n, 0.08)
    assert it == n and F == Fs and th == ths


# ---------------------------------------------------------------------------
# degenerate inputs and errors
# ---------------------------------------------------------------------------

def test_identity_field_is_fixed_point():
    ext = (4, 4, 4, 4)
    U = O.identity_links(ext)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        F, th = lat.measure()
        assert F == 1.0 and th == 0.0
        it, F, th, conv = lat.fix(1e-15, 100, 0.08)
        assert it == 0 and conv
        lat.step(0.08)
        assert np.array_equal(lat.get_links(), U)
        assert np.array_equal(lat.get_gauge(), O.identity_sites(ext))


def test_pure_gauge_driven_to_unit_links():
    ext = (4, 4, 4, 4)
    U = fields.pure_gauge_links(ext, seed=3)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        it, F, th, conv = lat.fix(1e-26, 500, 0.08)
        U1 = lat.get_links()
    assert conv and F > 1 - 1e-13
    assert np.max(np.abs(U1 - np.eye(3))) < 1e-6


def test_rejects_non_su3_and_nan_links():
    ext = (2, 2, 2, 2)
    U = fields.random_links(ext, eps=0.5, seed=0)
    with lgf.Lattice(ext, "fp64") as lat:
        bad = U.copy()
        bad[1, 0, 1, 0, 1] *= 1.001
        with pytest.raises(lgf.LgfError) as e:
            lat.set_links(bad)
        assert e.value.status == lgf.LGF_E_ARG
        nan = U.copy()
        nan[0, 0, 0, 0, 0, 1, 2] = np.nan
        with pytest.raises(lgf.LgfError) as e:
            lat.set_links(nan)
        assert e.value.status == lgf.LGF_E_NONFINITE
        with pytest.raises(lgf.LgfError) as e:
            lat.get_transform()
        assert e.value.status == lgf.LGF_E_STATE
        lat.set_links(U)  # still usable after rejected inputs
        with pytest.raises(lgf.LgfError) as e:
            lat.get_transform()
        assert e.value.status == lgf.LGF_E_STATE
        it, F, th, conv = lat.fix(1e-30, 3, 0.08)
        assert it == 3 and not conv


def test_device_pointers_roundtrip():
    import torch
    ext = (4, 4, 6, 4)
    U = fields.random_links(ext, eps=0.6, seed=9)
    Ut = torch.from_numpy(U).cuda()
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(Ut)
        out = torch.empty_like(Ut)
        lat.get_links(out)
        torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), U)


# ---------------------------------------------------------------------------
# full-size case of the 32^4 workload (the launch configuration the bench times)
# ---------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("prec,store12,tol", [("fp64", False, 1e-12), ("fp32", True, 2e-5)])
def test_full_size_32x4_one_step(prec, store12, tol):
    ext = (32, 32, 32, 32)
    U = fields.random_links(ext, eps=1.0, seed=0)
    with lgf.Lattice(ext, prec, store12=store12) as lat:
        lat.set_links(U)
        F0, th0 = lat.measure()
        lat.step(0.08)
        F1, th1 = lat.measure()
        U1 = lat.get_links()
    Fo0, tho0, D = O.measure(U)
    Uo, _ = O.fa_step(U, 0.08, D=D)
    Fo1, tho1, _ = O.measure(Uo)
    assert rel(F0, Fo0) < (1e-13 if prec == "fp64" else 1e-6)
    assert rel(th0, tho0) < (1e-12 if prec == "fp64" else 1e-5)
    assert rel(F1, Fo1) < (1e-12 if prec == "fp64" else 1e-5)
    assert rel(th1, tho1) < (1e-11 if prec == "fp64" else 1e-5)
    # sampled sites: every link of 64 random sites
    rng = np.random.default_rng(0)
    idx = tuple(rng.integers(0, 32, size=(4, 64)))
    assert np.max(np.abs(U1[:, idx[0], idx[1], idx[2], idx[3]] - Uo[:, idx[0], idx[1], idx[2], idx[3]])) < tol


@pytest.fixture(scope="module")
def aniso_case():
    """The 48^3 x 96 workload (eps = 0.7, seed 0) and one oracle step from it."""
    ext = (48, 48, 48, 96)
    U = fields.random_links(ext, eps=0.7, seed=0)
    Fo0, tho0, D = O.measure(U)
    Uo, _ = O.fa_step(U, 0.08, D=D)
    Fo1, tho1, _ = O.measure(Uo)
    rng = np.random.default_rng(1)
    idx = (rng.integers(0, 96, 128), rng.integers(0, 48, 128), rng.integers(0, 48, 128), rng.integers(0, 48, 128))
    return ext, U, (Fo0, tho0, Fo1, tho1), idx, Uo[:, idx[0], idx[1], idx[2], idx[3]]


@pytest.mark.slow
@pytest.mark.parametrize("prec,store12", [("fp64", False), ("fp32", True)])
def test_anisotropic_48x3_96_one_step(aniso_case, prec, store12):
    """48^3 x 96: one step against the oracle, links of 128 sampled sites."""
    ext, U, (Fo0, tho0, Fo1, tho1), idx, Uo_s = aniso_case
    with lgf.Lattice(ext, prec, store12=store12) as lat:
        lat.set_links(U)
        F0, th0 = lat.measure()
        lat.step(0.08)
        F1, th1 = lat.measure()
        U1 = lat.get_links()
    f64 = prec == "fp64"
    assert abs(F0 - Fo0) < (1e-13 if f64 else 1e-6) * abs(Fo0)
    assert rel(th0, tho0) < (1e-12 if f64 else 1e-5)
    assert abs(F1 - Fo1) < (1e-13 if f64 else 1e-6) * abs(Fo1)
    assert rel(th1, tho1) < (1e-11 if f64 else 1e-5)
    assert np.max(np.abs(U1[:, idx[0], idx[1], idx[2], idx[3]] - Uo_s)) < (1e-12 if f64 else 2e-5)


# ---------------------------------------------------------------------------
# per-measurement trace flags and the sampled link defect
# ---------------------------------------------------------------------------

def test_trace_flags_and_defect_of_a_mixed_fix():
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=1)
    with lgf.Lattice(ext, "mixed", store12=True) as lat:
        lat.set_links(U)
        Fh, Th, Fl, Dh = lat.set_trace(6001, flags=True)
        it, F, th, conv = lat.fix(1e-15, 6000, 0.08)
        d_last, repairs = lat.link_defect()
    assert conv and repairs == 0
    n = it + 1
    fp64 = (Fl[1:n] & lgf.LGF_TRACE_FP64) != 0
    k = int(np.argmax(fp64)) + 1          # first update run in FP64
    assert fp64[k - 1:].all() and not fp64[:k - 1].any()
    # every FP32 measurement before the switch had theta >= 1e-9 (entry k - 1
    # holds the FP64 re-measurement of the links rebuilt at the switch, whose
    # theta differs from the FP32 one that triggered it by the FP32 error of G)
    assert np.all(Th[:k - 1] >= 1e-9) and Th[k - 1] < 1e-8
    assert not np.any(Fl[1:n] & (lgf.LGF_TRACE_LEARNED | lgf.LGF_TRACE_REDO | lgf.LGF_TRACE_REPAIRED))
    # FP32 links drift from SU(3) by compounded FP32 roundings (1.4e-5 after
    # this phase, below the FP32 bound 1e-4); the links rebuilt in FP64 at the
    # switch carry a few FP64 roundings
    assert 1e-7 < Dh[:k - 1].max() < 1e-4
    assert Dh[k - 1:n].max() < 1e-13 and d_last == Dh[n - 1]


def test_defect_guard_beyond_the_convergent_alpha():
    """alpha = 0.11 (alpha p2max = 1.76) lies past FA-SD's convergent range:
    on this 8^4 field theta stalls near 1.8 in the oracle and on the GPU
    alike.  No step of Algorithm 1 reunitarises the links; the GPU path
    rebuilds row 3 from rows 1-2 at every update, and far from the fixed
    point that compounds the rounding defect of rows 1-2 (7.7e-10 after 3000
    steps here, against 6e-13 in the oracle's full products).  The guard
    reunitarises the links when the sampled defect passes 1e-10; the
    trajectory still follows the oracle's."""
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=0.5, seed=0)
    ref = O.fix(U, alpha=0.11, tol=1e-12, max_iter=3000, track_G=False)
    assert not ref["converged"]
    runs = {}
    for bound in (0.0, 1e-10):
        with lgf.Lattice(ext, "fp64") as lat:
            lat.set_defect_bound(bound, 1e-4)
            lat.set_links(U)
            Fh, Th, Fl, Dh = lat.set_trace(3001, flags=True)
            it, F, th, conv = lat.fix(1e-12, 3000, 0.11)
            runs[bound] = (it, F, th, conv, lat.link_defect(), Fl.copy(), Dh.copy())
    it, F, th, conv, (d, rep), Fl, Dh = runs[0.0]
    assert it == 3000 and not conv and rep == 0 and Dh.max() > 1e-10
    it, F, th, conv, (d, rep), Fl, Dh = runs[1e-10]
    assert it == 3000 and not conv and rep >= 1
    assert Dh.max() <= 1e-10 and np.count_nonzero(Fl & lgf.LGF_TRACE_REPAIRED) == rep
    assert rel(F, ref["F"][-1]) < 1e-9 and rel(th, ref["theta"][-1]) < 1e-9
