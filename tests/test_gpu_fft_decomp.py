"""The 1D x 4 and 3D + 1D decompositions of the 4D transform
(lgf_set_fft_decomposition) against the FP64 CPU oracle.

Sec. 3.2 of the paper compares the three decompositions for speed; they
compute the same transform, so every one of them must reproduce the oracle's
step to rounding, and a whole trajectory to the parity tolerances.
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


EXTENTS = [(2, 2, 2, 2), (4, 4, 4, 4), (8, 8, 8, 8), (3, 4, 6, 9), (12, 6, 4, 8), (6, 12, 9, 3), (16, 8, 16, 4)]


@pytest.mark.parametrize("decomp", ["1d4", "3d1d"])
@pytest.mark.parametrize("ext", EXTENTS)
def test_one_step_parity_fp64(decomp, ext):
    U = fields.random_links(ext, eps=0.8, seed=7)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_fft_decomposition(decomp)
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


@pytest.mark.parametrize("decomp", ["1d4", "3d1d"])
def test_step_fp32_12real_and_exact_exp(decomp):
    ext = (8, 4, 6, 8)
    U = fields.random_links(ext, eps=0.9, seed=3)
    Uo, go = O.fa_step(U, 0.08)
    with lgf.Lattice(ext, "fp32", store12=True) as lat:
        lat.set_fft_decomposition(decomp)
        lat.set_links(U)
        lat.step(0.08)
        assert np.max(np.abs(lat.get_gauge() - go)) < 2e-5
        assert np.max(np.abs(lat.get_links() - Uo)) < 2e-5
    Uo, go = O.fa_step(U, 0.08, exact_exp=True)
    with lgf.Lattice(ext, "fp64", store12=True, exact_exp=True) as lat:
        lat.set_fft_decomposition(decomp)
        lat.set_links(U)
        lat.step(0.08)
        assert np.max(np.abs(lat.get_gauge() - go)) < 1e-12


@pytest.mark.parametrize("decomp", ["1d4", "3d1d"])
def test_trajectory_50_and_transform(decomp):
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=0)
    ref = O.fix(U, tol=0.0, max_iter=50, track_G=True)
    with lgf.Lattice(ext, "fp64", track_G=True) as lat:
        lat.set_fft_decomposition(decomp)
        lat.set_links(U)
        Fh, Th = lat.set_trace(51)
        it, F, th, conv = lat.fix(0.0, 50, 0.08)
        G = lat.get_transform()
    assert it == 50
    for k in range(51):
        assert rel(Fh[k], ref["F"][k]) < 1e-11, k
        assert rel(Th[k], ref["theta"][k]) < 1e-11, k
    assert np.max(np.abs(G - ref["G"])) < 1e-10


def test_switching_decomposition_between_fixes_and_mixed_mode():
    """The loop graph is rebuilt when the decomposition changes; a mixed fix
    runs both phases with the chosen decomposition."""
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=0.7, seed=4)
    ref = O.fix(U, tol=1e-12, max_iter=3000, track_G=False)
    out = {}
    with lgf.Lattice(ext, "fp64") as lat:
        for d in ("2d2d", "1d4", "3d1d", "2d2d"):
            lat.set_fft_decomposition(d)
            lat.set_links(U)
            out[d] = lat.fix(1e-12, 3000, 0.08)
            assert abs(out[d][0] - ref["iters"]) <= max(1, 0.02 * ref["iters"])
            assert abs(out[d][1] - ref["F"][-1]) < 1e-10
    with lgf.Lattice(ext, "mixed", store12=True, track_G=True) as lat:
        lat.set_fft_decomposition("1d4")
        lat.set_links(U)
        it, F, th, conv = lat.fix(1e-15, 6000, 0.08)
        assert conv and lat.phase == 64 and abs(F - ref["F"][-1]) < 1e-10


def test_timing_categories_cover_all_passes():
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=0.7, seed=4)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_fft_decomposition("1d4")
        lat.set_links(U)
        lat.set_timing(True)
        for _ in range(4):
            lat.step(0.08)
        ms, steps = lat.get_timing()
    assert steps == 4 and all(t > 0 for t in ms[:5])


def test_unsupported_combinations():
    with lgf.Lattice((32, 32, 32, 32), "fp64") as lat:
        with pytest.raises(lgf.LgfError) as e:
            lat.set_fft_decomposition("3d1d")   # a 32^3 FP64 slab is 540 KB
        assert e.value.status == lgf.LGF_E_UNSUPPORTED
        lat.set_fft_decomposition("1d4")


@pytest.mark.parametrize("decomp", ["1d4", "3d1d"])
def test_learned_multiplier_in_the_filter_pass(decomp):
    """With LGF_LEARNED the t pass of 1D x 4 and 3D + 1D applies the network's
    multiplier exactly where pass B of 2D + 2D does: the same trajectory up to
    the transforms' rounding, and the same fallbacks."""
    from paper_1206_0675_gb300.preconditioner import DEFAULT_WEIGHTS
    weights = np.load(DEFAULT_WEIGHTS)
    ext = (8, 8, 8, 8)
    U = fields.random_links(ext, eps=1.0, seed=21)
    runs = {}
    for d in ("2d2d", decomp):
        with lgf.Lattice(ext, "fp64", learned=True) as lat:
            lat.load_preconditioner(weights)
            lat.set_fft_decomposition(d)
            lat.set_links(U)
            Fh, Th = lat.set_trace(41)
            lat.fix(0.0, 40, 0.08)
            runs[d] = (Fh.copy(), Th.copy(), lat.fallbacks())
    (F0, T0, n0), (F1, T1, n1) = runs["2d2d"], runs[decomp]
    assert n0 == n1
    assert np.allclose(F1, F0, rtol=1e-10, atol=0)
    assert np.allclose(T1, T0, rtol=1e-8, atol=0)


@pytest.mark.parametrize("prec,store12", [("fp64", False), ("mixed", True)])
def test_autotune_keeps_results_and_reports(prec, store12):
    """The autotuner picks the fastest plan or decomposition; the step is
    the same transform whichever it picks."""
    ext = (8, 12, 8, 6)
    U = fields.random_links(ext, eps=0.8, seed=2)
    with lgf.Lattice(ext, prec, store12=store12, track_G=True) as lat:
        lat.set_links(U)
        F0, th0 = lat.measure()
        rep = lat.autotune()
        assert lat.measure() == (F0, th0)   # the current links were re-measured
        lanes = ["fp64"] + (["fp32"] if prec == "mixed" else [])
        for lane in lanes:
            c = rep[lane]["candidates"]
            assert {x["decomposition"] for x in c} == {"2d2d", "1d4", "3d1d"}
            assert all(x["ms"] > 0 for x in c)
            assert c[rep[lane]["chosen"]]["ms"] == min(x["ms"] for x in c)
        with pytest.raises(lgf.LgfError):
            lat.get_gauge()                 # g was overwritten by the trials
        if prec == "fp64":
            lat.step(0.08)
            Uo, go = O.fa_step(U, 0.08)
            assert np.max(np.abs(lat.get_gauge() - go)) < 1e-12
            assert np.max(np.abs(lat.get_links() - Uo)) < 1e-12
        else:
            ref = O.fix(U, tol=1e-15, max_iter=6000, track_G=False)
            it, F, th, conv = lat.fix(1e-15, 6000, 0.08)
            assert conv and abs(F - ref["F"][-1]) < 1e-10


def test_autotune_cache_file_reuses_the_choice(tmp_path, monkeypatch):
    """With LGF_AUTOTUNE_CACHE set, the first tuning is recorded and a later
    handle of the same shape applies it without timing."""
    path = tmp_path / "tune.cache"
    monkeypatch.setenv("LGF_AUTOTUNE_CACHE", str(path))
    ext = (6, 8, 12, 4)
    U = fields.random_links(ext, eps=0.6, seed=9)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        first = lat.autotune()["fp64"]
    assert not first["cached"]
    chosen = first["candidates"][first["chosen"]]
    lines = path.read_text().splitlines()
    assert any(l.startswith("single,6,8,12,4,fp64,rows=3,learned=0,") for l in lines)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        again = lat.autotune()["fp64"]
        assert again["cached"]
        c = again["candidates"][0]
        for k in ("decomposition", "fields_per_cta_xy", "x_columns_zt", "threads"):
            assert c[k] == chosen[k]
        lat.step(0.08)
        Uo, _ = O.fa_step(U, 0.08)
        assert np.max(np.abs(lat.get_links() - Uo)) < 1e-12
