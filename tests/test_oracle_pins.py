"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each pin is chosen so that a plausible mistake in the oracle (a dropped
factor 1/2, a wrong sign of the step, a forward instead of backward
difference, a transposed momentum axis, a missing 1/V, a wrong p2max, a
non-SU(3) projection) fails at least one of them.  None of them re-types
the oracle's own formulas: they use closed forms derived from the
definitions, invariants, library routines (QR, numpy's FFT checked against
the defining DFT sum) and brute-force loops on tiny lattices.
"""

import itertools

import numpy as np
import pytest

from oracle import lgf_oracle as O
from paper_1206_0675_gb300 import fields

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------------------
# P1: identity field
# ---------------------------------------------------------------------------

def test_identity_field_is_exact_fixed_point():
    ext = (4, 3, 2, 6)
    U = O.identity_links(ext)
    F, th, D = O.measure(U)
    assert F == 1.0 and th == 0.0
    assert np.all(D == 0)
    U1, g = O.fa_step(U)
    assert np.array_equal(U1, U)
    assert np.array_equal(g, O.identity_sites(ext))


# ---------------------------------------------------------------------------
# P2: pure gauge driven back to F = 1
# ---------------------------------------------------------------------------

def test_pure_gauge_converges_to_unit_links():
    ext = (4, 4, 4, 4)
    U0 = fields.pure_gauge_links(ext, seed=3)
    h = fields.random_site_su3(ext, seed=3)  # the same stream: h used to build U0
    res = O.fix(U0, tol=1e-26, max_iter=400)
    assert res["converged"]
    assert res["F"][-1] > 1.0 - 1e-13
    assert np.max(np.abs(res["U"] - np.eye(3))) < 1e-6
    # U_final = G h h^dag(x+mu) G^dag(x+mu) = 1  =>  G(x) h(x) is the same matrix everywhere
    Gh = res["G"] @ h
    assert np.max(np.abs(Gh - Gh[0, 0, 0, 0])) < 1e-6


# ---------------------------------------------------------------------------
# P3: weak-field contraction factor (linearisation of Eq. (eq:gx))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ext", [(4, 4, 4, 4), (6, 4, 8, 4), (3, 4, 5, 6)])
def test_weak_field_contraction_factor(ext):
    """For U = exp(i eps a) with small eps, Delta^_{k+1}(p) = (1 - alpha p2max) Delta^_k(p)
    for every p != 0, so theta_{k+1}/theta_k = (1 - alpha p2max)^2 (+O(eps)).

    On a non-cubic lattice this fails if the filter's momentum axes are
    permuted or if p2max is not the largest eigenvalue of -d^2.
    """
    alpha = 0.08
    p2max = sum(4 * np.sin(np.pi * (L // 2) / L) ** 2 for L in ext)
    U = fields.random_links(ext, eps=1e-5, seed=11, gauge_rotate=False)
    _, th0, _ = O.measure(U)
    U1, _ = O.fa_step(U, alpha)
    _, th1, _ = O.measure(U1)
    expected = (1 - alpha * p2max) ** 2
    assert abs(th1 / th0 - expected) < 1e-3 * expected


def test_weak_field_factor_even_lattice_is_00784():
    # all-even extents: p2max = 16 and (1 - 0.08*16)^2 = 0.0784
    U = fields.random_links((4, 4, 4, 4), eps=1e-6, seed=1, gauge_rotate=False)
    _, th0, _ = O.measure(U)
    _, th1, _ = O.measure(O.fa_step(U, 0.08)[0])
    assert abs(th1 / th0 - 0.0784) < 1e-4


def test_weak_field_plain_sd_mode_by_mode():
    """Plain SD (filter = alpha): Delta^ contracts by (1 - alpha p2(k)) per mode."""
    ext = (4, 6, 4, 2)
    alpha = 0.08
    U = fields.random_links(ext, eps=1e-6, seed=5, gauge_rotate=False)
    D0 = O.divergence(U)
    U1, _ = O.fa_step(U, alpha, K=O.sd_filter(ext, alpha))
    D1 = O.divergence(U1)
    D0h = naive_dft4(D0)
    D1h = naive_dft4(D1)
    p2 = brute_p2(ext)
    pred = (1 - alpha * p2)[..., None, None] * D0h
    scale = np.max(np.abs(D0h))
    assert np.max(np.abs(D1h - pred)) < 1e-4 * scale


# ---------------------------------------------------------------------------
# P4: first-order ascent rate
# ---------------------------------------------------------------------------

def test_first_order_ascent_rate():
    """dF/dalpha at alpha = 0 equals (1/(12 V^2)) sum_k (p2max/p2(k)) ||Delta^(k)||_F^2.

    Derived from F = (1/12V) sum Re Tr(g U g^dag) with g = exp(X): dF = -(1/12V)
    sum_x Tr[X Delta_A] and Parseval.  Checks the sign of the step, the 1/2 in
    the exponent, the 1/V of the inverse transform and the filter.
    """
    ext = (3, 4, 2, 3)
    V = int(np.prod(ext))
    U = fields.random_links(ext, eps=0.4, seed=7)
    D = O.divergence(U)
    Dh = naive_dft4(D)
    p2 = brute_p2(ext)
    p2max = max(p2.ravel())
    w = np.zeros_like(p2)
    w[p2 > 0] = p2max / p2[p2 > 0]
    rate = np.sum(w[..., None, None] * np.abs(Dh) ** 2) / (12 * V * V)
    a = 1e-5
    Fp = O.functional_F(O.fa_step(U, a)[0])
    Fm = O.functional_F(O.fa_step(U, -a)[0])
    assert abs((Fp - Fm) / (2 * a) - rate) < 1e-7 * rate


def test_ascent_rate_plain_sd_equals_theta_over_16():
    """With the filter replaced by alpha (plain SD) the rate is theta/16 (theta paper-literal)."""
    ext = (4, 2, 3, 4)
    U = fields.random_links(ext, eps=0.6, seed=9)
    _, th, _ = O.measure(U)
    a = 1e-5
    Fp = O.functional_F(O.fa_step(U, a, K=O.sd_filter(ext, a))[0])
    Fm = O.functional_F(O.fa_step(U, -a, K=O.sd_filter(ext, -a))[0])
    assert abs((Fp - Fm) / (2 * a) - th / 16) < 1e-7 * th


# ---------------------------------------------------------------------------
# P5 / P6: gauge invariants, covariance, monotonicity, unitarity
# ---------------------------------------------------------------------------

def test_gauge_invariants_monotone_F_and_unitarity():
    ext = (4, 4, 4, 6)
    U = fields.random_links(ext, eps=0.5, seed=2)
    plaq0 = O.plaquette(U)
    poly0 = O.polyakov_loops(U)
    F_prev = O.functional_F(U)
    for _ in range(6):
        U, g = O.fa_step(U)
        assert abs(O.plaquette(U) - plaq0) < 1e-12
        assert np.max(np.abs(O.polyakov_loops(U) - poly0)) < 1e-12
        assert O.unitarity_defect(U) < 1e-13
        assert O.unitarity_defect(g) < 1e-13
        F = O.functional_F(U)
        assert F >= F_prev
        F_prev = F


def test_global_colour_rotation_covariance_of_measurement():
    """U -> C U C^dag (constant C) maps Delta -> C Delta C^dag and leaves F, theta unchanged.

    The step itself is covariant only to first order: Gram-Schmidt on the
    rows of 1 + Delta' does not commute with conjugation by C, so trajectories
    of rotated fields agree to O(|Delta'|^2) per step, not exactly.
    """
    ext = (4, 2, 4, 2)
    U = fields.random_links(ext, eps=0.7, seed=4)
    C = fields.haar_su3((), np.random.Generator(np.random.Philox(key=99)))
    Ur = C @ U @ np.conj(C.T)
    Fa, tha, Da = O.measure(U)
    Fb, thb, Db = O.measure(Ur)
    assert abs(Fa - Fb) < 1e-14 and abs(tha - thb) < 1e-13 * tha
    assert np.max(np.abs(C @ Da @ np.conj(C.T) - Db)) < 1e-13
    # first-order covariance of the step: weak field, tiny alpha
    Uw = fields.random_links(ext, eps=1e-4, seed=4, gauge_rotate=False)
    a = O.fix(Uw, tol=0.0, max_iter=3, track_G=False)
    b = O.fix(C @ Uw @ np.conj(C.T), tol=0.0, max_iter=3, track_G=False)
    assert np.allclose(a["theta"], b["theta"], rtol=1e-3, atol=0)  # deviation is O(eps)


def test_transform_reproduces_links():
    """G accumulated by fix() satisfies U_final = G U_0 G^dag(x+mu^)."""
    ext = (2, 4, 2, 4)
    U0 = fields.random_links(ext, eps=0.5, seed=8)
    res = O.fix(U0, tol=0.0, max_iter=7)
    rebuilt = O.apply_gauge(U0, res["G"])
    assert np.max(np.abs(rebuilt - res["U"])) < 1e-13


# ---------------------------------------------------------------------------
# P7: FFT and filter
# ---------------------------------------------------------------------------

def naive_dft4(f):
    """Defining sum f^(k) = sum_x f(x) exp(-2 pi i sum_mu k_mu x_mu / L_mu) over site axes 0..3."""
    shape = f.shape[:4]
    out = f.astype(np.complex128)
    for ax in range(4):
        L = shape[ax]
        n = np.arange(L)
        W = np.exp(-2j * np.pi * np.outer(n, n) / L)
        out = np.moveaxis(np.tensordot(W, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def full_dft4(f):
    """The 4D defining sum written as one sum over all sites (tiny lattices only)."""
    lt, lz, ly, lx = f.shape[:4]
    out = np.zeros_like(f, dtype=np.complex128)
    for kt, kz, ky, kx in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        acc = 0
        for t, z, y, x in itertools.product(range(lt), range(lz), range(ly), range(lx)):
            ph = kx * x / lx + ky * y / ly + kz * z / lz + kt * t / lt
            acc = acc + f[t, z, y, x] * np.exp(-2j * np.pi * ph)
        out[kt, kz, ky, kx] = acc
    return out


def brute_p2(ext):
    lx, ly, lz, lt = ext
    p2 = np.zeros((lt, lz, ly, lx))
    for kt, kz, ky, kx in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        p2[kt, kz, ky, kx] = sum(4 * np.sin(np.pi * k / L) ** 2
                                 for k, L in ((kx, lx), (ky, ly), (kz, lz), (kt, lt)))
    return p2


@pytest.mark.parametrize("ext", [(2, 2, 2, 2), (3, 3, 3, 3), (2, 3, 4, 6)])
def test_fft_matches_defining_sum(ext):
    lx, ly, lz, lt = ext
    rng = np.random.default_rng(0)
    f = rng.standard_normal((lt, lz, ly, lx, 2)) + 1j * rng.standard_normal((lt, lz, ly, lx, 2))
    ref = full_dft4(f)
    assert np.max(np.abs(O.fft4(f) - ref)) < 1e-12
    assert np.max(np.abs(naive_dft4(f) - ref)) < 1e-12
    assert np.max(np.abs(O.ifft4(ref) - f)) < 1e-13


def test_filter_plane_wave_and_eigenvalues():
    """A plane wave T cos(p.x) is an eigenfunction: filtered -> K(p) T cos(p.x);
    and p2 is the eigenvalue of -d^2 (second difference) on it."""
    ext = (6, 4, 8, 3)
    lx, ly, lz, lt = ext
    k = (1, 3, 2, 1)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ph = 2 * np.pi * (k[0] * x / lx + k[1] * y / ly + k[2] * z / lz + k[3] * t / lt)
    f = np.cos(ph)[..., None, None] * np.ones((1, 1))
    K = O.fa_filter(ext, 0.08)
    out = O.ifft4(O.fft4(f) * K[..., None, None]).real
    p2 = sum(4 * np.sin(np.pi * kk / L) ** 2 for kk, L in zip(k, ext))
    p2max = 4 * np.sin(np.pi * 3 / 6) ** 2 + 4 * np.sin(np.pi * 2 / 4) ** 2 + 4 * np.sin(np.pi * 4 / 8) ** 2 \
        + 4 * np.sin(np.pi * 1 / 3) ** 2
    assert abs(O.p2_max(ext) - p2max) < 1e-14
    assert np.max(np.abs(out - 0.08 * p2max / p2 * f)) < 1e-13
    # -d^2 cos(p.x) = p2 cos(p.x)
    lap = sum(2 * f - np.roll(f, 1, axis=a) - np.roll(f, -1, axis=a) for a in range(4))
    assert np.max(np.abs(lap - p2 * f)) < 1e-12


def test_p2max_even_lattice_is_16():
    assert O.p2_max((8, 8, 8, 8)) == pytest.approx(16.0, abs=1e-14)
    assert O.p2_max((48, 48, 48, 96)) == pytest.approx(16.0, abs=1e-13)


# ---------------------------------------------------------------------------
# reunitarisation against a library QR
# ---------------------------------------------------------------------------

def test_reunitarize_matches_phase_fixed_qr():
    """Gram-Schmidt of rows 1, 2 = the first two columns of Q in M^T = QR with R_ii > 0;
    row 3 is then fixed by det = 1 and orthogonality."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((50, 3, 3)) + 1j * rng.standard_normal((50, 3, 3))
    R = O.reunitarize(M)
    Q, Rr = np.linalg.qr(np.swapaxes(M, -1, -2))
    d = np.diagonal(Rr, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[..., None, :]
    assert np.max(np.abs(R[:, 0, :] - Q[:, :, 0])) < 1e-13
    assert np.max(np.abs(R[:, 1, :] - Q[:, :, 1])) < 1e-13
    assert O.unitarity_defect(R) < 1e-14
    # idempotent on SU(3)
    S = fields.haar_su3((20,), np.random.Generator(np.random.Philox(key=5)))
    assert np.max(np.abs(O.reunitarize(S) - S)) < 1e-14


def test_reunitarize_first_order_is_exponential():
    """reunitarize(1 + X) = exp(X) + O(X^2) for X traceless anti-Hermitian."""
    from scipy.linalg import expm
    rng = np.random.default_rng(4)
    H = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    H = H + H.conj().T
    H -= np.trace(H) / 3 * np.eye(3)
    for s in (1e-3, 1e-4):
        X = 1j * s * H
        err = np.max(np.abs(O.reunitarize(np.eye(3) + X) - expm(X)))
        assert err < 20 * s * s


# ---------------------------------------------------------------------------
# P8: brute force on tiny lattices
# ---------------------------------------------------------------------------

def brute_force_step(U, alpha):
    """Every quantity by explicit loops over sites, directions and colour indices."""
    _, lt, lz, ly, lx = U.shape[:5]
    L = (lx, ly, lz, lt)
    V = lx * ly * lz * lt

    def idx(c):  # c = (x, y, z, t) -> array index (t, z, y, x)
        return (c[3] % lt, c[2] % lz, c[1] % ly, c[0] % lx)

    sites = list(itertools.product(range(lx), range(ly), range(lz), range(lt)))
    unit = [[(1 if m == n else 0) for n in range(4)] for m in range(4)]

    def A(M):  # traceless anti-hermitian part, element by element
        out = np.zeros((3, 3), complex)
        for i in range(3):
            for j in range(3):
                out[i, j] = 0.5 * (M[i, j] - np.conj(M[j, i]))
        tr = (out[0, 0] + out[1, 1] + out[2, 2]) / 3
        for i in range(3):
            out[i, i] -= tr
        return out

    D = np.zeros((lt, lz, ly, lx, 3, 3), complex)
    Fsum = 0.0
    for c in sites:
        for mu in range(4):
            back = tuple(c[n] - unit[mu][n] for n in range(4))
            D[idx(c)] += A(U[mu][idx(back)]) - A(U[mu][idx(c)])
            Fsum += (U[mu][idx(c)][0, 0] + U[mu][idx(c)][1, 1] + U[mu][idx(c)][2, 2]).real
    F = Fsum / (12 * V)
    theta = 0.0
    for c in sites:
        P = 2 * D[idx(c)]
        theta += np.trace(P @ P.conj().T).real
    theta /= 3 * V
    # Fourier step by the defining sums
    p2 = {}
    for k in sites:
        p2[k] = sum(4 * np.sin(np.pi * k[m] / L[m]) ** 2 for m in range(4))
    p2max = max(p2.values())
    Dh = {}
    for k in sites:
        acc = np.zeros((3, 3), complex)
        for c in sites:
            ph = sum(k[m] * c[m] / L[m] for m in range(4))
            acc += D[idx(c)] * np.exp(-2j * np.pi * ph)
        Dh[k] = acc * (0 if p2[k] == 0 else alpha * p2max / p2[k])
    g = np.zeros((lt, lz, ly, lx, 3, 3), complex)
    for c in sites:
        acc = np.zeros((3, 3), complex)
        for k in sites:
            ph = sum(k[m] * c[m] / L[m] for m in range(4))
            acc += Dh[k] * np.exp(2j * np.pi * ph)
        M = np.eye(3) + acc / V
        a = M[0] / np.sqrt(sum(abs(M[0, j]) ** 2 for j in range(3)))
        b = M[1] - sum(np.conj(a[j]) * M[1, j] for j in range(3)) * a
        b = b / np.sqrt(sum(abs(b[j]) ** 2 for j in range(3)))
        cc = np.array([np.conj(a[1] * b[2] - a[2] * b[1]),
                       np.conj(a[2] * b[0] - a[0] * b[2]),
                       np.conj(a[0] * b[1] - a[1] * b[0])])
        g[idx(c)] = np.array([a, b, cc])
    Un = np.zeros_like(U)
    for c in sites:
        for mu in range(4):
            fwd = tuple(c[n] + unit[mu][n] for n in range(4))
            Un[mu][idx(c)] = g[idx(c)] @ U[mu][idx(c)] @ g[idx(fwd)].conj().T
    return F, theta, D, g, Un


@pytest.mark.parametrize("ext", [(2, 2, 2, 2), (2, 3, 2, 3)])
def test_brute_force_tiny_lattice(ext):
    U = fields.random_links(ext, eps=0.8, seed=6)
    F, th, D, g, Un = brute_force_step(U, 0.08)
    Fo, tho, Do = O.measure(U)
    Uo, go = O.fa_step(U, 0.08)
    assert abs(F - Fo) < 1e-14
    assert abs(th - tho) < 1e-13 * th
    assert np.max(np.abs(D - Do)) < 1e-14
    assert np.max(np.abs(g - go)) < 1e-13
    assert np.max(np.abs(Un - Uo)) < 1e-13


# ---------------------------------------------------------------------------
# field generator sanity (the shared input module)
# ---------------------------------------------------------------------------

def test_generator_fields_are_su3_and_seeded():
    ext = (4, 2, 3, 2)
    U = fields.random_links(ext, eps=0.5, seed=0)
    assert U.shape == (4, 2, 3, 2, 4, 3, 3)
    assert O.unitarity_defect(U) < 1e-13
    assert np.array_equal(U, fields.random_links(ext, eps=0.5, seed=0))
    assert not np.array_equal(U, fields.random_links(ext, eps=0.5, seed=1))
    R = fields.as_real(U)
    assert R.shape == U.shape + (2,) and np.array_equal(fields.from_real(R), U)


def test_generator_expi_matches_expm():
    from scipy.linalg import expm
    rng = np.random.default_rng(1)
    H = rng.standard_normal((5, 3, 3)) + 1j * rng.standard_normal((5, 3, 3))
    H = H + np.conj(np.swapaxes(H, -1, -2))
    E = fields.expi_hermitian(H)
    for i in range(5):
        assert np.max(np.abs(E[i] - expm(1j * H[i]))) < 1e-13


def test_generator_haar_moments():
    """For Haar SU(3): E[Tr h] = 0 and E[|Tr h|^2] = 1."""
    h = fields.haar_su3((40000,), np.random.Generator(np.random.Philox(key=2)))
    tr = np.trace(h, axis1=-2, axis2=-1)
    assert abs(np.mean(tr)) < 0.03
    assert abs(np.mean(np.abs(tr) ** 2) - 1.0) < 0.05
