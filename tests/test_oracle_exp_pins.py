"""Pins of the oracle's exact-exponential variant (g = exp(Delta'), Eq. (eq:gx)).

The paper expands the exponential of Eq. (eq:gx) to first order and
reunitarises; the variant evaluates the exponential itself.  The pins use
library routines (scipy's expm), closed forms (diagonal and SU(2)-embedded
exponents, abelian fields, where both variants have exact answers that differ)
and the linearisation facts that the two variants share: the weak-field
contraction factor and the first-order ascent rate.
"""

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import lgf_oracle as O
from paper_1206_0675_gb300 import fields


def random_su3_algebra(rng, n, scale):
    """n traceless anti-Hermitian 3x3 matrices of Frobenius norm `scale`."""
    A = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    H -= (np.trace(H, axis1=-2, axis2=-1) / 3)[:, None, None] * np.eye(3)
    H *= scale / np.linalg.norm(H, axis=(-2, -1))[:, None, None]
    return 1j * H


@pytest.mark.parametrize("scale", [1e-9, 1e-3, 0.3, 1.0, 3.0, 20.0])
def test_expm_antihermitian_matches_scipy(scale):
    rng = np.random.default_rng(int(scale * 1e3) + 1)
    X = random_su3_algebra(rng, 50, scale)
    E = O.expm_antihermitian(X)
    for i in range(len(X)):
        assert np.max(np.abs(E[i] - expm(X[i]))) < 5e-15 * max(1.0, scale)
    assert O.unitarity_defect(E) < 1e-13 * max(1.0, scale)


def test_expm_closed_forms():
    # diagonal: exp(i diag(a, b, -a-b)) = diag(e^{ia}, e^{ib}, e^{-i(a+b)})
    a, b = 0.7, -1.9
    X = 1j * np.diag([a, b, -a - b])
    assert np.max(np.abs(O.expm_antihermitian(X) - np.diag(np.exp(1j * np.array([a, b, -a - b]))))) < 1e-15
    # SU(2) embedding: exp(i phi n.sigma/2) = cos(phi/2) 1 + i sin(phi/2) n.sigma in the (1,2) block
    phi = 2.3
    n = np.array([0.36, -0.48, 0.8])
    sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    ns = sum(n[i] * sig[i] for i in range(3))
    X = np.zeros((3, 3), complex)
    X[:2, :2] = 0.5j * phi * ns
    want = np.eye(3, dtype=complex)
    want[:2, :2] = np.cos(phi / 2) * np.eye(2) + 1j * np.sin(phi / 2) * ns
    assert np.max(np.abs(O.expm_antihermitian(X) - want)) < 1e-15


def abelian_links(ext, seed):
    """Diagonal SU(3) links diag(e^{i p1}, e^{i p2}, e^{-i(p1+p2)})."""
    rng = np.random.default_rng(seed)
    lx, ly, lz, lt = ext
    ph = rng.uniform(-0.8, 0.8, size=(4, lt, lz, ly, lx, 2))
    U = np.zeros((4, lt, lz, ly, lx, 3, 3), complex)
    U[..., 0, 0] = np.exp(1j * ph[..., 0])
    U[..., 1, 1] = np.exp(1j * ph[..., 1])
    U[..., 2, 2] = np.exp(-1j * (ph[..., 0] + ph[..., 1]))
    return U


def test_abelian_field_gauge_transforms_in_closed_form():
    """On diagonal (abelian) links Delta' = i diag(d1, d2, d3) with d1 + d2 + d3 = 0.
    Then exp(Delta') = diag(e^{i d1}, e^{i d2}, e^{i d3}) exactly, while the
    first-order form reunitarises 1 + Delta' to diag(e^{i atan d1}, e^{i atan d2},
    e^{-i(atan d1 + atan d2)}): the two variants differ at third order in d."""
    ext = (4, 6, 4, 4)
    U = abelian_links(ext, 3)
    D = O.divergence(U)
    K = O.fa_filter(ext, 0.08)
    Dp = np.fft.ifftn(np.fft.fftn(D, axes=(0, 1, 2, 3)) * K[..., None, None], axes=(0, 1, 2, 3))
    d = np.stack([Dp[..., i, i].imag for i in range(3)], axis=-1)
    assert np.max(np.abs(Dp[..., 0, 1])) < 1e-15 and np.max(np.abs(d.sum(-1))) < 1e-14
    assert np.max(np.abs(d)) > 0.1  # the two variants really differ here
    g_exp = O.gauge_transform_from_divergence(D, K, exact_exp=True)
    g_fo = O.gauge_transform_from_divergence(D, K)
    want_exp = np.zeros_like(g_exp)
    want_fo = np.zeros_like(g_fo)
    at = np.arctan(d)
    for i in range(3):
        want_exp[..., i, i] = np.exp(1j * d[..., i])
    want_fo[..., 0, 0] = np.exp(1j * at[..., 0])
    want_fo[..., 1, 1] = np.exp(1j * at[..., 1])
    want_fo[..., 2, 2] = np.exp(-1j * (at[..., 0] + at[..., 1]))
    assert np.max(np.abs(g_exp - want_exp)) < 1e-14
    assert np.max(np.abs(g_fo - want_fo)) < 1e-14
    assert np.max(np.abs(g_exp - g_fo)) > 1e-4


def test_exact_and_first_order_differ_at_second_order():
    """|g_exp - g_first| scales as alpha^2 for a fixed divergence."""
    ext = (4, 4, 2, 4)
    U = fields.random_links(ext, eps=0.5, seed=8)
    D = O.divergence(U)
    diffs = []
    for a in (0.004, 0.002):
        K = O.fa_filter(ext, a)
        diffs.append(np.max(np.abs(O.gauge_transform_from_divergence(D, K, True)
                                   - O.gauge_transform_from_divergence(D, K))))
    assert 3.6 < diffs[0] / diffs[1] < 4.4


def test_exact_exp_weak_field_factor():
    """The linearised step is the same for both variants: theta contracts by (1 - alpha p2max)^2."""
    U = fields.random_links((4, 4, 4, 4), eps=1e-6, seed=1, gauge_rotate=False)
    _, th0, _ = O.measure(U)
    _, th1, _ = O.measure(O.fa_step(U, 0.08, exact_exp=True)[0])
    assert abs(th1 / th0 - 0.0784) < 1e-4


def test_exact_exp_ascent_rate_and_gauge_invariants():
    ext = (3, 4, 2, 3)
    U = fields.random_links(ext, eps=0.4, seed=7)
    a = 1e-5
    rate_fo = (O.functional_F(O.fa_step(U, a)[0]) - O.functional_F(O.fa_step(U, -a)[0])) / (2 * a)
    rate_ex = (O.functional_F(O.fa_step(U, a, exact_exp=True)[0])
               - O.functional_F(O.fa_step(U, -a, exact_exp=True)[0])) / (2 * a)
    assert abs(rate_ex - rate_fo) < 1e-8 * rate_fo
    U1, g = O.fa_step(U, 0.08, exact_exp=True)
    assert abs(O.plaquette(U1) - O.plaquette(U)) < 1e-12
    assert O.unitarity_defect(g) < 1e-13 and O.unitarity_defect(U1) < 1e-13


def test_exact_exp_pure_gauge_converges_to_unit_links():
    ext = (4, 4, 4, 4)
    U0 = fields.pure_gauge_links(ext, seed=3)
    res = O.fix(U0, tol=1e-26, max_iter=400, exact_exp=True)
    assert res["converged"] and res["F"][-1] > 1.0 - 1e-13
    assert np.max(np.abs(res["U"] - np.eye(3))) < 1e-6
    assert np.all(np.diff(res["F"]) > -1e-15)


def test_exact_exp_brute_force_tiny_lattice():
    """The variant on 2^4 against loops: the defining DFT sums, scipy's expm
    on each site's 3x3 exponent, then Gram-Schmidt written out."""
    ext = (2, 2, 2, 2)
    U = fields.random_links(ext, eps=0.8, seed=6)
    D = O.divergence(U)
    V = 16
    L = ext
    sites = [(x, y, z, t) for x in range(2) for y in range(2) for z in range(2) for t in range(2)]
    p2 = {k: sum(4 * np.sin(np.pi * k[m] / L[m]) ** 2 for m in range(4)) for k in sites}
    p2max = max(p2.values())
    g = np.zeros((2, 2, 2, 2, 3, 3), complex)
    for c in sites:
        acc = np.zeros((3, 3), complex)
        for k in sites:
            if p2[k] == 0:
                continue
            Dh = np.zeros((3, 3), complex)
            for c2 in sites:
                Dh += D[c2[3], c2[2], c2[1], c2[0]] * np.exp(-2j * np.pi * sum(k[m] * c2[m] / L[m] for m in range(4)))
            acc += 0.08 * p2max / p2[k] * Dh * np.exp(2j * np.pi * sum(k[m] * c[m] / L[m] for m in range(4)))
        X = acc / V
        X = 0.5 * (X - X.conj().T)
        X -= np.trace(X) / 3 * np.eye(3)
        M = expm(X)
        a = M[0] / np.linalg.norm(M[0])
        b = M[1] - np.vdot(a, M[1]) * a
        b /= np.linalg.norm(b)
        g[c[3], c[2], c[1], c[0]] = np.array([a, b, np.conj(np.cross(a, b))])
    _, go = O.fa_step(U, 0.08, exact_exp=True)
    assert np.max(np.abs(g - go)) < 1e-13
