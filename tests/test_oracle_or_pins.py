"""Pins of the overrelaxation oracle (oracle/lgf_or_oracle.py) to facts that
do not come from the oracle itself.

* The SU(2) maximiser reaches the maximum that a direct numerical
  maximisation of Re Tr(r B) over SU(2) (scipy, from many starts) finds.
* The overrelaxed element lies on the geodesic from 1 through r: it equals
  scipy's fractional matrix power r^t for an effective exponent 1 <= t <= omega
  that tends to omega for small rotations.
* One hit on a field w = c R^dag (R an SU(2) element embedded in SU(3))
  returns g = R exactly at omega = 1.
* Re Tr(g w) never decreases in one hit, and F never decreases in a colour
  update, for 1 <= omega < 2 (the cosine argument: the angle moves from phi
  to (1 - t) phi with |1 - t| <= 1).
* Gauge invariants (plaquette, Polyakov loops) and unitarity are kept.
* A pure-gauge field h(x) h^dag(x + mu^) is driven to F = 1, theta -> 0, and
  the accumulated G undoes h up to one global matrix.
* A colour update equals the same local maximisation done site by site in
  a plain loop, in any order, with explicit neighbour indexing.
"""

import numpy as np
import pytest
from scipy import linalg, optimize

from oracle import lgf_oracle as O
from oracle import lgf_or_oracle as R
from paper_1206_0675_gb300 import fields


def rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def su2_of_angles(a):
    """exp(i (a1 s1 + a2 s2 + a3 s3)) through scipy's expm (independent of the quaternion code)."""
    s1 = np.array([[0, 1], [1, 0]], dtype=complex)
    s2 = np.array([[0, -1j], [1j, 0]])
    s3 = np.array([[1, 0], [0, -1]], dtype=complex)
    return linalg.expm(1j * (a[0] * s1 + a[1] * s2 + a[2] * s3))


def test_su2_matrix_is_special_unitary():
    rng = np.random.default_rng(1)
    q = rng.standard_normal((50, 4))
    q /= np.linalg.norm(q, axis=-1, keepdims=True)
    m = R.su2_matrix(q)
    assert np.max(np.abs(m @ O.dagger(m) - np.eye(2))) < 1e-14
    assert np.max(np.abs(np.linalg.det(m) - 1)) < 1e-14


def test_components_reproduce_the_quaternion_part():
    """B = b0 + i b.s + i (c0 + i c.s) for real b, c: the components recover b."""
    rng = np.random.default_rng(2)
    b, c = rng.standard_normal(4), rng.standard_normal(4)
    B = R.su2_matrix(b) + 1j * R.su2_matrix(c)
    assert np.allclose(R.su2_components(B), b, atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_su2_maximizer_against_numerical_maximisation(seed):
    rng = np.random.default_rng(10 + seed)
    B = rand_c(rng, 2, 2)
    r = R.su2_matrix(R.su2_maximizer(R.su2_components(B)))
    best = np.real(np.trace(r @ B))

    def neg(a):
        return -np.real(np.trace(su2_of_angles(a) @ B))

    found = max(-optimize.minimize(neg, rng.uniform(-3, 3, 3), method="BFGS").fun for _ in range(20))
    assert best >= found - 1e-9
    assert abs(best - found) < 1e-7
    # and no random SU(2) element does better
    for _ in range(200):
        assert np.real(np.trace(su2_of_angles(rng.uniform(-3, 3, 3)) @ B)) <= best + 1e-12


def test_su2_maximizer_of_zero_block_is_identity():
    r = R.su2_maximizer(np.zeros((1, 4)))
    assert np.array_equal(r, [[1.0, 0.0, 0.0, 0.0]])


@pytest.mark.parametrize("omega", [1.0, 1.3, 1.7, 1.95])
def test_overrelaxed_element_is_a_power_along_the_geodesic(omega):
    rng = np.random.default_rng(3)
    for phi in (1e-3, 0.1, 0.7, 1.5, 2.5):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        r = np.concatenate([[np.cos(phi)], np.sin(phi) * n])
        ro = R.su2_overrelax(r[None].copy(), omega)[0]
        # effective exponent: the angle of r_omega over that of r, same axis
        psi = np.arctan2(np.linalg.norm(ro[1:]), ro[0])
        t = psi / phi
        assert 1.0 - 1e-12 <= t <= omega + 1e-12
        assert np.allclose(ro[1:] / np.linalg.norm(ro[1:]), n, atol=1e-12)
        Rt = linalg.fractional_matrix_power(R.su2_matrix(r), t)
        assert np.max(np.abs(R.su2_matrix(ro) - Rt)) < 1e-9
        if phi == 1e-3:
            assert abs(t - omega) < 1e-5


def embed(r2, i, j):
    m = np.eye(3, dtype=complex)
    m[np.ix_([i, j], [i, j])] = r2
    return m


def test_one_hit_on_an_embedded_su2_field():
    """w = c R^dag with R in the first subgroup (rows 0, 1): one hit at omega = 1 gives g = R,
    the maximiser of Re Tr(g w) over SU(3) (value 3c); the later subgroups then see c * 1."""
    rng = np.random.default_rng(4)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    Rm = embed(R.su2_matrix(q), 0, 1)
    w = 2.5 * O.dagger(Rm)
    g = R.or_site_transform(w[None], 1.0)[0]
    assert np.max(np.abs(g - Rm)) < 1e-13
    assert abs(np.real(np.trace(g @ w)) - 7.5) < 1e-13


@pytest.mark.parametrize("sub", R.SUBGROUPS)
def test_repeated_hits_reach_the_su3_maximum(sub):
    """For w = c R^dag (R in any subgroup) repeated hits converge to g = R."""
    rng = np.random.default_rng(5)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    Rm = embed(R.su2_matrix(q), *sub)
    w = 2.5 * O.dagger(Rm)
    G = np.eye(3, dtype=complex)
    for _ in range(60):
        G = R.or_site_transform((G @ w)[None], 1.0)[0] @ G
    assert np.max(np.abs(G - Rm)) < 1e-10


@pytest.mark.parametrize("omega", [1.0, 1.5, 1.9])
def test_one_hit_never_lowers_the_local_function(omega):
    rng = np.random.default_rng(5)
    w = rand_c(rng, 200, 3, 3)
    g = R.or_site_transform(w, omega)
    before = np.real(np.trace(w, axis1=-2, axis2=-1))
    after = np.real(np.trace(g @ w, axis1=-2, axis2=-1))
    assert np.all(after >= before - 1e-12)
    assert O.unitarity_defect(g) < 1e-14


def test_local_field_enters_F_as_re_tr_gw():
    """F(g at one site) - F(1) = (Re Tr(g w) - Re Tr w) / (12 V) for any SU(3) g at that site."""
    ext = (4, 4, 2, 4)
    U = fields.random_links(ext, 0.8, 6)
    V = int(np.prod(ext))
    w = R.or_local_field(U)
    g = O.identity_sites(ext)
    h = fields.random_site_su3(ext, 7)[1, 0, 2, 3]
    g[1, 0, 2, 3] = h
    dF = O.functional_F(O.apply_gauge(U, g)) - O.functional_F(U)
    pred = (np.real(np.trace(h @ w[1, 0, 2, 3])) - np.real(np.trace(w[1, 0, 2, 3]))) / (12 * V)
    assert abs(dF - pred) < 1e-15


def test_parity_mask_is_a_checkerboard():
    ext = (4, 2, 6, 4)
    m0, m1 = R.parity_mask(ext, 0), R.parity_mask(ext, 1)
    assert np.all(m0 ^ m1) and m0.sum() == m1.sum()
    for mu in range(4):
        # no site shares its colour with a neighbour
        assert not np.any(m0 & O.shift_fwd(m0, mu))


def test_odd_extent_is_rejected():
    U = fields.random_links((4, 4, 4, 3), 0.5, 1)
    with pytest.raises(ValueError):
        R.or_half_sweep(U, 0, 1.5)


@pytest.mark.parametrize("omega", [1.0, 1.5, 1.9])
def test_F_never_decreases_and_invariants_hold(omega):
    ext = (4, 4, 4, 6)
    U0 = fields.random_links(ext, 1.0, 8)
    U = U0.copy()
    F = O.functional_F(U)
    for k in range(6):
        U, _ = R.or_half_sweep(U, k % 2, omega)
        F2 = O.functional_F(U)
        assert F2 >= F - 1e-15
        F = F2
    assert abs(O.plaquette(U) - O.plaquette(U0)) < 1e-13
    assert np.max(np.abs(O.polyakov_loops(U) - O.polyakov_loops(U0))) < 1e-12
    assert O.unitarity_defect(U) < 1e-13


def test_sweep_transform_reproduces_the_links():
    ext = (4, 2, 4, 4)
    U0 = fields.random_links(ext, 0.9, 9)
    U1, g = R.or_sweep(U0, 1.6)
    assert np.max(np.abs(O.apply_gauge(U0, g) - U1)) < 1e-13


def test_pure_gauge_field_is_driven_to_the_identity():
    ext = (4, 4, 4, 4)
    U0 = fields.pure_gauge_links(ext, 11)
    res = R.or_fix(U0, omega=1.7, tol=1e-24, max_sweeps=400, check_every=2)
    assert res["converged"]
    assert abs(res["F"][-1] - 1.0) < 1e-13
    # G U0 G^dag(x+mu) = 1 on every link: G(x) h(x) is the same matrix everywhere
    U = O.apply_gauge(U0, res["G"])
    assert np.max(np.abs(U - O.identity_links(ext))) < 1e-10
    assert np.all(np.diff(res["F"]) >= -1e-15)


def test_converged_field_is_a_fixed_point():
    ext = (4, 4, 4, 4)
    res = R.or_fix(fields.random_links(ext, 0.6, 12), omega=1.7, tol=1e-26, max_sweeps=3000, check_every=5)
    assert res["converged"]
    D = O.divergence(res["U"])
    assert np.max(np.abs(D)) < 1e-12      # the Landau condition (Sec. 2)
    U2, _ = R.or_sweep(res["U"], 1.7)
    assert abs(O.functional_F(U2) - res["F"][-1]) < 1e-15


def _loop_half_sweep(U, parity, omega, order):
    """One colour updated site by site (plain loops, explicit neighbour indexing)."""
    U = U.copy()
    lt, lz, ly, lx = U.shape[1:5]
    sites = [(t, z, y, x) for t in range(lt) for z in range(lz) for y in range(ly) for x in range(lx)
             if (x + y + z + t) % 2 == parity]
    for k in order(len(sites)):
        t, z, y, x = sites[k]
        c = [x, y, z, t]
        w = np.zeros((3, 3), dtype=complex)
        back = []
        for mu in range(4):
            b = list(c)
            b[mu] = (b[mu] - 1) % (lx, ly, lz, lt)[mu]
            bi = (mu, b[3], b[2], b[1], b[0])
            w += U[mu, t, z, y, x] + U[bi].conj().T
            back.append(bi)
        g = R.or_site_transform(w[None], omega)[0]
        for mu in range(4):
            U[mu, t, z, y, x] = g @ U[mu, t, z, y, x]
            U[back[mu]] = U[back[mu]] @ g.conj().T
    return U


@pytest.mark.parametrize("ext", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_colour_update_equals_a_site_by_site_loop(ext):
    U = fields.random_links(ext, 1.0, 13)
    rng = np.random.default_rng(14)
    for parity in (0, 1):
        want, _ = R.or_half_sweep(U, parity, 1.7)
        fwd = _loop_half_sweep(U, parity, 1.7, lambda n: range(n))
        shuf = _loop_half_sweep(U, parity, 1.7, lambda n: rng.permutation(n))
        assert np.max(np.abs(fwd - want)) < 1e-13
        assert np.max(np.abs(shuf - want)) < 1e-13
        U = want
