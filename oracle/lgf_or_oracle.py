"""Plain FP64 CPU oracle for overrelaxation Landau gauge fixing.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
use it.  It shares no code with the CUDA library; from the FA-SD oracle it
takes the lattice helpers and the measurement of Sec. 2 (Delta, F, theta),
which define the functional being maximised and the stopping quantity.

Source.  arXiv:1206.0675 (Sec. 3.2) names overrelaxation as the gauge
fixing method that needs less memory than the Fourier-accelerated one, and
gives no algorithm for it.  The method written out here is the published
one it refers to:

* local maximisation of the gauge functional one site at a time (the
  "Los Alamos" method), over the sites of one checkerboard colour at once;
* J. E. Mandula and M. Ogilvie, Phys. Lett. B 248 (1990) 156: replace the
  locally optimal transformation r by r^omega, 1 <= omega < 2, where the
  power is taken to first order in (r - 1), r^omega ~ 1 + omega (r - 1), and
  the result projected back onto the group;
* N. Cabibbo and E. Marinari, Phys. Lett. B 119 (1982) 387: the SU(3)
  maximisation is done in its three SU(2) subgroups in turn.

The steps, in order
-------------------
F[g] = (1/(4 Nc V)) sum_x sum_mu Re Tr g(x) U_mu(x) g^dag(x + mu^) (Sec. 2).
Holding every g(y), y != x, at 1, the part of F that depends on g(x) is
Re Tr[g(x) w(x)] with

    w(x) = sum_mu [ U_mu(x) + U_mu^dag(x - mu^) ].

Sites of one colour (x + y + z + t even, or odd; every extent even) have no
neighbour of their own colour, so their w(x) do not depend on each other's
g and a colour is updated at once.  At one site:

1. M = w(x), g = 1.
2. For each subgroup (i, j) in (0, 1), (0, 2), (1, 2): the 2x2 block B of M
   on rows/columns i, j is written as B = b0 + i (b1 s1 + b2 s2 + b3 s3) plus
   a part that does not contribute to Re Tr (s_k the Pauli matrices):
   b0 = Re(B00 + B11)/2, b1 = Im(B01 + B10)/2, b2 = Re(B01 - B10)/2,
   b3 = Im(B00 - B11)/2.  Over SU(2), Re Tr(r B) = 2 (r0 b0 - r.b) is largest
   at r = (b0, -b1, -b2, -b3)/|b| (r = 1 when |b| = 0).
3. Overrelaxation: q = (1 - omega) + omega r (quaternion sum), r_omega = q/|q|.
   |q| >= 1 for 1 <= omega <= 2, so the division is always safe.
4. R = r_omega embedded on rows/columns i, j of the 3x3 identity;
   M <- R M, g <- R g.

Then U_mu(x) <- g(x) U_mu(x) and U_mu(x - mu^) <- U_mu(x - mu^) g^dag(x) for
the sites of the colour, i.e. the gauge transformation of Sec. 2 with
g = 1 on the other colour.  One sweep is the even colour then the odd one.
The loop measures theta (Sec. 2) every ``check_every`` sweeps and stops
once theta < tol (the strict test of Algorithm 1).

Readings (where the sources leave a choice)
-------------------------------------------
* Colour order: even (x + y + z + t even) first, then odd.
* One pass over the three subgroups per site and colour ("one hit").
* The overrelaxed element is the first-order binomial form, projected by
  normalising the quaternion (not the exact r^omega).
* Counting: the sweep count advances by check_every per measurement, so a
  stop on max_sweeps can overshoot it by less than check_every.

Pins (tests/test_oracle_or_pins.py): the SU(2) maximiser against a direct
numerical maximisation, the overrelaxed element against the matrix power
along the same geodesic, the one-hit SU(3) update of an embedded SU(2)
field, monotone F for 1 <= omega < 2, gauge invariants, a pure-gauge field
driven to F = 1, and the colour update against a site-by-site loop.
"""

from __future__ import annotations

import numpy as np

from oracle import lgf_oracle as O

SUBGROUPS = ((0, 1), (0, 2), (1, 2))  # Cabibbo-Marinari order


# ---------------------------------------------------------------------------
# SU(2) in quaternion form: r = r0 + i (r1 s1 + r2 s2 + r3 s3)
# ---------------------------------------------------------------------------

def su2_components(B: np.ndarray) -> np.ndarray:
    """(b0, b1, b2, b3) of 2x2 complex blocks B (shape (..., 2, 2)) -> (..., 4)."""
    b0 = 0.5 * (B[..., 0, 0].real + B[..., 1, 1].real)
    b1 = 0.5 * (B[..., 0, 1].imag + B[..., 1, 0].imag)
    b2 = 0.5 * (B[..., 0, 1].real - B[..., 1, 0].real)
    b3 = 0.5 * (B[..., 0, 0].imag - B[..., 1, 1].imag)
    return np.stack([b0, b1, b2, b3], axis=-1)


def su2_matrix(q: np.ndarray) -> np.ndarray:
    """2x2 complex matrix q0 + i (q1 s1 + q2 s2 + q3 s3), shape (..., 2, 2)."""
    m = np.empty(q.shape[:-1] + (2, 2), dtype=np.complex128)
    m[..., 0, 0] = q[..., 0] + 1j * q[..., 3]
    m[..., 0, 1] = q[..., 2] + 1j * q[..., 1]
    m[..., 1, 0] = -q[..., 2] + 1j * q[..., 1]
    m[..., 1, 1] = q[..., 0] - 1j * q[..., 3]
    return m


def su2_maximizer(b: np.ndarray) -> np.ndarray:
    """The r in SU(2) that maximises Re Tr(r B) for B with components b: (b0, -b1, -b2, -b3)/|b|."""
    n = np.sqrt(np.sum(b * b, axis=-1))
    r = np.empty_like(b)
    r[..., 0] = b[..., 0]
    r[..., 1:] = -b[..., 1:]
    zero = n == 0.0
    r[~zero] /= n[~zero][..., None]
    r[zero] = (1.0, 0.0, 0.0, 0.0)
    return r


def su2_overrelax(r: np.ndarray, omega: float) -> np.ndarray:
    """Mandula-Ogilvie: r^omega ~ 1 + omega (r - 1), projected back onto SU(2)."""
    q = omega * r
    q[..., 0] += 1.0 - omega
    return q / np.sqrt(np.sum(q * q, axis=-1))[..., None]


# ---------------------------------------------------------------------------
# one site: the Cabibbo-Marinari hit
# ---------------------------------------------------------------------------

def or_site_transform(w: np.ndarray, omega: float) -> np.ndarray:
    """g(x) of one overrelaxation hit for local fields w (shape (..., 3, 3))."""
    M = w.copy()
    g = np.zeros_like(w)
    g[..., 0, 0] = g[..., 1, 1] = g[..., 2, 2] = 1.0
    for i, j in SUBGROUPS:
        idx = [i, j]
        B = M[..., idx, :][..., :, idx]
        r = su2_overrelax(su2_maximizer(su2_components(B)), omega)
        R2 = su2_matrix(r)
        M[..., idx, :] = R2 @ M[..., idx, :]
        g[..., idx, :] = R2 @ g[..., idx, :]
    return g


def or_local_field(U: np.ndarray) -> np.ndarray:
    """w(x) = sum_mu [U_mu(x) + U_mu^dag(x - mu^)] for every site."""
    w = np.zeros(U.shape[1:], dtype=np.complex128)
    for mu in range(4):
        w += U[mu] + O.dagger(O.shift_back(U[mu], mu))
    return w


def parity_mask(extents, parity: int) -> np.ndarray:
    """Boolean site field, True where (x + y + z + t) % 2 == parity; shape (Lt, Lz, Ly, Lx)."""
    lx, ly, lz, lt = extents
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x + y + z + t) % 2 == parity


def check_extents(extents) -> None:
    if any(L % 2 for L in extents):
        raise ValueError("the checkerboard needs every extent even")


# ---------------------------------------------------------------------------
# colours, sweeps and the loop
# ---------------------------------------------------------------------------

def or_half_sweep(U: np.ndarray, parity: int, omega: float) -> tuple[np.ndarray, np.ndarray]:
    """Update the sites of one colour; returns (new links, g) with g = 1 off the colour."""
    ext = O.extents_of(U)
    check_extents(ext)
    g = or_site_transform(or_local_field(U), omega)
    g[~parity_mask(ext, parity)] = np.eye(3)
    return O.apply_gauge(U, g), g


def or_sweep(U: np.ndarray, omega: float) -> tuple[np.ndarray, np.ndarray]:
    """Even colour, then odd.  Returns (new links, g of the sweep): each site
    is transformed once, so g is g_even on even sites and g_odd on odd ones."""
    U, g0 = or_half_sweep(U, 0, omega)
    U, g1 = or_half_sweep(U, 1, omega)
    return U, g1 @ g0


def or_fix(U: np.ndarray, omega: float = 1.7, tol: float = 1e-15, max_sweeps: int = 10000,
           check_every: int = 1, track_G: bool = True):
    """Measure; while theta >= tol and sweeps < max_sweeps: check_every sweeps, then measure.

    Returns a dict like lgf_oracle.fix: final links, accumulated transform G
    (U_final = G U_0 G^dag(x + mu^)), the sweep count, F and theta of every
    measurement (entry 0 before the first sweep) and whether theta < tol.
    """
    if not (1.0 <= omega < 2.0) or check_every < 1:
        raise ValueError("need 1 <= omega < 2 and check_every >= 1")
    G = O.identity_sites(O.extents_of(U)) if track_G else None
    F, th, _ = O.measure(U)
    F_hist, th_hist = [F], [th]
    n = 0
    while th >= tol and n < max_sweeps:
        for _ in range(check_every):
            U, g = or_sweep(U, omega)
            if track_G:
                G = g @ G
        n += check_every
        F, th, _ = O.measure(U)
        F_hist.append(F)
        th_hist.append(th)
    return {"U": U, "G": G, "sweeps": n, "F": np.array(F_hist), "theta": np.array(th_hist),
            "converged": th < tol}
