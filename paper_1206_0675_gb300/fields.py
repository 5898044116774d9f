"""Seeded synthetic SU(3) link fields (the workload recipe, not the method).

This module builds the input configurations that both the CUDA path and the
CPU oracle consume; it contains none of the gauge-fixing arithmetic
(no divergence, no functional, no Fourier filter, no reunitarisation).

Recipe (the shape of the paper's Sec. 4 workloads, with synthetic fields
standing in for its beta = 5.8/6.0/6.2 Wilson-action configurations):

    U_mu(x) = h(x) . exp(i eps sum_a c_a lambda_a / 2) . h^dagger(x + mu^)

* c_a ~ N(0, 1) i.i.d. per link and generator, lambda_a the Gell-Mann
  matrices; exp(iH) of the Hermitian traceless H is formed from its
  eigendecomposition.
* h(x) is Haar-random in SU(3): QR of a 3x3 complex Gaussian with the
  diagonal-phase fix of Mezzadri (2007), divided by a cube root of its
  determinant.
* Random numbers: one Philox-4x64 counter-based stream per seed
  (``numpy.random.Philox(key=seed)``), drawn in this fixed order:
  c (shape (4, Lt, Lz, Ly, Lx, 8)), then Re Z and Im Z of h (each of shape
  (Lt, Lz, Ly, Lx, 3, 3)).

Layout of the returned links: complex128 ``(4, Lt, Lz, Ly, Lx, 3, 3)`` -
direction mu (x, y, z, t) first, site with x fastest, then the matrix
``[row, col]``.  ``as_real`` views it as the library's float64 user layout
``[mu][t][z][y][x][row][col][re, im]``.
"""

from __future__ import annotations

import numpy as np


def _gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


GELL_MANN = _gell_mann()


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _site_shape(extents) -> tuple[int, int, int, int]:
    lx, ly, lz, lt = (int(e) for e in extents)
    return (lt, lz, ly, lx)


def expi_hermitian(H: np.ndarray) -> np.ndarray:
    """exp(iH) for a stack of Hermitian 3x3 matrices via eigendecomposition."""
    w, Q = np.linalg.eigh(H)
    return (Q * np.exp(1j * w)[..., None, :]) @ np.conj(np.swapaxes(Q, -1, -2))


def haar_su3(shape, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed SU(3) matrices of the given batch shape."""
    Z = rng.standard_normal(tuple(shape) + (3, 3)) + 1j * rng.standard_normal(tuple(shape) + (3, 3))
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(Q)
    return Q * np.exp(-1j * np.angle(det) / 3.0)[..., None, None]


def _fwd(field: np.ndarray, mu: int) -> np.ndarray:
    return np.roll(field, -1, axis=3 - mu)


def random_links(extents, eps: float, seed: int, gauge_rotate: bool = True) -> np.ndarray:
    """U_mu(x) = h(x) exp(i eps sum_a c_a lambda_a/2) h^dagger(x+mu^).

    With ``gauge_rotate=False`` the links are the bare exp(i eps H) (h = 1),
    which is the weak-field workload when eps is small.
    """
    sites = _site_shape(extents)
    rng = _rng(seed)
    c = rng.standard_normal((4,) + sites + (8,))
    H = 0.5 * eps * np.einsum("...a,aij->...ij", c, GELL_MANN)
    Vl = expi_hermitian(H)
    if not gauge_rotate:
        return Vl
    h = haar_su3(sites, rng)
    hd = np.conj(np.swapaxes(h, -1, -2))
    return np.stack([h @ Vl[mu] @ _fwd(hd, mu) for mu in range(4)])


def pure_gauge_links(extents, seed: int) -> np.ndarray:
    """U_mu(x) = h(x) h^dagger(x + mu^): a gauge copy of the identity field."""
    sites = _site_shape(extents)
    rng = _rng(seed)
    h = haar_su3(sites, rng)
    hd = np.conj(np.swapaxes(h, -1, -2))
    return np.stack([h @ _fwd(hd, mu) for mu in range(4)])


def random_site_su3(extents, seed: int) -> np.ndarray:
    """Haar SU(3) matrix per site, shape (Lt, Lz, Ly, Lx, 3, 3)."""
    return haar_su3(_site_shape(extents), _rng(seed))


def as_real(U: np.ndarray) -> np.ndarray:
    """float64 view [..., row, col, re/im] of a complex128 field (C-contiguous copy)."""
    return np.ascontiguousarray(U).view(np.float64).reshape(U.shape + (2,))


def from_real(R: np.ndarray) -> np.ndarray:
    """Inverse of ``as_real``."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    return R.view(np.complex128).reshape(R.shape[:-1])


# Batch workload: 64 configurations of uneven sizes with eps ~ U[0.3, 1.0].
BATCH64_EXTENTS = ([(8, 8, 8, 8)] * 16 + [(12, 12, 12, 12)] * 16 + [(16, 16, 16, 16)] * 16
                   + [(16, 16, 16, 32)] * 8 + [(24, 24, 24, 24)] * 8)


def batch_eps(i: int) -> float:
    """eps of batch member i: uniform in [0.3, 1.0] from its own Philox stream."""
    return 0.3 + 0.7 * float(_rng(1_000_000 + int(i)).random())
