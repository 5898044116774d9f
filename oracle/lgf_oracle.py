"""Plain FP64 CPU oracle for Fourier-accelerated steepest-descent Landau gauge fixing.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (no kernels, headers, tables or helpers); the only thing the
two sides share is the seeded field generator in
``paper_1206_0675_gb300/fields.py``, which holds none of the method's
arithmetic.

Source: N. Cardoso, P. J. Silva, P. Bicudo, O. Oliveira, "Landau Gauge Fixing
on GPUs", arXiv:1206.0675 (Comput. Phys. Commun.), Section 2 and Algorithm 1.

Representation
--------------
* Links ``U`` are complex128 arrays of shape ``(4, Lt, Lz, Ly, Lx, 3, 3)``:
  direction mu first (0..3 = x, y, z, t), then the site with x fastest, then
  the 3x3 colour matrix ``[row, col]``.  This is the library's user layout.
* Site fields (``g``, ``G``, ``Delta``) drop the leading mu axis.
* Every 3x3 matrix is stored in full (all 9 complex entries); the oracle never
  uses the 12-real or packed-8-real forms of the GPU path.

Readings of the paper (where it is silent or ambiguous)
-------------------------------------------------------
1. theta normalisation.  The Delta of Sec. 2 (the equation defining the
   lattice divergence) is built from ``U - U^dagger``, i.e. it is twice the
   divergence ``Delta_A`` of the traceless anti-Hermitian parts ``A_mu``.
   ``theta = (1/(Nc V)) sum_x Tr[Delta Delta^dagger]`` is therefore evaluated
   as ``(4/(3V)) sum_x ||Delta_A(x)||_F^2`` (``THETA_FACTOR = 4``).
2. The gauge-transform exponent of Eq. (eq:gx) is
   ``(alpha/2) (p2max/p2) F[ sum_nu Delta_{-nu}(U_nu - U_nu^dagger) - trace ]``
   ``= alpha (p2max/p2) F[Delta_A]``.
3. ``p^2`` are the eigenvalues of the lattice ``-d^2``:
   ``p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu)``; ``p2max`` is their maximum over
   the lattice (16 for all-even extents).
4. The zero mode k = 0 gets multiplier 0 (Delta_A is a lattice divergence, so
   its k = 0 component vanishes up to rounding).
5. The exponential is expanded to first order, ``g~ = 1 + Delta'``, then
   reunitarised (Sec. 2, the sentence after Eq. (eq:gx)).  Reunitarisation is
   Gram-Schmidt on rows 1 and 2 with row 3 = (a x b)^* (Sec. 3.2, the
   12-real reconstruction formula), so that det g = 1.
   The exact-exponential variant (``exact_exp=True``) evaluates the
   exponential of Eq. (eq:gx) itself, ``g = exp(Delta')`` with Delta'
   traceless anti-Hermitian, and then applies the same Gram-Schmidt
   projection (a change at rounding level only for a matrix that is
   already in SU(3)), so that both variants hand the update a g built
   the same way.
6. The stop test is strict: iterate while theta >= tol (Algorithm 1); the
   iteration count is the number of link updates performed.
7. The FFT is applied to all 9 complex entries of the 3x3 matrix Delta_A
   (Algorithm 1, "for all elements of Delta(x)").

Pins (see tests/test_oracle_pins.py): identity field, pure-gauge field driven
to F = 1, the weak-field contraction factor (1 - alpha p2max)^2, the
first-order ascent rate dF/dalpha, gauge invariants (plaquette, Polyakov
loops), unitarity, FFT against the defining DFT sum, reunitarisation against
a QR factorisation, and a brute-force loop implementation on 2^4.
"""

from __future__ import annotations

import numpy as np

NC = 3
ALPHA_DEFAULT = 0.08  # Sec. 2: the recommended value of alpha
THETA_FACTOR = 4.0  # reading 1: Delta of Sec. 2 is 2 * Delta_A


# ---------------------------------------------------------------------------
# lattice helpers
# ---------------------------------------------------------------------------

def site_axis(mu: int) -> int:
    """Axis of a site field ``(Lt, Lz, Ly, Lx, ...)`` that runs along mu."""
    return 3 - mu


def extents_of(U: np.ndarray) -> tuple[int, int, int, int]:
    """(Lx, Ly, Lz, Lt) of a link array of shape (4, Lt, Lz, Ly, Lx, 3, 3)."""
    lt, lz, ly, lx = U.shape[1:5]
    return (lx, ly, lz, lt)


def shift_back(field: np.ndarray, mu: int) -> np.ndarray:
    """f(x - mu^) for a site field with periodic boundaries."""
    return np.roll(field, 1, axis=site_axis(mu))


def shift_fwd(field: np.ndarray, mu: int) -> np.ndarray:
    """f(x + mu^) for a site field with periodic boundaries."""
    return np.roll(field, -1, axis=site_axis(mu))


def dagger(M: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(M, -1, -2))


def trace(M: np.ndarray) -> np.ndarray:
    return np.trace(M, axis1=-2, axis2=-1)


def identity_links(extents) -> np.ndarray:
    lx, ly, lz, lt = extents
    U = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def identity_sites(extents) -> np.ndarray:
    lx, ly, lz, lt = extents
    g = np.zeros((lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    g[..., 0, 0] = g[..., 1, 1] = g[..., 2, 2] = 1.0
    return g


# ---------------------------------------------------------------------------
# Sec. 2: divergence, functional, stopping quantity
# ---------------------------------------------------------------------------

def traceless_antihermitian(M: np.ndarray) -> np.ndarray:
    """A = (M - M^dagger)/2 - (1/3) Tr[(M - M^dagger)/2] * 1."""
    A = 0.5 * (M - dagger(M))
    tr = trace(A) / NC
    A = A.copy()
    for i in range(NC):
        A[..., i, i] -= tr
    return A


def divergence(U: np.ndarray) -> np.ndarray:
    """Delta_A(x) = sum_mu [A_mu(x - mu^) - A_mu(x)]  (Sec. 2, lattice d.A).

    The backward difference Delta_{-nu} f(x) = f(x - nu^) - f(x) is the one
    that defines Eq. (eq:gx); A_mu is the traceless anti-Hermitian part of
    U_mu (reading 1: this is half of the paper's Delta).
    """
    D = np.zeros(U.shape[1:], dtype=np.complex128)
    for mu in range(4):
        A = traceless_antihermitian(U[mu])
        D += shift_back(A, mu) - A
    return D


def functional_F(U: np.ndarray) -> float:
    """F = (1/(4 Nc V)) sum_x sum_mu Re Tr U_mu(x)  (Sec. 2, at g = 1)."""
    V = int(np.prod(U.shape[1:5]))
    return float(np.sum(trace(U).real) / (4 * NC * V))


def theta_of_divergence(D: np.ndarray) -> float:
    """theta = (1/(Nc V)) sum_x Tr[Delta Delta^dagger] with Delta = 2 Delta_A."""
    V = int(np.prod(D.shape[:4]))
    return float(THETA_FACTOR * np.sum(np.abs(D) ** 2) / (NC * V))


def measure(U: np.ndarray) -> tuple[float, float, np.ndarray]:
    """Algorithm 1 first step: Delta(x), F and theta of the current links."""
    D = divergence(U)
    return functional_F(U), theta_of_divergence(D), D


# ---------------------------------------------------------------------------
# Eq. (eq:gx): momentum-space filter
# ---------------------------------------------------------------------------

def lattice_p2(extents) -> np.ndarray:
    """p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu), shape (Lt, Lz, Ly, Lx).

    These are the eigenvalues of the lattice operator -d^2 (Sec. 2).
    """
    lx, ly, lz, lt = extents
    s = [4.0 * np.sin(np.pi * np.arange(L) / L) ** 2 for L in (lx, ly, lz, lt)]
    return (s[3][:, None, None, None] + s[2][None, :, None, None]
            + s[1][None, None, :, None] + s[0][None, None, None, :])


def p2_max(extents) -> float:
    """Largest eigenvalue of -d^2 on the lattice: sum_mu 4 sin^2(pi floor(L/2)/L)."""
    return float(sum(4.0 * np.sin(np.pi * (L // 2) / L) ** 2 for L in extents))


def fa_filter(extents, alpha: float = ALPHA_DEFAULT, multiplier=None) -> np.ndarray:
    """K(k) = alpha * p2max / p2(k) * m(k), with K(0) = 0 (readings 2-4).

    ``multiplier`` m(k) defaults to 1 (the paper's filter).
    """
    p2 = lattice_p2(extents)
    K = np.zeros_like(p2)
    nz = p2 > 0
    K[nz] = alpha * p2_max(extents) / p2[nz]
    if multiplier is not None:
        K = K * multiplier
    return K


def sd_filter(extents, alpha: float = ALPHA_DEFAULT) -> np.ndarray:
    """Plain steepest descent (no Fourier acceleration): K(k) = alpha, K(0) = 0."""
    lx, ly, lz, lt = extents
    K = np.full((lt, lz, ly, lx), alpha)
    K[0, 0, 0, 0] = 0.0
    return K


def fft4(f: np.ndarray) -> np.ndarray:
    """Forward 4D DFT over the site axes, f^(k) = sum_x f(x) e^{-2 pi i k.x/L}."""
    return np.fft.fftn(f, axes=(0, 1, 2, 3))


def ifft4(f: np.ndarray) -> np.ndarray:
    """Inverse 4D DFT including the 1/V normalisation (Algorithm 1, 'normalize')."""
    return np.fft.ifftn(f, axes=(0, 1, 2, 3))


# ---------------------------------------------------------------------------
# Sec. 2 / Sec. 3.2: g(x) and reunitarisation
# ---------------------------------------------------------------------------

def reunitarize(M: np.ndarray) -> np.ndarray:
    """Project 3x3 matrices to SU(3) (reading 5).

    a = r1/|r1|;  b = (r2 - <a,r2> a)/|.|  with <a,r> = sum_j conj(a_j) r_j;
    c = (a x b)^*  (the third-row reconstruction of Sec. 3.2).
    """
    r1 = M[..., 0, :]
    r2 = M[..., 1, :]
    a = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1))[..., None]
    ip = np.sum(np.conj(a) * r2, axis=-1)
    b = r2 - ip[..., None] * a
    b = b / np.sqrt(np.sum(np.abs(b) ** 2, axis=-1))[..., None]
    c = np.conj(np.cross(a, b))
    return np.stack([a, b, c], axis=-2)


def expm_antihermitian(X: np.ndarray) -> np.ndarray:
    """exp(X) for traceless anti-Hermitian 3x3 matrices X (reading 5, exact variant).

    X = i Q with Q Hermitian; Q = W diag(lambda) W^dagger (eigendecomposition),
    so exp(X) = W diag(exp(i lambda)) W^dagger.
    """
    Q = -1j * X
    Q = 0.5 * (Q + dagger(Q))  # Hermitian part: removes rounding asymmetry only
    lam, W = np.linalg.eigh(Q)
    return (W * np.exp(1j * lam)[..., None, :]) @ dagger(W)


def gauge_transform_from_divergence(D: np.ndarray, K: np.ndarray, exact_exp: bool = False) -> np.ndarray:
    """Eq. (eq:gx) to first order, then reunitarised.

    Algorithm 1: for every element of the Delta matrix, FFT forward, apply
    the momentum filter, FFT backward, normalise; then for all x obtain
    g(x) = reunitarize(1 + Delta'(x)).  With ``exact_exp`` the exponential is
    evaluated instead: g(x) = reunitarize(exp(Delta'(x))), Delta' taken as
    its traceless anti-Hermitian part (it is one up to rounding, because the
    filter is real and even in k).
    """
    Dhat = fft4(D)
    Dp = ifft4(Dhat * K[..., None, None])
    if exact_exp:
        return reunitarize(expm_antihermitian(traceless_antihermitian(Dp)))
    gt = Dp.copy()
    for i in range(NC):
        gt[..., i, i] += 1.0
    return reunitarize(gt)


def apply_gauge(U: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_mu(x) -> g(x) U_mu(x) g^dagger(x + mu^)  (Sec. 2, gauge transformation)."""
    out = np.empty_like(U)
    for mu in range(4):
        out[mu] = g @ U[mu] @ dagger(shift_fwd(g, mu))
    return out


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------

def fa_step(U: np.ndarray, alpha: float = ALPHA_DEFAULT, K: np.ndarray | None = None,
            D: np.ndarray | None = None, exact_exp: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """One body of the Algorithm 1 loop: FFT, filter, IFFT, g, link update.

    Returns (new links, g).  ``D`` may be passed when the divergence of ``U``
    is already known (it is the measurement that ends the previous body).
    ``exact_exp`` selects g = exp(Delta') over the first-order form.
    """
    if K is None:
        K = fa_filter(extents_of(U), alpha)
    if D is None:
        D = divergence(U)
    g = gauge_transform_from_divergence(D, K, exact_exp)
    return apply_gauge(U, g), g


def fix(U: np.ndarray, alpha: float = ALPHA_DEFAULT, tol: float = 1e-15,
        max_iter: int = 1000, K: np.ndarray | None = None, track_G: bool = True,
        callback=None, exact_exp: bool = False):
    """Algorithm 1: measure; while theta >= tol: step and measure again.

    Returns a dict with the final links, the accumulated transform
    G(x) = g_k(x) ... g_1(x) (so that U_final = G U_0 G^dagger(x+mu^)),
    the iteration count and the per-iteration F and theta histories
    (entry 0 is the initial measurement).
    """
    if K is None:
        K = fa_filter(extents_of(U), alpha)
    G = identity_sites(extents_of(U)) if track_G else None
    F, th, D = measure(U)
    F_hist, th_hist = [F], [th]
    k = 0
    while th >= tol and k < max_iter:
        U, g = fa_step(U, alpha, K, D, exact_exp)
        if track_G:
            G = g @ G
        F, th, D = measure(U)
        F_hist.append(F)
        th_hist.append(th)
        k += 1
        if callback is not None:
            callback(k, U, g)
    return {"U": U, "G": G, "iters": k, "F": np.array(F_hist), "theta": np.array(th_hist),
            "converged": th < tol}


# ---------------------------------------------------------------------------
# gauge invariants and group checks (used by the pins)
# ---------------------------------------------------------------------------

def plaquette(U: np.ndarray) -> float:
    """(1/(18 V)) sum_x sum_{mu<nu} Re Tr U_mu(x) U_nu(x+mu) U_mu^dag(x+nu) U_nu^dag(x)."""
    V = int(np.prod(U.shape[1:5]))
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = U[mu] @ shift_fwd(U[nu], mu) @ dagger(shift_fwd(U[mu], nu)) @ dagger(U[nu])
            s += float(np.sum(trace(P).real))
    return s / (18.0 * V)


def polyakov_loops(U: np.ndarray) -> np.ndarray:
    """Tr prod_t U_t(x, t) for every spatial site, shape (Lz, Ly, Lx)."""
    Ut = U[3]
    P = Ut[0].copy()
    for t in range(1, Ut.shape[0]):
        P = P @ Ut[t]
    return trace(P)


def unitarity_defect(M: np.ndarray) -> float:
    """max |M M^dagger - 1| and |det M - 1| over all matrices."""
    eye = np.eye(3)
    d1 = np.max(np.abs(M @ dagger(M) - eye))
    d2 = np.max(np.abs(np.linalg.det(M) - 1.0))
    return float(max(d1, d2))
