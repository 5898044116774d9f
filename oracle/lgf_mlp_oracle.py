"""FP64 CPU oracle of the learned momentum-space multiplier (test infrastructure only).

Nothing on the product path imports this module (see oracle/lgf_oracle.py).
The paper has no learned part: this is the reference for the library's
additions -- a per-mode multiplier m(k) applied on top of the
Fourier-acceleration filter alpha p2max/p2(k) of Eq. (eq:gx), predicted by a
small MLP and trained on statistics logged from plain FA-SD trajectories.

Network (flat parameter vector, the library's layout, 8961 numbers)
-------------------------------------------------------------------
    h1 = relu(W1 x + b1)      W1: [64][8]   offset 0,    b1: [64] offset 512
    h2 = relu(W2 h1 + b2)     W2: [64][64]  offset 576,  b2: [64] offset 4672
    h3 = relu(W3 h2 + b3)     W3: [64][64]  offset 4736, b3: [64] offset 8832
    z  = w4 . h3 + b4         w4: [64]      offset 8896, b4: [1]  offset 8960
    m  = softplus(z) = log(1 + e^z)

Features of a momentum mode k at iteration k_it with stopping quantity theta
--------------------------------------------------------------------------
    x = (p2_x/4, p2_y/4, p2_z/4, p2_t/4, -bucket(theta)/16, iter_frac, rate, r_class)
    p2_mu = 4 sin^2(pi k_mu / L_mu)        (per direction, as in the filter)
    bucket(theta) = floor(2 log10 theta) / 2   (half decades; theta <= 0 -> -20)
    iter_frac = min(k_it / 10000, 1)
    rate = clamp(log10(theta / theta_prev), -2, 1) / 2   (0 on the first step),
           theta_prev being the stopping quantity one step earlier
    r_class = clamp(r, -1, 1): the contraction of the mode's class (modes with
           the same p2 tuple) over the last step whose two Fourier-space
           divergences are known, under the plain filter:
           r = sum Re<D^_new, D^_old> / sum |D^_old|^2 over the class
           (0 while fewer than two divergences are known)

Inference on the GPU uses BF16 weights with FP32 accumulation: ``forward``
with ``bf16=True`` emulates it (weights and the inputs of the three mma
layers rounded to BF16 with round-to-nearest-even; the last hidden layer and
the output layer stay in full precision).

Training target (defined here; nothing in the paper fixes it)
--------------------------------------------------------------
From a plain FA-SD trajectory, for every mode class c (modes with the same
p2 tuple) and theta bucket b, the logged ratio
    r = sum Re<D^_{k+1}, D^_k> / sum |D^_k|^2
estimates the per-step contraction 1 - K0 lambda_eff of that class.  The
multiplier that would remove it in one step in the linear model is
m* = 1/(1 - r); it is clamped to [M_LO, M_HI].  M_HI = 2 bounds the step a
slowly contracting class may take: with the class's own contraction as an
input the multiplier can stay near 1 (or below) on classes that contract
fast or oscillate, so the cap that a uniform multiplier needed for stability
(1.25) no longer binds.  The linear model holds only once the step is small:
in buckets with theta >= THETA_LINEAR the target is the plain filter,
m* = 1.  The loss is the weighted mean square error of log m against log m*,
with weight |D^_k|^2 normalised per bucket.
"""

from __future__ import annotations

import numpy as np

NIN, NH = 8, 64
OFF_W1, OFF_B1 = 0, 512
OFF_W2, OFF_B2 = 576, 4672
OFF_W3, OFF_B3 = 4736, 8832
OFF_W4, OFF_B4 = 8896, 8960
NPARAM = 8961
ITER_SCALE = 10000.0
M_LO, M_HI = 0.25, 2.0
THETA_LINEAR = 1e-4


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    W1 = p[OFF_W1:OFF_B1].reshape(NH, NIN)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(NH, NH)
    b2 = p[OFF_B2:OFF_W3]
    W3 = p[OFF_W3:OFF_B3].reshape(NH, NH)
    b3 = p[OFF_B3:OFF_W4]
    w4 = p[OFF_W4:OFF_B4]
    b4 = p[OFF_B4]
    return W1, b1, W2, b2, W3, b3, w4, b4


def pack(W1, b1, W2, b2, W3, b3, w4, b4) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3, w4, [b4]]).astype(np.float64)


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def softplus(z):
    z = np.asarray(z, dtype=np.float64)
    return np.where(z > 30, z, np.log1p(np.exp(np.minimum(z, 30))))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-np.asarray(z, dtype=np.float64)))


def theta_bucket(theta: float) -> float:
    if not theta > 0:
        return -20.0
    return np.floor(2.0 * np.log10(theta)) / 2.0


def rate_feature(theta: float, theta_prev: float) -> float:
    if not (theta > 0 and theta_prev > 0):
        return 0.0
    return 0.5 * float(np.clip(np.log10(theta / theta_prev), -2.0, 1.0))


def features(p2_tuple, theta: float, iteration: int, theta_prev: float = 0.0, r_class=0.0) -> np.ndarray:
    """Feature rows for an array of per-direction p2 tuples, shape (n, 4) -> (n, 8);
    r_class (scalar or one value per row) is the class contraction, clamped to [-1, 1]."""
    p2 = np.atleast_2d(np.asarray(p2_tuple, dtype=np.float64))
    n = p2.shape[0]
    x = np.empty((n, NIN))
    x[:, :4] = p2 / 4.0
    x[:, 4] = -theta_bucket(theta) / 16.0
    x[:, 5] = min(iteration / ITER_SCALE, 1.0)
    x[:, 6] = rate_feature(theta, theta_prev) if iteration > 0 else 0.0
    x[:, 7] = np.clip(np.broadcast_to(np.asarray(r_class, dtype=np.float64), (n,)), -1.0, 1.0)
    return x


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation with the output layer zero and b4 = log(e-1), so m = 1."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    W1 = rng.standard_normal((NH, NIN)) * np.sqrt(2.0 / NIN)
    W2 = rng.standard_normal((NH, NH)) * np.sqrt(2.0 / NH)
    W3 = rng.standard_normal((NH, NH)) * np.sqrt(2.0 / NH)
    return pack(W1, np.zeros(NH), W2, np.zeros(NH), W3, np.zeros(NH), np.zeros(NH), np.log(np.e - 1.0))


def forward(p: np.ndarray, X: np.ndarray, bf16: bool = False):
    """m(x) for feature rows X (n, 7); returns (m, cache)."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(bf16_round(p) if bf16 else p)
    r = bf16_round if bf16 else (lambda a: a)
    X = np.asarray(X, dtype=np.float64)
    a1 = r(X) @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = r(h1) @ W2.T + b2
    h2 = np.maximum(a2, 0)
    a3 = r(h2) @ W3.T + b3
    h3 = np.maximum(a3, 0)
    z = h3 @ w4 + b4
    return softplus(z), (X, a1, h1, a2, h2, a3, h3, z)


def loss_and_grad(p: np.ndarray, X: np.ndarray, Y: np.ndarray, Wt: np.ndarray):
    """Weighted MSE of log m against Y = log m*, and its gradient (backpropagation by hand)."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p)
    m, (X, a1, h1, a2, h2, a3, h3, z) = forward(p, X)
    sw = float(np.sum(Wt))
    e = np.log(m) - Y
    loss = float(np.sum(Wt * e * e) / sw)
    dz = 2.0 * Wt * e / sw * sigmoid(z) / m          # d log softplus(z)/dz = sigmoid(z)/softplus(z)
    gw4 = h3.T @ dz
    gb4 = np.sum(dz)
    dh3 = np.outer(dz, w4)
    da3 = dh3 * (a3 > 0)
    gW3 = da3.T @ h2
    gb3 = np.sum(da3, axis=0)
    dh2 = da3 @ W3
    da2 = dh2 * (a2 > 0)
    gW2 = da2.T @ h1
    gb2 = np.sum(da2, axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    gW1 = da1.T @ X
    gb1 = np.sum(da1, axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gW3, gb3, gw4, gb4)


def targets_from_stats(num: np.ndarray, den: np.ndarray, bucket=None) -> np.ndarray:
    """log m* = log clamp(1/(1 - r), M_LO, M_HI) with r = num/den (den > 0 entries only);
    0 (the plain filter) where bucket(theta) >= log10(THETA_LINEAR)."""
    r = num / den
    with np.errstate(divide="ignore"):
        m = np.where(r < 1.0, 1.0 / (1.0 - r), M_HI)
    y = np.log(np.clip(m, M_LO, M_HI))
    if bucket is not None:
        y = np.where(np.asarray(bucket) < np.log10(THETA_LINEAR), y, 0.0)
    return y
