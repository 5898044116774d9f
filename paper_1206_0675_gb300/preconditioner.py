"""Training of the learned per-mode multiplier on the GPU with the library's kernels.

Data: plain FA-SD trajectories (FP64, alpha = 0.08) of synthetic SU(3)
configurations at 16^4 and 24^4 with eps uniform in [0.3, 1.0], run through
``lgf_step`` with the mode log on.  For every configuration, theta bucket b
and momentum class c the log gives

    r = sum Re<D^_{k+1}, D^_k> / sum |D^_k|^2

(D^ the 4D Fourier transform of the packed divergence), the per-step
contraction of that class under the plain filter.  The training target is
the multiplier that would remove it in one step in a linear model,
m* = 1/(1 - r), clamped to [0.25, 2].  The linear model
holds only once the gauge transformations are small: for theta >= 1e-4
(the first, non-linear part of every trajectory, where a uniformly larger
step was measured to slow fast-converging fields) the target is the plain
filter, m* = 1.  Buckets below theta = 1e-15 (rounding noise) are left out.
The loss is the mean square error of log m, weighted by |D^_k|^2
normalised within each (configuration, bucket).

Features (identical to the ones the inference kernel builds):
    (p2_x/4, p2_y/4, p2_z/4, p2_t/4, -bucket/16, iter_frac, rate, r_class)
with p2_mu = 4 sin^2(pi f_mu / L_mu), bucket = floor(2 log10 theta)/2 of the
step's starting links, iter_frac = min(iteration / 10000, 1),
rate = clamp(log10(theta/theta_prev), -2, 1)/2 the contraction of theta over
the previous step (0 on the first step), averaged over the steps of a bucket,
and r_class = sum Re<D^_k, D^_{k-1}> / sum |D^_{k-1}|^2 the class's own
contraction over the previous step (summed over the steps of the bucket,
clamped to [-1, 1]; 0 where the previous step is not logged).  The inference
kernel forms the same quantity one step later than the step it predicts for,
from the divergences it keeps.

The network is trained with Adam by ``lgf_mlp_train`` (FP32 forward and
backward kernels of liblgf) and stored as BF16 (``lgf_mlp_to_bf16``).

    python -m paper_1206_0675_gb300.preconditioner [--configs 200] [--out FILE]
"""

from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import fields, lgf

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "preconditioner_bf16.npy")
M_LO, M_HI = 0.25, 2.0
THETA_LINEAR = 1e-4
NPARAM = lgf.LGF_MLP_NPARAM


def class_p2(extents) -> np.ndarray:
    """Per-direction p2 of every momentum class, shape (nclass, 4), class order of the library."""
    H = [L // 2 + 1 for L in extents]
    tabs = [4.0 * np.sin(np.pi * np.arange(h) / L) ** 2 for h, L in zip(H, extents)]
    ft, fz, fy, fx = np.meshgrid(np.arange(H[3]), np.arange(H[2]), np.arange(H[1]), np.arange(H[0]), indexing="ij")
    return np.stack([tabs[0][fx], tabs[1][fy], tabs[2][fz], tabs[3][ft]], -1).reshape(-1, 4)


def targets(r: np.ndarray, bucket: np.ndarray) -> np.ndarray:
    """log m*: log clamp(1/(1 - r), M_LO, M_HI) where the linear model holds, else 0."""
    m = np.where(r < 1.0, 1.0 / np.maximum(1.0 - r, 1e-12), M_HI)
    y = np.log(np.clip(m, M_LO, M_HI))
    return np.where(bucket < np.log10(THETA_LINEAR), y, 0.0)


def samples_from_log(extents, stats: np.ndarray, rng: np.random.Generator, per_bucket: int = 256):
    """(X, r, w) rows from one configuration's mode log [bucket][class][7]: features,
    logged contraction ratio and weight.  Buckets below theta = 1e-15 are left out."""
    p2 = class_p2(extents)
    X, Rr, W = [], [], []
    for b in range(stats.shape[0]):
        if (4 - b) / 2.0 < -15.0:
            continue
        num, den, cnt, itf, rate, num_lag, den_lag = stats[b].T
        ok = np.nonzero((cnt > 0) & (den > 0))[0]
        if ok.size == 0:
            continue
        if ok.size > per_bucket:
            ok = rng.choice(ok, per_bucket, replace=False)
        bucket = (4 - b) / 2.0
        x = np.empty((ok.size, 8))
        x[:, :4] = p2[ok] / 4.0
        x[:, 4] = -bucket / 16.0
        x[:, 5] = np.minimum(itf[ok] / cnt[ok], 1.0)
        x[:, 6] = rate[ok] / cnt[ok]
        with np.errstate(divide="ignore", invalid="ignore"):
            x[:, 7] = np.where(den_lag[ok] > 0, np.clip(num_lag[ok] / den_lag[ok], -1.0, 1.0), 0.0)
        X.append(x)
        Rr.append(num[ok] / den[ok])
        W.append(den[ok] / den[ok].sum())
    if not X:
        return np.zeros((0, 8)), np.zeros(0), np.zeros(0)
    return np.concatenate(X), np.concatenate(Rr), np.concatenate(W)


def collect(extents, eps: float, seed: int, tol: float = 1e-15, max_iter: int = 6000):
    """Plain FP64 trajectory with the mode log on; returns (stats, iterations, theta)."""
    U = fields.random_links(extents, eps, seed)
    with lgf.Lattice(extents, "fp64") as lat:
        lat.set_links(U)
        lat.set_mode_log(True)
        k = 0
        F, th = lat.measure()
        while th >= tol and k < max_iter:
            n = 25 if th > 1e-9 else 2
            for _ in range(n):
                lat.step(0.08)
            k += n
            F, th = lat.measure()
        return lat.get_mode_log(), k, th


def init_params(seed: int) -> np.ndarray:
    """He initialisation; the output layer starts at zero with b4 = log(e - 1) (m = 1)."""
    rng = np.random.Generator(np.random.Philox(key=seed + 7))
    p = np.zeros(NPARAM, dtype=np.float32)
    p[0:512] = rng.standard_normal(512) * np.sqrt(2.0 / 8)
    p[576:4672] = rng.standard_normal(4096) * np.sqrt(2.0 / 64)
    p[4736:8832] = rng.standard_normal(4096) * np.sqrt(2.0 / 64)
    p[8960] = np.log(np.e - 1.0)
    return p


def train(X, Y, W, steps=(8000, 4000), lrs=(1e-3, 3e-4), batch=4096, seed=0, verbose=True):
    """Adam on the GPU through lgf_mlp_train; returns (fp32 params, bf16 params, loss history)."""
    import torch
    dev = torch.device("cuda")
    Xd = torch.tensor(X, dtype=torch.float32, device=dev).contiguous()
    Yd = torch.tensor(Y, dtype=torch.float32, device=dev).contiguous()
    Wn = W / W.mean()
    Wd = torch.tensor(Wn, dtype=torch.float32, device=dev).contiguous()
    P = torch.tensor(init_params(seed), device=dev)
    adam = torch.zeros(2 * NPARAM, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    hist = []
    t0 = 0
    for n_steps, lr in zip(steps, lrs):
        h = lgf.lgf_mlp_train(P.data_ptr(), adam.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Wd.data_ptr(), Xd.shape[0],
                              batch, n_steps, lr, seed, t0, stream)
        hist.extend(h.tolist())
        t0 += n_steps
        if verbose:
            print(f"  {t0} steps: minibatch loss {np.mean(h[-200:]):.5f}", flush=True)
    full = lgf.lgf_mlp_loss_grad(P.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Wd.data_ptr(), Xd.shape[0],
                                 torch.empty(NPARAM, device=dev).data_ptr(), stream)
    Pb = torch.empty(NPARAM, dtype=torch.int16, device=dev)
    lgf.lgf_mlp_to_bf16(P.data_ptr(), Pb.data_ptr(), stream)
    torch.cuda.synchronize()
    return P.cpu().numpy(), Pb.cpu().numpy().view(np.uint16), hist, full


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", type=int, default=200, help="configurations, split evenly over 16^4 and 24^4")
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--per-bucket", type=int, default=256)
    ap.add_argument("--save-data", default=None, help="also write the training rows to this .npz file")
    ap.add_argument("--from-data", default=None, help="train on rows saved by --save-data instead of collecting")
    args = ap.parse_args()
    import torch
    assert torch.cuda.is_available()
    lgf.load_library()
    rng = np.random.Generator(np.random.Philox(key=args.seed0))
    Xs, Ys, Ws, meta = [], [], [], []
    t_start = time.time()
    if args.from_data:
        d = np.load(args.from_data)
        Xs, Ys, Ws = [d["X"].astype(np.float64)], [d["R"].astype(np.float64)], [d["W"].astype(np.float64)]
        args.configs = 0
    for i in range(args.configs):
        ext = (16,) * 4 if i % 2 == 0 else (24,) * 4
        seed = args.seed0 + i
        eps = 0.3 + 0.7 * float(np.random.Generator(np.random.Philox(key=seed)).random())
        stats, k, th = collect(ext, eps, seed)
        x, y, w = samples_from_log(ext, stats, rng, args.per_bucket)
        Xs.append(x)
        Ys.append(y)
        Ws.append(w)
        meta.append({"extents": ext[0], "eps": eps, "seed": seed, "iters": k, "theta": th})
        if i % 20 == 0:
            print(f"config {i}: L={ext[0]} eps={eps:.3f} iters={k} theta={th:.2e} samples={y.size} "
                  f"({time.time() - t_start:.0f} s)", flush=True)
    X, Rr, W = np.concatenate(Xs), np.concatenate(Ys), np.concatenate(Ws)
    print(f"dataset: {Rr.size} samples from {len(meta)} configurations ({time.time() - t_start:.0f} s)", flush=True)
    if args.save_data:
        np.savez_compressed(args.save_data, X=X.astype(np.float32), R=Rr.astype(np.float32), W=W.astype(np.float32))
    Y = targets(Rr, -16.0 * X[:, 4])
    P32, Pbf, hist, full = train(X, Y, W)
    np.save(args.out, Pbf)
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump({"samples": int(Y.size), "configs": meta, "final_full_loss": full,
                   "loss_first": hist[:5], "loss_last": hist[-5:], "m_range": [M_LO, M_HI],
                   "train_seconds": time.time() - t_start}, f, indent=1)
    print(f"saved {args.out}; full-data loss {full:.5f}", flush=True)


if __name__ == "__main__":
    main()
