"""The learned multiplier on the GPU against its CPU oracle (oracle/lgf_mlp_oracle.py).

* tensor-core inference (BF16 weights, FP32 accumulation) vs the oracle's
  BF16-emulating forward pass;
* training gradients vs the oracle's hand-written backward pass (which is
  itself checked against finite differences in test_mlp_oracle.py);
* the learned step with a constant multiplier and the F-monotonicity
  fallback vs the FA oracle driven the same way;
* the mode log (training data) vs the same sums formed from the oracle's
  Fourier-space divergence.
"""

import numpy as np
import pytest

from oracle import lgf_mlp_oracle as M
from oracle import lgf_oracle as O
from paper_1206_0675_gb300 import fields, lgf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    lgf.load_library()
    return torch


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    p[M.OFF_W4:M.OFF_B4] = rng.standard_normal(64) * 0.3
    p[M.OFF_B1:M.OFF_W2] = rng.standard_normal(64) * 0.1
    p[M.OFF_B2:M.OFF_W3] = rng.standard_normal(64) * 0.1
    p[M.OFF_B3:M.OFF_W4] = rng.standard_normal(64) * 0.1
    p[M.OFF_B4] = 0.2
    return p


def bf16_bits(p):
    return (M.bf16_round(p).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def gpu_eval(torch, bits, X):
    Pb = torch.from_numpy(bits.view(np.int16).copy()).cuda()
    Xd = torch.tensor(X, dtype=torch.float32).cuda()
    m = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    lgf.lgf_mlp_eval(Pb.data_ptr(), Xd.data_ptr(), X.shape[0], m.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return m.cpu().numpy().astype(np.float64)


def _bf16_other(h):
    """For each entry of h (float64), its BF16 rounding r and the adjacent BF16
    value on the other side of h, and the midpoint between the two."""
    r = M.bf16_round(h)
    bits = r.astype(np.float32).view(np.uint32).astype(np.int64)
    up = (h > r) == (r >= 0)  # move away from zero when h lies beyond r in magnitude
    ob = np.where(up, bits + 0x10000, bits - 0x10000)
    ob = np.where((r == 0) & (h < 0), 0x80010000, ob)
    other = (ob & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    return r, other, 0.5 * (r + other)


def _rounding_options(a, S, nterms, cap):
    """Every BF16 rounding of relu(a) that an FP32 accumulation of nterms products
    could produce: a entry whose exact value lies within the accumulation error
    bound (2 nterms 2^-24 S) of a BF16 rounding midpoint may round either way.
    None when more than cap entries are in doubt."""
    h = np.maximum(a, 0.0)
    r, other, mid = _bf16_other(h)
    dmax = 2.0 * nterms * 2.0 ** -24 * S
    doubt = np.nonzero((np.abs(h - mid) <= dmax) & (h > 0))[0]
    if len(doubt) > cap:
        return None
    opts = []
    for mask in range(1 << len(doubt)):
        v = r.copy()
        for j, i in enumerate(doubt):
            if mask >> j & 1:
                v[i] = other[i]
        opts.append(v)
    return opts


def test_inference_matches_bf16_oracle_row_by_row(torch):
    """Tensor-core inference against the oracle's BF16 emulation, row by row.

    The kernel rounds the hidden activations h1 and h2 to BF16 (the operands
    of the next mma) after accumulating them in FP32; the oracle accumulates
    in FP64.  Where an exact activation lies within the FP32 accumulation
    error of a BF16 rounding midpoint, the two may round it to neighbouring
    BF16 values (2^-8 apart, relative): that, and nothing else, may separate
    them by more than FP32 rounding.  So every row must agree to 1e-5
    relative with one of the oracle's evaluations over the admissible
    roundings of its doubtful activations."""
    rng = np.random.default_rng(0)
    p = random_params(0)
    X = rng.random((1000 + 13, 8))  # ragged tail: not a multiple of the 16-row tile
    m_gpu = gpu_eval(torch, bf16_bits(p), X)
    W1, b1, W2, b2, W3, b3, w4, b4 = M.unpack(M.bf16_round(p))
    Xb = M.bf16_round(X)
    n_doubt, worst = 0, 0.0
    for i in range(X.shape[0]):
        a1 = W1 @ Xb[i] + b1
        S1 = np.abs(W1) @ np.abs(Xb[i]) + np.abs(b1)
        best = np.inf
        opts1 = _rounding_options(a1, S1, 9, 6)
        assert opts1 is not None, i
        for h1 in opts1:
            a2 = W2 @ h1 + b2
            S2 = np.abs(W2) @ np.abs(h1) + np.abs(b2)
            opts2 = _rounding_options(a2, S2, 65, 6)
            assert opts2 is not None, i
            for h2 in opts2:
                h3 = np.maximum(W3 @ h2 + b3, 0.0)
                m = M.softplus(w4 @ h3 + b4)
                best = min(best, abs(m_gpu[i] - m) / m)
        n_doubt += (len(opts1) > 1) or best > 0
        worst = max(worst, best)
        assert best < 2e-5, (i, best)
    print(f"rows {X.shape[0]}, worst relative deviation from an admissible BF16 evaluation {worst:.2e}")


def test_gradient_matches_oracle(torch):
    rng = np.random.default_rng(1)
    p = random_params(1).astype(np.float32)
    n = 777
    X = rng.random((n, 8)).astype(np.float32)
    Y = (rng.standard_normal(n) * 0.2).astype(np.float32)
    W = rng.random(n) + 0.2
    W = (W / W.mean()).astype(np.float32)
    loss_ref, g_ref = M.loss_and_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                                      W.astype(np.float64))
    dev = torch.device("cuda")
    Pd, Xd, Yd, Wd = (torch.from_numpy(a).to(dev) for a in (p, X, Y, W))
    g = torch.empty(M.NPARAM, dtype=torch.float32, device=dev)
    loss = lgf.lgf_mlp_loss_grad(Pd.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Wd.data_ptr(), n, g.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - loss_ref) < 1e-5 * loss_ref
    assert np.max(np.abs(g - g_ref)) < 1e-4 * np.max(np.abs(g_ref))


def test_training_reduces_loss(torch):
    rng = np.random.default_rng(2)
    n = 20000
    X = rng.random((n, 8)).astype(np.float32)
    Y = (0.15 * np.sin(3 * X[:, 0]) - 0.1 * X[:, 4] + 0.05 * X[:, 5]).astype(np.float32)
    W = np.ones(n, dtype=np.float32)
    dev = torch.device("cuda")
    Pd = torch.from_numpy(M.init_params(3).astype(np.float32)).to(dev)
    adam = torch.zeros(2 * M.NPARAM, dtype=torch.float32, device=dev)
    Xd, Yd, Wd = (torch.from_numpy(a).to(dev) for a in (X, Y, W))
    st = torch.cuda.current_stream().cuda_stream
    g = torch.empty(M.NPARAM, dtype=torch.float32, device=dev)
    l0 = lgf.lgf_mlp_loss_grad(Pd.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Wd.data_ptr(), n, g.data_ptr(), st)
    hist = lgf.lgf_mlp_train(Pd.data_ptr(), adam.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Wd.data_ptr(), n, 1024,
                             600, 1e-3, 11, 0, st)
    l1 = lgf.lgf_mlp_loss_grad(Pd.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Wd.data_ptr(), n, g.data_ptr(), st)
    assert hist.shape == (600,) and np.all(np.isfinite(hist))
    assert l1 < 0.1 * l0
    # the oracle agrees on the trained network's loss
    lo, _ = M.loss_and_grad(Pd.cpu().numpy().astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                            W.astype(np.float64))
    assert abs(lo - l1) < 1e-4 * lo + 1e-9


def constant_multiplier_bits(z0):
    p = np.zeros(M.NPARAM)
    p[M.OFF_B4] = z0
    return bf16_bits(p)


def oracle_learned_fix(U, K, m, n_steps):
    """Algorithm 1 with filter K*m and the fallback: a step that lowers F is redone with K."""
    F, th, D = O.measure(U)
    Fs, ths, nf = [F], [th], 0
    for _ in range(n_steps):
        Un, _ = O.fa_step(U, 0.08, K * m, D)
        Fn, thn, Dn = O.measure(Un)
        if Fn < F:
            nf += 1
            Un, _ = O.fa_step(U, 0.08, K, D)
            Fn, thn, Dn = O.measure(Un)
        U, F, th, D = Un, Fn, thn, Dn
        Fs.append(F)
        ths.append(th)
    return np.array(Fs), np.array(ths), nf


@pytest.mark.parametrize("alpha_scale,z0", [(1.0, 0.7), (1.6, 3.0)])
def test_learned_constant_multiplier_and_fallback_match_oracle(torch, alpha_scale, z0):
    """z0 = 0.7: m = softplus(0.7) = 1.10, no fallback.  z0 = 3: m clamps to 2 and,
    with alpha scaled by 1.6, steps overshoot and are redone with the plain filter."""
    ext = (6, 4, 8, 4)
    alpha = 0.08 * alpha_scale
    U = fields.random_links(ext, eps=0.9, seed=21)
    bits = constant_multiplier_bits(z0)
    m = float(np.clip(gpu_eval(torch, bits, np.zeros((1, 8)))[0], 0.25, 2.0))
    n = 30
    with lgf.Lattice(ext, "fp64", learned=True) as lat:
        lat.load_preconditioner(bits)
        lat.set_links(U)
        Fh, Th = lat.set_trace(n + 1)
        it, F, th, conv = lat.fix(0.0, n, alpha)
        nf = lat.fallbacks()
    K = O.fa_filter(ext, alpha)
    Fo, tho, nfo = oracle_learned_fix(U, K, m, n)
    assert it == n
    assert nf == nfo
    if z0 > 1:
        assert nf > 0
    assert np.max(np.abs(Fh - Fo) / np.abs(Fo)) < 1e-11
    assert np.max(np.abs(Th - tho) / tho) < 1e-9


def test_learned_step_api_redoes_rejected_steps(torch):
    ext = (4, 4, 4, 6)
    U = fields.random_links(ext, eps=0.9, seed=5)
    bits = constant_multiplier_bits(3.0)
    with lgf.Lattice(ext, "fp64", learned=True) as lat:
        lat.load_preconditioner(bits)
        lat.set_links(U)
        F_prev = lat.measure()[0]
        for _ in range(10):
            lat.step(0.13)
            F, _ = lat.measure()
            assert F >= F_prev  # every accepted step raises F
            F_prev = F


def test_learned_level_zero_is_the_plain_method(torch):
    """With the learned level at 0 no step uses the table: a learned handle
    runs the plain method bit for bit (a multiplier of 2 would otherwise
    overshoot at this alpha and be redone)."""
    ext = (6, 4, 8, 4)
    U = fields.random_links(ext, eps=0.9, seed=21)
    out = []
    for learned in (True, False):
        with lgf.Lattice(ext, "fp64", learned=learned) as lat:
            if learned:
                lat.load_preconditioner(constant_multiplier_bits(3.0))
                lat.set_learned_theta(0.0)
            lat.set_links(U)
            Fh, Th = lat.set_trace(31)
            it, F, th, conv = lat.fix(0.0, 30, 0.128)
            out.append((Fh.copy(), Th.copy(), lat.get_links(), lat.fallbacks() if learned else 0))
    a, b = out
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert a[3] == 0


def test_learned_level_gates_steps_by_theta(torch):
    """Steps from links with theta at or above the level use the plain filter
    (no learned flag in the trace); the others use the table (m = 1.10)."""
    ext = (6, 4, 8, 4)
    U = fields.random_links(ext, eps=0.9, seed=21)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        Fp, Tp = lat.set_trace(41)
        lat.fix(0.0, 40, 0.08)
    level = float(Tp[12])  # about a third of the way down
    with lgf.Lattice(ext, "fp64", learned=True) as lat:
        lat.load_preconditioner(constant_multiplier_bits(0.7))
        lat.set_learned_theta(level)
        lat.set_links(U)
        Fh, Th, Fl, Dh = lat.set_trace(41, flags=True)
        it, F, th, conv = lat.fix(0.0, 40, 0.08)
        assert lat.fallbacks() == 0
    on = [(Fl[k] & lgf.LGF_TRACE_LEARNED) != 0 for k in range(1, 41)]
    for k in range(1, 41):
        assert on[k - 1] == (Th[k - 1] < level), k
    assert any(on) and not all(on)
    # until the level is reached the run is the plain one
    first = on.index(True) + 1
    assert np.array_equal(Fh[:first], Fp[:first]) and np.array_equal(Th[:first], Tp[:first])
    with pytest.raises(lgf.LgfError):
        lat2 = lgf.Lattice(ext, "fp64")
        try:
            lat2.set_learned_theta(1e-6)  # not a learned handle
        finally:
            lat2.close()


def packed_hat(D):
    """Fourier transforms of the four packed divergence fields from the oracle's 3x3 Delta_A."""
    Dh = O.fft4(D)
    return np.stack([-1j * Dh[..., 0, 0] + Dh[..., 1, 1], Dh[..., 0, 1], Dh[..., 0, 2], Dh[..., 1, 2]])


def test_mode_log_matches_oracle(torch):
    ext = (6, 4, 4, 6)
    steps = 3
    U = fields.random_links(ext, eps=0.8, seed=2)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        lat.set_mode_log(True)
        for _ in range(steps):
            lat.step(0.08)
        stats = lat.get_mode_log()
    lx, ly, lz, lt = ext
    H = [L // 2 + 1 for L in ext]
    t, z, y, x = np.meshgrid(range(lt), range(lz), range(ly), range(lx), indexing="ij")
    f = [np.minimum(c, L - c) for c, L in ((x, lx), (y, ly), (z, lz), (t, lt))]
    cls = ((f[3] * H[2] + f[2]) * H[1] + f[1]) * H[0] + f[0]
    nclass = int(np.prod(H))
    ref = np.zeros_like(stats)
    Ucur = U
    F, th, D = O.measure(Ucur)
    prev = packed_hat(D)
    prev2 = None
    th_before = 0.0
    for k in range(steps):
        b = int(np.clip(4 - 2 * np.floor(2 * np.log10(th)) / 2, 0, 39))
        Ucur, _ = O.fa_step(Ucur, 0.08, D=D)
        F, th_new, D = O.measure(Ucur)
        cur = packed_hat(D)
        num = np.sum(np.real(np.conj(prev) * cur), axis=0)
        den = np.sum(np.abs(prev) ** 2, axis=0)
        ref[b, :, 0] += np.bincount(cls.ravel(), num.ravel(), nclass)
        ref[b, :, 1] += np.bincount(cls.ravel(), den.ravel(), nclass)
        ref[b, :, 2] += np.bincount(cls.ravel(), minlength=nclass)
        ref[b, :, 3] += np.bincount(cls.ravel(), minlength=nclass) * min(k / 10000.0, 1.0)
        ref[b, :, 4] += np.bincount(cls.ravel(), minlength=nclass) * (M.rate_feature(th, th_before) if k else 0.0)
        if prev2 is not None:
            ref[b, :, 5] += np.bincount(cls.ravel(), np.sum(np.real(np.conj(prev2) * prev), axis=0).ravel(), nclass)
            ref[b, :, 6] += np.bincount(cls.ravel(), np.sum(np.abs(prev2) ** 2, axis=0).ravel(), nclass)
        prev2, prev, th_before, th = prev, cur, th, th_new
    scale = np.max(np.abs(ref[..., 1]))
    assert np.array_equal(stats[..., 2], ref[..., 2])
    assert np.max(np.abs(stats[..., 0] - ref[..., 0])) < 1e-10 * scale
    assert np.max(np.abs(stats[..., 1] - ref[..., 1])) < 1e-10 * scale
    assert np.max(np.abs(stats[..., 3] - ref[..., 3])) < 1e-6
    assert np.max(np.abs(stats[..., 4] - ref[..., 4])) < 1e-3
    assert np.max(np.abs(stats[..., 5] - ref[..., 5])) < 1e-10 * scale
    assert np.max(np.abs(stats[..., 6] - ref[..., 6])) < 1e-10 * scale
    assert np.any(ref[..., 6] > 0)


def test_trained_preconditioner_gains_on_slow_fields(torch):
    """The committed network (trained on 16^4 and 24^4 trajectories) against plain
    FA-SD on twelve held-out rough 16^4 fields (eps = 1, seeds 100-111), to
    theta < 1e-12: fewer iterations in all, and on nearly every field (one of
    these fields, seed 105, sits on a plateau of theta near 1e-11 for
    thousands of steps, which the larger steps lengthen); same gauge orbit
    (plaquette unchanged); every accepted step raises F."""
    from paper_1206_0675_gb300.preconditioner import DEFAULT_WEIGHTS
    weights = np.load(DEFAULT_WEIGHTS)
    ext = (16, 16, 16, 16)
    total_plain = total_learned = wins = 0
    for seed in range(100, 112):
        U = fields.random_links(ext, eps=1.0, seed=seed)
        with lgf.Lattice(ext, "fp64") as lat:
            lat.set_links(U)
            it_p, F_p, th_p, conv_p = lat.fix(1e-12, 20000, 0.08)
        with lgf.Lattice(ext, "fp64", learned=True) as lat:
            lat.load_preconditioner(weights)
            lat.set_links(U)
            Fh, _ = lat.set_trace(20001)
            it_l, F_l, th_l, conv_l = lat.fix(1e-12, 20000, 0.08)
            U_l = lat.get_links()
        assert conv_p and conv_l
        assert np.all(np.diff(Fh[: it_l + 1]) >= 0)
        assert abs(O.plaquette(U_l) - O.plaquette(U)) < 1e-12
        total_plain += it_p
        total_learned += it_l
        wins += it_l < it_p
    print(f"iterations to 1e-12 on twelve held-out 16^4 eps=1 fields: plain {total_plain}, learned {total_learned}, "
          f"learned fewer on {wins}")
    assert total_learned < 0.9 * total_plain
    assert wins >= 10


def test_trained_preconditioner_on_fast_fields(torch):
    """On smooth fields that plain FA-SD fixes in a few dozen steps the network
    keeps the multiplier near 1 on the classes that contract fast (their own
    contraction is an input) and costs no iterations; the result stays on the
    gauge orbit."""
    from paper_1206_0675_gb300.preconditioner import DEFAULT_WEIGHTS
    weights = np.load(DEFAULT_WEIGHTS)
    ext = (16, 16, 16, 16)
    U = fields.random_links(ext, eps=0.7, seed=100)
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        it_p, _, _, conv_p = lat.fix(1e-12, 20000, 0.08)
    with lgf.Lattice(ext, "fp64", learned=True) as lat:
        lat.load_preconditioner(weights)
        lat.set_links(U)
        it_l, _, _, conv_l = lat.fix(1e-12, 20000, 0.08)
        U_l = lat.get_links()
    print(f"iterations to 1e-12 on a held-out 16^4 eps=0.7 field: plain {it_p}, learned {it_l}")
    assert conv_p and conv_l
    assert it_l <= it_p
    assert abs(O.plaquette(U_l) - O.plaquette(U)) < 1e-12
