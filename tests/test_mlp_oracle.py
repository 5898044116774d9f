"""Pins of the CPU oracle of the learned multiplier (no GPU)."""

import numpy as np
import pytest

from oracle import lgf_mlp_oracle as M


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    p[M.OFF_W4:M.OFF_B4] = rng.standard_normal(64) * 0.2
    p[M.OFF_B1:M.OFF_W2] = rng.standard_normal(64) * 0.1
    p[M.OFF_B2:M.OFF_W3] = rng.standard_normal(64) * 0.1
    p[M.OFF_B3:M.OFF_W4] = rng.standard_normal(64) * 0.1
    return p


def test_parameter_layout_roundtrip():
    p = random_params(0)
    assert p.size == M.NPARAM == 8961
    assert np.array_equal(M.pack(*M.unpack(p)), p)


def test_initial_network_is_the_plain_filter():
    p = M.init_params(3)
    X = np.random.default_rng(0).random((50, 8))
    m, _ = M.forward(p, X)
    assert np.allclose(m, 1.0, rtol=0, atol=1e-15)


def test_gradient_against_central_differences():
    rng = np.random.default_rng(1)
    p = random_params(1)
    X = rng.random((40, 8))
    Y = rng.standard_normal(40) * 0.2
    Wt = rng.random(40) + 0.1
    loss, g = M.loss_and_grad(p, X, Y, Wt)
    idx = np.concatenate([rng.choice(np.arange(M.OFF_W1, M.OFF_B1), 8), rng.choice(np.arange(M.OFF_W2, M.OFF_B2), 8),
                          rng.choice(np.arange(M.OFF_W3, M.OFF_B3), 8), np.arange(M.OFF_W4, M.OFF_W4 + 8),
                          [M.OFF_B1, M.OFF_B2 + 3, M.OFF_B3 + 5, M.OFF_B4]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, X, Y, Wt)[0] - M.loss_and_grad(pm, X, Y, Wt)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).standard_normal(10000) * np.exp(np.random.default_rng(3).standard_normal(10000) * 5)
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)


def test_targets_and_features():
    r = np.array([0.0, 0.5, -0.28, 0.993, 1.2, -5.0])
    m = np.exp(M.targets_from_stats(r, np.ones_like(r)))
    assert np.allclose(m, [1.0, M.M_HI, 1 / 1.28, M.M_HI, M.M_HI, M.M_LO])
    x = M.features([[0.0, 4.0, 2.0, 1.0]], 3e-10, 2500, 3e-9, 0.75)
    assert np.allclose(x, [[0.0, 1.0, 0.5, 0.25, 10.0 / 16.0, 0.25, -0.5, 0.75]])
    assert M.features([[1, 1, 1, 1]], 1e-3, 0, 1e-1)[0, 6] == 0.0  # no previous step
    x2 = M.features([[1, 1, 1, 1], [2, 2, 2, 2]], 1e-3, 5, 1e-2, [3.0, -7.0])
    assert np.array_equal(x2[:, 7], [1.0, -1.0])                     # class contraction clamped
    assert M.rate_feature(1e-9, 1e-3) == -1.0 and M.rate_feature(1e-3, 1e-9) == 0.5
    assert M.theta_bucket(1e-9) == -9.0 and M.theta_bucket(0.0) == -20.0


def test_training_targets_match_the_oracle_definition():
    from paper_1206_0675_gb300 import preconditioner as P
    rng = np.random.default_rng(5)
    r = rng.uniform(-3, 1.5, 2000)
    bucket = rng.integers(-30, 5, 2000) / 2.0
    assert np.allclose(P.targets(r, bucket), M.targets_from_stats(r, np.ones_like(r), bucket), atol=1e-12)
    assert np.all(P.targets(r, np.full_like(r, -3.5)) == 0.0)
