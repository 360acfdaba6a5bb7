"""Pins for the float64 MLP reference (runs without a GPU)."""

import numpy as np

from oracle import mlp


def _params(rng, scale=0.3):
    d = {
        "mean": rng.normal(size=mlp.NF), "std": rng.uniform(0.5, 2.0, size=mlp.NF),
        "W1": rng.normal(scale=scale, size=(mlp.H, mlp.NF)), "b1": rng.normal(scale=0.1, size=mlp.H),
        "W2": rng.normal(scale=scale / 2, size=(mlp.H, mlp.H)), "b2": rng.normal(scale=0.1, size=mlp.H),
        "W3": rng.normal(scale=scale, size=(1, mlp.H)), "b3": rng.normal(scale=0.1, size=1),
    }
    return mlp.pack(d)


def test_layout_size():
    assert mlp.NPARAMS == 12 + 12 + 64 * 12 + 64 + 64 * 64 + 64 + 64 + 1
    p = np.arange(mlp.NPARAMS, dtype=np.float64)
    d = mlp.unpack(p)
    assert d["W1"][1, 0] == 24 + 12 and d["b3"][0] == mlp.NPARAMS - 1
    assert np.array_equal(mlp.pack(d), p)


def test_bf16_rounding_definition():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5, 3.0e-3, 65504.0],
                 dtype=np.float32)
    r = mlp.to_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # tie, round to even (mantissa ...0)
    assert r[2] == 1.0 + 2 ** -6       # tie, round to even (mantissa ...10)
    assert r[3] == 1.0 + 2 ** -7       # exactly representable
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2 ** -8
    assert r[6] == 65536.0             # 65504 rounds up to 2^16


def test_hand_computed_network():
    d = {k: np.zeros_like(v, dtype=np.float64) for k, v in mlp.unpack(np.zeros(mlp.NPARAMS)).items()}
    d["std"] = np.ones(mlp.NF)
    d["W1"][0, 0] = 2.0      # h1_0 = relu(2 x0 - 1)
    d["b1"][0] = -1.0
    d["W1"][1, 1] = -1.0     # h1_1 = relu(-x1)
    d["W2"][0, 0] = 3.0      # h2_0 = relu(3 h1_0 + h1_1 + 0.5)
    d["W2"][0, 1] = 1.0
    d["b2"][0] = 0.5
    d["W3"][0, 0] = -0.25    # y = -0.25 h2_0 + 4
    d["b3"][0] = 4.0
    feats = np.zeros((3, mlp.NF), dtype=np.float32)
    feats[0, :2] = [1.0, -2.0]   # h1 = (1, 2), h2_0 = 5.5, y = 2.625
    feats[1, :2] = [0.25, 3.0]   # h1 = (0, 0), h2_0 = 0.5, y = 3.875
    feats[2, :2] = [0.0, 0.0]    # h1 = (0, 0), y = 3.875
    y, _ = mlp.forward(d, feats)
    assert np.allclose(y, [2.625, 3.875, 3.875], rtol=0, atol=1e-15)


def test_zero_weights_give_bias():
    rng = np.random.default_rng(0)
    d = mlp.unpack(_params(rng))
    d["W3"][:] = 0.0
    y, _ = mlp.forward(d, rng.normal(size=(5, mlp.NF)))
    assert np.all(y == d["b3"][0])


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    feats = rng.normal(size=(16, mlp.NF))
    labels = rng.normal(size=16)
    loss, g = mlp.loss_and_grad(mlp.unpack(p), feats, labels)
    gflat = mlp.pack(g)
    idx = np.concatenate([rng.choice(np.arange(24, mlp.NPARAMS), size=60, replace=False), [mlp.NPARAMS - 1]])
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp, _ = mlp.loss_and_grad(mlp.unpack(pp), feats, labels)
        lm, _ = mlp.loss_and_grad(mlp.unpack(pm), feats, labels)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, gflat[i])


def test_adam_reduces_loss_on_a_linear_target():
    rng = np.random.default_rng(2)
    p = _params(rng, scale=0.2)
    feats = rng.normal(size=(200, mlp.NF))
    labels = feats[:, 0] * 0.5 - feats[:, 3]
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    first, _ = mlp.loss_and_grad(mlp.unpack(p), feats, labels)
    for t in range(1, 301):
        _, g = mlp.loss_and_grad(mlp.unpack(p), feats, labels)
        p, m, v = mlp.adam_step(p, m, v, mlp.pack(g), t, 1e-2)
    last, _ = mlp.loss_and_grad(mlp.unpack(p), feats, labels)
    assert last < 0.05 * first
    # mean and std are never moved (their gradient is zero)
    assert np.array_equal(p[:24], _params(np.random.default_rng(2), scale=0.2)[:24])
