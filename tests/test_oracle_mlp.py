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


def test_adam_two_steps_worked_by_hand():
    """Two Adam steps (Kingma & Ba, 2015) on a 3-parameter vector from p = 0,
    beta1 = 0.9, beta2 = 0.999, lr = 0.1, eps = 1e-8, worked out by hand:

    step 1, g1 = (1, -2, 1/2):
      m1 = 0.1 g1 = (1/10, -1/5, 1/20);  v1 = 0.001 g1^2 = (1/1000, 1/250, 1/4000)
      m_hat = m1 / 0.1 = g1;  v_hat = v1 / 0.001 = g1^2 = (1, 4, 1/4)
      p1 = -lr g1 / (|g1| + eps) = (-0.1/(1+eps), 0.2/(2+eps), -0.05/(1/2+eps))
    step 2, g2 = (3, 0, -1):
      m2 = 0.9 m1 + 0.1 g2 = (39/100, -9/50, -11/200)
      v2 = 0.999 v1 + 0.001 g2^2 = (9999/10^6, 999/250000, 4999/(4 10^6))
      1 - 0.9^2 = 19/100;  1 - 0.999^2 = 1999/10^6
      m_hat = (39/19, -18/19, -11/38);  v_hat = (9999/1999, 3996/1999, 4999/7996)
      p2 = p1 - lr m_hat / (sqrt(v_hat) + eps)

    Swapped betas leave step 1 unchanged but not step 2; a missing bias
    correction or sqrt(v) without the correction changes step 1.
    """
    eps = 1e-8
    p1_want = np.array([-0.1 / (1 + eps), 0.2 / (2 + eps), -0.05 / (0.5 + eps)])
    mh2 = np.array([39 / 19, -18 / 19, -11 / 38])
    vh2 = np.array([9999 / 1999, 3996 / 1999, 4999 / 7996])
    p2_want = p1_want - 0.1 * mh2 / (np.sqrt(vh2) + eps)
    m2_want = np.array([39 / 100, -9 / 50, -11 / 200])
    v2_want = np.array([9999e-6, 999 / 250000, 4999 / 4e6])

    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    p, m, v = mlp.adam_step(p, m, v, np.array([1.0, -2.0, 0.5]), 1, 0.1)
    assert np.allclose(m, [0.1, -0.2, 0.05], rtol=1e-14, atol=0)
    assert np.allclose(v, [1e-3, 4e-3, 2.5e-4], rtol=1e-12, atol=0)
    assert np.allclose(p, p1_want, rtol=1e-12, atol=0)
    p, m, v = mlp.adam_step(p, m, v, np.array([3.0, 0.0, -1.0]), 2, 0.1)
    assert np.allclose(m, m2_want, rtol=1e-12, atol=0)
    assert np.allclose(v, v2_want, rtol=1e-12, atol=0)
    assert np.allclose(p, p2_want, rtol=1e-12, atol=0)
    # swapped betas: the same first step, a different second one
    q, mq, vq = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), np.array([1.0, -2.0, 0.5]), 1, 0.1,
                              b1=0.999, b2=0.9)
    assert np.allclose(q, p1_want, rtol=1e-9, atol=0)
    q, mq, vq = mlp.adam_step(q, mq, vq, np.array([3.0, 0.0, -1.0]), 2, 0.1, b1=0.999, b2=0.9)
    assert np.max(np.abs(q - p2_want)) > 1e-3
