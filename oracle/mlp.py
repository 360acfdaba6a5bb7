"""Float64 reference of the stepping-threshold MLP.  TEST INFRASTRUCTURE ONLY.

The paper tunes Delta of Delta*-stepping by doubling until the time stops
improving (Sec. 6.1, "Tested Algorithms"); Delta changes only speed, never the
answer (Theorems 3.3/3.4 hold for any stepping schedule).  The library learns
Delta instead with a small MLP; this module is the plain definition of that
network, written out in float64:

  x  = (features - mean) / std                                 12 inputs
  h1 = relu(W1 x + b1)        W1: 64 x 12 (bf16 values), b1: 64 (fp32)
  h2 = relu(W2 h1 + b2)       W2: 64 x 64 (bf16 values), b2: 64 (fp32)
  y  = W3 h2 + b3             W3:  1 x 64 (bf16 values), b3: 1  (fp32)

y predicts log2(Delta_best / Delta_default).  The flat parameter vector is
[mean(12), std(12), W1(768, row-major), b1(64), W2(4096), b2(64), W3(64), b3(1)]
= 5,081 floats.  Training minimises the mean squared error with Adam
(Kingma & Ba, 2015: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
p <- p - lr * m_hat / (sqrt(v_hat) + eps)); mean and std are not trained.
"""

from __future__ import annotations

import numpy as np

NF, H = 12, 64
SIZES = [("mean", NF), ("std", NF), ("W1", H * NF), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H), ("b3", 1)]
NPARAMS = sum(s for _, s in SIZES)
BF16_PARTS = ("W1", "W2", "W3")


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, size in SIZES:
        out[name] = p[o:o + size]
        o += size
    out["W1"] = out["W1"].reshape(H, NF)
    out["W2"] = out["W2"].reshape(H, H)
    out["W3"] = out["W3"].reshape(1, H)
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even); returns
    the rounded values as float64.  NaN inputs are not expected."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def inference_params(p32: np.ndarray) -> dict:
    """Parameters as the inference kernel sees them: W in bf16, the rest fp32."""
    d = unpack(np.asarray(p32, dtype=np.float32).astype(np.float64))
    for name in BF16_PARTS:
        d[name] = to_bf16(np.asarray(d[name], dtype=np.float32))
    return d


def forward(d: dict, feats: np.ndarray):
    """Returns (y [N], cache) in float64."""
    x = (np.asarray(feats, dtype=np.float32).astype(np.float64) - d["mean"]) / d["std"]
    z1 = x @ d["W1"].T + d["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ d["W2"].T + d["b2"]
    h2 = np.maximum(z2, 0.0)
    y = (h2 @ d["W3"].T)[:, 0] + d["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(d: dict, feats: np.ndarray, labels: np.ndarray):
    """Mean squared error and its gradient w.r.t. every parameter (mean/std: 0)."""
    y, (x, z1, h1, z2, h2) = forward(d, feats)
    n = y.shape[0]
    r = y - np.asarray(labels, dtype=np.float64)
    loss = float(np.mean(r * r))
    gy = 2.0 * r / n
    g = {"mean": np.zeros(NF), "std": np.zeros(NF)}
    g["W3"] = gy[None, :] @ h2
    g["b3"] = np.array([gy.sum()])
    gh2 = gy[:, None] * d["W3"]
    gz2 = gh2 * (z2 > 0)
    g["W2"] = gz2.T @ h1
    g["b2"] = gz2.sum(axis=0)
    gh1 = gz2 @ d["W2"]
    gz1 = gh1 * (z1 > 0)
    g["W1"] = gz1.T @ x
    g["b1"] = gz1.sum(axis=0)
    return loss, g


def adam_step(p: np.ndarray, m: np.ndarray, v: np.ndarray, grad: np.ndarray, t: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
