"""Parity of the stepping-increment MLP kernels with the float64 oracle."""

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2506_16488_gb300 import ppsp
from workloads import road_like_graph, random_pairs, clique_pairs

pytestmark = pytest.mark.gpu

U = 2.0 ** -24  # fp32 unit roundoff


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    d = {
        "mean": rng.normal(size=12), "std": rng.uniform(0.5, 2.0, size=12),
        "W1": rng.normal(scale=scale, size=(64, 12)), "b1": rng.normal(scale=0.2, size=64),
        "W2": rng.normal(scale=scale / 2, size=(64, 64)), "b2": rng.normal(scale=0.2, size=64),
        "W3": rng.normal(scale=scale, size=(1, 64)), "b3": rng.normal(scale=0.2, size=1),
    }
    return omlp.pack(d).astype(np.float32)


def _gamma(n):
    return n * U / (1 - n * U)


def _fp32_bound(d, feats, n1=13, n2=65, n3=65):
    """First-order bound on |y_fp32 - y_exact| for fp32 evaluation in any
    summation order: gamma_{n+1} * sum of |terms| per dot product, propagated
    through the layers (ReLU is 1-Lipschitz).  The tensor-core kernel sums
    three bf16 terms of every fp32 activation (an exact split up to 2^-24 of
    the value) in 16-product steps per k-chunk: 3 * 16 * chunks + 1 additions
    per dot product, hence n1 = 49, n2 = n3 = 193 for it."""
    f = np.asarray(feats, dtype=np.float32).astype(np.float64)
    x = (f - d["mean"]) / d["std"]
    ex = np.abs(x) * 3 * U
    z1 = x @ d["W1"].T + d["b1"]
    e1 = _gamma(n1) * (np.abs(x) @ np.abs(d["W1"]).T + np.abs(d["b1"])) + ex @ np.abs(d["W1"]).T
    h1 = np.maximum(z1, 0)
    z2 = h1 @ d["W2"].T + d["b2"]
    e2 = _gamma(n2) * (h1 @ np.abs(d["W2"]).T + np.abs(d["b2"])) + (e1 + h1 * U) @ np.abs(d["W2"]).T
    h2 = np.maximum(z2, 0)
    e3 = _gamma(n3) * (h2 @ np.abs(d["W3"]).T + np.abs(d["b3"])) + (e2 + h2 * U) @ np.abs(d["W3"]).T
    return e3[:, 0]


@pytest.mark.parametrize("count", [1, 15, 16, 17, 300, 4099])
def test_inference_matches_oracle_within_fp32_bound(count):
    # 16 samples per warp on the tensor cores: single, partial, exact and
    # ragged tiles, and more tiles than the CTAs of one pass
    p = _params(1)
    rng = np.random.default_rng(2)
    feats = rng.normal(scale=2.0, size=(count, 12)).astype(np.float32)
    m = ppsp.DeltaModel(p)
    y = m.predict(feats).astype(np.float64)
    d = omlp.inference_params(p)
    y_ref, _ = omlp.forward(d, feats)
    bound = _fp32_bound(d, feats, 49, 193, 193)
    assert np.all(np.abs(y - y_ref) <= 2 * bound + 1e-30), np.max(np.abs(y - y_ref) / bound)
    # the bound separates rounding from real mistakes: the oracle with a
    # planted mistake (second-layer weights transposed, or the output bias
    # dropped) lands outside it on most samples
    for planted in ("W2T", "b3"):
        bad = {k: np.array(v, copy=True) for k, v in d.items()}
        if planted == "W2T":
            bad["W2"] = bad["W2"].T.copy()
        else:
            bad["b3"][:] = 0.0
        y_bad, _ = omlp.forward(bad, feats)
        assert np.mean(np.abs(y_bad - y_ref) > 2 * bound) > 0.5, planted
    assert np.array_equal(m.params(), p)
    m.close()


@pytest.mark.parametrize("count", [37, 256, 3001])
def test_gradient_matches_oracle(count):
    # 16 samples per warp on the tensor cores: ragged last tile, several
    # tiles per warp
    p = _params(3)
    rng = np.random.default_rng(4)
    feats = rng.normal(size=(count, 12)).astype(np.float32)
    labels = rng.normal(size=count).astype(np.float32)
    m = ppsp.DeltaModel(p)
    g, loss = m.grad(feats, labels)
    d = omlp.inference_params(p)
    loss_ref, gref = omlp.loss_and_grad(d, feats, labels.astype(np.float64))
    gref = omlp.pack(gref)
    # fp32 accumulation over the samples and 64-term sums: relative error of
    # order (count + 64) * 2^-24 of each block's magnitude (2e-4 at 3,001
    # samples in the worst case; the sums are random-signed, so far less)
    assert abs(loss - loss_ref) <= 1e-4 * max(1.0, loss_ref)
    for name, size in omlp.SIZES:
        lo = sum(s for nm, s in omlp.SIZES[:[n for n, _ in omlp.SIZES].index(name)])
        blk, ref = g[lo:lo + size], gref[lo:lo + size]
        scale = max(np.abs(ref).max(), 1e-12)
        assert np.all(np.abs(blk - ref) <= 1e-4 * scale), name
    assert np.all(g[:24] == 0)
    m.close()


def test_adam_step_matches_oracle_and_training_converges():
    p = _params(5, scale=0.2)
    rng = np.random.default_rng(6)
    feats = rng.normal(size=(400, 12)).astype(np.float32)
    labels = (0.5 * feats[:, 0] - feats[:, 3]).astype(np.float32)
    m = ppsp.DeltaModel(p)
    first = m.train(feats, labels, 1, 1e-2)
    # one Adam step from the same start, in float64 on the same bf16-rounded forward
    d = omlp.inference_params(p)
    loss_ref, g = omlp.loss_and_grad(d, feats, labels.astype(np.float64))
    assert abs(first - loss_ref) <= 1e-4 * max(1.0, loss_ref)
    pref, _, _ = omlp.adam_step(p.astype(np.float64), np.zeros(p.shape), np.zeros(p.shape), omlp.pack(g), 1, 1e-2)
    got = m.params().astype(np.float64)
    # Adam's first step moves each parameter by lr * g/|g| (= +-lr) unless |g| is
    # tiny; allow a sign flip only where the oracle gradient is within fp32 noise.
    diff = np.abs(got - pref)
    small = np.abs(omlp.pack(g)) < 1e-6 * np.abs(omlp.pack(g)).max()
    assert np.all((diff <= 1e-5 + 1e-6 * np.abs(pref)) | small)
    last = m.train(feats, labels, 300, 1e-2)
    assert last < 0.05 * first
    m.close()


def test_plan_with_model_keeps_answers_and_uses_features():
    g = road_like_graph(96, seed=61)
    pairs = np.concatenate([random_pairs(g, 60, 62), clique_pairs(g, 6, 63)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    with ppsp.Graph.from_csr(g) as G:
        plan = G.plan(pairs, mode="bidastar")
        feats = plan.features()
        assert feats.shape[1] == 12 and feats.shape[0] >= 2
        assert np.all(feats[:, 9] >= 1.0)  # log2(1 + |V_q|) >= log2(3)
        plan.close()
        for bias in (-6.0, 0.0, 4.0):
            p = _params(7)
            p[-1] = bias  # b3: the prediction is dominated by the bias
            model = ppsp.DeltaModel(p)
            G.set_delta_model("bidastar", model)
            G.set_delta_model("bids", model)
            for mode in ("bidastar", "bids"):
                assert np.array_equal(G.batch(pairs, mode=mode), want)
            G.set_delta_model("bidastar", None)
            G.set_delta_model("bids", None)
            model.close()
