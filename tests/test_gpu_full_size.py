"""Parity at the full workload sizes, in the launch configuration the bench
times: the whole batch runs as one plan (learned Delta, CUDA-graph replay,
default block and team layout) and a stratified sample of its answers is
checked against the oracle's Dijkstra one query at a time.  Sizes: the
1024^2 road-like batch of 1,000 BiD-A* queries, RMAT-22 with its three query
patterns (AUTO strategy), the 2048^2 mixed batch (AUTO), and the 4096^2
serving graph with uint64 distances.
"""

import numpy as np
import pytest

import oracle
from paper_2506_16488_gb300 import learned_delta, ppsp
from workloads import config_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _run_plan(G, pairs, **opts):
    import torch

    stream = torch.cuda.Stream()
    out = torch.zeros(pairs.shape[0], dtype=torch.int64, device="cuda")
    plan = G.plan(pairs, stream=stream.cuda_stream, cuda_graph=True, **opts)
    for _ in range(2):  # the second run replays the captured graph
        plan.run(out.data_ptr())
        plan.sync()
    plan.close()
    return out.cpu().numpy().view(np.uint64).copy()


def _sample(labels, per, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.choice(np.nonzero(labels == b)[0], size=min(per, int((labels == b).sum())),
                                      replace=False) for b in np.unique(labels)])


def _check(g, pairs, got, idx):
    import os

    want = oracle.pairs_threaded(g.offsets, g.targets, g.weights, pairs[idx], os.cpu_count() or 1)
    assert np.array_equal(got[idx], want), np.nonzero(got[idx] != want)


def _batch(wl):
    names = list(wl["batches"])
    pairs = np.concatenate([wl["batches"][k] for k in names])
    labels = np.concatenate([np.full(wl["batches"][k].shape[0], j) for j, k in enumerate(names)])
    if "labels" in wl:
        labels = np.asarray(wl["labels"])
    return pairs, labels


def test_road_1024_batch_of_1000():
    wl = config_workload(2)
    g = wl["graph"]
    pairs, labels = _batch(wl)
    with ppsp.Graph.from_csr(g) as G:
        G.set_delta_model("bidastar", learned_delta.load_model("bidastar"))
        got = _run_plan(G, pairs, mode="bidastar", strategy="multi")
    _check(g, pairs, got, _sample(labels, 12, 1))


def test_rmat22_patterns_auto():
    wl = config_workload(3)
    g = wl["graph"]
    pairs, labels = _batch(wl)
    with ppsp.Graph.from_csr(g, with_coords=False) as G:
        G.set_delta_model("bids", learned_delta.load_model("bids"))
        got = _run_plan(G, pairs, mode="bids", strategy="auto")
    _check(g, pairs, got, _sample(labels, 2, 2))


def test_road_2048_mixed_auto():
    wl = config_workload(4)
    g = wl["graph"]
    pairs, _ = _batch(wl)
    labels = np.r_[np.zeros(1552, dtype=np.int64), np.ones(pairs.shape[0] - 1552, dtype=np.int64)]  # pairs, clique
    with ppsp.Graph.from_csr(g) as G:
        G.set_delta_model("bidastar", learned_delta.load_model("bidastar"))
        got = _run_plan(G, pairs, mode="bidastar", strategy="auto")
    _check(g, pairs, got, _sample(labels, 4, 3))


def test_road_4096_uint64():
    wl = config_workload(5)
    g = wl["graph"]
    pairs = wl["batches"]["random"][:152]
    with ppsp.Graph.from_csr(g) as G:
        G.set_delta_model("bidastar", learned_delta.load_model("bidastar"))
        got = _run_plan(G, pairs, mode="bidastar", dist_bits=64)
    _check(g, pairs, got, np.arange(0, 152, 38))
