"""Autotuner: every configuration it tries returns the same distances, and the
chosen options are cached per (graph, batch shape, mode)."""

import json
import os

import numpy as np
import pytest

import oracle
from paper_2506_16488_gb300 import autotune, ppsp
from workloads import clique_pairs, random_pairs, road_like_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def test_tune_keeps_answers_and_caches(tmp_path):
    g = road_like_graph(96, seed=95)
    pairs = np.concatenate([random_pairs(g, 80, 96), clique_pairs(g, 8, 97)])
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    cache = str(tmp_path / "cache.json")
    with ppsp.Graph.from_csr(g) as G:
        opts = autotune.cached_or_tune(G, pairs, "bidastar", path=cache, budget_s=30, reps=1)
        assert opts["mode"] == "bidastar"
        assert np.array_equal(G.batch(pairs, **opts), want)
        with open(cache) as f:
            saved = json.load(f)
        assert autotune.signature(G, pairs, "bidastar") in saved
        # a second call is served from the cache
        assert autotune.cached_or_tune(G, pairs, "bidastar", path=cache, allow_tune=False) == opts
