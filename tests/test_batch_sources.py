"""Source selection of the SSSP-based batch strategies (Sec. 4.3), host only.

VC-SSSP runs one full search from every vertex of a vertex cover of the query
graph G_q; the library enumerates covers of small components exactly and
covers large ones greedily.  The pins: every query is answered from one of its
own endpoints (so the sources form a cover), the exact covers are minimum
(brute force over all vertex subsets of small random query graphs), and the
closed forms of the paper's query-graph patterns (Sec. 4.1): a star needs one
search, a k-clique k - 1, a chain of k vertices floor(k / 2) (every other
vertex).
"""

import itertools

import numpy as np
import pytest

from paper_2506_16488_gb300 import ppsp

NONE = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()


def brute_min_cover(pairs):
    verts = sorted({int(x) for p in pairs for x in p if p[0] != p[1]})
    idx = {v: k for k, v in enumerate(verts)}
    edges = [(1 << idx[int(a)]) | (1 << idx[int(b)]) for a, b in pairs if a != b]
    for r in range(len(verts) + 1):
        for sub in itertools.combinations(range(len(verts)), r):
            m = sum(1 << k for k in sub)
            if all(e & m for e in edges):
                return r
    return len(verts)


def check_cover(pairs, src):
    for (s, t), x in zip(pairs, src):
        if s == t:
            assert x == NONE
        else:
            assert x in (s, t)


def test_patterns_closed_forms():
    v = np.arange(100, 111, dtype=np.uint32)
    clique = np.array([(a, b) for i, a in enumerate(v) for b in v[i + 1:]], dtype=np.uint32)
    src, n = ppsp.batch_sources(clique, "vc")
    check_cover(clique, src)
    assert n == 10
    star = np.array([(5, x) for x in range(10, 74)], dtype=np.uint32)
    assert ppsp.batch_sources(star, "vc")[1] == 1
    assert ppsp.batch_sources(star[:, ::-1], "vc")[1] == 1
    assert ppsp.batch_sources(star[:, ::-1], "sssp")[1] == 64
    for k in (2, 3, 10, 17):
        chain = np.array([(i, i + 1) for i in range(k - 1)], dtype=np.uint32)
        src, n = ppsp.batch_sources(chain, "vc")
        check_cover(chain, src)
        assert n == k // 2, k


def test_plain_sssp_uses_each_source():
    rng = np.random.default_rng(3)
    pairs = rng.integers(0, 50, size=(200, 2)).astype(np.uint32)
    src, n = ppsp.batch_sources(pairs, "sssp")
    for (s, t), x in zip(pairs, src):
        assert x == (NONE if s == t else s)
    assert n == len({int(s) for s, t in pairs if s != t})


@pytest.mark.parametrize("seed", range(16))
def test_exact_cover_is_minimum(seed):
    rng = np.random.default_rng(seed)
    nv = int(rng.integers(2, 15))
    ne = int(rng.integers(1, 3 * nv + 1))
    ids = rng.choice(10 ** 6, size=nv, replace=False).astype(np.uint32)
    pairs = ids[rng.integers(0, nv, size=(ne, 2))]
    src, n = ppsp.batch_sources(pairs, "vc")
    check_cover(pairs, src)
    assert n == brute_min_cover(pairs)
    assert n == len({int(x) for x in src if x != NONE})


def test_components_are_covered_separately():
    # two disjoint triangles and an isolated pair: 2 + 2 + 1
    pairs = np.array([(0, 1), (1, 2), (2, 0), (10, 11), (11, 12), (12, 10), (20, 21)], dtype=np.uint32)
    src, n = ppsp.batch_sources(pairs, "vc")
    check_cover(pairs, src)
    assert n == 5


def test_exact_cover_of_32_vertex_components():
    # the largest exact case: a 32-clique (31) and a 32-cycle (16)
    v = np.arange(32, dtype=np.uint32)
    clique = np.array([(a, b) for i, a in enumerate(v) for b in v[i + 1:]], dtype=np.uint32)
    src, n = ppsp.batch_sources(clique, "vc")
    check_cover(clique, src)
    assert n == 31
    cycle = np.stack([v, np.roll(v, -1)], axis=1)
    src, n = ppsp.batch_sources(cycle, "vc")
    check_cover(cycle, src)
    assert n == 16


def test_greedy_cover_of_large_components():
    # components above the exhaustive limit are covered greedily; the cover
    # must still hold every query, and greedy finds the obvious optimum of a
    # complete bipartite K(3, 40) and of a 100-leaf star
    kb = np.array([(a, 1000 + b) for a in range(3) for b in range(40)], dtype=np.uint32)
    src, n = ppsp.batch_sources(kb, "vc")
    check_cover(kb, src)
    assert n == 3
    star = np.array([(7, 100 + i) for i in range(100)], dtype=np.uint32)
    assert ppsp.batch_sources(star, "vc")[1] == 1
    rng = np.random.default_rng(11)
    pairs = rng.integers(0, 60, size=(300, 2)).astype(np.uint32)
    src, n = ppsp.batch_sources(pairs, "vc")
    check_cover(pairs, src)
    # a maximal matching of G_q bounds any cover from below
    used, match = set(), 0
    for s, t in pairs:
        if s != t and s not in used and t not in used:
            used |= {int(s), int(t)}
            match += 1
    assert match <= n <= len({int(x) for p in pairs for x in p})


def test_duplicates_reversed_and_self_pairs():
    pairs = np.array([(4, 9), (9, 4), (4, 9), (3, 3), (9, 2)], dtype=np.uint32)
    src, n = ppsp.batch_sources(pairs, "vc")
    check_cover(pairs, src)
    assert src[0] == src[1] == src[2] and src[3] == NONE
    assert n == 1  # vertex 9 covers every query
    assert ppsp.batch_sources(np.zeros((0, 2), np.uint32), "vc")[1] == 0


def brute_min_bipartite_cover(pairs):
    # nodes: (vertex, 0) for a source, (vertex, 1) for a target
    nodes = sorted({(int(s), 0) for s, t in pairs if s != t} | {(int(t), 1) for s, t in pairs if s != t})
    idx = {x: k for k, x in enumerate(nodes)}
    edges = [(1 << idx[(int(s), 0)]) | (1 << idx[(int(t), 1)]) for s, t in pairs if s != t]
    for r in range(len(nodes) + 1):
        for sub in itertools.combinations(range(len(nodes)), r):
            m = sum(1 << k for k in sub)
            if all(e & m for e in edges):
                return r
    return len(nodes)


@pytest.mark.parametrize("seed", range(12))
def test_directed_cover_is_minimum(seed):
    # directed G_q is bipartite (sources, targets): the cover is minimum
    # (Konig), every query is answered forward from its source or backward
    # from its target
    rng = np.random.default_rng(100 + seed)
    nv = int(rng.integers(2, 9))
    ne = int(rng.integers(1, 2 * nv + 1))
    ids = rng.choice(10 ** 6, size=nv, replace=False).astype(np.uint32)
    pairs = ids[rng.integers(0, nv, size=(ne, 2))]
    src, n, dirs = ppsp.batch_sources(pairs, "vc", undirected=False, return_dirs=True)
    for (s, t), x, d in zip(pairs, src, dirs):
        if s == t:
            assert x == NONE
        else:
            assert (x, d) in ((s, 0), (t, 1))
    assert n == brute_min_bipartite_cover(pairs)
    assert n == len({(int(x), int(d)) for x, d in zip(src, dirs) if x != NONE})


def test_directed_cover_equals_maximum_matching():
    # Konig: a minimum bipartite cover has the size of a maximum matching
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_bipartite_matching

    rng = np.random.default_rng(7)
    for _ in range(5):
        pairs = rng.integers(0, 300, size=(2000, 2)).astype(np.uint32)
        pairs = pairs[pairs[:, 0] != pairs[:, 1]]
        _, n = ppsp.batch_sources(pairs, "vc", undirected=False)
        uniq = np.unique(pairs, axis=0)
        a = csr_matrix((np.ones(uniq.shape[0]), (uniq[:, 0], uniq[:, 1])), shape=(300, 300))
        match = maximum_bipartite_matching(a, perm_type="column")
        assert n == int((match >= 0).sum())
    # a reversed star is one backward search from its centre
    rs = np.array([(x, 5) for x in range(10, 40)], dtype=np.uint32)
    src, n, dirs = ppsp.batch_sources(rs, "vc", undirected=False, return_dirs=True)
    assert n == 1 and set(src.tolist()) == {5} and set(dirs.tolist()) == {1}
    # (a, b) and (b, a) are two queries on a directed graph, one undirected
    assert ppsp.batch_sources(np.array([(1, 2), (2, 1)]), "vc", undirected=False)[1] == 2
    assert ppsp.batch_sources(np.array([(1, 2), (2, 1)]), "vc")[1] == 1


def test_invalid_strategy():
    with pytest.raises(ppsp.PPSPError):
        ppsp.batch_sources(np.array([[0, 1]]), "multi")


def test_golden_query_graph_patterns():
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "query_graph_patterns.json")
    with open(path) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        pairs = np.array(c["pairs"], dtype=np.uint32)
        assert ppsp.batch_sources(pairs, "vc")[1] == c["vc_sources"], c["name"]
        assert ppsp.batch_sources(pairs, "sssp")[1] == c["plain_sssp_sources"], c["name"]
