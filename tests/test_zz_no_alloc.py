"""The allocation-free single-query entry point (ppsp_query_noalloc).

Some callers cannot allocate device memory: code that runs inside a memory
pool it does not own, a serving process under a no-allocation policy, or a
caller that cannot accept cudaMalloc's implicit device synchronisation.
ppsp_query_noalloc answers one BiDS query with all of its scratch in a fixed
array inside the library.  These tests call it through the C ABI on graphs
the caller keeps in its own device memory and check two calls in a row
against the CPU Dijkstra oracle (distances are integers: the tolerance is
zero), also on a graph of about a million vertices whose far queries
overflow the touched list, and check that calls after the first allocate no
device memory.  The file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2506_16488_gb300 import ppsp
from workloads import grid_graph, random_pairs, road_like_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    lib = ppsp.load()
    fn = lib.ppsp_query_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    return lib


def _device_csr(g):
    torch = pytest.importorskip("torch")
    off = torch.from_numpy(g.offsets.astype(np.int64).astype(np.int32)).cuda()
    ed = np.empty(2 * g.m, dtype=np.uint32)
    ed[0::2] = g.targets
    ed[1::2] = g.weights
    edges = torch.from_numpy(ed.view(np.int32)).cuda()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    return off, edges, out


def _call(lib, off, edges, out, n, m, s, t, delta, stream):
    out.fill_(-7)
    st = lib.ppsp_query_noalloc(off.data_ptr(), edges.data_ptr(), n, m, s, t, delta, out.data_ptr(), stream)
    got = int(out.cpu().numpy().view(np.uint64)[0])
    return st, got


@pytest.mark.parametrize("which", ["grid64", "road128"])
def test_noalloc_matches_oracle_on_two_calls(lib, which):
    import torch

    g = grid_graph(64, seed=1001) if which == "grid64" else road_like_graph(128, seed=77)
    pairs = random_pairs(g, 12, seed=5)
    pairs = np.concatenate([pairs, [[3, 3]]])  # s == t
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    off, edges, out = _device_csr(g)
    stream = torch.cuda.Stream()
    for (s, t), w in zip(pairs.tolist(), want.tolist()):
        for call in range(2):  # two calls in a row on the same array
            st, got = _call(lib, off, edges, out, g.n, g.m, s, t, 0, stream.cuda_stream)
            assert st == ppsp.OK, (st, call)
            assert got == w, (s, t, call, got, w)


def test_noalloc_million_vertex_graph_and_no_allocation(lib):
    """A graph just under the vertex limit (1024^2 road-like, about 1.05 M
    vertices): far BiDS queries touch more entries than the touched list
    holds, so the search resets the whole array; every later call must still
    be exact.  Device memory in use must not change after the first call."""
    import torch

    g = road_like_graph(1024, seed=2001)
    assert g.n <= (1 << 20)
    xy = g.grid_xy.astype(np.int64)
    far = np.argsort(xy[:, 0] + xy[:, 1])
    pairs = np.array([[far[0], far[-1]], [far[5], far[-7]], [far[-3], far[11]], [far[100], far[g.n // 2]]],
                     dtype=np.uint32)
    want = oracle.pairs(g.offsets, g.targets, g.weights, pairs)
    off, edges, out = _device_csr(g)
    stream = torch.cuda.Stream()
    st, got = _call(lib, off, edges, out, g.n, g.m, int(pairs[0, 0]), int(pairs[0, 1]), 0, stream.cuda_stream)
    assert st == ppsp.OK and got == int(want[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for (s, t), w in zip(pairs.tolist(), want.tolist()):
        for delta in (0, 0, 3000):  # two calls in a row with the default Delta, one with another
            st, got = _call(lib, off, edges, out, g.n, g.m, s, t, delta, stream.cuda_stream)
            assert st == ppsp.OK, (s, t, delta, st)
            assert got == w, (s, t, delta, got, w)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_the_limit(lib):
    import torch

    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    big = (1 << 20) + 1
    assert lib.ppsp_query_noalloc(dummy.data_ptr(), dummy.data_ptr(), big, 2, 0, 1, 0, out.data_ptr(),
                                  None) == ppsp.ERR_INVALID_ARG
    assert lib.ppsp_query_noalloc(dummy.data_ptr(), dummy.data_ptr(), 2, 2, 0, 5, 0, out.data_ptr(),
                                  None) == ppsp.ERR_INVALID_ARG
    assert lib.ppsp_query_noalloc(None, dummy.data_ptr(), 2, 2, 0, 1, 0, out.data_ptr(),
                                  None) == ppsp.ERR_INVALID_ARG
    # misaligned adjacency (8-byte records) or output: refused before any launch
    assert lib.ppsp_query_noalloc(dummy.data_ptr(), dummy.data_ptr() + 4, 2, 2, 0, 1, 0, out.data_ptr(),
                                  None) == ppsp.ERR_INVALID_ARG
    assert lib.ppsp_query_noalloc(dummy.data_ptr(), dummy.data_ptr(), 2, 2, 0, 1, 0, out.data_ptr() + 4,
                                  None) == ppsp.ERR_INVALID_ARG
