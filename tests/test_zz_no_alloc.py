"""The allocation-free single-query entry point (ppsp_query_noalloc).

Some callers cannot allocate device memory (a pool they do not own, a
no-allocation serving policy, or no tolerance for cudaMalloc's implicit
synchronisation).  ppsp_query_noalloc answers one BiDS query with all
scratch in a fixed array inside the library.  This test calls it through the
C ABI on graphs the caller keeps in its own device memory and checks that two
calls in a row give exactly what ppsp_query gives (distances are integers,
so the tolerance is zero).  The file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("which", ["grid64", "road128"])
def test_noalloc_matches_query_on_two_calls(lib, which):
    import torch

    g = grid_graph(64, seed=1001) if which == "grid64" else road_like_graph(128, seed=77)
    pairs = random_pairs(g, 12, seed=5)
    pairs = np.concatenate([pairs, [[3, 3]]])  # s == t
    off, edges, out = _device_csr(g)
    stream = torch.cuda.Stream()
    with ppsp.Graph.from_csr(g) as G:
        for s, t in pairs.tolist():
            want = G.query(s, t, mode="bids")
            for call in range(2):  # two calls in a row on the same array
                out.fill_(-7)
                torch.cuda.synchronize()
                st = lib.ppsp_query_noalloc(off.data_ptr(), edges.data_ptr(), g.n, g.m, s, t, 0,
                                            out.data_ptr(), stream.cuda_stream)
                assert st == ppsp.OK, (st, call)
                got = int(out.cpu().numpy().view(np.uint64)[0])
                assert got == want, (s, t, call, got, want)


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
