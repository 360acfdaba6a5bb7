"""Object lifetimes in the Python binding, on the host with a stand-in for the
library: a plan belongs to its graph (ppsp_plan_destroy takes the graph's
lock), so closing a graph destroys its open plans first; a graph borrows its
Delta model, so closing a model detaches it from the graphs that use it;
calls on a closed object raise instead of passing a freed handle to C."""

import ctypes

import numpy as np
import pytest

from paper_2506_16488_gb300 import ppsp


class FakeLib:
    def __init__(self):
        self.calls = []
        self.live = set()
        self.next = 1

    def _new(self, kind, out):
        h = self.next
        self.next += 1
        self.live.add((kind, h))
        out._obj.value = h
        return ppsp.OK

    def _free(self, kind, h):
        h = h.value if isinstance(h, ctypes.c_void_p) else h
        assert (kind, h) in self.live, f"{kind} {h} freed twice or never created"
        self.live.remove((kind, h))
        self.calls.append(("destroy", kind, h))

    def ppsp_options_init(self, o):
        pass

    def ppsp_graph_create(self, n, m, off, tgt, w, xy, flags, out):
        return self._new("graph", out)

    def ppsp_graph_destroy(self, h):
        self._free("graph", h)

    def ppsp_plan_create(self, g, pairs, k, opt, out):
        assert ("graph", g.value) in self.live
        return self._new("plan", out)

    def ppsp_batch(self, g, pairs, k, opt, out, paths, offs, lens, cnt):
        assert ("graph", g.value) in self.live
        self.calls.append(("batch", pairs.value, out.value))
        arr = ctypes.cast(out, ctypes.POINTER(ctypes.c_uint64))
        for q in range(k):
            arr[q] = 7 + q
        return ppsp.OK

    def ppsp_plan_destroy(self, h):
        self._free("plan", h)

    def ppsp_plan_run(self, h, out):
        raise AssertionError("a closed plan's handle reached the library")

    def ppsp_delta_model_create(self, params, out):
        return self._new("model", out)

    def ppsp_delta_model_destroy(self, h):
        self._free("model", h)

    def ppsp_graph_set_delta_model(self, g, mode, m):
        assert ("graph", g.value) in self.live
        mv = m.value if isinstance(m, ctypes.c_void_p) else m
        assert mv is None or ("model", mv) in self.live
        self.calls.append(("set_model", g.value, mode, mv))
        return ppsp.OK


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(ppsp, "_lib", lib)
    return lib


def _graph():
    off = np.array([0, 1, 2], dtype=np.uint64)
    return ppsp.Graph(off, np.array([1, 0], np.uint32), np.array([3, 3], np.uint32))


def test_closing_a_graph_destroys_its_plans_first(fake):
    g = _graph()
    p1 = g.plan(np.array([[0, 1]]))
    p2 = g.plan(np.array([[1, 0]]))
    g.close()
    kinds = [c[1] for c in fake.calls if c[0] == "destroy"]
    assert kinds == ["plan", "plan", "graph"]
    assert not fake.live
    p1.close()  # already destroyed: no second free
    del p2
    with pytest.raises(ppsp.PPSPError):
        p1.run(0)
    with pytest.raises(ppsp.PPSPError):
        g.plan(np.array([[0, 1]]))


def test_plans_closed_early_are_not_destroyed_again(fake):
    with _graph() as g:
        with g.plan(np.array([[0, 1]])):
            pass
    assert [c[1] for c in fake.calls if c[0] == "destroy"] == ["plan", "graph"]
    assert not fake.live


def test_closing_a_model_detaches_it(fake):
    g = _graph()
    m = ppsp.DeltaModel(np.ones(ppsp.MLP_PARAMS, np.float32))
    g.set_delta_model("bidastar", m)
    m.close()
    sets = [c for c in fake.calls if c[0] == "set_model"]
    assert sets[-1][2:] == (ppsp.MODES["bidastar"], None)
    assert m._h is None and [c[1] for c in fake.calls if c[0] == "destroy"] == ["model"]
    g.close()
    assert not fake.live


def test_model_outlives_graph(fake):
    m = ppsp.DeltaModel(np.ones(ppsp.MLP_PARAMS, np.float32))
    with _graph() as g:
        g.set_delta_model("bids", m)
    m.close()  # the graph is gone: nothing to detach
    assert not fake.live
    with pytest.raises(ValueError):
        ppsp.DeltaModel(np.ones(7, np.float32))


def test_batch_writes_a_caller_buffer(fake):
    g = _graph()
    pairs = np.array([[0, 1], [1, 0], [1, 1]], dtype=np.uint32)
    out = np.zeros(3, dtype=np.uint64)
    res = g.batch(pairs, out=out)
    assert res is out and out.tolist() == [7, 8, 9]
    call = [c for c in fake.calls if c[0] == "batch"][-1]
    assert call[1] == pairs.ctypes.data and call[2] == out.ctypes.data  # read and written in place
    assert g.batch(pairs).tolist() == [7, 8, 9]
    for bad in (np.zeros(3, np.int64), np.zeros(4, np.uint64), np.zeros(6, np.uint64)[::2]):
        with pytest.raises(ValueError):
            g.batch(pairs, out=bad)
    g.close()
