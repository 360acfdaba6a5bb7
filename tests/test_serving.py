"""Serving: admission by memory and continuous batching (scheduler on CPU,
results alone vs in the mix on the GPU)."""

import time

import numpy as np
import pytest

from paper_2506_16488_gb300.serving import (CANCELLED, REJECTED, Request, Scheduler, memory_model, poisson_arrivals,
                                            serve)


def _req(i, k, t=0.0):
    return Request(i, np.stack([np.arange(k), np.arange(k) + 1], axis=1).astype(np.uint32) + i * 1000, t)


def test_scheduler_packs_oldest_first_within_limits():
    sch = Scheduler(lanes=2, max_pairs=8, budget=100, bytes_for=lambda p: 10 * p.shape[0])
    for i, k in enumerate([3, 4, 2, 5, 1]):
        sch.add(_req(i, k))
    a = sch.next_batch()  # 3 + 4 fit (7 pairs, 70 bytes); adding 2 would exceed 8 pairs
    assert [r.rid for r in a.requests] == [0, 1] and a.bytes == 70 and a.lane == 0
    b = sch.next_batch()  # 2 fits (20 bytes -> 90); 5 more would exceed the budget
    assert [r.rid for r in b.requests] == [2] and b.lane == 1
    assert sch.next_batch() is None  # no free lane
    sch.finish(a)
    c = sch.next_batch()
    assert [r.rid for r in c.requests] == [3, 4] and sch.in_use == 20 + 60


def test_scheduler_rejects_requests_that_can_never_fit():
    sch = Scheduler(lanes=1, max_pairs=4, budget=30, bytes_for=lambda p: 10 * p.shape[0])
    sch.add(_req(0, 5))   # more pairs than a micro-batch
    sch.add(_req(1, 4))   # needs 40 bytes > budget
    sch.add(_req(2, 2))
    assert [r.rid for r in sch.rejected] == [0, 1]
    assert [r.rid for r in sch.next_batch().requests] == [2]


class FakeExecutor:
    """Completes a micro-batch 2 ms after it starts; answer = s + t."""

    def __init__(self):
        self.live = 0
        self.max_live = 0

    def start(self, pairs, lane):
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return (time.perf_counter() + 0.002, pairs)

    def poll(self, h):
        t, pairs = h
        if time.perf_counter() < t:
            return None
        self.live -= 1
        return 0, pairs[:, 0].astype(np.uint64) + pairs[:, 1]


def test_serve_loop_continuous_batching_with_fake_executor():
    rng = np.random.default_rng(0)
    arrivals = poisson_arrivals(4000, 0.05, lambda k: rng.integers(0, 1000, size=(k, 2)), seed=1,
                                batch_sizes=(1, 2, 8))
    ex = FakeExecutor()
    sch = Scheduler(lanes=3, max_pairs=16, budget=10 ** 9, bytes_for=lambda p: p.shape[0])
    out = serve(arrivals, ex, sch)
    assert ex.max_live <= 3 and out["rejected"] == 0
    for (t, p), r in zip(arrivals, out["requests"]):
        assert np.array_equal(r.result, p[:, 0].astype(np.uint64) + p[:, 1])
        assert r.done >= r.arrival
    assert out["latency_p99_ms"] >= out["latency_p50_ms"] > 0


def test_scheduler_cancel_withdraws_only_waiting_requests():
    sch = Scheduler(lanes=1, max_pairs=4, budget=100, bytes_for=lambda p: p.shape[0])
    for i in range(3):
        sch.add(_req(i, 2))
    a = sch.next_batch()  # requests 0 and 1 start
    assert [r.rid for r in a.requests] == [0, 1]
    assert not sch.cancel(0)  # already started
    assert sch.cancel(2) and not sch.cancel(2)
    assert [r.rid for r in sch.cancelled] == [2] and sch.cancelled[0].status == CANCELLED
    sch.finish(a)
    assert sch.next_batch() is None and not sch.waiting


class SlowExecutor(FakeExecutor):
    """One lane; each micro-batch takes 20 ms."""

    def start(self, pairs, lane):
        h = super().start(pairs, lane)
        return (h[0] + 0.018, h[1])


def test_serve_cancellations():
    pairs = lambda i: np.array([[i, i + 1]], dtype=np.uint32)
    # 0 runs first; 1 and 2 wait behind it; 3 arrives late
    arrivals = [(0.0, pairs(0)), (0.001, pairs(1)), (0.001, pairs(2)), (0.08, pairs(3)), (0.08, pairs(4))]
    # 0 is cancelled while on the device (its answer is dropped), 1 while
    # waiting, 3 before it arrives; 9 does not exist; 4 after it finished
    cancels = [(0.005, 0), (0.006, 1), (0.007, 3), (0.008, 9), (0.3, 4)]
    ex = SlowExecutor()
    sch = Scheduler(lanes=1, max_pairs=1, budget=10 ** 9, bytes_for=lambda p: p.shape[0])
    out = serve(arrivals, ex, sch, cancels=cancels)
    st = [r.status for r in out["requests"]]
    assert st == [CANCELLED, CANCELLED, 0, CANCELLED, 0]
    r = out["requests"]
    assert r[0].result is None and r[1].result is None and r[1].start is None and r[3].start is None
    assert r[2].result.tolist() == [5] and r[4].result.tolist() == [9]
    assert out["cancelled"] == 3 and out["failed"] == 0 and out["queries"] == 2


class FailingExecutor(FakeExecutor):
    """The plan for a micro-batch holding vertex 666 cannot get device memory."""

    class OOM(RuntimeError):
        status = 3  # PPSP_ERR_OOM

    def start(self, pairs, lane):
        if (pairs == 666).any():
            raise self.OOM("ppsp_plan_create: PPSP_ERR_OOM")
        return super().start(pairs, lane)


def test_serve_survives_a_failed_micro_batch():
    arrivals = [(0.0, np.array([[1, 2]])), (0.001, np.array([[666, 3]])), (0.002, np.array([[4, 5]])),
                (0.003, np.array([[1, 2]] * 9))]
    # one pair per micro-batch: the failure stays with the request that caused it
    sch = Scheduler(lanes=1, max_pairs=1, budget=10 ** 9, bytes_for=lambda p: p.shape[0])
    out = serve(arrivals, FailingExecutor(), sch)
    assert [r.status for r in out["requests"]] == [0, 3, 0, REJECTED]
    assert out["failed"] == 1 and out["rejected"] == 1 and out["queries"] == 2
    assert out["requests"][1].result is None and out["requests"][2].result.tolist() == [9]

    class Broken(FakeExecutor):
        def start(self, pairs, lane):
            raise ValueError("not a library error")

    with pytest.raises(ValueError):
        serve(arrivals[:1], Broken(), Scheduler(lanes=1, max_pairs=4, budget=10, bytes_for=lambda p: 1))


def test_memory_model_counts_one_slot_per_team():
    f = memory_model(slot_bytes=12345, lane_ctas=8)
    assert f(np.zeros((3, 2))) == 3 * 12345 and f(np.zeros((100, 2))) == 8 * 12345
    assert f(np.zeros((0, 2))) == 12345


@pytest.mark.gpu
def test_serving_results_alone_equal_in_mix():
    import __graft_entry__

    __graft_entry__.build()
    import oracle
    from paper_2506_16488_gb300 import ppsp
    from paper_2506_16488_gb300.serving import GpuExecutor
    from workloads import random_pairs, road_like_graph

    g = road_like_graph(96, seed=81)
    rng = np.random.default_rng(82)
    src = lambda k: g.lcc[rng.integers(0, g.lcc.shape[0], size=(k, 2))]
    arrivals = poisson_arrivals(3000, 0.3, src, seed=83, batch_sizes=(1, 1, 4, 16, 64))
    with ppsp.Graph.from_csr(g) as G:
        lanes, lane_ctas = 3, 32
        ex = GpuExecutor(G, lanes, mode="bidastar", dist_bits=64, lane_ctas=lane_ctas)
        model = memory_model(ex.slot_bytes(), lane_ctas)
        sch = Scheduler(lanes, 256, 2 ** 34, model)
        out = serve(arrivals, ex, sch)
        assert out["rejected"] == 0
        for r in out["requests"]:
            assert r.status == 0
            alone = G.batch(r.pairs, mode="bidastar", dist_bits=64)
            assert np.array_equal(r.result, alone)
        sample = np.concatenate([r.pairs for r in out["requests"][:20]])
        want = oracle.pairs(g.offsets, g.targets, g.weights, sample)
        got = np.concatenate([r.result for r in out["requests"][:20]])
        assert np.array_equal(got, want)


@pytest.mark.gpu
def test_memory_model_bounds_the_plans_device_memory():
    """The admission model takes its slot size from the library: every
    micro-batch plan the executor creates holds at most what the model
    charges for it (one pair slot per team, teams <= min(lane CTAs, queries))."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_2506_16488_gb300 import ppsp
    from paper_2506_16488_gb300.serving import GpuExecutor
    from workloads import road_like_graph

    g = road_like_graph(64, seed=91)
    rng = np.random.default_rng(92)
    with ppsp.Graph.from_csr(g) as G:
        lane_ctas = 12
        ex = GpuExecutor(G, 1, mode="bidastar", dist_bits=64, lane_ctas=lane_ctas)
        per = ex.slot_bytes()
        assert per >= 2 * g.n * 8  # at least the two distance arrays
        assert G.slot_bytes(1, 64) < per <= G.slot_bytes(4, 64)
        model = memory_model(per, lane_ctas)
        star = np.stack([np.full(9, g.lcc[0]), g.lcc[1:10]], axis=1)
        clique = np.array([[a, b] for a in g.lcc[20:26] for b in g.lcc[20:26] if a < b])
        for pairs in (g.lcc[rng.integers(0, g.lcc.shape[0], size=(k, 2))] for k in (1, 5, 12, 40)):
            for batch in (pairs, np.concatenate([pairs, star]), np.concatenate([pairs, clique])):
                plan, out, ev = ex.start(batch.astype(np.uint32), 0)
                b = plan.device_bytes()
                assert b["teams"] <= min(lane_ctas, batch.shape[0])
                assert b["slot_bytes"] <= model(batch), (b, model(batch))
                ev.synchronize()
                status, d = ex.poll((plan, out, ev))
                assert status == 0
                assert np.array_equal(d, G.batch(batch, mode="bidastar", dist_bits=64))
