"""Continuous-batching query serving on one GPU.

Requests (single queries or batches of pairs) arrive over time.  The
scheduler packs waiting requests, oldest first, into micro-batches and starts
one whenever an execution lane (a CUDA stream with its share of the GPU's
CTAs) is free and the device memory the micro-batch's searches need fits the
budget; finished micro-batches free their lane and memory immediately, so new
arrivals join while earlier work is still on the device.  Each micro-batch is
one plan (query graph of its pairs, Sec. 4.1; Multi-BiDS, Sec. 4.2) run by the
persistent engine on a fraction of the SMs, so several micro-batches overlap
on the device.  Answers never depend on how requests were packed (Theorems
3.3/3.4: any schedule of the searches returns d(s,t)); `tests/` checks that
each result is the same alone and in the mix.

The scheduling core (:class:`Scheduler`) has no GPU dependency; the executor
(:class:`GpuExecutor`) runs plans through the C ABI.

Request status: 0 answered; REJECTED (-1) can never fit one micro-batch or
the memory budget; CANCELLED (-2) withdrawn by the client; a positive value
is the library's ppsp_status for the micro-batch that carried it (for
example PPSP_ERR_OOM when its plan could not get device memory); the loop
goes on with the other requests.
"""

from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

REJECTED = -1
CANCELLED = -2


@dataclass
class Request:
    """One client request: its pairs, arrival time and, once final, result
    and status (0, REJECTED, CANCELLED or a library status)."""

    rid: int
    pairs: np.ndarray  # uint32 [k, 2]
    arrival: float
    start: Optional[float] = None
    done: Optional[float] = None
    result: Optional[np.ndarray] = None
    status: int = 0


@dataclass
class MicroBatch:
    """Requests packed into one plan on one lane, with the bytes they hold."""

    requests: list
    pairs: np.ndarray
    bytes: int
    lane: int
    handle: object = None
    started: float = 0.0


class Scheduler:
    """Admission and packing (no device code).

    lanes        number of concurrent micro-batches
    max_pairs    pairs per micro-batch (requests are never split)
    budget       device bytes available for in-flight searches
    bytes_for    callable(pairs) -> device bytes the micro-batch needs
    """

    def __init__(self, lanes: int, max_pairs: int, budget: int, bytes_for: Callable[[np.ndarray], int]):
        assert lanes >= 1 and max_pairs >= 1
        self.lanes = lanes
        self.max_pairs = max_pairs
        self.budget = budget
        self.bytes_for = bytes_for
        self.waiting: deque = deque()
        self.free_lanes = list(range(lanes))
        self.in_use = 0
        self.rejected: list = []
        self.cancelled: list = []

    def add(self, req: Request):
        """Queue a request, or reject it if it can never be admitted."""
        need = self.bytes_for(req.pairs)
        if need > self.budget or req.pairs.shape[0] > self.max_pairs:
            # can never be admitted in one piece: refuse instead of waiting forever
            req.status = REJECTED
            self.rejected.append(req)
            return
        self.waiting.append(req)

    def cancel(self, rid: int) -> bool:
        """Withdraw a waiting request; False if it is not waiting (not yet
        added, already started or finished)."""
        for req in self.waiting:
            if req.rid == rid:
                self.waiting.remove(req)
                req.status = CANCELLED
                self.cancelled.append(req)
                return True
        return False

    def next_batch(self) -> Optional[MicroBatch]:
        """Pack the oldest waiting requests that fit one lane and the memory budget."""
        if not self.free_lanes or not self.waiting:
            return None
        reqs, k = [], 0
        for req in list(self.waiting):
            if k + req.pairs.shape[0] > self.max_pairs:
                break
            trial = np.concatenate([r.pairs for r in reqs] + [req.pairs])
            if self.in_use + self.bytes_for(trial) > self.budget:
                break
            reqs.append(req)
            k += req.pairs.shape[0]
        if not reqs:
            return None
        for _ in reqs:
            self.waiting.popleft()
        pairs = np.concatenate([r.pairs for r in reqs])
        mb = MicroBatch(reqs, pairs, self.bytes_for(pairs), self.free_lanes.pop(0))
        self.in_use += mb.bytes
        return mb

    def finish(self, mb: MicroBatch):
        """Return a finished micro-batch's lane and memory."""
        self.in_use -= mb.bytes
        self.free_lanes.append(mb.lane)
        self.free_lanes.sort()


def serve(arrivals: list, executor, scheduler: Scheduler, clock=time.perf_counter, poll_s: float = 2e-4,
          cancels=()) -> dict:
    """Run requests arriving at the given times (seconds from start).

    arrivals: list of (t_arrival, pairs) sorted by time; request ids are the
    list positions.  cancels: (t, request id) sorted by time: a request that
    has not started by then never runs; one already on the device completes
    there (a running search is not interrupted) and its answer is dropped.
    An executor error that carries a library status (``.status``) fails the
    micro-batch's requests with that status; other exceptions propagate.
    Returns per-request results and latencies, p50/p99 and sustained
    queries/sec (over answered requests), and the rejected / cancelled /
    failed counts.
    """
    reqs = [Request(i, np.ascontiguousarray(p, dtype=np.uint32).reshape(-1, 2), t) for i, (t, p) in
            enumerate(arrivals)]
    t0 = clock()
    nxt = nc = 0
    running: list = []
    closed = 0  # requests that reached a final state
    total = len(reqs)
    withdrawn: set = set()  # cancelled before arrival, or while running

    def close(mb, status, dists):
        nonlocal closed
        end = clock() - t0
        off = 0
        for r in mb.requests:
            k = r.pairs.shape[0]
            if r.rid in withdrawn:
                r.status = CANCELLED
            else:
                r.result = None if dists is None else dists[off:off + k]
                r.status = status
                r.done = end
            off += k
        closed += len(mb.requests)
        scheduler.finish(mb)

    while closed + len(scheduler.rejected) + len(scheduler.cancelled) < total:
        now = clock() - t0
        while nc < len(cancels) and cancels[nc][0] <= now:
            rid = int(cancels[nc][1])
            nc += 1
            if not scheduler.cancel(rid) and 0 <= rid < total and reqs[rid].done is None:
                withdrawn.add(rid)
        while nxt < total and reqs[nxt].arrival <= now:
            r = reqs[nxt]
            nxt += 1
            if r.rid in withdrawn:
                r.status = CANCELLED
                scheduler.cancelled.append(r)
            else:
                scheduler.add(r)
        while True:
            mb = scheduler.next_batch()
            if mb is None:
                break
            for r in mb.requests:
                r.start = clock() - t0
            mb.started = clock() - t0
            try:
                mb.handle = executor.start(mb.pairs, mb.lane)
            except Exception as e:
                if not isinstance(getattr(e, "status", None), int):
                    raise
                close(mb, e.status, None)
                continue
            running.append(mb)
        for mb in list(running):
            res = executor.poll(mb.handle)
            if res is None:
                continue
            status, dists = res
            close(mb, status, dists)
            running.remove(mb)
        if not running and nxt < total and not scheduler.waiting:
            # idle until the next arrival
            wait = reqs[nxt].arrival - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.01))
        else:
            time.sleep(poll_s)
    ok = [r for r in reqs if r.status == 0 and r.done is not None]
    span = max((r.done for r in ok), default=0.0)
    lat = np.array([r.done - r.arrival for r in ok])
    nq = sum(r.pairs.shape[0] for r in ok)
    return {
        "requests": reqs,
        "latency_p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
        "latency_p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
        "queries": int(nq),
        "span_s": float(span),
        "qps": float(nq / span) if span > 0 else None,
        "rejected": len(scheduler.rejected),
        "cancelled": sum(r.status == CANCELLED for r in reqs),
        "failed": sum(r.status > 0 for r in reqs),
    }


def poisson_arrivals(rate_qps: float, duration_s: float, pair_source: Callable[[int], np.ndarray], seed: int,
                     batch_sizes=(1, 1, 1, 4, 16, 64, 256)) -> list:
    """Poisson request stream whose query rate is rate_qps: each request is a
    single query or a batch (size drawn from batch_sizes)."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(batch_sizes)
    mean_size = sizes.mean()
    req_rate = rate_qps / mean_size
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / req_rate)
        if t > duration_s:
            break
        k = int(rng.choice(sizes))
        out.append((t, pair_source(k)))
    return out


class GpuExecutor:
    """Runs a micro-batch as one plan on a lane's stream with lane_ctas CTAs."""

    def __init__(self, graph, lanes: int, mode: str = "bids", dist_bits: int = 32, lane_ctas: int = 0,
                 strategy: str = "auto", **opts):
        import torch

        from . import ppsp

        self.ppsp = ppsp
        self.torch = torch
        self.graph = graph
        self.streams = [torch.cuda.Stream() for _ in range(lanes)]
        self.mode = mode
        self.dist_bits = dist_bits
        self.lane_ctas = lane_ctas
        self.opts = dict(opts, strategy=strategy)

    def slot_bytes(self) -> int:
        """Device bytes of the pair slot each team of a micro-batch holds."""
        return self.graph.slot_bytes(2, self.dist_bits)

    def start(self, pairs: np.ndarray, lane: int):
        """Create the micro-batch's plan and launch it on the lane's stream."""
        s = self.streams[lane]
        plan = self.graph.plan(pairs, mode=self.mode, dist_bits=self.dist_bits, stream=s.cuda_stream,
                               max_ctas=self.lane_ctas, **self.opts)
        try:
            # the output is allocated and cleared on the lane's stream, so the
            # clear is ordered before the plan's writes (on another stream it
            # could land after them)
            with self.torch.cuda.stream(s):
                out = self.torch.zeros(pairs.shape[0], dtype=self.torch.int64, device="cuda")
            plan.run(out.data_ptr())
        except BaseException:
            plan.close()
            raise
        ev = self.torch.cuda.Event()
        ev.record(s)
        return (plan, out, ev)

    def poll(self, handle):
        """None while running, else (status, distances); frees the plan."""
        plan, out, ev = handle
        if not ev.query():
            return None
        try:
            plan.sync()
            status = 0
        except self.ppsp.PPSPError as e:
            status = e.status
        d = out.cpu().numpy().view(np.uint64).copy()
        plan.close()
        return status, d


def memory_model(slot_bytes: int, lane_ctas: int) -> Callable[[np.ndarray], int]:
    """bytes_for(pairs): the search memory a micro-batch's plan holds.  A
    plan has at most one team per group and at most lane_ctas teams, and each
    team holds one slot; with BiD-A* and the AUTO strategy every group has at
    most two searches, so a pair slot bounds each.  `slot_bytes` is the
    library's own size of that slot (``Graph.slot_bytes(2, dist_bits)``, i.e.
    ppsp_slot_bytes), so the model follows the library's capacities."""
    per = int(slot_bytes)

    def f(pairs: np.ndarray) -> int:
        return int(min(lane_ctas, max(1, pairs.shape[0])) * per)

    return f
