"""Benchmark: exact PPSP queries/sec and GTEPS on one GB300.

Workload (default): the largest single-launch configuration, the road-like
2048 x 2048 jittered grid (about 4.19 M vertices, 10% of grid edges deleted,
0.5% shortcuts of at most 20 cells, weights round(1000 * length)) with a
batch of 2,048 queries: 1,552 random pairs and every pair of a 32-vertex
clique (496 pairs), answered with bidirectional A* (Sec. 3.5) in one
persistent launch replayed as a CUDA graph.  The launch configuration (batch
strategy, block size, team size, frontier policy, GetDist rule) is chosen by
the autotuner at the start of the run; a step is one pass of the whole batch.

Reported:
  value        queries/sec with the graph, the pairs and the output in HBM
               (CUDA events on the launching stream around each step; the L2
               is flushed between steps by writing a 256 MB buffer)
  e2e          queries/sec through ppsp_batch with pinned host buffers (query graph
               build, host->device copy of the pairs, search, device->host
               copy of the distances inside the timed region)
  plain        the same queries one at a time (Plain-BiDS, best team size)
  strategies   the paper's Multi-BiDS (Sec. 4.2) and other batch strategies
               on the same batch
  roofline     algorithmic bytes of the engine kernel per step / step time
  cpu_baseline the CPU Dijkstra oracle on a bounded sample, all host cores
  config3      RMAT-22 with its three query patterns (BiDS): AUTO, Multi-BiDS,
               plain, GTEPS and roofline
  config5      the 4096^2 road-like graph with uint64 distances: a batch of
               256 queries and the serving loop at 1K, 5K and 20K queries/s
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


WORKLOAD_NAMES = {
    1: "64x64 jittered grid, 100 random pairs",
    2: "road-like 1024x1024 grid, 1000 near/mid/far queries",
    3: "RMAT scale 22 (edge factor 16), 64 random pairs + 64-leaf star + 11-clique",
    4: "road-like 2048x2048 grid, 1552 random pairs + 32-clique (496 pairs)",
    5: "road-like 4096x4096 grid, uint64 distances, Poisson arrivals (serving)",
}


METRIC = "PPSP queries/sec (exact distances), batched vs plain one-at-a-time"


def workload_name(cfg: int, g, k: int, mode: str) -> str:
    return "%s (%d vertices, %d CSR entries, %d queries per step), %s" % (WORKLOAD_NAMES[cfg], g.n, g.m, k, mode)


def load_workload(cfg: int):
    from workloads import config_workload

    wl = config_workload(cfg)
    # every batch of the configuration, as one batch (its query graph keeps
    # the random pairs, the star and the clique as separate components)
    names = list(wl["batches"])
    pairs = np.concatenate([wl["batches"][b] for b in names])
    # strata of the bounded CPU samples: near/mid/far, or the query patterns
    wl["labels_all"] = np.asarray(wl["labels"]) if "labels" in wl else np.concatenate(
        [np.full(wl["batches"][b].shape[0], j, dtype=np.int32) for j, b in enumerate(names)])
    mode = {"bids": "bids", "bidastar": "bidastar", "multi_astar": "bidastar", "serving": "bidastar"}[wl["mode"]]
    return wl, pairs, mode


def algorithmic_bytes(cnt: dict, dist_bytes: int, astar: bool) -> int:
    """Bytes the method must touch (offsets, edges, distances, queue entries)."""
    X, E, R, P, T = cnt["extracted"], cnt["edges"], cnt["relaxed"], cnt["pushed"], cnt["touched"]
    coord = 8 if astar else 0
    return int(X * (2 * 4 + dist_bytes + coord) + E * (4 + 4 + dist_bytes) + R * (dist_bytes + coord)
               + P * 4 * 2 + T * dist_bytes)


def group_time_stats(plan):
    """Device time per group in the plan's last run (a pair group is one
    query), summarised as the paper summarises query times (geometric mean),
    with the median, 99th percentile and maximum, in ms."""
    from paper_2506_16488_gb300 import ppsp

    try:
        ns = np.asarray(plan.group_times(), dtype=np.float64)
    except ppsp.PPSPError:
        return None
    ms = ns[ns > 0] / 1e6
    if ms.size == 0:
        return None
    return {"groups": int(ms.size), "geomean": float(np.exp(np.log(ms).mean())), "p50": float(np.median(ms)),
            "p99": float(np.percentile(ms, 99)), "max": float(ms.max())}


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def engine_source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2506_16488_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_2506_16488_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(workload: str):
    """DRAM bytes per engine launch from the committed ncu summary, if it
    was taken on the current sources; else None."""
    p = os.path.join(ROOT, "profiles", "engine_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != engine_source_hash() or d.get("workload") != workload:
        return None
    return d.get("dram_bytes_per_launch")


def cpu_baseline(g, pairs, labels, per_stratum: int = 0):
    import oracle

    threads = os.cpu_count() or 1
    # a bounded, stratified sample: equal numbers of queries per stratum
    # (near/mid/far, or each query pattern)
    rng = np.random.default_rng(7)
    per = per_stratum or max(1, min(20, threads * 2))
    idx = np.concatenate([rng.choice(np.nonzero(labels == b)[0], size=min(per, int((labels == b).sum())),
                                     replace=False) for b in np.unique(labels)])
    sample = pairs[idx]
    t0 = time.perf_counter()
    oracle.pairs_threaded(g.offsets, g.targets, g.weights, sample, threads)
    dt = time.perf_counter() - t0
    # single-threaded on a third of the sample (same strata), which also
    # counts the edges Dijkstra scans (the work ratio's denominator)
    sub = sample[::3]
    t0 = time.perf_counter()
    _, scanned = oracle.pairs(g.offsets, g.targets, g.weights, sub, return_scanned=True)
    dt1 = time.perf_counter() - t0
    return {"value": sample.shape[0] / dt, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"{sample.shape[0]} queries ({per} per stratum: near/mid/far, or each batch pattern), "
                      f"one Dijkstra per query, {threads} threads",
            "single_thread_qps": sub.shape[0] / dt1,
            "dijkstra_edges_per_query": scanned / max(1, sub.shape[0])}


def run_reference(args):
    """The CPU oracle timed as the reference arm (rank 0 only)."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    import oracle

    wl, pairs, mode = load_workload(args.config)
    g = wl["graph"]
    labels = wl["labels_all"]
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    per = max(1, min(6, threads // 2))
    times = []
    nq = 0
    for step in range(args.warmup + args.steps):
        idx = np.concatenate([rng.choice(np.nonzero(labels == b)[0], size=min(per, int((labels == b).sum())),
                                         replace=False) for b in np.unique(labels)])
        t0 = time.perf_counter()
        oracle.pairs_threaded(g.offsets, g.targets, g.weights, pairs[idx], threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            nq += idx.shape[0]
    total = sum(times)
    value = nq / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name(args.config, g, pairs.shape[0], mode),
                   "sample_per_step": int(idx.shape[0])},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle",
                         "sample": f"{idx.shape[0]} stratified queries per step, binary-heap Dijkstra, "
                                   f"{threads} threads"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _timed_plan_runs(G, pairs, opts, reps, warmup, stream, flush):
    """Warm-up and timed runs of one plan (CUDA events on its stream, L2
    flushed before each timed run); returns (ms list, counters of the last
    run, distances, plan's group times)."""
    import torch

    k = pairs.shape[0]
    with torch.cuda.stream(stream):  # cleared on the stream the plan writes on
        out = torch.zeros(k, dtype=torch.int64, device="cuda")
    plan = G.plan(pairs, stream=stream.cuda_stream, cuda_graph=True, **opts)
    for _ in range(warmup):
        plan.run(out.data_ptr())
        plan.sync()
    ms, cnt = [], None
    for i in range(reps):
        with torch.cuda.stream(stream):
            flush.fill_(i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(out.data_ptr())
        e1.record(stream)
        cnt = plan.sync()
        ms.append(e0.elapsed_time(e1))
    gms = group_time_stats(plan)
    plan.close()
    return ms, cnt, out.cpu().numpy().view(np.uint64).copy(), gms


def _plain(G, pairs, got, nq, teams, stream, **popts):
    """One query at a time (Plain strategy) on a strided subset, best of the
    given team sizes; answers checked against the batched run's."""
    import torch

    sel = np.linspace(0, pairs.shape[0] - 1, min(pairs.shape[0], nq)).astype(np.int64)
    pp_pairs = pairs[sel]
    kp = pp_pairs.shape[0]
    runs = []
    for tc in teams:
        pp = G.plan(pp_pairs, strategy="plain", stream=stream.cuda_stream, team_ctas=tc, **popts)
        with torch.cuda.stream(stream):
            po = torch.zeros(kp, dtype=torch.int64, device="cuda")
        pp.run(po.data_ptr())
        pp.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pp.run(po.data_ptr())
        e1.record(stream)
        pc = pp.sync()
        ms = e0.elapsed_time(e1)
        assert np.array_equal(po.cpu().numpy().view(np.uint64), got[sel])
        runs.append({"value": kp / (ms / 1000.0), "unit": "queries/s", "ms": ms, "queries": kp,
                     "gteps": pc["edges"] / (ms / 1000.0) / 1e9, "rounds": pc["rounds"],
                     "query_ms": group_time_stats(pp), "team_ctas": tc if tc else "all resident CTAs"})
        pp.close()
    best = max(runs, key=lambda r: r["value"])
    best["tried"] = [{"team_ctas": r["team_ctas"], "value": r["value"]} for r in runs]
    return best


def ms_per_step_median(step_ms):
    return float(np.median(step_ms))


def _roofline(cnt, ms, dist_bytes, astar, peak, peak_kind, traffic=None):
    alg = algorithmic_bytes(cnt, dist_bytes, astar)
    achieved = alg / (ms / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "traffic": traffic, "algorithmic_bytes_per_launch": alg}


def _delta_rule(G, mode, args):
    from paper_2506_16488_gb300 import learned_delta

    if args.delta:
        return f"fixed {args.delta}", None
    if args.no_learned:
        return "default (mean edge weight)", None
    model = learned_delta.load_model(mode)
    if model is None:
        return "default (mean edge weight)", None
    G.set_delta_model(mode, model)
    return f"learned MLP ({os.path.relpath(learned_delta.weights_path(mode), ROOT)})", model


def _choose_opts(G, pairs, mode, args, world):
    """Launch configuration of the headline batch: the autotuner's choice
    (coordinate descent from the AUTO strategy, every trial checked for the
    same answers) or a fixed strategy."""
    from paper_2506_16488_gb300 import autotune

    base = {"mode": mode, "strategy": "auto" if args.strategy == "tuned" else args.strategy}
    if args.delta:
        base["delta"] = args.delta
    if args.config == 5:
        base["dist_bits"] = 64  # the serving graph's configuration keeps uint64 distances
    if args.strategy != "tuned" or world > 1:
        if args.block_threads:
            base["block_threads"] = args.block_threads
        return base, None
    t0 = time.perf_counter()
    res = autotune.tune(G, pairs, mode, base=base, reps=2, budget_s=args.tune_budget)
    trials = [{"opts": {k: v for k, v in t["opts"].items() if k not in ("mode", "delta")},
               "ms": round(t["ms"], 3)} for t in res["trials"]]
    return res["opts"], {"seconds": time.perf_counter() - t0, "trials": trials,
                         "chosen": {k: v for k, v in res["opts"].items() if k not in ("mode", "delta")}}


def extra_config3(args, peak, peak_kind, flush, stream):
    """RMAT-22 (power-law shape), its three query patterns in one batch, BiDS:
    the AUTO strategy, the paper's Multi-BiDS, and plain one at a time."""
    from paper_2506_16488_gb300 import ppsp

    wl, pairs, mode = load_workload(3)
    g = wl["graph"]
    labels = wl["labels_all"]
    k = pairs.shape[0]
    res = {"workload": workload_name(3, g, k, mode)}
    with ppsp.Graph.from_csr(g, with_coords=False) as G:
        res["delta"], _ = _delta_rule(G, mode, args)
        ms, cnt, got, gms = _timed_plan_runs(G, pairs, {"mode": mode, "strategy": "auto"}, 3, 1, stream, flush)
        t = float(np.median(ms))
        res["auto"] = {"value": k / (t / 1000.0), "unit": "queries/s", "ms": t, "gteps": cnt["edges"] / t / 1e6,
                       "searches": cnt["searches"], "roofline": _roofline(cnt, t, 4, False, peak, peak_kind),
                       "group_ms": gms}
        ms, cnt, got_m, _ = _timed_plan_runs(G, pairs, {"mode": mode, "strategy": "multi"}, 1, 1, stream, flush)
        assert np.array_equal(got_m, got)
        res["multi"] = {"value": k / (ms[0] / 1000.0), "unit": "queries/s", "ms": ms[0],
                        "gteps": cnt["edges"] / ms[0] / 1e6, "searches": cnt["searches"]}
        # one query at a time on 16 CTAs or on all of them (one CTA per query
        # measured about 10x slower than all on this graph)
        res["plain"] = _plain(G, pairs, got, args.plain_queries // 4, [16, 0], stream, mode=mode)
    res["speedup_vs_plain"] = res["auto"]["value"] / res["plain"]["value"]
    res["cpu_baseline"] = cpu_baseline(g, pairs, labels, per_stratum=4)
    return res


def extra_config5(args, flush, stream):
    """The 4096^2 road-like graph with uint64 distances: a batch of 256
    random queries (AUTO, BiD-A*) and the continuous-batching serving loop."""
    import torch

    from paper_2506_16488_gb300 import ppsp
    from paper_2506_16488_gb300.serving import GpuExecutor, Scheduler, memory_model, poisson_arrivals, serve

    wl, pairs, mode = load_workload(5)
    g = wl["graph"]
    k = pairs.shape[0]
    res = {"workload": workload_name(5, g, k, mode) + ", uint64 distances"}
    with ppsp.Graph.from_csr(g) as G:
        res["delta"], _ = _delta_rule(G, mode, args)
        ms, cnt, got, gms = _timed_plan_runs(G, pairs, {"mode": mode, "strategy": "auto", "dist_bits": 64}, 3, 1,
                                             stream, flush)
        t = float(np.median(ms))
        res["batch"] = {"value": k / (t / 1000.0), "unit": "queries/s", "ms": t, "gteps": cnt["edges"] / t / 1e6,
                        "group_ms": gms}
        if args.next2:
            ms, _, got_m, _ = _timed_plan_runs(G, pairs, {"mode": mode, "strategy": "auto", "dist_bits": 64,
                                                          "memo_potential": True}, 3, 1, stream, flush)
            assert np.array_equal(got_m, got)
            res["batch_memo_potential"] = {"value": k / (float(np.median(ms)) / 1000.0), "ms": float(np.median(ms))}
        free, _ = torch.cuda.mem_get_info()
        lanes = args.lanes
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        lane_ctas = args.lane_ctas or max(1, sms // lanes)
        rng = np.random.default_rng(5003)
        src = lambda n: g.lcc[rng.integers(0, g.lcc.shape[0], size=(n, 2))]
        ex = GpuExecutor(G, lanes, mode=mode, dist_bits=64, lane_ctas=lane_ctas, team_ctas=args.team_ctas)
        model = memory_model(ex.slot_bytes(), lane_ctas)
        budget = int(0.6 * free)
        serve(poisson_arrivals(2000, 0.2, src, seed=5004), ex, Scheduler(lanes, 256, budget, model))  # warm-up
        rates = []
        for rate in args.rates:
            out = serve(poisson_arrivals(rate, args.duration, src, seed=int(rate)), ex,
                        Scheduler(lanes, 256, budget, model))
            rates.append({"offered_qps": rate, "sustained_qps": out["qps"], "p50_ms": out["latency_p50_ms"],
                          "p99_ms": out["latency_p99_ms"], "queries": out["queries"],
                          "requests": len(out["requests"]), "rejected": out["rejected"],
                          "failed": sum(1 for r in out["requests"] if r.status != 0)})
        res["serving"] = {"lanes": lanes, "lane_ctas": lane_ctas, "memory_budget_bytes": budget,
                          "seconds_per_rate": args.duration, "rates": rates}
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2506_16488_gb300 import ppsp

    wl, pairs, mode = load_workload(args.config)
    g = wl["graph"]
    labels = wl["labels_all"]
    if world > 1 and rank > 0:
        # weak scaling over query-parallel replicas: every rank answers its own
        # batch of the same shape (same size and pattern mix) on its copy
        from paper_2506_16488_gb300.replicas import rank_seed
        from workloads import near_mid_far_pairs, random_pairs

        if "labels" in wl and args.config == 2:
            pairs, labels = near_mid_far_pairs(g, pairs.shape[0], rank_seed(args.config * 1000 + 2, rank))
        else:
            keep = labels != 0  # the patterns (clique, star) stay; the random pairs are redrawn
            fresh = random_pairs(g, int((labels == 0).sum()), rank_seed(args.config * 1000 + 2, rank))
            pairs = np.concatenate([fresh, pairs[keep]])
            labels = np.concatenate([np.zeros(fresh.shape[0], dtype=labels.dtype), labels[keep]])
    if args.queries and args.queries < pairs.shape[0]:
        # an evenly strided subset keeps the pattern mix
        sel = np.linspace(0, pairs.shape[0] - 1, args.queries).astype(np.int64)
        pairs, labels = pairs[sel], labels[sel]
    k = pairs.shape[0]
    workload = workload_name(args.config, g, k, mode)
    if args.max_ctas:
        workload += f", at most {args.max_ctas} CTAs"
    G = ppsp.Graph.from_csr(g)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    delta_rule, model = _delta_rule(G, mode, args)
    opts, tuning = _choose_opts(G, pairs, mode, args, world)
    if args.max_ctas:
        opts["max_ctas"] = args.max_ctas
    plan = G.plan(pairs, stream=stream.cuda_stream, cuda_graph=True, **opts)
    with torch.cuda.stream(stream):
        out = torch.zeros(k, dtype=torch.int64, device="cuda")

    def step():
        plan.run(out.data_ptr())

    for _ in range(args.warmup):
        step()
        plan.sync()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    counters = []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        counters.append(plan.sync())
    torch.cuda.synchronize()
    plan_used_graph = plan.uses_graph()
    group_ms = group_time_stats(plan)  # the last timed step
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    clocks = sampler.stop()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    got = out.cpu().numpy().view(np.uint64)
    plan.close()

    # e2e through the C ABI with host buffers, in pinned (page-locked)
    # memory as a serving process keeps them (pageable if pinning is refused)
    try:
        t_pairs = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.uint32).view(np.int32)).pin_memory()
        t_res = torch.empty(k, dtype=torch.int64).pin_memory()
        h_pairs, h_res, host_memory = t_pairs.numpy().view(np.uint32), t_res.numpy().view(np.uint64), "pinned"
    except RuntimeError:
        h_pairs = np.ascontiguousarray(pairs, dtype=np.uint32)
        h_res, host_memory = np.zeros(k, dtype=np.uint64), "pageable"
    bopts = {kk: v for kk, v in opts.items() if kk not in ("mode",)}
    e2e_ms = []
    for i in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = G.batch(h_pairs, out=h_res, mode=mode, **bopts)
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    assert np.array_equal(res, got)
    e2e_step_ms = float(np.median(e2e_ms))
    if world > 1:  # the slowest rank's end-to-end step, as for the device time
        t = torch.tensor([e2e_step_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step_ms = float(t.item())

    # plain: one query at a time (Plain-BiDS), with the default Delta and
    # with the same Delta rule as the batched run
    default_delta = max(1, int(round(G.info()["w_mean"])))
    plain = _plain(G, pairs, got, args.plain_queries, args.plain_default_teams, stream, mode=mode,
                   delta=args.delta or default_delta)
    plain["delta"] = f"default {default_delta}" if not args.delta else f"fixed {args.delta}"
    plain_same = _plain(G, pairs, got, args.plain_queries, args.plain_teams, stream, mode=mode,
                        **({"delta": args.delta} if args.delta else {}))
    plain_same["delta"] = delta_rule

    # other batch strategies on the same batch (Sec. 4.2 Multi-BiDS, Plain*,
    # Sec. 4.3 Plain-SSSP and VC-SSSP), one timed run each after one untimed run
    compare = {}
    for strat in args.compare:
        copts = dict(mode=mode, strategy=strat.replace("_potential", ""), max_ctas=args.max_ctas,
                     multi_potential=strat == "multi_potential")
        if args.delta:
            copts["delta"] = args.delta
        ms, cc, co, _ = _timed_plan_runs(G, pairs, copts, 1, 1, stream, flush)
        assert np.array_equal(co, got), strat
        compare[strat] = {"value": k / (ms[0] / 1000.0), "unit": "queries/s", "ms": ms[0],
                          "searches": cc["searches"], "edges": cc["edges"]}
    # the paper's two implementation optimisations, on and off: heuristic
    # memoization (Sec. 5) on the headline launch, and pull-then-push
    # relaxation (App. B) where it applies, on groups run by several CTAs
    # (the plain one-at-a-time baseline on all CTAs, and Multi-BiDS)
    next2 = None
    if args.next2 and world == 1:
        next2 = {}
        ms, _, co, _ = _timed_plan_runs(G, pairs, dict(opts, memo_potential=True), 3, 1, stream, flush)
        assert np.array_equal(co, got)
        t = float(np.median(ms))
        next2["memo_potential"] = {"value": k / (t / 1000.0), "ms": t, "off_ms": ms_per_step_median(step_ms)}
        pl = {}
        for pull in (False, True):
            r = _plain(G, pairs, got, args.plain_queries, [0], stream, mode=mode, pull_push=pull)
            pl["on" if pull else "off"] = {"value": r["value"], "ms": r["ms"], "queries": r["queries"]}
        next2["pull_push_plain_all_ctas"] = pl
        ml = {}
        for pull in (False, True):
            mopts = dict(mode=mode, strategy="multi", pull_push=pull)
            if args.delta:
                mopts["delta"] = args.delta
            ms, cc, co, _ = _timed_plan_runs(G, pairs, mopts, 1, 1, stream, flush)
            assert np.array_equal(co, got)
            ml["on" if pull else "off"] = {"value": k / (ms[0] / 1000.0), "ms": ms[0], "edges": cc["edges"]}
        next2["pull_push_multi"] = ml
    G.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cnt = counters[-1]
    astar = mode in ("bidastar", "astar")
    dist_bytes = opts.get("dist_bits", 32) // 8
    ms_per_step = total_ms / args.steps
    qps = world * k * args.steps / (total_ms / 1000.0)
    peak, peak_kind = read_peaks()
    cpu = cpu_baseline(g, pairs, labels) if world == 1 else None
    extras = {}
    if world == 1:
        for c in (c for c in args.extras if c != args.config):
            extras[f"config{c}"] = (extra_config3(args, peak, peak_kind, flush, stream) if c == 3
                                    else extra_config5(args, flush, stream))
    chosen = {kk: v for kk, v in opts.items() if kk not in ("mode", "delta", "dist_bits")}
    line = {
        "metric": METRIC,
        "value": qps,
        "unit": "queries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "ms_per_step_median": float(np.median(step_ms)),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64" if dist_bytes == 8 else "u32",
        "data": "synthetic",
        "config": {"workload": workload, "queries_per_step": k,
                   "strategy": chosen.get("strategy", "multi"), "launch": chosen,
                   "tuned": tuning is not None, "delta": delta_rule,
                   "l2": "flushed between steps (256 MB write)",
                   "inputs": "plan (query graph, schedule) built before the timed region; graph, plan and "
                             "output resident in HBM", "parallelism": f"replicas x{world}"},
        "gteps": cnt["edges"] / (ms_per_step / 1000.0) / 1e9,
        # edges scanned per query, GPU batch mean over the oracle's Dijkstra on
        # the stratified sample
        "work_ratio": (cnt["edges"] / k) / cpu["dijkstra_edges_per_query"]
        if cpu and cpu.get("dijkstra_edges_per_query") else None,
        "plain": plain,
        "plain_same_delta": plain_same,
        "speedup_vs_plain": qps / world / plain["value"],
        "speedup_vs_plain_same_delta": qps / world / plain_same["value"],
        **({"strategies": compare} if compare else {}),
        **({"autotune": tuning} if tuning else {}),
        **({"next2": next2} if next2 else {}),
        "counters": cnt,
        # per-group device time within the batch (start of its Init to the
        # end of its tidy step on its team)
        "group_ms": group_ms,
        "roofline": _roofline(cnt, ms_per_step, dist_bytes, astar, peak, peak_kind, read_traffic(workload)),
        "e2e": {"value": world * k / (e2e_step_ms / 1000.0), "unit": "queries/s",
                "h2d_bytes_per_step": int(h_pairs.nbytes), "d2h_bytes_per_step": int(h_res.nbytes),
                "host_memory": host_memory},
        "gpu_launches": (3 if model is not None else 2) * args.steps,
        "cuda_graph": plan_used_graph,
        "clocks": clocks,
        "cpu_baseline": cpu,
        **extras,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--strategy", default="tuned",
                    choices=["tuned", "auto", "multi", "plain_star", "vc", "sssp"],
                    help="batch strategy of the headline run; tuned = autotuner from AUTO")
    ap.add_argument("--tune-budget", type=float, default=40.0, help="seconds of autotuning (tuned strategy)")
    ap.add_argument("--delta", type=int, default=0)
    ap.add_argument("--no-learned", action="store_true", help="use the default Delta, not the learned model")
    ap.add_argument("--queries", type=int, default=0, help="strided subset of the batch (profiling)")
    ap.add_argument("--plain-queries", type=int, default=100,
                    help="plain baseline: strided subset of the batch, answered one at a time")
    ap.add_argument("--plain-default-teams", type=int, nargs="*", default=[16, 0],
                    help="team sizes tried for the plain baseline with the default Delta (0 = all CTAs; one CTA "
                         "answers about one query per second there, so it is not tried by default)")
    ap.add_argument("--plain-teams", type=int, nargs="*", default=[1, 16, 0],
                    help="team sizes tried for the plain one-query-at-a-time baseline (0 = all CTAs)")
    ap.add_argument("--max-ctas", type=int, default=0, help="cap on resident CTAs (profiling)")
    ap.add_argument("--block-threads", type=int, default=0, choices=[0, 256, 512, 1024],
                    help="threads per CTA of the headline plan with a fixed strategy (0 = the library's choice; "
                         "profiling the tuner's launch)")
    ap.add_argument("--compare", nargs="*", default=["multi", "multi_potential"],
                    choices=["multi", "multi_potential", "auto", "plain_star", "sssp", "vc"],
                    help="also time these batch strategies on the same batch (one run each)")
    ap.add_argument("--no-next2", dest="next2", action="store_false",
                    help="skip the memoization and pull-then-push on/off measurements")
    ap.add_argument("--extras", type=int, nargs="*", default=[3, 5], choices=[3, 5],
                    help="also measure these configurations (RMAT-22; the 4096^2 graph with serving)")
    ap.add_argument("--rates", type=float, nargs="*", default=[1000, 5000, 20000],
                    help="serving (config 5): offered query rates")
    ap.add_argument("--duration", type=float, default=2.0, help="serving (config 5): seconds per rate")
    ap.add_argument("--lanes", type=int, default=8, help="serving (config 5): concurrent micro-batches")
    ap.add_argument("--lane-ctas", type=int, default=0, help="serving (config 5): CTAs per lane (0 = SMs / lanes)")
    ap.add_argument("--team-ctas", type=int, default=1, help="serving (config 5): CTAs per query (0 = auto)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
