"""Learned stepping increment: sweep labels, train the MLP on the GPU, measure regret.

The paper picks Delta for Delta*-stepping by doubling it until the geometric
mean time stops improving (Sec. 6.1).  Here the same sweep produces training
labels: every group of a batch is timed on the device (ppsp_plan_group_times)
for Delta = Delta_default * 2^j over a grid of j, and its label is the
smallest j whose time is within 5% of its fastest run (time rises slowly
below the best increment and steeply above it).  The model (12 -> 64 -> 64
-> 1, ppsp_delta_model_*) is trained with the library's own Adam kernel, and
a safety margin chosen on the training sets (the smallest that minimises
their summed regret when a prediction between grid points is charged the
larger increment) is subtracted from its output bias.  Its regret is the total
group time at the predicted grid point over the total at each group's best
grid point, minus one.  Delta never changes an answer (Theorems 3.3/3.4), so a bad
prediction costs time only; without a model the library uses Delta_default
(mean edge weight).

Weights are stored as a flat float32 file plus a JSON file of metadata.
"""

from __future__ import annotations

import json
import os
import time

import numpy as np

from . import ppsp

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS_DIR = os.path.join(HERE, "weights")
GRID = tuple(range(-12, 4))  # log2(Delta / Delta_default) the sweep may visit


def weights_path(mode: str) -> str:
    return os.path.join(WEIGHTS_DIR, f"delta_{mode}.bin")


def sweep(G: ppsp.Graph, pairs: np.ndarray, mode: str, grid=GRID, stream=None, reps: int = 1,
          patience: int = 2, start: int = 0, **opts):
    """Time every group of the batch for Delta = Delta_default * 2^j.

    Like the paper's doubling search (Sec. 6.1) the sweep starts at j = start
    (0: the default increment; large graphs start lower, where the default is
    far too coarse and slow to time) and walks down, then up, while the
    batch's total time improves (stopping after `patience` worse points).
    Grid points it never visits get time +inf.
    Returns (features [groups, 12], times_ns [groups, len(grid)], default_delta).
    """
    import torch

    default = max(1, int(round(G.info()["w_mean"])))
    s = stream or torch.cuda.Stream()
    with torch.cuda.stream(s):  # cleared on the stream the plans write on
        out = torch.zeros(pairs.shape[0], dtype=torch.int64, device="cuda")
    grid = list(grid)
    cols = {}
    state = {"feats": None, "ref": None}

    def run(j):
        delta = max(1, int(round(default * 2.0 ** j)))
        plan = G.plan(pairs, mode=mode, delta=delta, stream=s.cuda_stream, **opts)
        if state["feats"] is None:
            state["feats"] = plan.features()
        best = None
        for _ in range(reps + 1):  # first run warms up
            plan.run(out.data_ptr())
            plan.sync()
            t = plan.group_times().astype(np.float64)
            best = t if best is None else np.minimum(best, t)
        res = out.cpu().numpy().copy()
        if state["ref"] is None:
            state["ref"] = res
        elif not np.array_equal(state["ref"], res):  # Delta must not change answers
            raise AssertionError(f"answers changed with delta={delta}")
        plan.close()
        cols[j] = best
        return best.sum()

    j0 = grid.index(start)
    best_total = run(start)
    for direction in (-1, 1):
        worse, k = 0, j0 + direction
        while 0 <= k < len(grid) and worse < patience:
            tot = run(grid[k])
            if tot < best_total:
                best_total, worse = tot, 0
            else:
                worse += 1
                if tot > 5 * best_total:  # far past the optimum: stop walking this way
                    break
            k += direction
    ng = state["feats"].shape[0]
    times = np.full((ng, len(grid)), np.inf)
    for j, col in cols.items():
        times[:, grid.index(j)] = col
    return state["feats"], times, default


def labels_from_times(times: np.ndarray, grid=GRID, tie: float = 0.05) -> np.ndarray:
    """Label of each group: the smallest grid point whose time is within
    `tie` of the group's best.  Time grows slowly as Delta shrinks below the
    best and steeply (many more re-extractions) as it grows above it, so a
    near-tie is broken towards the smaller increment."""
    best = times.min(axis=1, keepdims=True)
    ok = times <= best * (1.0 + tie)
    first = np.argmax(ok, axis=1)  # grid is increasing: the first True is the smallest Delta
    return np.asarray(grid, dtype=np.float32)[first]


def regret(times: np.ndarray, y_pred: np.ndarray, grid=GRID) -> float:
    """Time at the measured grid point nearest each prediction over the best."""
    ok = _finite_cols(times)
    g = np.asarray(grid, dtype=np.float64)[ok]
    times = times[:, ok]
    idx = np.abs(np.clip(y_pred, g[0], g[-1])[:, None] - g[None, :]).argmin(axis=1)
    chosen = times[np.arange(times.shape[0]), idx].sum()
    return float(chosen / times.min(axis=1).sum() - 1.0)


def doubling_regret(times: np.ndarray, grid=GRID):
    """Regret of the paper's rule (Sec. 6.1): one Delta for the whole graph,
    found by doubling until the time stops improving -- here the grid point
    with the smallest total time over the swept points (the sweep walks the
    grid the same way, so it visits the rule's choice).  Returns (regret,
    chosen grid point)."""
    ok = _finite_cols(times)
    if not ok.any():
        return None, None
    tot = times[:, ok].sum(axis=0)
    j = int(np.argmin(tot))
    return float(tot[j] / times.min(axis=1).sum() - 1.0), int(np.asarray(grid)[ok][j])


def default_regret(times: np.ndarray, grid=GRID):
    """Regret of the default increment, or None when the sweep never timed it."""
    j0 = list(grid).index(0)
    if not np.isfinite(times[:, j0]).all():
        return None
    return float(times[:, j0].sum() / times.min(axis=1).sum() - 1.0)


def _finite_cols(times: np.ndarray) -> np.ndarray:
    return np.isfinite(times).all(axis=0)


def init_params(feats: np.ndarray, seed: int = 0) -> np.ndarray:
    """Standardisation from the training features; He-normal weights."""
    rng = np.random.default_rng(seed)
    mean = feats.mean(axis=0)
    std = feats.std(axis=0)
    std = np.where(std < 1e-3, 1.0, std)
    parts = [mean, std,
             rng.normal(scale=np.sqrt(2.0 / 12), size=64 * 12), np.zeros(64),
             rng.normal(scale=np.sqrt(2.0 / 64), size=64 * 64), np.zeros(64),
             rng.normal(scale=np.sqrt(1.0 / 64), size=64), np.zeros(1)]
    p = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in parts]).astype(np.float32)
    assert p.shape == (ppsp.MLP_PARAMS,)
    return p


def train(feats: np.ndarray, labels: np.ndarray, epochs: int = 600, lr: float = 3e-3, seed: int = 0):
    model = ppsp.DeltaModel(init_params(feats, seed))
    loss = model.train(feats, labels, epochs, lr)
    return model, loss


def save(model: ppsp.DeltaModel, mode: str, meta: dict, directory: str = WEIGHTS_DIR) -> str:
    os.makedirs(directory, exist_ok=True)
    path = os.path.join(directory, f"delta_{mode}.bin")
    model.params().astype("<f4").tofile(path)
    with open(path[:-4] + ".json", "w") as f:
        json.dump(meta, f, indent=1, sort_keys=True)
    return path


def load_model(mode: str, directory: str = WEIGHTS_DIR):
    path = os.path.join(directory, f"delta_{mode}.bin")
    if not os.path.exists(path):
        return None
    p = np.fromfile(path, dtype="<f4")
    if p.shape != (ppsp.MLP_PARAMS,):
        return None
    return ppsp.DeltaModel(p)


def _training_sets(mode: str, build: bool = True):
    """Query sets used for training: held-out seeds, several graph shapes.
    With build=False only the names and sweep starts are returned (graphs and
    pairs None), for training from stored sweeps."""
    from workloads import near_mid_far_pairs, random_pairs, rmat_graph, road_like_graph, grid_graph, clique_pairs

    if not build:
        names = [("road1024", 0), ("road512", 0), ("grid64", 0), ("road2048", -3), ("road4096", -4)]
        if mode == "bids":
            names.append(("rmat18", 0))
        return [(n, None, None, st) for n, st in names]
    # (name, graph, pairs, first grid point of the sweep)
    sets = []
    # a 1024^2 road-like graph of its own seed (the benchmark graphs of every
    # size are held out for evaluation)
    g = road_like_graph(1024, seed=9601)
    p, _ = near_mid_far_pairs(g, 1000, seed=9602)
    sets.append(("road1024", g, p, 0))
    g = road_like_graph(512, seed=9001)
    p, _ = near_mid_far_pairs(g, 600, seed=9002)
    sets.append(("road512", g, np.concatenate([p, clique_pairs(g, 12, 9003)]), 0))
    g = grid_graph(64, seed=9101)
    sets.append(("grid64", g, random_pairs(g, 300, 9102), 0))
    # larger road-like graphs (other seeds than the benchmark and serving
    # graphs): the increment that works shrinks with graph size
    g = road_like_graph(2048, seed=9401)
    p, _ = near_mid_far_pairs(g, 300, seed=9402)
    sets.append(("road2048", g, p, -3))
    g = road_like_graph(4096, seed=9501)
    p, _ = near_mid_far_pairs(g, 120, seed=9502)
    sets.append(("road4096", g, p, -4))
    if mode == "bids":
        g = rmat_graph(18, seed=9201)
        sets.append(("rmat18", g, random_pairs(g, 128, 9202), 0))
    return sets


def ceil_regret(times: np.ndarray, y_pred: np.ndarray, grid=GRID) -> float:
    """Like `regret`, but a prediction between two grid points is charged the
    time of the larger increment (the pessimistic side of the steep curve)."""
    ok = _finite_cols(times)
    g = np.asarray(grid, dtype=np.float64)[ok]
    times = times[:, ok]
    idx = np.searchsorted(g, np.clip(y_pred, g[0], g[-1]) - 1e-6)
    chosen = times[np.arange(times.shape[0]), np.minimum(idx, g.shape[0] - 1)].sum()
    return float(chosen / times.min(axis=1).sum() - 1.0)


MARGINS = tuple(np.arange(0.0, 1.51, 0.25))


def build_and_train(mode: str, out_dir: str = WEIGHTS_DIR, epochs: int = 600, log=print,
                    sweeps_dir: str | None = None, evaluate_sets: bool = True) -> dict:
    """Sweep Delta on the training sets (or load earlier sweeps from
    `sweeps_dir`), train, pick a safety margin, report regret, save weights.

    The margin m is subtracted from every prediction (folded into the output
    bias): the smallest m in MARGINS that minimises the summed pessimistic
    regret (`ceil_regret`) over the training sets."""
    feats_all, labels_all, times_all, meta_sets = [], [], [], []
    t0 = time.time()
    os.makedirs(out_dir, exist_ok=True)
    for name, g, pairs, start in _training_sets(mode, build=sweeps_dir is None):
        if sweeps_dir is not None:
            d = np.load(os.path.join(sweeps_dir, f"sweep_{mode}_{name}.npz"))
            feats, times, default = d["feats"], d["times"], int(d["default"])
        else:
            with ppsp.Graph.from_csr(g, with_coords=g.coords is not None) as G:
                m = mode if (mode != "bidastar" or g.coords is not None) else "bids"
                feats, times, default = sweep(G, pairs, m, start=start)
        lab = labels_from_times(times)
        np.savez_compressed(os.path.join(out_dir, f"sweep_{mode}_{name}.npz"), feats=feats, times=times,
                            default=default)
        feats_all.append(feats)
        labels_all.append(lab)
        times_all.append(times)
        meta_sets.append({"set": name, "groups": int(feats.shape[0]), "default_delta": default,
                          "default_regret": default_regret(times),
                          "swept": [j for j, ok in zip(GRID, _finite_cols(times)) if ok],
                          "label_hist": {str(j): int((lab == j).sum()) for j in GRID if (lab == j).any()}})
        log(json.dumps(meta_sets[-1]))
    F = np.concatenate(feats_all)
    Y = np.concatenate(labels_all)
    model, loss = train(F, Y, epochs=epochs)
    pred = model.predict(F)
    # safety margin against the steep side of the time curve
    offs = np.cumsum([0] + [f.shape[0] for f in feats_all])
    scores = []
    for mg in MARGINS:
        scores.append(sum(ceil_regret(t, pred[offs[i]:offs[i + 1]] - mg) for i, t in enumerate(times_all)))
    margin = float(MARGINS[int(np.argmin(scores))])
    if margin:
        params = model.params()
        params[-1] -= margin  # output bias b3
        model.close()
        model = ppsp.DeltaModel(params)
    for i, t in enumerate(times_all):
        meta_sets[i]["regret_learned"] = regret(t, pred[offs[i]:offs[i + 1]] - margin)
        meta_sets[i]["ceil_regret_learned"] = ceil_regret(t, pred[offs[i]:offs[i + 1]] - margin)
        meta_sets[i]["regret_doubling_rule"], meta_sets[i]["doubling_grid_point"] = doubling_regret(t)
    meta = {"mode": mode, "grid": list(GRID), "epochs": epochs, "train_loss": loss,
            "train_groups": int(F.shape[0]), "sets": meta_sets, "seconds": time.time() - t0,
            "features": "log2(1 + raw): h(s,t), deg(s), deg(t), w mean/std/min/max, n, m, |V_q|, |E_q|, "
                        "mean query-graph degree",
            "label_rule": "smallest grid point within 5% of the group's best time",
            "margin": margin, "margin_scores": {str(float(m)): float(v) for m, v in zip(MARGINS, scores)},
            "train_mae": float(np.abs(pred - Y).mean())}
    if evaluate_sets:
        meta["eval"] = evaluate(mode, log=log, model=model)
        meta["eval_large"] = evaluate_large(mode, log=log, model=model)
        if mode == "bidastar":
            meta["eval_batch2048"] = evaluate_batch2048(log=log, model=model)
    path = save(model, mode, meta, out_dir)
    log(json.dumps({"saved": path, "train_loss": loss, "train_mae": meta["train_mae"], "margin": margin}))
    model.close()
    return meta


def evaluate(mode: str, log=print, model=None) -> dict:
    """Regret of the model (default: the saved one) on the held-out road-like
    benchmark queries (the 1,000 near/mid/far pairs; training used other seeds)."""
    from workloads import config_workload

    wl = config_workload(2)
    g, pairs = wl["graph"], wl["batches"]["nmf"]
    own = model is None
    if own:
        model = load_model(mode)
    if model is None:
        raise FileNotFoundError(weights_path(mode))
    with ppsp.Graph.from_csr(g) as G:
        feats, times, default = sweep(G, pairs, mode)
    y = model.predict(feats)
    lab = labels_from_times(times)
    dr, dj = doubling_regret(times)
    res = {"mode": mode, "eval_set": "road1024 benchmark graph (held out of training), its 1,000 near/mid/far "
                                     "queries", "groups": int(feats.shape[0]),
           "regret_learned": regret(times, y), "regret_default": default_regret(times),
           "regret_doubling_rule": dr, "doubling_grid_point": dj,
           "best_grid_hist": {str(j): int((lab == j).sum()) for j in GRID if (lab == j).any()},
           "pred_mean": float(y.mean())}
    if own:
        model.close()
    log(json.dumps(res))
    return res


def evaluate_large(mode: str, log=print, model=None, k: int = 96) -> dict:
    """Regret on k random queries of the 4096^2 road-like serving graph (its own
    seed; training used other graphs of that size)."""
    from workloads import config_workload, random_pairs

    g = config_workload(5)["graph"]
    pairs = random_pairs(g, k, 5501)
    own = model is None
    if own:
        model = load_model(mode)
    if model is None:
        raise FileNotFoundError(weights_path(mode))
    with ppsp.Graph.from_csr(g) as G:
        feats, times, default = sweep(G, pairs, mode, start=-4)
    y = model.predict(feats)
    dr, dj = doubling_regret(times)
    res = {"mode": mode, "eval_set": f"road4096 serving graph, {k} random pairs", "groups": int(feats.shape[0]),
           "regret_learned": regret(times, y), "regret_default": default_regret(times),
           "regret_doubling_rule": dr, "doubling_grid_point": dj, "pred_mean": float(y.mean())}
    if own:
        model.close()
    log(json.dumps(res))
    return res


def evaluate_batch2048(log=print, model=None) -> dict:
    """Regret on the 2,048-query batch of the 2048^2 road-like graph (random
    pairs and a 32-clique answered as independent BiD-A* pairs, as the AUTO
    strategy runs them; held out of training)."""
    from workloads import config_workload

    wl = config_workload(4)
    g, pairs = wl["graph"], wl["batches"]["mixed"]
    own = model is None
    if own:
        model = load_model("bidastar")
    if model is None:
        raise FileNotFoundError(weights_path("bidastar"))
    with ppsp.Graph.from_csr(g) as G:
        feats, times, default = sweep(G, pairs, "bidastar", start=-3, strategy="auto")
    y = model.predict(feats)
    dr, dj = doubling_regret(times)
    res = {"mode": "bidastar", "eval_set": "road2048 batch of 2,048 queries (AUTO strategy)",
           "groups": int(feats.shape[0]), "regret_learned": regret(times, y), "regret_default": default_regret(times),
           "regret_doubling_rule": dr, "doubling_grid_point": dj, "pred_mean": float(y.mean())}
    if own:
        model.close()
    log(json.dumps(res))
    return res


if __name__ == "__main__":
    import sys

    root = os.path.dirname(HERE)
    sys.path.insert(0, root)
    import __graft_entry__

    __graft_entry__.build()
    args = sys.argv[1:]
    if args and args[0] == "eval":
        for md in args[1:] or ["bidastar", "bids"]:
            evaluate(md)
    else:
        for md in args or ["bidastar", "bids"]:
            build_and_train(md)
