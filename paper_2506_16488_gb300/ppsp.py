"""Python binding of the C ABI in include/ppsp.h (argument marshalling only).

Every search step runs in the CUDA library lib/libppsp.so.  There is no
fallback: if the library is missing or cannot load, :func:`load` raises.
Names follow the C ABI (ppsp_graph_create -> Graph, ppsp_query -> Graph.query,
ppsp_batch -> Graph.batch, ppsp_plan_* -> Plan).
"""

from __future__ import annotations

import ctypes
import os
import threading
import weakref
from typing import Optional

import numpy as np

from . import _build

INF = 0xFFFFFFFFFFFFFFFF

# status codes
OK, ERR_INVALID_ARG, ERR_BAD_GRAPH, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NO_COORDS, \
    ERR_BUFFER_TOO_SMALL, ERR_OVERFLOW, ERR_UNSUPPORTED = range(10)
STATUS_NAMES = ["OK", "INVALID_ARG", "BAD_GRAPH", "OOM", "CUDA", "TIMEOUT", "NO_COORDS",
                "BUFFER_TOO_SMALL", "OVERFLOW", "UNSUPPORTED"]

MODES = {"bids": 0, "bidastar": 1, "et": 2, "astar": 3}
FRONTIER = {"auto": 0, "sparse": 1, "dense": 2}
LAYOUT = {"auto": 0, "interleaved": 1, "stacked": 2}
STRATEGY = {"multi": 0, "plain_star": 1, "plain": 2, "sssp": 3, "vc": 4, "auto": 5}
UNDIRECTED = 1
KEEP_VERTEX_ORDER = 2
DEBUG_BARRIER_NEVER_RELEASES = 1
MLP_FEATURES = 12
MLP_PARAMS = 5081


class Options(ctypes.Structure):
    """ppsp_options (include/ppsp.h), field for field; see make_options."""

    _fields_ = [
        ("mode", ctypes.c_int32),
        ("dist_bits", ctypes.c_int32),
        ("delta", ctypes.c_uint64),
        ("frontier", ctypes.c_int32),
        ("layout", ctypes.c_int32),
        ("batch_strategy", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("team_ctas", ctypes.c_int32),
        ("big_team_ctas", ctypes.c_int32),
        ("dense_den", ctypes.c_uint32),
        ("want_paths", ctypes.c_int32),
        ("max_ctas", ctypes.c_int32),
        ("spin_limit", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("debug_flags", ctypes.c_uint32),
        ("cuda_graph", ctypes.c_uint32),
        ("stepping_rho", ctypes.c_uint32),
        ("memo_potential", ctypes.c_uint32),
        ("pull_push", ctypes.c_uint32),
        ("ring_entries", ctypes.c_uint32),
        ("multi_potential", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 1),
    ]


class Counters(ctypes.Structure):
    """ppsp_counters: work done by one call (extracted X, edges E, relaxed R,
    pushed P, rounds, groups, searches, touched, dense rounds)."""

    _fields_ = [(name, ctypes.c_uint64) for name in
                ("extracted", "edges", "relaxed", "pushed", "rounds", "groups", "searches",
                 "touched", "dense_rounds")] + [("reserved", ctypes.c_uint64 * 7)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "reserved"}


class GraphInfo(ctypes.Structure):
    """ppsp_graph_info: properties computed when the graph was created."""

    _fields_ = [
        ("n", ctypes.c_uint64), ("m", ctypes.c_uint64),
        ("w_min", ctypes.c_uint64), ("w_max", ctypes.c_uint64),
        ("w_mean", ctypes.c_double), ("w_std", ctypes.c_double),
        ("deg_max", ctypes.c_uint64),
        ("potential_scale", ctypes.c_double),
        ("potential_shift", ctypes.c_int32),
        ("has_coords", ctypes.c_int32),
        ("undirected", ctypes.c_int32),
        ("has_zero_weight", ctypes.c_int32),
        ("device_bytes", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class PPSPError(RuntimeError):
    """A non-OK ppsp_status; ``status`` holds the code."""

    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{what}: PPSP_ERR_{name}" if what else f"PPSP_ERR_{name}")


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """Path of the in-tree CUDA library (lib/libppsp.so)."""
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load lib/libppsp.so (raises if absent unless build_if_missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"{_build.LIB} is missing: run __graft_entry__.build() first")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        p, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
        S = ctypes.c_int
        sig = {
            "ppsp_options_init": (None, [p]),
            "ppsp_status_string": (ctypes.c_char_p, [S]),
            "ppsp_last_error_detail": (ctypes.c_char_p, []),
            "ppsp_graph_create": (S, [u64, u64, p, p, p, p, u32, p]),
            "ppsp_graph_destroy": (None, [p]),
            "ppsp_graph_get_info": (S, [p, p]),
            "ppsp_query": (S, [p, u32, u32, p, p, p, u64, p]),
            "ppsp_batch": (S, [p, p, u64, p, p, p, p, p, p]),
            "ppsp_plan_create": (S, [p, p, u64, p, p]),
            "ppsp_plan_run": (S, [p, p]),
            "ppsp_plan_sync": (S, [p, p]),
            "ppsp_plan_destroy": (None, [p]),
            "ppsp_potential_coords": (S, [p, p]),
            "ppsp_potential_eval": (S, [p, u32, p, u64, p]),
            "ppsp_plan_features": (S, [p, p, u64, p]),
            "ppsp_plan_group_times": (S, [p, p, u64, p]),
            "ppsp_plan_uses_graph": (S, [p, p]),
            "ppsp_plan_device_bytes": (S, [p, p, p, p]),
            "ppsp_slot_bytes": (S, [p, u32, i32, i32, p]),
            "ppsp_batch_sources": (S, [p, u64, i32, u32, p, p, p]),
            "ppsp_vertex_order": (S, [u64, p, p]),
            "ppsp_delta_model_create": (S, [p, p]),
            "ppsp_delta_model_destroy": (None, [p]),
            "ppsp_delta_model_get_params": (S, [p, p]),
            "ppsp_delta_model_predict": (S, [p, p, u64, p]),
            "ppsp_delta_model_grad": (S, [p, p, p, u64, p, p]),
            "ppsp_delta_model_train": (S, [p, p, p, u64, u32, ctypes.c_float, p]),
            "ppsp_graph_set_delta_model": (S, [p, i32, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != OK:
        detail = ""
        if status == ERR_CUDA:
            d = load().ppsp_last_error_detail()
            detail = f" ({d.decode()})" if d else ""
        raise PPSPError(status, what + detail)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def batch_sources(pairs, strategy: str | int = "vc", undirected: bool = True, return_dirs: bool = False):
    """Sources of an SSSP-based batch (Sec. 4.3), computed on the host:
    (per-pair source vertex, 0xFFFFFFFF where s == t; number of distinct
    searches) and, with return_dirs, each pair's search direction (1 =
    backward from its target over in-edges).  strategy "sssp" = each query's
    own source, "vc" = an endpoint in a vertex cover of the query graph
    (bipartite and minimum on a directed graph)."""
    pa = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    k = pa.shape[0]
    out = np.zeros(max(1, k), dtype=np.uint32)
    dirs = np.zeros(max(1, k), dtype=np.uint32)
    n = ctypes.c_uint64(0)
    st = STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    _check(load().ppsp_batch_sources(_ptr(pa), k, st, UNDIRECTED if undirected else 0, _ptr(out), _ptr(dirs),
                                     ctypes.byref(n)), "ppsp_batch_sources")
    if return_dirs:
        return out[:k], int(n.value), dirs[:k]
    return out[:k], int(n.value)


def vertex_order(coords) -> np.ndarray:
    """perm[v] = the device id ppsp_graph_create gives vertex v of a graph
    with these coordinates (float [n, 2]; host only)."""
    xy = np.ascontiguousarray(coords, dtype=np.float32).reshape(-1, 2)
    out = np.zeros(xy.shape[0], dtype=np.uint32)
    _check(load().ppsp_vertex_order(xy.shape[0], _ptr(xy), _ptr(out)), "ppsp_vertex_order")
    return out


def make_options(mode: str | int = "bids", dist_bits: int = 32, delta: int = 0, frontier="auto",
                 layout="auto", strategy="multi", block_threads: int = 0, team_ctas: int = 0,
                 big_team_ctas: int = 0, dense_den: int = 0, want_paths: bool = False, max_ctas: int = 0,
                 spin_limit: int = 0, stream: int | None = None, debug_flags: int = 0,
                 cuda_graph: bool = False, stepping_rho: int = 0, memo_potential: bool = False,
                 pull_push: bool = False, ring_entries: int = 0, multi_potential: bool = False) -> Options:
    """ppsp_options from keyword arguments: the library's defaults
    (ppsp_options_init) overridden by the given values; enum fields accept
    names ("bidastar", "auto", ...) or numbers.  `stream` is a cudaStream_t
    as an int (e.g. torch.cuda.Stream().cuda_stream)."""
    o = Options()
    load().ppsp_options_init(ctypes.byref(o))
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.dist_bits = dist_bits
    o.delta = delta
    o.frontier = FRONTIER[frontier] if isinstance(frontier, str) else int(frontier)
    o.layout = LAYOUT[layout] if isinstance(layout, str) else int(layout)
    o.batch_strategy = STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    o.block_threads = block_threads
    o.team_ctas = team_ctas
    o.big_team_ctas = big_team_ctas
    o.dense_den = dense_den
    o.want_paths = int(bool(want_paths))
    o.max_ctas = max_ctas
    o.spin_limit = spin_limit
    o.stream = stream
    o.debug_flags = debug_flags
    o.cuda_graph = int(bool(cuda_graph))
    o.stepping_rho = stepping_rho
    o.memo_potential = int(bool(memo_potential))
    o.pull_push = int(bool(pull_push))
    o.ring_entries = ring_entries
    o.multi_potential = int(bool(multi_potential))
    return o


class Graph:
    """Device-resident CSR graph (ppsp_graph_create / ppsp_graph_destroy)."""

    def __init__(self, offsets, targets, weights, coords=None, undirected: bool = True, keep_order: bool = False):
        lib = load()
        self._off = np.ascontiguousarray(offsets, dtype=np.uint64)
        tgt = np.ascontiguousarray(targets, dtype=np.uint32)
        w = np.ascontiguousarray(weights, dtype=np.uint32)
        xy = None if coords is None else np.ascontiguousarray(coords, dtype=np.float32).reshape(-1)
        n = self._off.shape[0] - 1
        h = ctypes.c_void_p()
        st = lib.ppsp_graph_create(n, tgt.shape[0], _ptr(self._off), _ptr(tgt), _ptr(w), _ptr(xy),
                                   (UNDIRECTED if undirected else 0) | (KEEP_VERTEX_ORDER if keep_order else 0),
                                   ctypes.byref(h))
        _check(st, "ppsp_graph_create")
        self._h = h
        self.n = n
        self.m = int(tgt.shape[0])
        self._plans = weakref.WeakSet()
        self._models = {}

    @classmethod
    def from_csr(cls, g, undirected: bool = True, with_coords: bool = True, keep_order: bool = False):
        """From an object with offsets, targets, weights and coords (a
        workloads.CSRGraph).  keep_order keeps the caller's vertex order on
        the device (default: a Hilbert-curve order over the coordinates;
        ids are mapped at the boundary either way)."""
        return cls(g.offsets, g.targets, g.weights, g.coords if with_coords else None, undirected, keep_order)

    def close(self):
        """Destroy the graph; its open plans are destroyed first (a plan
        belongs to its graph and must not outlive it)."""
        for p in list(getattr(self, "_plans", ())):
            p.close()
        if getattr(self, "_h", None):
            load().ppsp_graph_destroy(self._h)
            self._h = None
        self._models = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _handle(self):
        if not getattr(self, "_h", None):
            raise PPSPError(ERR_INVALID_ARG, "graph is closed")
        return self._h

    def info(self) -> dict:
        """ppsp_graph_get_info as a dict."""
        gi = GraphInfo()
        _check(load().ppsp_graph_get_info(self._handle(), ctypes.byref(gi)), "ppsp_graph_get_info")
        return gi.as_dict()

    def query(self, s: int, t: int, **opts) -> int:
        """d(s, t) (INF if unreachable) by ppsp_query; opts as make_options."""
        o = make_options(**opts)
        d = ctypes.c_uint64(0)
        plen = ctypes.c_uint64(0)
        st = load().ppsp_query(self._handle(), s, t, ctypes.byref(o), ctypes.byref(d), None, 0, ctypes.byref(plen))
        _check(st, "ppsp_query")
        return int(d.value)

    def query_status(self, s: int, t: int, **opts) -> tuple:
        """(status, distance) without raising (for error-path tests)."""
        o = make_options(**opts)
        d = ctypes.c_uint64(0)
        st = load().ppsp_query(self._handle(), s, t, ctypes.byref(o), ctypes.byref(d), None, 0, None)
        return int(st), int(d.value)

    def batch(self, pairs, return_counters: bool = False, out: Optional[np.ndarray] = None, **opts):
        """Distances of k pairs (uint64 [k], input order) by ppsp_batch, and
        the work counters with return_counters=True.  `out` (optional) is a
        caller-owned contiguous uint64 [k] array to write them to, e.g. in
        pinned host memory; contiguous uint32 pairs are read in place."""
        o = make_options(**opts)
        pa = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        k = pa.shape[0]
        if out is None:
            out = np.zeros(k, dtype=np.uint64)
        elif out.dtype != np.uint64 or out.shape != (k,) or not out.flags.c_contiguous:
            raise ValueError(f"out must be a contiguous uint64 array of {k} elements")
        c = Counters()
        st = load().ppsp_batch(self._handle(), _ptr(pa), k, ctypes.byref(o), _ptr(out), None, None, None,
                               ctypes.byref(c))
        _check(st, "ppsp_batch")
        return (out, c.as_dict()) if return_counters else out

    def query_path(self, s: int, t: int, cap: int = 1 << 16, **opts) -> tuple:
        """(status, distance, path as uint32 array or None if it did not fit, needed length)."""
        o = make_options(want_paths=True, **opts)
        d = ctypes.c_uint64(0)
        plen = ctypes.c_uint64(0)
        buf = np.zeros(max(1, cap), dtype=np.uint32)
        st = load().ppsp_query(self._handle(), s, t, ctypes.byref(o), ctypes.byref(d), _ptr(buf), cap, ctypes.byref(plen))
        n = int(plen.value)
        path = buf[:n].copy() if st == OK else None
        return int(st), int(d.value), path, n

    def batch_paths(self, pairs, caps, **opts) -> tuple:
        """(status, distances, list of paths (None where it did not fit), needed lengths)."""
        o = make_options(want_paths=True, **opts)
        pa = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        k = pa.shape[0]
        caps = np.broadcast_to(np.asarray(caps, dtype=np.uint64), (k,))
        off = np.zeros(k + 1, dtype=np.uint64)
        np.cumsum(caps, out=off[1:])
        buf = np.zeros(max(1, int(off[-1])), dtype=np.uint32)
        out = np.zeros(k, dtype=np.uint64)
        lens = np.zeros(k, dtype=np.uint64)
        st = load().ppsp_batch(self._handle(), _ptr(pa), k, ctypes.byref(o), _ptr(out), _ptr(buf), _ptr(off), _ptr(lens),
                               None)
        paths = [buf[int(off[q]):int(off[q]) + int(lens[q])].copy() if lens[q] <= caps[q] else None
                 for q in range(k)]
        return int(st), out, paths, lens

    def batch_status(self, pairs, **opts) -> tuple:
        """(status, distances) without raising (for error-path tests)."""
        o = make_options(**opts)
        pa = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        out = np.zeros(pa.shape[0], dtype=np.uint64)
        st = load().ppsp_batch(self._handle(), _ptr(pa), pa.shape[0], ctypes.byref(o), _ptr(out), None, None,
                               None, None)
        return int(st), out

    def plan(self, pairs, **opts) -> "Plan":
        """A prepared batch (ppsp_plan_create) owned by this graph."""
        return Plan(self, pairs, **opts)

    def slot_bytes(self, searches: int = 2, dist_bits: int = 32, frontier="auto") -> int:
        """Device bytes of the slot one team of a batch allocates for groups
        of `searches` searches (ppsp_slot_bytes; host only)."""
        out = ctypes.c_uint64(0)
        f = FRONTIER[frontier] if isinstance(frontier, str) else int(frontier)
        _check(load().ppsp_slot_bytes(self._handle(), searches, dist_bits, f, ctypes.byref(out)), "ppsp_slot_bytes")
        return int(out.value)

    def set_delta_model(self, mode: str | int, model: Optional["DeltaModel"]):
        """Plans of this mode with delta=0 use the model (kept alive by the graph)."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        _check(load().ppsp_graph_set_delta_model(self._handle(), m, model._handle() if model else None),
               "ppsp_graph_set_delta_model")
        self._models[m] = model
        if model is not None:
            model._graphs.add(self)

    def potential_coords(self) -> np.ndarray:
        """Integer potential coordinates P(v) (int64 [n, 2])."""
        out = np.empty(2 * self.n, dtype=np.int64)
        _check(load().ppsp_potential_coords(self._handle(), _ptr(out)), "ppsp_potential_coords")
        return out.reshape(-1, 2)

    def potential_eval(self, anchor: int, vertices) -> np.ndarray:
        """h_anchor(v) for the given vertices, computed on the device."""
        v = np.ascontiguousarray(vertices, dtype=np.uint32)
        out = np.empty(v.shape[0], dtype=np.int64)
        _check(load().ppsp_potential_eval(self._handle(), anchor, _ptr(v), v.shape[0], _ptr(out)),
               "ppsp_potential_eval")
        return out


class Plan:
    """A prepared batch (ppsp_plan_create); run() writes distances to a device buffer."""

    def __init__(self, graph: Graph, pairs, **opts):
        self.graph = graph
        self._opts = make_options(**opts)
        pa = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        self.k = pa.shape[0]
        h = ctypes.c_void_p()
        _check(load().ppsp_plan_create(graph._handle(), _ptr(pa), self.k, ctypes.byref(self._opts),
                                       ctypes.byref(h)), "ppsp_plan_create")
        self._h = h
        graph._plans.add(self)

    def _handle(self):
        if not getattr(self, "_h", None):
            raise PPSPError(ERR_INVALID_ARG, "plan is closed")
        return self._h

    def run(self, d_out_ptr: int):
        """Launch the batch on the plan's stream; distances go to the device
        uint64 buffer at d_out_ptr (input order)."""
        _check(load().ppsp_plan_run(self._handle(), ctypes.c_void_p(d_out_ptr)), "ppsp_plan_run")

    def sync(self) -> dict:
        """Wait for the last run; raise on a device error; its counters."""
        c = Counters()
        _check(load().ppsp_plan_sync(self._handle(), ctypes.byref(c)), "ppsp_plan_sync")
        return c.as_dict()

    def features(self) -> np.ndarray:
        """Per-group model features, float32 [groups, 12]."""
        ng = ctypes.c_uint64(0)
        _check(load().ppsp_plan_features(self._handle(), None, 0, ctypes.byref(ng)), "ppsp_plan_features")
        out = np.zeros((ng.value, MLP_FEATURES), dtype=np.float32)
        _check(load().ppsp_plan_features(self._handle(), _ptr(out), ng.value, ctypes.byref(ng)), "ppsp_plan_features")
        return out

    def device_bytes(self) -> dict:
        """Device memory the plan holds (ppsp_plan_device_bytes): its teams'
        slots (one per team) and the rest (descriptors, paths)."""
        sb, nt, ob = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(load().ppsp_plan_device_bytes(self._handle(), ctypes.byref(sb), ctypes.byref(nt), ctypes.byref(ob)),
               "ppsp_plan_device_bytes")
        return {"slot_bytes": int(sb.value), "teams": int(nt.value), "other_bytes": int(ob.value)}

    def uses_graph(self) -> bool:
        """Whether the last run replayed a captured CUDA graph."""
        v = ctypes.c_int32(0)
        _check(load().ppsp_plan_uses_graph(self._handle(), ctypes.byref(v)), "ppsp_plan_uses_graph")
        return bool(v.value)

    def group_times(self) -> np.ndarray:
        """Device ns per group of the last run, uint64 [groups]."""
        ng = ctypes.c_uint64(0)
        _check(load().ppsp_plan_group_times(self._handle(), None, 0, ctypes.byref(ng)), "ppsp_plan_group_times")
        out = np.zeros(ng.value, dtype=np.uint64)
        _check(load().ppsp_plan_group_times(self._handle(), _ptr(out), ng.value, ctypes.byref(ng)),
               "ppsp_plan_group_times")
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().ppsp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class DeltaModel:
    """The stepping-increment MLP on the device (ppsp_delta_model_*)."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (MLP_PARAMS,):
            raise ValueError(f"expected {MLP_PARAMS} parameters, got shape {p.shape}")
        h = ctypes.c_void_p()
        _check(load().ppsp_delta_model_create(_ptr(p), ctypes.byref(h)), "ppsp_delta_model_create")
        self._h = h
        self._graphs = weakref.WeakSet()  # graphs that borrow this model

    def _handle(self):
        if not getattr(self, "_h", None):
            raise PPSPError(ERR_INVALID_ARG, "model is closed")
        return self._h

    def params(self) -> np.ndarray:
        """The fp32 master copy of the parameters."""
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(load().ppsp_delta_model_get_params(self._handle(), _ptr(out)), "ppsp_delta_model_get_params")
        return out

    def predict(self, feats) -> np.ndarray:
        """y = log2(Delta / Delta_default) per feature row."""
        f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, MLP_FEATURES)
        out = np.empty(f.shape[0], dtype=np.float32)
        _check(load().ppsp_delta_model_predict(self._handle(), _ptr(f), f.shape[0], _ptr(out)),
               "ppsp_delta_model_predict")
        return out

    def grad(self, feats, labels) -> tuple:
        """(gradient of the mean squared error, the loss)."""
        f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, MLP_FEATURES)
        y = np.ascontiguousarray(labels, dtype=np.float32)
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float(0)
        _check(load().ppsp_delta_model_grad(self._handle(), _ptr(f), _ptr(y), f.shape[0], _ptr(g), ctypes.byref(loss)),
               "ppsp_delta_model_grad")
        return g, float(loss.value)

    def train(self, feats, labels, epochs: int, lr: float) -> float:
        """Full-batch Adam steps on the device; the loss before the last."""
        f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, MLP_FEATURES)
        y = np.ascontiguousarray(labels, dtype=np.float32)
        loss = ctypes.c_float(0)
        _check(load().ppsp_delta_model_train(self._handle(), _ptr(f), _ptr(y), f.shape[0], epochs, lr,
                                             ctypes.byref(loss)), "ppsp_delta_model_train")
        return float(loss.value)

    def close(self):
        """Destroy the model after detaching it from every open graph that
        borrows it (graphs keep a pointer to it, not a copy)."""
        for g in list(getattr(self, "_graphs", ())):
            for mode, mm in list(g._models.items()):
                if mm is self and getattr(g, "_h", None):
                    g.set_delta_model(mode, None)
        if getattr(self, "_h", None):
            load().ppsp_delta_model_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
