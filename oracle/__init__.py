"""CPU oracle for the PPSP hot path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  It shares no code with the CUDA path
(``paper_2506_16488_gb300``) and never imports it.

* ``ppsp_oracle.c`` -- binary-heap Dijkstra (the plain definition of d(s,t),
  which Theorems 3.3/3.4 say BiDS and BiD-A* return exactly), full SSSP with
  parents, Floyd-Warshall for tiny graphs.
* ``potential.py`` -- the integer A* potential h_x(v) = floor(scaled Euclidean
  distance) (Sec. 3.3; Fact 3.1 consistency).
* ``mlp.py`` -- float64 forward/backward of the small stepping-threshold MLP.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppsp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF = np.uint64(0xFFFFFFFFFFFFFFFF)
INF_INT = 0xFFFFFFFFFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
            lib.oracle_dijkstra_pair.restype = u64
            lib.oracle_dijkstra_pair.argtypes = [u64, p, p, p, u32, u32, p]
            lib.oracle_sssp.restype = ctypes.c_int
            lib.oracle_sssp.argtypes = [u64, p, p, p, u32, p, p]
            lib.oracle_dijkstra_path.restype = u64
            lib.oracle_dijkstra_path.argtypes = [u64, p, p, p, u32, u32, p, u64, p]
            lib.oracle_floyd_warshall.restype = None
            lib.oracle_floyd_warshall.argtypes = [u64, p, p, p, p]
            lib.oracle_pairs.restype = ctypes.c_int
            lib.oracle_pairs.argtypes = [u64, p, p, p, p, u64, p, p]
            _lib = lib
    return _lib


def _csr(off, tgt, w):
    off = np.ascontiguousarray(off, dtype=np.uint64)
    tgt = np.ascontiguousarray(tgt, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    return off, tgt, w


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def dijkstra_pair(off, tgt, w, s: int, t: int, return_scanned: bool = False):
    """Exact d(s, t) (uint64 INF if unreachable)."""
    off, tgt, w = _csr(off, tgt, w)
    n = off.shape[0] - 1
    sc = ctypes.c_uint64(0)
    d = _load().oracle_dijkstra_pair(n, _ptr(off), _ptr(tgt), _ptr(w), s, t, ctypes.byref(sc))
    if d == INF_INT - 1:
        raise MemoryError("oracle allocation failed")
    return (d, sc.value) if return_scanned else d


def pairs(off, tgt, w, pairs_arr: np.ndarray, return_scanned: bool = False):
    """Distances of a [k, 2] pair array, answered one pair at a time."""
    off, tgt, w = _csr(off, tgt, w)
    pa = np.ascontiguousarray(pairs_arr, dtype=np.uint32).reshape(-1, 2)
    out = np.empty(pa.shape[0], dtype=np.uint64)
    sc = ctypes.c_uint64(0)
    rc = _load().oracle_pairs(off.shape[0] - 1, _ptr(off), _ptr(tgt), _ptr(w), _ptr(pa),
                              pa.shape[0], _ptr(out), ctypes.byref(sc))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (out, sc.value) if return_scanned else out


def pairs_threaded(off, tgt, w, pairs_arr: np.ndarray, threads: int):
    """Same as :func:`pairs`, one pair per worker thread (the C call releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    off, tgt, w = _csr(off, tgt, w)
    pa = np.ascontiguousarray(pairs_arr, dtype=np.uint32).reshape(-1, 2)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(lambda q: dijkstra_pair(off, tgt, w, int(q[0]), int(q[1])), pa))
    return np.array(res, dtype=np.uint64)


def sssp(off, tgt, w, s: int, with_parent: bool = False):
    off, tgt, w = _csr(off, tgt, w)
    n = off.shape[0] - 1
    dist = np.empty(n, dtype=np.uint64)
    par = np.empty(n, dtype=np.uint32) if with_parent else None
    rc = _load().oracle_sssp(n, _ptr(off), _ptr(tgt), _ptr(w), s, _ptr(dist),
                             _ptr(par) if par is not None else None)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (dist, par) if with_parent else dist


def path(off, tgt, w, s: int, t: int):
    """(d(s,t), one shortest path as a uint32 array; empty if unreachable)."""
    off, tgt, w = _csr(off, tgt, w)
    n = off.shape[0] - 1
    cap = 1024
    while True:
        buf = np.empty(cap, dtype=np.uint32)
        ln = ctypes.c_uint64(0)
        d = _load().oracle_dijkstra_path(n, _ptr(off), _ptr(tgt), _ptr(w), s, t, _ptr(buf), cap,
                                         ctypes.byref(ln))
        if d == INF_INT - 1:
            raise MemoryError("oracle allocation failed")
        if ln.value <= cap:
            return d, buf[: ln.value].copy()
        cap = int(ln.value)


def floyd_warshall(off, tgt, w):
    off, tgt, w = _csr(off, tgt, w)
    n = off.shape[0] - 1
    d = np.empty(n * n, dtype=np.uint64)
    _load().oracle_floyd_warshall(n, _ptr(off), _ptr(tgt), _ptr(w), _ptr(d))
    return d.reshape(n, n)


def path_weight(off, tgt, w, p) -> int:
    """Sum of edge weights along path p (the lightest parallel edge per hop);
    raises ValueError if two consecutive vertices are not adjacent."""
    total = 0
    for a, b in zip(p[:-1], p[1:]):
        lo, hi = int(off[a]), int(off[a + 1])
        row = tgt[lo:hi]
        hit = np.nonzero(row == b)[0]
        if hit.shape[0] == 0:
            raise ValueError(f"no edge {a}->{b}")
        total += int(w[lo:hi][hit].min())
    return total
