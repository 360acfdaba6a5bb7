"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, and rejects malformed input on the host before touching the device."""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_2506_16488_gb300 import ppsp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return ppsp.load()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ppsp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "ppsp_query" in names and "ppsp_batch" in names and "ppsp_graph_create" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_options_defaults(lib):
    o = ppsp.Options()
    lib.ppsp_options_init(ctypes.byref(o))
    assert o.mode == 0 and o.dist_bits == 32 and o.delta == 0 and o.batch_strategy == 0
    assert o.block_threads == 0 and o.stepping_rho == 0 and o.cuda_graph == 0 and o.want_paths == 0
    assert lib.ppsp_status_string(ppsp.ERR_TIMEOUT) == b"device wait timed out"


def _create(lib, off, tgt, w, flags=1):
    h = ctypes.c_void_p()
    off = np.ascontiguousarray(off, dtype=np.uint64)
    tgt = np.ascontiguousarray(tgt, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    st = lib.ppsp_graph_create(off.shape[0] - 1, tgt.shape[0], off.ctypes.data, tgt.ctypes.data,
                               w.ctypes.data, None, flags, ctypes.byref(h))
    return st, h


def test_host_validation_rejects_bad_graphs(lib):
    # offsets not ending at m
    assert _create(lib, [0, 1, 3], [1, 0], [5, 5])[0] == ppsp.ERR_BAD_GRAPH
    # decreasing offsets
    assert _create(lib, [0, 2, 1, 2], [1, 2], [1, 1])[0] == ppsp.ERR_BAD_GRAPH
    # target out of range
    assert _create(lib, [0, 1, 2], [1, 7], [1, 1])[0] == ppsp.ERR_BAD_GRAPH
    # undirected flag but asymmetric weights
    assert _create(lib, [0, 1, 2], [1, 0], [3, 4])[0] == ppsp.ERR_BAD_GRAPH
    # undirected flag but a missing reverse edge
    assert _create(lib, [0, 1, 1], [1], [3])[0] == ppsp.ERR_BAD_GRAPH
    # n = 0
    h = ctypes.c_void_p()
    off = np.zeros(1, dtype=np.uint64)
    assert lib.ppsp_graph_create(0, 0, off.ctypes.data, None, None, None, 1, ctypes.byref(h)) == \
        ppsp.ERR_INVALID_ARG
    # null out pointer
    assert lib.ppsp_graph_create(1, 0, off.ctypes.data, None, None, None, 1, None) == ppsp.ERR_INVALID_ARG


def test_null_handles_are_rejected(lib):
    d = ctypes.c_uint64()
    assert lib.ppsp_query(None, 0, 0, None, ctypes.byref(d), None, 0, None) == ppsp.ERR_INVALID_ARG
    assert lib.ppsp_batch(None, None, 0, None, None, None, None, None, None) == ppsp.ERR_INVALID_ARG
    assert lib.ppsp_plan_run(None, None) == ppsp.ERR_INVALID_ARG
    lib.ppsp_graph_destroy(None)
    lib.ppsp_plan_destroy(None)


def test_python_structs_mirror_the_c_layout(tmp_path):
    # sizes and field offsets of the option / counter / info structs as the C
    # compiler lays them out from include/ppsp.h
    import os
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    fields = [f for f, _ in ppsp.Options._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ppsp.h"', "int main(void) {",
             '  printf("%zu %zu %zu\\n", sizeof(ppsp_options), sizeof(ppsp_counters), sizeof(ppsp_graph_info));']
    for f in fields:
        lines.append(f'  printf("%zu\\n", offsetof(ppsp_options, {f}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    so, sc, si = (int(x) for x in out[:3])
    assert so == ctypes.sizeof(ppsp.Options)
    assert sc == ctypes.sizeof(ppsp.Counters)
    assert si == ctypes.sizeof(ppsp.GraphInfo)
    for f, off in zip(fields, out[3:]):
        assert getattr(ppsp.Options, f).offset == int(off), f
