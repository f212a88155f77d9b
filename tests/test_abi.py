"""The C-ABI library loads and exports every symbol include/bfs.h declares;
host-side argument checks reject bad calls before any launch. CPU only."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_1704_02259_gb300 as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"BFS_API\s+[\w\s\*]+?\b(\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    gb.build()
    return gb.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly what the header declares
    assert names == set(gb.SIGNATURES)


def test_config_defaults(lib):
    c = gb.default_config()
    assert c.policy == gb.POLICY_EDGE and c.alpha == 20.0 and c.beta == 200.0
    assert 1 <= c.bu_probe <= 64 and c.td_warp_degree <= c.td_grid_degree


def _last_error(lib):
    return lib.bfs_last_error().decode()


def test_generate_rejects_bad_arguments(lib):
    P = ctypes.c_void_p
    buf = P(0x1000)  # never dereferenced: the checks run first
    assert lib.bfs_generate_edges(0, 0, 16, 1, .57, .19, .19, buf, buf, None) == 1
    assert lib.bfs_generate_edges(0, 31, 16, 1, .57, .19, .19, buf, buf, None) == 1
    assert lib.bfs_generate_edges(7, 10, 16, 1, .57, .19, .19, buf, buf, None) == 1
    assert lib.bfs_generate_edges(0, 10, 16, 1, .6, .3, .2, buf, buf, None) == 1
    assert lib.bfs_generate_edges(0, 10, 16, 1, .57, .19, .19, None, buf, None) == 1
    assert _last_error(lib) != ""


def test_csr_and_roots_reject_bad_arguments(lib):
    P = ctypes.c_void_p
    buf = P(0x1000)
    nnz = ctypes.c_int64(0)
    assert lib.bfs_build_csr(0, 1, buf, buf, buf, buf, ctypes.byref(nnz), None) == 1
    assert lib.bfs_build_csr(1 << 31, 1, buf, buf, buf, buf, ctypes.byref(nnz), None) == 1
    assert lib.bfs_build_csr(10, 5, None, buf, buf, buf, ctypes.byref(nnz), None) == 1
    got = ctypes.c_int32(0)
    assert lib.bfs_sample_roots(buf, 10, 1, 0, 100, buf, ctypes.byref(got), None) == 1
    assert lib.bfs_sample_roots(buf, 10, 1, 5000, 100, buf, ctypes.byref(got), None) == 1


def test_graph_and_run_reject_bad_arguments(lib):
    h = ctypes.c_void_p(0)
    buf = ctypes.c_void_p(0x1000)
    assert lib.bfs_graph_create(buf, buf, 0, 0, 0, None, ctypes.byref(h)) == 1
    assert lib.bfs_graph_create(buf, buf, 10, -1, 0, None, ctypes.byref(h)) == 1
    assert lib.bfs_graph_create(buf, buf, 10, 5, gb.BORROW, None, ctypes.byref(h)) == 1
    bad = gb.default_config()
    bad.bu_probe = 0
    assert lib.bfs_graph_create(buf, buf, 10, 5, gb.DEVICE_PTRS | gb.BORROW, ctypes.byref(bad),
                                ctypes.byref(h)) == 1
    assert lib.bfs_run(None, 0, buf, buf, None) == 1
    assert lib.bfs_graph_destroy(None) == 0
    assert lib.bfs_last_run_stats(None, None, 0, None, None) == 1


STRUCTS = {"Config": "bfs_config", "LayerStats": "bfs_layer_stats",
           "BatchConfig": "bfs_batch_config", "BatchLayerStats": "bfs_batch_layer_stats",
           "ServeConfig": "bfs_serve_config", "ServeStats": "bfs_serve_stats"}


def test_struct_layouts_match_the_header(tmp_path):
    # a C program compiled against include/bfs.h prints every field's offset
    # and every struct's size; the ctypes classes must agree exactly
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bfs.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        cls = getattr(gb, py)
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in cls._fields_:
            lines.append(f'printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        py, field, value = line.split()
        cls = getattr(gb, py)
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (py, field, got, value)
