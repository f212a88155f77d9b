"""The scripts that write the full-size expected values (tests/golden/make_*.py)
run at small sizes and must give the digests of plain, unchunked oracle calls;
the committed files must have the shape the GPU tests read. CPU only."""
from __future__ import annotations

import hashlib
import importlib.util
import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(GOLDEN, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype=a.dtype.newbyteorder("<")).data).hexdigest()


def _graph(scale, ef, seed):
    s, d = oracle.gen_edges(oracle.RMAT, scale, ef, seed)      # one call, no chunks
    return oracle.build_csr(1 << scale, s, d)


def test_single_source_script(tmp_path, monkeypatch):
    m = _load("make_rmat26_bfs")
    monkeypatch.setattr(m, "SCALE", 11)
    monkeypatch.setattr(m, "N_ROOTS", 8)
    monkeypatch.setattr(m, "N_EXACT", 3)
    monkeypatch.setattr(m, "OUT", str(tmp_path / "g.json"))
    m.main()
    rec = json.loads((tmp_path / "g.json").read_text())
    off, idx = _graph(11, m.EF, m.GRAPH_SEED)
    assert rec["nnz"] == idx.size
    assert rec["offsets_sha256"] == _sha(off) and rec["indices_sha256"] == _sha(idx)
    roots = oracle.sample_roots(off, 1 << 11, m.ROOT_SEED, 8)
    assert rec["roots"] == roots.tolist()
    for e, r in zip(rec["exact"], roots[:3]):
        lv, _ = oracle.bfs(off, idx, int(r))
        assert e["levels_sha256"] == _sha(lv)
        assert e["min_parent_sha256"] == _sha(oracle.min_parent(off, idx, int(r), lv))
        assert e["layer_sizes"] == np.bincount(lv[lv >= 0]).tolist()
        assert e["component_edges"] == oracle.component_edges(off, lv)


def test_batch_script(tmp_path, monkeypatch):
    m = _load("make_rmat22_batch")
    monkeypatch.setattr(m, "SCALE", 10)
    monkeypatch.setattr(m, "K", 16)
    monkeypatch.setattr(m, "OUT", str(tmp_path / "b.json"))
    m.main()
    rec = json.loads((tmp_path / "b.json").read_text())
    off, idx = _graph(10, m.EF, m.GRAPH_SEED)
    assert rec["indices_sha256"] == _sha(idx)
    roots = oracle.sample_roots(off, 1 << 10, m.ROOT_SEED, 16)
    assert [r["root"] for r in rec["rows"]] == roots.tolist()
    for row, r in zip(rec["rows"], roots):
        lv, _ = oracle.bfs(off, idx, int(r))
        assert row["int8_levels_sha256"] == hashlib.sha256(lv.astype(np.int8).data).hexdigest()
        assert row["reached"] == int((lv >= 0).sum())


def test_serve_script(tmp_path, monkeypatch):
    m = _load("make_serve8")
    monkeypatch.setattr(m, "SCALES", [8, 9])
    monkeypatch.setattr(m, "POOL", 64)
    monkeypatch.setattr(m, "PER_GRAPH", 2)
    monkeypatch.setattr(m, "OUT", str(tmp_path / "s.json"))
    m.main()
    rec = json.loads((tmp_path / "s.json").read_text())
    for i, gg in enumerate(rec["graphs"]):
        off, idx = _graph(gg["scale"], m.EF, 10 + i)
        assert gg["indices_sha256"] == _sha(idx)
        pool = oracle.sample_roots(off, 1 << gg["scale"], 5 + i, 64)
        assert gg["pool_sha256"] == _sha(pool)
        for q, r in zip(gg["queries"], pool[:2]):
            lv, _ = oracle.bfs(off, idx, int(r))
            assert q["root"] == int(r) and q["levels_sha256"] == _sha(lv)


def test_committed_files_have_the_expected_shape():
    g26 = json.load(open(os.path.join(GOLDEN, "rmat26_ef16_seed1_bfs.json")))
    assert (g26["scale"], g26["edgefactor"], g26["graph_seed"], g26["root_seed"]) == (26, 16, 1, 2)
    assert len(g26["roots"]) == 64 and len(g26["exact"]) == 8
    assert [e["root"] for e in g26["exact"]] == g26["roots"][:8]
    assert all(sum(e["layer_sizes"]) > 1 and e["layer_sizes"][0] == 1 for e in g26["exact"])
    b22 = json.load(open(os.path.join(GOLDEN, "rmat22_ef16_seed1_batch.json")))
    assert (b22["scale"], b22["root_seed"]) == (22, 4) and len(b22["rows"]) == 512
    assert all(0 < r["depth"] <= 127 for r in b22["rows"])
    s8 = json.load(open(os.path.join(GOLDEN, "serve8_rmat_levels.json")))
    assert [g["scale"] for g in s8["graphs"]] == [14, 16, 18, 19, 20, 21, 22, 23]
    assert all(len(g["queries"]) == 8 for g in s8["graphs"])
