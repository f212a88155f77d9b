"""GPU tests of the serving loop: every query's levels equal the oracle's
single-source levels of that root, whether it ran alone or batched into a
mixed stream; admission, capacity and shutdown behave as documented."""
from __future__ import annotations

import hashlib
import json
import threading
import time
from pathlib import Path

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02259_gb300 as gb
from tests.gpu_common import both_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graphs():
    out = []
    for kind, scale, seed in [(oracle.RMAT, 12, 10), (oracle.RMAT, 14, 11), (oracle.ER, 13, 12)]:
        n = 1 << scale
        s, d = oracle.gen_edges(kind, scale, 8, seed)
        o_off, o_idx, g_off, g_idx = both_csr(n, s, d)
        out.append((n, o_off, o_idx, gb.Graph(g_off, g_idx)))
    return out


def server_with(graphs, **kw):
    c = gb.default_serve_config()
    for k, v in kw.items():
        setattr(c, k, v)
    srv = gb.Server(c)
    ids = [srv.add_graph(g) for (_, _, _, g) in graphs]
    return srv, ids


def expected(graphs, gi, root, cache={}):
    key = (id(graphs[gi][1]), root)
    if key not in cache:
        cache[key] = oracle.bfs(graphs[gi][1], graphs[gi][2], root)[0]
    return cache[key]


def test_each_result_same_alone_and_in_the_mix(graphs):
    rng = np.random.default_rng(0)
    srv, ids = server_with(graphs, workers=3, max_batch=64)
    reqs = []
    for i in range(400):
        gi = int(rng.integers(0, len(graphs)))
        n = graphs[gi][0]
        root = int(rng.integers(0, n))
        if i % 3 == 0:
            out = torch.full((n,), 99, dtype=torch.int32).pin_memory()
        elif i % 3 == 1:
            out = torch.full((n,), 99, dtype=torch.int32)
        else:
            out = torch.full((n,), 99, dtype=torch.int32, device="cuda")
        reqs.append((gi, root, out, srv.submit(ids[gi], root, out)))
    for gi, root, out, t in reqs:
        assert srv.wait(t) == 0
    torch.cuda.synchronize()
    for gi, root, out, t in reqs:
        assert np.array_equal(out.cpu().numpy(), expected(graphs, gi, root))
    st = srv.stats()
    assert st["completed"] == 400 and st["failed"] == 0 and st["mean_batch"] >= 1
    srv.close()
    # alone: one query at a time through the same server path and through bfs_run
    srv, ids = server_with(graphs, workers=1, max_batch=1)
    for gi, root, _, _ in reqs[:12]:
        out = torch.empty(graphs[gi][0], dtype=torch.int32, device="cuda")
        assert srv.wait(srv.submit(ids[gi], root, out)) == 0
        solo, _ = graphs[gi][3].run(root)
        assert np.array_equal(out.cpu().numpy(), solo.cpu().numpy())
        assert np.array_equal(out.cpu().numpy(), expected(graphs, gi, root))
    srv.close()


def test_deep_queries_fall_back_to_single_source(graphs):
    # a 400-vertex path is 399 levels deep from its end, more than an int8
    # batch level holds: the batch returns BFS_ERR_DEPTH inside the worker,
    # which answers each of its queries with the single-source traversal;
    # mixed with ordinary queries of the other graphs, every result equals
    # the oracle's
    from tests import inputs
    n = 400
    s, d = inputs.path_edges(n)
    o_off, o_idx, g_off, g_idx = both_csr(n, s, d)
    path = (n, o_off, o_idx, gb.Graph(g_off, g_idx))
    allg = graphs + [path]
    srv, ids = server_with(allg, workers=2, max_batch=8)
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(60):
        gi = len(allg) - 1 if i % 3 == 0 else int(rng.integers(0, len(graphs)))
        nn = allg[gi][0]
        root = [0, n - 1, 150, 300][i % 4] if gi == len(allg) - 1 else int(rng.integers(0, nn))
        out = (torch.full((nn,), 99, dtype=torch.int32).pin_memory() if i % 2 else
               torch.full((nn,), 99, dtype=torch.int32, device="cuda"))
        reqs.append((gi, root, out, srv.submit(ids[gi], root, out)))
    for gi, root, out, t in reqs:
        assert srv.wait(t) == 0
    torch.cuda.synchronize()
    for gi, root, out, t in reqs:
        assert np.array_equal(out.cpu().numpy(), expected(allg, gi, root)), (gi, root)
    assert (expected(allg, len(allg) - 1, 0) == np.arange(n)).all()   # depth 399
    st = srv.stats()
    assert st["failed"] == 0 and st["deep_fallbacks"] >= 1
    srv.close()


def test_poisson_stream_reports_latency(graphs):
    srv, ids = server_with(graphs, workers=2, max_batch=128)
    rng = np.random.default_rng(1)
    reqs, lock = [], threading.Lock()

    def producer():
        for _ in range(300):
            gi = int(rng.integers(0, len(graphs)))
            root = int(rng.integers(0, graphs[gi][0]))
            out = torch.empty(graphs[gi][0], dtype=torch.int32, device="cuda")
            t = srv.submit(ids[gi], root, out)
            with lock:
                reqs.append((gi, root, out, t))
            time.sleep(rng.exponential(1 / 3000))

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    for gi, root, out, t in reqs:
        assert srv.wait(t) == 0
        assert np.array_equal(out.cpu().numpy(), expected(graphs, gi, root))
    st = srv.stats()
    assert st["completed"] == 300 and 0 < st["p50_us"] <= st["p99_us"] and st["qps"] > 0
    srv.close()


def test_stats_reset_starts_a_new_interval(graphs):
    srv, ids = server_with(graphs[:2], workers=2)
    n = graphs[0][0]
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(20)]
    for i, out in enumerate(outs):
        assert srv.wait(srv.submit(ids[0], i, out)) == 0
    assert srv.stats()["completed"] == 20
    srv.reset_stats()
    st = srv.stats()
    assert st["completed"] == 0 and st["batches"] == 0 and st["p99_us"] == 0
    for i, out in enumerate(outs[:5]):
        assert srv.wait(srv.submit(ids[0], 40 + i, out)) == 0
        assert np.array_equal(out.cpu().numpy(), expected(graphs, 0, 40 + i))
    st = srv.stats()
    assert st["completed"] == 5 and st["p50_us"] > 0 and st["qps"] > 0
    srv.close()


def test_memory_admission_splits_and_defers(graphs):
    n = graphs[1][0]
    # room for a few rows but not for a 256-root batch with its lane state
    # (a worker's view: 21n + 64 KiB of scratch; one lane word: seen and 8
    # frontier slots, 72n bytes; then 12 int8 level rows)
    budget = 21 * n + (1 << 16) + 72 * n + 4 * n + 8 * n
    srv, ids = server_with(graphs[1:2], workers=1, max_batch=256, memory_budget=budget)
    reqs = []
    for r in range(0, 200):
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        reqs.append((r, out, srv.submit(ids[0], r, out)))
    for r, out, t in reqs:
        assert srv.wait(t) == 0
        assert np.array_equal(out.cpu().numpy(), expected(graphs, 1, r))
    st = srv.stats()
    assert st["deferred"] > 0 and st["mean_batch"] < 256
    srv.close()


def test_memory_admission_rejects_what_never_fits(graphs):
    srv, ids = server_with(graphs[:1], workers=1, memory_budget=16)
    out = torch.empty(graphs[0][0], dtype=torch.int32, device="cuda")
    assert srv.wait(srv.submit(ids[0], 0, out)) == 2   # BFS_ERR_OOM
    assert srv.stats()["failed"] == 1
    srv.close()


def test_queue_capacity_and_bad_requests(graphs):
    srv, ids = server_with(graphs[1:2], workers=1, queue_capacity=4, max_batch=1)
    n = graphs[1][0]
    busy = 0
    outs = []
    for r in range(200):
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        try:
            outs.append((r, out, srv.submit(ids[0], r, out)))
        except gb.BfsError as e:
            assert e.status == 6          # BFS_ERR_BUSY
            busy += 1
    assert busy > 0
    for r, out, t in outs:
        assert srv.wait(t) == 0
        assert np.array_equal(out.cpu().numpy(), expected(graphs, 1, r))
    with pytest.raises(gb.BfsError):
        srv.submit(7, 0, outs[0][1])
    with pytest.raises(gb.BfsError):
        srv.submit(ids[0], n, outs[0][1])
    with pytest.raises(gb.BfsError):
        srv.wait(123456789)
    srv.close()


def test_shutdown_drains_or_cancels(graphs):
    n = graphs[1][0]
    srv, ids = server_with(graphs[1:2], workers=1, max_batch=8)
    outs = [torch.full((n,), 99, dtype=torch.int32, device="cuda") for _ in range(40)]
    for r, out in enumerate(outs):
        srv.submit(ids[0], r, out)
    srv.close()                                   # drains: every query completes
    torch.cuda.synchronize()
    for r, out in enumerate(outs):
        assert np.array_equal(out.cpu().numpy(), expected(graphs, 1, r))
    srv, ids = server_with(graphs[1:2], workers=1, max_batch=1, cancel_on_destroy=1)
    outs = [torch.full((n,), 99, dtype=torch.int32, device="cuda") for _ in range(60)]
    for r, out in enumerate(outs):
        srv.submit(ids[0], r, out)
    srv.close()                                   # cancels what is still queued
    torch.cuda.synchronize()
    for r, out in enumerate(outs):
        got = out.cpu().numpy()
        assert (got == 99).all() or np.array_equal(got, expected(graphs, 1, r))


GOLDEN_SERVE = Path(__file__).parent / "golden" / "serve8_rmat_levels.json"


def _sha(t: torch.Tensor) -> str:
    a = t.cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(a, dtype=a.dtype.newbyteorder("<")).data).hexdigest()


def test_serving_workload_full_size_matches_oracle_digests():
    """The serving workload at full size: 8 resident R-MAT graphs (scales 14,
    16, 18-23, edgefactor 16, seeds 10-17), the benchmark's server settings,
    a mixed stream of 2,000 queries submitted back to back; 8 queries per
    graph, spread through the stream, must equal the oracle's levels
    (digests written by tests/golden/make_serve8.py), and every CSR and root
    pool the oracle's."""
    gold = json.loads(GOLDEN_SERVE.read_text())
    graphs, pools = [], []
    for gg in gold["graphs"]:
        n = 1 << gg["scale"]
        off, idx = gb.rmat_graph(gg["scale"], gold["edgefactor"], gg["graph_seed"])
        assert idx.numel() == gg["nnz"]
        assert _sha(off) == gg["offsets_sha256"] and _sha(idx) == gg["indices_sha256"]
        pool = gb.sample_roots(off, n, gg["root_seed"], gold["pool"])
        assert _sha(pool) == gg["pool_sha256"]
        graphs.append(gb.Graph(off, idx))
        pools.append(pool.cpu().numpy())
    cfg = gb.default_serve_config()
    cfg.workers = 4
    cfg.max_batch = 512
    srv = gb.Server(cfg)
    ids = [srv.add_graph(g) for g in graphs]
    rng = np.random.default_rng(5)
    scratch = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    checked = [(gi, q) for gi, gg in enumerate(gold["graphs"]) for q in gg["queries"]]
    at = {int(p): c for p, c in zip(rng.choice(2000, len(checked), replace=False), checked)}
    tickets, outs = [], []
    for i in range(2000):
        if i in at:
            gi, q = at[i]
            out = torch.full((graphs[gi].n,), 99, dtype=torch.int32, device="cuda")
            outs.append((gi, q, out, srv.submit(ids[gi], q["root"], out)))
        else:
            gi = int(rng.integers(0, len(graphs)))
            r = int(pools[gi][rng.integers(0, len(pools[gi]))])
            tickets.append(srv.submit(ids[gi], r, scratch[gi]))
    assert all(srv.wait(t) == 0 for t in tickets)
    assert all(srv.wait(t) == 0 for _, _, _, t in outs)
    torch.cuda.synchronize()
    for gi, q, out, _ in outs:
        assert _sha(out) == q["levels_sha256"], f"graph {gi}, root {q['root']}"
        assert int((out >= 0).sum().item()) == q["reached"]
    st = srv.stats()
    assert st["failed"] == 0 and st["mean_batch"] > 1
    srv.close()
