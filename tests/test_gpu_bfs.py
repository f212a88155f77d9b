"""GPU parity for the single-source hybrid BFS: levels bit-exact against the
oracle, parents by the tree invariants, bottom-up parents and per-layer
counters exact against the oracle's run of Alg. 3 under the same policy."""
from __future__ import annotations

import hashlib
import json
from pathlib import Path

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02259_gb300 as gb
from tests import inputs
from tests.gpu_common import both_csr, config, run_gpu

pytestmark = pytest.mark.gpu


def check_run(o_off, o_idx, graph, root, policy=None, forced=None, alpha=None, beta=None):
    """Runs the GPU BFS and compares it with the oracle's Alg. 3 run (under the
    graph's own switch thresholds unless given)."""
    alpha = graph.config.alpha if alpha is None else alpha
    beta = graph.config.beta if beta is None else beta
    lv, pa = run_gpu(graph, root)
    ref, _ = oracle.bfs(o_off, o_idx, root)
    assert np.array_equal(lv, ref), "levels differ from the oracle"
    assert oracle.check_parents(o_off, o_idx, root, lv, pa) == 0
    if policy is None:
        policy = oracle.POLICY_FORCED if forced is not None else oracle.POLICY_EDGE
    # bu_head 2: the bottom-up step tests each vertex's hub before its row
    hint = oracle.hub(o_off, o_idx) if graph.config.bu_head == 2 else None
    h_lv, h_pa, dirs, tr = oracle.hybrid_bfs(o_off, o_idx, root, policy, alpha, beta,
                                             forced=forced, hint=hint)
    st = graph.stats()
    L = st.layers
    assert [x["direction"] for x in L] == dirs.tolist()
    # with component pruning the bottom-up step skips vertices outside the
    # root's component, so only its edges-examined count may be smaller
    pruned = graph.config.prune_components
    for d, x in enumerate(L):
        got = (x["n_f"], x["m_f"], x["n_u"], x["m_u"], x["examined"], x["found"])
        exp = tuple(int(t) for t in tr[d])
        if pruned and x["direction"] == 1:
            assert got[:4] + got[5:] == exp[:4] + exp[5:], f"layer {d}"
            assert got[4] <= exp[4], f"layer {d}"
        else:
            assert got == exp, f"layer {d}"
        if x["direction"] == 1:
            nxt = ref == d + 1
            assert np.array_equal(pa[nxt], h_pa[nxt]), f"bottom-up parents, layer {d}"
    assert st.component_edges == oracle.component_edges(o_off, ref)
    return lv, pa


def make(n, s, d, **cfg):
    o_off, o_idx, g_off, g_idx = both_csr(n, s, d)
    g = gb.Graph(g_off, g_idx, config(**cfg) if cfg else None, validate=True)
    return o_off, o_idx, g


FORCED = {"td": [0], "bu": [1], "alt": [0, 1] * 32, "alt2": [1, 0] * 32,
          "late_bu": [0, 0, 1], "rand": [1, 0, 0, 1, 1, 0, 1, 0, 0, 0, 1, 1, 1, 0, 1, 1]}


@pytest.mark.parametrize("name", ["path", "cycle", "star", "grid", "hypercube", "complete",
                                  "union", "single", "ragged"])
@pytest.mark.parametrize("pat", list(FORCED))
@pytest.mark.parametrize("prune", [0, 1])
@pytest.mark.parametrize("loop", [0, 1, 3, 4])
def test_closed_form_graphs_forced_directions(name, pat, prune, loop):
    if name == "path":
        n, (s, d) = 77, inputs.path_edges(77)
    elif name == "cycle":
        n, (s, d) = 65, inputs.cycle_edges(65)
    elif name == "star":
        n, (s, d) = 100, inputs.star_edges(100, centre=3)
    elif name == "grid":
        n, (s, d) = 15 * 17, inputs.grid_edges(15, 17)
    elif name == "hypercube":
        n, (s, d) = 256, inputs.hypercube_edges(8)
    elif name == "complete":
        n, (s, d) = 40, inputs.complete_edges(40)
    elif name == "union":
        n, s, d = inputs.union((30, *inputs.path_edges(30)), (9, *inputs.cycle_edges(9)),
                               (5, [], []))
    elif name == "single":
        n, s, d = 1, np.zeros(0, np.int32), np.zeros(0, np.int32)
    else:
        n = 1000 + 13
        s, d = inputs.random_edges(n, 3 * n, 5)
    forced = FORCED[pat]
    o_off, o_idx, g = make(n, s, d, forced=forced, prune_components=prune,
                           bu_list_percent=100 if prune else 0, device_loop=loop,
                           bu_head=(prune + 2 * loop) % 3)
    for r in sorted({0, n // 2, n - 1}):
        check_run(o_off, o_idx, g, r, forced=forced)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("policy", [gb.POLICY_EDGE, gb.POLICY_VERTEX])
@pytest.mark.parametrize("claim", [0, 1])
def test_policies_on_skewed_graphs(seed, policy, claim):
    n = [300, 2049, 5000, 10007, 40000, 65536][seed]
    if seed % 2:
        s, d = inputs.powerlaw_edges(n, 8 * n, seed, hubs=5)
    else:
        s, d = oracle.gen_edges(oracle.RMAT, 12 + seed // 2, 8, seed)
        n = 1 << (12 + seed // 2)
    o_off, o_idx, g = make(n, s, d, policy=policy, td_claim=claim, bu_words=[1, 2, 4][seed % 3],
                           bu_head=(seed // 2 + claim) % 3, prune_components=(seed + claim) % 2,
                           bu_list_percent=[0, 10, 100][(seed + claim) % 3],
                           device_loop=[0, 1, 3, 4][(seed + 2 * claim) % 4])
    for r in oracle.sample_roots(o_off, n, seed, 4):
        check_run(o_off, o_idx, g, int(r), policy=policy)


@pytest.mark.parametrize("deg", [1, 7, 8, 9, 31, 32, 33, 63, 64, 65, 127, 128, 129, 1023, 1024, 1025,
                                 4095, 4096, 4097])
@pytest.mark.parametrize("pat", ["td", "bu"])
def test_degree_bin_boundaries(deg, pat):
    # hub 0 with `deg` leaves, each leaf also on a path, plus a second hub
    n = deg + 200
    hs, hd = inputs.star_edges(deg + 1, centre=0)
    ps, pd = inputs.path_edges(n)
    s = np.concatenate([hs, ps, np.full(50, 5, np.int32)]).astype(np.int32)
    d = np.concatenate([hd, pd, np.arange(100, 150, dtype=np.int32)]).astype(np.int32)
    forced = FORCED[pat]
    for cfg in [dict(forced=forced), dict(forced=forced, td_warp_degree=8, td_grid_degree=64),
                dict(forced=forced, bu_probe=1), dict(forced=forced, bu_probe=33),
                dict(forced=forced, bu_words=1, bu_probe=5),
                dict(forced=forced, bu_words=4, bu_probe=7, td_claim=1),
                dict(forced=forced, bu_head=0, prune_components=0),
                dict(forced=forced, bu_list_percent=100, bu_probe=3),
                dict(forced=forced, device_loop=1),
                dict(forced=forced, device_loop=1, bu_list_percent=100, td_grid_degree=64),
                dict(forced=forced, bu_head=1, bu_probe=2),
                dict(forced=forced, bu_head=1, bu_probe=4, bu_words=2),
                dict(forced=forced, bu_head=2, bu_probe=2),
                dict(forced=forced, bu_head=2, bu_probe=1, bu_words=4),
                dict(forced=forced, bu_head=2, bu_list_percent=100, bu_probe=1),
                dict(forced=forced, bu_head=2, device_loop=1),
                dict(forced=forced, bu_head=2, device_loop=1, bu_list_percent=100),
                dict(forced=forced, device_loop=3),
                dict(forced=forced, device_loop=3, bu_list_percent=100, td_grid_degree=64),
                dict(forced=forced, bu_head=2, device_loop=3, bu_probe=2),
                dict(forced=forced, bu_head=1, bu_words=4, device_loop=3),
                dict(forced=forced, bu_head=0, bu_words=1, device_loop=3, td_claim=0)]:
        o_off, o_idx, g = make(n, s, d, **cfg)
        for r in [0, 1, n - 1, deg // 2]:
            check_run(o_off, o_idx, g, r, forced=forced)


def test_vertex_adjacent_to_all():
    n = 5000
    s, d = inputs.star_edges(n, centre=4321)
    s2, d2 = inputs.random_edges(n, n, 3)
    s = np.concatenate([s, s2]); d = np.concatenate([d, d2])
    for pat in ["td", "bu", "alt"]:
        o_off, o_idx, g = make(n, s, d, forced=FORCED[pat], td_grid_degree=256)
        for r in [4321, 0, 17]:
            check_run(o_off, o_idx, g, r, forced=FORCED[pat])


def _rmat_both(scale, ef, seed, kind=oracle.RMAT):
    n = 1 << scale
    s, d = gb.generate_edges(kind, scale, ef, seed)
    g_off, g_idx = gb.build_csr(n, s, d)
    os_, od = oracle.gen_edges(kind, scale, ef, seed)
    o_off, o_idx = oracle.build_csr(n, os_, od)
    assert np.array_equal(g_off.cpu().numpy(), o_off)
    assert np.array_equal(g_idx.cpu().numpy(), o_idx)
    return n, o_off, o_idx, g_off, g_idx


def test_rmat_scale16_all_64_roots():
    # R-MAT scale 16, edgefactor 16, graph seed 1, 64 roots from seed 2
    n, o_off, o_idx, g_off, g_idx = _rmat_both(16, 16, 1)
    g = gb.Graph(g_off, g_idx)
    roots = gb.sample_roots(g_off, n, 2, 64).cpu().numpy()
    assert np.array_equal(roots, oracle.sample_roots(o_off, n, 2, 64))
    for r in roots:
        check_run(o_off, o_idx, g, int(r))
    g.set_config(config(device_loop=0))    # the same 64 roots with the host-driven loop
    for r in roots:
        check_run(o_off, o_idx, g, int(r))
    for head in (1, 2):                     # and with each kind of head record
        g.set_config(config(device_loop=0, bu_head=head))
        for r in roots[:16]:
            check_run(o_off, o_idx, g, int(r))
    g.set_config(config(device_loop=3))     # the graph loop, rebuilt per configuration
    for r in roots:
        check_run(o_off, o_idx, g, int(r))
    for head in (0, 1):
        g.set_config(config(device_loop=3, bu_head=head))
        for r in roots[:16]:
            check_run(o_off, o_idx, g, int(r))


@pytest.mark.parametrize("pat", ["td", "late_bu", "alt"])
@pytest.mark.parametrize("loop", [0, 1, 3])
def test_large_top_down_layers(pat, loop):
    # forced top-down layers with more than 2^18 frontier edges leave only the
    # next bitmap, and with many vertices still findable they defer level
    # stores and counts to a pass over that bitmap: counters stay exact
    n, o_off, o_idx, g_off, g_idx = _rmat_both(17, 16, 4)
    g = gb.Graph(g_off, g_idx, config(forced=FORCED[pat], device_loop=loop))
    for r in oracle.sample_roots(o_off, n, 5, 3):
        check_run(o_off, o_idx, g, int(r), forced=FORCED[pat])
    if pat == "td":
        assert max(x["m_f"] for x in g.stats().layers) > (1 << 18)


@pytest.mark.parametrize("cfg", [dict(), dict(forced=[0, 0, 1]), dict(forced=[1]),
                                 dict(bu_list_percent=100), dict(forced=[0]), dict(level_pass=0),
                                 dict(level_pass=0, forced=[1])])
@pytest.mark.parametrize("loop", [0, 3, 4])
def test_outputs_written_by_first_sweep(cfg, loop):
    # scale 21 with the host loop: dense bottom-up layers run in two passes
    # and (td_claim = 1) the first hub sweep writes the -1 of every vertex not
    # reached before it; traversals without such a sweep (top-down only,
    # list layers first, a degree-0 root, a small component) fill at the end
    n, o_off, o_idx, g_off, g_idx = _rmat_both(21, 16, 7)
    full = dict(device_loop=loop, td_claim=1, **cfg)
    g = gb.Graph(g_off, g_idx, config(**full))
    deg = np.diff(o_off)
    ref_big = oracle.bfs(o_off, o_idx, int(np.argmax(deg)))[0]
    small = [v for v in range(n) if deg[v] > 0 and ref_big[v] < 0][:1]
    roots = [int(r) for r in oracle.sample_roots(o_off, n, 9, 3)] + small
    roots.append(int(np.nonzero(deg == 0)[0][0]))
    lv = torch.full((n,), 77, dtype=torch.int32, device="cuda")
    pa = torch.full((n,), 77, dtype=torch.int32, device="cuda")
    for r in roots:
        lv.fill_(77)
        pa.fill_(77)       # stale values that must all be overwritten
        g.run(r, lv, pa)
        torch.cuda.synchronize()
        got, par = lv.cpu().numpy(), pa.cpu().numpy()
        ref, _ = oracle.bfs(o_off, o_idx, r)
        assert np.array_equal(got, ref)
        assert oracle.check_parents(o_off, o_idx, r, got, par) == 0
        assert (par[ref < 0] == -1).all()
    check_run(o_off, o_idx, g, roots[0], forced=cfg.get("forced"))


_R21 = {}


def _rmat21_seed11():
    if not _R21:
        _R21["g"] = _rmat_both(21, 16, 11)
    return _R21["g"]


@pytest.mark.parametrize("stages", [0, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("percent", [0, 50])
def test_streaming_hub_sweep(stages, percent):
    # scale 21 (two-pass bottom-up layers): the hub sweep that streams whole
    # tiles of head records through shared memory (every sweep at percent 0,
    # only the dense ones at 50) gives the same levels, bottom-up parents,
    # counters and -1 outputs as the oracle's hub-first Alg. 3 run
    n, o_off, o_idx, g_off, g_idx = _rmat21_seed11()
    g = gb.Graph(g_off, g_idx, config(device_loop=0, hub_stream_stages=stages,
                                      hub_stream_percent=percent))
    deg = np.diff(o_off)
    roots = [int(r) for r in oracle.sample_roots(o_off, n, 5, 3)]
    roots.append(int(np.nonzero(deg == 0)[0][0]))
    lv = torch.full((n,), 77, dtype=torch.int32, device="cuda")
    pa = torch.full((n,), 77, dtype=torch.int32, device="cuda")
    for r in roots:
        lv.fill_(77)
        pa.fill_(77)       # stale values that must all be overwritten
        g.run(r, lv, pa)
        torch.cuda.synchronize()
        got, par = lv.cpu().numpy(), pa.cpu().numpy()
        ref, _ = oracle.bfs(o_off, o_idx, r)
        assert np.array_equal(got, ref)
        assert oracle.check_parents(o_off, o_idx, r, got, par) == 0
        assert (par[ref < 0] == -1).all()
    for r in roots[:2]:
        check_run(o_off, o_idx, g, r)
        assert any(x["converted"] == 3 for x in g.stats().layers)


@pytest.mark.parametrize("cfg", [dict(), dict(device_loop=1), dict(device_loop=3),
                                 dict(parent_min=1), dict(prune_components=1),
                                 dict(host_async=1), dict(timing=1), dict(bu_head=1)])
def test_reserved_runs_allocate_nothing(cfg):
    # after bfs_graph_reserve, traversals under that configuration make no
    # device or pinned allocation in the library (scale 21: two-pass layers)
    n, o_off, o_idx, g_off, g_idx = _rmat21_seed11()
    g = gb.Graph(g_off, g_idx, config(**cfg))
    host = cfg.get("host_async", 0) == 1
    g.reserve(host_out=host, no_parent=True)
    roots = [int(r) for r in oracle.sample_roots(o_off, n, 7, 3)]
    if host:
        bufs = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
    else:
        bufs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(2)]
    before = gb.alloc_count()
    for r in roots:
        g.run(r, bufs[0], bufs[1])
        g.run(r, bufs[0], None, want_parent=False)
    g.sync()
    torch.cuda.synchronize()
    assert gb.alloc_count() == before, "bfs_run allocated after bfs_graph_reserve"
    ref, _ = oracle.bfs(o_off, o_idx, roots[-1])
    assert np.array_equal(bufs[0].cpu().numpy(), ref)


def test_first_run_allocates_then_warm_runs_do_not():
    # without a reserve call the first traversal of a configuration may
    # allocate (host-output scratch here); the warmed-up ones do not
    n, o_off, o_idx, g_off, g_idx = _rmat21_seed11()
    g = gb.Graph(g_off, g_idx)
    lv = torch.empty(n, dtype=torch.int32)
    pa = torch.empty(n, dtype=torch.int32)
    a0 = gb.alloc_count()
    g.run(0, lv, pa)
    a1 = gb.alloc_count()
    assert a1 > a0
    for r in (1, 2, 3):
        g.run(r, lv, pa)
    assert gb.alloc_count() == a1


@pytest.mark.parametrize("kind,seed", [(oracle.RMAT, 1), (oracle.ER, 3)])
def test_scale20_all_64_roots(kind, seed):
    # R-MAT scale 20 (the paper's one-million-vertex size) and its ER control
    n, o_off, o_idx, g_off, g_idx = _rmat_both(20, 16, seed, kind)
    g = gb.Graph(g_off, g_idx)
    roots = gb.sample_roots(g_off, n, 2, 64).cpu().numpy()
    for i, r in enumerate(roots):
        lv, pa = run_gpu(g, int(r))
        ref, _ = oracle.bfs(o_off, o_idx, int(r))
        assert np.array_equal(lv, ref)
        assert oracle.check_parents(o_off, o_idx, int(r), lv, pa) == 0
        if i < 4:
            check_run(o_off, o_idx, g, int(r))


def test_host_output_buffers_match_device():
    n, o_off, o_idx, g_off, g_idx = _rmat_both(14, 16, 1)
    g = gb.Graph(g_off, g_idx)
    r = int(oracle.sample_roots(o_off, n, 2, 1)[0])
    lv_d, _ = run_gpu(g, r)
    lv_h = torch.empty(n, dtype=torch.int32).pin_memory()
    pa_h = torch.empty(n, dtype=torch.int32)
    g.run(r, lv_h, pa_h)
    assert np.array_equal(lv_h.numpy(), lv_d)
    assert oracle.check_parents(o_off, o_idx, r, lv_h.numpy(), pa_h.numpy()) == 0


@pytest.mark.parametrize("loop", [0, 1, 3])
def test_host_async_outputs(loop):
    # host_async: each run returns once its traversal is done; the copies of
    # two runs may still be in flight and all land by sync()
    n, o_off, o_idx, g_off, g_idx = _rmat_both(14, 16, 1)
    g = gb.Graph(g_off, g_idx, config(host_async=1, device_loop=loop))
    roots = [int(r) for r in oracle.sample_roots(o_off, n, 3, 7)]
    bufs = [(torch.full((n,), 55, dtype=torch.int32).pin_memory(),
             torch.full((n,), 55, dtype=torch.int32).pin_memory()) for _ in roots]
    for r, (lv, pa) in zip(roots, bufs):
        g.run(r, lv, pa)
    g.sync()
    for r, (lv, pa) in zip(roots, bufs):
        ref, _ = oracle.bfs(o_off, o_idx, r)
        assert np.array_equal(lv.numpy(), ref)
        assert oracle.check_parents(o_off, o_idx, r, lv.numpy(), pa.numpy()) == 0
    g.sync()                                # nothing pending: returns at once


def test_run_rejects_bad_root():
    o_off, o_idx, g = make(10, *inputs.path_edges(10))
    with pytest.raises(gb.BfsError):
        g.run(10)
    with pytest.raises(gb.BfsError):
        g.run(-1)


def test_validate_rejects_bad_csr():
    off = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    idx = torch.tensor([1, 5], dtype=torch.int32, device="cuda")
    with pytest.raises(gb.BfsError):
        gb.Graph(off, idx, validate=True)
    off = torch.tensor([0, 2, 1], dtype=torch.int64, device="cuda")
    with pytest.raises(gb.BfsError):
        gb.Graph(off, idx, validate=True)
    with pytest.raises(gb.BfsError):           # range checks come first
        gb.Graph(off, idx, validate="symmetric")


def _dev(off, idx):
    return (torch.tensor(off, dtype=torch.int64, device="cuda"),
            torch.tensor(idx, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("case,ok", [
    (([0, 1, 2], [1, 0]), True),                  # one undirected edge
    (([0, 1, 1], [1]), False),                    # 0 -> 1 without 1 -> 0
    (([0, 2, 3, 4], [2, 1, 0, 0]), False),        # symmetric, row 0 descending
    (([0, 2, 4], [1, 1, 0, 0]), False),           # duplicate entries
    (([0, 1, 1], [0]), True),                     # a self-loop is its own reverse
    (([0, 0, 0], []), True),                      # no edges
])
def test_validate_symmetric(case, ok):
    off, idx = _dev(*case)
    gb.Graph(off, idx, validate=True)             # all pass the range checks
    if ok:
        gb.Graph(off, idx, validate="symmetric")
    else:
        with pytest.raises(gb.BfsError):
            gb.Graph(off, idx, validate="symmetric")


def test_validate_symmetric_generated_graphs():
    # the library's own CSR builder output is symmetric with ascending rows;
    # dropping one direction of one edge, or reversing a row, is caught
    n, o_off, o_idx, g_off, g_idx = _rmat_both(16, 16, 1)
    gb.Graph(g_off, g_idx, validate="symmetric")
    rev = torch.as_tensor(_reversed_rows(o_off, o_idx)).cuda()
    with pytest.raises(gb.BfsError):
        gb.Graph(g_off, rev, validate="symmetric")
    # move the first entry u0 of some row v up to u0 + 1 (< the next entry, so
    # the row stays ascending): v -> u0 + 1 has no reverse entry
    for v in range(n):
        lo, hi = o_off[v], o_off[v + 1]
        if hi - lo >= 2 and o_idx[lo + 1] - o_idx[lo] >= 2 and o_idx[lo] + 1 != v:
            break
    cut = o_idx.copy()
    cut[lo] += 1
    w = int(cut[lo])
    assert v not in o_idx[o_off[w]:o_off[w + 1]]
    with pytest.raises(gb.BfsError):
        gb.Graph(g_off, torch.as_tensor(cut).cuda(), validate="symmetric")


GOLDEN26 = Path(__file__).parent / "golden" / "rmat26_ef16_seed1_bfs.json"


def _sha(t: torch.Tensor) -> str:
    a = t.cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(a, dtype=a.dtype.newbyteorder("<")).data).hexdigest()


@pytest.fixture(scope="module")
def rmat26():
    """The full-size single-source workload as the benchmark runs it: R-MAT
    SCALE 26, edgefactor 16, graph seed 1, 64 roots of seed 2, default
    configuration (host-driven loop at this size)."""
    gold = json.loads(GOLDEN26.read_text())
    n = 1 << gold["scale"]
    off, idx = gb.rmat_graph(gold["scale"], gold["edgefactor"], gold["graph_seed"])
    g = gb.Graph(off, idx)
    roots = gb.sample_roots(off, n, gold["root_seed"], 64).tolist()
    src = torch.repeat_interleave(torch.arange(n, dtype=torch.int32, device="cuda"),
                                  off[1:] - off[:-1])       # row of every CSR entry
    yield gold, off, idx, g, roots, src
    del g, src


def _full_check(off, idx, src, root, level, parent, minimal):
    """The BFS characterisation over every edge (any size): level[root] = 0;
    no edge joins a reached and an unreached vertex or two levels more than
    one apart; every reached v != root has a neighbour one level up. The
    parent of such v is a neighbour one level up (exactly one row entry
    equals it: rows are deduplicated), and with `minimal` the smallest one.
    Unreached vertices hold -1 in both arrays. Returns the component edges."""
    n = level.numel()
    lu = level[src]
    lv = torch.index_select(level, 0, idx)
    assert bool(((lu >= 0) == (lv >= 0)).all()), "an edge leaves the reached set"
    assert int((lu - lv).abs().max().item()) <= 1, "an edge spans two layers"
    up = (lv == lu - 1) & (lu > 0)
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda").index_add_(0, src, up.int())
    reached = level >= 0
    inner = reached.clone()
    inner[root] = False
    assert level[root].item() == 0 and parent[root].item() == root
    assert bool((cnt[inner] > 0).all()), "a reached vertex without a neighbour one level up"
    assert bool((level[~reached] == -1).all()) and bool((parent[~reached] == -1).all())
    is_par = (idx == parent[src]) & up
    pc = torch.zeros(n, dtype=torch.int32, device="cuda").index_add_(0, src, is_par.int())
    assert bool((pc[inner] == 1).all()), "a parent that is not a neighbour one level up"
    if minimal:
        big = torch.iinfo(torch.int32).max
        cand = torch.where(up, idx, torch.full_like(idx, big))
        best = torch.full((n,), big, dtype=torch.int32, device="cuda")
        best.scatter_reduce_(0, src.long(), cand, "amin")
        assert torch.equal(parent[inner], best[inner]), "parent is not the smallest one"
    deg = off[1:] - off[:-1]
    return int(deg[reached].sum().item()) // 2


def test_scale26_csr_and_roots_match_oracle_digests(rmat26):
    # the whole generated CSR and the 64 roots, against digests that the
    # oracle wrote for the same seeds (tests/golden/make_rmat26_bfs.py)
    gold, off, idx, g, roots, src = rmat26
    assert idx.numel() == gold["nnz"]
    assert _sha(off) == gold["offsets_sha256"]
    assert _sha(idx) == gold["indices_sha256"]
    assert roots == gold["roots"]


def test_scale26_levels_and_min_parents_exact(rmat26):
    # 8 roots: levels bit-exact against the oracle's FIFO BFS (digest), and
    # with parent_min the whole parent array against the oracle's post-pass
    gold, off, idx, g, roots, src = rmat26
    n = off.numel() - 1
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    gm = gb.Graph(off, idx, config(parent_min=1), borrow=True)
    g3 = gb.Graph(off, idx, config(device_loop=3), borrow=True)
    for e in gold["exact"]:
        r = e["root"]
        g3.run(r, level, parent)                # the graph loop
        torch.cuda.synchronize()
        assert _sha(level) == e["levels_sha256"], f"graph loop levels of root {r}"
        layers3 = g3.stats().layers
        g.run(r, level, parent)
        torch.cuda.synchronize()
        assert _sha(level) == e["levels_sha256"], f"levels of root {r}"
        keys = ("direction", "converted", "n_f", "m_f", "n_u", "m_u", "examined", "found",
                "hub_found")
        assert [{k: x[k] for k in keys} for x in layers3] == \
            [{k: x[k] for k in keys} for x in g.stats().layers]
        ce = _full_check(off, idx, src, r, level, parent, minimal=False)
        assert ce == e["component_edges"] == g.stats().component_edges
        sizes = torch.bincount(level[level >= 0].long()).tolist()
        assert sizes == e["layer_sizes"]
        parent.fill_(7)
        gm.run(r, level, parent)
        torch.cuda.synchronize()
        assert _sha(level) == e["levels_sha256"]
        assert _sha(parent) == e["min_parent_sha256"], f"min parents of root {r}"


def test_scale26_all_64_roots_full_check(rmat26):
    # every root of the benchmark: the characterisation over all 2^31 CSR
    # entries, parents included; then with parent_min, minimality too
    gold, off, idx, g, roots, src = rmat26
    n = off.numel() - 1
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots:
        g.run(r, level, parent)
        torch.cuda.synchronize()
        ce = _full_check(off, idx, src, r, level, parent, minimal=False)
        assert ce == g.stats().component_edges
    gm = gb.Graph(off, idx, config(parent_min=1), borrow=True)
    for r in roots[::4]:
        gm.run(r, level, parent)
        torch.cuda.synchronize()
        _full_check(off, idx, src, r, level, parent, minimal=True)


def _reversed_rows(o_off, o_idx):
    """The same graph with every CSR row in descending order."""
    idx = o_idx.copy()
    for v in range(len(o_off) - 1):
        idx[o_off[v]:o_off[v + 1]] = idx[o_off[v]:o_off[v + 1]][::-1]
    return idx


@pytest.mark.parametrize("loop", [0, 1, 3])
@pytest.mark.parametrize("rows", ["sorted", "reversed"])
def test_parent_min_matches_oracle(loop, rows):
    # parent_min: every reached vertex's parent is its smallest neighbour one
    # level up, whatever the direction of the layer that found it (Sec. 7.1
    # allows any such tree; this one is unique), so parents compare exactly
    n, o_off, o_idx, g_off, g_idx = _rmat_both(16, 16, 1)
    if rows == "reversed":
        o_idx = _reversed_rows(o_off, o_idx)
        g_idx = torch.as_tensor(o_idx).cuda()
    cases = [dict(), dict(forced=FORCED["alt"]), dict(forced=FORCED["td"]),
             dict(bu_head=0, td_claim=0), dict(prune_components=1)]
    roots = [int(r) for r in oracle.sample_roots(o_off, n, 2, 6)]
    for c in cases:
        g = gb.Graph(g_off, g_idx, config(parent_min=1, device_loop=loop, **c))
        for r in roots:
            lv, pa = run_gpu(g, r)
            ref, _ = oracle.bfs(o_off, o_idx, r)
            assert np.array_equal(lv, ref)
            assert np.array_equal(pa, oracle.min_parent(o_off, o_idx, r, ref)), (c, r)


@pytest.mark.parametrize("name", ["star", "grid", "hypercube", "complete", "union", "ragged"])
def test_parent_min_closed_forms(name):
    if name == "star":
        n, (s, d) = 100, inputs.star_edges(100, centre=3)
    elif name == "grid":
        n, (s, d) = 15 * 17, inputs.grid_edges(15, 17)
    elif name == "hypercube":
        n, (s, d) = 256, inputs.hypercube_edges(8)
    elif name == "complete":
        n, (s, d) = 40, inputs.complete_edges(40)
    elif name == "union":
        n, s, d = inputs.union((30, *inputs.path_edges(30)), (9, *inputs.cycle_edges(9)),
                               (5, [], []))
    else:
        n = 1000 + 13
        s, d = inputs.powerlaw_edges(n, 6 * n, 5)
    o_off, o_idx, g = make(n, s, d, parent_min=1)
    for r in sorted({0, n // 2, n - 1}):
        lv, pa = run_gpu(g, r)
        ref, _ = oracle.bfs(o_off, o_idx, r)
        assert np.array_equal(lv, ref)
        assert np.array_equal(pa, oracle.min_parent(o_off, o_idx, r, ref))


def test_parent_min_host_outputs():
    n, o_off, o_idx, g_off, g_idx = _rmat_both(14, 16, 1)
    roots = [int(r) for r in oracle.sample_roots(o_off, n, 3, 4)]
    for extra in (dict(), dict(host_async=1)):
        g = gb.Graph(g_off, g_idx, config(parent_min=1, **extra))
        bufs = [(torch.full((n,), 55, dtype=torch.int32).pin_memory(),
                 torch.full((n,), 55, dtype=torch.int32).pin_memory()) for _ in roots]
        for r, (lv, pa) in zip(roots, bufs):
            g.run(r, lv, pa)
        g.sync()
        for r, (lv, pa) in zip(roots, bufs):
            ref, _ = oracle.bfs(o_off, o_idx, r)
            assert np.array_equal(lv.numpy(), ref)
            assert np.array_equal(pa.numpy(), oracle.min_parent(o_off, o_idx, r, ref))


@pytest.mark.parametrize("pat", ["td", "bu", "alt"])
def test_graph_loop_runs_past_its_layer_cap(pat):
    # a path of 600 vertices has up to 599 layers: the graph loop stops every
    # 256 layers and is launched again until the traversal ends
    n = 600
    o_off, o_idx, g = make(n, *inputs.path_edges(n), forced=FORCED[pat], device_loop=3)
    for r in (0, 299, n - 1):
        check_run(o_off, o_idx, g, r, forced=FORCED[pat])
    g.run(0)
    assert len(g.stats().layers) == n


@pytest.mark.parametrize("scale", [20, 21])
def test_graph_loop_layer_records_equal_host_loop(scale):
    # the same decisions and the same per-layer variant (queue rebuilt,
    # list, two-pass) and hub hits as the host-driven loop
    n, o_off, o_idx, g_off, g_idx = _rmat_both(scale, 16, 3)
    # (and so does the hybrid loop, whose top-down stretches run on the device)
    gh = gb.Graph(g_off, g_idx, config(device_loop=0))
    g3 = gb.Graph(g_off, g_idx, config(device_loop=3))
    g4 = gb.Graph(g_off, g_idx, config(device_loop=4))
    keys = ("direction", "converted", "n_f", "m_f", "n_u", "m_u", "examined", "found",
            "hub_found")
    for r in oracle.sample_roots(o_off, n, 11, 6):
        lh, ph = run_gpu(gh, int(r))
        recs_h = [{k: x[k] for k in keys} for x in gh.stats().layers]
        ce_h = gh.stats().component_edges
        for gx in (g3, g4):
            lx, px = run_gpu(gx, int(r))
            assert np.array_equal(lh, lx)
            assert oracle.check_parents(o_off, o_idx, int(r), lx, px) == 0
            assert [{k: x[k] for k in keys} for x in gx.stats().layers] == recs_h
            assert gx.stats().component_edges == ce_h


@pytest.mark.parametrize("level_pass", [0, 1])
@pytest.mark.parametrize("pat", ["td", "bu", "alt"])
def test_level_pass_on_deep_paths(level_pass, pat):
    # paths of 15, 16, 17 and 300 vertices: depths around the 16-slot ring
    # of the level pass (levels written after the traversal, or written so
    # far at the flush before the ring wraps and stored as found after it)
    for n in (15, 16, 17, 18, 300):
        s, d = inputs.path_edges(n)
        o_off, o_idx, g = make(n, s, d, forced=FORCED[pat], level_pass=level_pass,
                               device_loop=0)
        for r in sorted({0, n // 2, n - 1}):
            check_run(o_off, o_idx, g, r, forced=FORCED[pat])


def test_timing_modes():
    # timing 1: events around every layer; 2: only around the hub sweeps
    n, o_off, o_idx, g_off, g_idx = _rmat_both(21, 16, 7)
    r = int(oracle.sample_roots(o_off, n, 9, 1)[0])
    g = gb.Graph(g_off, g_idx, config(device_loop=0, timing=1))
    lv1, _ = run_gpu(g, r)
    L1 = g.stats().layers
    assert all(x["ms_total"] > 0 for x in L1)
    assert any(x["converted"] == 3 for x in L1)
    g.set_config(config(device_loop=0, timing=2))
    lv2, _ = run_gpu(g, r)
    L2 = g.stats().layers
    assert np.array_equal(lv1, lv2)
    for x in L2:
        assert x["ms_total"] == 0 and x["ms_main"] == 0
        assert (x["ms_sweep"] > 0) == (x["converted"] == 3)
    with pytest.raises(gb.BfsError):
        g.set_config(config(timing=3))
