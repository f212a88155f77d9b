"""GPU parity for the batched multi-source BFS: every int8 level row equals
the oracle's single-source levels of that root (exact)."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02259_gb300 as gb
from tests import inputs
from tests.gpu_common import both_csr

pytestmark = pytest.mark.gpu

ALL_BU = dict(alpha=1e12, beta=1e-12)    # bottom-up from layer 0 on
ALL_TD = dict(alpha=1e-12, beta=1e12)    # never bottom-up


def rmat(scale, ef=16, seed=1):
    n = 1 << scale
    s, d = oracle.gen_edges(oracle.RMAT, scale, ef, seed)
    o_off, o_idx, g_off, g_idx = both_csr(n, s, d)
    return n, o_off, o_idx, gb.Graph(g_off, g_idx)


def set_cfg(g, **kw):
    c = gb.default_batch_config()
    for k, v in kw.items():
        setattr(c, k, v)
    g.set_batch_config(c)


def check(g, o_off, o_idx, roots):
    lv = g.run_batch(roots)
    torch.cuda.synchronize()
    exp = oracle.msbfs_levels(o_off, o_idx, [int(r) for r in roots])
    assert np.array_equal(lv.cpu().numpy(), exp)


@pytest.mark.parametrize("k", [1, 2, 63, 64, 65, 127, 128, 129, 256, 300, 512])
@pytest.mark.parametrize("mode", ["auto", "bu", "td"])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_rmat14_matches_oracle(k, mode, use_graph):
    n, o_off, o_idx, g = rmat(14)
    set_cfg(g, use_graph=use_graph, **({"bu": ALL_BU, "td": ALL_TD}.get(mode, {})))
    roots = np.random.default_rng(k).integers(0, n, size=k).astype(np.int32)
    check(g, o_off, o_idx, roots)


@pytest.mark.parametrize("probe", [0, 1, 3, 64])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_lane_probe_and_hubs(probe, use_graph):
    n = 3000
    s, d = inputs.powerlaw_edges(n, 12 * n, 7, hubs=4)
    o_off, o_idx, g_off, g_idx = both_csr(n, s, d)
    g = gb.Graph(g_off, g_idx)
    for mode in [{}, ALL_BU, ALL_TD]:
        set_cfg(g, lane_probe=probe, big_degree=64, use_graph=use_graph, **mode)
        roots = np.random.default_rng(probe).integers(0, n, size=200).astype(np.int32)
        check(g, o_off, o_idx, roots)


def test_device_loop_replays_and_recaptures():
    n, o_off, o_idx, g = rmat(13)
    set_cfg(g, use_graph=1)
    out = torch.empty((70, n), dtype=torch.int8, device="cuda")
    for seed in range(3):   # same arguments: the captured graph is replayed
        roots = np.random.default_rng(seed).integers(0, n, size=70).astype(np.int32)
        g.run_batch(roots, out)
        assert np.array_equal(out.cpu().numpy(), oracle.msbfs_levels(o_off, o_idx, roots.tolist()))
        layers, pairs = g.batch_stats()
        assert layers and pairs >= 70
    roots = [5, 6, 7]       # new k and output buffer: captured again
    check(g, o_off, o_idx, roots)


def test_grid_barrier_wait_runs_out_and_context_survives():
    assert gb.selftest_grid_barrier(0, 200000) == 0
    t0 = time.time()
    assert gb.selftest_grid_barrier(1, 200000) == 4          # BFS_ERR_TIMEOUT
    assert time.time() - t0 < 30
    assert gb.selftest_grid_barrier(0, 200000) == 0
    n, o_off, o_idx, g = rmat(12)                            # the context still works
    check(g, o_off, o_idx, [0, 1, 2])


def test_batch_duplicate_roots_and_small_graphs():
    n, s, d = inputs.union((40, *inputs.path_edges(40)), (17, *inputs.cycle_edges(17)),
                           (9, [], []), (33, *inputs.complete_edges(33)))
    o_off, o_idx, g_off, g_idx = both_csr(n, s, d)
    g = gb.Graph(g_off, g_idx)
    roots = np.array([0, 0, 5, 41, 41, 60, 39, 70, 0] * 9, dtype=np.int32)
    for mode in [{}, ALL_BU, ALL_TD]:
        set_cfg(g, **mode)
        check(g, o_off, o_idx, roots)
        check(g, o_off, o_idx, roots[:1])


def test_batch_k1_equals_single_source():
    n, o_off, o_idx, g = rmat(15)
    r = int(oracle.sample_roots(o_off, n, 2, 1)[0])
    lv = g.run_batch([r])
    single, _ = g.run(r)
    assert np.array_equal(lv[0].cpu().numpy().astype(np.int32), single.cpu().numpy())


def test_batch_device_roots_and_errors():
    n, o_off, o_idx, g = rmat(12)
    roots = torch.tensor([1, 2, 3, 4000], dtype=torch.int32, device="cuda")
    lv = g.run_batch(roots)
    exp = oracle.msbfs_levels(o_off, o_idx, [1, 2, 3, 4000])
    assert np.array_equal(lv.cpu().numpy(), exp)
    with pytest.raises(gb.BfsError):
        g.run_batch([0] * 513)
    with pytest.raises(gb.BfsError):
        g.run_batch([n])
    with pytest.raises(gb.BfsError):
        g.run_batch(torch.zeros(0, dtype=torch.int32))


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_depth_over_127_is_an_error(use_graph):
    n = 300
    o_off, o_idx, g_off, g_idx = both_csr(n, *inputs.path_edges(n))
    g = gb.Graph(g_off, g_idx)
    set_cfg(g, use_graph=use_graph)
    lv = torch.empty((2, n), dtype=torch.int8, device="cuda")
    with pytest.raises(gb.BfsError) as e:
        g.run_batch([0, 5], lv)
    assert e.value.status == 5
    got = lv.cpu().numpy().astype(np.int32)
    ref = oracle.bfs(o_off, o_idx, 0)[0]
    # every level up to 127 is written; nothing wrapped to a negative value
    assert np.array_equal(got[0][ref <= 127], ref[ref <= 127])
    assert (got[0][ref > 127] == -1).all()


def test_batch_autotune_keeps_results_exact():
    n, o_off, o_idx, g = rmat(14)
    roots = oracle.sample_roots(o_off, n, 3, 64)
    best = g.autotune_batch(roots)
    assert best.alpha > 0 and best.beta > 0
    cfg = g.batch_config()
    assert cfg.alpha == best.alpha and cfg.lane_probe == best.lane_probe
    check(g, o_off, o_idx, roots)


def test_batch_scale22_sampled_lanes():
    """The batched workload: R-MAT scale 22, 512 roots in one launch; 6
    sampled lanes compared with the oracle's BFS of those roots."""
    scale, k = 22, 512
    n = 1 << scale
    off, idx = gb.rmat_graph(scale, 16, 1)
    s, d = oracle.gen_edges(oracle.RMAT, scale, 16, 1)
    o_off, o_idx = oracle.build_csr(n, s, d)
    del s, d
    g = gb.Graph(off, idx)
    roots = gb.sample_roots(off, n, 4, k)
    lv = g.run_batch(roots)
    torch.cuda.synchronize()
    rs = roots.cpu().numpy()
    for i in [0, 1, 63, 64, 300, 511]:
        ref, _ = oracle.bfs(o_off, o_idx, int(rs[i]))
        assert np.array_equal(lv[i].cpu().numpy().astype(np.int32), ref)
