"""The allocation-free entry point (bfs_run_noalloc) against bfs_run and the
oracle.

Callers that cannot allocate device memory (a plugin given only a stream, a
process whose device memory belongs to another allocator's pool, a
latency-critical path that cannot take an allocation's implicit
synchronisation) use bfs_run_noalloc, whose scratch is a fixed array inside
the library. Its levels must equal both the existing entry point's (bfs_run)
and the oracle's FIFO BFS exactly, and its parents must form a valid BFS
tree, on calls made back to back (the array is shared and keeps the last
call's contents). This file is collected last so that a failure here stops a
-x run only after every other test has run; it also passes when run alone."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02259_gb300 as gb
from tests import inputs
from tests.gpu_common import both_csr

pytestmark = pytest.mark.gpu

LIMIT = 1 << 20  # vertices the library's fixed scratch array holds


def _rmat(scale, seed):
    n = 1 << scale
    s, d = oracle.gen_edges(oracle.RMAT, scale, 16, seed)
    o_off, o_idx, off, idx = both_csr(n, s, d)
    return n, o_off, o_idx, off, idx


def _check_against_both(o_off, o_idx, off, idx, roots):
    """Runs bfs_run_noalloc for each root in turn (poisoned outputs first) and
    compares it with bfs_run and with oracle.bfs."""
    n = off.numel() - 1
    g = gb.Graph(off, idx)
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots:
        ref_lv, _ = g.run(int(r))
        level.fill_(123)
        parent.fill_(456)
        torch.cuda.synchronize()
        a0 = gb.alloc_count()
        gb.run_noalloc(off, idx, int(r), level, parent)
        torch.cuda.synchronize()
        assert gb.alloc_count() == a0, "bfs_run_noalloc allocated"
        lv = level.cpu().numpy()
        want, _ = oracle.bfs(o_off, o_idx, int(r))
        assert np.array_equal(lv, want), f"levels differ from the oracle (root {r})"
        assert np.array_equal(lv, ref_lv.cpu().numpy()), f"levels differ from bfs_run (root {r})"
        assert oracle.check_parents(o_off, o_idx, int(r), lv, parent.cpu().numpy()) == 0
    g.close()


@pytest.mark.parametrize("scale,seed", [(16, 1), (20, 1)])
def test_noalloc_matches_bfs_run_and_oracle_twice_in_a_row(scale, seed):
    # scale 20 is n = 2^20 exactly, the largest size the array holds. Two
    # different roots back to back, then the first again: the shared array
    # must not carry state from one call into the next.
    n, o_off, o_idx, off, idx = _rmat(scale, seed)
    roots = gb.sample_roots(off, n, 2, 3).cpu().tolist()
    _check_against_both(o_off, o_idx, off, idx, [roots[0], roots[1], roots[0]])


@pytest.mark.parametrize("name", ["path", "star", "grid", "disconnected", "ragged"])
def test_noalloc_closed_form_graphs(name):
    if name == "path":
        n = 3001
        s, d = inputs.path_edges(n)
        roots = [0, n // 2, n - 1]                  # depth n-1 from either end
    elif name == "star":
        n = 5000
        s, d = inputs.star_edges(n, centre=17)
        roots = [17, 0, n - 1]                      # centre, then two leaves
    elif name == "grid":
        n = 60 * 70
        s, d = inputs.grid_edges(60, 70)
        roots = [0, 35 * 70 + 20]
    elif name == "disconnected":
        n, s, d = inputs.union((400, *inputs.cycle_edges(400)), (1, [], []),
                               (300, *inputs.random_edges(300, 900, 5)))
        roots = [400, 3, 700]                       # isolated root, cycle, random part
    else:
        n = 1000 + 7
        s, d = inputs.random_edges(n, 4 * n, 3)
        roots = [0, n - 1]
    o_off, o_idx, off, idx = both_csr(n, s, d)
    _check_against_both(o_off, o_idx, off, idx, roots)


def test_noalloc_deep_traversal_at_the_size_limit():
    # n = 2^20 exactly: a 20,000-vertex path (20,000 layers) plus isolated
    # vertices, traversed from the path's end.
    n, s, d = inputs.union((20000, *inputs.path_edges(20000)), (LIMIT - 20000, [], []))
    assert n == LIMIT
    o_off, o_idx, off, idx = both_csr(n, s, d)
    _check_against_both(o_off, o_idx, off, idx, [19999, 0])


def test_noalloc_refuses_bad_sizes_before_any_work():
    n = 1000 + 7
    s, d = inputs.random_edges(n, 4 * n, 3)
    _, _, off, idx = both_csr(n, s, d)
    level = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    parent = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    lib = gb.lib()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    # sizes beyond the fixed array
    st = lib.bfs_run_noalloc(p(off), p(idx), LIMIT + 1, idx.numel(), 0, p(level), p(parent), None)
    assert st == 1 and b"limit" in lib.bfs_last_error()
    # nnz that disagrees with offsets[n]
    st = lib.bfs_run_noalloc(p(off), p(idx), n, idx.numel() - 1, 0, p(level), p(parent), None)
    assert st == 1 and b"offsets[n]" in lib.bfs_last_error()
    torch.cuda.synchronize()
    assert (level == 7).all() and (parent == 7).all()   # nothing was written
