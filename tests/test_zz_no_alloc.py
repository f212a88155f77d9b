"""The allocation-free entry point (bfs_run_noalloc) against bfs_run.

Callers that cannot allocate device memory (a plugin given only a stream, a
process whose device memory belongs to another allocator, a latency-critical
path) use bfs_run_noalloc, whose scratch is a fixed array inside the library.
This file is collected last so that a failure here stops a -x run only after
every other test has run; it also passes when run alone."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02259_gb300 as gb

pytestmark = pytest.mark.gpu


def _graph(scale, seed):
    n = 1 << scale
    s, d = gb.generate_edges(gb.GEN_RMAT, scale, 16, seed)
    off, idx = gb.build_csr(n, s, d)
    os_, od = oracle.gen_edges(oracle.RMAT, scale, 16, seed)
    o_off, o_idx = oracle.build_csr(n, os_, od)
    assert np.array_equal(off.cpu().numpy(), o_off) and np.array_equal(idx.cpu().numpy(), o_idx)
    return n, off, idx, o_off, o_idx


@pytest.mark.parametrize("scale,seed", [(16, 1), (20, 1)])
def test_noalloc_matches_bfs_run_twice_in_a_row(scale, seed):
    n, off, idx, o_off, o_idx = _graph(scale, seed)
    g = gb.Graph(off, idx)
    roots = gb.sample_roots(off, n, 2, 3).cpu().tolist()
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    # two different roots back to back, then the first again: the shared
    # array must not carry state from one call into the next
    for r in [roots[0], roots[1], roots[0]]:
        ref_lv, ref_pa = g.run(r)
        level.fill_(123)
        parent.fill_(456)
        gb.run_noalloc(off, idx, r, level, parent)
        torch.cuda.synchronize()
        lv = level.cpu().numpy()
        assert np.array_equal(lv, ref_lv.cpu().numpy())
        assert oracle.check_parents(o_off, o_idx, r, lv, parent.cpu().numpy()) == 0


def test_noalloc_ragged_size_and_limit():
    n = 1000 + 7
    rng = np.random.default_rng(3)
    s = rng.integers(0, n, 4 * n).astype(np.int32)
    d = rng.integers(0, n, 4 * n).astype(np.int32)
    off, idx = gb.build_csr(n, torch.as_tensor(s).cuda(), torch.as_tensor(d).cuda())
    o_off, o_idx = oracle.build_csr(n, s, d)
    g = gb.Graph(off, idx)
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in [0, n - 1]:
        ref_lv, _ = g.run(r)
        gb.run_noalloc(off, idx, r, level, parent)
        torch.cuda.synchronize()
        assert np.array_equal(level.cpu().numpy(), ref_lv.cpu().numpy())
        assert oracle.check_parents(o_off, o_idx, r, level.cpu().numpy(),
                                    parent.cpu().numpy()) == 0
    # sizes beyond the fixed array are refused before any work
    big_n = (1 << 20) + 1
    st = gb.lib().bfs_run_noalloc(ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(idx.data_ptr()),
                                  big_n, idx.numel(), 0, ctypes.c_void_p(level.data_ptr()),
                                  ctypes.c_void_p(parent.data_ptr()), None)
    assert st == 1 and b"limit" in gb.lib().bfs_last_error()
