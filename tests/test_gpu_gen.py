"""GPU parity for graph input: generator, symmetric CSR build, root sampling.
Integer work, so every comparison is exact."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02259_gb300 as gb
from tests import inputs
from tests.gpu_common import both_csr, gpu_csr_from_edges

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,scale,ef,seed", [
    (gb.GEN_RMAT, 1, 1, 0), (gb.GEN_RMAT, 5, 3, 7), (gb.GEN_RMAT, 12, 16, 1),
    (gb.GEN_RMAT, 16, 16, 1), (gb.GEN_ER, 3, 2, 9), (gb.GEN_ER, 16, 16, 3)])
def test_generator_matches_oracle(kind, scale, ef, seed):
    s, d = gb.generate_edges(kind, scale, ef, seed)
    os_, od = oracle.gen_edges(kind, scale, ef, seed)
    assert np.array_equal(s.cpu().numpy(), os_)
    assert np.array_equal(d.cpu().numpy(), od)


def test_generator_degenerate_initiator():
    s, d = gb.generate_edges(gb.GEN_RMAT, 9, 2, 5, a=0.0, b=1.0, c=0.0)
    os_, od = oracle.gen_edges(oracle.RMAT, 9, 2, 5, a=0.0, b=1.0, c=0.0)
    assert np.array_equal(s.cpu().numpy(), os_) and np.array_equal(d.cpu().numpy(), od)


@pytest.mark.parametrize("seed", range(8))
def test_csr_random_edge_lists(seed):
    rng = np.random.default_rng(seed)
    n = int([1, 2, 31, 32, 33, 1000, 4097, 70000][seed])
    m = int(rng.integers(0, 6 * n + 10))
    s, d = inputs.random_edges(n, m, seed)
    both_csr(n, s, d)


def test_csr_special_cases():
    both_csr(10, np.zeros(0, np.int32), np.zeros(0, np.int32))         # no edges
    both_csr(5, np.array([0, 3, 3], np.int32), np.array([0, 3, 3], np.int32))  # only self-loops
    both_csr(1, np.array([0], np.int32), np.array([0], np.int32))
    both_csr(64, *inputs.star_edges(64, centre=63))
    n, s, d = inputs.union((40, *inputs.path_edges(40)), (3000, [], []), (7, *inputs.complete_edges(7)))
    both_csr(n, s, d)
    # many duplicates of one edge in both orientations
    s = np.array([1, 2] * 5000, np.int32); d = np.array([2, 1] * 5000, np.int32)
    both_csr(3, s, d)


def test_csr_rejects_out_of_range_endpoint():
    with pytest.raises(gb.BfsError) as e:
        gpu_csr_from_edges(4, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    assert e.value.status == 1
    with pytest.raises(gb.BfsError):
        gpu_csr_from_edges(4, np.array([0, -1], np.int32), np.array([1, 2], np.int32))


@pytest.mark.parametrize("kind,scale", [(gb.GEN_RMAT, 16), (gb.GEN_RMAT, 20), (gb.GEN_ER, 20)])
def test_csr_of_generated_graphs(kind, scale):
    # scale 16 and 20 R-MAT and the scale 20 Erdos-Renyi control, edgefactor 16
    seed = 1 if kind == gb.GEN_RMAT else 3
    s, d = gb.generate_edges(kind, scale, 16, seed)
    off, idx = gb.build_csr(1 << scale, s, d)
    os_, od = oracle.gen_edges(kind, scale, 16, seed)
    o_off, o_idx = oracle.build_csr(1 << scale, os_, od)
    assert np.array_equal(off.cpu().numpy(), o_off)
    assert np.array_equal(idx.cpu().numpy(), o_idx)


@pytest.mark.parametrize("k,seed", [(1, 2), (64, 2), (64, 4), (512, 4)])
def test_roots_match_oracle(k, seed):
    s, d = gb.generate_edges(gb.GEN_RMAT, 16, 16, 1)
    off, _ = gb.build_csr(1 << 16, s, d)
    r = gb.sample_roots(off, 1 << 16, seed, k)
    o = oracle.sample_roots(off.cpu().numpy(), 1 << 16, seed, k)
    assert np.array_equal(r.cpu().numpy(), o)


def test_roots_when_few_vertices_qualify():
    n, s, d = inputs.union((3, *inputs.path_edges(3)), (50, [], []))
    off, _ = gpu_csr_from_edges(n, s, d)
    r = gb.sample_roots(off, n, 1, 10, max_draws=100000)
    assert sorted(r.cpu().tolist()) == [0, 1, 2]


def test_scale26_graph_sampled():
    """The full-size workload: sampled generated edges equal the oracle's,
    one by one; the CSR satisfies the structural invariants on sampled rows,
    and every sampled generated edge is present in both directions."""
    scale, ef = 26, 16
    n = 1 << scale
    s, d = gb.generate_edges(gb.GEN_RMAT, scale, ef, 1)
    m = s.numel()
    rng = np.random.default_rng(0)
    picks = np.sort(rng.choice(m, 4096, replace=False))
    for e0 in picks[:64]:
        os_, od = oracle.gen_edges(oracle.RMAT, scale, ef, 1, first=int(e0), count=1)
        assert s[int(e0)].item() == os_[0] and d[int(e0)].item() == od[0]
    ps = torch.as_tensor(picks).cuda()
    es, ed = s[ps].cpu().numpy(), d[ps].cpu().numpy()
    off, idx = gb.build_csr(n, s, d)
    del s, d
    nnz = idx.numel()
    assert off[0].item() == 0 and off[-1].item() == nnz and nnz <= 2 * m
    assert bool((off[1:] >= off[:-1]).all())
    offh_cache = {}

    def row(v):
        if v not in offh_cache:
            a, b = off[v].item(), off[v + 1].item()
            offh_cache[v] = idx[a:b].cpu().numpy()
        return offh_cache[v]

    for a_, b_ in zip(es[:512], ed[:512]):
        if a_ == b_:
            continue
        ra, rb = row(int(a_)), row(int(b_))
        assert np.searchsorted(ra, b_) < ra.size and ra[np.searchsorted(ra, b_)] == b_
        assert np.searchsorted(rb, a_) < rb.size and rb[np.searchsorted(rb, a_)] == a_
    for v in rng.choice(n, 256, replace=False):
        r = row(int(v))
        assert (np.diff(r) > 0).all() and not (r == v).any()
        for u in r[:8]:
            ru = row(int(u))
            k = np.searchsorted(ru, v)
            assert k < ru.size and ru[k] == v
