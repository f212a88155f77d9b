"""Helpers for the GPU parity tests: each side builds its own CSR from the
same seeded edge list, and the two CSRs are compared before any BFS runs."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_1704_02259_gb300 as gb


def gpu_csr_from_edges(n, s, d):
    src = torch.as_tensor(np.asarray(s, dtype=np.int32)).cuda()
    dst = torch.as_tensor(np.asarray(d, dtype=np.int32)).cuda()
    return gb.build_csr(n, src, dst)


def both_csr(n, s, d):
    """(oracle offsets, oracle indices, gpu offsets, gpu indices), checked equal."""
    o_off, o_idx = oracle.build_csr(n, s, d)
    g_off, g_idx = gpu_csr_from_edges(n, s, d)
    assert np.array_equal(g_off.cpu().numpy(), o_off), "CSR offsets differ from the oracle"
    assert np.array_equal(g_idx.cpu().numpy(), o_idx), "CSR indices differ from the oracle"
    return o_off, o_idx, g_off, g_idx


def config(**kw):
    c = gb.default_config()
    for k, v in kw.items():
        if k == "forced":
            c.policy = gb.POLICY_FORCED
            c.forced_len = len(v)
            for i, x in enumerate(v):
                c.forced[i] = int(x)
        else:
            setattr(c, k, v)
    return c


def run_gpu(graph, root):
    lv, pa = graph.run(int(root))
    torch.cuda.synchronize()
    return lv.cpu().numpy(), pa.cpu().numpy()
