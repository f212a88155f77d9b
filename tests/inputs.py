"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This module holds no step of the method: it only draws random numbers and
writes down edge lists of textbook graphs. Each side then builds its own CSR
from the same edge list (the oracle with ``oracle.build_csr``, the library with
its GPU CSR builder), so nothing computed by one side feeds the other.
"""
from __future__ import annotations

import numpy as np


def path_edges(n):
    v = np.arange(n - 1, dtype=np.int32)
    return v, v + 1


def cycle_edges(n):
    v = np.arange(n, dtype=np.int32)
    return v, ((v + 1) % n).astype(np.int32)


def star_edges(n, centre=0):
    leaves = np.array([v for v in range(n) if v != centre], dtype=np.int32)
    return np.full(leaves.size, centre, dtype=np.int32), leaves


def complete_edges(n):
    s, d = np.triu_indices(n, k=1)
    return s.astype(np.int32), d.astype(np.int32)


def grid_edges(rows, cols):
    src, dst = [], []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                src.append(v); dst.append(v + 1)
            if r + 1 < rows:
                src.append(v); dst.append(v + cols)
    return np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32)


def hypercube_edges(dim):
    src, dst = [], []
    for v in range(1 << dim):
        for b in range(dim):
            u = v ^ (1 << b)
            if v < u:
                src.append(v); dst.append(u)
    return np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32)


def random_edges(n, m, seed, self_loops=True, duplicates=True):
    """m uniform random endpoint pairs (with repeats and self-loops unless disabled)."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    d = rng.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    if not self_loops:
        keep = s != d
        s, d = s[keep], d[keep]
    if duplicates and m >= 4:
        k = max(1, m // 10)
        s = np.concatenate([s, d[:k]]).astype(np.int32)
        d = np.concatenate([d, s[:k]]).astype(np.int32)
    return s, d


def powerlaw_edges(n, m, seed, hubs=3):
    """Skewed random graph: a few hubs adjacent to many vertices plus noise."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, size=m, dtype=np.int64)
    d = rng.integers(0, n, size=m, dtype=np.int64)
    h = rng.integers(0, n, size=hubs, dtype=np.int64)
    half = m // 2
    s[:half] = h[rng.integers(0, hubs, size=half)]
    return s.astype(np.int32), d.astype(np.int32)


def union(*parts):
    """Disjoint union of (n_i, src_i, dst_i) graphs, relabelled consecutively."""
    src, dst, base = [], [], 0
    for n, s, d in parts:
        src.append(np.asarray(s, dtype=np.int64) + base)
        dst.append(np.asarray(d, dtype=np.int64) + base)
        base += n
    return base, np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32)


def roots(n, k, seed):
    return np.random.default_rng(seed).integers(0, n, size=k).astype(np.int32)
