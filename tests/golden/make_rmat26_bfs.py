"""Writes rmat26_ef16_seed1_bfs.json: digests of the oracle's results on the
full-size single-source workload, so that GPU runs at that size compare
bit-exactly without the oracle's minutes of CPU time in the test.

Workload: R-MAT graph (Sec. 6.2: initiator A, B, C, D = 0.57, 0.19, 0.19,
0.05, edgefactor 16, SCALE 26, graph seed 1), symmetric CSR with self-loops
dropped and rows sorted and deduplicated (Sec. 6.2-6.3), the 64 roots of
seed 2 (Sec. 6.3). For the first 8 roots: levels (Sec. 4 layer definition,
the oracle's FIFO BFS) and the smallest-id-parent tree (one of the valid
trees of Sec. 7.1). Every value comes from `oracle/` only; the edge list is
generated in chunks on host threads (the C generator is a pure function of
the edge number). Digests are SHA-256 of the arrays' little-endian bytes.

    python tests/golden/make_rmat26_bfs.py      # ~60 GB of host memory, ~20 min
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))
import oracle  # noqa: E402

SCALE, EF, GRAPH_SEED, ROOT_SEED, N_ROOTS, N_EXACT = 26, 16, 1, 2, 64, 8
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat26_ef16_seed1_bfs.json")


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=a.dtype.newbyteorder("<")).data).hexdigest()


def main() -> None:
    n = 1 << SCALE
    m = EF << SCALE
    t0 = time.time()
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    chunks = 64
    step = (m + chunks - 1) // chunks

    def gen(i):
        a, b = i * step, min(m, (i + 1) * step)
        oracle.gen_edges(oracle.RMAT, SCALE, EF, GRAPH_SEED, first=a, count=b - a,
                         out=(src[a:b], dst[a:b]))

    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        list(ex.map(gen, range(chunks)))
    print(f"edges {time.time() - t0:.0f} s", flush=True)
    off, idx = oracle.build_csr(n, src, dst)
    del src, dst
    print(f"csr {time.time() - t0:.0f} s, nnz {idx.size}", flush=True)
    roots = oracle.sample_roots(off, n, ROOT_SEED, N_ROOTS)
    rec = {
        "what": "oracle results on R-MAT SCALE 26, edgefactor 16, graph seed 1 "
                "(Sec. 6.2-6.3), roots of seed 2; SHA-256 of little-endian arrays",
        "scale": SCALE, "edgefactor": EF, "graph_seed": GRAPH_SEED, "root_seed": ROOT_SEED,
        "n": n, "nnz": int(idx.size),
        "offsets_sha256": sha(off), "indices_sha256": sha(idx),
        "roots": [int(r) for r in roots], "exact": [],
    }
    for r in roots[:N_EXACT]:
        r = int(r)
        level, _ = oracle.bfs(off, idx, r)
        mp = oracle.min_parent(off, idx, r, level)
        reached = level[level >= 0]
        rec["exact"].append({
            "root": r,
            "levels_sha256": sha(level),
            "min_parent_sha256": sha(mp),
            "layer_sizes": np.bincount(reached).tolist(),
            "component_edges": int(oracle.component_edges(off, level)),
        })
        print(f"root {r}: depth {int(reached.max())}, {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
