"""Writes serve8_rmat_levels.json: digests of the oracle's results for the
serving workload, so that queries served at full size compare bit-exactly
without the oracle's CPU time in the test.

Workload: 8 R-MAT graphs (Sec. 6.2: initiator 0.57, 0.19, 0.19, 0.05),
SCALE 14, 16, 18, 19, 20, 21, 22, 23, edgefactor 16, graph seeds 10..17;
symmetric CSRs with self-loops dropped, rows sorted and deduplicated
(Sec. 6.2-6.3); each graph's root pool is the 4096 roots of seed 5 + i
(Sec. 6.3 root rule). For the first 8 roots of every pool: the SHA-256 of
the int32 level array (Sec. 4 hop distances, -1 = unreached) and the
reached count. Every value comes from `oracle/` only.

    python tests/golden/make_serve8.py       # ~6 GB of host memory, a few minutes
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))
import oracle  # noqa: E402

SCALES = [14, 16, 18, 19, 20, 21, 22, 23]
EF, POOL, PER_GRAPH = 16, 4096, 8
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serve8_rmat_levels.json")


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=a.dtype.newbyteorder("<")).data).hexdigest()


def main() -> None:
    t0 = time.time()
    graphs = []
    for i, scale in enumerate(SCALES):
        n = 1 << scale
        s, d = oracle.gen_edges(oracle.RMAT, scale, EF, 10 + i)
        off, idx = oracle.build_csr(n, s, d)
        del s, d
        pool = oracle.sample_roots(off, n, 5 + i, POOL)
        queries = []
        for r in pool[:PER_GRAPH]:
            level, _ = oracle.bfs(off, idx, int(r))
            queries.append({"root": int(r), "levels_sha256": sha(level),
                            "reached": int((level >= 0).sum())})
        graphs.append({"scale": scale, "graph_seed": 10 + i, "root_seed": 5 + i,
                       "nnz": int(idx.size), "offsets_sha256": sha(off),
                       "indices_sha256": sha(idx), "pool_sha256": sha(pool),
                       "queries": queries})
        print(f"scale {scale}: {time.time() - t0:.0f} s", flush=True)
    rec = {"what": "oracle results for 8 R-MAT graphs (Sec. 6.2-6.3), edgefactor 16; "
                   "SHA-256 of little-endian arrays",
           "edgefactor": EF, "pool": POOL, "graphs": graphs}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
