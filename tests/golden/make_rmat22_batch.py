"""Writes rmat22_ef16_seed1_batch.json: digests of the oracle's levels for
the batched workload, so that GPU batches at full size compare bit-exactly
without the oracle's CPU time in the test.

Workload: R-MAT graph (Sec. 6.2: initiator 0.57, 0.19, 0.19, 0.05),
SCALE 22, edgefactor 16, graph seed 1; symmetric CSR with self-loops
dropped, rows sorted and deduplicated (Sec. 6.2-6.3); 512 roots of seed 4
(Sec. 6.3 root rule). For every root, the SHA-256 of its level row as int8
(levels are hop distances, Sec. 4; -1 = unreached; every depth here is far
below 127), its depth and its reached count. Every value comes from
`oracle/` only; roots run on host threads (the C BFS is reentrant).

    python tests/golden/make_rmat22_batch.py     # ~3 GB of host memory, a few minutes
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

SCALE, EF, GRAPH_SEED, ROOT_SEED, K = 22, 16, 1, 4, 512
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat22_ef16_seed1_batch.json")


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=a.dtype.newbyteorder("<")).data).hexdigest()


def main() -> None:
    n = 1 << SCALE
    t0 = time.time()
    s, d = oracle.gen_edges(oracle.RMAT, SCALE, EF, GRAPH_SEED)
    off, idx = oracle.build_csr(n, s, d)
    del s, d
    roots = oracle.sample_roots(off, n, ROOT_SEED, K)
    print(f"graph {time.time() - t0:.0f} s, nnz {idx.size}", flush=True)

    def one(r):
        level, _ = oracle.bfs(off, idx, int(r))
        assert level.max() <= 127
        return {"root": int(r), "int8_levels_sha256": sha(level.astype(np.int8)),
                "depth": int(level.max()), "reached": int((level >= 0).sum())}

    with ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        rows = list(ex.map(one, roots))
    rec = {"what": "oracle levels (int8 rows) on R-MAT SCALE 22, edgefactor 16, graph seed 1 "
                   "(Sec. 6.2-6.3), 512 roots of seed 4; SHA-256 of little-endian arrays",
           "scale": SCALE, "edgefactor": EF, "graph_seed": GRAPH_SEED, "root_seed": ROOT_SEED,
           "n": n, "nnz": int(idx.size), "offsets_sha256": sha(off), "indices_sha256": sha(idx),
           "rows": rows}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
