"""The N > 1 bench path on CPU: two gloo ranks gather their per-rank figures
and combine them the way bench.py does (independent replicas: rates add,
times take the max); the reference arm prints only on rank 0."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    rows = bench.gather_ranks(dist, world, [100.0 * (rank + 1), 2.0 + rank, 3.0 - rank], "cpu")
    q.put((rank, rows.tolist(), bench.combine_ranks(rows)))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rows, comb in out:
        assert np.allclose(rows, [[100.0, 2.0, 3.0], [200.0, 3.0, 2.0]])
        assert comb == (300.0, 3.0, 3.0)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "1", "--scale", "12"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "1", "--scale", "12"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["cores"] == 1
    # the same metric, unit, direction and workload as the GPU arm's line
    sys.path.insert(0, ROOT)
    import bench
    assert line["metric"] == bench.METRIC and line["unit"] == "GTEPS"
    assert line["higher_is_better"] is True
    # the workload it ran is the one it names: the GPU arm's config for the
    # same arguments, on the graph the oracle built
    import argparse
    args = argparse.Namespace(scale=12, edgefactor=16, roots=64, graph_seed=1, root_seed=2)
    import oracle
    s, d = oracle.gen_edges(oracle.RMAT, 12, 16, 1)
    off, idx = oracle.build_csr(1 << 12, s, d)
    assert line["config"] == bench.workload_config(args, 1 << 12, int(idx.size))
    assert line["config"]["workload"] == "rmat-scale12-ef16-64roots"
    assert line["steps"] == 3 and line["warmup"] == 1 and line["cpu_baseline"]["roots"] == 3
    for k in ("n_gpus", "steps", "warmup", "ms_per_step", "scaling", "vs_baseline", "dtype", "data"):
        assert k in line, k
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == "GTEPS"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
