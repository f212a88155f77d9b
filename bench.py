#!/usr/bin/env python3
"""Benchmark: single-source hybrid BFS, harmonic-mean TEPS over 64 roots on a
scale-26 R-MAT graph (edgefactor 16), one JSON line on stdout.

One step = one BFS from each of the 64 sampled roots on the resident graph
(init, direction switch, top-down / bottom-up layers, conversions, counters:
the whole traversal). Graph generation and CSR build are Graph500's untimed
kernels 0/1 and are reported separately (`graph_build_s`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--scale S] [--impl gb300|reference]

With N > 1 (torchrun) every rank traverses its own replica of the graph from
its own roots (weak scaling, no data-path collective); value is the sum of
the ranks' harmonic-mean TEPS and the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "GTEPS (harmonic mean, 64 roots)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--scale", type=int, default=26)
    p.add_argument("--edgefactor", type=int, default=16)
    p.add_argument("--roots", type=int, default=64)
    p.add_argument("--graph-seed", type=int, default=1)
    p.add_argument("--root-seed", type=int, default=2)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-scale", type=int, default=20,
                   help="scale of the oracle's bounded sample graph")
    p.add_argument("--cpu-roots", type=int, default=8)
    return p.parse_args()


def peaks():
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def hmean(x):
    x = np.asarray(x, dtype=np.float64)
    return float(len(x) / np.sum(1.0 / x)) if len(x) and (x > 0).all() else 0.0


def cpu_baseline(args, n_steps=None):
    """The oracle (plain single-threaded C FIFO BFS) on a bounded sample of the
    workload: the same R-MAT recipe at --cpu-scale, built by the oracle itself,
    --cpu-roots roots from the same root seed. Returns per-root TEPS."""
    import oracle
    scale = args.cpu_scale
    n = 1 << scale
    s, d = oracle.gen_edges(oracle.RMAT, scale, args.edgefactor, args.graph_seed)
    off, idx = oracle.build_csr(n, s, d)
    del s, d
    roots = oracle.sample_roots(off, n, args.root_seed, args.cpu_roots)
    teps, secs = [], 0.0
    for r in roots:
        t0 = time.perf_counter()
        lv, _ = oracle.bfs(off, idx, int(r))
        dt = time.perf_counter() - t0
        secs += dt
        teps.append(oracle.component_edges(off, lv) / dt)
    return {"value": hmean(teps) / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"oracle FIFO BFS, {len(roots)} roots on the same R-MAT recipe at scale "
                      f"{scale} (edgefactor {args.edgefactor}), CSR built by the oracle; the "
                      f"single-threaded oracle cannot build the scale-{args.scale} CSR in "
                      f"the bench's time bound",
            "seconds": round(secs, 3)}


def run_reference(args, rank, world):
    """--impl reference: the oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args)
        if i >= args.warmup:
            steps.append(cb)
    val = hmean([s["value"] for s in steps])
    ms = 1000.0 * sum(s["seconds"] for s in steps) / max(1, len(steps))
    cb = dict(steps[-1])
    cb["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"rmat-scale{args.scale}-ef{args.edgefactor}-64roots",
                       "sample_scale": args.cpu_scale, "roots_per_step": args.cpu_roots},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1704_02259_gb300 as gb

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    gb.lib()
    scale, ef = args.scale, args.edgefactor
    n = 1 << scale
    t0 = time.perf_counter()
    off, idx = gb.rmat_graph(scale, ef, args.graph_seed)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    torch.cuda.empty_cache()
    nnz = idx.numel()
    cfg = gb.default_config()
    cfg.timing = 1
    g = gb.Graph(off, idx, cfg)
    roots = gb.sample_roots(off, n, args.root_seed + rank, args.roots).cpu().tolist()
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def one_step(record=None):
        for r in roots:
            if record is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            g.run(r, level, parent)
            if record is not None:
                e1.record(stream)
                st = g.stats()
                record.append((e0, e1, st))

    for _ in range(args.warmup):
        one_step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = gb.launch_count()
    recs = []
    barrier()
    tw0 = time.perf_counter()
    for _ in range(args.steps):
        one_step(recs)
    barrier()
    wall = time.perf_counter() - tw0
    launches = gb.launch_count() - launches0
    clk = clocks.stop()

    times = [a.elapsed_time(b) / 1e3 for a, b, _ in recs]
    edges = [st.component_edges for _, _, st in recs]
    teps = [e / t for e, t in zip(edges, times)]
    my_hmean = hmean(teps)
    my_total_s = sum(times)
    # roofline of the bottom-up step kernel (the dominant kernel): algorithmic
    # bytes per launch over its CUDA-event duration
    bu_bytes = bu_ms = 0.0
    td_bytes = td_ms = 0.0
    for _, _, st in recs:
        for L in st.layers:
            if L["direction"] == 1:
                bu_bytes += n / 4 + 8 * L["n_u"] + 4 * L["examined"] + 8 * L["found"]
                bu_ms += L["ms_main"]
            else:
                td_bytes += 20 * L["n_f"] + 4 * L["m_f"] + 28 * L["found"]
                td_ms += L["ms_main"]
    n_bu = sum(1 for _, _, st in recs for L in st.layers if L["direction"] == 1)

    if dist is not None:
        t = torch.tensor([my_hmean, my_total_s, wall], dtype=torch.float64, device="cuda")
        allv = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(allv, t)
        vals = torch.stack(allv).cpu().numpy()
        value = float(vals[:, 0].sum())
        total_s = float(vals[:, 1].max())
        wall = float(vals[:, 2].max())
    else:
        value, total_s = my_hmean, my_total_s

    # end to end through the public API with host buffers: the results of
    # every root are copied back to pinned host memory inside the timed region
    lv_h = torch.empty(n, dtype=torch.int32).pin_memory()
    pa_h = torch.empty(n, dtype=torch.int32).pin_memory()
    cfg.timing = 0
    g.set_config(cfg)
    barrier()
    e2e_teps = []
    for r in roots:
        t1 = time.perf_counter()
        g.run(r, lv_h, pa_h)
        dt = time.perf_counter() - t1
        e2e_teps.append(g.stats().component_edges / dt)
    barrier()
    e2e_val = hmean(e2e_teps)
    if dist is not None:
        t = torch.tensor([e2e_val], dtype=torch.float64, device="cuda")
        allv = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(allv, t)
        e2e_val = float(sum(x.item() for x in allv))

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    achieved = (bu_bytes / (bu_ms / 1e3)) / 1e9 if bu_ms > 0 else 0.0
    m_c = statistics.median(edges)
    b_sweep = 4 * nnz + 8 * (n + 1) + 2 * n / 8 + 8 * n
    roof_teps = m_c * peak * 1e9 / b_sweep
    line = {
        "metric": METRIC, "value": value / 1e9, "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"rmat-scale{scale}-ef{ef}-64roots", "scale": scale,
                   "edgefactor": ef, "n": n, "nnz": nnz, "roots": len(roots),
                   "graph_seed": args.graph_seed, "root_seed": args.root_seed,
                   "l2": "inputs larger than L2 (CSR of scale 26 is ~8 GB)",
                   "policy": "edge alpha=14 beta=24", "bu_probe": cfg.bu_probe},
        "roofline": {"bound": "hbm", "kernel": "bu_kernel", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": bu_bytes / max(1, n_bu),
                     "avg_launch_ms": bu_ms / max(1, n_bu)},
        "sweep_roofline": {"bytes": b_sweep, "teps": roof_teps / 1e9, "unit": "GTEPS",
                           "frac": value / roof_teps if world == 1 else None},
        "td_step": {"achieved_gbs": (td_bytes / (td_ms / 1e3)) / 1e9 if td_ms > 0 else 0.0,
                    "ms": td_ms},
        "aggregate_teps": sum(edges) / sum(times) / 1e9,
        "teps_min_median_max": [min(teps) / 1e9, statistics.median(teps) / 1e9, max(teps) / 1e9],
        "component_edges_median": m_c,
        "graph_build_s": build_s,
        "e2e": {"value": e2e_val / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": 4 * len(roots),
                "d2h_bytes_per_step": 8 * n * len(roots)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
