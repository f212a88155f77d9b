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
    p.add_argument("--cpu-roots", type=int, default=4,
                   help="most roots the cpu_baseline leg times (in order, from the 64)")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="cpu_baseline stops after the root that passes this much traversal time")
    p.add_argument("--mode", default="single", choices=["single", "serve", "batch", "study"],
                   help="single: the headline line (single-source + batched); "
                        "serve: the serving stream over 8 resident graphs; "
                        "batch: one batched configuration timed alone; "
                        "study: the switch-policy trace (Table 2 form) and the "
                        "scale x edgefactor sweep (Figure 3 form)")
    p.add_argument("--batch-k", type=int, default=512, help="roots per batch (--mode batch)")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched comparison, the Table 3 analogue and the layer-loop "
                        "comparison")
    p.add_argument("--device-loop", type=int, default=2, choices=[0, 1, 2, 3],
                   help="bfs_config.device_loop: 0 host loop, 1 persistent device loop, "
                        "2 library default, 3 graph loop (the timed region records hub-sweep "
                        "events, so 3 falls back to the host loop there)")
    p.add_argument("--batch-scale", type=int, default=22)
    p.add_argument("--serve-queries", type=int, default=10000)
    p.add_argument("--serve-seconds", type=float, default=4.0,
                   help="cap on each rate's arrival window")
    return p.parse_args()


def peaks():
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def hub_sweep_bytes(n, probed, written, out_bytes=8):
    """Algorithmic bytes of one hub sweep launch (compact records): the
    visited words read and the next, pend and visited words written (n/8
    bytes each), the base and rank words read (n/4), one 4-byte hub record
    per probed vertex (unvisited, degree >= 1), and out_bytes per written
    vertex (the hub hits, or in the first sweep of a traversal every vertex
    not reached before it): 8 for parent and level, 4 for the parent alone
    when the levels are written by the level pass after the traversal."""
    return 3 * n / 4 + 4 * probed + out_bytes * written


def one_sweep_bytes(n, nnz):
    """The one-sweep model: every CSR index and row bound read once, the
    frontier and visited bitmaps once each, level and parent written once."""
    return 4 * nnz + 8 * (n + 1) + 2 * n / 8 + 8 * n


def roofline_teps(m_c, peak_gbs, bytes_per_bfs):
    """TEPS of a traversal that moves bytes_per_bfs at peak_gbs GB/s and
    counts m_c edges."""
    return m_c * peak_gbs * 1e9 / bytes_per_bfs


def batch_bytes(n, k, layers):
    """The batched byte model (W = k/64 lane words of 8 bytes): per layer,
    4 bytes per CSR entry read (the examined count), one 8W-byte lane-word
    gather or OR per entry, and the seen, frontier and next words of every
    vertex (3 x 8W x n); once per batch the k x n int8 level rows."""
    W = max(1, (k + 63) // 64)
    total = 0.0
    for L in layers:
        total += 4 * L["examined"] + 8 * W * L["examined"] + 3 * 8 * W * n
    return total + k * n


# source text each recorded ncu capture belongs to (start, end markers in bfs.cu)
KERNEL_TEXT = {
    "bu_hubc_stream_kernel": ("// Streaming sweep, one pipeline per warp",
                              "// Per-vertex step of the compact gather sweep"),
    "bu_hubc_kernel": ("// Per-vertex step of the compact gather sweep",
                       "__global__ void __launch_bounds__(kBlock) bu_list_kernel("),
}


def kernel_source_sha1(name):
    import hashlib
    src = open(os.path.join(HERE, "paper_1704_02259_gb300", "csrc", "bfs.cu")).read()
    a = src.find(KERNEL_TEXT[name][0])
    b = src.find(KERNEL_TEXT[name][1], a + 1)
    if a < 0 or b < 0:
        return None
    return hashlib.sha1(src[a:b].encode()).hexdigest()


def measured_traffic(name, scale, edgefactor, launches, first):
    """DRAM bytes per launch of a hub sweep kernel, from its committed ncu
    summary (profiles/<kernel>_rmat24.md: dram__bytes_read.sum +
    dram__bytes_write.sum of captured first sweeps and later sweeps at R-MAT
    scale 24), weighted by this run's mix of first and later sweeps and
    scaled to the run's n (the sweep's bytes grow with n: every bitmap word,
    record and output is per vertex). None when there is no summary, the
    edgefactor differs, or the kernel's source text changed since the
    capture (the summary records its SHA-1)."""
    path = os.path.join(HERE, "profiles", f"{name}_rmat24.md")
    if name not in KERNEL_TEXT or edgefactor != 16 or not os.path.exists(path) or launches < 1:
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if kernel_source_sha1(name) != vals.get("kernel_source_sha1"):
        return None
    try:
        t1 = float(vals["traffic_first_sweep_bytes"])
        t2 = float(vals["traffic_later_sweep_bytes"])
        cap = int(vals["capture_scale"])
    except (KeyError, ValueError):
        return None
    per = (first * t1 + (launches - first) * t2) / launches
    return per * 2.0 ** (scale - cap)


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


def gather_ranks(dist, world, vals, device):
    """All ranks' value vectors, as a [world, len(vals)] float64 array."""
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    allv = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(allv, t)
    return torch.stack(allv).cpu().numpy()


def combine_ranks(rows):
    """Whole-job figures from per-rank [hmean TEPS, timed seconds, wall]:
    ranks run independent replicas, so rates add and times take the max."""
    rows = np.asarray(rows, dtype=np.float64)
    return float(rows[:, 0].sum()), float(rows[:, 1].max()), float(rows[:, 2].max())


def hmean(x):
    x = np.asarray(x, dtype=np.float64)
    return float(len(x) / np.sum(1.0 / x)) if len(x) and (x > 0).all() else 0.0


GOLDEN = os.path.join(HERE, "tests", "golden")
# oracle-written digests of the workloads whose CSR the single-threaded oracle
# takes minutes to build (tests/golden/make_*.py write them from oracle/ only)
GOLDEN_CSR = {(26, 16, 1): "rmat26_ef16_seed1_bfs.json", (22, 16, 1): "rmat22_ef16_seed1_batch.json"}
ORACLE_BUILD_MAX_SCALE = 20   # above this the oracle's own CSR build takes minutes


def workload_config(args, n, nnz):
    """The workload both arms name in `config`: the graph and its root set."""
    return {"workload": f"rmat-scale{args.scale}-ef{args.edgefactor}-{args.roots}roots",
            "scale": args.scale, "edgefactor": args.edgefactor, "n": n, "nnz": nnz,
            "roots": args.roots, "graph_seed": args.graph_seed, "root_seed": args.root_seed,
            "l2": f"inputs larger than L2 (CSR of scale {args.scale} is "
                  f"{(8 * (n + 1) + 4 * nnz) / 1e9:.2f} GB)"}


def _sha256(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a, dtype=a.dtype.newbyteorder("<")).data).hexdigest()


_HOST_CSR = {}


def host_csr(scale, ef, seed, device_csr=None):
    """(offsets, indices) of an R-MAT graph on the host, for the oracle legs.

    Up to ORACLE_BUILD_MAX_SCALE the oracle generates and builds it itself.
    Above that its single-threaded build takes minutes (about 20 at scale
    26), so the library's GPU build (`device_csr`, or one made here) is
    copied to the host in untimed setup and used only if the SHA-256 of both
    arrays equals the digest the oracle itself wrote for that graph: the
    bytes are then the oracle's own CSR. Returns None when no digest exists
    for a graph that large."""
    key = (scale, ef, seed)
    if key in _HOST_CSR:
        return _HOST_CSR[key]
    import oracle
    n = 1 << scale
    if scale <= ORACLE_BUILD_MAX_SCALE:
        s, d = oracle.gen_edges(oracle.RMAT, scale, ef, seed)
        _HOST_CSR[key] = oracle.build_csr(n, s, d)
        return _HOST_CSR[key]
    if key not in GOLDEN_CSR:
        return None
    with open(os.path.join(GOLDEN, GOLDEN_CSR[key])) as f:
        gold = json.load(f)
    if device_csr is None:
        import torch
        import paper_1704_02259_gb300 as gb
        device_csr = gb.rmat_graph(scale, ef, seed)
        torch.cuda.synchronize()
    off = device_csr[0].cpu().numpy()
    idx = device_csr[1].cpu().numpy()
    if _sha256(off) != gold["offsets_sha256"] or _sha256(idx) != gold["indices_sha256"]:
        raise RuntimeError(f"the GPU-built CSR of scale {scale} differs from the oracle's digests")
    _HOST_CSR[key] = (off, idx)
    return _HOST_CSR[key]


def oracle_roots(off, args, rank=0):
    """The workload's roots, drawn by the oracle's own sampler."""
    import oracle
    return oracle.sample_roots(off, off.size - 1, args.root_seed + rank, args.roots)


def oracle_root_teps(off, idx, root):
    """One timed oracle traversal (plain single-threaded C FIFO BFS): TEPS and
    seconds. Only the BFS call is timed; the component edge count after it is
    the TEPS numerator (undirected deduplicated edges reached)."""
    import oracle
    t0 = time.perf_counter()
    lv, _ = oracle.bfs(off, idx, int(root))
    dt = time.perf_counter() - t0
    return oracle.component_edges(off, lv) / dt, dt


def cpu_baseline(args, device_csr=None):
    """The oracle on a bounded sample of the bench's own workload: the first
    roots of the same 64 on the same graph, one after another, until
    --cpu-roots roots or --cpu-seconds of traversal time are reached (at
    least one root)."""
    host = host_csr(args.scale, args.edgefactor, args.graph_seed, device_csr)
    if host is None:
        return {"value": None, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                "sample": f"none: no oracle digest for a scale-{args.scale} CSR"}
    off, idx = host
    roots = oracle_roots(off, args)
    teps, secs = [], 0.0
    for r in roots[:max(1, args.cpu_roots)]:
        t, dt = oracle_root_teps(off, idx, r)
        teps.append(t)
        secs += dt
        if secs >= args.cpu_seconds:
            break
    return {"value": hmean(teps) / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"oracle FIFO BFS, single-threaded, from the first {len(teps)} of the "
                      f"{args.roots} roots on the bench's own graph (R-MAT scale {args.scale}, "
                      f"edgefactor {args.edgefactor}); harmonic mean of per-root TEPS",
            "roots": len(teps), "seconds": round(secs, 3)}


def cpu_throughput(args, device_csr=None):
    """The oracle's throughput on all host cores, one independent root per
    thread (the C BFS runs outside the interpreter lock): aggregate TEPS =
    sum of component edges / wall time, the CPU comparison point for the
    batched GPU runs, on the batched workload's graph (R-MAT
    --batch-scale)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    host = host_csr(args.batch_scale, 16, 1, device_csr)
    if host is None:
        return None
    off, idx = host
    n = off.size - 1
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    roots = oracle.sample_roots(off, n, 4, 2 * cores)

    def one(r):
        lv, _ = oracle.bfs(off, idx, int(r))
        return oracle.component_edges(off, lv)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        edges = sum(ex.map(one, roots))
    dt = time.perf_counter() - t0
    return {"value": edges / dt / 1e9, "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": f"{len(roots)} independent roots, one per thread, on the batched "
                      f"workload's graph (R-MAT scale {args.batch_scale}, edgefactor 16); "
                      f"aggregate edges / wall time",
            "seconds": round(dt, 3)}


def run_reference(args, rank, world):
    """--impl reference: the oracle, timed on the host cores (rank 0 only),
    on the bench's own workload: each step is one traversal from the next of
    the 64 roots (cycling), on the same graph; value = harmonic mean of the
    timed steps' TEPS. The graph is set up untimed (host_csr)."""
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    off, idx = host_csr(args.scale, args.edgefactor, args.graph_seed)
    roots = oracle_roots(off, args)
    # the untimed warm-up steps (a plain C program has nothing to warm but
    # its first page faults) run side by side, one per core, so a warm-up
    # costs one traversal's wall time; the timed steps then run one at a
    # time on an otherwise idle host
    if args.warmup > 0:
        with ThreadPoolExecutor(max(1, min(args.warmup, os.cpu_count() or 1))) as ex:
            list(ex.map(lambda i: oracle_root_teps(off, idx, roots[i % len(roots)]),
                        range(args.warmup)))
    teps, secs = [], []
    for i in range(args.warmup, args.warmup + args.steps):
        t, dt = oracle_root_teps(off, idx, roots[i % len(roots)])
        teps.append(t)
        secs.append(dt)
    val = hmean(teps) / 1e9
    cb = {"value": val, "unit": "GTEPS", "cores": 1, "kind": "oracle",
          "sample": f"oracle FIFO BFS, single-threaded, one root per step (roots "
                    f"{args.warmup}..{args.warmup + args.steps - 1} of the {args.roots}, "
                    f"cycling) on the bench's own graph (R-MAT scale {args.scale}, edgefactor "
                    f"{args.edgefactor})",
          "roots": len(teps), "seconds": round(sum(secs), 3)}
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(secs) / max(1, len(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": workload_config(args, off.size - 1, int(idx.size)),
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


TABLE3_PAPER = [2879193, 30910, 34, 1.06, 2.51, 41.06]   # Table 3, per layer


def table3_analogue(gb, torch, scale=18, ef=16, seed=1, root_seed=2):
    """Table 3 on the GPU: every layer bottom-up from 64 roots at SCALE 18,
    edgefactor 16; per layer, edges examined per newly visited vertex
    (averaged over the roots that reach the layer) and the layer's device
    time. Variants: the row scan with a per-lane probe of P entries before
    the warp-cooperative tail (the paper's MAX_POS structure, P = 2, 8, 32),
    and the hub probe first (this library's default bottom-up step)."""
    n = 1 << scale
    off, idx = gb.rmat_graph(scale, ef, seed)
    roots = gb.sample_roots(off, n, root_seed, 64).tolist()
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    pa = torch.empty_like(lv)
    out = {"workload": f"rmat-scale{scale}-ef{ef}-64roots, every layer bottom-up",
           "paper_edges_per_visited": TABLE3_PAPER}
    for name, head, probe in (("scan_p2", 0, 2), ("scan_p8", 0, 8), ("scan_p32", 0, 32),
                              ("hub", 2, 8)):
        cfg = gb.default_config()
        cfg.policy = gb.POLICY_FORCED
        cfg.forced_len = 1
        cfg.forced[0] = 1
        cfg.bu_head = head
        cfg.bu_probe = probe
        cfg.device_loop = 0
        cfg.timing = 1
        g = gb.Graph(off, idx, cfg)
        for r in roots[:4]:
            g.run(r, lv, pa)
        ratio, ms = {}, {}
        for r in roots:
            g.run(r, lv, pa)
            torch.cuda.synchronize()
            layers = g.stats().layers
            if sum(L["found"] for L in layers) < n // 100:
                continue                    # root outside the large component
            for d, L in enumerate(layers):
                if L["found"] > 0:
                    ratio.setdefault(d, []).append(L["examined"] / L["found"])
                    ms.setdefault(d, []).append(L["ms_total"])
        out[name] = {"edges_per_visited": [round(float(np.mean(ratio[d])), 2) for d in sorted(ratio)],
                     "layer_ms": [round(float(np.mean(ms[d])), 4) for d in sorted(ms)]}
        del g
    return out


def batched_comparison(gb, torch, scale, seed=1, root_seed=4, ks=(64, 128, 256, 512)):
    """Batched multi-source BFS against k sequential single-source runs on the
    same GPU (R-MAT scale 22): aggregate TEPS = sum of the roots' component
    edges / wall time on the stream (CUDA events)."""
    n = 1 << scale
    off, idx = gb.rmat_graph(scale, 16, seed)
    g = gb.Graph(off, idx)
    allroots = gb.sample_roots(off, n, root_seed, max(ks))
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    pa = torch.empty_like(lv)
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for r in allroots[:4].tolist():
        g.run(r, lv, pa)
    mc, seq_ms = {}, {}
    for r in allroots.tolist():
        ev[0].record(st)
        g.run(r, lv, pa)
        ev[1].record(st)
        ev[1].synchronize()
        seq_ms[r] = ev[0].elapsed_time(ev[1])
        mc[r] = g.stats().component_edges
    out = {"workload": f"rmat-scale{scale}-ef16", "per_k": []}
    launches0 = gb.launch_count()
    for k in ks:
        roots = allroots[:k]
        rl = roots.tolist()
        edges = sum(mc[r] for r in rl)
        t_seq = sum(seq_ms[r] for r in rl)
        best = g.autotune_batch(roots)
        levels = torch.empty((k, n), dtype=torch.int8, device="cuda")
        g.run_batch(roots, levels)
        ts = []
        for _ in range(3):
            ev[0].record(st)
            g.run_batch(roots, levels)
            ev[1].record(st)
            ev[1].synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        t = statistics.median(ts)
        layers, _ = g.batch_stats()
        bb = batch_bytes(n, k, layers)
        peak, peak_kind = peaks()
        out["per_k"].append({
            "k": k, "batch_ms": t, "sequential_ms": t_seq,
            "batch_gteps": edges / t / 1e6, "sequential_gteps": edges / t_seq / 1e6,
            "speedup": t_seq / t, "alpha": best.alpha, "beta": best.beta,
            "lane_probe": best.lane_probe,
            "roofline": {"bound": "hbm", "bytes": bb, "achieved": bb / (t / 1e3) / 1e9,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": bb / (t / 1e3) / 1e9 / peak,
                         "directions": "".join("B" if L["direction"] else "T" for L in layers)}})
    out["gpu_launches_batched"] = gb.launch_count() - launches0
    g.close()
    return out


def run_study(args):
    """Two studies of the paper's evaluation, one JSON line.

    table2: one root at SCALE 18, edgefactor 16, run under the vertex policy
    read off Table 2 (f = n_u / 1024, g = n / 64 on the frontier size) and
    under the edge policy (the defaults): per layer the frontier size v_f,
    the unvisited count n_u, f, g, the direction taken and the layer's device
    time, and the run's TEPS.
    sweep: R-MAT and the Erdos-Renyi control at SCALE 14-22 and edgefactor
    16, 32, 64 (the axes of Figure 3), 16 roots each, harmonic-mean GTEPS of
    the hybrid (edge policy), top-down only and bottom-up from the first
    layer on."""
    import torch
    import paper_1704_02259_gb300 as gb
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()

    def timed(g, roots, level, parent):
        for r in roots[:2]:
            g.run(r, level, parent)
        teps = []
        for r in roots:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.run(r, level, parent)
            e1.record(stream)
            e1.synchronize()
            teps.append(g.stats().component_edges / (e0.elapsed_time(e1) / 1e3))
        return hmean(teps) / 1e9

    def forced(pattern):
        c = gb.default_config()
        c.policy = gb.POLICY_FORCED
        c.forced_len = len(pattern)
        for i, x in enumerate(pattern):
            c.forced[i] = x
        return c

    out = {"metric": "policy trace and scale sweep", "mode": "study", "n_gpus": 1,
           "data": "synthetic", "dtype": "int32"}
    # Table 2 form
    n = 1 << 18
    off, idx = gb.rmat_graph(18, 16, 1)
    root = gb.sample_roots(off, n, 2, 1).tolist()[0]
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty_like(level)
    t2 = {"workload": "rmat-scale18-ef16, one root", "root": root}
    for name, policy in (("vertex", gb.POLICY_VERTEX), ("edge", gb.POLICY_EDGE)):
        c = gb.default_config()
        c.policy = policy
        c.device_loop = 0
        c.timing = 1
        g = gb.Graph(off, idx, c)
        for _ in range(3):
            g.run(root, level, parent)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.run(root, level, parent)
        e1.record(stream)
        e1.synchronize()
        st = g.stats()
        rows = [{"layer": d + 1, "v_f": L["n_f"], "n_u": L["n_u"], "f": L["n_u"] >> 10,
                 "g": n >> 6, "approach": "BU" if L["direction"] else "TD",
                 "ms": round(L["ms_total"], 4)} for d, L in enumerate(st.layers)]
        t2[name] = {"layers": rows,
                    "gteps": st.component_edges / (e0.elapsed_time(e1) / 1e3) / 1e9}
        g.close()
    out["table2"] = t2
    del off, idx, level, parent
    # Figure 3 form
    sweep = []
    for kind_name, kind in (("rmat", gb.GEN_RMAT), ("er", gb.GEN_ER)):
        for scale in (14, 16, 18, 20, 22):
            for ef in (16, 32, 64):
                n = 1 << scale
                off, idx = gb.rmat_graph(scale, ef, 1, kind=kind)
                roots = gb.sample_roots(off, n, 2, 16).tolist()
                level = torch.empty(n, dtype=torch.int32, device="cuda")
                parent = torch.empty_like(level)
                row = {"graph": kind_name, "scale": scale, "edgefactor": ef,
                       "nnz": idx.numel()}
                for name, cfg in (("hybrid", gb.default_config()), ("top_down", forced([0])),
                                  ("bottom_up", forced([1]))):
                    g = gb.Graph(off, idx, cfg)
                    row[name + "_gteps"] = timed(g, roots, level, parent)
                    g.close()
                sweep.append(row)
                del off, idx, level, parent
                torch.cuda.empty_cache()
    out["sweep"] = sweep
    print(json.dumps(out), flush=True)


def run_batch_mode(args):
    """One batched configuration timed alone (R-MAT --batch-scale, --batch-k
    roots, the default batch configuration, host-driven layers): W untimed
    and K timed batches, CUDA events on the stream; value = aggregate GTEPS
    (sum of the roots' component edges per batch / batch time)."""
    import torch
    import paper_1704_02259_gb300 as gb
    torch.cuda.set_device(0)
    scale, k = args.batch_scale, args.batch_k
    n = 1 << scale
    off, idx = gb.rmat_graph(scale, 16, 1)
    g = gb.Graph(off, idx)
    roots = gb.sample_roots(off, n, 4, k)
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    pa = torch.empty_like(lv)
    edges = 0
    for r in roots.tolist():
        g.run(r, lv, pa)
        edges += g.stats().component_edges
    levels = torch.empty((k, n), dtype=torch.int8, device="cuda")
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(args.warmup):
        g.run_batch(roots, levels)
    launches0 = gb.launch_count()
    ts = []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        ev[0].record(st)
        g.run_batch(roots, levels)
        ev[1].record(st)
        ev[1].synchronize()
        ts.append(ev[0].elapsed_time(ev[1]))
    torch.cuda.nvtx.range_pop()
    ms = statistics.median(ts)
    layers, pairs = g.batch_stats()
    print(json.dumps({
        "metric": "batched multi-source BFS, aggregate GTEPS", "mode": "batch",
        "value": edges / ms / 1e6, "unit": "GTEPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": f"rmat-scale{scale}-ef16-k{k}", "k": k, "n": n,
                   "directions": "".join("B" if L["direction"] else "T" for L in layers)},
        "pairs_reached": pairs, "gpu_launches": gb.launch_count() - launches0}), flush=True)
    g.close()


def serve_sweep(gb, torch, rates, queries, seconds, seed=5):
    """Serving: 8 resident R-MAT graphs (scales 14, 16, 18..23, edgefactor 16,
    seeds 10..17), Poisson arrivals at each rate, graph uniform, root uniform
    among degree >= 1 vertices; p50/p99 latency and queries/s per rate.
    Each rate sends min(queries, rate * seconds) queries to one long-running
    server whose workers were warmed by a burst first."""
    scales = [14, 16, 18, 19, 20, 21, 22, 23]
    graphs, roots, pools = [], [], []
    csr_bytes = 0
    for i, sc in enumerate(scales):
        off, idx = gb.rmat_graph(sc, 16, 10 + i)
        csr_bytes += off.numel() * 8 + idx.numel() * 4
        g = gb.Graph(off, idx)
        graphs.append(g)
        roots.append(gb.sample_roots(off, 1 << sc, 5 + i, 4096).cpu().numpy())
        pools.append([torch.empty(1 << sc, dtype=torch.int32, device="cuda") for _ in range(16)])
    cfg = gb.default_serve_config()
    cfg.workers = 4
    cfg.max_batch = 512
    rng = np.random.default_rng(seed)
    results = []
    srv = gb.Server(cfg)
    ids = [srv.add_graph(g) for g in graphs]
    warm = []
    for rep in range(3):
        for gi in range(len(graphs)):
            for j in range(64 if rep else 1):
                r = int(roots[gi][j % len(roots[gi])])
                warm.append(srv.submit(ids[gi], r, pools[gi][j % len(pools[gi])]))
        for t in warm:
            srv.wait(t)
        warm = []
    for rate in rates:
        srv.reset_stats()
        nq = int(min(queries, rate * seconds))
        gsel = rng.integers(0, len(graphs), size=nq)
        gaps = rng.exponential(1.0 / rate, size=nq)
        tickets = []
        t0 = time.perf_counter()
        due = t0
        for q in range(nq):
            due += gaps[q]
            while time.perf_counter() < due:
                pass
            gi = int(gsel[q])
            r = int(roots[gi][rng.integers(0, len(roots[gi]))])
            tickets.append(srv.submit(ids[gi], r, pools[gi][q % len(pools[gi])]))
        bad = sum(1 for t in tickets if srv.wait(t) != 0)
        st = srv.stats()
        results.append({"rate_qps": rate, "queries": nq, "p50_ms": st["p50_us"] / 1e3,
                        "p99_ms": st["p99_us"] / 1e3, "achieved_qps": st["qps"],
                        "mean_batch": st["mean_batch"], "batches": st["batches"],
                        "failed": bad})
    srv.close()
    for g in graphs:
        g.close()
    meta = {"workload": "8 R-MAT graphs, scales 14,16,18-23, ef 16, Poisson stream",
            "csr_bytes": csr_bytes, "workers": cfg.workers, "max_batch": cfg.max_batch}
    return results, meta


def run_serve(args):
    """--mode serve: the serving sweep over arrival rates 100 to 20,000/s."""
    import torch
    import paper_1704_02259_gb300 as gb
    torch.cuda.set_device(0)
    results, meta = serve_sweep(gb, torch, [100, 300, 1000, 3000, 10000, 20000],
                                args.serve_queries, args.serve_seconds)
    line = {"metric": "serving latency p50/p99 and queries/s", "mode": "serve",
            "value": max(r["achieved_qps"] for r in results), "unit": "queries/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "int32", "data": "synthetic",
            "config": meta, "rates": results}
    print(json.dumps(line), flush=True)


def small_config(gb, torch, scale, kind=None, seed=1, root_seed=2, roots=64):
    """A smaller single-source configuration timed as the headline is (per
    root CUDA events, harmonic mean of per-root TEPS) with the library's
    default configuration, plus its one-sweep roofline fraction."""
    n = 1 << scale
    kind = gb.GEN_RMAT if kind is None else kind
    off, idx = gb.rmat_graph(scale, 16, seed, kind=kind)
    g = gb.Graph(off, idx)
    rl = gb.sample_roots(off, n, root_seed, roots).cpu().tolist()
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    pa = torch.empty_like(lv)
    st = torch.cuda.current_stream()
    for r in rl[:4]:
        g.run(r, lv, pa)
    teps, edges = [], []
    for r in rl:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.run(r, lv, pa)
        e1.record(st)
        e1.synchronize()
        edges.append(g.stats().component_edges)
        teps.append(edges[-1] / (e0.elapsed_time(e1) / 1e3))
    g.close()
    peak, kind_p = peaks()
    v = hmean(teps)
    roof = roofline_teps(statistics.median(edges), peak, one_sweep_bytes(n, idx.numel()))
    return {"workload": f"{'er' if kind == gb.GEN_ER else 'rmat'}-scale{scale}-ef16-{roots}roots",
            "value": v / 1e9, "unit": "GTEPS", "nnz": idx.numel(),
            "teps_min_median_max": [min(teps) / 1e9, statistics.median(teps) / 1e9,
                                    max(teps) / 1e9],
            "sweep_roofline_frac": v / roof, "peak_kind": kind_p}


def main():
    args = parse()
    if args.mode == "study":
        run_study(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "batch":
        run_batch_mode(args)
        return
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
    deg1 = int(((off[1:] - off[:-1]) > 0).sum().item())  # vertices of degree >= 1
    cfg = gb.default_config()
    # events only around the hub sweeps inside the timed region (the kernel
    # the roofline is quoted for); per-layer events for the other sections
    # come from an untimed pass afterwards
    cfg.timing = 2
    cfg.device_loop = args.device_loop
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
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
    for _ in range(args.steps):
        one_step(recs)
    barrier()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - tw0
    launches = gb.launch_count() - launches0
    clk = clocks.stop()

    times = [a.elapsed_time(b) / 1e3 for a, b, _ in recs]
    edges = [st.component_edges for _, _, st in recs]
    teps = [e / t for e, t in zip(edges, times)]
    my_hmean = hmean(teps)
    my_total_s = sum(times)
    # roofline of the hub sweep (the first pass of the dense bottom-up
    # layers, the dominant kernel): algorithmic bytes per launch over its own
    # CUDA-event duration, per kernel that ran it (the streaming sweep for
    # layers with at least hub_stream_percent of n left to find, the
    # gathering sweep for the rest); see hub_sweep_bytes
    sweeps = {}
    scan_ms = 0.0
    bl_bytes = bl_ms = 0.0
    bu1_bytes = bu1_ms = 0.0
    td_bytes = td_ms = 0.0
    n_bl = n_bu1 = 0
    fills_outputs = cfg.td_claim == 1 and not cfg.prune_components
    for _, _, st in recs:
        first_sweep = fills_outputs
        for L in st.layers:
            active = L["n_u"] - (n - deg1)  # unvisited vertices of degree >= 1
            if L["direction"] == 1 and L["converted"] == 3:
                written = L["n_u"] if first_sweep else L["hub_found"]
                stream = (cfg.hub_stream_stages > 0 and
                          active * 100 >= cfg.hub_stream_percent * n)
                name = "bu_hubc_stream_kernel" if stream else "bu_hubc_kernel"
                e = sweeps.setdefault(name, {"bytes": 0.0, "ms": 0.0, "launches": 0,
                                             "first": 0})
                e["bytes"] += hub_sweep_bytes(n, active, written,
                                              4 if cfg.level_pass else 8)
                e["ms"] += L["ms_sweep"]
                e["launches"] += 1
                e["first"] += 1 if first_sweep else 0
                first_sweep = False
    # the other kernels' sections: one untimed pass over the same roots with
    # events around every layer
    pcfg = gb.default_config()
    pcfg.timing = 1
    pcfg.device_loop = args.device_loop
    g.set_config(pcfg)
    prof = []
    for r in roots:
        g.run(r, level, parent)
        prof.append(g.stats())
    g.set_config(cfg)
    for st in prof:
        for L in st.layers:
            active = L["n_u"] - (n - deg1)
            if L["direction"] == 1 and L["converted"] == 3:
                scan_ms += L["ms_main"] - L["ms_sweep"]
            elif L["direction"] == 1 and L["converted"] == 2:
                bl_bytes += n / 8 + 12 * active + 4 * L["examined"] + 16 * L["found"]
                bl_ms += L["ms_main"]
                n_bl += 1
            elif L["direction"] == 1:
                bu1_bytes += n / 4 + 8 * L["n_u"] + 4 * L["examined"] + 8 * L["found"]
                bu1_ms += L["ms_main"]
                n_bu1 += 1
            else:
                td_bytes += 20 * L["n_f"] + 4 * L["m_f"] + 28 * L["found"]
                td_ms += L["ms_main"]

    if dist is not None:
        value, total_s, wall = combine_ranks(
            gather_ranks(dist, world, [my_hmean, my_total_s, wall], "cuda"))
    else:
        value, total_s = my_hmean, my_total_s

    # the layer loops compared on the same roots, untimed per layer: host
    # loop (counters polled per layer), cooperative persistent kernel, CUDA
    # graph with device-side control flow
    loops = {}
    if not args.no_batch:
        for name, mode in (("host", 0), ("persistent", 1), ("graph", 3)):
            lc = gb.default_config()
            lc.device_loop = mode
            g.set_config(lc)
            for r in roots[:4]:
                g.run(r, level, parent)
            ts = []
            for r in roots:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.run(r, level, parent)
                e1.record(stream)
                e1.synchronize()
                ts.append(g.stats().component_edges / (e0.elapsed_time(e1) / 1e3))
            loops[name] = hmean(ts) / 1e9

    # end to end through the public API with host buffers: every root's level
    # and parent arrays are copied back to pinned host memory inside the timed
    # region (host_async: a root's copy overlaps the next root's traversal;
    # the step ends when the last copy has landed)
    bufs = [(torch.empty(n, dtype=torch.int32).pin_memory(),
             torch.empty(n, dtype=torch.int32).pin_memory()) for _ in range(2)]
    cfg.timing = 0
    cfg.host_async = 1
    g.set_config(cfg)
    for i, r in enumerate(roots[:4]):       # untimed: allocate the output pairs
        g.run(r, *bufs[i % 2])
    g.sync()
    barrier()
    # --steps passes over the 64 roots, as in the device-timed region
    e2e_edges = 0
    t1 = time.perf_counter()
    for _ in range(args.steps):
        for i, r in enumerate(roots):
            g.run(r, *bufs[i % 2])
            e2e_edges += g.stats().component_edges
    g.sync()
    dt = time.perf_counter() - t1
    barrier()
    e2e_val = e2e_edges / dt
    if dist is not None:
        e2e_val = float(gather_ranks(dist, world, [e2e_val], "cuda")[:, 0].sum())

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    roofs = {}
    for name, e in sweeps.items():
        ach = e["bytes"] / (e["ms"] / 1e3) / 1e9 if e["ms"] > 0 else 0.0
        roofs[name] = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak,
                       "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                       "traffic": measured_traffic(name, scale, ef, e["launches"], e["first"]),
                       "algorithmic_bytes_per_launch": e["bytes"] / max(1, e["launches"]),
                       "avg_launch_ms": e["ms"] / max(1, e["launches"]),
                       "launches": e["launches"], "first_sweeps": e["first"]}
    dominant = max(roofs, key=lambda k: sweeps[k]["ms"]) if roofs else None
    m_c = statistics.median(edges)
    b_sweep = one_sweep_bytes(n, nnz)
    roof_teps = roofline_teps(m_c, peak, b_sweep)
    line = {
        "metric": METRIC, "value": value / 1e9, "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": workload_config(args, n, nnz),
        "method": {"policy": f"edge alpha={cfg.alpha:g} beta={cfg.beta:g}",
                   "bu_probe": cfg.bu_probe, "bu_head": cfg.bu_head,
                   "device_loop": args.device_loop},
        "roofline": roofs.get(dominant),
        "roofline_other_sweeps": [v for k, v in roofs.items() if k != dominant],
        "sweep_roofline": {"bytes": b_sweep, "teps": roof_teps / 1e9, "unit": "GTEPS",
                           "frac": value / roof_teps if world == 1 else None},
        "bu_scan_step": {"ms": scan_ms, "pass": "untimed, per-layer events"},
        "bu_list_step": {"achieved_gbs": (bl_bytes / (bl_ms / 1e3)) / 1e9 if bl_ms > 0 else 0.0,
                         "ms": bl_ms, "launches": n_bl, "pass": "untimed, per-layer events"},
        "bu_one_pass_step": {"achieved_gbs": (bu1_bytes / (bu1_ms / 1e3)) / 1e9
                             if bu1_ms > 0 else 0.0, "ms": bu1_ms, "launches": n_bu1},
        "td_step": {"achieved_gbs": (td_bytes / (td_ms / 1e3)) / 1e9 if td_ms > 0 else 0.0,
                    "ms": td_ms, "pass": "untimed, per-layer events"},
        "aggregate_teps": sum(edges) / sum(times) / 1e9,
        "teps_min_median_max": [min(teps) / 1e9, statistics.median(teps) / 1e9, max(teps) / 1e9],
        "component_edges_median": m_c,
        "graph_build_s": build_s,
        "e2e": {"value": e2e_val / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": 4 * len(roots),
                "d2h_bytes_per_step": 8 * n * len(roots)},
        "gpu_launches": launches,
        "layer_loops_gteps": loops,
        "clocks": clk,
    }
    if not args.no_batch and world == 1:
        line["batched"] = batched_comparison(gb, torch, args.batch_scale)
        line["table3"] = table3_analogue(gb, torch)
        # the other single-source configurations: scale 16, and scale 20 with
        # its Erdos-Renyi control
        line["configs"] = [small_config(gb, torch, 16), small_config(gb, torch, 20),
                           small_config(gb, torch, 20, kind=gb.GEN_ER, seed=3)]
        res, meta = serve_sweep(gb, torch, [3000, 10000, 20000], args.serve_queries,
                                args.serve_seconds)
        line["serving"] = dict(meta, rates=res)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args, (off, idx))
        line["cpu_throughput"] = cpu_throughput(args)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
