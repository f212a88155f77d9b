"""Python binding of the GB300 hybrid BFS library (include/bfs.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are passed as raw pointers, streams as ``torch.cuda.current_stream()``
handles. If the shared library has not been built this module raises; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

BFS_OK = 0
STATUS = {0: "BFS_OK", 1: "BFS_ERR_INVALID", 2: "BFS_ERR_OOM", 3: "BFS_ERR_CUDA",
          4: "BFS_ERR_TIMEOUT", 5: "BFS_ERR_DEPTH", 6: "BFS_ERR_BUSY", 7: "BFS_ERR_SHUTDOWN",
          8: "BFS_ERR_INTERNAL"}

GEN_RMAT = 0
GEN_ER = 1
POLICY_EDGE = 0
POLICY_VERTEX = 1
POLICY_FORCED = 2
DEVICE_PTRS = 1
BORROW = 2
VALIDATE = 4
VALIDATE_SYMMETRIC = 8


class BfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("forced_len", ctypes.c_int32),
                ("forced", ctypes.c_uint8 * 64), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("bu_probe", ctypes.c_int32),
                ("td_warp_degree", ctypes.c_int32), ("td_grid_degree", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("bu_words", ctypes.c_int32),
                ("td_claim", ctypes.c_int32), ("bu_head", ctypes.c_int32),
                ("prune_components", ctypes.c_int32), ("bu_list_percent", ctypes.c_int32),
                ("device_loop", ctypes.c_int32), ("host_async", ctypes.c_int32),
                ("parent_min", ctypes.c_int32), ("hub_stream_stages", ctypes.c_int32),
                ("hub_stream_percent", ctypes.c_int32), ("level_pass", ctypes.c_int32)]


class LayerStats(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int32), ("converted", ctypes.c_int32),
                ("n_f", ctypes.c_int64), ("m_f", ctypes.c_int64), ("n_u", ctypes.c_int64),
                ("m_u", ctypes.c_int64), ("examined", ctypes.c_int64), ("found", ctypes.c_int64),
                ("ms_total", ctypes.c_float), ("ms_main", ctypes.c_float),
                ("ms_sweep", ctypes.c_float), ("pad", ctypes.c_float),
                ("hub_found", ctypes.c_int64)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("lane_probe", ctypes.c_int32), ("big_degree", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("layer_slots", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class BatchLayerStats(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("v_f", ctypes.c_int64), ("e_f", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("v_u", ctypes.c_int64), ("e_u", ctypes.c_int64), ("ms", ctypes.c_float),
                ("pad2", ctypes.c_float), ("examined", ctypes.c_int64)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("queue_capacity", ctypes.c_int32),
                ("cancel_on_destroy", ctypes.c_int32), ("reserved", ctypes.c_int32 * 8)]


class ServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("deferred", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("qps", ctypes.c_double),
                ("deep_fallbacks", ctypes.c_int64)]


_lib = None
P = ctypes.c_void_p
I32, I64, U32, U64, DBL = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double

# name -> (restype, argtypes); exactly the entry points include/bfs.h declares
SIGNATURES = {
    "bfs_last_error": (ctypes.c_char_p, []),
    "bfs_launch_count": (I64, []),
    "bfs_alloc_count": (I64, []),
    "bfs_generate_edges": (I32, [I32, I32, I32, U64, DBL, DBL, DBL, P, P, P]),
    "bfs_build_csr": (I32, [I64, I64, P, P, P, P, P, P]),
    "bfs_sample_roots": (I32, [P, I64, U64, I32, I64, P, P, P]),
    "bfs_config_default": (None, [P]),
    "bfs_graph_create": (I32, [P, P, I64, I64, U32, P, P]),
    "bfs_graph_set_config": (I32, [P, P]),
    "bfs_graph_info": (I32, [P, P, P, P, P]),
    "bfs_graph_destroy": (I32, [P]),
    "bfs_graph_reserve": (I32, [P, U32, P]),
    "bfs_run": (I32, [P, I32, P, P, P]),
    "bfs_graph_sync": (I32, [P]),
    "bfs_last_run_stats": (I32, [P, P, I32, P, P]),
    "bfs_run_noalloc": (I32, [P, P, I64, I64, I32, P, P, P]),
    "bfs_batch_config_default": (None, [P]),
    "bfs_graph_set_batch_config": (I32, [P, P]),
    "bfs_graph_get_batch_config": (I32, [P, P]),
    "bfs_run_batch": (I32, [P, P, I32, P, P]),
    "bfs_last_batch_stats": (I32, [P, P, I32, P, P]),
    "bfs_batch_autotune": (I32, [P, P, I32, P, P, P]),
    "bfs_selftest_grid_barrier": (I32, [I32, I64, P]),
    "bfs_serve_config_default": (None, [P]),
    "bfs_serve_create": (I32, [P, P]),
    "bfs_serve_add_graph": (I32, [P, P, P]),
    "bfs_serve_submit": (I32, [P, I32, I32, P, P]),
    "bfs_serve_wait": (I32, [P, U64, I64, P]),
    "bfs_serve_stats_get": (I32, [P, P]),
    "bfs_serve_stats_reset": (I32, [P]),
    "bfs_serve_destroy": (I32, [P]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the built library; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def build(force: bool = False) -> str:
    return _build.build(force=force)


def _check(status: int):
    if status != BFS_OK:
        raise BfsError(status, lib().bfs_last_error().decode())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def launch_count() -> int:
    return int(lib().bfs_launch_count())


def alloc_count() -> int:
    """Device and pinned-host allocations the library has made so far."""
    return int(lib().bfs_alloc_count())


RESERVE_HOST_OUT = 1
RESERVE_NO_PARENT = 2


def default_batch_config() -> BatchConfig:
    c = BatchConfig()
    lib().bfs_batch_config_default(ctypes.byref(c))
    return c


def default_config() -> Config:
    c = Config()
    lib().bfs_config_default(ctypes.byref(c))
    return c


# ------------------------------------------------------------- graph input
def generate_edges(kind: int, scale: int, edgefactor: int, seed: int,
                   a: float = 0.57, b: float = 0.19, c: float = 0.19, device="cuda", stream=None):
    m = edgefactor << scale
    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    _check(lib().bfs_generate_edges(kind, scale, edgefactor, seed, a, b, c, _ptr(src), _ptr(dst),
                                    _stream(stream)))
    return src, dst


def build_csr(n: int, src: torch.Tensor, dst: torch.Tensor, stream=None):
    m = src.numel()
    dev = src.device
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    indices = torch.empty(max(2 * m, 1), dtype=torch.int32, device=dev)
    nnz = ctypes.c_int64(0)
    _check(lib().bfs_build_csr(n, m, _ptr(src if m else None), _ptr(dst if m else None),
                               _ptr(offsets), _ptr(indices), ctypes.byref(nnz), _stream(stream)))
    return offsets, indices[:nnz.value]


def sample_roots(offsets: torch.Tensor, n: int, seed: int, k: int, max_draws: int = 1 << 24,
                 stream=None):
    roots = torch.empty(k, dtype=torch.int32, device=offsets.device)
    got = ctypes.c_int32(0)
    _check(lib().bfs_sample_roots(_ptr(offsets), n, seed, k, max_draws, _ptr(roots),
                                  ctypes.byref(got), _stream(stream)))
    return roots[:got.value]


def rmat_graph(scale: int, edgefactor: int, seed: int, kind: int = GEN_RMAT, stream=None):
    """Generate edges and build the symmetric CSR on the GPU."""
    src, dst = generate_edges(kind, scale, edgefactor, seed, stream=stream)
    off, idx = build_csr(1 << scale, src, dst, stream=stream)
    del src, dst
    return off, idx


# --------------------------------------------------------------------- BFS
@dataclass
class RunStats:
    layers: list
    component_edges: int


class Graph:
    """A CSR graph resident on the GPU (bfs_graph)."""

    def __init__(self, offsets: torch.Tensor, indices: torch.Tensor, config: Config | None = None,
                 borrow: bool = True, validate: bool | str = False):
        """validate: True = range checks (BFS_VALIDATE); "symmetric" = also
        ascending rows and every entry's reverse (BFS_VALIDATE_SYMMETRIC)."""
        n = offsets.numel() - 1
        nnz = indices.numel()
        offsets = offsets.contiguous()
        indices = indices.contiguous()
        flags = 0
        if offsets.is_cuda:
            flags |= DEVICE_PTRS
            if borrow:
                flags |= BORROW
                self._keep = (offsets, indices)
        if validate == "symmetric":
            flags |= VALIDATE | VALIDATE_SYMMETRIC
        elif validate:
            flags |= VALIDATE
        h = ctypes.c_void_p(0)
        _check(lib().bfs_graph_create(_ptr(offsets), _ptr(indices if nnz else None), n, nnz, flags,
                                      ctypes.byref(config) if config is not None else None,
                                      ctypes.byref(h)))
        self._h = h
        self.n = n
        self.nnz = nnz
        self.config = config if config is not None else default_config()

    def set_config(self, config: Config | None):
        _check(lib().bfs_graph_set_config(self._h, ctypes.byref(config) if config else None))
        self.config = config if config is not None else default_config()

    def run(self, root: int, level: torch.Tensor | None = None, parent: torch.Tensor | None = None,
            want_parent: bool = True, stream=None):
        dev = "cuda"
        if level is None:
            level = torch.empty(self.n, dtype=torch.int32, device=dev)
        if parent is None and want_parent:
            parent = torch.empty(self.n, dtype=torch.int32, device=level.device)
        _check(lib().bfs_run(self._h, int(root), _ptr(level), _ptr(parent), _stream(stream)))
        return level, parent

    def reserve(self, host_out: bool = False, no_parent: bool = False, stream=None):
        """bfs_graph_reserve: allocate now what bfs_run would allocate on
        first use under the current configuration."""
        flags = (RESERVE_HOST_OUT if host_out else 0) | (RESERVE_NO_PARENT if no_parent else 0)
        _check(lib().bfs_graph_reserve(self._h, flags, _stream(stream)))

    def sync(self):
        """Waits for host copies left in flight by run() with config.host_async."""
        _check(lib().bfs_graph_sync(self._h))

    def stats(self) -> RunStats:
        L = ctypes.c_int32(0)
        ce = ctypes.c_int64(0)
        _check(lib().bfs_last_run_stats(self._h, None, 0, ctypes.byref(L), None))
        arr = (LayerStats * max(L.value, 1))()
        _check(lib().bfs_last_run_stats(self._h, arr, L.value, ctypes.byref(L), ctypes.byref(ce)))
        layers = [{f: getattr(arr[i], f) for f, _ in LayerStats._fields_} for i in range(L.value)]
        return RunStats(layers, ce.value)

    # ---------------------------------------------------------- batched BFS
    def batch_config(self) -> BatchConfig:
        c = BatchConfig()
        _check(lib().bfs_graph_get_batch_config(self._h, ctypes.byref(c)))
        return c

    def set_batch_config(self, config: BatchConfig | None):
        _check(lib().bfs_graph_set_batch_config(self._h, ctypes.byref(config) if config else None))

    def run_batch(self, roots, levels: torch.Tensor | None = None, stream=None):
        """Levels from every root at once: int8 [k, n] (row i = roots[i])."""
        if not isinstance(roots, torch.Tensor):
            roots = torch.tensor(list(roots), dtype=torch.int32)
        roots = roots.to(torch.int32).contiguous()
        k = roots.numel()
        if levels is None:
            levels = torch.empty((k, self.n), dtype=torch.int8, device="cuda")
        _check(lib().bfs_run_batch(self._h, _ptr(roots), k, _ptr(levels), _stream(stream)))
        return levels

    def batch_stats(self):
        L = ctypes.c_int32(0)
        pairs = ctypes.c_int64(0)
        _check(lib().bfs_last_batch_stats(self._h, None, 0, ctypes.byref(L), None))
        arr = (BatchLayerStats * max(L.value, 1))()
        _check(lib().bfs_last_batch_stats(self._h, arr, L.value, ctypes.byref(L),
                                          ctypes.byref(pairs)))
        layers = [{f: getattr(arr[i], f) for f, _ in BatchLayerStats._fields_}
                  for i in range(L.value)]
        return layers, pairs.value

    def autotune_batch(self, roots, stream=None) -> BatchConfig:
        if not isinstance(roots, torch.Tensor):
            roots = torch.tensor(list(roots), dtype=torch.int32)
        roots = roots.to(torch.int32).contiguous()
        k = roots.numel()
        scratch = torch.empty((k, self.n), dtype=torch.int8, device="cuda")
        best = BatchConfig()
        _check(lib().bfs_batch_autotune(self._h, _ptr(roots), k, _ptr(scratch), ctypes.byref(best),
                                        _stream(stream)))
        return best

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().bfs_graph_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_noalloc(offsets: torch.Tensor, indices: torch.Tensor, root: int, level: torch.Tensor,
                parent: torch.Tensor, stream=None):
    """bfs_run_noalloc: the traversal with library-resident scratch (n <= 2^20)."""
    n = offsets.numel() - 1
    _check(lib().bfs_run_noalloc(_ptr(offsets), _ptr(indices if indices.numel() else None), n,
                                 indices.numel(), int(root), _ptr(level), _ptr(parent),
                                 _stream(stream)))
    return level, parent


def default_serve_config() -> ServeConfig:
    c = ServeConfig()
    lib().bfs_serve_config_default(ctypes.byref(c))
    return c


class Server:
    """bfs_server: batches single-root queries per graph (continuous batching)."""

    def __init__(self, config: ServeConfig | None = None):
        h = ctypes.c_void_p(0)
        _check(lib().bfs_serve_create(ctypes.byref(config) if config else None, ctypes.byref(h)))
        self._h = h
        self._graphs = []

    def add_graph(self, graph: Graph) -> int:
        gid = ctypes.c_int32(0)
        _check(lib().bfs_serve_add_graph(self._h, graph._h, ctypes.byref(gid)))
        self._graphs.append(graph)
        return gid.value

    def submit(self, graph_id: int, root: int, level_out: torch.Tensor) -> int:
        t = ctypes.c_uint64(0)
        _check(lib().bfs_serve_submit(self._h, graph_id, int(root), _ptr(level_out),
                                      ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1) -> int:
        """Returns the request's own status (0 = BFS_OK)."""
        r = ctypes.c_int32(0)
        _check(lib().bfs_serve_wait(self._h, ctypes.c_uint64(ticket), timeout_us, ctypes.byref(r)))
        return r.value

    def stats(self) -> dict:
        o = ServeStats()
        _check(lib().bfs_serve_stats_get(self._h, ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in ServeStats._fields_}

    def reset_stats(self):
        _check(lib().bfs_serve_stats_reset(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().bfs_serve_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_grid_barrier(missing_blocks: int, timeout_us: int, stream=None) -> int:
    """Status of one bounded grid barrier that lacks `missing_blocks` arrivals."""
    return int(lib().bfs_selftest_grid_barrier(missing_blocks, timeout_us, _stream(stream)))
