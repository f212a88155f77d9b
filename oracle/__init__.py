"""CPU oracle for the hybrid BFS library (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU library never imports, links or
calls it. The arithmetic lives in ``oracle.c`` (plain single-threaded C, each
function citing the passage of the paper it restates); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

POLICY_EDGE = 0      # e_f > e_u / alpha  /  |in| < n / beta
POLICY_VERTEX = 1    # f = n_u >> 10, g = n >> 6 (read off Table 2)
POLICY_FORCED = 2

RMAT = 0
ER = 1


def build() -> str:
    """Compile oracle.c into _build/liboracle.so (portable flags: no -march)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "orc_sm64": (u64, [u64, u64]),
            "orc_relabel": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_int, u64]),
            "orc_gen_edges": (None, [ctypes.c_int, ctypes.c_int, u64, dbl, dbl, dbl,
                                     i64, i64, P, P]),
            "orc_build_csr": (i64, [i64, i64, P, P, P, P]),
            "orc_sample_roots": (i32, [P, i64, u64, i32, i64, P]),
            "orc_bfs": (i32, [P, P, i64, i32, P, P]),
            "orc_policy_decide": (i32, [i32, i32, i64, i64, i64, i64, i64, dbl, dbl]),
            "orc_hybrid_bfs": (i32, [P, P, i64, i32, i32, dbl, dbl, P, P, P, P, P, i32, P]),
            "orc_hub": (None, [P, P, i64, P]),
            "orc_check_levels": (i64, [P, P, i64, i32, P]),
            "orc_check_parents": (i64, [P, P, i64, i32, P, P]),
            "orc_min_parent": (None, [P, P, i64, i32, P, P]),
            "orc_component_edges": (i64, [P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _csr(offsets, indices):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(indices, dtype=np.int32)
    if idx.size == 0:
        idx = np.zeros(1, dtype=np.int32)
    return off, idx


# --------------------------------------------------------------------------
def sm64(seed: int, i: int) -> int:
    """Output i (0-based) of SplitMix64 seeded with `seed`."""
    return int(_load().orc_sm64(seed & (2**64 - 1), i & (2**64 - 1)))


def relabel(x: int, scale: int, seed: int) -> int:
    return int(_load().orc_relabel(x, scale, seed))


def gen_edges(kind: int, scale: int, edgefactor: int, seed: int,
              a: float = 0.57, b: float = 0.19, c: float = 0.19,
              first: int = 0, count: int | None = None, out=None):
    """Edge list of the R-MAT (kind=RMAT) or uniform (kind=ER) generator.
    `out` = (src, dst): contiguous int32 arrays of at least `count` entries
    to fill instead of new ones (lets a caller fill chunks of one list)."""
    m = edgefactor << scale
    if count is None:
        count = m - first
    if out is None:
        src = np.empty(max(count, 1), dtype=np.int32)
        dst = np.empty(max(count, 1), dtype=np.int32)
    else:
        src, dst = out
        if not (src.dtype == dst.dtype == np.int32 and src.flags.c_contiguous
                and dst.flags.c_contiguous and min(src.size, dst.size) >= count):
            raise ValueError("out: two contiguous int32 arrays of >= count entries")
    if count > 0:
        _load().orc_gen_edges(kind, scale, seed, a, b, c, first, count, _p(src), _p(dst))
    return src[:count], dst[:count]


def build_csr(n: int, src, dst):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = src.size
    off = np.empty(n + 1, dtype=np.int64)
    idx = np.empty(max(2 * m, 1), dtype=np.int32)
    s = src if m else np.zeros(1, np.int32)
    d = dst if m else np.zeros(1, np.int32)
    nnz = _load().orc_build_csr(n, m, _p(s), _p(d), _p(off), _p(idx))
    if nnz < 0:
        raise ValueError("edge endpoint out of range or out of memory")
    return off, idx[:nnz].copy()


def sample_roots(offsets, n: int, seed: int, k: int, max_draws: int = 1 << 24):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    roots = np.empty(max(k, 1), dtype=np.int32)
    got = _load().orc_sample_roots(_p(off), n, seed, k, max_draws, _p(roots))
    return roots[:got].copy()


def bfs(offsets, indices, root: int):
    off, idx = _csr(offsets, indices)
    n = off.size - 1
    level = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    depth = _load().orc_bfs(_p(off), _p(idx), n, root, _p(level), _p(parent))
    if depth < 0:
        raise ValueError("bad root")
    return level, parent


def policy_decide(policy: int, cur_bottom_up: bool, n: int, n_f: int, m_f: int,
                  n_u: int, m_u: int, alpha: float = 14.0, beta: float = 24.0) -> int:
    return int(_load().orc_policy_decide(policy, int(cur_bottom_up), n, n_f, m_f,
                                         n_u, m_u, alpha, beta))


def hybrid_bfs(offsets, indices, root: int, policy: int = POLICY_EDGE,
               alpha: float = 14.0, beta: float = 24.0, forced=None,
               max_levels: int | None = None, hint=None):
    """Alg. 3 run sequentially. Returns level, parent, dirs, trace[L, 6].
    ``hint`` (int32 [n] or None): a neighbour the bottom-up step tests first."""
    off, idx = _csr(offsets, indices)
    n = off.size - 1
    if max_levels is None:
        max_levels = n + 1
    f = np.zeros(max_levels, dtype=np.int32)
    if forced is not None:
        forced = list(forced)
        for d in range(max_levels):
            f[d] = forced[min(d, len(forced) - 1)] if forced else 0
    level = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    dirs = np.empty(max_levels, dtype=np.int32)
    trace = np.empty(6 * max_levels, dtype=np.int64)
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, dtype=np.int32)
        if h.size != n:
            raise ValueError("hint must have one entry per vertex")
    L = _load().orc_hybrid_bfs(_p(off), _p(idx), n, root, policy, alpha, beta, _p(f),
                               _p(level), _p(parent), _p(dirs), _p(trace), max_levels,
                               None if h is None else _p(h))
    if L < 0:
        raise ValueError("bad root or too many layers")
    return level, parent, dirs[:L].copy(), trace[:6 * L].reshape(L, 6).copy()


def hub(offsets, indices):
    """Neighbour of largest degree per vertex (smallest id on ties; -1 if none)."""
    off, idx = _csr(offsets, indices)
    n = off.size - 1
    out = np.empty(n, dtype=np.int32)
    _load().orc_hub(_p(off), _p(idx), n, _p(out))
    return out


def check_levels(offsets, indices, root: int, level) -> int:
    off, idx = _csr(offsets, indices)
    lv = np.ascontiguousarray(level, dtype=np.int32)
    return int(_load().orc_check_levels(_p(off), _p(idx), off.size - 1, root, _p(lv)))


def check_parents(offsets, indices, root: int, level, parent) -> int:
    off, idx = _csr(offsets, indices)
    lv = np.ascontiguousarray(level, dtype=np.int32)
    pa = np.ascontiguousarray(parent, dtype=np.int32)
    return int(_load().orc_check_parents(_p(off), _p(idx), off.size - 1, root,
                                         _p(lv), _p(pa)))


def min_parent(offsets, indices, root: int, level):
    off, idx = _csr(offsets, indices)
    n = off.size - 1
    lv = np.ascontiguousarray(level, dtype=np.int32)
    out = np.empty(n, dtype=np.int32)
    _load().orc_min_parent(_p(off), _p(idx), n, root, _p(lv), _p(out))
    return out


def component_edges(offsets, level) -> int:
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    lv = np.ascontiguousarray(level, dtype=np.int32)
    return int(_load().orc_component_edges(_p(off), off.size - 1, _p(lv)))


def msbfs_levels(offsets, indices, roots):
    """int8 level rows, one single-source BFS per root (cast from int32).

    Raises ValueError when a level does not fit in int8 (depth > 127)."""
    off, idx = _csr(offsets, indices)
    n = off.size - 1
    out = np.empty((len(roots), n), dtype=np.int8)
    for i, r in enumerate(roots):
        lv, _ = bfs(off, idx, int(r))
        if lv.max(initial=0) > 127:
            raise ValueError("BFS depth exceeds 127")
        out[i] = lv.astype(np.int8)
    return out
