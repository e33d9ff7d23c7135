"""Python side of the CPU oracle (test infrastructure only).

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
use this module; the CUDA library never imports it and it never imports the
CUDA library.  The walks themselves run in ppr_oracle.c (single-threaded,
plain C); this module builds that library with gcc, marshals arrays, and does
the estimator's counting (Algorithm 2, final grouping of terminated walks by
(head, tail); Sec. 2.1 estimator pi_hat(s, t) = omega'/omega) with numpy.

Result conventions:
    ends     uint32[S, R]   endpoint of walk j of source s_begin + i
    rows     (row_ptr int64[S+1], col int32[nnz], cnt uint32[nnz]) per source,
             end ids strictly ascending, counts summing to R
    topk     idx int32[S, k], cnt uint32[S, k]: count descending, ties by the
             smaller end id, padded with (-1, 0)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppr_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "libppr_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (single-threaded, no OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Graph(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("P", C.c_void_p),
                ("W", C.c_void_p), ("seg_off", C.c_void_p), ("seg_node", C.c_void_p),
                ("seg_mark_len", C.c_void_p), ("seg_cum", C.c_void_p), ("w", C.c_void_p), ("lazy", C.c_void_p),
                ("alias_thr", C.c_void_p), ("alias_idx", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("T", C.c_uint32), ("R", C.c_uint32), ("seed", C.c_uint64), ("s_begin", C.c_int64),
                ("s_end", C.c_int64), ("ctr_base", C.c_int64), ("tag", C.c_uint32),
                ("dangling_mode", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.ppr_oracle_philox4x32.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.ppr_oracle_philox4x32_run.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
        L.ppr_oracle_philox4x64.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.ppr_oracle_mulhi64.argtypes = [C.c_uint64, C.c_uint64]
        L.ppr_oracle_mulhi64.restype = C.c_uint64
        L.ppr_oracle_threshold.argtypes = [C.c_double]
        L.ppr_oracle_threshold.restype = C.c_uint32
        L.ppr_oracle_row_prefix.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.ppr_oracle_pick.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_uint64]
        L.ppr_oracle_pick.restype = C.c_int64
        L.ppr_oracle_segment_table.argtypes = [C.c_void_p] * 4 + [C.c_uint32, C.c_uint32] + [C.c_void_p] * 3
        L.ppr_oracle_segment_table.restype = C.c_int
        L.ppr_oracle_segments.argtypes = ([C.c_int64] + [C.c_void_p] * 4 + [C.c_uint32] + [C.c_void_p] * 5
                                          + [C.c_int64])
        L.ppr_oracle_segments.restype = C.c_int64
        L.ppr_oracle_walks.argtypes = [C.POINTER(_Graph), C.POINTER(_Params), C.c_void_p, C.c_void_p]
        L.ppr_oracle_walks.restype = C.c_int
        L.ppr_oracle_lazy_new.argtypes = [C.c_int64]
        L.ppr_oracle_lazy_new.restype = C.c_void_p
        L.ppr_oracle_lazy_free.argtypes = [C.c_void_p]
        L.ppr_oracle_alias_table.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        L.ppr_oracle_alias_table.restype = C.c_int
        L.ppr_oracle_alias_pick.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_uint64]
        L.ppr_oracle_alias_pick.restype = C.c_int64
        L.ppr_oracle_alias_tables.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.ppr_oracle_alias_tables.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# --- primitive entry points (used by the pins) ------------------------------

def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ppr_oracle_philox4x32(_p(c), _p(k), rounds, _p(out))
    return out


def philox4x32_run(ctr, key, count: int) -> np.ndarray:
    """Philox4x32-10 words uint32[count, 4] for counters (ctr[0] + i, ctr[1], ctr[2], ctr[3])."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros((count, 4), dtype=np.uint32)
    lib().ppr_oracle_philox4x32_run(_p(c), _p(k), count, _p(out))
    return out


def philox4x64(ctr, key, rounds: int = 10) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().ppr_oracle_philox4x64(_p(c), _p(k), rounds, _p(out))
    return out


def mulhi64(a: int, b: int) -> int:
    return int(lib().ppr_oracle_mulhi64(a, b))


def threshold(alpha: float) -> int:
    return int(lib().ppr_oracle_threshold(alpha))


def pick(P: np.ndarray, lo: int, hi: int, x: int) -> int:
    P = np.ascontiguousarray(P, dtype=np.uint64)
    return int(lib().ppr_oracle_pick(_p(P), lo, hi, x))


# --- graphs and walks --------------------------------------------------------

@dataclass
class OracleGraph:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    P: np.ndarray
    W: np.ndarray
    seg_T: int = 0
    seg_off: np.ndarray | None = None
    seg_node: np.ndarray | None = None
    seg_mark_len: np.ndarray | None = None
    seg_weight: np.ndarray | None = None
    seg_cum: np.ndarray | None = None
    lazy: object = None  # on-demand segment tables (large graphs)
    alias_thr: np.ndarray | None = None
    alias_idx: np.ndarray | None = None

    def __del__(self):
        if self.lazy:
            lib().ppr_oracle_lazy_free(self.lazy)
            self.lazy = None


def prepare(n: int, row_ptr, col, w) -> OracleGraph:
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    m = int(row_ptr[-1])
    P = np.zeros(max(m, 1), dtype=np.uint64)
    W = np.zeros(max(n, 1), dtype=np.uint64)
    lib().ppr_oracle_row_prefix(n, _p(row_ptr), _p(w), _p(P), _p(W))
    return OracleGraph(n, row_ptr, col, w, P, W)


def segment_table(g: OracleGraph, T: int, v: int):
    """Outcome table of node v: list of (node, active, len, weight), canonical order; [] if ineligible."""
    node = np.zeros(64, dtype=np.uint32)
    ml = np.zeros(64, dtype=np.uint32)
    wt = np.zeros(64, dtype=np.uint64)
    k = lib().ppr_oracle_segment_table(_p(g.row_ptr), _p(g.col), _p(g.w), _p(g.W), T, v,
                                       _p(node), _p(ml), _p(wt))
    return [(int(node[i]), int(ml[i]) >> 8, int(ml[i]) & 0xFF, int(wt[i])) for i in range(k)]


def build_segments(g: OracleGraph, T: int) -> OracleGraph:
    cap = 64 * g.n + 1
    seg_off = np.zeros(g.n + 1, dtype=np.int64)
    node = np.zeros(cap, dtype=np.uint32)
    ml = np.zeros(cap, dtype=np.uint32)
    wt = np.zeros(cap, dtype=np.uint64)
    cum = np.zeros(cap, dtype=np.uint64)
    total = lib().ppr_oracle_segments(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(g.W), T, _p(seg_off),
                                      _p(node), _p(ml), _p(wt), _p(cum), cap)
    if total < 0:
        raise RuntimeError("segment table capacity exceeded")
    g.seg_T = T
    g.seg_off, g.seg_node, g.seg_mark_len = seg_off, node[:total].copy(), ml[:total].copy()
    g.seg_weight, g.seg_cum = wt[:total].copy(), cum[:total].copy()
    return g


def alias_table(weights):
    """Integer alias table of one row: (thr uint64[d], alias int64[d]) as Algorithm 1."""
    w = np.ascontiguousarray(weights, dtype=np.uint32)
    thr = np.zeros(len(w), dtype=np.uint64)
    ali = np.zeros(len(w), dtype=np.int64)
    if lib().ppr_oracle_alias_table(_p(w), len(w), _p(thr), _p(ali)) != 0:
        raise MemoryError
    return thr, ali


def alias_pick(thr, ali, W: int, r: int) -> int:
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    ali = np.ascontiguousarray(ali, dtype=np.int64)
    return int(lib().ppr_oracle_alias_pick(_p(thr), _p(ali), len(thr), W, r))


def build_alias(g: OracleGraph) -> OracleGraph:
    m = int(g.row_ptr[-1])
    g.alias_thr = np.zeros(max(m, 1), dtype=np.uint64)
    g.alias_idx = np.zeros(max(m, 1), dtype=np.int64)
    if lib().ppr_oracle_alias_tables(g.n, _p(g.row_ptr), _p(g.w), _p(g.alias_thr), _p(g.alias_idx)) != 0:
        raise MemoryError
    return g


def walks(g: OracleGraph, alpha: float, R: int, seed: int, s_begin: int = 0, s_end: int | None = None,
          tag: int = 0, dangling: int = 0, segments: bool = False, lazy_segments: bool = False,
          sampler: int = 0):
    """Endpoints uint32[S, R] and the number of draws consumed.  With
    lazy_segments, segment tables are built only for the nodes the walks
    visit (same tables; for sampled runs on large graphs)."""
    if s_end is None:
        s_end = g.n
    T = threshold(alpha)
    if T == 0:
        raise ValueError("alpha must satisfy floor(alpha * 2^32) >= 1 and alpha < 1")
    if sampler == 1 and g.alias_thr is None:
        build_alias(g)
    use_lazy = segments and lazy_segments
    if use_lazy and not g.lazy:
        g.lazy = lib().ppr_oracle_lazy_new(g.n)
    if segments and not use_lazy and (g.seg_off is None or g.seg_T != T):
        build_segments(g, T)
    S = s_end - s_begin
    ends = np.zeros((S, R), dtype=np.uint32)
    steps = np.zeros(1, dtype=np.uint64)
    flat = segments and not use_lazy
    gr = _Graph(g.n, g.row_ptr.ctypes.data, g.col.ctypes.data, g.P.ctypes.data, g.W.ctypes.data,
                g.seg_off.ctypes.data if flat else None,
                g.seg_node.ctypes.data if flat else None,
                g.seg_mark_len.ctypes.data if flat else None,
                g.seg_cum.ctypes.data if flat else None,
                g.w.ctypes.data, g.lazy if use_lazy else None,
                g.alias_thr.ctypes.data if sampler == 1 else None,
                g.alias_idx.ctypes.data if sampler == 1 else None)
    pr = _Params(T, R, seed, s_begin, s_end, 0, tag, dangling)
    if S > 0 and R > 0:
        rc = lib().ppr_oracle_walks(C.byref(gr), C.byref(pr), _p(ends), _p(steps))
        if rc != 0:
            raise RuntimeError(f"oracle walks failed: {rc}")
    return ends, int(steps[0])


def rows(ends: np.ndarray, n: int):
    """Per-source sparse count rows (end ascending) from the endpoint matrix."""
    S, R = ends.shape
    key = (np.repeat(np.arange(S, dtype=np.int64), R) * n) + ends.reshape(-1).astype(np.int64)
    uk, cnt = np.unique(key, return_counts=True)
    src = uk // n
    col = (uk - src * n).astype(np.int32)
    row_ptr = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=S), out=row_ptr[1:])
    return row_ptr, col, cnt.astype(np.uint32)


def topk(row_ptr: np.ndarray, col: np.ndarray, cnt: np.ndarray, k: int):
    """Top-k per row: count descending, ties by the smaller end id, padded with (-1, 0)."""
    S = len(row_ptr) - 1
    src = np.repeat(np.arange(S, dtype=np.int64), np.diff(row_ptr))
    order = np.lexsort((col, -cnt.astype(np.int64), src))
    rank = np.arange(len(order), dtype=np.int64) - row_ptr[src[order]]
    sel = order[rank < k]
    r = rank[rank < k]
    idx = np.full((S, k), -1, dtype=np.int32)
    cc = np.zeros((S, k), dtype=np.uint32)
    idx[src[sel], r] = col[sel]
    cc[src[sel], r] = cnt[sel]
    return idx, cc


def dense(ends: np.ndarray, n: int) -> np.ndarray:
    """Dense S x n endpoint counts."""
    S, R = ends.shape
    out = np.zeros((S, n), dtype=np.uint32)
    np.add.at(out, (np.repeat(np.arange(S), R), ends.reshape(-1).astype(np.int64)), 1)
    return out
