"""Seeded synthetic graph generators.

These build the weighted CSR inputs that both the CUDA path and the CPU oracle
consume.  The module holds none of the method's arithmetic (no prefix sums, no
draws, no walks): it only fixes a graph, deterministically, from a seed.

The paper evaluates on SNAP graphs (Table 2) that are not available here; the
generators below stand in for their shape: most nodes with a small out-degree,
a few very large hubs, strictly positive edge weights (Sec. 2.1 requires
w(e) > 0; here weights are integers >= 1).

CSR convention (shared by every generator):
    row_ptr : int64[n + 1], row_ptr[0] == 0, non-decreasing, row_ptr[n] == m
    col     : int32[m], each in [0, n)
    w       : uint32[m], each >= 1
Multi-edges and self-loops are kept as separate entries.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _csr_from_pairs(n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray):
    """Group (src, dst, w) triples by source with a stable counting order."""
    order = np.argsort(src, kind="stable")
    counts = np.bincount(src, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, dst[order].astype(np.int32), w[order].astype(np.uint32)


def zipf_weights(rng: np.random.Generator, size: int, s: float = 1.5, wmax: int = 1000) -> np.ndarray:
    """Integer weights with P(k) proportional to k^-s on {1..wmax}, drawn by inverse CDF."""
    k = np.arange(1, wmax + 1, dtype=np.float64)
    pmf = k ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = rng.random(size)
    idx = np.searchsorted(cdf, u, side="right")
    np.minimum(idx, wmax - 1, out=idx)
    return (idx + 1).astype(np.uint32)


def er_graph(n: int = 1000, m: int = 10_000, wlo: int = 1, whi: int = 10, seed: int = 12345) -> Graph:
    """Directed Erdos-Renyi multigraph: m uniform (src, dst) pairs, weights U[wlo, whi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    src = rng.integers(0, n, size=m, dtype=np.int64)
    dst = rng.integers(0, n, size=m, dtype=np.int64)
    w = rng.integers(wlo, whi + 1, size=m, dtype=np.int64)
    row_ptr, col, ww = _csr_from_pairs(n, src, dst, w)
    return Graph(n, row_ptr, col, ww, name=f"er_n{n}_m{m}", meta={"seed": seed})


_GEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gen")
_gen_lib = None


def _gen():
    """The C R-MAT generator (built with gcc on first use)."""
    global _gen_lib
    if _gen_lib is None:
        src = os.path.join(_GEN_DIR, "rmat_gen.c")
        out_dir = os.path.join(_GEN_DIR, "_build")
        lib = os.path.join(out_dir, "librmat_gen.so")
        os.makedirs(out_dir, exist_ok=True)
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, src, "-lm"])
            os.replace(tmp, lib)
        L = ctypes.CDLL(lib)
        L.rmat_begin.restype = ctypes.c_void_p
        L.rmat_begin.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_uint64, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
        L.rmat_edges.restype = ctypes.c_int64
        L.rmat_edges.argtypes = [ctypes.c_void_p]
        L.rmat_hub.restype = ctypes.c_int64
        L.rmat_hub.argtypes = [ctypes.c_void_p]
        L.rmat_finish.restype = ctypes.c_int
        L.rmat_finish.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                  ctypes.c_int]
        _gen_lib = L
    return _gen_lib


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 2020, dangling_frac: float = 0.05, zipf_s: float = 1.5, wmax: int = 1000,
               hub_degree: int = 0, threads: int | None = None) -> Graph:
    """R-MAT graph with 2^scale nodes and edge_factor * 2^scale directed edges
    (gen/rmat_gen.c; every random choice is a counter-based hash, so the graph
    does not depend on the thread count).

    Source-major: the out-degrees come from the R-MAT source marginal (each
    source bit is 1 with probability c + d); each edge's destination bits are
    drawn conditionally on the source bit at the same level (probability
    b / (a + b) when it is 0, d / (c + d) when it is 1).  Plain R-MAT leaves
    about half the nodes without out-edges; to match a ~dangling_frac share of
    dangling nodes, an empty row stays empty with probability
    dangling_frac * n / #empty and every other empty row gets one edge to a
    uniform target.  With hub_degree > 0, every edge outside row 0 moves to
    row 0 with probability hub_degree / (m - deg(0)), planting a hub of about
    that out-degree.  Weights are Zipf(zipf_s) on {1..wmax}.
    """
    n = 1 << scale
    L = _gen()
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    threads = threads or min(32, os.cpu_count() or 1)
    h = L.rmat_begin(scale, edge_factor, a, b, c, seed, dangling_frac, hub_degree, threads, row_ptr.ctypes.data)
    if not h:
        raise MemoryError("rmat generator: allocation failed")
    m = int(L.rmat_edges(h))
    hub = int(L.rmat_hub(h))
    col = np.empty(m, dtype=np.int32)
    w = np.empty(m, dtype=np.uint32)
    L.rmat_finish(h, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data, zipf_s, wmax)
    deg = np.diff(row_ptr)
    meta = {"seed": seed, "scale": scale, "m_rmat": edge_factor * n, "hub_moved": hub,
            "dangling": int((deg == 0).sum()), "max_degree": int(deg.max())}
    return Graph(n, row_ptr, col, w, name=f"rmat_s{scale}", meta=meta)


def chung_lu_graph(n: int, avg_deg: float = 12.0, exponent: float = 2.3, wlo: int = 1, whi: int = 100,
                   rng: np.random.Generator | None = None, seed: int = 7) -> Graph:
    """Directed Chung-Lu graph: node weights proportional to i^(-1/(exponent-1)),
    round(avg_deg * n) edges whose source and destination are both drawn
    proportionally to those weights; edge weights U[wlo, whi]."""
    if rng is None:
        rng = np.random.Generator(np.random.PCG64(seed))
    i = np.arange(1, n + 1, dtype=np.float64)
    pw = i ** (-1.0 / (exponent - 1.0))
    pw /= pw.sum()
    m = int(round(avg_deg * n))
    deg = rng.multinomial(m, pw).astype(np.int64)
    cdf = np.cumsum(pw)
    cdf /= cdf[-1]
    dst = np.searchsorted(cdf, rng.random(m), side="right")
    np.minimum(dst, n - 1, out=dst)
    w = rng.integers(wlo, whi + 1, size=m, dtype=np.int64).astype(np.uint32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    return Graph(n, row_ptr, dst.astype(np.int32), w, name=f"chunglu_n{n}")


@dataclass
class Instances:
    """Many independent graphs stored block-diagonally: instance g owns global
    nodes [node_off[g], node_off[g+1]); col holds instance-local ids."""
    node_off: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray

    @property
    def count(self) -> int:
        return len(self.node_off) - 1

    def instance(self, g: int) -> Graph:
        a, b = int(self.node_off[g]), int(self.node_off[g + 1])
        rp = self.row_ptr[a: b + 1] - self.row_ptr[a]
        e0, e1 = int(self.row_ptr[a]), int(self.row_ptr[b])
        return Graph(b - a, rp.astype(np.int64), self.col[e0:e1].copy(), self.w[e0:e1].copy(),
                     name=f"instance{g}")


def chung_lu_instances(count: int = 2048, nmin: int = 100, nmax: int = 50_000, avg_deg: float = 12.0,
                       exponent: float = 2.3, wlo: int = 1, whi: int = 100, seed: int = 4242) -> Instances:
    """count independent Chung-Lu graphs, n drawn as floor(exp(U(ln nmin, ln nmax)))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(np.int64)
    node_off = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(ns, out=node_off[1:])
    rps, cols, ws = [], [], []
    edge_base = 0
    for g in range(count):
        gr = chung_lu_graph(int(ns[g]), avg_deg, exponent, wlo, whi, rng=rng)
        rps.append(gr.row_ptr[:-1] + edge_base)
        cols.append(gr.col)
        ws.append(gr.w)
        edge_base += gr.m
    row_ptr = np.concatenate(rps + [np.array([edge_base], dtype=np.int64)])
    return Instances(node_off, row_ptr, np.concatenate(cols), np.concatenate(ws))


def random_small_graph(n: int, m: int, seed: int, wmax: int = 10, dangling: int = 0) -> Graph:
    """Tiny random multigraph for exhaustive tests; the last `dangling` nodes get no out-edge."""
    rng = np.random.Generator(np.random.PCG64(seed))
    live = n - dangling
    src = rng.integers(0, live, size=m, dtype=np.int64)
    dst = rng.integers(0, n, size=m, dtype=np.int64)
    w = rng.integers(1, wmax + 1, size=m, dtype=np.int64)
    row_ptr, col, ww = _csr_from_pairs(n, src, dst, w)
    return Graph(n, row_ptr, col, ww, name=f"small_n{n}_m{m}_s{seed}")


def from_edges(n: int, edges) -> Graph:
    """CSR from an explicit list of (src, dst, weight) triples, kept in the given order per source."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 3)
    row_ptr, col, w = _csr_from_pairs(n, e[:, 0], e[:, 1], e[:, 2])
    return Graph(n, row_ptr, col, w)


# Named workloads.  Each returns the graph plus the run parameters.
WORKLOADS = {
    "er1k": dict(alpha=0.15, R=1000, seed=1, topk=32, dense=True),
    "rmat20": dict(alpha=0.2, R=100, seed=1, topk=32),
    "rmat24": dict(alpha=0.15, R=50, seed=1, topk=64, segments=True),
    "chunglu2048": dict(alpha=0.15, R=200, seed=1, topk=32),
}


def _make_workload_graph(name: str) -> Graph:
    if name == "er1k":
        return er_graph(1000, 10_000, 1, 10, seed=12345)
    if name == "rmat20":
        return rmat_graph(20, 16, seed=2020)
    if name == "rmat24":
        return rmat_graph(24, 16, seed=2424, hub_degree=1_200_000)
    raise KeyError(name)


def workload_graph(name: str) -> Graph:
    """The named workload's graph.  With PPR_GRAPH_CACHE set to a directory,
    a generated graph is saved there (raw .npy arrays) and later calls load it
    instead of generating it again; the arrays are the generator's, unchanged."""
    cache = os.environ.get("PPR_GRAPH_CACHE")
    if not cache:
        return _make_workload_graph(name)
    d = os.path.join(cache, name)
    parts = ("row_ptr", "col", "w")
    if all(os.path.exists(os.path.join(d, p + ".npy")) for p in parts):
        a = [np.load(os.path.join(d, p + ".npy")) for p in parts]
        return Graph(len(a[0]) - 1, a[0], a[1], a[2], name=name, meta={"cached": d})
    g = _make_workload_graph(name)
    os.makedirs(d, exist_ok=True)
    for p_, arr in zip(parts, (g.row_ptr, g.col, g.w)):
        tmp = os.path.join(d, f"{p_}.tmp{os.getpid()}.npy")
        np.save(tmp, arr)
        os.replace(tmp, os.path.join(d, p_ + ".npy"))
    return g
