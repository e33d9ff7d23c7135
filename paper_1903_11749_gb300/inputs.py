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

import math
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


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 2020, dangling_frac: float = 0.05, zipf_s: float = 1.5, wmax: int = 1000,
               hub_degree: int = 0) -> Graph:
    """R-MAT graph with 2^scale nodes and edge_factor * 2^scale directed edges.

    Generated source-major: the out-degree vector is one multinomial draw over
    the R-MAT source marginal (each source bit is 1 with probability c + d),
    then each edge's destination bits are drawn conditionally on the source
    bit at the same level (P(dst bit = 1) = b / (a + b) when the source bit is
    0 and d / (c + d) when it is 1; probabilities quantised to 1/65536).  This
    gives the R-MAT joint law without a global sort.

    Plain R-MAT leaves roughly half the nodes with no out-edge; to match a
    ~5 % dangling fraction, a seeded random dangling_frac * n of the
    zero-out-degree nodes stay dangling and every other one receives a single
    out-edge to a uniform target.  With hub_degree > 0, that many uniformly
    chosen edges of other sources are re-sourced to node 0 (m unchanged).
    Weights are Zipf(zipf_s) on {1..wmax}.
    """
    n = 1 << scale
    m0 = edge_factor * n
    d = 1.0 - a - b - c
    rng = np.random.Generator(np.random.PCG64(seed))

    # Out-degree per source: P(src) = prod over levels of (a+b) or (c+d).
    pop = np.zeros(n, dtype=np.int64)
    ids = np.arange(n, dtype=np.int64)
    for lvl in range(scale):
        pop += (ids >> lvl) & 1
    p_src = np.exp((scale - pop) * math.log(a + b) + pop * math.log(c + d))
    p_src /= p_src.sum()
    deg = rng.multinomial(m0, p_src).astype(np.int64)
    del pop, p_src

    src = np.repeat(ids.astype(np.int32), deg)
    del ids
    thr0 = np.uint16(min(65535, int(round(b / (a + b) * 65536))))
    thr1 = np.uint16(min(65535, int(round(d / (c + d) * 65536))))
    dst = np.zeros(m0, dtype=np.int32)
    for lvl in range(scale):
        u = rng.integers(0, 65536, size=m0, dtype=np.uint16)
        sbit = ((src >> lvl) & 1).astype(bool)
        thr = np.where(sbit, thr1, thr0)
        dst |= (u < thr).astype(np.int32) << lvl
        del u, sbit, thr
    del src

    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])

    if hub_degree > 0:
        # Re-source hub_degree uniformly chosen edges (not already node 0's) to node 0.
        lo = int(row_ptr[1])
        pick = lo + rng.choice(m0 - lo, size=hub_degree, replace=False)
        pick.sort()
        keep = np.ones(m0, dtype=bool)
        keep[pick] = False
        moved = dst[pick]
        # Count removals per source row.
        src_of_pick = np.searchsorted(row_ptr, pick, side="right") - 1
        removed = np.bincount(src_of_pick, minlength=n).astype(np.int64)
        deg = deg - removed
        deg[0] += hub_degree
        dst = np.concatenate([dst[: lo], moved, dst[lo:][keep[lo:]]])
        row_ptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(deg, out=row_ptr[1:])
        del keep, moved, pick, src_of_pick

    # Dangling repair: keep a random dangling_frac * n of the empty rows empty.
    empty = np.flatnonzero(deg == 0)
    n_keep = min(len(empty), int(round(dangling_frac * n)))
    keep_empty = rng.choice(len(empty), size=n_keep, replace=False)
    fill_mask = np.ones(len(empty), dtype=bool)
    fill_mask[keep_empty] = False
    fill = empty[fill_mask]
    if len(fill):
        extra_dst = rng.integers(0, n, size=len(fill), dtype=np.int64).astype(np.int32)
        new_deg = deg.copy()
        new_deg[fill] = 1
        new_row_ptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(new_deg, out=new_row_ptr[1:])
        new_dst = np.empty(int(new_row_ptr[-1]), dtype=np.int32)
        # Old edges keep their order; each filled row gets its single new edge.
        old_pos = np.repeat(new_row_ptr[:-1] - row_ptr[:-1], deg) + np.arange(int(row_ptr[-1]), dtype=np.int64)
        new_dst[old_pos] = dst
        new_dst[new_row_ptr[fill]] = extra_dst
        dst, deg, row_ptr = new_dst, new_deg, new_row_ptr
        del old_pos, new_dst
    w = zipf_weights(rng, int(row_ptr[-1]), zipf_s, wmax)
    meta = {"seed": seed, "scale": scale, "m_rmat": m0, "hub_degree": hub_degree,
            "dangling": int((deg == 0).sum()), "max_degree": int(deg.max())}
    return Graph(n, row_ptr, dst, w, name=f"rmat_s{scale}", meta=meta)


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


def workload_graph(name: str):
    if name == "er1k":
        return er_graph(1000, 10_000, 1, 10, seed=12345)
    if name == "rmat20":
        return rmat_graph(20, 16, seed=2020)
    if name == "rmat24":
        return rmat_graph(24, 16, seed=2424, hub_degree=1_200_000)
    raise KeyError(name)
