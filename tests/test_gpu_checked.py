"""The checked build (-DPPR_CHECKED): every node index and row extent a walk
step reads is tested against its array, a bad one recorded as a flag (no
trap) and reported by ppr_wait.  On valid graphs of every layout (narrow,
wide, segment tables, alias tables, batched) the checked library reports no
flag and gives the oracle's counts.  It runs in a child process so that it
loads the checked library instead of the one this process has loaded."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/oracle"); sys.path.insert(0, sys.argv[1] + "/tests")
from paper_1903_11749_gb300 import ppr, inputs as I
import oracle as O
assert ppr.LIB_PATH.endswith("libppr_checked.so"), ppr.LIB_PATH
ctx = ppr.Context(0)

def same(G, g, **kw):
    og = O.prepare(g.n, g.row_ptr, g.col, g.w)
    s_end = kw.pop("src_end", g.n)
    lazy = kw.get("segments", False)
    ends, steps = O.walks(og, kw["alpha"], kw["R"], kw["seed"], 0, s_end, kw.get("tag", 0), kw.get("dangling", 0),
                          kw.get("segments", False), sampler=kw.get("sampler", 0))
    rp, col, cnt = O.rows(ends, g.n)
    res = G.run(src_end=s_end, **kw)
    a = res.sparse_rows()
    assert np.array_equal(a[0], rp) and np.array_equal(a[1], col) and np.array_equal(a[2], cnt), kw
    assert res.info().steps == steps

g = I.random_small_graph(500, 4000, seed=3, wmax=20, dangling=9)
G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
for kernel in (0, 1):
    for dangling in (0, 1):
        same(G, g, alpha=0.2, R=40, seed=2, kernel=kernel, dangling=dangling)
        same(G, g, alpha=0.2, R=40, seed=2, kernel=kernel, dangling=dangling, sampler=1)
        same(G, g, alpha=0.3, R=40, seed=2, kernel=kernel, dangling=dangling, segments=True)
rng = np.random.Generator(np.random.PCG64(1))
edges = [(0, int(t), int(w)) for t, w in zip(rng.integers(0, 3000, 70001), rng.integers(1, 900, 70001))]
edges += [(u, int(rng.integers(0, 3000)), int(rng.integers(1, 9))) for u in range(1, 3000)]
h = I.from_edges(3000, edges)
H = ctx.load_graph(h.n, h.row_ptr, h.col, h.w)
same(H, h, alpha=0.2, R=30, seed=4, src_end=200)
same(H, h, alpha=0.2, R=30, seed=4, src_end=200, sampler=1)
big = 2**32 - 5
wg = I.from_edges(4, [(0, 1, big), (0, 2, big), (1, 0, 1), (2, 3, 7), (3, 0, big), (3, 1, 2)])
W = ctx.load_graph(wg.n, wg.row_ptr, wg.col, wg.w)
assert W.info().wide
same(W, wg, alpha=0.25, R=200, seed=5)
inst = I.chung_lu_instances(count=6, nmin=50, nmax=400, seed=3)
B = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
for sampler in (0, 1):
    res = B.run(alpha=0.15, R=30, seed=1, sampler=sampler)
    rp, col, cnt = res.sparse_rows()
    for gi in range(inst.count):
        sub = inst.instance(gi)
        og = O.prepare(sub.n, sub.row_ptr, sub.col, sub.w)
        e, _ = O.walks(og, 0.15, 30, 1, tag=gi, sampler=sampler)
        orp, ocol, ocnt = O.rows(e, sub.n)
        a, b = int(inst.node_off[gi]), int(inst.node_off[gi + 1])
        assert np.array_equal(col[rp[a]:rp[b]], ocol) and np.array_equal(cnt[rp[a]:rp[b]], ocnt)
print("checked build: no flag, counts equal the oracle")
"""


def test_checked_build_matches_oracle_without_flags(oracle):
    from paper_1903_11749_gb300 import build as B
    lib = B.build(checked=True)
    env = dict(os.environ, PPR_LIBRARY_PATH=lib)
    res = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "no flag" in res.stdout
