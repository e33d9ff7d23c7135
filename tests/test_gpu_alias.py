"""The alias sampler (integer Algorithm 1) on the GPU against the oracle's
alias mode, element by element.

The alias tables are built on the device (one thread per row, the same
first-in first-out pairing as the oracle), so equal counts check the tables
and the selection rule together.  Counts are integers: every comparison is
bit-exact.  Cases: ragged R and both dangling modes on both kernels, rows long
enough to exercise long pairing chains, self-loops and parallel edges,
single-edge rows, batched instances, caller-workspace runs, sampled sources of
the R-MAT scale-20 workload, and the unsupported combinations.
"""
import numpy as np
import pytest

from paper_1903_11749_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppr():
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr as P
    return P


@pytest.fixture(scope="module")
def ctx(ppr):
    return ppr.Context(0)


def ref_rows(oracle, g, alpha, R, seed, s_begin=0, s_end=None, tag=0, dangling=0, topk=0, og=None):
    og = og or oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    ends, steps = oracle.walks(og, alpha, R, seed, s_begin, s_end, tag, dangling, sampler=1)
    rp, col, cnt = oracle.rows(ends, g.n)
    out = {"rows": (rp, col, cnt), "steps": steps}
    if topk:
        out["topk"] = oracle.topk(rp, col, cnt, topk)
    return out


def assert_same(res, ref, topk=0):
    rp, col, cnt = res.sparse_rows()
    orp, ocol, ocnt = ref["rows"]
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    assert np.array_equal(cnt, ocnt)
    if topk:
        idx, tc = res.topk(topk)
        assert np.array_equal(idx, ref["topk"][0])
        assert np.array_equal(tc, ref["topk"][1])
    assert res.info().steps == ref["steps"]


@pytest.mark.parametrize("R", [1, 33, 100])
@pytest.mark.parametrize("kernel", [0, 1])
def test_alias_small_graphs(ppr, ctx, oracle, R, kernel):
    g = I.random_small_graph(211, 1500, seed=100 + R, wmax=13, dangling=7)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for dangling in (0, 1):
        ref = ref_rows(oracle, g, 0.25, R, seed=9 + R, dangling=dangling, topk=min(R, 6), og=og)
        res = G.run(alpha=0.25, R=R, seed=9 + R, dangling=dangling, topk=min(R, 6), kernel=kernel, sampler=1)
        assert_same(res, ref, topk=min(R, 6))
        if kernel == 0:  # lanes refilled in groups: the same walks
            res = G.run(alpha=0.25, R=R, seed=9 + R, dangling=dangling, topk=min(R, 6), sampler=1, refill_lanes=20)
            assert_same(res, ref, topk=min(R, 6))


def test_alias_differs_from_prefix_but_same_rows_sum(ppr, ctx, oracle):
    """Same law, different draws-to-edges map: the two samplers give different
    counts on the same seed, each row still sums to R."""
    g = I.random_small_graph(300, 3000, seed=3, wmax=50)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    a = G.run(alpha=0.15, R=64, seed=1, sampler=1).sparse_rows()
    b = G.run(alpha=0.15, R=64, seed=1, sampler=0).sparse_rows()
    assert not (np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]))
    for rp, _, cnt in (a, b):
        assert (np.add.reduceat(cnt.astype(np.int64), rp[:-1]) == 64).all()


def test_alias_long_rows_skew_self_loops(ppr, ctx, oracle):
    """Rows in every build tier (inline up to 32 edges, one warp with the row
    in shared memory up to 512, one warp up to 1024, one block up to 8192,
    tiles of blocks above) and on each side of its limits, with Zipf weights
    (long pairing chains, edges re-entering S^s many times), a heavy
    self-loop, parallel edges, single-edge rows and a dangling node."""
    rng = np.random.Generator(np.random.PCG64(17))
    n = 1200
    edges = []
    for u, d in ((0, 20000), (1, 2500), (2, 700), (4, 256), (5, 257), (6, 100), (7, 33), (8, 70001),
                 (9, 512), (10, 513), (11, 1024), (12, 1025), (13, 8192), (14, 8193)):
        ws = I.zipf_weights(rng, d, s=1.2, wmax=5000)
        dst = rng.integers(0, n, d)
        edges += [(u, int(v), int(x)) for v, x in zip(dst, ws)]
    edges += [(3, 3, 1000), (3, 4, 1), (3, 4, 1), (3, 5, 7)]  # self-loop, parallel edges
    edges += [(u, (u * 7) % n, 3) for u in range(15, 200)]  # single-edge rows
    edges += [(u, int(v), int(x)) for u in range(200, n - 1)
              for v, x in zip(rng.integers(0, n, 5), rng.integers(1, 30, 5))]
    g = I.from_edges(n, edges)  # node n-1 dangling
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for kernel in (0, 1):
        for dangling in (0, 1):
            ref = ref_rows(oracle, g, 0.1, 77, seed=4, dangling=dangling, topk=8, og=og)
            res = G.run(alpha=0.1, R=77, seed=4, dangling=dangling, topk=8, kernel=kernel, sampler=1)
            assert_same(res, ref, topk=8)


def test_alias_batched_instances(ppr, ctx, oracle):
    inst = I.chung_lu_instances(count=10, nmin=20, nmax=500, seed=8)
    G = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
    for kernel in (0, 1):
        res = G.run(alpha=0.15, R=40, seed=1, topk=4, kernel=kernel, sampler=1)
        rp, col, cnt = res.sparse_rows()
        idx, tc = res.topk()
        for gi in range(inst.count):
            sub = inst.instance(gi)
            ref = ref_rows(oracle, sub, 0.15, 40, 1, tag=gi, topk=4)
            a, b = int(inst.node_off[gi]), int(inst.node_off[gi + 1])
            orp, ocol, ocnt = ref["rows"]
            assert np.array_equal(rp[a: b + 1] - rp[a], orp)
            assert np.array_equal(col[rp[a]: rp[b]], ocol)
            assert np.array_equal(cnt[rp[a]: rp[b]], ocnt)
            assert np.array_equal(idx[a:b], ref["topk"][0])
            assert np.array_equal(tc[a:b], ref["topk"][1])


def test_alias_run_into_and_lists(ppr, ctx, oracle):
    """Caller-workspace runs need the tables built first; source lists equal
    the rows of a range run."""
    import torch
    g = I.random_small_graph(500, 5000, seed=21, wmax=20, dangling=10)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    kw = dict(alpha=0.2, R=50, seed=3, topk=5)
    dev = torch.device("cuda:0")
    cap = 50
    ws = torch.zeros(G.workspace_size(**kw), dtype=torch.uint8, device=dev)
    nnz = torch.zeros(g.n, dtype=torch.int32, device=dev)
    cols = torch.zeros(g.n * cap, dtype=torch.int32, device=dev)
    cnts = torch.zeros(g.n * cap, dtype=torch.int32, device=dev)
    ti = torch.zeros((g.n, 5), dtype=torch.int32, device=dev)
    tc = torch.zeros((g.n, 5), dtype=torch.int32, device=dev)
    with pytest.raises(ppr.PPRError) as ei:
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, sampler=1, **kw)
    assert ei.value.code == ppr.PPR_ENOTSUP
    full = G.run(sampler=1, **kw)
    G.run_into(ws, nnz, cols, cnts, cap, ti, tc, sampler=1, **kw)
    torch.cuda.synchronize()
    rp, col, cnt = full.sparse_rows()
    k = nnz.cpu().numpy()
    assert np.array_equal(k, np.diff(rp))
    C_, N_ = cols.cpu().numpy().reshape(g.n, cap), cnts.cpu().numpy().reshape(g.n, cap)
    for s in range(g.n):
        assert np.array_equal(C_[s, :k[s]], col[rp[s]:rp[s + 1]])
        assert np.array_equal(N_[s, :k[s]], cnt[rp[s]:rp[s + 1]])
    assert np.array_equal(ti.cpu().numpy(), full.topk()[0])
    ref = ref_rows(oracle, g, 0.2, 50, 3, topk=5)
    assert_same(full, ref, topk=5)
    src = np.array([7, 3, 3, 499, 0], dtype=np.int32)
    lst = G.run_list(src, sampler=1, **kw)
    lrp, lcol, lcnt = lst.sparse_rows()
    for i, s in enumerate(src):
        assert np.array_equal(lcol[lrp[i]:lrp[i + 1]], col[rp[s]:rp[s + 1]])
        assert np.array_equal(lcnt[lrp[i]:lrp[i + 1]], cnt[rp[s]:rp[s + 1]])


def test_alias_unsupported_combinations(ppr, ctx):
    g = I.random_small_graph(50, 200, seed=1)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    with pytest.raises(ppr.PPRError) as ei:
        G.run(alpha=0.2, R=10, seed=1, segments=True, sampler=1)
    assert ei.value.code == ppr.PPR_ENOTSUP
    with pytest.raises(ppr.PPRError) as ei:
        G.run(alpha=0.2, R=10, seed=1, sampler=2)
    assert ei.value.code == ppr.PPR_EINVAL
    # a row total at or above 2^32 needs the wide layout: no alias tables
    wide = I.from_edges(3, [(0, 1, 4_000_000_000), (0, 2, 400_000_000), (1, 0, 1)])
    Gw = ctx.load_graph(wide.n, wide.row_ptr, wide.col, wide.w)
    assert Gw.info().wide
    with pytest.raises(ppr.PPRError) as ei:
        Gw.run(alpha=0.2, R=10, seed=1, sampler=1)
    assert ei.value.code == ppr.PPR_ENOTSUP


@pytest.mark.slow
def test_alias_rmat20_full_size_sampled(ppr, ctx, oracle):
    """The R-MAT scale-20 workload (alpha 0.2, R 100, top-32) with the alias
    sampler, every source on the GPU; 300 sampled sources (largest rows,
    dangling nodes, random ones) recomputed by the oracle, compared exactly."""
    g = I.workload_graph("rmat20")
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    res = G.run(alpha=0.2, R=100, seed=1, topk=32, sampler=1)
    rp, col, cnt = res.sparse_rows()
    idx, tc = res.topk()
    assert (np.add.reduceat(cnt.astype(np.int64), rp[:-1]) == 100).all()
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    rng = np.random.Generator(np.random.PCG64(2))
    sample = np.unique(np.concatenate([rng.integers(0, g.n, 280), np.argsort(-g.degrees())[:10],
                                       np.flatnonzero(g.degrees() == 0)[:10]]))
    for s in sample:
        ref = ref_rows(oracle, g, 0.2, 100, 1, int(s), int(s) + 1, topk=32, og=og)
        orp, ocol, ocnt = ref["rows"]
        assert np.array_equal(col[rp[s]: rp[s + 1]], ocol)
        assert np.array_equal(cnt[rp[s]: rp[s + 1]], ocnt)
        assert np.array_equal(idx[s], ref["topk"][0][0])
        assert np.array_equal(tc[s], ref["topk"][1][0])
