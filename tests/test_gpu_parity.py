"""GPU path (through the C ABI) against the CPU oracle, element by element.

Counts are integers: every comparison is bit-exact.  Cases span several
chunks and warps with ragged tails (R not a multiple of 32, source counts not
a multiple of the chunk), dangling nodes in both modes, self-loops and
parallel edges, rows long enough for the cooperative search, both kernels,
tags and seeds, sub-ranges of sources, batch splits and the error paths.
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


def oracle_rows(oracle, g, alpha, R, seed, s_begin=0, s_end=None, tag=0, dangling=0, segments=False, topk=0,
                og=None):
    og = og or oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    lazy = segments and g.n > 100_000  # large graphs: tables of the visited nodes only
    ends, steps = oracle.walks(og, alpha, R, seed, s_begin, s_end, tag, dangling, segments, lazy_segments=lazy)
    rp, col, cnt = oracle.rows(ends, g.n)
    out = {"rows": (rp, col, cnt), "steps": steps, "ends": ends}
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
        oidx, otc = ref["topk"]
        assert np.array_equal(idx, oidx)
        assert np.array_equal(tc, otc)
    assert res.info().steps == ref["steps"]


def test_er1k_dense_matches_oracle(ppr, ctx, oracle):
    """The 1000-node ER workload (alpha 0.15, R 1000, seed 1), all n*n counts."""
    g = I.er_graph(1000, 10_000, 1, 10, seed=12345)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ref = oracle_rows(oracle, g, 0.15, 1000, 1, topk=32)
    for kernel in (ppr.KERNEL_PERSISTENT, ppr.KERNEL_PLAIN):
        res = G.run(alpha=0.15, R=1000, seed=1, topk=32, kernel=kernel)
        assert_same(res, ref, topk=32)
        D = res.dense()
        assert np.array_equal(D, oracle.dense(ref["ends"], g.n))
        assert (D.sum(axis=1) == 1000).all()


@pytest.mark.parametrize("R", [1, 7, 31, 33, 100, 257])
@pytest.mark.parametrize("kernel", [0, 1])
def test_small_graphs_ragged(ppr, ctx, oracle, R, kernel):
    g = I.random_small_graph(97, 400, seed=R, wmax=9, dangling=5)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    for dangling in (0, 1):
        ref = oracle_rows(oracle, g, 0.3, R, seed=5 + R, dangling=dangling, topk=min(R, 5))
        res = G.run(alpha=0.3, R=R, seed=5 + R, dangling=dangling, topk=min(R, 5), kernel=kernel)
        assert_same(res, ref, topk=min(R, 5))


@pytest.mark.parametrize("R,topk", [(1025, 40), (1500, 1500), (4096, 4096), (2048, 7)])
def test_large_R_shared_memory_reduction(ppr, ctx, oracle, R, topk):
    """R above 1024 takes the shared-memory reduction (next_pow2(R) > 1024);
    top-k up to the largest k (4096), both kernels, both samplers."""
    g = I.random_small_graph(600, 3000, seed=R, wmax=30, dangling=6)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for sampler in (0, 1):
        ends, steps = oracle.walks(og, 0.25, R, 3, 0, 40, sampler=sampler)
        orp, ocol, ocnt = oracle.rows(ends, g.n)
        oidx, otc = oracle.topk(orp, ocol, ocnt, topk)
        for kernel in (0, 1):
            res = G.run(alpha=0.25, R=R, seed=3, src_end=40, topk=topk, kernel=kernel, sampler=sampler)
            rp, col, cnt = res.sparse_rows()
            assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(cnt, ocnt)
            idx, tc = res.topk(topk)
            assert np.array_equal(idx, oidx) and np.array_equal(tc, otc)
            assert res.info().steps == steps


def test_topk_larger_than_R(ppr, ctx, oracle):
    """k above R (and above next_pow2(R)) returns the whole row by count, padded."""
    g = I.er_graph(300, 2000, seed=6)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    for R, k in ((50, 64), (20, 100), (7, 33)):
        ref = oracle_rows(oracle, g, 0.15, R, 2, topk=k)
        for kernel in (0, 1):
            assert_same(G.run(alpha=0.15, R=R, seed=2, topk=k, kernel=kernel), ref, topk=k)


@pytest.mark.parametrize("R", [2, 33, 50, 64, 65, 100, 200, 256])
def test_whole_row_in_topk_order(ppr, ctx, oracle, R):
    """k at or above the row length returns the whole row in top-k order:
    runs counted twice or more sorted, runs counted once after them in id
    order (the fast path when at most 32 runs repeat), and the full sort
    when more repeat (an 80-node graph at R >= 100); every padding slot is
    (-1, 0)."""
    for g, alpha in ((I.er_graph(30, 300, 1, 4, seed=R), 0.25), (I.er_graph(80, 900, 1, 4, seed=R + 1), 0.15),
                     (I.random_small_graph(3000, 20000, seed=R, wmax=5), 0.1)):
        G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
        og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
        for k in (R, R + 7, 64, 300):
            if k < min(R, g.n):
                continue
            ref = oracle_rows(oracle, g, alpha, R, 5, s_end=min(g.n, 200), topk=k, og=og)
            res = G.run(alpha=alpha, R=R, seed=5, src_end=min(g.n, 200), topk=k)
            assert_same(res, ref, topk=k)


@pytest.mark.parametrize("R", [33, 64, 100, 200, 513, 1024])
def test_topk_selection_at_count_ties(ppr, ctx, oracle, R):
    """Top-k below the number of distinct endpoints (k <= 32, R > 32) is
    selected by a count threshold instead of a full sort: rows where many
    endpoints tie at the threshold count (a 40-node dense graph, a few counts
    shared by many ids) and rows of mostly singletons (a 3,000-node graph)
    give the oracle's order, count descending then id ascending."""
    for g, alpha in ((I.er_graph(40, 600, 1, 3, seed=R), 0.2), (I.random_small_graph(3000, 20000, seed=R, wmax=5), 0.1)):
        G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
        og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
        for k in (1, 2, 17, 31, 32):
            ref = oracle_rows(oracle, g, alpha, R, 9, s_end=min(g.n, 300), topk=k, og=og)
            res = G.run(alpha=alpha, R=R, seed=9, src_end=min(g.n, 300), topk=k)
            assert_same(res, ref, topk=k)


def test_self_loops_parallel_edges_and_skew(ppr, ctx, oracle):
    g = I.from_edges(6, [(0, 1, 1000), (0, 2, 1), (0, 1, 3), (1, 1, 2), (1, 3, 5), (2, 0, 1), (2, 4, 7), (3, 0, 1),
                         (3, 5, 1), (4, 2, 2)])
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    for kernel in (0, 1):
        ref = oracle_rows(oracle, g, 0.15, 4000, seed=9, topk=6)
        assert_same(G.run(alpha=0.15, R=4000, seed=9, topk=6, kernel=kernel), ref, topk=6)


def test_tags_seeds_and_subranges(ppr, ctx, oracle):
    g = I.er_graph(500, 4000, 1, 10, seed=3)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for seed, tag, a, b in [(1, 0, 0, 500), (2**40 + 17, 3, 17, 389), (123456789, 0xFFFFFFFF, 499, 500)]:
        ref = oracle_rows(oracle, g, 0.2, 45, seed, a, b, tag, topk=10, og=og)
        for kernel in (0, 1):
            res = G.run(alpha=0.2, R=45, seed=seed, src_begin=a, src_end=b, tag=tag, topk=10, kernel=kernel)
            assert_same(res, ref, topk=10)


def test_batches_and_chunking_do_not_change_results(ppr, ctx, oracle):
    g = I.er_graph(700, 6000, 1, 10, seed=4)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ref = oracle_rows(oracle, g, 0.15, 60, 7, topk=4)
    for kw in (dict(kernel=1, max_batch_sources=33), dict(chunk_sources=1), dict(chunk_sources=13, warps_per_block=2),
               dict(chunk_sources=64, warps_per_block=1), dict(max_batch_sources=250),
               dict(chunk_sources=3, max_batch_sources=101), dict(refill_lanes=32), dict(refill_lanes=7, chunk_sources=3),
               dict(refill_lanes=24, warps_per_block=4), dict(refill_lanes=16, chunk_sources=64)):
        assert_same(G.run(alpha=0.15, R=60, seed=7, topk=4, **kw), ref, topk=4)


def _hub_graph(deg_hub=20000, n=30000, seed=11):
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = [(0, int(t), int(w)) for t, w in zip(rng.integers(1, n, deg_hub), rng.integers(1, 1000, deg_hub))]
    # mid-size rows (5000 edges) and small rows pointing back at the hub
    for h in (1, 2):
        edges += [(h, int(t), int(w)) for t, w in zip(rng.integers(0, n, 5000), rng.integers(1, 50, 5000))]
    for u in range(3, n):
        edges.append((u, 0, int(rng.integers(1, 10))))
        edges.append((u, int(rng.integers(0, n)), int(rng.integers(1, 10))))
    return I.from_edges(n, edges)


def test_large_rows_cooperative_search(ppr, ctx, oracle):
    """Rows above the cooperative threshold (default 4096, and 1 to force every
    row through it) give the same edge as the bisection."""
    g = _hub_graph()
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ref = oracle_rows(oracle, g, 0.15, 50, 3, 0, 2000, topk=8)
    for large in (0, 1, 32, 100000):
        assert_same(G.run(alpha=0.15, R=50, seed=3, src_end=2000, topk=8, large_degree=large), ref, topk=8)


def _mixed_depth_graph(seed=17):
    """Rows of every search depth (1 to 150,000 edges), dangling nodes, and
    small rows whose 3-step neighbourhoods carry segment tables."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 6000
    degs = np.concatenate([[150_000, 40_000, 9000, 3000, 2561, 600, 321, 70, 41, 9],
                           rng.integers(0, 9, n - 10)])
    degs[-40:] = 0  # dangling
    src = np.repeat(np.arange(n), degs)
    dst = rng.integers(0, n, len(src))
    w = rng.integers(1, 1000, len(src))
    row_ptr, col, ww = I._csr_from_pairs(n, src, dst, w)
    return I.Graph(n, row_ptr, col, ww)


@pytest.mark.parametrize("segments", [False, True])
def test_step_bound_does_not_change_results(ppr, ctx, oracle, segments):
    """The bounded step (a deep search resumes in the next warp iteration)
    gives the oracle's rows, steps and top-k for every bound, including 2 (the
    node record and one more load per iteration: every search of two or more
    loads resumes), and without a bound; both dangling modes."""
    g = _mixed_depth_graph()
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    for dangling in (0, 1):
        ref = oracle_rows(oracle, g, 0.2, 40, 9, dangling=dangling, segments=segments, topk=6)
        for sl in (0, -1, 2, 3, 5, 16):
            res = G.run(alpha=0.2, R=40, seed=9, dangling=dangling, segments=segments, topk=6, step_loads=sl,
                        refill_lanes=24 if sl == 3 else 0)
            assert_same(res, ref, topk=6)
    with pytest.raises(ppr.PPRError):
        G.run(alpha=0.2, R=4, step_loads=1)


def test_huge_rows_built_by_tiles(ppr, ctx, oracle):
    """Rows above 8,192 edges are built by tiles of 8,192 edges (a hub of
    150,001 edges, rows of 65,537 and 65,536 edges), in a plain and in a
    batched graph; every count equals the oracle's."""
    rng = np.random.Generator(np.random.PCG64(5))
    n = 40000
    edges = []
    for u, d in ((0, 150_001), (1, 65_537), (2, 65_536)):
        edges += [(u, int(t), int(w)) for t, w in zip(rng.integers(0, n, d), rng.integers(1, 3000, d))]
    for u in range(3, n):
        edges.append((u, int(rng.integers(0, 3)), int(rng.integers(1, 9))))
        edges.append((u, int(rng.integers(0, n)), int(rng.integers(1, 9))))
    g = I.from_edges(n, edges)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ref = oracle_rows(oracle, g, 0.2, 40, 6, 0, 600, topk=5)
    for kernel in (0, 1):
        assert_same(G.run(alpha=0.2, R=40, seed=6, src_end=600, topk=5, kernel=kernel), ref, topk=5)
    # the same graph twice as a batched graph: each instance as its own run
    rp2 = np.concatenate([g.row_ptr[:-1], g.row_ptr + g.m])
    Gb = ctx.load_graph_batch(np.array([0, n, 2 * n]), rp2, np.concatenate([g.col, g.col]),
                              np.concatenate([g.w, g.w]))
    res = Gb.run(alpha=0.2, R=40, seed=6, src_begin=n, src_end=n + 600, topk=5)
    ref1 = oracle_rows(oracle, g, 0.2, 40, 6, 0, 600, tag=1, topk=5)
    rp, col, cnt = res.sparse_rows()
    orp, ocol, ocnt = ref1["rows"]
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(cnt, ocnt)  # instance-local ids


def test_rows_at_every_build_tier_boundary(ppr, ctx, oracle):
    """Rows whose degrees sit on each side of every build tier (thread per row
    up to 32 edges, warp per row up to 1,024, block per row up to 8,192, tiles
    of 8,192 edges above), of the 8-ary summary levels (8, 64, 512, 4,096) and
    of the top levels kept in the node record (at most five keys: 40, 320,
    2,560, 20,480), in a plain and in a batched graph: the walks return to
    those rows often enough to draw from most of their edges, and every count
    equals the oracle's."""
    rng = np.random.Generator(np.random.PCG64(17))
    degs = [2, 8, 9, 31, 32, 33, 40, 41, 64, 65, 127, 128, 129, 320, 321, 512, 513, 1023, 1024, 1025, 2560, 2561,
            4096, 4097, 8191, 8192, 8193, 16384, 16385, 20480, 20481, 24577]
    h = len(degs)
    n = 6000
    edges = []
    for u, d in enumerate(degs):
        edges += [(u, int(t), int(w)) for t, w in zip(rng.integers(h, n, d), rng.integers(1, 4000, d))]
    for u in range(h, n):  # small rows lead back to the tier rows
        edges.append((u, int(rng.integers(0, h)), int(rng.integers(1, 9))))
        if u % 3 == 0:
            edges.append((u, int(rng.integers(0, n)), int(rng.integers(1, 9))))
    g = I.from_edges(n, edges)
    assert [int(g.row_ptr[u + 1] - g.row_ptr[u]) for u in range(h)] == degs
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ref = oracle_rows(oracle, g, 0.15, 1000, 8, 0, 400, topk=6)
    for sampler in (0, 1):
        og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
        ends, steps = oracle.walks(og, 0.15, 1000, 8, 0, 400, sampler=sampler)
        orp, ocol, ocnt = oracle.rows(ends, g.n)
        res = G.run(alpha=0.15, R=1000, seed=8, src_end=400, sampler=sampler)
        rp, col, cnt = res.sparse_rows()
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(cnt, ocnt), sampler
        assert res.info().steps == steps
    assert_same(G.run(alpha=0.15, R=1000, seed=8, src_end=400, topk=6), ref, topk=6)
    # the same rows in the second instance of a batched graph (instance-local ids, tag 1)
    rp2 = np.concatenate([g.row_ptr[:-1], g.row_ptr + g.m])
    Gb = ctx.load_graph_batch(np.array([0, n, 2 * n]), rp2, np.concatenate([g.col, g.col]), np.concatenate([g.w, g.w]))
    res = Gb.run(alpha=0.15, R=1000, seed=8, src_begin=n, src_end=n + 400)
    ref1 = oracle_rows(oracle, g, 0.15, 1000, 8, 0, 400, tag=1)
    rp, col, cnt = res.sparse_rows()
    orp, ocol, ocnt = ref1["rows"]
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(cnt, ocnt)


def test_segment_mode_matches_segment_oracle(ppr, ctx, oracle):
    g = I.random_small_graph(400, 1100, seed=21, wmax=30, dangling=20)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for alpha, dangling in ((0.15, 0), (0.5, 1)):
        ref = oracle_rows(oracle, g, alpha, 77, 2, dangling=dangling, segments=True, topk=5, og=og)
        assert (np.diff(og.seg_off) > 0).sum() > 50
        for kernel in (0, 1):
            res = G.run(alpha=alpha, R=77, seed=2, dangling=dangling, segments=True, topk=5, kernel=kernel)
            assert_same(res, ref, topk=5)
        info = G.info()
        assert info.segment_nodes == int((np.diff(og.seg_off) > 0).sum())
        assert info.segment_entries == int(og.seg_off[-1])


@pytest.mark.parametrize("n,dmin", [(12, 8), (40, 1), (400, 4)])
def test_segment_tables_every_tier(ppr, ctx, oracle, n, dmin):
    """Segment tables where every node is eligible (all degrees <= 8): 12
    nodes of degree 8 give 1,096 raw path contributions per table (the large
    hash tier) folded into at most 48 outcomes; 40 nodes of degree 1..8 mix
    both tiers with tables above 64 outcomes (rejected); 400 nodes of degree
    4..8 reject most.  Tables, rows and counts equal the oracle's."""
    rng = np.random.Generator(np.random.PCG64(n))
    edges = []
    for u in range(n):
        for _ in range(int(rng.integers(dmin, 9))):
            edges.append((u, int(rng.integers(0, n)), int(rng.integers(1, 1000))))
    g = I.from_edges(n, edges)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for alpha in (0.15, 0.6):
        ref = oracle_rows(oracle, g, alpha, 300, 4, segments=True, topk=6, og=og)
        for kernel in (0, 1):
            assert_same(G.run(alpha=alpha, R=300, seed=4, segments=True, topk=6, kernel=kernel), ref, topk=6)
        info = G.info()
        assert info.segment_nodes == int((np.diff(og.seg_off) > 0).sum())
        assert info.segment_entries == int(og.seg_off[-1])
    if n == 12:
        assert info.segment_nodes == n  # every table kept
    if n == 40:
        assert 0 < info.segment_nodes < n  # some tables above 64 outcomes


def test_batched_instances_equal_each_instance_alone(ppr, ctx, oracle):
    inst = I.chung_lu_instances(count=12, nmin=20, nmax=400, seed=5)
    G = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
    for kernel in (0, 1):
        _check_instances(oracle, inst, G.run(alpha=0.15, R=40, seed=1, topk=4, kernel=kernel))
    _check_instances(oracle, inst, G.run(alpha=0.15, R=40, seed=1, topk=4, refill_lanes=24))
    # a sub-range cutting through instances
    a, b = int(inst.node_off[3]) + 5, int(inst.node_off[7]) - 3
    res = G.run(alpha=0.15, R=40, seed=1, topk=4, src_begin=a, src_end=b, chunk_sources=2)
    full = G.run(alpha=0.15, R=40, seed=1, topk=4)
    frp, fcol, fcnt = full.sparse_rows()
    rp, col, cnt = res.sparse_rows()
    assert np.array_equal(col, fcol[frp[a]:frp[b]]) and np.array_equal(cnt, fcnt[frp[a]:frp[b]])


def _check_instances(oracle, inst, res):
    rp, col, cnt = res.sparse_rows()
    idx, tc = res.topk()
    for gi in range(inst.count):
        sub = inst.instance(gi)
        ref = oracle_rows(oracle, sub, 0.15, 40, 1, tag=gi, topk=4)
        a, b = int(inst.node_off[gi]), int(inst.node_off[gi + 1])
        orp, ocol, ocnt = ref["rows"]
        assert np.array_equal(rp[a: b + 1] - rp[a], orp)
        assert np.array_equal(col[rp[a]: rp[b]], ocol)
        assert np.array_equal(cnt[rp[a]: rp[b]], ocnt)
        assert np.array_equal(idx[a:b], ref["topk"][0])
        assert np.array_equal(tc[a:b], ref["topk"][1])


def test_autotune_picks_a_valid_launch(ppr, ctx, oracle):
    """The tuner times the candidates and returns one; results under any
    tuning are the same counts."""
    g = I.random_small_graph(3000, 30000, seed=44, wmax=20, dangling=30)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    t = G.autotune(sample_sources=1000, alpha=0.2, R=30, seed=1, topk=4)
    assert t["candidates"] >= 10 and t["ms"] > 0 and t["warps_per_block"] in (4, 8)
    ref = G.run(alpha=0.2, R=30, seed=1, topk=4)
    tuned = G.run(alpha=0.2, R=30, seed=1, topk=4, chunk_sources=t["chunk_sources"],
                  large_degree=t["large_degree"], warps_per_block=t["warps_per_block"])
    a, b = ref.sparse_rows(), tuned.sparse_rows()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(ref.topk()[0], tuned.topk()[0])
    inst = I.chung_lu_instances(count=20, nmin=50, nmax=800, seed=6)
    Gb = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
    tb = Gb.autotune(sample_sources=2000, alpha=0.15, R=20, seed=1)
    assert tb["candidates"] >= 10


def test_device_inputs_and_outputs(ppr, ctx, oracle):
    import torch
    g = I.er_graph(400, 3000, 1, 10, seed=8)
    dev = torch.device("cuda:0")
    G = ctx.load_graph(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                       torch.from_numpy(g.w.view(np.int32)).to(dev))
    res = G.run(alpha=0.15, R=32, seed=4, topk=3)
    ref = oracle_rows(oracle, g, 0.15, 32, 4, topk=3)
    nnz = res.nnz()
    rp = torch.zeros(g.n + 1, dtype=torch.int64, device=dev)
    col = torch.zeros(nnz, dtype=torch.int32, device=dev)
    cnt = torch.zeros(nnz, dtype=torch.int32, device=dev)
    assert res.sparse_rows_into(rp, col, cnt) == nnz
    orp, ocol, ocnt = ref["rows"]
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(col.cpu().numpy(), ocol)
    assert np.array_equal(cnt.cpu().numpy().view(np.uint32), ocnt)
    idx = torch.zeros((g.n, 2), dtype=torch.int32, device=dev)
    tc = torch.zeros((g.n, 2), dtype=torch.int32, device=dev)
    res.topk_into(2, idx, tc)
    assert np.array_equal(idx.cpu().numpy(), ref["topk"][0][:, :2])


def test_dangling_sources_and_single_node(ppr, ctx, oracle):
    g = I.from_edges(4, [(0, 1, 1), (1, 2, 1), (2, 0, 1)])
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    for mode in (0, 1):
        res = G.run(alpha=0.15, R=100, seed=1, src_begin=3, src_end=4, dangling=mode, topk=2)
        rp, col, cnt = res.sparse_rows()
        assert col.tolist() == [3] and cnt.tolist() == [100]
    g1 = I.from_edges(1, [])
    G1 = ctx.load_graph(1, g1.row_ptr, np.zeros(0, np.int32), np.zeros(0, np.uint32))
    for mode in (0, 1):
        rp, col, cnt = G1.run(alpha=0.5, R=10, seed=1, dangling=mode).sparse_rows()
        assert col.tolist() == [0] and cnt.tolist() == [10]


def test_wide_rows(ppr, ctx, oracle):
    """Row totals above 2^32 switch to the 64-bit prefix layout."""
    big = 2**32 - 5
    g = I.from_edges(5, [(0, 1, big), (0, 2, big), (0, 3, 7), (1, 0, 1), (2, 4, big), (2, 0, 3), (3, 0, 1),
                         (4, 4, 1), (4, 0, big)])
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    assert G.info().wide == 1
    ref = oracle_rows(oracle, g, 0.25, 500, 3, topk=3)
    for kernel in (0, 1):
        assert_same(G.run(alpha=0.25, R=500, seed=3, topk=3, kernel=kernel), ref, topk=3)


def test_source_lists_equal_range_rows(ppr, ctx, oracle):
    """A run over an explicit list (repeats, any order) gives each listed
    source the same row and top-k as the range run."""
    g = I.random_small_graph(800, 6000, seed=41, wmax=20, dangling=10)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ref = G.run(alpha=0.2, R=50, seed=3, topk=6)
    rp, col, cnt = ref.sparse_rows()
    idx, tc = ref.topk()
    rng = np.random.Generator(np.random.PCG64(4))
    lst = np.concatenate([rng.integers(0, g.n, 333), [5, 5, 5, g.n - 1, 0]]).astype(np.int32)
    for kernel in (0, 1):
        res = G.run_list(lst, alpha=0.2, R=50, seed=3, topk=6, kernel=kernel, max_batch_sources=97)
        lrp, lcol, lcnt = res.sparse_rows()
        lidx, ltc = res.topk()
        for i, s_ in enumerate(lst):
            assert np.array_equal(lcol[lrp[i]:lrp[i + 1]], col[rp[s_]:rp[s_ + 1]])
            assert np.array_equal(lcnt[lrp[i]:lrp[i + 1]], cnt[rp[s_]:rp[s_ + 1]])
            assert np.array_equal(lidx[i], idx[s_]) and np.array_equal(ltc[i], tc[s_])
    with pytest.raises(ppr.PPRError):
        G.run_list(np.array([0, g.n], dtype=np.int32))


def _rows_from_fixed(nnz, cols, cnts, cap):
    nnz = nnz.cpu().numpy().astype(np.int64)
    S = len(nnz)
    cols = cols.cpu().numpy().reshape(S, cap)
    cnts = cnts.cpu().numpy().view(np.uint32).reshape(S, cap)
    rp = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(nnz, out=rp[1:])
    return rp, np.concatenate([cols[s, :nnz[s]] for s in range(S)]), np.concatenate([cnts[s, :nnz[s]] for s in range(S)])


@pytest.mark.parametrize("batched", [False, True])
def test_run_into_and_cuda_graph_replay(ppr, ctx, oracle, batched):
    """ppr_run_into (caller workspace, no allocation) gives the oracle's rows,
    also when recorded into a CUDA graph and replayed twice."""
    import torch
    dev = torch.device("cuda:0")
    if batched:
        inst = I.chung_lu_instances(count=9, nmin=30, nmax=500, seed=8)
        G = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
        n, cap = int(inst.node_off[-1]), min(64, int(np.diff(inst.node_off).max()))
    else:
        g = I.random_small_graph(1200, 9000, seed=43, wmax=20, dangling=10)
        G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
        n, cap = g.n, 64
    kw = dict(alpha=0.15, R=64, seed=9, topk=5, chunk_sources=3)
    # expected rows from the oracle: batched instances walk alone with their id as tag
    if batched:
        parts = [oracle_rows(oracle, inst.instance(gi), 0.15, 64, 9, tag=gi, topk=5) for gi in range(inst.count)]
        rp0 = np.concatenate([[0], np.cumsum(np.concatenate([np.diff(p["rows"][0]) for p in parts]))])
        col0 = np.concatenate([p["rows"][1] for p in parts])
        cnt0 = np.concatenate([p["rows"][2] for p in parts])
        ti0 = np.concatenate([p["topk"][0] for p in parts])
        tc0 = np.concatenate([p["topk"][1] for p in parts])
    else:
        ref = oracle_rows(oracle, g, 0.15, 64, 9, topk=5)
        (rp0, col0, cnt0), (ti0, tc0) = ref["rows"], ref["topk"]
    ws = torch.zeros(G.workspace_size(**kw), dtype=torch.uint8, device=dev)
    nnz = torch.zeros(n, dtype=torch.int32, device=dev)
    cols = torch.zeros(n * cap, dtype=torch.int32, device=dev)
    cnts = torch.zeros(n * cap, dtype=torch.int32, device=dev)
    ti = torch.zeros((n, 5), dtype=torch.int32, device=dev)
    tc = torch.zeros((n, 5), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, **kw)
    s.synchronize()
    got = _rows_from_fixed(nnz, cols, cnts, cap)
    for a_, b_ in zip(got, (rp0, col0, cnt0)):
        assert np.array_equal(a_, b_)
    assert np.array_equal(ti.cpu().numpy(), ti0)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, **kw)
    for _ in range(2):
        nnz.zero_()
        cols.zero_()
        graph.replay()
        torch.cuda.synchronize()
        got = _rows_from_fixed(nnz, cols, cnts, cap)
        for a_, b_ in zip(got, (rp0, col0, cnt0)):
            assert np.array_equal(a_, b_)
        assert np.array_equal(tc.cpu().numpy().view(np.uint32), tc0)


def test_invalid_inputs_are_rejected(ppr, ctx):
    E = ppr.PPRError
    g = I.er_graph(50, 200, seed=1)
    bad_w = g.w.copy()
    bad_w[7] = 0
    with pytest.raises(E) as ei:
        ctx.load_graph(g.n, g.row_ptr, g.col, bad_w)
    assert ei.value.code == ppr.PPR_EINVAL
    bad_c = g.col.copy()
    bad_c[3] = 50
    with pytest.raises(E):
        ctx.load_graph(g.n, g.row_ptr, bad_c, g.w)
    bad_rp = g.row_ptr.copy()
    bad_rp[10], bad_rp[11] = bad_rp[11], bad_rp[10] - 1
    with pytest.raises(E):
        ctx.load_graph(g.n, bad_rp, g.col, g.w)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    for kw, code in ((dict(alpha=0.0), ppr.PPR_EINVAL), (dict(alpha=1.0), ppr.PPR_EINVAL),
                     (dict(alpha=2.0**-40), ppr.PPR_EINVAL), (dict(R=0), ppr.PPR_EINVAL),
                     (dict(R=5000), ppr.PPR_ERANGE), (dict(src_begin=10, src_end=10), ppr.PPR_EINVAL),
                     (dict(src_end=51), ppr.PPR_EINVAL), (dict(topk=4097), ppr.PPR_EINVAL),
                     (dict(dangling=2), ppr.PPR_EINVAL), (dict(refill_lanes=33), ppr.PPR_EINVAL),
                     (dict(refill_lanes=-1), ppr.PPR_EINVAL), (dict(warps_per_block=33), ppr.PPR_EINVAL)):
        with pytest.raises(E) as ei:
            G.run(**kw)
        assert ei.value.code == code, kw
    res = G.run(R=10, topk=3)
    with pytest.raises(E):
        res.topk(4)


@pytest.mark.slow
def test_rmat20_full_size_sampled(ppr, ctx, oracle):
    """The R-MAT scale-20 workload (alpha 0.2, R 100, top-32), every source on
    the GPU in the benchmark's launch configuration; 400 sampled sources
    recomputed by the oracle and compared exactly; every row sums to R."""
    g = I.workload_graph("rmat20")
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    res = G.run(alpha=0.2, R=100, seed=1, topk=32)
    rp, col, cnt = res.sparse_rows()
    idx, tc = res.topk()
    rowsum = np.add.reduceat(cnt.astype(np.int64), rp[:-1]) if len(cnt) else np.zeros(0)
    assert (np.diff(rp) >= 1).all() and (rowsum == 100).all()
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    rng = np.random.Generator(np.random.PCG64(0))
    sample = np.unique(np.concatenate([rng.integers(0, g.n, 380), np.argsort(-g.degrees())[:10],
                                       np.flatnonzero(g.degrees() == 0)[:10]]))
    for s in sample:
        ref = oracle_rows(oracle, g, 0.2, 100, 1, int(s), int(s) + 1, topk=32, og=og)
        orp, ocol, ocnt = ref["rows"]
        assert np.array_equal(col[rp[s]: rp[s + 1]], ocol)
        assert np.array_equal(cnt[rp[s]: rp[s + 1]], ocnt)
        assert np.array_equal(idx[s], ref["topk"][0][0])
        assert np.array_equal(tc[s], ref["topk"][1][0])


@pytest.mark.slow
def test_rmat24_full_size_sampled(ppr, ctx, oracle):
    """The R-MAT scale-24 workload with its hub above 10^6 edges (alpha 0.15,
    R 50, top-64, depth-3 segment tables), every source on the GPU; 160
    sampled sources (the hub, large rows, dangling nodes, random ones)
    recomputed by the oracle with the same segment tables, compared exactly;
    every row sums to R.  The plain mode is sampled the same way."""
    import torch
    g = I.workload_graph("rmat24")
    dev = torch.device("cuda:0")
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    deg = g.degrees()
    rng = np.random.Generator(np.random.PCG64(1))
    sample = np.unique(np.concatenate([[0], np.argsort(-deg)[:20], np.flatnonzero(deg == 0)[:20],
                                       np.flatnonzero((deg >= 1) & (deg <= 8))[:20], rng.integers(0, g.n, 100)]))
    for segments in (True, False):
        res = G.run(alpha=0.15, R=50, seed=1, topk=64, segments=segments)
        nnz = res.nnz()
        rp = torch.zeros(g.n + 1, dtype=torch.int64, device=dev)
        col = torch.zeros(nnz, dtype=torch.int32, device=dev)
        cnt = torch.zeros(nnz, dtype=torch.int32, device=dev)
        res.sparse_rows_into(rp, col, cnt)
        sums = torch.zeros(g.n, dtype=torch.int64, device=dev)
        rows = torch.repeat_interleave(torch.arange(g.n, device=dev), rp[1:] - rp[:-1])
        sums.index_add_(0, rows, cnt.to(torch.int64))
        assert bool((sums == 50).all())
        ti = torch.zeros((g.n, 64), dtype=torch.int32, device=dev)
        tc = torch.zeros((g.n, 64), dtype=torch.int32, device=dev)
        res.topk_into(64, ti, tc)
        rp_h = rp.cpu().numpy()
        idx = torch.from_numpy(sample).to(dev)
        ti_s, tc_s = ti[idx].cpu().numpy(), tc[idx].cpu().numpy().view(np.uint32)
        for n_i, s in enumerate(sample):
            ref = oracle_rows(oracle, g, 0.15, 50, 1, int(s), int(s) + 1, topk=64, og=og, segments=segments)
            a, b = int(rp_h[s]), int(rp_h[s + 1])
            assert np.array_equal(col[a:b].cpu().numpy(), ref["rows"][1])
            assert np.array_equal(cnt[a:b].cpu().numpy().view(np.uint32), ref["rows"][2])
            assert np.array_equal(ti_s[n_i], ref["topk"][0][0])
            assert np.array_equal(tc_s[n_i], ref["topk"][1][0])
        del res, rp, col, cnt, rows, sums, ti, tc
