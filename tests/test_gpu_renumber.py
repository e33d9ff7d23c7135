"""The layout's own node numbering (PPR_RENUMBER: nodes by descending
in-degree class) against the CPU oracle and against the caller's numbering.

The numbering is internal: sources, rows and top-k use the caller's ids, the
draws are keyed by the caller's source id, and the segment tables rank
their outcomes by the caller's node ids (the canonical order of Algorithm
4's tables).  So every count, every row and every top-k must equal the
oracle's bit for bit, on every layout path: rows of every search depth and
build tier, dangling nodes in both modes, segment tables, alias tables,
both kernels, source lists, caller workspaces replayed from a CUDA graph,
the allocation-free entry point and both serving modes."""
import numpy as np
import pytest

from paper_1903_11749_gb300 import inputs as I
from test_gpu_parity import _mixed_depth_graph, assert_same, oracle_rows

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


def _skewed_graph(seed=3):
    """R-MAT scale 13 with a planted hub (tile-built row) and 5 % dangling
    nodes: in-degrees span every class from 0 to thousands."""
    return I.rmat_graph(13, 12, seed=seed, hub_degree=20_000)


@pytest.mark.parametrize("kernel", [0, 1])
def test_renumbered_layout_equals_oracle(ppr, ctx, oracle, kernel):
    g = _mixed_depth_graph()
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    assert G.info().renumbered == 1
    for dangling in (0, 1):
        ref = oracle_rows(oracle, g, 0.2, 40, 9, dangling=dangling, topk=6)
        assert_same(G.run(alpha=0.2, R=40, seed=9, dangling=dangling, topk=6, kernel=kernel), ref, topk=6)


def test_renumbered_skewed_graph_all_paths(ppr, ctx, oracle):
    """A hub of 20,000 edges, rows of every depth, dangling nodes: the bounded
    step, the unbounded step, refill thresholds, a sub-range and a tag."""
    g = _skewed_graph()
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    Gk = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=False)
    assert G.info().renumbered == 1 and Gk.info().renumbered == 0
    ref = oracle_rows(oracle, g, 0.15, 50, 4, 100, 2100, tag=3, topk=9)
    for sl, refill in ((0, 0), (-1, 0), (2, 24), (5, 24)):
        kw = dict(alpha=0.15, R=50, seed=4, src_begin=100, src_end=2100, tag=3, topk=9, step_loads=sl,
                  refill_lanes=refill)
        assert_same(G.run(**kw), ref, topk=9)
        assert_same(Gk.run(**kw), ref, topk=9)


def test_renumbered_segment_tables(ppr, ctx, oracle):
    """Segment tables built on the renumbered layout rank their outcomes by
    the caller's ids: the segment-mode oracle's counts, both dangling modes."""
    g = I.random_small_graph(400, 1100, seed=21, wmax=30, dangling=20)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for alpha, dangling in ((0.15, 0), (0.5, 1)):
        ref = oracle_rows(oracle, g, alpha, 77, 2, dangling=dangling, segments=True, topk=5, og=og)
        for kernel in (0, 1):
            res = G.run(alpha=alpha, R=77, seed=2, dangling=dangling, segments=True, topk=5, kernel=kernel)
            assert_same(res, ref, topk=5)
        assert G.info().segment_entries == int(og.seg_off[-1])
    # and on the graph of every search depth, bounded step
    g = _mixed_depth_graph()
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    ref = oracle_rows(oracle, g, 0.2, 40, 9, segments=True, topk=6)
    for sl in (0, 3):
        assert_same(G.run(alpha=0.2, R=40, seed=9, segments=True, topk=6, step_loads=sl), ref, topk=6)


def test_renumbered_alias_tables(ppr, ctx, oracle):
    g = _skewed_graph(seed=8)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    ends, steps = oracle.walks(og, 0.2, 30, 5, 0, 1500, sampler=1)
    orp, ocol, ocnt = oracle.rows(ends, g.n)
    for kernel in (0, 1):
        res = G.run(alpha=0.2, R=30, seed=5, src_end=1500, sampler=1, kernel=kernel)
        rp, col, cnt = res.sparse_rows()
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(cnt, ocnt)
        assert res.info().steps == steps


def test_renumbered_source_lists_and_caller_workspace(ppr, ctx, oracle):
    import torch
    g = _skewed_graph(seed=5)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    ref = oracle_rows(oracle, g, 0.2, 33, 6, topk=4)
    orp, ocol, ocnt = ref["rows"]
    rng = np.random.Generator(np.random.PCG64(2))
    lst = np.concatenate([rng.integers(0, g.n, 500), [0, 0, g.n - 1]]).astype(np.int32)
    res = G.run_list(lst, alpha=0.2, R=33, seed=6, topk=4, max_batch_sources=111)
    lrp, lcol, lcnt = res.sparse_rows()
    lidx, ltc = res.topk()
    for i, s_ in enumerate(lst):
        assert np.array_equal(lcol[lrp[i]:lrp[i + 1]], ocol[orp[s_]:orp[s_ + 1]])
        assert np.array_equal(lcnt[lrp[i]:lrp[i + 1]], ocnt[orp[s_]:orp[s_ + 1]])
        assert np.array_equal(lidx[i], ref["topk"][0][s_]) and np.array_equal(ltc[i], ref["topk"][1][s_])
    # caller workspace, recorded into a CUDA graph and replayed
    dev = torch.device("cuda:0")
    S, cap = 1200, 33
    kw = dict(alpha=0.2, R=33, seed=6, topk=4, src_end=S)
    ws = torch.empty(G.workspace_size(**kw), dtype=torch.uint8, device=dev)
    nnz = torch.zeros(S, dtype=torch.int32, device=dev)
    cols = torch.zeros(S * cap, dtype=torch.int32, device=dev)
    cnts = torch.zeros(S * cap, dtype=torch.int32, device=dev)
    ti = torch.zeros((S, 4), dtype=torch.int32, device=dev)
    tc = torch.zeros((S, 4), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, **kw)
    s.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s, capture_error_mode="thread_local"):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, **kw)
    nnz.zero_()
    cols.fill_(-1)
    cg.replay()
    torch.cuda.synchronize(dev)
    nz = nnz.cpu().numpy().astype(np.int64)
    assert np.array_equal(nz, np.diff(orp[:S + 1]))
    c = cols.cpu().numpy().reshape(S, cap)
    n_ = cnts.cpu().numpy().view(np.uint32).reshape(S, cap)
    keep = np.arange(cap)[None, :] < nz[:, None]
    assert np.array_equal(c[keep], ocol[:orp[S]])
    assert np.array_equal(n_[keep], ocnt[:orp[S]])
    assert np.array_equal(ti.cpu().numpy(), ref["topk"][0][:S])


def test_renumbered_noalloc_and_host_outputs(ppr, ctx, oracle):
    import torch
    g = _skewed_graph(seed=6)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    S, R, K = 900, 21, 5
    ref = oracle_rows(oracle, g, 0.15, R, 3, 0, S, topk=K)
    orp, ocol, ocnt = ref["rows"]
    dev = torch.device("cuda:0")
    cap = R
    nnz = torch.zeros(S, dtype=torch.int32, device=dev)
    cols = torch.zeros(S * cap, dtype=torch.int32, device=dev)
    cnts = torch.zeros(S * cap, dtype=torch.int32, device=dev)
    ti = torch.zeros((S, K), dtype=torch.int32, device=dev)
    tc = torch.zeros((S, K), dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)
    G.run_noalloc(nnz, cols, cnts, cap, ti, tc, alpha=0.15, R=R, seed=3, src_end=S, topk=K, stream=st)
    st.synchronize()
    nz = nnz.cpu().numpy().astype(np.int64)
    assert np.array_equal(nz, np.diff(orp))
    keep = np.arange(cap)[None, :] < nz[:, None]
    assert np.array_equal(cols.cpu().numpy().reshape(S, cap)[keep], ocol)
    assert np.array_equal(ti.cpu().numpy(), ref["topk"][0])
    # pinned host outputs, rows copied batch by batch
    h_rp = torch.empty(S + 1, dtype=torch.int64).pin_memory()
    h_col = torch.empty(S * R, dtype=torch.int32).pin_memory()
    h_cnt = torch.empty(S * R, dtype=torch.int32).pin_memory()
    total, _ = G.run_to_host(h_rp, h_col, h_cnt, alpha=0.15, R=R, seed=3, src_end=S, max_batch_sources=256)
    assert np.array_equal(h_rp.numpy(), orp)
    assert np.array_equal(h_col.numpy()[:total], ocol)
    assert np.array_equal(h_cnt.numpy()[:total].view(np.uint32), ocnt)


@pytest.mark.parametrize("mode", [0, 1])
def test_renumbered_serving(ppr, oracle, mode):
    """Queries served from a renumbered graph (device loop and streams) give
    the oracle's top-k of their sources."""
    g = I.random_small_graph(5000, 50000, seed=61, wmax=50, dangling=50)
    c = ppr.Context(0)
    G = c.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=True)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    ends, _ = oracle.walks(og, 0.15, 40, 7)
    rp, col, cnt = oracle.rows(ends, g.n)
    oidx, ocnt = oracle.topk(rp, col, cnt, 6)
    rng = np.random.Generator(np.random.PCG64(9))
    qs = [rng.choice(g.n, size=int(s), replace=False).astype(np.int32) for s in (1, 17, 400, 2500)]
    c.serve_start(G, streams=2, mode=mode)
    try:
        ids = [c.submit(q, alpha=0.15, R=40, seed=7, topk=6) for q in qs]
        for q, qid in zip(qs, ids):
            idx, cn = c.poll(qid, len(q), 6, timeout_ms=60000)[:2]
            assert np.array_equal(idx, oidx[q]) and np.array_equal(cn, ocnt[q])
    finally:
        c.serve_stop()


def test_numbering_policy_and_flags(ppr, ctx, oracle):
    """Without a flag the layout renumbers when its node records exceed twice
    the L2 (here 2^24 nodes, 512 MiB of records); a small graph keeps the
    caller's order; a wide graph (a row total of 2^32 or more) keeps it too;
    the flags exclude each other and do not apply to batched graphs."""
    small = I.random_small_graph(300, 900, seed=2, wmax=9, dangling=3)
    assert ctx.load_graph(small.n, small.row_ptr, small.col, small.w).info().renumbered == 0
    n = 1 << 24
    rng = np.random.Generator(np.random.PCG64(1))
    row_ptr = np.arange(n + 1, dtype=np.int64)
    col = rng.integers(0, n, n).astype(np.int32)
    w = np.ones(n, dtype=np.uint32)
    Gb = ctx.load_graph(n, row_ptr, col, w)
    assert Gb.info().renumbered == 1
    # a functional graph: each walk follows col; compare a few sources with the oracle
    big = I.Graph(n, row_ptr, col, w)
    ref = oracle_rows(oracle, big, 0.3, 8, 2, 0, 64)
    assert_same(Gb.run(alpha=0.3, R=8, seed=2, src_end=64), ref)
    del Gb
    huge = 2**32 - 5
    gw = I.from_edges(4, [(0, 1, huge), (0, 2, huge), (1, 0, 1), (2, 3, 5), (3, 0, 2)])
    Gw = ctx.load_graph(gw.n, gw.row_ptr, gw.col, gw.w, renumber=True)
    assert Gw.info().wide == 1 and Gw.info().renumbered == 0
    assert_same(Gw.run(alpha=0.25, R=300, seed=3, topk=3), oracle_rows(oracle, gw, 0.25, 300, 3, topk=3), topk=3)
    lib = ppr.lib()
    h = ppr.C.c_void_p()
    rp, cp, wp = small.row_ptr.ctypes.data, small.col.ctypes.data, small.w.ctypes.data
    rc = lib.ppr_load_graph(ctx.h, small.n, small.m, rp, cp, wp, ppr.PPR_RENUMBER | ppr.PPR_KEEP_IDS, None,
                            ppr.C.byref(h))
    assert rc == -1  # PPR_EINVAL
    off = np.array([0, small.n], dtype=np.int64)
    rc = lib.ppr_load_graph_batch(ctx.h, 1, off.ctypes.data, small.m, rp, cp, wp, ppr.PPR_RENUMBER, None,
                                  ppr.C.byref(h))
    assert rc == -1
