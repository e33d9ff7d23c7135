"""ppr_run_to_host: rows and top-k written straight to host memory, the output
copies of each batch pipelined against the next batch's walks.  Every split
gives exactly the rows and top-k of the CPU oracle (and of ppr_run) on the
same arguments."""
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


def _host_run(G, S, R, k, parts, pinned, **kw):
    import torch
    cap = S * R
    if pinned:
        rp = torch.empty(S + 1, dtype=torch.int64).pin_memory()
        col = torch.empty(cap, dtype=torch.int32).pin_memory()
        cnt = torch.empty(cap, dtype=torch.int32).pin_memory()
        ti = torch.empty((S, k), dtype=torch.int32).pin_memory() if k else None
        tc = torch.empty((S, k), dtype=torch.int32).pin_memory() if k else None
    else:
        rp = np.empty(S + 1, dtype=np.int64)
        col = np.empty(cap, dtype=np.int32)
        cnt = np.empty(cap, dtype=np.uint32)
        ti = np.empty((S, k), dtype=np.int32) if k else None
        tc = np.empty((S, k), dtype=np.uint32) if k else None
    nnz, info = G.run_to_host(rp, col, cnt, ti, tc, parts=parts, R=R, topk=k, **kw)
    conv = (lambda x: x.numpy()) if pinned else (lambda x: x)
    out = [conv(rp), conv(col)[:nnz], conv(cnt)[:nnz].view(np.uint32)]
    if k:
        out += [conv(ti), conv(tc).view(np.uint32)]
    return nnz, info, out


@pytest.mark.parametrize("parts,pinned,segments", [(1, True, False), (3, True, False), (7, False, False),
                                                   (0, True, False), (4, True, True)])
def test_run_to_host_equals_oracle(ppr, ctx, oracle, parts, pinned, segments):
    g = I.random_small_graph(3001, 24000, seed=61, wmax=30, dangling=25)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    kw = dict(alpha=0.2, seed=4, src_begin=5, src_end=2990, segments=segments)
    S, R, k = 2985, 37, 6
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    ends, steps = oracle.walks(og, 0.2, R, 4, 5, 2990, segments=segments)
    rp0, col0, cnt0 = oracle.rows(ends, g.n)
    ti0, tc0 = oracle.topk(rp0, col0, cnt0, k)
    nnz, info, got = _host_run(G, S, R, k, parts, pinned, **kw)
    assert nnz == len(col0)
    for a_, b_ in zip(got, (rp0, col0, cnt0, ti0, tc0)):
        assert np.array_equal(a_, b_)
    assert info.steps == steps and info.walks == S * R and info.kernel_ms > 0
    ref = G.run(R=R, topk=k, **kw)
    for a_, b_ in zip(got, (*ref.sparse_rows(), *ref.topk())):
        assert np.array_equal(a_, b_)


def test_run_to_host_batched_graph_and_alias(ppr, ctx, oracle):
    """Each instance's rows equal the oracle run on that instance alone with
    the instance id as tag (both samplers)."""
    inst = I.chung_lu_instances(count=9, nmin=30, nmax=600, seed=12)
    G = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
    N = int(inst.node_off[-1])
    for sampler in (0, 1):
        nnz, _, (rp, col, cnt, ti, tc) = _host_run(G, N, 40, 4, 4, True, alpha=0.15, seed=2, sampler=sampler)
        for gi in range(inst.count):
            sub = inst.instance(gi)
            og = oracle.prepare(sub.n, sub.row_ptr, sub.col, sub.w)
            ends, _ = oracle.walks(og, 0.15, 40, 2, tag=gi, sampler=sampler)
            orp, ocol, ocnt = oracle.rows(ends, sub.n)
            oti, otc = oracle.topk(orp, ocol, ocnt, 4)
            a, b = int(inst.node_off[gi]), int(inst.node_off[gi + 1])
            assert np.array_equal(rp[a: b + 1] - rp[a], orp)
            assert np.array_equal(col[rp[a]: rp[b]], ocol) and np.array_equal(cnt[rp[a]: rp[b]], ocnt)
            assert np.array_equal(ti[a:b], oti) and np.array_equal(tc[a:b], otc)


def test_run_to_host_capacity_and_arguments(ppr, ctx):
    g = I.random_small_graph(500, 4000, seed=3)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    rp = np.empty(501, dtype=np.int64)
    col = np.empty(10, dtype=np.int32)
    cnt = np.empty(10, dtype=np.uint32)
    with pytest.raises(ppr.PPRError) as ei:
        G.run_to_host(rp, col, cnt, parts=2, alpha=0.2, R=20, seed=1)
    assert ei.value.code == ppr.PPR_ERANGE
    with pytest.raises(ppr.PPRError):  # top-k requested without buffers
        G.run_to_host(rp, np.empty(10000, np.int32), np.empty(10000, np.uint32), alpha=0.2, R=20, seed=1, topk=3)
    # the context stays usable
    nnz, _, _ = _host_run(G, 500, 20, 0, 2, False, alpha=0.2, seed=1)
    assert nnz == len(G.run(alpha=0.2, R=20, seed=1).sparse_rows()[1])
