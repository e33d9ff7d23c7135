"""The allocation-free entry point (ppr_run_noalloc) against ppr_run.

Callers that cannot allocate device memory mid-run (their device memory is
held by another framework's pool, or a serving loop must not pay for or risk
a driver allocation) pass their own output buffers; the walk endpoints live
in the library's fixed scratch array.  Two calls in a row must each give the
same rows and top-k as ppr_run with the same arguments: counts are integers,
so "the same" is bit-exact.  This file is collected last so that a failure
here does not stop the other GPU tests of a -x run.
"""
import numpy as np
import pytest

from paper_1903_11749_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    import torch
    ctx = ppr.Context(0)
    g = I.random_small_graph(3000, 24000, seed=31, wmax=50, dangling=40)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    return ppr, torch, ctx, g, G


def _noalloc_rows(torch, G, n, S, R, topk, **kw):
    dev = torch.device("cuda:0")
    cap = min(R, n)
    nnz = torch.zeros(S, dtype=torch.int32, device=dev)
    cols = torch.full((S * cap,), -5, dtype=torch.int32, device=dev)
    cnts = torch.zeros(S * cap, dtype=torch.int32, device=dev)
    ti = torch.zeros((S, topk), dtype=torch.int32, device=dev)
    tc = torch.zeros((S, topk), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    G.run_noalloc(nnz, cols, cnts, cap, ti, tc, R=R, topk=topk, stream=stream, **kw)
    stream.synchronize()
    nnz = nnz.cpu().numpy().astype(np.int64)
    cols = cols.cpu().numpy().reshape(S, cap)
    cnts = cnts.cpu().numpy().view(np.uint32).reshape(S, cap)
    row_ptr = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(nnz, out=row_ptr[1:])
    col = np.concatenate([cols[s, : nnz[s]] for s in range(S)])
    cnt = np.concatenate([cnts[s, : nnz[s]] for s in range(S)])
    return row_ptr, col, cnt, ti.cpu().numpy(), tc.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("calls", [[dict(seed=5, src_begin=0, src_end=3000, alpha=0.15),
                                    dict(seed=6, src_begin=100, src_end=2901, alpha=0.3, dangling=1)]])
def test_noalloc_matches_ppr_run_twice(env, calls):
    ppr, torch, ctx, g, G = env
    R, topk = 37, 7
    for kw in calls:  # two calls in a row share the one scratch array
        S = kw["src_end"] - kw["src_begin"]
        rp, col, cnt, ti, tc = _noalloc_rows(torch, G, g.n, S, R, topk, **kw)
        ref = G.run(R=R, topk=topk, **kw)
        orp, ocol, ocnt = ref.sparse_rows()
        oi, oc = ref.topk()
        assert np.array_equal(rp, orp)
        assert np.array_equal(col, ocol)
        assert np.array_equal(cnt, ocnt)
        assert np.array_equal(ti, oi)
        assert np.array_equal(tc, oc)


def test_noalloc_rejects_oversize_calls(env):
    ppr, torch, ctx, g, G = env
    dev = torch.device("cuda:0")
    big = I.random_small_graph(5000, 20000, seed=2)
    Gb = ctx.load_graph(big.n, big.row_ptr, big.col, big.w)
    S, R = 5000, 4096  # 20,480,000 walks: more than the scratch holds, rejected before any work
    nnz = torch.zeros(S, dtype=torch.int32, device=dev)
    cols = torch.zeros(S, dtype=torch.int32, device=dev)
    with pytest.raises(ppr.PPRError) as ei:
        Gb.run_noalloc(nnz, cols, cols, R, R=R)
    assert ei.value.code == ppr.PPR_ERANGE
