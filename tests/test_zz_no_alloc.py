"""The allocation-free entry point (ppr_run_noalloc) against the oracle and
against ppr_run.

Callers that cannot allocate device memory mid-run (their device memory is
held by another framework's pool, or a serving loop must not pay for or risk
a driver allocation) pass their own output buffers; the walk endpoints live
in the library's fixed scratch array.  Two calls in a row must each give the
rows and top-k of the CPU oracle and of ppr_run with the same arguments:
counts are integers, so "the same" is bit-exact.  While a call is queued,
every device allocation of the library is made to fail (host-side fault
injection), so a call that allocated anything would return PPR_ENOMEM.
This file is collected last so that a failure here does not stop the other
GPU tests of a -x run.
"""
import numpy as np
import pytest

from paper_1903_11749_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R, TOPK = 37, 7


@pytest.fixture(scope="module")
def env(oracle):
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    import torch
    ctx = ppr.Context(0)
    g = I.random_small_graph(3000, 24000, seed=31, wmax=50, dangling=40)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    return ppr, torch, ctx, g, G, og


def _noalloc_rows(ppr, torch, G, n, S, **kw):
    dev = torch.device("cuda:0")
    cap = min(R, n)
    nnz = torch.zeros(S, dtype=torch.int32, device=dev)
    cols = torch.full((S * cap,), -5, dtype=torch.int32, device=dev)
    cnts = torch.zeros(S * cap, dtype=torch.int32, device=dev)
    ti = torch.zeros((S, TOPK), dtype=torch.int32, device=dev)
    tc = torch.zeros((S, TOPK), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    stream.synchronize()
    ppr.debug_fail_allocs(0)  # any device allocation by the library now fails with PPR_ENOMEM
    try:
        G.run_noalloc(nnz, cols, cnts, cap, ti, tc, R=R, topk=TOPK, stream=stream, **kw)
    finally:
        ppr.debug_fail_allocs(-1)
    stream.synchronize()
    nnz = nnz.cpu().numpy().astype(np.int64)
    cols = cols.cpu().numpy().reshape(S, cap)
    cnts = cnts.cpu().numpy().view(np.uint32).reshape(S, cap)
    row_ptr = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(nnz, out=row_ptr[1:])
    col = np.concatenate([cols[s, : nnz[s]] for s in range(S)])
    cnt = np.concatenate([cnts[s, : nnz[s]] for s in range(S)])
    return row_ptr, col, cnt, ti.cpu().numpy(), tc.cpu().numpy().view(np.uint32)


def _oracle(oracle, og, g, kw):
    ends, _ = oracle.walks(og, kw["alpha"], R, kw["seed"], kw["src_begin"], kw["src_end"], kw.get("tag", 0),
                           kw.get("dangling", 0), kw.get("segments", False), sampler=kw.get("sampler", 0))
    rp, col, cnt = oracle.rows(ends, g.n)
    return (rp, col, cnt, *oracle.topk(rp, col, cnt, TOPK))


def _check_twice(env, oracle, calls):
    ppr, torch, ctx, g, G, og = env
    for kw in calls:  # calls in a row share the one scratch array
        S = kw["src_end"] - kw["src_begin"]
        got = _noalloc_rows(ppr, torch, G, g.n, S, **kw)
        ref = G.run(R=R, topk=TOPK, **kw)
        for a_, b_ in zip(got, (*ref.sparse_rows(), *ref.topk())):
            assert np.array_equal(a_, b_)
        for a_, b_ in zip(got, _oracle(oracle, og, g, kw)):
            assert np.array_equal(a_, b_)


def test_noalloc_matches_oracle_and_ppr_run_twice(env, oracle):
    _check_twice(env, oracle, [dict(seed=5, src_begin=0, src_end=3000, alpha=0.15),
                               dict(seed=6, src_begin=100, src_end=2901, alpha=0.3, dangling=1, tag=3)])


def test_noalloc_segment_tables_and_alias_sampler(env, oracle):
    """Segment mode and the alias sampler, with their tables built by an
    earlier ppr_run (the allocation-free call builds nothing)."""
    ppr, torch, ctx, g, G, og = env
    G.run(alpha=0.2, R=1, seed=1, src_begin=0, src_end=1, segments=True)  # builds the tables for alpha 0.2
    G.run(alpha=0.2, R=1, seed=1, src_begin=0, src_end=1, sampler=1)      # builds the alias tables
    _check_twice(env, oracle, [dict(seed=8, src_begin=0, src_end=3000, alpha=0.2, segments=True),
                               dict(seed=9, src_begin=17, src_end=2999, alpha=0.2, sampler=1, refill_lanes=24)])


def test_noalloc_needs_prebuilt_tables(env):
    ppr, torch, ctx, g, G, og = env
    dev = torch.device("cuda:0")
    fresh = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    nnz = torch.zeros(g.n, dtype=torch.int32, device=dev)
    cols = torch.zeros(g.n * R, dtype=torch.int32, device=dev)
    for kw in (dict(segments=True, alpha=0.25), dict(sampler=1)):
        with pytest.raises(ppr.PPRError) as ei:
            fresh.run_noalloc(nnz, cols, cols, R, R=R, **kw)
        assert ei.value.code == ppr.PPR_ENOTSUP
    # the same argument limits as ppr_run
    for kw, code in ((dict(refill_lanes=33), ppr.PPR_EINVAL), (dict(warps_per_block=33), ppr.PPR_EINVAL),
                     (dict(chunk_sources=30000), ppr.PPR_ERANGE)):
        with pytest.raises(ppr.PPRError) as ei:
            fresh.run_noalloc(nnz, cols, cols, R, R=R, **kw)
        assert ei.value.code == code, kw


def test_noalloc_rejects_oversize_calls(env):
    ppr, torch, ctx, g, G, og = env
    dev = torch.device("cuda:0")
    big = I.random_small_graph(5000, 20000, seed=2)
    Gb = ctx.load_graph(big.n, big.row_ptr, big.col, big.w)
    S, RR = 5000, 4096  # 20,480,000 walks: more than the scratch holds, rejected before any work
    nnz = torch.zeros(S, dtype=torch.int32, device=dev)
    cols = torch.zeros(S, dtype=torch.int32, device=dev)
    with pytest.raises(ppr.PPRError) as ei:
        Gb.run_noalloc(nnz, cols, cols, RR, R=RR)
    assert ei.value.code == ppr.PPR_ERANGE
