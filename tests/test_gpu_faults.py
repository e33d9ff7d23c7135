"""Failure paths, injected on the host (no device fault, trap or hang).

Every device allocation the library makes is made to fail in turn: each call
either succeeds or returns PPR_ENOMEM with a message, the context stays
usable, and once injection is off every result equals the undisturbed run.
A run that has not finished reports PPR_ETIMEOUT at its deadline and
completes normally afterwards."""
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


def _pipeline(ppr, ctx, g):
    """Load, alias tables, segment tables, list run, host-output run; returns
    every result as arrays."""
    out = []
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    for kw in (dict(sampler=1), dict(segments=True), dict()):
        r = G.run(alpha=0.3, R=24, seed=5, topk=3, **kw)
        out += [*r.sparse_rows(), *r.topk()]
    r = G.run_list(np.array([3, 1, 4, 1, 5], dtype=np.int32), alpha=0.3, R=24, seed=5)
    out += list(r.sparse_rows())
    rp = np.empty(g.n + 1, np.int64)
    col = np.empty(g.n * 24, np.int32)
    cnt = np.empty(g.n * 24, np.uint32)
    nnz, _ = G.run_to_host(rp, col, cnt, parts=3, alpha=0.3, R=24, seed=5)
    out += [rp, col[:nnz], cnt[:nnz]]
    return out


def test_every_allocation_failure_is_reported(ppr):
    g = I.random_small_graph(400, 2400, seed=9, wmax=7, dangling=4)
    ctx = ppr.Context(0)
    ref = _pipeline(ppr, ctx, g)
    failures = 0
    try:
        for k in range(120):
            ppr.debug_fail_allocs(k)
            try:
                got = _pipeline(ppr, ctx, g)
            except ppr.PPRError as e:
                assert e.code == ppr.PPR_ENOMEM, e
                assert "injected" in str(e)
                failures += 1
                continue
            finally:
                ppr.debug_fail_allocs(-1)
            # no allocation failed within the budget: the whole pipeline ran
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
            break
    finally:
        ppr.debug_fail_allocs(-1)
    assert failures >= 10
    for a, b in zip(_pipeline(ppr, ctx, g), ref):
        assert np.array_equal(a, b)


def test_deadline_then_completion(ppr):
    g = I.random_small_graph(3000, 30000, seed=2, wmax=5)
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    G.run(alpha=0.5, R=2, seed=1)  # the first launch of a kernel may wait for its module to load
    r = G.run(alpha=0.0002, R=400, seed=1, wait=False)  # ~5000-step walks
    with pytest.raises(ppr.PPRError) as ei:
        r.wait(timeout_ms=0)
    assert ei.value.code == ppr.PPR_ETIMEOUT
    r.wait()
    rp, col, cnt = r.sparse_rows()
    assert (np.add.reduceat(cnt.astype(np.int64), rp[:-1]) == 400).all()


def test_handles_freed_in_any_order(ppr):
    """A context dropped before its graph and result stays alive for them;
    freeing them afterwards leaves no error behind for the next caller."""
    g = I.random_small_graph(300, 2000, seed=4)
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    r = G.run(alpha=0.2, R=16, seed=1, topk=2)
    ctx.close()
    rp, col, cnt = r.sparse_rows()
    assert (np.add.reduceat(cnt.astype(np.int64), rp[:-1]) == 16).all()
    r.free()
    G.free()
    ctx2 = ppr.Context(0)
    G2 = ctx2.load_graph(g.n, g.row_ptr, g.col, g.w)
    r2 = G2.run(alpha=0.2, R=16, seed=1, topk=2)
    for a, b in zip(r2.sparse_rows(), (rp, col, cnt)):
        assert np.array_equal(a, b)
