"""Serving: multi-source queries admitted by continuous batching, in both
modes (the resident device loop, and one launch per query on a few streams).

Each query's top-k must equal the CPU oracle's (walks from each listed
source at tag 0, Sec. 2.1 estimator, top-k order of count then id) when it
runs alone, when it runs in a mix of overlapping queries, and as a
ppr_run_list of the same sources (tolerance 0: the counts are integers).
The device loop's bounded waits are exercised from the host: an idle loop
exits and is launched again by the next query, and a published slot that
was never written makes the loop exit with an error status while the
context stays usable."""
import threading

import numpy as np
import pytest

from paper_1903_11749_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    g = I.random_small_graph(6000, 60000, seed=51, wmax=50, dangling=60)
    return ppr, g


def _oracle_topk(oracle, g, alpha, R, seed, k, sampler=0):
    """Top-k of every node as a source under the oracle; a query's answer is
    the rows of its sources, in the order listed."""
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    ends, _ = oracle.walks(og, alpha, R, seed, sampler=sampler)
    rp, col, cnt = oracle.rows(ends, g.n)
    return oracle.topk(rp, col, cnt, k)


def _same_as_oracle(ref, src, idx, cnt):
    return np.array_equal(idx, ref[0][src]) and np.array_equal(cnt, ref[1][src])


def _queries(n, count, seed, smax=3000):
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.floor(np.exp(rng.uniform(0, np.log(smax), count))).astype(int)
    return [rng.choice(n, size=int(s), replace=False).astype(np.int32) for s in sizes]


MODES = [0, 1]  # ppr.SERVE_DEVICE_LOOP, ppr.SERVE_STREAMS


@pytest.mark.parametrize("mode", MODES)
def test_alone_equals_mix_equals_oracle(env, oracle, mode):
    ppr, g = env
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    qs = _queries(g.n, 24, seed=1)
    kw = dict(alpha=0.15, R=60, seed=7, topk=8)
    ref = _oracle_topk(oracle, g, 0.15, 60, 7, 8)
    ctx.serve_start(G, streams=3, mode=mode)
    alone = []
    for src in qs:
        qid = ctx.submit(src, **kw)
        alone.append(ctx.poll(qid, len(src), kw["topk"], timeout_ms=60000)[:2])
        assert _same_as_oracle(ref, src, *alone[-1])
    # the mix: two submitting threads, then poll everything
    ids = [None] * len(qs)

    def submitter(part):
        for i in part:
            ids[i] = ctx.submit(qs[i], **kw)

    th = [threading.Thread(target=submitter, args=(range(k, len(qs), 2),)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    stats = []
    for i, src in enumerate(qs):
        idx, cnt, st = ctx.poll(ids[i], len(src), kw["topk"], timeout_ms=60000)
        assert np.array_equal(idx, alone[i][0]) and np.array_equal(cnt, alone[i][1])
        assert _same_as_oracle(ref, src, idx, cnt)
        stats.append(st)
    assert all(st["done_ns"] >= st["admit_ns"] >= st["submit_ns"] for st in stats)
    # several queries were in flight at once
    spans = sorted((st["admit_ns"], st["done_ns"]) for st in stats)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    ctx.serve_stop()
    for i, src in enumerate(qs[:6]):
        ref = G.run_list(src, alpha=kw["alpha"], R=kw["R"], seed=kw["seed"], topk=kw["topk"])
        ridx, rcnt = ref.topk()
        assert np.array_equal(ridx, alone[i][0]) and np.array_equal(rcnt, alone[i][1])


@pytest.mark.parametrize("mode", MODES)
def test_memory_admission_and_errors(env, oracle, mode):
    ppr, g = env
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    with pytest.raises(ppr.PPRError):
        ctx.submit(np.arange(5, dtype=np.int32))  # not started
    # a budget that fits one large query at a time: queries wait for memory
    ctx.serve_start(G, streams=4, memory_budget=3 << 20, max_sources=4000, mode=mode)
    qs = _queries(g.n, 10, seed=2, smax=3000)
    kw = dict(alpha=0.2, R=40, seed=3, topk=5)
    ref = _oracle_topk(oracle, g, 0.2, 40, 3, 5)
    ids = [ctx.submit(s, **kw) for s in qs]
    res = [ctx.poll(q, len(s), 5, timeout_ms=60000) for q, s in zip(ids, qs)]
    for (idx, cnt, st), s in zip(res, qs):
        assert _same_as_oracle(ref, s, idx, cnt)
    with pytest.raises(ppr.PPRError):
        ctx.submit(np.array([0, g.n], dtype=np.int32), **kw)  # source out of range
    with pytest.raises(ppr.PPRError):
        ctx.submit(np.arange(10, dtype=np.int32), alpha=0.0)
    with pytest.raises(ppr.PPRError):
        ctx.poll(123456789, 1, 5, timeout_ms=10)  # unknown query
    with pytest.raises(ppr.PPRError) as ei:
        ctx.submit(np.arange(4000, dtype=np.int32), alpha=0.2, R=400, seed=1, topk=5)  # beyond the budget
    assert ei.value.code == ppr.PPR_ERANGE
    big = np.arange(4000, dtype=np.int32)
    q = ctx.submit(big, alpha=0.001, R=40, seed=1, topk=5)  # ~1000-step walks: still running after 0 ms
    with pytest.raises(ppr.PPRError) as ei:
        ctx.poll(q, len(big), 5, timeout_ms=0)
    assert ei.value.code in (ppr.PPR_ETIMEOUT,)
    ctx.poll(q, len(big), 5, timeout_ms=120000)
    # stop with queries waiting: they are cancelled, running ones finish
    for _ in range(6):
        ctx.submit(big, **kw)
    ctx.serve_stop()
    with pytest.raises(ppr.PPRError):
        ctx.poll(1, 1, 5, timeout_ms=10)


@pytest.mark.parametrize("mode", MODES)
def test_alias_sampler_queries_equal_oracle(env, oracle, mode):
    ppr, g = env
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ctx.serve_start(G, streams=2, sampler=1, mode=mode)
    qs = _queries(g.n, 6, seed=9, smax=800)
    kw = dict(alpha=0.15, R=50, seed=11, topk=6)
    ids = [ctx.submit(src, **kw) for src in qs]
    got = [ctx.poll(q, len(src), kw["topk"], timeout_ms=60000)[:2] for q, src in zip(ids, qs)]
    ctx.serve_stop()
    ref = _oracle_topk(oracle, g, 0.15, 50, 11, 6, sampler=1)
    for (idx, cnt), src in zip(got, qs):
        assert _same_as_oracle(ref, src, idx, cnt)
        ridx, rcnt = G.run_list(src, sampler=1, **kw).topk()
        assert np.array_equal(idx, ridx) and np.array_equal(cnt, rcnt)


@pytest.mark.parametrize("mode", MODES)
def test_refilled_warps_serve_the_same_counts(env, oracle, mode):
    """A server whose warps start new walks 24 lanes at a time returns the
    oracle's counts."""
    ppr, g = env
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ctx.serve_start(G, streams=2, refill_lanes=24, mode=mode)
    qs = _queries(g.n, 5, seed=13, smax=900)
    kw = dict(alpha=0.15, R=50, seed=12, topk=6)
    ids = [ctx.submit(src, **kw) for src in qs]
    got = [ctx.poll(q, len(src), kw["topk"], timeout_ms=60000)[:2] for q, src in zip(ids, qs)]
    ctx.serve_stop()
    ref = _oracle_topk(oracle, g, 0.15, 50, 12, 6)
    for (idx, cnt), src in zip(got, qs):
        assert _same_as_oracle(ref, src, idx, cnt)


def test_device_loop_idle_exit_and_relaunch(env, oracle):
    """The resident loop exits after its idle bound with no work; the next
    query launches it again and is served exactly."""
    import time
    ppr, g = env
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ctx.serve_start(G, idle_us=20_000)
    deadline = time.time() + 10
    while ctx.serve_info()["running"] and time.time() < deadline:
        time.sleep(0.01)
    info = ctx.serve_info()
    assert info["running"] == 0 and info["idle_exits"] >= 1 and info["status"] & ppr.LOOP_IDLE
    launches = info["launches"]
    kw = dict(alpha=0.2, R=30, seed=5, topk=4)
    ref = _oracle_topk(oracle, g, 0.2, 30, 5, 4)
    for src in _queries(g.n, 3, seed=21, smax=500):
        idx, cnt, st = ctx.poll(ctx.submit(src, **kw), len(src), 4, timeout_ms=60000)
        assert _same_as_oracle(ref, src, idx, cnt)
    assert ctx.serve_info()["launches"] > launches
    ctx.serve_stop()


def test_device_loop_slot_wait_runs_out(env, oracle):
    """A ring slot published without its descriptor (a host-side test hook):
    the loop's bounded wait ends it with PPR_LOOP_SLOT_TIMEOUT, no GPU fault;
    the server refuses further queries and the context keeps working."""
    import time
    ppr, g = env
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ctx.serve_start(G)
    ctx.debug_serve_publish_unwritten()
    deadline = time.time() + 20
    while time.time() < deadline:
        info = ctx.serve_info()
        if not info["running"] and info["status"] & ppr.LOOP_SLOT_TIMEOUT:
            break
        time.sleep(0.05)
    assert info["status"] & ppr.LOOP_SLOT_TIMEOUT and not info["running"]
    with pytest.raises(ppr.PPRError) as ei:
        ctx.submit(np.arange(5, dtype=np.int32))
    assert ei.value.code == ppr.PPR_ECUDA
    with pytest.raises(ppr.PPRError):
        ctx.serve_stop()  # reports the failed loop, and stops serving
    ref = _oracle_topk(oracle, g, 0.15, 20, 3, 4)
    idx, cnt = G.run(alpha=0.15, R=20, seed=3, topk=4).topk()
    assert np.array_equal(idx, ref[0]) and np.array_equal(cnt, ref[1])
    ctx.serve_start(G)  # serving starts again on the same context
    src = np.arange(0, 50, dtype=np.int32)
    idx, cnt, _ = ctx.poll(ctx.submit(src, alpha=0.15, R=20, seed=3, topk=4), 50, 4, timeout_ms=60000)
    assert _same_as_oracle(ref, src, idx, cnt)
    ctx.serve_stop()


def test_device_loop_limits(env):
    ppr, g = env
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ctx.serve_start(G)
    with pytest.raises(ppr.PPRError) as ei:
        ctx.submit(np.arange(10, dtype=np.int32), R=1025)  # the loop's reduction takes R <= 1024
    assert ei.value.code == ppr.PPR_ERANGE
    assert ctx.serve_info()["mode"] == ppr.SERVE_DEVICE_LOOP
    ctx.serve_stop()
    with pytest.raises(ppr.PPRError):
        ctx.serve_start(G, mode=2)
