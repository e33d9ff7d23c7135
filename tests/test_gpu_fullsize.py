"""Full-size parity: every source of the R-MAT scale-20 workload (1,048,576
sources, R 100, alpha 0.2, top-32) on the GPU against the oracle run over
the same sources, in source ranges on host threads (the oracle's C walk loop
releases the interpreter lock; the ranges are independent because every draw
is keyed by (source, walk, step)).  Both samplers; counts, rows, top-k and
the number of draws are compared exactly."""
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1903_11749_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def graph():
    return I.workload_graph("rmat20")


@pytest.mark.parametrize("sampler", [0, 1])
def test_rmat20_every_source_equals_threaded_oracle(oracle, graph, sampler):
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    g = graph
    kw = dict(alpha=0.2, R=100, seed=1)
    G = ppr.Context(0).load_graph(g.n, g.row_ptr, g.col, g.w)
    res = G.run(topk=32, sampler=sampler, **kw)
    rp, col, cnt = res.sparse_rows()
    idx, tc = res.topk()
    steps_gpu = res.info().steps

    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    if sampler == 1:
        oracle.build_alias(og)  # once, before the threads share the graph
    block = 1 << 15
    ranges = [(a, min(g.n, a + block)) for a in range(0, g.n, block)]

    def check(r):
        a, b = r
        ends, steps = oracle.walks(og, kw["alpha"], kw["R"], kw["seed"], a, b, sampler=sampler)
        orp, ocol, ocnt = oracle.rows(ends, g.n)
        oidx, otc = oracle.topk(orp, ocol, ocnt, 32)
        ok = (np.array_equal(rp[a:b + 1] - rp[a], orp) and np.array_equal(col[rp[a]:rp[b]], ocol)
              and np.array_equal(cnt[rp[a]:rp[b]], ocnt) and np.array_equal(idx[a:b], oidx)
              and np.array_equal(tc[a:b], otc))
        return ok, steps

    threads = min(32, os.cpu_count() or 1)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        out = list(ex.map(check, ranges))
    dt = time.perf_counter() - t0
    bad = [r for r, (ok, _) in zip(ranges, out) if not ok]
    assert not bad, f"ranges differing from the oracle: {bad[:5]}"
    assert sum(s for _, s in out) == steps_gpu
    print(f"oracle over {g.n} sources on {threads} threads: {dt:.1f} s ({steps_gpu / dt / 1e6:.1f} M steps/s)")


@pytest.mark.skipif(os.environ.get("PPR_FULLSIZE_C3") != "1",
                    reason="several minutes of host oracle time; set PPR_FULLSIZE_C3=1 to run")
@pytest.mark.parametrize("mode", ["segments", "alias"])
def test_rmat24_every_source_equals_threaded_oracle(oracle, mode):
    """The scale-24 workload (16,777,216 sources, R 50, alpha 0.15, hub of
    1.57 M edges): every source against the oracle in source ranges on host
    threads, with depth-3 segment tables (the oracle builds every table up
    front, so the threads only read them) or with alias tables, each in the
    launch shape the benchmark times (segments: refill 16)."""
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    g = I.workload_graph("rmat24")
    kw = dict(alpha=0.15, R=50, seed=1)
    seg, sampler = (True, 0) if mode == "segments" else (False, 1)
    G = ppr.Context(0).load_graph(g.n, g.row_ptr, g.col, g.w)
    res = G.run(segments=seg, sampler=sampler, refill_lanes=16 if seg else 0, **kw)
    rp, col, cnt = res.sparse_rows()
    steps_gpu = res.info().steps
    del res, G
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    if seg:
        oracle.build_segments(og, oracle.threshold(kw["alpha"]))
    else:
        oracle.build_alias(og)
    block = 1 << 16
    ranges = [(a, min(g.n, a + block)) for a in range(0, g.n, block)]

    def check(r):
        a, b = r
        ends, steps = oracle.walks(og, kw["alpha"], kw["R"], kw["seed"], a, b, segments=seg, sampler=sampler)
        orp, ocol, ocnt = oracle.rows(ends, g.n)
        ok = (np.array_equal(rp[a:b + 1] - rp[a], orp) and np.array_equal(col[rp[a]:rp[b]], ocol)
              and np.array_equal(cnt[rp[a]:rp[b]], ocnt))
        return ok, steps

    threads = min(32, os.cpu_count() or 1)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        out = list(ex.map(check, ranges))
    dt = time.perf_counter() - t0
    bad = [r for r, (ok, _) in zip(ranges, out) if not ok]
    assert not bad, f"ranges differing from the oracle: {bad[:5]}"
    assert sum(s for _, s in out) == steps_gpu
    print(f"oracle over {g.n} sources ({mode}) on {threads} threads: {dt:.1f} s ({steps_gpu / dt / 1e6:.1f} M draws/s)")


@pytest.mark.skipif(os.environ.get("PPR_FULLSIZE_C4") != "1",
                    reason="several minutes of host oracle time; set PPR_FULLSIZE_C4=1 to run")
@pytest.mark.parametrize("sampler", [0, 1])
def test_chunglu2048_every_source_equals_threaded_oracle(oracle, sampler):
    """The 2,048-instance batched workload (16.3 M sources, R 200, alpha 0.15,
    top-32) in one fused launch: every instance against the oracle run on
    that instance alone with its id as the tag, instances spread over host
    threads."""
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    inst = I.chung_lu_instances(2048, 100, 50_000, 12.0, 2.3, 1, 100, seed=4242)
    kw = dict(alpha=0.15, R=200, seed=1)
    G = ppr.Context(0).load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
    res = G.run(topk=32, sampler=sampler, chunk_sources=8, refill_lanes=8, **kw)  # the tuner's launch shape
    rp, col, cnt = res.sparse_rows()
    idx, tc = res.topk()
    steps_gpu = res.info().steps
    del res, G

    def check(gi):
        sub = inst.instance(gi)
        og = oracle.prepare(sub.n, sub.row_ptr, sub.col, sub.w)
        ends, steps = oracle.walks(og, kw["alpha"], kw["R"], kw["seed"], tag=gi, sampler=sampler)
        orp, ocol, ocnt = oracle.rows(ends, sub.n)
        oidx, otc = oracle.topk(orp, ocol, ocnt, 32)
        a, b = int(inst.node_off[gi]), int(inst.node_off[gi + 1])
        ok = (np.array_equal(rp[a:b + 1] - rp[a], orp) and np.array_equal(col[rp[a]:rp[b]], ocol)
              and np.array_equal(cnt[rp[a]:rp[b]], ocnt) and np.array_equal(idx[a:b], oidx)
              and np.array_equal(tc[a:b], otc))
        return ok, steps

    threads = min(32, os.cpu_count() or 1)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        out = list(ex.map(check, range(inst.count)))
    dt = time.perf_counter() - t0
    bad = [gi for gi, (ok, _) in enumerate(out) if not ok]
    assert not bad, f"instances differing from the oracle: {bad[:5]}"
    assert sum(s for _, s in out) == steps_gpu
    print(f"oracle over {inst.count} instances ({int(inst.node_off[-1])} sources, sampler {sampler}) on "
          f"{threads} threads: {dt:.1f} s ({steps_gpu / dt / 1e6:.1f} M draws/s)")
