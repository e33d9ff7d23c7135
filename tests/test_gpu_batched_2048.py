"""The batched workload at its own size: 2,048 independent Chung-Lu graphs
(exponent 2.3, n log-uniform in [100, 50,000], mean degree 12, integer
weights U[1,100]; alpha 0.15, R 200, top-32) walked in one fused persistent
launch in the autotuner's launch shape, recorded as a CUDA graph and
replayed.  Every 64th instance, plus the smallest and the largest, is
recomputed by the CPU oracle on that instance alone with the instance id as
tag (Algorithm 2's walks, Sec. 2.1 estimator) and compared exactly, row by
row and top-k by top-k; every row of the launch sums to R."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1903_11749_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ALPHA, R, SEED, K = 0.15, 200, 1, 32


@pytest.fixture(scope="module")
def ppr():
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr as P
    return P


@pytest.fixture(scope="module")
def c4(ppr):
    inst = I.chung_lu_instances(2048, 100, 50_000, 12.0, 2.3, 1, 100, seed=4242)
    ctx = ppr.Context(0)
    G = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
    return inst, ctx, G


def _oracle_instance(oracle, inst, gi, sampler):
    sub = inst.instance(gi)
    og = oracle.prepare(sub.n, sub.row_ptr, sub.col, sub.w)
    ends, _ = oracle.walks(og, ALPHA, R, SEED, tag=gi, sampler=sampler)  # ctypes drops the GIL here
    rp, col, cnt = oracle.rows(ends, sub.n)
    return gi, (rp, col, cnt), oracle.topk(rp, col, cnt, K)


@pytest.mark.parametrize("sampler", [0, 1])
def test_2048_instances_one_fused_replayed_launch(ppr, oracle, c4, sampler):
    import torch
    dev = torch.device("cuda:0")
    inst, ctx, G = c4
    ns = np.diff(inst.node_off)
    N = int(inst.node_off[-1])
    kw = dict(alpha=ALPHA, R=R, seed=SEED, topk=K, sampler=sampler)
    t = G.autotune(sample_sources=200_000, **kw)
    kw.update(chunk_sources=t["chunk_sources"], large_degree=t["large_degree"],
              warps_per_block=t["warps_per_block"], refill_lanes=t["refill_lanes"])
    cap = min(R, int(ns.max()))
    ws = torch.empty(G.workspace_size(**kw), dtype=torch.uint8, device=dev)
    nnz = torch.zeros(N, dtype=torch.int32, device=dev)
    cols = torch.zeros(N * cap, dtype=torch.int32, device=dev)
    cnts = torch.zeros(N * cap, dtype=torch.int32, device=dev)
    ti = torch.zeros((N, K), dtype=torch.int32, device=dev)
    tc = torch.zeros((N, K), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, **kw)  # tables built, kernels loaded
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, **kw)
    sample = sorted(set(range(0, inst.count, 64)) | {int(ns.argmin()), int(ns.argmax())})
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as pool:
        futs = [pool.submit(_oracle_instance, oracle, inst, gi, sampler) for gi in sample]
        for rep in range(2):
            nnz.zero_()
            cols.fill_(-1)
            cnts.zero_()
            ti.fill_(-7)
            graph.replay()
            torch.cuda.synchronize(dev)
            rows = cnts.view(N, cap).sum(dim=1, dtype=torch.int64)
            assert bool((rows == R).all())  # every row of every instance holds its R walks
            assert bool((nnz >= 1).all()) and bool((nnz <= cap).all())
        for f in futs:
            gi, (orp, ocol, ocnt), (oti, otc) = f.result()
            a, b = int(inst.node_off[gi]), int(inst.node_off[gi + 1])
            nz = nnz[a:b].cpu().numpy().astype(np.int64)
            assert np.array_equal(nz, np.diff(orp))
            c = cols[a * cap: b * cap].view(b - a, cap).cpu().numpy()
            n_ = cnts[a * cap: b * cap].view(b - a, cap).cpu().numpy().view(np.uint32)
            keep = np.arange(cap)[None, :] < nz[:, None]
            assert np.array_equal(c[keep], ocol)
            assert np.array_equal(n_[keep], ocnt)
            assert np.array_equal(ti[a:b].cpu().numpy(), oti)
            assert np.array_equal(tc[a:b].cpu().numpy().view(np.uint32), otc)
