"""Accuracy evaluation (the Sec. 5.2 analog) and the Definition 1 walk count.

CPU: the FP64 ground truth against exact rational pi, the ranking metrics on
hand-worked rankings, and the walk count against exact binomial tails.
GPU: estimates from the CUDA path meet Definition 1 at the walk count the
library derives, and their rankings improve with R.
"""
import math

import numpy as np
import pytest

import exact_ppr as X
from paper_1903_11749_gb300 import accuracy as A
from paper_1903_11749_gb300 import inputs as I


def _graphs():
    return [I.from_edges(6, [(0, 1, 1000), (0, 2, 1), (0, 1, 3), (1, 1, 2), (1, 3, 5), (2, 0, 1),
                             (2, 4, 7), (3, 0, 1), (3, 5, 1), (4, 2, 2)]),
            I.random_small_graph(8, 16, seed=4, wmax=9, dangling=2)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("gi", [0, 1])
def test_fp64_truth_equals_exact_rational_pi(gi, mode):
    g = _graphs()[gi]
    T = int(0.2 * 2**32)
    exact = X.exact_pi(g.n, g.row_ptr, g.col, g.w, T, mode)
    got = A.exact_ppr_rows(g.n, g.row_ptr, g.col, g.w, np.arange(g.n), T, dangling=mode, tol=1e-15)
    want = np.array([[float(p) for p in row] for row in exact])
    assert np.abs(got - want).max() < 1e-12
    assert np.allclose(got.sum(axis=1), 1.0, atol=1e-12)


def test_ndcg_and_average_precision_by_hand():
    truth = [5, 3, 9, 1]
    assert A.ndcg_at_k([5, 3, 9, 1], truth, 4) == pytest.approx(1.0)
    assert A.average_precision_at_k([5, 3, 9, 1], truth, 4) == pytest.approx(1.0)
    assert A.ndcg_at_k([7, 8, 2, 0], truth, 4) == 0.0
    # hits at positions 2 and 4 of 4: DCG = 1/log2(3) + 1/log2(5)
    dcg = 1 / math.log2(3) + 1 / math.log2(5)
    idcg = 1 + 1 / math.log2(3) + 1 / math.log2(4) + 1 / math.log2(5)
    assert A.ndcg_at_k([7, 3, 8, 9], truth, 4) == pytest.approx(dcg / idcg)
    # precision 1/2 at position 2, 2/4 at position 4, two relevant items missed
    assert A.average_precision_at_k([7, 3, 8, 9], truth, 4) == pytest.approx((1 / 2 + 2 / 4) / 4)
    # k cuts both lists; a short prediction is scored against the ideal of min(k, |rel|)
    assert A.ndcg_at_k([5], truth, 2) == pytest.approx(1 / (1 + 1 / math.log2(3)))
    assert A.average_precision_at_k([3, 5, 1], truth, 2) == pytest.approx(1.0)


def test_exact_topk_order_and_ties():
    pi = np.array([0.1, 0.3, 0.0, 0.3, 0.05, 0.25])
    assert A.exact_topk(pi, 4).tolist() == [1, 3, 5, 0]
    assert A.exact_topk(pi, 10).tolist() == [1, 3, 5, 0, 4]


@pytest.mark.parametrize("eps,delta,p_f", [(0.5, 0.01, 0.01), (0.5, 0.001, 0.1), (0.2, 0.05, 0.001),
                                           (1.0, 0.1, 0.05), (0.1, 0.2, 0.01)])
def test_walk_count_meets_definition1_by_exact_binomial_tails(eps, delta, p_f):
    """For the omega the library returns, a pair with pi = delta (the hardest
    case) and larger ones miss by more than eps * pi with probability <= p_f,
    computed exactly from the binomial law of the count."""
    from scipy.stats import binom
    from paper_1903_11749_gb300 import ppr
    omega = ppr.walks_for_accuracy(eps, delta, p_f)
    assert omega == math.ceil((2 + 2 * eps / 3) * math.log(2 / p_f) / (eps * eps * delta))
    for pi in (delta, 2 * delta, min(1.0, 10 * delta)):
        if pi >= 1.0:
            continue
        mu = omega * pi
        tail = binom.cdf(math.ceil(mu * (1 - eps)) - 1, omega, pi) + binom.sf(math.floor(mu * (1 + eps)), omega, pi)
        assert tail <= p_f
    assert A.delta_for_walks(omega, eps, p_f) <= delta
    assert ppr.walks_for_accuracy(eps, delta / 2, p_f) >= 2 * omega - 1


def test_walk_count_rejects_bad_parameters():
    from paper_1903_11749_gb300 import ppr
    for args in [(0.0, 0.1, 0.1), (0.5, 0.0, 0.1), (0.5, 1.5, 0.1), (0.5, 0.1, 1.0), (0.5, 0.1, 0.0)]:
        with pytest.raises(ppr.PPRError):
            ppr.walks_for_accuracy(*args)
    with pytest.raises(ppr.PPRError):
        ppr.walks_for_accuracy(1e-9, 1e-9, 0.5)  # beyond 2^53


@pytest.mark.gpu
def test_gpu_estimates_meet_definition1_and_rank_better_with_R():
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    g = I.chung_lu_graph(5000, avg_deg=8.0, seed=77)
    T = ppr.alpha_threshold(0.15)
    src = np.arange(0, g.n, 50, dtype=np.int32)
    pi = A.exact_ppr_rows(g.n, g.row_ptr, g.col, g.w, src, T)
    ctx = ppr.Context(0)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    k = 10
    ndcg = {}
    for R in (64, 4096):
        res = G.run_list(src, alpha=0.15, R=R, seed=3, topk=k)
        idx, cnt = res.topk()
        ndcg[R] = np.mean([A.ndcg_at_k(A.estimated_ranking(idx[i], cnt[i]), A.exact_topk(pi[i], k), k)
                           for i in range(len(src))])
    assert ndcg[4096] > ndcg[64] and ndcg[4096] > 0.9
    # Definition 1 at eps = 0.5, p_f = 0.01 with 4 runs of 4096 walks summed over tags
    eps, p_f, R, runs = 0.5, 0.01, 4096, 4
    delta = A.delta_for_walks(R * runs, eps, p_f)
    assert ppr.walks_for_accuracy(eps, delta, p_f) <= R * runs
    est = np.zeros((len(src), g.n))
    for tag in range(runs):
        rp, col, c = G.run_list(src, alpha=0.15, R=R, seed=3, tag=tag).sparse_rows()
        rows = np.repeat(np.arange(len(src)), np.diff(rp))
        np.add.at(est, (rows, col), c)
    est /= R * runs
    bad, pairs = A.definition1_violations(est, pi, eps, delta)
    assert pairs > 50
    # each pair fails with probability <= p_f; allow the binomial 99.9 % upper quantile
    from scipy.stats import binom
    assert bad <= binom.ppf(0.999, pairs, p_f)
