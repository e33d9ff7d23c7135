"""Accuracy of the Monte Carlo estimates against exact PPR (host-side evaluation).

Nothing here is on the walk path: it scores results the CUDA library produced.

Ground truth is FP64 power iteration of the law the walks sample (Sec. 2.1):
each step moves to an out-neighbour with probability w(e)/W_u and then stops
with probability t = T / 2^32, T = floor(alpha * 2^32); at a node without
out-edges, mode 0 moves to the source (the step counts) and mode 1 ends the
walk there without a step.  The scores follow the paper's accuracy
experiment (Sec. 5.2): per source, nodes are ranked by pi, the first k of each
ranking are kept, and the estimate's ranking is scored against the exact one
with NDCG@k and average precision under binary relevance (relevant = the exact
top k), the definitions of the ranking-metrics library the paper cites.  The
(eps, delta) check is Definition 1 applied pair by pair.
"""
from __future__ import annotations

import math

import numpy as np


def transition(n: int, row_ptr, col, w):
    """Row-stochastic sparse P (scipy CSR, parallel edges summed) and the mask
    of nodes without out-edges."""
    from scipy.sparse import csr_matrix
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(row_ptr)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    wf = np.asarray(w, dtype=np.float64)
    Wu = np.zeros(n, dtype=np.float64)
    np.add.at(Wu, src, wf)
    P = csr_matrix((wf / Wu[src], (src, np.asarray(col, dtype=np.int64))), shape=(n, n))
    P.sum_duplicates()
    return P, deg == 0


def exact_ppr_rows(n: int, row_ptr, col, w, sources, T: int, dangling: int = 0, tol: float = 1e-13):
    """pi(s, .) in FP64 for each s in `sources`: float64[len(sources), n].

    A_0 = e_s holds the walks still active; each round (mode 1 first ends the
    active mass sitting on dangling nodes) moves A one step, Y = A P (mode 0
    adds the mass on dangling nodes to column s), ends t * Y and keeps
    (1 - t) * Y active, until the active mass is below tol."""
    P, dang = transition(n, row_ptr, col, w)
    PT = P.T.tocsr()
    t = T / 2.0 ** 32
    src = np.asarray(sources, dtype=np.int64)
    S = len(src)
    A = np.zeros((n, S), dtype=np.float64)  # column i: walks of source i
    A[src, np.arange(S)] = 1.0
    pi = np.zeros((n, S), dtype=np.float64)
    has_dang = bool(dang.any())
    while True:
        if has_dang and dangling == 1:
            pi[dang] += A[dang]
            A[dang] = 0.0
        Y = PT @ A
        if has_dang and dangling == 0:
            Y[src, np.arange(S)] += A[dang].sum(axis=0)
        pi += t * Y
        A = (1.0 - t) * Y
        if A.sum(axis=0).max() < tol:
            break
    return pi.T.copy()


def exact_topk(pi_row, k: int) -> np.ndarray:
    """The first k nodes of the exact ranking (pi descending, ties by smaller
    id; nodes with pi = 0 are not ranked)."""
    pi_row = np.asarray(pi_row)
    nz = np.flatnonzero(pi_row > 0)
    order = np.lexsort((nz, -pi_row[nz]))
    return nz[order[:k]]


def estimated_ranking(idx_row, cnt_row) -> np.ndarray:
    """A top-k row as the library returns it (count descending, ties by id,
    padding -1) as a ranking without the padding."""
    idx_row = np.asarray(idx_row)
    return idx_row[(idx_row >= 0) & (np.asarray(cnt_row) > 0)]


def ndcg_at_k(pred, relevant_ranked, k: int) -> float:
    """NDCG@k with binary relevance: DCG = sum over the first n = min(max(|pred|,
    |rel|), k) positions i of [pred_i in rel] / log2(i + 2); the ideal DCG puts
    the |rel| relevant items first."""
    rel = set(int(x) for x in relevant_ranked[:k])
    if not rel:
        return 0.0
    pred = [int(x) for x in pred[:k]]
    n = min(max(len(pred), len(rel)), k)
    dcg = sum(1.0 / math.log2(i + 2) for i in range(min(n, len(pred))) if pred[i] in rel)
    idcg = sum(1.0 / math.log2(i + 2) for i in range(min(n, len(rel))))
    return dcg / idcg


def average_precision_at_k(pred, relevant_ranked, k: int) -> float:
    """Average precision of the first k predictions against the relevant set
    (the exact top k): the mean over relevant items of the precision at the
    position where each is found, unfound ones counting 0."""
    rel = set(int(x) for x in relevant_ranked[:k])
    if not rel:
        return 0.0
    hits, acc = 0, 0.0
    for i, x in enumerate(pred[:k]):
        if int(x) in rel:
            hits += 1
            acc += hits / (i + 1)
    return acc / len(rel)


def definition1_violations(est, pi, eps: float, delta: float):
    """(violations, pairs): among pairs with pi >= delta, those whose estimate
    misses pi by more than eps * pi (Definition 1)."""
    est = np.asarray(est, dtype=np.float64)
    pi = np.asarray(pi, dtype=np.float64)
    mask = pi >= delta
    bad = np.abs(est[mask] - pi[mask]) > eps * pi[mask]
    return int(bad.sum()), int(mask.sum())


def delta_for_walks(R: int, eps: float, p_f: float) -> float:
    """The smallest delta that R walks cover under the bound of
    ppr_walks_for_accuracy (its inverse in delta)."""
    return (2.0 + 2.0 * eps / 3.0) * math.log(2.0 / p_f) / (eps * eps * R)
