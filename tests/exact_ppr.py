"""Ground truth for the oracle pins: exact rational PPR, brute-force path
enumeration, and FP64 power iteration.

The quantity is the endpoint law of the walk of Sec. 2.1: from the current
node move along an out-edge chosen with probability w(e)/W_u, then stop with
probability t (move-then-stop, so every walk has at least one step).  A node
with no out-edge sends the walk back to its head (mode 0, as Sec. 2.1 states),
or ends the walk in place (mode 1).  With t = T / 2^32 (T = floor(alpha*2^32))
these are the laws the integer sampler realises.

Mode 0, P_s = P with dangling rows replaced by the unit row of s:
    pi_s = t * e_s P_s (I - (1-t) P_s)^-1
Mode 1, N = diag(non-dangling), D = diag(dangling):
    pi_s = e_s (I - (1-t) N P)^-1 (D + t N P)
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def transition_fractions(n, row_ptr, col, w):
    P = [[Fraction(0)] * n for _ in range(n)]
    for u in range(n):
        a, b = int(row_ptr[u]), int(row_ptr[u + 1])
        W = sum(int(w[e]) for e in range(a, b))
        for e in range(a, b):
            P[u][int(col[e])] += Fraction(int(w[e]), W)
    return P


def _solve_left(A, b):
    """x such that x A = b, exact Gauss-Jordan on A^T."""
    n = len(A)
    M = [[A[j][i] for j in range(n)] + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [vr - f * vc for vr, vc in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def exact_pi(n, row_ptr, col, w, T: int, mode: int = 0):
    """Exact rational pi[s][v] for every source s."""
    t = Fraction(T, 1 << 32)
    P = transition_fractions(n, row_ptr, col, w)
    dang = [int(row_ptr[u + 1]) == int(row_ptr[u]) for u in range(n)]
    out = []
    for s in range(n):
        if mode == 0:
            Ps = [row[:] for row in P]
            for u in range(n):
                if dang[u]:
                    Ps[u] = [Fraction(0)] * n
                    Ps[u][s] = Fraction(1)
            A = [[(1 if i == j else 0) - (1 - t) * Ps[i][j] for j in range(n)] for i in range(n)]
            es = [Fraction(0)] * n
            es[s] = Fraction(1)
            y = _solve_left(A, es)  # y = e_s (I - (1-t) P_s)^-1
            pi = [t * sum(y[i] * Ps[i][j] for i in range(n)) for j in range(n)]
        else:
            NP = [[(0 if dang[i] else 1) * P[i][j] for j in range(n)] for i in range(n)]
            A = [[(1 if i == j else 0) - (1 - t) * NP[i][j] for j in range(n)] for i in range(n)]
            es = [Fraction(0)] * n
            es[s] = Fraction(1)
            y = _solve_left(A, es)
            pi = [(y[j] if dang[j] else 0) + t * sum(y[i] * NP[i][j] for i in range(n)) for j in range(n)]
        out.append(pi)
    return out


def enumerate_paths(n, row_ptr, col, w, T: int, s: int, depth: int, mode: int = 0):
    """Endpoint law of walks from s, by listing every walk of at most `depth`
    steps with its probability.  Returns (pi_truncated, unresolved_mass)."""
    t = Fraction(T, 1 << 32)
    P = transition_fractions(n, row_ptr, col, w)
    dang = [int(row_ptr[u + 1]) == int(row_ptr[u]) for u in range(n)]
    pi = [Fraction(0)] * n
    frontier = {s: Fraction(1)}  # active mass by position, before the next move
    for _ in range(depth):
        nxt = {}
        for u, q in frontier.items():
            if dang[u]:
                if mode == 1:
                    pi[u] += q
                    continue
                targets = {s: Fraction(1)}
            else:
                targets = {v: p for v, p in enumerate(P[u]) if p != 0}
            for v, p in targets.items():
                pi[v] += q * p * t
                nxt[v] = nxt.get(v, Fraction(0)) + q * p * (1 - t)
        frontier = nxt
    if mode == 1:
        # dangling positions left in the frontier end there on the next round
        for u, q in list(frontier.items()):
            if dang[u]:
                pi[u] += q
                del frontier[u]
    return pi, sum(frontier.values(), Fraction(0))


def power_iteration(n, row_ptr, col, w, T: int, tol: float = 1e-16):
    """FP64 pi for all sources at once (mode 0), dense n x n."""
    t = T / 2.0 ** 32
    P = np.zeros((n, n), dtype=np.float64)
    deg = np.diff(row_ptr)
    src = np.repeat(np.arange(n), deg)
    Wu = np.zeros(n)
    np.add.at(Wu, src, w.astype(np.float64))
    np.add.at(P, (src, col.astype(np.int64)), w.astype(np.float64) / Wu[src])
    dang = deg == 0

    def step(X):
        Y = X @ P
        if dang.any():
            Y[np.arange(n), np.arange(n)] += X[:, dang].sum(axis=1)
        return Y

    X = step(np.eye(n))
    pi = t * X
    scale = 1.0
    while scale > tol:
        X = (1.0 - t) * step(X)
        pi += t * X
        scale *= (1.0 - t)
    return pi


def binomial_pvalues(counts, R: int, pi):
    """Two-sided exact binomial tail probability of each observed count under
    Binomial(R, pi); entries with pi == 0 get 1 if the count is 0, else 0."""
    from scipy.stats import binom
    counts = np.asarray(counts, dtype=np.float64)
    pi = np.clip(np.asarray(pi, dtype=np.float64), 0.0, 1.0)
    lo = binom.cdf(counts, R, pi)
    hi = binom.sf(counts - 1, R, pi)
    p = np.minimum(1.0, 2.0 * np.minimum(lo, hi))
    zero = pi <= 0
    p = np.where(zero, (counts == 0).astype(np.float64), p)
    return p


def check_estimates(counts, R: int, pi, family_alpha: float = 1e-3):
    """Acceptance rule for Monte Carlo counts against the exact law.

    (a) at most 0.5 % of entries have |pi_hat - pi| > 3 sigma + 1/(2R),
        sigma = sqrt(pi (1 - pi) / R);
    (b) no entry has a two-sided exact binomial p-value below
        family_alpha / (number of entries) (Bonferroni), so the chance that a
        correct sampler fails (b) is at most family_alpha.
    A Gaussian 6-sigma cap is not used for (b): for pi*R of order 1 the count
    is close to Poisson and its upper tail is much heavier than 6 sigma.
    Returns (fraction_beyond_3_sigma, smallest_p_value)."""
    counts = np.asarray(counts, dtype=np.float64)
    pi = np.asarray(pi, dtype=np.float64)
    sig = np.sqrt(np.clip(pi * (1 - pi), 0, None) / R)
    frac = float((np.abs(counts / R - pi) > 3 * sig + 0.5 / R).mean())
    pv = binomial_pvalues(counts, R, pi)
    assert frac <= 0.005, frac
    assert pv.min() >= family_alpha / pv.size, (pv.min(), np.unravel_index(np.argmin(pv), pv.shape))
    return frac, float(pv.min())
