"""Pins of the CPU oracle against things other than itself: library routines
(numpy's Philox4x64, cuRAND's host Philox4x32), exact integer arithmetic, exact rational PPR, brute-force
path enumeration, FP64 power iteration, the paper's worked examples, and the
invariants the paper states (Lemma 2, expected walk length 1/alpha)."""
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import exact_ppr as X
from paper_1903_11749_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----

def test_philox4x64_matches_numpy(oracle):
    """numpy's Philox bit generator is Philox4x64-10; its raw output for
    counter c is the block of c + 1.  The oracle's 4x64 instance is produced
    by the same round definition as its 4x32 instance, so this pins the round
    structure, the key schedule and the output order of both."""
    rng = np.random.Generator(np.random.PCG64(99))
    for _ in range(200):
        key = rng.integers(0, 2**64, size=2, dtype=np.uint64)
        ctr = rng.integers(1, 2**64, size=4, dtype=np.uint64)
        prev = ctr.copy()
        prev[0] -= np.uint64(1)
        ref = np.random.Philox(counter=prev, key=key).random_raw(4)
        got = oracle.philox4x64(ctr, key)
        assert [int(v) for v in got] == [int(v) for v in ref]


def test_philox_weyl_constants_are_the_published_irrationals(oracle):
    """The key bumps are the fractional parts of the golden ratio and of
    sqrt(3) scaled to the word size.  With rounds=2 the key bump enters the
    second round exactly once; recover it from a zero counter and check it."""
    getcontext().prec = 60
    phi_frac = (Decimal(1) + Decimal(5).sqrt()) / 2 - 1
    s3_frac = Decimal(3).sqrt() - 1
    for bits, fn, dt in ((32, oracle.philox4x32, np.uint32), (64, oracle.philox4x64, np.uint64)):
        w0 = int(phi_frac * (1 << bits))
        w1 = int(s3_frac * (1 << bits))
        # With a zero counter and zero key, round 1 outputs all zeros (0 * M = 0),
        # so round 2's output words 0 and 2 are exactly the bumped key words.
        out = fn(np.zeros(4, dtype=dt), np.zeros(2, dtype=dt), rounds=2)
        assert int(out[0]) == w0
        assert int(out[2]) == w1


def _curand_host():
    """The CUDA toolkit's host-side random number library (runs on the CPU), or None."""
    import ctypes
    import ctypes.util
    cands = [ctypes.util.find_library("curand")]
    for root in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if root:
            cands += [os.path.join(root, d, "libcurand.so") for d in ("lib64", "lib", "targets/sbsa-linux/lib")]
    for c in cands:
        if c:
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    return None


def test_philox4x32_matches_curand_host_generator(oracle):
    """cuRAND's host generator of type PHILOX4_32_10 (computed on the CPU) is
    an independent Philox4x32-10: seeded with s, its i-th block of four words
    is the block of counter (0, 0, i, 0) under key (s mod 2^32, s >> 32).
    This pins the 4x32 instance itself -- its multipliers, key bumps and word
    order -- over 4,096 blocks for each of four seeds."""
    import ctypes
    lib = _curand_host()
    if lib is None:
        pytest.skip("the CUDA random number library is not installed")
    PHILOX4_32_10 = 161  # curandRngType_t
    for seed in (0, 5, 0xDEADBEEF12345678, 2**64 - 1):
        gen = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX4_32_10) == 0
        try:
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            ref = np.zeros(4 * 4096, dtype=np.uint32)
            assert lib.curandGenerate(gen, ref.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(ref.size)) == 0
        finally:
            lib.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = np.stack([oracle.philox4x32([0, 0, i, 0], key) for i in range(4096)])
        assert np.array_equal(got, ref.reshape(-1, 4)), hex(seed)


def test_philox4x32_words_are_uniform(oracle):
    """Chi-square of the four 32-bit output words over 16 bins each."""
    counts = np.zeros((4, 16), dtype=np.int64)
    N = 20000
    for i in range(N):
        out = oracle.philox4x32([i, 7, 3, 1], [0xDEADBEEF, 0x12345678])
        for wi in range(4):
            counts[wi, int(out[wi]) >> 28] += 1
    exp = N / 16
    for wi in range(4):
        chi2 = float(((counts[wi] - exp) ** 2 / exp).sum())
        assert chi2 < 45.0  # 15 dof; p ~ 1e-4


def test_philox4x32_distinct_counters_give_distinct_blocks(oracle):
    seen = set()
    for s in range(8):
        for j in range(8):
            for k in range(8):
                seen.add(tuple(int(v) for v in oracle.philox4x32([s, j, k, 0], [1, 0])))
    assert len(seen) == 512


# --------------------------------------------------- integer sampling rule ----

def test_mulhi64_is_exact_floor(oracle):
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(2000):
        a = int(rng.integers(0, 2**64, dtype=np.uint64))
        b = int(rng.integers(0, 2**64, dtype=np.uint64))
        assert oracle.mulhi64(a, b) == (a * b) >> 64
    assert oracle.mulhi64(2**64 - 1, 2**64 - 1) == 2**64 - 2


def test_threshold_is_floor_alpha_2_32(oracle):
    rng = np.random.Generator(np.random.PCG64(6))
    for alpha in list(rng.random(500)) + [0.15, 0.2, 0.5, 1e-9, 0.999999999]:
        want = math.floor(Fraction(alpha) * 2**32)
        assert oracle.threshold(float(alpha)) == want
    assert oracle.threshold(0.15) == 644245094
    assert oracle.threshold(0.2) == 858993459
    assert oracle.threshold(0.5) == 2**31
    for bad in (0.0, 1.0, -0.1, 1.5, 2.0**-33, float("nan")):
        assert oracle.threshold(bad) == 0


@pytest.mark.parametrize("weights", [[1], [3, 1], [1, 1, 1, 1], [2, 3, 3], [5, 1, 7, 1, 1, 9], [1000, 1, 1]])
def test_pick_inverts_the_prefix_exactly(oracle, weights):
    """Every x in [0, W) selects index e exactly w_e times: the routing
    probability w(e)/W_u of Sec. 2.1 is realised exactly over x."""
    P = np.cumsum(np.asarray(weights, dtype=np.uint64))
    W = int(P[-1])
    hits = np.zeros(len(weights), dtype=np.int64)
    pad = np.concatenate([np.zeros(3, dtype=np.uint64), P])  # row starting at offset 3
    for x in range(W):
        e = oracle.pick(pad, 3, 3 + len(weights), x)
        hits[e - 3] += 1
    assert hits.tolist() == list(weights)


def test_one_step_law_on_a_hub(oracle):
    """With alpha close to 1 almost every walk stops after one step, so the
    endpoint histogram of a 200-edge hub follows w(e)/W_u (chi-square)."""
    rng = np.random.Generator(np.random.PCG64(8))
    deg = 200
    w = rng.integers(1, 50, size=deg)
    edges = [(0, 1 + i, int(w[i])) for i in range(deg)] + [(1 + i, 0, 1) for i in range(deg)]
    g = I.from_edges(deg + 1, edges)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    R = 200000
    ends, _ = oracle.walks(og, 1.0 - 2.0**-20, R, seed=3, s_begin=0, s_end=1)
    cnt = np.bincount(ends[0].astype(np.int64), minlength=deg + 1)[1:]
    exp = R * w / w.sum()
    chi2 = float(((cnt - exp) ** 2 / exp).sum())
    assert chi2 < 199 + 6 * math.sqrt(2 * 199)


# ------------------------------------------------------- law of the walk ----

def _small_graphs():
    gs = []
    # parallel edges, a self-loop, a dangling node and a 1000:1 weight skew
    gs.append(I.from_edges(6, [(0, 1, 1000), (0, 2, 1), (0, 1, 3), (1, 1, 2), (1, 3, 5), (2, 0, 1),
                               (2, 4, 7), (3, 0, 1), (3, 5, 1), (4, 2, 2)]))
    gs.append(I.from_edges(5, [(0, 1, 1), (1, 2, 1), (2, 0, 1), (2, 3, 9), (3, 4, 1), (4, 0, 4), (4, 4, 1)]))
    for seed in (1, 2, 3):
        gs.append(I.random_small_graph(7 + seed % 2, 14, seed, wmax=20, dangling=1))
    return gs


def _check_counts(ends_rows, pi_rows, R):
    """Estimator pi_hat = omega'/omega (Sec. 2.1) against the exact law, with
    the acceptance rule of exact_ppr.check_estimates."""
    n = len(pi_rows[0])
    cnt = np.stack([np.bincount(e.astype(np.int64), minlength=n) for e in ends_rows])
    assert (cnt.sum(axis=1) == R).all()
    X.check_estimates(cnt, R, np.array([[float(p) for p in row] for row in pi_rows]))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("gi", range(5))
def test_oracle_law_matches_exact_pi(oracle, gi, mode):
    g = _small_graphs()[gi]
    alpha = [0.15, 0.3, 0.5, 0.2, 0.7][gi]
    T = oracle.threshold(alpha)
    pi = X.exact_pi(g.n, g.row_ptr, g.col, g.w, T, mode)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    R = 40000
    ends, _ = oracle.walks(og, alpha, R, seed=11 + gi, dangling=mode)
    for s in range(g.n):
        assert sum(pi[s]) == 1
    _check_counts(ends, pi, R)


@pytest.mark.parametrize("mode", [0, 1])
def test_exact_pi_matches_path_enumeration(mode):
    """The closed form used as ground truth agrees with listing every walk up
    to depth L, within the unresolved mass (1-t)^L."""
    g = _small_graphs()[0]
    T = 2**31
    pi = X.exact_pi(g.n, g.row_ptr, g.col, g.w, T, mode)
    for s in range(g.n):
        enum, rest = X.enumerate_paths(g.n, g.row_ptr, g.col, g.w, T, s, depth=24, mode=mode)
        assert rest <= Fraction(1, 2**24)
        for v in range(g.n):
            assert 0 <= pi[s][v] - enum[v] <= rest


def test_dangling_source_ends_at_itself(oracle):
    g = I.from_edges(4, [(0, 1, 1), (1, 2, 1), (2, 0, 1)])  # node 3 dangling
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for mode in (0, 1):
        ends, _ = oracle.walks(og, 0.15, 500, seed=1, s_begin=3, s_end=4, dangling=mode)
        assert (ends == 3).all()


def test_mean_walk_length_is_one_over_alpha(oracle):
    """Sec. 2.1: the expected length of a walk is 1/alpha (here 2^32/T)."""
    g = I.er_graph(200, 2000, seed=4)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    alpha, R = 0.15, 500
    ends, steps = oracle.walks(og, alpha, R, seed=1)
    walks = g.n * R
    T = oracle.threshold(alpha)
    mean = steps / walks
    t = T / 2**32
    sd = math.sqrt((1 - t) / t**2 / walks)
    assert abs(mean - 1 / t) < 5 * sd


def test_power_iteration_er1k(oracle):
    """Oracle on the 1000-node ER workload (alpha 0.15, R 1000, seed 1) against
    FP64 power iteration under the acceptance rule of check_estimates; every
    row sums to R; count > 0 only where pi > 0."""
    g = I.er_graph(1000, 10_000, 1, 10, seed=12345)
    T = oracle.threshold(0.15)
    pi = X.power_iteration(g.n, g.row_ptr, g.col, g.w, T)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    R = 1000
    ends, _ = oracle.walks(og, 0.15, R, seed=1)
    cnt = oracle.dense(ends, g.n)
    assert (cnt.sum(axis=1) == R).all()
    X.check_estimates(cnt, R, pi)
    assert not ((cnt > 0) & (pi <= 0)).any()


# ------------------------------------------------- big moves (segments) ----

def _golden_example5():
    rows = []
    with open(os.path.join(GOLDEN, "example5_big_moves.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                node, mark, p = line.split()
                rows.append((int(node[1:]), int(mark), Fraction(p)))
    return rows


def test_example5_big_moves_exact(oracle):
    """Sec. 4.2 Example 5 (alpha = 0.5): BM(v2) = <v3,0,0.625>, <v4,0,0.25>,
    <v3,1,0.125>, reproduced exactly in 2^62 fixed point."""
    # nodes v2, v3, v4 as ids 2, 3, 4; v0, v1 unused (give them edges so they are not dangling)
    g = I.from_edges(5, [(0, 1, 1), (1, 0, 1), (2, 3, 1), (3, 4, 1), (4, 3, 1)])
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    T = oracle.threshold(0.5)
    table = oracle.segment_table(og, T, 2)
    got = {(node, active): wt for node, active, _, wt in table}
    for node, mark, p in _golden_example5():
        assert got[(node, mark)] == p * 2**62
    assert len(table) == 3
    assert [ln for _, a, ln, _ in table if a] == [3]


def _exact_outcomes(g, T, v):
    """Exact rational outcome masses of the depth-3 big move of v, and the
    number of (edge, depth) sites the enumeration visits."""
    t = Fraction(T, 2**32)
    rp, col, w = g.row_ptr, g.col, g.w
    Wt = [sum(int(w[e]) for e in range(int(rp[u]), int(rp[u + 1]))) for u in range(g.n)]
    out = {}
    sites = [0]

    def rec(u, depth, q):
        for e in range(int(rp[u]), int(rp[u + 1])):
            x = int(col[e])
            sites[0] += 1
            qe = q * Fraction(int(w[e]), Wt[u]) * (1 if depth == 0 else (1 - t))
            out[(x, 0, 0)] = out.get((x, 0, 0), 0) + qe * t
            if depth + 1 == 3 or Wt[x] == 0:
                key = (x, 1, depth + 1)
                out[key] = out.get(key, 0) + qe * (1 - t)
            else:
                rec(x, depth + 1, qe)

    rec(v, 0, Fraction(1))
    return out, sites[0]


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_segment_tables_match_exact_masses_and_lemma2(oracle, seed):
    """Each fixed-point outcome weight is within the flooring error of the
    exact mass x 2^62, and the weights sum to 2^62 minus at most 4 units per
    enumerated path (Lemma 2: the big moves form a full probability space)."""
    g = I.random_small_graph(9, 20, seed, wmax=30, dangling=1)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for alpha in (0.15, 0.5):
        T = oracle.threshold(alpha)
        for v in range(g.n):
            table = oracle.segment_table(og, T, v)
            deg = int(g.row_ptr[v + 1] - g.row_ptr[v])
            if deg == 0:
                assert table == []
                continue
            ex, sites = _exact_outcomes(g, T, v)
            # per visited edge: the ratio floor loses < 1 unit and the split of its
            # mass into the terminated share and the continuing (or active) share
            # loses < 2 units; later factors are <= 1 and do not amplify a loss
            for node, active, ln, wt in table:
                e = ex[(node, active, ln if active else 0)] * 2**62
                assert abs(wt - e) <= 3 * sites
            Q = sum(wt for *_, wt in table)
            assert 0 <= 2**62 - Q <= 3 * sites
            # canonical order: terminated by node, then active by (node, len)
            keys = [(a, nd, ln) for nd, a, ln, _ in table]
            assert keys == sorted(keys)


def test_segment_eligibility_rules(oracle):
    # node 0 has degree 9 -> ineligible; node 1 -> node 0 (deg 9) at depth 1 -> ineligible
    edges = [(0, 2 + i, 1) for i in range(9)] + [(1, 0, 1)] + [(2 + i, 1, 1) for i in range(9)]
    g = I.from_edges(11, edges)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    T = oracle.threshold(0.2)
    assert oracle.segment_table(og, T, 0) == []
    assert oracle.segment_table(og, T, 1) == []
    # node 2 -> 1 -> 0: node 0 sits at depth 2 with degree 9 -> ineligible
    assert oracle.segment_table(og, T, 2) == []


@pytest.mark.parametrize("mode", [0, 1])
def test_segment_mode_law_matches_exact_pi(oracle, mode):
    """Segment steps change which draws are consumed but not the law of the
    walk (up to 2^-60 flooring): the counts still match the exact pi."""
    g = _small_graphs()[0]
    alpha = 0.3
    T = oracle.threshold(alpha)
    pi = X.exact_pi(g.n, g.row_ptr, g.col, g.w, T, mode)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    oracle.build_segments(og, T)
    assert (np.diff(og.seg_off) > 0).sum() >= 3
    R = 40000
    ends, _ = oracle.walks(og, alpha, R, seed=5, dangling=mode, segments=True)
    _check_counts(ends, pi, R)


# ------------------------------------------------------------ aggregation ----

def test_rows_and_topk_invariants(oracle):
    g = I.er_graph(300, 1500, seed=9)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    R = 77
    ends, _ = oracle.walks(og, 0.25, R, seed=2)
    rp, col, cnt = oracle.rows(ends, g.n)
    for s in range(g.n):
        c = col[rp[s]:rp[s + 1]]
        assert (np.diff(c) > 0).all()
        assert int(cnt[rp[s]:rp[s + 1]].sum()) == R
        ref = np.bincount(ends[s].astype(np.int64), minlength=g.n)
        assert (ref[c] == cnt[rp[s]:rp[s + 1]]).all()
    idx, tc = oracle.topk(rp, col, cnt, 8)
    for s in range(g.n):
        ref = np.bincount(ends[s].astype(np.int64), minlength=g.n)
        order = sorted([(-int(ref[v]), v) for v in range(g.n) if ref[v] > 0])[:8]
        want = [v for _, v in order] + [-1] * (8 - len(order))
        assert idx[s].tolist() == want
        assert tc[s].tolist() == [-c for c, _ in order] + [0] * (8 - len(order))


def test_lazy_segment_tables_equal_full_tables(oracle):
    """Tables built on first visit give the same walks as tables built for
    every node up front."""
    g = I.random_small_graph(500, 1400, seed=21, wmax=30, dangling=20)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    for alpha, mode in ((0.15, 0), (0.5, 1)):
        e1, s1 = oracle.walks(og, alpha, 50, 3, dangling=mode, segments=True)
        e2, s2 = oracle.walks(og, alpha, 50, 3, dangling=mode, segments=True, lazy_segments=True)
        assert np.array_equal(e1, e2) and s1 == s2


# ------------------------------------------------------------- alias rule ----

def _golden_example2():
    rows = []
    with open(os.path.join(GOLDEN, "example2_alias.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                e, p, a = line.split()
                rows.append((int(e[1:]) - 1, Fraction(p), int(a[1:]) - 1))
    return rows


def test_example2_alias_setup_exact(oracle):
    """Sec. 2.2 Example 2: weights in ratio 2:3:3 give switch probabilities
    (0.75, 0.875, 1) and aliases (e2, e3, e3), exactly (thr / W)."""
    for scale in (1, 7):
        w = np.array([2, 3, 3]) * scale
        thr, ali = oracle.alias_table(w)
        W = int(w.sum())
        for e, p, a in _golden_example2():
            assert Fraction(int(thr[e]), W) == p
            assert int(ali[e]) == a


def test_alias_pairing_order_worked_by_hand(oracle):
    """The pairing order Algorithm 1 leaves open (any x of S^s, any y of S^l),
    fixed as: y the first of S^l, x the element that just joined S^s, else the
    next initial small one.  Weights (1,1,2,2,2): d = 5, W = 8, p = (5,5,10,10,10).
    Round 1: x=e1, y=e3 -> a(e1)=e3, p(e3) = 10-3 = 7 < 8, e3 joins S^s.
    Round 2: x=e3, y=e4 -> a(e3)=e4, p(e4) = 10-1 = 9.
    Round 3: x=e2, y=e4 -> a(e2)=e4, p(e4) = 9-3 = 6 < 8, e4 joins S^s.
    Round 4: x=e4, y=e5 -> a(e4)=e5, p(e5) = 10-2 = 8, S^l empty.
    (A first-in first-out S^s would pair e3 with e5 instead.)"""
    thr, ali = oracle.alias_table(np.array([1, 1, 2, 2, 2]))
    assert [int(t) for t in thr] == [5, 5, 7, 6, 8]
    assert [int(a) for a in ali][:4] == [2, 3, 3, 4]


@pytest.mark.parametrize("seed", range(6))
def test_alias_table_equals_prefix_sum_closed_form(oracle, seed):
    """With that order the table has a closed form in prefix sums: for the
    small edges (p < W, ascending) let D_i be the running sum of W - p, for the
    large ones (p > W, ascending) E_j the running sum of p - W.  Small edge i
    takes thr = p and the alias of the first large j with E_j > D_(i-1);
    large edge j (not the last) takes thr = W - (D_q - E_j) for the first q
    with D_q >= E_j and the alias of large j+1; the last large edge and the
    edges with p = W keep thr = W."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = int(rng.integers(2, 300))
    w = (I.zipf_weights(rng, d, s=1.1, wmax=10_000) if seed % 2 else rng.integers(1, 50, d)).astype(np.uint64)
    if seed == 5:
        w[:] = 7  # every p equals W
    W = int(w.sum())
    p = [d * int(x) for x in w]
    small = [e for e in range(d) if p[e] < W]
    large = [e for e in range(d) if p[e] > W]
    D = np.cumsum([W - p[e] for e in small]).tolist()
    E = np.cumsum([p[e] - W for e in large]).tolist()
    thr, ali = oracle.alias_table(w)
    want_thr = [W] * d
    want_ali = {}
    for i, e in enumerate(small):
        prev = D[i - 1] if i else 0
        j = next(j for j in range(len(large)) if E[j] > prev)
        want_thr[e] = p[e]
        want_ali[e] = large[j]
    for j, e in enumerate(large[:-1]):
        q = next(q for q in range(len(small)) if D[q] >= E[j])
        want_thr[e] = W - (D[q] - E[j])
        want_ali[e] = large[j + 1]
    assert [int(t) for t in thr] == want_thr
    for e, a in want_ali.items():
        if want_thr[e] < W:
            assert int(ali[e]) == a


@pytest.mark.parametrize("weights", [[1], [3, 1], [2, 3, 3], [5, 1, 7, 1, 1, 9], [1000, 1, 1], [4, 4, 4, 4],
                                     [1, 2, 3, 4, 5, 6, 7, 8, 9]])
def test_alias_rule_realises_routing_probability_exactly(oracle, weights):
    """Over all d * W (slot, y) pairs, edge e is chosen exactly d * w_e times:
    the selection law is r(e) = w_e / W exactly (Sec. 2.2)."""
    w = np.asarray(weights, dtype=np.uint64)
    d, W = len(w), int(w.sum())
    thr, ali = oracle.alias_table(w)
    hits = np.zeros(d, dtype=np.int64)
    for j in range(d):
        for y in range(W):
            hits[j if y < int(thr[j]) else int(ali[j])] += 1
    assert hits.tolist() == [d * int(x) for x in w]
    assert all(0 <= int(t) <= W for t in thr)


def test_alias_pick_uses_slot_and_fraction(oracle):
    """alias_pick with draw r equals the rule computed with exact integers."""
    rng = np.random.Generator(np.random.PCG64(12))
    w = rng.integers(1, 1000, 37).astype(np.uint64)
    thr, ali = oracle.alias_table(w)
    W = int(w.sum())
    for _ in range(3000):
        r = int(rng.integers(0, 2**64, dtype=np.uint64))
        j, frac = divmod(r * len(w), 2**64)
        y = (frac * W) >> 64
        want = j if y < int(thr[j]) else int(ali[j])
        assert oracle.alias_pick(thr, ali, W, r) == want


@pytest.mark.parametrize("mode", [0, 1])
def test_alias_sampler_law_matches_exact_pi(oracle, mode):
    g = _small_graphs()[0]
    alpha = 0.3
    T = oracle.threshold(alpha)
    pi = X.exact_pi(g.n, g.row_ptr, g.col, g.w, T, mode)
    og = oracle.prepare(g.n, g.row_ptr, g.col, g.w)
    R = 40000
    ends, _ = oracle.walks(og, alpha, R, seed=15, dangling=mode, sampler=1)
    _check_counts(ends, pi, R)
