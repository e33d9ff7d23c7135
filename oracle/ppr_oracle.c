/*
 * ppr_oracle.c -- plain single-threaded CPU oracle for Monte Carlo
 * edge-weighted Personalized PageRank (Lin, "Distributed Algorithms for Fully
 * Personalized PageRank on Large Graphs", WWW'19).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA library; it is written directly from the
 * paper and from the published definition of Philox (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *
 * What it computes (paper Sec. 2.1, Algorithm 2, Algorithm 4):
 *   For every source s in [s_begin, s_end) and walk j in [0, R): start at u=s,
 *   repeatedly move to an out-neighbour chosen with probability w(e)/W_u
 *   (routing probability, Sec. 2.1), then stop with probability t = T/2^32
 *   (move-then-stop, Sec. 2.1 and Algorithm 2).  A node with no
 *   out-edge restarts the walk at its head (Sec. 2.1, mode 0) or ends the walk
 *   where it is (mode 1).  The endpoint of walk j of source s is written to
 *   ends[(s - s_begin) * R + j].
 *
 * Integer sampling rule (the readings used wherever the paper is silent):
 *   T      = floor(alpha * 2^32); the walk stops after a step iff x2 < T.
 *   draw   = Philox4x32-10, key (seed mod 2^32, seed >> 32),
 *            counter (s_ctr, j, k, tag) where k counts steps taken so far.
 *   r64    = x0 | x1 << 32.
 *   pick   = the smallest edge index e of u's row with P[e] > floor(r64*W_u/2^64),
 *            P the inclusive prefix sum of the row's weights.
 *   segment step (Algorithm 4 adapted to a fixed depth of 3, nodes of
 *            out-degree <= 8): x = floor(r64*Q_v/2^64) selects an outcome by
 *            the same first-prefix-above rule over the node's outcome table.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox, one definition for both word sizes (SC'11, Sec. 3 and Table 2).   */
/* A round multiplies two counter words by fixed constants, splits each      */
/* product into hi/lo halves, and mixes the hi halves with the other two     */
/* counter words and the round key; the key is bumped by the Weyl constants  */
/* between rounds.  The 64-bit instance is checked against numpy's Philox,    */
/* which pins this shared round structure.                                    */
/* ------------------------------------------------------------------------ */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

#define DEFINE_PHILOX4(NAME, UINT, MULHILO, M0, M1, W0, W1)                    \
    static void NAME(const UINT ctr[4], const UINT key[2], int rounds, UINT out[4]) \
    {                                                                          \
        UINT c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];               \
        UINT k0 = key[0], k1 = key[1];                                         \
        for (int r = 0; r < rounds; ++r) {                                     \
            if (r > 0) {                                                       \
                k0 = (UINT)(k0 + (W0));                                        \
                k1 = (UINT)(k1 + (W1));                                        \
            }                                                                  \
            UINT hi0, lo0, hi1, lo1;                                           \
            MULHILO((M0), c0, &hi0, &lo0);                                     \
            MULHILO((M1), c2, &hi1, &lo1);                                     \
            UINT n0 = hi1 ^ c1 ^ k0;                                           \
            UINT n2 = hi0 ^ c3 ^ k1;                                           \
            c0 = n0;                                                           \
            c1 = lo1;                                                          \
            c2 = n2;                                                           \
            c3 = lo0;                                                          \
        }                                                                      \
        out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;                    \
    }

DEFINE_PHILOX4(philox4x32, uint32_t, mulhilo32,
               UINT32_C(0xD2511F53), UINT32_C(0xCD9E8D57),
               UINT32_C(0x9E3779B9), UINT32_C(0xBB67AE85))
DEFINE_PHILOX4(philox4x64, uint64_t, mulhilo64,
               UINT64_C(0xD2E7470EE14C6C93), UINT64_C(0xCA5A826395121157),
               UINT64_C(0x9E3779B97F4A7C15), UINT64_C(0xBB67AE8584CAA73B))

void ppr_oracle_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds, uint32_t out[4])
{
    philox4x32(ctr, key, rounds, out);
}

/* Words of `count` consecutive counters: counter word 0 = ctr[0] + i (mod 2^32). */
void ppr_oracle_philox4x32_run(const uint32_t ctr[4], const uint32_t key[2], int64_t count, uint32_t *out)
{
    for (int64_t i = 0; i < count; ++i) {
        uint32_t c[4] = {ctr[0] + (uint32_t)i, ctr[1], ctr[2], ctr[3]};
        philox4x32(c, key, 10, out + 4 * i);
    }
}

void ppr_oracle_philox4x64(const uint64_t ctr[4], const uint64_t key[2], int rounds, uint64_t out[4])
{
    philox4x64(ctr, key, rounds, out);
}

/* floor(a * b / 2^64), exact. */
uint64_t ppr_oracle_mulhi64(uint64_t a, uint64_t b)
{
    uint64_t hi, lo;
    mulhilo64(a, b, &hi, &lo);
    return hi;
}

/* T = floor(alpha * 2^32); the scaling by a power of two is exact in binary64.
 * Returns 0 when alpha is outside (0, 1) or T would be 0. */
uint32_t ppr_oracle_threshold(double alpha)
{
    if (!(alpha > 0.0) || !(alpha < 1.0))
        return 0;
    double t = alpha * 4294967296.0;
    return (uint32_t)t; /* truncation == floor for t >= 0 */
}

/* Inclusive per-row prefix sums of the weights: P[e] = sum of w over the row
 * up to and including e; W[u] = total weight of row u (0 if u has no edge). */
void ppr_oracle_row_prefix(int64_t n, const int64_t *row_ptr, const uint32_t *w,
                           uint64_t *P, uint64_t *W)
{
    for (int64_t u = 0; u < n; ++u) {
        uint64_t acc = 0;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            acc += w[e];
            P[e] = acc;
        }
        W[u] = acc;
    }
}

/* Smallest index e in [lo, hi) with P[e] > x.  Requires P non-decreasing and
 * P[hi-1] > x (true for x < W_u).  Plain bisection. */
int64_t ppr_oracle_pick(const uint64_t *P, int64_t lo, int64_t hi, uint64_t x)
{
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (P[mid] > x)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Alias method (Algorithm 1) in integers.  For a row of d edges with         */
/* weights w_e and total W, the switch probability p(e) = d * r(e) of the     */
/* paper becomes the integer p_e = d * w_e out of a slot capacity of W (so    */
/* sum_e p_e = d * W exactly).  S^l holds the e with p_e > W, S^s those with   */
/* p_e < W.  Algorithm 1 lets each round take any x of S^s and any y of S^l;  */
/* here y is always the first element of S^l in ascending edge order, and x   */
/* is the element that joined S^s in the previous round if there is one,     */
/* else the first not yet processed element of the initial S^s in ascending   */
/* order.  Each round sets a(x) = y, keeps thr(x) = p_x and lowers p_y by      */
/* W - p_x; y leaves S^l once p_y <= W and joins S^s if p_y < W.  Edges that  */
/* are never in S^s keep thr = W and a(e) = e.  Selection with one 64-bit     */
/* draw r: slot j = floor(r*d/2^64), y = floor(((r*d) mod 2^64) * W / 2^64);  */
/* the edge is j if y < thr(j), else a(j).  Edge e is chosen for exactly      */
/* d * w_e of the d * W (j, y) pairs.                                         */
/* ------------------------------------------------------------------------ */

/* thr/alias: d entries each (alias as an index within the row).  Work space
 * of d int64 is allocated here. */
int ppr_oracle_alias_table(const uint32_t *w, int64_t d, uint64_t *thr, int64_t *alias)
{
    uint64_t W = 0;
    for (int64_t e = 0; e < d; ++e)
        W += w[e];
    int64_t *small = (int64_t *)malloc(sizeof(int64_t) * (size_t)(d > 0 ? d : 1));
    int64_t *large = (int64_t *)malloc(sizeof(int64_t) * (size_t)(d > 0 ? d : 1));
    if (!small || !large) {
        free(small);
        free(large);
        return -1;
    }
    int64_t n_small = 0, n_large = 0;
    for (int64_t e = 0; e < d; ++e) {
        thr[e] = (uint64_t)d * w[e];
        alias[e] = e;
        if (thr[e] < W)
            small[n_small++] = e;
        else if (thr[e] > W)
            large[n_large++] = e;
    }
    int64_t next_small = 0, first_large = 0;
    int64_t rejoined = -1; /* the element that joined S^s in the previous round */
    while (first_large < n_large) {
        int64_t x;
        if (rejoined >= 0) {
            x = rejoined;
            rejoined = -1;
        } else if (next_small < n_small) {
            x = small[next_small++];
        } else { /* unreachable: the sum of p is d * W exactly */
            free(small);
            free(large);
            return -2;
        }
        int64_t y = large[first_large];
        alias[x] = y;
        thr[y] -= W - thr[x];
        if (thr[y] <= W) {
            ++first_large;
            if (thr[y] < W)
                rejoined = y;
        }
    }
    free(small);
    free(large);
    return 0;
}

/* Index (within the row) the alias rule selects for draw r. */
int64_t ppr_oracle_alias_pick(const uint64_t *thr, const int64_t *alias, int64_t d, uint64_t W, uint64_t r)
{
    unsigned __int128 t = (unsigned __int128)r * (uint64_t)d;
    int64_t j = (int64_t)(uint64_t)(t >> 64);
    uint64_t frac = (uint64_t)t;
    uint64_t y = ppr_oracle_mulhi64(frac, W);
    return y < thr[j] ? j : alias[j];
}

/* Alias tables of every row: thr[e], alias[e] (index within e's row). */
int ppr_oracle_alias_tables(int64_t n, const int64_t *row_ptr, const uint32_t *w, uint64_t *thr, int64_t *alias)
{
    for (int64_t u = 0; u < n; ++u) {
        int64_t a = row_ptr[u], d = row_ptr[u + 1] - a;
        if (d == 0)
            continue;
        if (ppr_oracle_alias_table(w + a, d, thr + a, alias + a) != 0)
            return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Segment tables: Algorithm 4 ("big moves") with the loop fixed at depth 3   */
/* for nodes of out-degree 1..8.                                              */
/*                                                                            */
/* For every path v=u0 -> u1 -> ... -> uj (j <= 3) the fixed-point mass q is  */
/* built edge by edge, in path order:                                         */
/*     q = 2^62;  for each edge i:  if i > 0: q = (q * (2^32 - T)) >> 32      */
/*                                   q = floor(q * w(u_i,u_i+1) / W(u_i))      */
/* A path ending at step j contributes  (q * T) >> 32  to the terminated     */
/* outcome (u_j) -- the set B(v) of Algorithm 4 scaled by alpha.     */
/* A path of length 3, or one that reaches a node with no out-edge before     */
/* step 3, contributes (q * (2^32 - T)) >> 32 to the active outcome           */
/* (u_j, j) -- the set F(v) of Algorithm 4 scaled by 1 - alpha.                    */
/* A node v is eligible iff 1 <= deg(v) <= 8, every node with an out-edge at  */
/* depth 1 or 2 has out-degree <= 8, and at most 64 outcomes have q > 0.      */
/* Outcomes with q == 0 are dropped.  Canonical order: terminated outcomes by */
/* node ascending, then active outcomes by (node, len) ascending.             */
/* ------------------------------------------------------------------------ */

#define SEG_MAXDEG 8
#define SEG_MAXOUT 64

typedef struct {
    uint32_t node;
    uint32_t active; /* 0 terminated, 1 active */
    uint32_t len;    /* steps consumed; 0 for terminated outcomes */
    uint64_t q;
} seg_outcome;

static uint64_t mul_shift32(uint64_t q, uint64_t f)
{
    unsigned __int128 p = (unsigned __int128)q * f;
    return (uint64_t)(p >> 32);
}

static uint64_t mul_div(uint64_t q, uint64_t num, uint64_t den)
{
    unsigned __int128 p = (unsigned __int128)q * num;
    return (uint64_t)(p / den);
}

typedef struct {
    seg_outcome out[2048];
    int count;
} seg_acc;

static void seg_add(seg_acc *acc, uint32_t node, uint32_t active, uint32_t len, uint64_t q)
{
    for (int i = 0; i < acc->count; ++i) {
        seg_outcome *o = &acc->out[i];
        if (o->node == node && o->active == active && o->len == len) {
            o->q += q;
            return;
        }
    }
    seg_outcome *o = &acc->out[acc->count++];
    o->node = node;
    o->active = active;
    o->len = len;
    o->q = q;
}

static int seg_cmp(const void *a, const void *b)
{
    const seg_outcome *x = (const seg_outcome *)a, *y = (const seg_outcome *)b;
    if (x->active != y->active)
        return x->active < y->active ? -1 : 1;
    if (x->node != y->node)
        return x->node < y->node ? -1 : 1;
    if (x->len != y->len)
        return x->len < y->len ? -1 : 1;
    return 0;
}

/* Depth-first enumeration of the paths out of the current tail. */
static void seg_expand(const int64_t *row_ptr, const int32_t *col, const uint32_t *w, const uint64_t *W,
                       uint32_t T, uint32_t u, uint32_t depth, uint64_t q, seg_acc *acc)
{
    /* q is the mass of having arrived at u after `depth` steps without stopping
     * after any earlier step (the stop test of step `depth` not yet applied). */
    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        uint64_t qe = q;
        if (depth > 0)
            qe = mul_shift32(qe, (uint64_t)(UINT64_C(4294967296) - T));
        qe = mul_div(qe, w[e], W[u]);
        uint32_t v = (uint32_t)col[e];
        uint32_t j = depth + 1;
        seg_add(acc, v, 0, 0, mul_shift32(qe, T));
        int dangling = (row_ptr[v + 1] == row_ptr[v]);
        if (j == 3 || dangling)
            seg_add(acc, v, 1, j, mul_shift32(qe, UINT64_C(4294967296) - T));
        else
            seg_expand(row_ptr, col, w, W, T, v, j, qe, acc);
    }
}

static int seg_eligible_shape(const int64_t *row_ptr, const int32_t *col, uint32_t v)
{
    int64_t dv = row_ptr[v + 1] - row_ptr[v];
    if (dv < 1 || dv > SEG_MAXDEG)
        return 0;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        uint32_t a = (uint32_t)col[e];
        int64_t da = row_ptr[a + 1] - row_ptr[a];
        if (da > SEG_MAXDEG)
            return 0;
        for (int64_t f = row_ptr[a]; f < row_ptr[a + 1]; ++f) {
            uint32_t b = (uint32_t)col[f];
            int64_t db = row_ptr[b + 1] - row_ptr[b];
            if (db > SEG_MAXDEG)
                return 0;
        }
    }
    return 1;
}

/* Builds the table of node v into out[] (capacity SEG_MAXOUT).  Returns the
 * number of outcomes, or 0 when v is not eligible. */
int ppr_oracle_segment_table(const int64_t *row_ptr, const int32_t *col, const uint32_t *w,
                             const uint64_t *W, uint32_t T, uint32_t v,
                             uint32_t *node, uint32_t *mark_len, uint64_t *weight)
{
    if (!seg_eligible_shape(row_ptr, col, v))
        return 0;
    static seg_acc acc;
    acc.count = 0;
    seg_expand(row_ptr, col, w, W, T, v, 0, UINT64_C(1) << 62, &acc);
    int k = 0;
    for (int i = 0; i < acc.count; ++i)
        if (acc.out[i].q > 0)
            acc.out[k++] = acc.out[i];
    if (k > SEG_MAXOUT)
        return 0;
    qsort(acc.out, (size_t)k, sizeof(seg_outcome), seg_cmp);
    for (int i = 0; i < k; ++i) {
        node[i] = acc.out[i].node;
        mark_len[i] = (acc.out[i].active << 8) | acc.out[i].len;
        weight[i] = acc.out[i].q;
    }
    return k;
}

/* Builds all tables.  seg_off[v]..seg_off[v+1] delimits v's outcomes in the
 * flat arrays (empty for ineligible nodes); cum is the inclusive prefix of
 * the outcome weights within each table, so Q_v is its last entry.
 * Capacity cap entries; returns the total count or -1 if cap is too small. */
int64_t ppr_oracle_segments(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint32_t *w,
                            const uint64_t *W, uint32_t T, int64_t *seg_off,
                            uint32_t *node, uint32_t *mark_len, uint64_t *weight, uint64_t *cum,
                            int64_t cap)
{
    int64_t pos = 0;
    uint32_t tn[SEG_MAXOUT], tm[SEG_MAXOUT];
    uint64_t tw[SEG_MAXOUT];
    for (int64_t v = 0; v < n; ++v) {
        seg_off[v] = pos;
        int k = ppr_oracle_segment_table(row_ptr, col, w, W, T, (uint32_t)v, tn, tm, tw);
        if (pos + k > cap)
            return -1;
        uint64_t acc = 0;
        for (int i = 0; i < k; ++i) {
            node[pos + i] = tn[i];
            mark_len[pos + i] = tm[i];
            weight[pos + i] = tw[i];
            acc += tw[i];
            cum[pos + i] = acc;
        }
        pos += k;
    }
    seg_off[n] = pos;
    return pos;
}

/* ------------------------------------------------------------------------ */
/* The walks (Algorithm 2 for one source at a time; every walk is simulated  */
/* to its end before the next one starts -- the order does not change any    */
/* result because every draw is keyed by (source, walk, step, tag)).          */
/* ------------------------------------------------------------------------ */

/* Segment tables built on first visit and kept (for runs that visit a small
 * part of a large graph).  Each table is the same as ppr_oracle_segment_table
 * gives; off[v] = -1 until v is visited. */
typedef struct {
    int64_t n;
    uint32_t T;
    int64_t *off;
    int32_t *cnt;
    uint32_t *node, *mark_len;
    uint64_t *cum;
    int64_t used, cap;
} lazy_segments;

void *ppr_oracle_lazy_new(int64_t n)
{
    lazy_segments *L = (lazy_segments *)calloc(1, sizeof(lazy_segments));
    if (!L)
        return NULL;
    L->n = n;
    L->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    L->cnt = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!L->off || !L->cnt)
        return NULL;
    for (int64_t v = 0; v < n; ++v)
        L->off[v] = -1;
    return L;
}

void ppr_oracle_lazy_free(void *p)
{
    lazy_segments *L = (lazy_segments *)p;
    if (!L)
        return;
    free(L->off);
    free(L->cnt);
    free(L->node);
    free(L->mark_len);
    free(L->cum);
    free(L);
}

typedef struct {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col;
    const uint64_t *P;       /* inclusive row prefix */
    const uint64_t *W;       /* row totals */
    const int64_t *seg_off;  /* NULL when segments are off (or built lazily) */
    const uint32_t *seg_node;
    const uint32_t *seg_mark_len;
    const uint64_t *seg_cum; /* inclusive prefix of outcome weights within each table */
    const uint32_t *w;       /* edge weights (lazy segment tables) */
    void *lazy;              /* lazy_segments, or NULL */
    const uint64_t *alias_thr;   /* alias sampler (NULL: first-prefix-above rule) */
    const int64_t *alias_idx;
} oracle_graph;

/* Outcome table of v: returns its length (0 if v has none) and its arrays. */
static int64_t seg_lookup(const oracle_graph *g, uint32_t T, uint32_t v, const uint32_t **node,
                          const uint32_t **ml, const uint64_t **cum)
{
    if (g->seg_off) {
        int64_t a = g->seg_off[v], b = g->seg_off[v + 1];
        *node = g->seg_node + a;
        *ml = g->seg_mark_len + a;
        *cum = g->seg_cum + a;
        return b - a;
    }
    lazy_segments *L = (lazy_segments *)g->lazy;
    if (!L)
        return 0;
    if (L->T != T) { /* tables depend on the threshold */
        for (int64_t u = 0; u < L->n; ++u)
            L->off[u] = -1;
        L->used = 0;
        L->T = T;
    }
    if (L->off[v] < 0) {
        uint32_t tn[SEG_MAXOUT], tm[SEG_MAXOUT];
        uint64_t tw[SEG_MAXOUT];
        int k = ppr_oracle_segment_table(g->row_ptr, g->col, g->w, g->W, T, v, tn, tm, tw);
        if (L->used + k > L->cap) {
            int64_t cap = L->cap ? 2 * L->cap : 4096;
            while (cap < L->used + k)
                cap *= 2;
            L->node = (uint32_t *)realloc(L->node, sizeof(uint32_t) * (size_t)cap);
            L->mark_len = (uint32_t *)realloc(L->mark_len, sizeof(uint32_t) * (size_t)cap);
            L->cum = (uint64_t *)realloc(L->cum, sizeof(uint64_t) * (size_t)cap);
            L->cap = cap;
        }
        uint64_t acc = 0;
        for (int i = 0; i < k; ++i) {
            acc += tw[i];
            L->node[L->used + i] = tn[i];
            L->mark_len[L->used + i] = tm[i];
            L->cum[L->used + i] = acc;
        }
        L->off[v] = L->used;
        L->cnt[v] = k;
        L->used += k;
    }
    *node = L->node + L->off[v];
    *ml = L->mark_len + L->off[v];
    *cum = L->cum + L->off[v];
    return L->cnt[v];
}

typedef struct {
    uint32_t T;
    uint32_t R;
    uint64_t seed;
    int64_t s_begin, s_end;
    int64_t ctr_base;        /* counter source id = s - ctr_base; end ids are also reported minus it */
    uint32_t tag;
    int32_t dangling_mode;   /* 0 restart at the head, 1 end at the dangling node */
} oracle_params;

/* Returns 0 on success.  ends has (s_end - s_begin) * R entries.  steps_out,
 * if non-NULL, receives the number of draws consumed (one per plain step and
 * one per segment step). */
int ppr_oracle_walks(const oracle_graph *g, const oracle_params *p, uint32_t *ends, uint64_t *steps_out)
{
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint64_t steps = 0;
    for (int64_t s = p->s_begin; s < p->s_end; ++s) {
        for (uint32_t j = 0; j < p->R; ++j) {
            uint32_t u = (uint32_t)s;
            uint32_t k = 0;
            uint32_t end;
            for (;;) {
                int64_t lo = g->row_ptr[u], hi = g->row_ptr[u + 1];
                if (hi == lo && p->dangling_mode == 1) {
                    end = u;
                    break;
                }
                uint32_t ctr[4] = {(uint32_t)(s - p->ctr_base), j, k, p->tag};
                uint32_t x[4];
                philox4x32(ctr, key, 10, x);
                uint64_t r64 = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
                const uint32_t *sn, *sml;
                const uint64_t *scum;
                int64_t cnt = (g->seg_off || g->lazy) ? seg_lookup(g, p->T, u, &sn, &sml, &scum) : 0;
                if (cnt > 0) {
                    uint64_t xs = ppr_oracle_mulhi64(r64, scum[cnt - 1]);
                    int64_t o = ppr_oracle_pick(scum, 0, cnt, xs);
                    uint32_t ml = sml[o];
                    steps += 1;
                    if ((ml >> 8) == 0) {
                        end = sn[o];
                        break;
                    }
                    u = sn[o];
                    k += ml & 0xff;
                    continue;
                }
                uint32_t next;
                if (hi == lo) {
                    next = (uint32_t)s;
                } else if (g->alias_thr) {
                    int64_t j = ppr_oracle_alias_pick(g->alias_thr + lo, g->alias_idx + lo, hi - lo, g->W[u], r64);
                    next = (uint32_t)g->col[lo + j];
                } else {
                    uint64_t xp = ppr_oracle_mulhi64(r64, g->W[u]);
                    int64_t e = ppr_oracle_pick(g->P, lo, hi, xp);
                    next = (uint32_t)g->col[e];
                }
                k += 1;
                steps += 1;
                u = next;
                if (x[2] < p->T) {
                    end = u;
                    break;
                }
            }
            ends[(s - p->s_begin) * (int64_t)p->R + j] = (uint32_t)(end - p->ctr_base);
        }
    }
    if (steps_out)
        *steps_out = steps;
    return 0;
}
