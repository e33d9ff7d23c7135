/*
 * rmat_gen.c -- seeded R-MAT graph generator for the synthetic workloads.
 *
 * Input generation only: none of the walk method's arithmetic lives here.
 * Every random choice is a counter-based hash of (seed, purpose, index), so
 * the graph is the same whatever the number of threads.
 *
 * Recipe (source-major R-MAT):
 *   1. out-degrees: each of the m0 edges draws its source bits independently
 *      per level, bit = 1 with probability c + d; a histogram gives the
 *      out-degree of every node.
 *   2. destinations: edge k of row u draws each destination bit with
 *      probability b / (a + b) if the same bit of u is 0, d / (c + d) if it
 *      is 1 (the R-MAT quadrant law conditioned on the source).
 *   3. hub (optional): each edge outside row 0 is moved to row 0 with
 *      probability hub / (m0 - deg(0)); moved edges keep their targets and
 *      are appended to row 0 in edge order.
 *   4. dangling repair: an empty row stays empty with probability
 *      min(1, keep * n / #empty); every other empty row gets one edge to a
 *      uniform target.
 *   5. weights: Zipf(s) on {1..wmax} by inverse CDF.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z)
{
    z += UINT64_C(0x9E3779B97F4A7C15);
    z = (z ^ (z >> 30)) * UINT64_C(0xBF58476D1CE4E5B9);
    z = (z ^ (z >> 27)) * UINT64_C(0x94D049BB133111EB);
    return z ^ (z >> 31);
}

static inline uint64_t rnd(uint64_t seed, uint64_t purpose, uint64_t i)
{
    return mix64(seed ^ mix64((purpose << 56) ^ i));
}

typedef struct {
    void (*fn)(void *ctx, int64_t lo, int64_t hi);
    void *ctx;
    int64_t lo, hi;
} job;

static void *run_job(void *p)
{
    job *j = (job *)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_for(int threads, int64_t n, void (*fn)(void *, int64_t, int64_t), void *ctx)
{
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    pthread_t th[256];
    job jobs[256];
    int64_t per = (n + threads - 1) / threads;
    int used = 0;
    for (int t = 0; t < threads; ++t) {
        int64_t lo = t * per, hi = lo + per < n ? lo + per : n;
        if (lo >= hi)
            break;
        jobs[t] = (job){fn, ctx, lo, hi};
        if (pthread_create(&th[t], NULL, run_job, &jobs[t]) != 0) {
            run_job(&jobs[t]);
            th[t] = 0;
        }
        used = t + 1;
    }
    for (int t = 0; t < used; ++t)
        if (th[t])
            pthread_join(th[t], NULL);
}

typedef struct {
    int scale;
    uint64_t seed;
    uint32_t t_src, t_dst0, t_dst1; /* thresholds on 32-bit words */
    int64_t *deg;                   /* atomic histogram */
    const int64_t *rp;              /* row_ptr after step 1 */
    int32_t *dst;
    uint8_t *moved;
    uint32_t t_move;
    int64_t n;
    const double *cdf;
    int wmax;
    uint32_t *w;
} gen_ctx;

static void k_degrees(void *p, int64_t lo, int64_t hi)
{
    gen_ctx *g = (gen_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        uint64_t s = 0;
        for (int l = 0; l < g->scale; l += 2) {
            uint64_t r = rnd(g->seed, 1, (uint64_t)e * (uint64_t)g->scale + (uint64_t)l);
            if ((uint32_t)r < g->t_src)
                s |= UINT64_C(1) << l;
            if (l + 1 < g->scale && (uint32_t)(r >> 32) < g->t_src)
                s |= UINT64_C(1) << (l + 1);
        }
        __atomic_fetch_add(&g->deg[s], 1, __ATOMIC_RELAXED);
    }
}

static void k_dests(void *p, int64_t lo, int64_t hi)
{
    gen_ctx *g = (gen_ctx *)p;
    for (int64_t u = lo; u < hi; ++u) {
        for (int64_t e = g->rp[u]; e < g->rp[u + 1]; ++e) {
            uint64_t d = 0;
            for (int l = 0; l < g->scale; l += 2) {
                uint64_t r = rnd(g->seed, 2, (uint64_t)e * (uint64_t)g->scale + (uint64_t)l);
                uint32_t t0 = ((u >> l) & 1) ? g->t_dst1 : g->t_dst0;
                if ((uint32_t)r < t0)
                    d |= UINT64_C(1) << l;
                if (l + 1 < g->scale) {
                    uint32_t t1 = ((u >> (l + 1)) & 1) ? g->t_dst1 : g->t_dst0;
                    if ((uint32_t)(r >> 32) < t1)
                        d |= UINT64_C(1) << (l + 1);
                }
            }
            g->dst[e] = (int32_t)d;
        }
    }
}

static void k_move(void *p, int64_t lo, int64_t hi)
{
    gen_ctx *g = (gen_ctx *)p;
    for (int64_t e = lo; e < hi; ++e)
        g->moved[e] = (e >= g->rp[1]) && ((uint32_t)rnd(g->seed, 3, (uint64_t)e) < g->t_move);
}

static void k_weights(void *p, int64_t lo, int64_t hi)
{
    gen_ctx *g = (gen_ctx *)p;
    for (int64_t e = lo; e < hi; ++e) {
        double u = (double)(rnd(g->seed, 6, (uint64_t)e) >> 11) * (1.0 / 9007199254740992.0);
        int a = 0, b = g->wmax - 1; /* first k with cdf[k] > u */
        while (a < b) {
            int mid = (a + b) / 2;
            if (g->cdf[mid] > u)
                b = mid;
            else
                a = mid + 1;
        }
        g->w[e] = (uint32_t)(a + 1);
    }
}

static uint32_t prob32(double p)
{
    if (p <= 0)
        return 0;
    if (p >= 1)
        return UINT32_MAX;
    return (uint32_t)(p * 4294967296.0);
}

/*
 * Pass 1: returns the final edge count (after hub and dangling repair) so the
 * caller can size col/w; fills row_ptr (n+1).  Pass 2 (rmat_finish) fills col/w.
 * Work arrays are allocated here and kept in the handle.
 */
typedef struct {
    int64_t n, m0, m;
    int64_t *rp0;     /* rows before hub / repair */
    int32_t *dst0;
    uint8_t *moved;
    uint8_t *fill;    /* repaired empty rows */
    int64_t hub;
    gen_ctx g;
    int threads;
} rmat_state;

void *rmat_begin(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed, double keep_dangling,
                 int64_t hub_degree, int threads, int64_t *row_ptr)
{
    rmat_state *S = (rmat_state *)calloc(1, sizeof(rmat_state));
    if (!S)
        return NULL;
    int64_t n = (int64_t)1 << scale, m0 = edge_factor * n;
    double d = 1.0 - a - b - c;
    S->n = n;
    S->m0 = m0;
    S->threads = threads;
    gen_ctx *g = &S->g;
    g->scale = scale;
    g->seed = seed;
    g->n = n;
    g->t_src = prob32(c + d);
    g->t_dst0 = prob32(b / (a + b));
    g->t_dst1 = prob32(d / (c + d));
    int64_t *deg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    S->rp0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    S->dst0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)m0);
    S->moved = (uint8_t *)calloc((size_t)m0, 1);
    S->fill = (uint8_t *)calloc((size_t)n, 1);
    if (!deg || !S->rp0 || !S->dst0 || !S->moved || !S->fill)
        return NULL;
    g->deg = deg;
    parallel_for(threads, m0, k_degrees, g);
    S->rp0[0] = 0;
    for (int64_t u = 0; u < n; ++u)
        S->rp0[u + 1] = S->rp0[u] + deg[u];
    g->rp = S->rp0;
    g->dst = S->dst0;
    parallel_for(threads, n, k_dests, g);
    /* hub */
    int64_t nmoved = 0;
    if (hub_degree > 0) {
        double q = (double)hub_degree / (double)(m0 - S->rp0[1]);
        g->t_move = prob32(q);
        g->moved = S->moved;
        parallel_for(threads, m0, k_move, g);
        for (int64_t e = 0; e < m0; ++e)
            nmoved += S->moved[e];
        /* degrees after the move */
        for (int64_t u = 1; u < n; ++u) {
            int64_t k = 0;
            for (int64_t e = S->rp0[u]; e < S->rp0[u + 1]; ++e)
                k += S->moved[e];
            deg[u] -= k;
        }
        deg[0] += nmoved;
    }
    S->hub = nmoved;
    /* dangling repair */
    int64_t empty = 0;
    for (int64_t u = 0; u < n; ++u)
        empty += deg[u] == 0;
    double pkeep = empty ? keep_dangling * (double)n / (double)empty : 0.0;
    uint32_t tkeep = prob32(pkeep);
    for (int64_t u = 0; u < n; ++u) {
        if (deg[u] == 0 && (uint32_t)rnd(seed, 4, (uint64_t)u) >= tkeep) {
            S->fill[u] = 1;
            deg[u] = 1;
        }
    }
    row_ptr[0] = 0;
    for (int64_t u = 0; u < n; ++u)
        row_ptr[u + 1] = row_ptr[u] + deg[u];
    S->m = row_ptr[n];
    free(deg);
    g->deg = NULL;
    return S;
}

int64_t rmat_edges(void *h) { return ((rmat_state *)h)->m; }
int64_t rmat_hub(void *h) { return ((rmat_state *)h)->hub; }

typedef struct {
    rmat_state *S;
    const int64_t *rp;
    int32_t *col;
} fill_ctx;

static void k_fill(void *p, int64_t lo, int64_t hi)
{
    fill_ctx *f = (fill_ctx *)p;
    rmat_state *S = f->S;
    for (int64_t u = lo; u < hi; ++u) {
        if (u == 0)
            continue; /* row 0 is filled serially (it gathers the moved edges) */
        int64_t o = f->rp[u];
        if (S->fill[u]) {
            f->col[o] = (int32_t)(rnd(S->g.seed, 5, (uint64_t)u) % (uint64_t)S->n);
            continue;
        }
        for (int64_t e = S->rp0[u]; e < S->rp0[u + 1]; ++e)
            if (!S->moved[e])
                f->col[o++] = S->dst0[e];
    }
}

/* Fills col/w (m entries each) and frees the handle. */
int rmat_finish(void *h, const int64_t *row_ptr, int32_t *col, uint32_t *w, double zipf_s, int wmax)
{
    rmat_state *S = (rmat_state *)h;
    fill_ctx f = {S, row_ptr, col};
    parallel_for(S->threads, S->n, k_fill, &f);
    int64_t o = row_ptr[0];
    if (S->fill[0]) {
        col[o] = (int32_t)(rnd(S->g.seed, 5, 0) % (uint64_t)S->n);
    } else {
        for (int64_t e = S->rp0[0]; e < S->rp0[1]; ++e)
            col[o++] = S->dst0[e];
        for (int64_t e = S->rp0[1]; e < S->m0; ++e)
            if (S->moved[e])
                col[o++] = S->dst0[e];
    }
    double *cdf = (double *)malloc(sizeof(double) * (size_t)wmax);
    double acc = 0;
    for (int k = 1; k <= wmax; ++k) {
        acc += pow((double)k, -zipf_s);
        cdf[k - 1] = acc;
    }
    for (int k = 0; k < wmax; ++k)
        cdf[k] /= acc;
    S->g.cdf = cdf;
    S->g.wmax = wmax;
    S->g.w = w;
    parallel_for(S->threads, S->m, k_weights, &S->g);
    free(cdf);
    free(S->rp0);
    free(S->dst0);
    free(S->moved);
    free(S->fill);
    free(S);
    return 0;
}
