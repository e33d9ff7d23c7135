/*
 * ppr.h -- C ABI of the GB300 Monte Carlo edge-weighted Personalized
 * PageRank library (libppr.so).
 *
 * The library computes, on one GPU, the Monte Carlo estimator of fully
 * personalized PageRank on an edge-weighted directed graph (Lin, "Distributed
 * Algorithms for Fully Personalized PageRank on Large Graphs", WWW'19):
 * R random walks from every source of a range; each step moves to an
 * out-neighbour with probability w(e)/W_u (routing probability, Sec. 2.1) and
 * then stops with probability alpha (Sec. 2.1, Algorithm 2); the endpoint
 * counts of each source form its sparse row, pi_hat(s,t) = count/R (Sec. 2.1
 * estimator, Definition 1).  Results are exact integer counts, identical for
 * any launch shape, batch split or kernel choice.
 *
 * Integer sampling rule (fixed; every result is a function of it):
 *   T = floor(alpha * 2^32), 1 <= T; a walk stops after a step iff x2 < T.
 *   (x0,x1,x2,x3) = Philox4x32-10(key = (seed mod 2^32, seed >> 32),
 *                    counter = (s_local, j, k, tag)), j = walk index,
 *                    k = steps taken so far (mod 2^32).
 *   r64 = x0 | x1 << 32; next edge = smallest e of the row with
 *   P[e] > floor(r64 * W_u / 2^64), P the inclusive row prefix of weights.
 *   With sampler = 1 the next edge comes from the row's integer alias table
 *   instead (Algorithm 1, Sec. 2.2): slot j = floor(r64 * d / 2^64),
 *   y = floor(((r64 * d) mod 2^64) * W_u / 2^64), edge j if y < thr(j), else
 *   its alias; the same law, a different map from draws to edges.
 *   A node with no out-edge restarts the walk at its source (Sec. 2.1;
 *   dangling = 0) or ends the walk there without a step (dangling = 1).
 *   Segment mode (Algorithm 4, "big moves", fixed depth 3, out-degree <= 8)
 *   replaces a plain step at an eligible node by one draw over that node's
 *   precomputed outcome table; its counts follow a different draw sequence
 *   and are therefore compared against the segment-mode oracle.
 *
 * Conventions
 *   - Every function returns an int status: PPR_OK (0) or a negative code.
 *     No C++ exception, abort or device trap crosses this boundary.
 *     ppr_last_error() gives a message for the last failure on this thread.
 *   - Host inputs are copied during the call; device inputs (flag
 *     PPR_PTRS_DEVICE) are read during the call and not retained.
 *   - The library owns graphs and results until ppr_free_graph /
 *     ppr_free_result.  Output arrays are caller-allocated, host memory unless
 *     PPR_PTRS_DEVICE is passed.
 *   - A context is used by one host thread at a time.
 */
#ifndef PPR_H
#define PPR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPR_ABI_VERSION 1

enum {
    PPR_OK = 0,
    PPR_EINVAL = -1,   /* invalid argument or malformed graph */
    PPR_ENOMEM = -2,   /* device or pinned-host allocation failed */
    PPR_ECUDA = -3,    /* CUDA runtime error (no device, launch failure, ...) */
    PPR_ETIMEOUT = -4, /* deadline passed before the work finished */
    PPR_ERANGE = -5,   /* size beyond a documented limit */
    PPR_EBUSY = -6,    /* result not ready (ppr_wait not yet successful) */
    PPR_ENOTSUP = -7   /* combination not supported */
};

/* flags */
#define PPR_PTRS_DEVICE 0x1u /* pointer arguments are device pointers */
/* Node numbering of the device layout (ppr_load_graph; plain graphs only).
 * With PPR_RENUMBER the layout numbers nodes by descending in-degree (counted
 * on every fourth edge, eight classes per power of two, ties in caller
 * order) so that the records and rows of the most visited nodes are
 * contiguous; PPR_KEEP_IDS keeps the caller's order; with neither, the
 * layout renumbers when its node records (32 bytes a node) exceed twice the
 * device's L2.  The numbering is internal:
 * sources, rows and top-k use the caller's ids, walks draw by the caller's
 * source id, and every result is the same either way. */
#define PPR_RENUMBER 0x2u
#define PPR_KEEP_IDS 0x4u

/* Documented limits. */
#define PPR_MAX_NODES 2147483647LL        /* n < 2^31 */
#define PPR_MAX_EDGES 1099511627775LL     /* m < 2^40 */
#define PPR_MAX_DEGREE 8388607LL          /* out-degree < 2^23 */
#define PPR_MAX_R 4096u                   /* walks per source */

typedef struct ppr_ctx ppr_ctx;
typedef struct ppr_graph ppr_graph;
typedef struct ppr_result ppr_result;

/* Library ABI version (PPR_ABI_VERSION).  Needs no GPU. */
int ppr_version(void);

/* T = floor(alpha * 2^32) (Sec. 2.1 termination probability as an integer
 * threshold), or 0 if alpha is not in (0,1) or T would be 0.  Needs no GPU. */
uint32_t ppr_alpha_threshold(double alpha);

/* Walks per source for Definition 1 (fully approximate PPR): the smallest
 * omega with
 *     omega >= (2 + 2*eps/3) * ln(2 / p_f) / (eps^2 * delta),
 * so that every pi(s,t) >= delta is estimated within eps * pi(s,t) with
 * probability at least 1 - p_f.  The paper fixes omega only up to a constant,
 * Omega(log(1/p_f) / (eps^2 delta)) (Sec. 2.1); the constant here is the
 * two-sided Bernstein bound P(|X - mu| >= eps mu) <= 2 exp(-eps^2 mu / (2 + 2 eps/3))
 * for X a sum of omega independent indicators with mean mu = omega * pi >=
 * omega * delta.  Needs no GPU.  PPR_EINVAL unless eps > 0, 0 < delta <= 1,
 * 0 < p_f < 1; PPR_ERANGE if omega >= 2^53.  An omega above PPR_MAX_R is
 * reached by summing the rows of runs that differ only in their tag (the tag
 * is a Philox counter word, so the runs' walks are independent). */
int ppr_walks_for_accuracy(double eps, double delta, double p_f, uint64_t *omega);

/* Message describing the last failure on the calling thread ("" if none).
 * Owned by the library; valid until the next call on this thread. */
const char *ppr_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts).  Needs no GPU. */
int64_t ppr_kernel_launches(void);

/* Creates a context on CUDA device `device`; *out receives it.
 * PPR_ECUDA if the device cannot be used. */
int ppr_create(int device, ppr_ctx **out);
/* Stops serving and drops the caller's handle.  Graphs and results made in
 * the context keep it alive until they are freed, so handles may be freed
 * in any order; the handle itself must not be used again. */
void ppr_destroy(ppr_ctx *ctx);

/* Number of streaming multiprocessors of the context's device. */
int ppr_device_sms(const ppr_ctx *ctx);

/*
 * Loads a weighted directed graph G = (V, E, w), w(e) > 0 (Sec. 2.1), in CSR
 * form and builds its device layout: node records (32 bytes, with the top
 * level of the row's search tree, when every row total is below 2^32; else
 * 16 bytes) and per-row inclusive 64-bit weight prefix sums (stored as
 * 32-bit values when every row total is below 2^32), built by device kernels.
 *   n        number of nodes, 1 <= n <= PPR_MAX_NODES
 *   m        number of edges, 0 <= m <= PPR_MAX_EDGES
 *   row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col      int32[m], each in [0, n)      (edge targets, row order kept)
 *   w        uint32[m], each >= 1          (integer edge weights)
 *   flags    PPR_PTRS_DEVICE if the three arrays are device pointers;
 *            PPR_RENUMBER or PPR_KEEP_IDS (not both) to force the layout's
 *            node numbering (above)
 *   stream   cudaStream_t for the build, or NULL for the legacy stream
 * Errors: PPR_EINVAL (malformed CSR, col out of range, w = 0),
 *         PPR_ERANGE (n, m or an out-degree beyond the limits), PPR_ENOMEM.
 * The call returns after the build has finished.
 */
int ppr_load_graph(ppr_ctx *ctx, int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                   const uint32_t *w, uint32_t flags, void *stream, ppr_graph **out);

/*
 * Loads `count` independent graphs as one block-diagonal graph.  Instance g
 * owns global nodes [node_off[g], node_off[g+1]); row_ptr (n_total+1 entries,
 * n_total = node_off[count]) indexes the concatenated edge arrays; col holds
 * INSTANCE-LOCAL target ids.  Walks of a source s of instance g draw with
 * counter (s - node_off[g], j, k, g): identical to running instance g alone
 * with tag = g.  Result rows of such a graph hold instance-local end ids.
 * Errors as ppr_load_graph.
 */
int ppr_load_graph_batch(ppr_ctx *ctx, int32_t count, const int64_t *node_off, int64_t m,
                         const int64_t *row_ptr, const int32_t *col, const uint32_t *w, uint32_t flags,
                         void *stream, ppr_graph **out);

typedef struct {
    int64_t n, m;
    int64_t max_degree;
    int64_t dangling;        /* nodes with no out-edge */
    int32_t wide;            /* 1 if some row total is >= 2^32 (64-bit prefix layout) */
    int32_t instances;       /* 0 for a plain graph */
    int64_t device_bytes;    /* device memory held by the graph */
    int64_t segment_nodes;   /* nodes with a segment table (last built threshold) */
    int64_t segment_entries;
    int32_t renumbered;      /* 1 if the layout numbers nodes by in-degree (PPR_RENUMBER) */
    int32_t reserved;
} ppr_graph_info;

int ppr_graph_get_info(const ppr_graph *g, ppr_graph_info *info);
/* Frees the graph's device memory after waiting for the device to go idle
 * (runs on any stream may still read it). */
void ppr_free_graph(ppr_graph *g);

/* Walker kernels. */
enum {
    PPR_KERNEL_PERSISTENT = 0, /* persistent warps, work queue, lane refill; per-source reduction kernel */
    PPR_KERNEL_PLAIN = 1       /* one thread per walk, endpoints to HBM, separate aggregation */
};

typedef struct {
    double alpha;        /* termination probability, floor(alpha*2^32) >= 1, alpha < 1 */
    uint32_t R;          /* walks per source, 1 <= R <= PPR_MAX_R */
    uint64_t seed;       /* Philox key */
    int64_t src_begin;   /* sources [src_begin, src_end), global node ids */
    int64_t src_end;
    uint32_t tag;        /* fourth counter word (plain graphs; batched graphs use the instance id) */
    int32_t dangling;    /* 0 restart at the source (Sec. 2.1), 1 end at the dangling node */
    int32_t segments;    /* 1: depth-3 segment tables for out-degree <= 8 (Algorithm 4) */
    int32_t topk;        /* 0..PPR_MAX_R: per-source top-k (count desc, end id asc) kept with the
                            rows; entries past the row's distinct endpoints are (-1, 0) */
    int32_t kernel;      /* PPR_KERNEL_PERSISTENT or PPR_KERNEL_PLAIN */
    int32_t large_degree;/* out-degree above which the whole warp searches a lane's row
                            cooperatively (persistent kernel); 0 = never (default) */
    int32_t warps_per_block;  /* persistent kernel: 4 or 8 warps per CTA (0 = 8) */
    int32_t chunk_sources;    /* sources per queue item, 0 = default */
    int64_t max_batch_sources;/* sources per device batch, 0 = sized to free device memory */
    int32_t stats;       /* 1: also count the algorithmic 32-byte sectors of every step (slower;
                            rows, counts and steps are unchanged) */
    int32_t sampler;     /* neighbour choice: 0 = first prefix above floor(r*W/2^64) (default);
                            1 = integer alias method (Algorithm 1): slot j = floor(r*d/2^64),
                            y = floor(((r*d) mod 2^64) * W / 2^64), edge j if y < thr(j) else
                            its alias.  Same law, different counts.  Alias tables are built on
                            the first run that asks for them (every row total < 2^32; no
                            segment mode) */
    int32_t l2_persist;  /* 1: walker launches mark the node records persisting in L2 (an
                            access-policy window; the device's persisting set-aside is raised
                            for this context on first use); 0: off.  Results are unchanged */
    int32_t refill_lanes;/* persistent kernel: a warp starts new walks once at least this many of
                            its 32 lanes are idle, and then fills every idle lane (1..32; 0 = 1,
                            at once).  32 starts a warp's walks together, like one thread per
                            walk, so the first steps of a source's walks share their loads.
                            Results are unchanged */
    void *stream;        /* cudaStream_t, NULL = legacy default stream */
    int32_t step_loads;  /* persistent kernel, prefix sampler on 32-bit rows, no cooperative
                            search, no statistics: the dependent loads one lane may spend on a
                            draw in one warp iteration (the node record counts as one); a
                            deeper search resumes in the next iteration while the warp's other
                            lanes start new draws.  0 = the library's choice (6); -1 = none
                            (each iteration finishes every lane's draw); 2..16.  Results are
                            unchanged */
} ppr_run_args;

/* Fills *args with defaults (alpha 0.15, R 100, seed 1, all sources of
 * nothing: src_end = src_begin = 0, persistent kernel). */
void ppr_run_args_init(ppr_run_args *args);

/*
 * Runs the walks of every source in [src_begin, src_end) (Algorithm 2 with
 * all walks of a source counted, then grouped by endpoint) and keeps, per
 * source, its sparse count row (end id ascending, counts summing to R) and
 * its top-k.  Work is enqueued on args->stream; call ppr_wait before reading.
 * Errors: PPR_EINVAL (alpha, R, range, topk), PPR_ERANGE (R > PPR_MAX_R),
 *         PPR_ENOMEM, PPR_ECUDA.
 */
int ppr_run(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *args, ppr_result **out);

/*
 * As ppr_run, for an explicit list of `count` source node ids (host memory,
 * copied; each in [0, n); repeats allowed).  Row i of the result belongs to
 * sources[i]; walks of that source use its node id in the counter, so a row
 * equals the row ppr_run gives for the same node.  args->src_begin/src_end are
 * ignored.  Plain graphs only (PPR_ENOTSUP for batched graphs).
 */
int ppr_run_list(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *args, const int32_t *sources, int64_t count,
                 ppr_result **out);

/* Bytes of device workspace ppr_run_into needs for these arguments. */
int ppr_workspace_size(const ppr_graph *g, const ppr_run_args *args, size_t *bytes);

/*
 * ppr_run into caller-owned device memory: the workspace (>= ppr_workspace_size
 * bytes, 256-byte aligned) holds the per-walk endpoints and counters, and the
 * rows and top-k go to the caller's buffers (layout as ppr_run_noalloc below).
 * Persistent kernel only; segment tables must already exist for this alpha.
 * The call only enqueues work on args->stream: no allocation, no host copy and
 * no synchronization, so it may be recorded into a CUDA graph.  Two calls that
 * share a workspace and overlap on the GPU race.
 */
int ppr_run_into(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *args, void *workspace, size_t bytes,
                 uint32_t *nnz, int32_t *cols, uint32_t *cnts, uint32_t cap, int32_t *topk_idx, uint32_t *topk_cnt);

/* Launch tuning chosen by ppr_autotune. */
typedef struct {
    int32_t chunk_sources;   /* sources per work-queue item */
    int32_t large_degree;    /* cooperative-search threshold (0 = off) */
    int32_t warps_per_block; /* walkers per CTA / 32 (4 or 8) */
    float ms;                /* device time of the best candidate on the sample */
    int32_t candidates;      /* candidates timed */
    int64_t sample_sources;  /* sources in the sample */
    int32_t refill_lanes;    /* idle lanes before a warp starts new walks (1..32) */
} ppr_tuning;

/*
 * Times the persistent walker on a sample of the run's sources (at most
 * sample_sources, 0 = 65536; evenly strided for plain graphs, a leading range
 * for batched graphs) for each candidate of walkers per CTA (128, 256), queue
 * chunk (1/4x .. 4x of 400/R sources) and cooperative threshold (off, 4096,
 * 65536), then, with the fastest of those, for refill thresholds of 8, 16,
 * 24 and 32 idle lanes (against 1), and returns the fastest.  Synchronous;
 * allocates scratch for the sample.  Tuning never changes results.
 */
int ppr_autotune(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *args, int64_t sample_sources, ppr_tuning *best);

/* Waits for the run; PPR_ETIMEOUT if not finished within timeout_ms
 * (timeout_ms < 0: wait without deadline).  The result stays valid. */
int ppr_wait(ppr_result *r, int64_t timeout_ms);

typedef struct {
    int64_t sources;       /* S = src_end - src_begin */
    uint32_t R;
    int32_t topk;
    int64_t nnz;           /* total stored (source, end) pairs */
    uint64_t steps;        /* draws consumed by all walks */
    uint64_t walks;        /* S * R */
    float kernel_ms;       /* device time of the walker launches alone (CUDA events) */
    uint64_t sectors;      /* stats runs: 32-byte sectors the row searches read, node records
                              included (0 otherwise) */
    float run_ms;          /* device time of the whole run: walkers and reductions */
    uint64_t model_sectors; /* stats runs: the same draws costed on a flat CSR searched by
                               bisection, in 32-byte sectors without reuse: per draw at a node
                               of out-degree d >= 1, one row_ptr sector, max(1, ceil(log2 d) - 1)
                               prefix-probe sectors and one col sector; 1 at a dangling node;
                               1 + (1 or 2) table sectors for a segment draw (<= 2 outcomes: 1);
                               the alias sampler's node and slot sectors as counted (0 otherwise) */
} ppr_result_info;

int ppr_result_get_info(const ppr_result *r, ppr_result_info *info);

/*
 * Runs the walks of args (range of sources) and delivers the compacted rows
 * and the top-k straight into host memory, pipelined against the walks
 * (the batching of the paper's pipelines, Sec. 4.3, with the output stream
 * of each batch overlapped with the next batch's walks): the sources are
 * cut into `parts` batches (0 = the library's choice), the last of which is
 * cut once more into three quarters and a quarter (when there are two or
 * more), so that little copying is left after the last walk; while batch
 * i+1 walks on args->stream, batch i's rows are compacted and copied to the
 * host on a second stream of the library's own.  Returns when every row is
 * in place.
 *   row_ptr  int64[S+1] (row s = entries [row_ptr[s], row_ptr[s+1]))
 *   col, cnt int32 / uint32 [cap]; cap >= nnz or PPR_ERANGE (nothing beyond
 *            cap is written; row_ptr is then incomplete)
 *   nnz      out: total entries (may be NULL)
 *   topk_idx, topk_cnt  [S * args->topk] or NULL when args->topk == 0
 *   info     out: steps, walks, walker time (may be NULL)
 * Host buffers should be page-locked (cudaHostAlloc or cudaHostRegister) for
 * the copies to overlap the walks; pageable buffers work, serialised.
 * Plain and batched graphs; source lists are not taken here.  Errors as
 * ppr_run, plus PPR_ERANGE for cap.
 */
int ppr_run_to_host(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *args, int32_t parts, int64_t *row_ptr,
                    int32_t *col, uint32_t *cnt, int64_t cap, int64_t *nnz, int32_t *topk_idx, uint32_t *topk_cnt,
                    ppr_result_info *info);


/*
 * Copies the sparse rows: row_ptr (S+1 entries), then col/cnt (nnz entries).
 * If col == NULL only row_ptr (may be NULL too) and *nnz are produced.
 * PPR_ERANGE if cap < nnz.  flags: PPR_PTRS_DEVICE for device outputs.
 */
int ppr_sparse_rows(const ppr_result *r, int64_t *row_ptr, int32_t *col, uint32_t *cnt, int64_t cap,
                    int64_t *nnz, uint32_t flags);

/* Top-k per source, S*k entries each: idx (end ids, -1 padded) and cnt
 * (counts, 0 padded), count descending then end id ascending.
 * 1 <= k <= the run's topk, else PPR_EINVAL. */
int ppr_topk(const ppr_result *r, int32_t k, int32_t *idx, uint32_t *cnt, uint32_t flags);

/* Dense S x n uint32 counts (plain graphs only). */
int ppr_dense(const ppr_result *r, uint32_t *out, uint32_t flags);

void ppr_free_result(ppr_result *r);

/*
 * Allocation-free run (no counterpart in the paper: it serves callers, not the
 * method).  Some callers cannot allocate device memory while they work: a
 * process whose other framework already holds nearly all device memory in its
 * own caching pool, or a serving loop that must not take the time or the risk
 * of a driver allocation once it is running.  This entry point runs the same
 * walks and reduction as ppr_run with the persistent kernel but makes no
 * allocation of any kind: the caller passes the graph (already loaded) and
 * device output buffers, and the per-walk endpoints live in a fixed 64 MiB
 * scratch array that the library keeps in device memory on every GPU that
 * loads it, until the process exits.
 *   nnz      uint32[S]            distinct endpoints of each source
 *   cols     int32[S * cap]       row s at cols[s*cap .. s*cap+nnz[s]), end ids ascending
 *   cnts     uint32[S * cap]      the matching counts (each row sums to R)
 *   cap      >= min(R, n)
 *   topk_idx, topk_cnt  S * topk entries as ppr_topk, or NULL when topk = 0
 * S * R may be at most 16,777,152 walks (64 MiB minus a 256-byte header, 4 B
 * per walk); larger calls fail with PPR_ERANGE before any work is queued.
 * Arguments are checked as ppr_run checks them (same limits, same codes),
 * then: plain graphs and args->kernel = PPR_KERNEL_PERSISTENT only, no
 * statistics; segment mode needs tables already built for this alpha, and
 * the alias sampler tables already built, by an earlier ppr_run (else
 * PPR_ENOTSUP: building them would allocate).
 * The work is queued on args->stream and the call returns at once: the
 * outputs are valid after that stream is synchronized.  The first call on a
 * device looks up the scratch array's device address (cudaGetSymbolAddress)
 * for that device; make that first call before any stream capture.  The
 * address is kept per device ordinal for the life of the process, so it
 * assumes the device's primary context is never reset (cudaDeviceReset, or
 * a framework's equivalent) while the library is loaded.  Every
 * call shares the one scratch array, whose counters each call clears and
 * whose contents a later call overwrites: calls whose work overlaps on the
 * GPU (other streams, or without a synchronization between them) race.
 */
int ppr_run_noalloc(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *args, uint32_t *nnz, int32_t *cols,
                    uint32_t *cnts, uint32_t cap, int32_t *topk_idx, uint32_t *topk_cnt);

/* Fault injection for tests (host side; no device fault): after `after`
 * further device allocations by this library, every allocation fails with
 * PPR_ENOMEM as if the device were full, until the next call; after < 0
 * turns it off.  Process-wide. */
void ppr_debug_fail_allocs(int64_t after);

/* ------------------------------------------------------------- probes ----
 * Measurement beside the walk path; neither is part of a run.
 *
 * ppr_probe_philox: the device's Philox4x32-10 words (the generator of every
 * walk step, Salmon et al., SC'11) for counters (c0 + i mod 2^32, c1, c2, c3),
 * i in [0, count), key (seed mod 2^32, seed >> 32); out: host uint32[4*count],
 * words x0..x3 of each counter in turn.  1 <= count <= 2^28.
 *
 * ppr_probe_rate: kind 0 = chains of dependent random 32-byte sector reads
 * over a device buffer of `bytes` (the access pattern of a walk step on
 * uniform addresses; one resident wave of threads, 256 reads per thread);
 * kind 2 = independent random 32-byte sector reads, four in flight per
 * thread (the random-access bandwidth for sector-sized reads); both give
 * *per_second = sectors read per second.  kind 1 = Philox4x32-10 draws per
 * second (bytes ignored).  *ms (may be NULL) = the timed kernel's duration.
 * Allocates and frees its buffer on the legacy default stream.
 */
int ppr_probe_philox(ppr_ctx *ctx, uint64_t seed, const uint32_t counter[4], int64_t count, uint32_t *out);
int ppr_probe_rate(ppr_ctx *ctx, int32_t kind, int64_t bytes, double *per_second, float *ms);

/* ---------------------------------------------------------------- serving
 * Multi-source queries with continuous batching: a scheduler thread admits
 * queries in arrival order as soon as one of `streams` device slots is free
 * and the query's device memory fits the budget left by the queries in
 * flight; queries run concurrently on their own streams.  Each query returns
 * the top-k of every one of its sources (same counts as ppr_run_list with
 * the same alpha, R and seed; tag 0, dangling mode 0, plain steps).
 */
/*
 * Serving (continuous batching of multi-source queries, Sec. 3's pipelines
 * applied to a query stream).  Two modes:
 *   PPR_SERVE_DEVICE_LOOP (default): one persistent kernel stays resident and
 *     serves every query.  The host admits queries in arrival order as device
 *     memory and one of 64 ring slots allow, copies their sources to the
 *     device and publishes them through host-mapped memory; walker warps take
 *     chunks of walks from all published queries (each warp starting at its
 *     own query, so small queries are not held behind large ones) and refill
 *     lanes as walks end, a lane carrying walks of different queries at once;
 *     a query whose walks are all done is reduced source by source by the
 *     loop's aggregator warps, which write its top-k rows straight into pinned
 *     host memory and mark it done.  Every wait on the device is bounded: the
 *     loop exits after `idle_us` without work and is launched again with the
 *     next query.  R <= 1024 per query.
 *   PPR_SERVE_STREAMS: a host scheduler runs each admitted query as its own
 *     persistent walker launch and reduction on one of `streams` streams.
 * Results are identical in both modes: query rows are ppr_run_list's rows of
 * the same sources (tag 0, dangling mode 0, no segment tables).
 */
enum { PPR_SERVE_DEVICE_LOOP = 0, PPR_SERVE_STREAMS = 1 };

typedef struct {
    int32_t streams;        /* stream mode: concurrent queries on the device (default 4) */
    int64_t max_sources;    /* sources per query (default 100000) */
    int32_t max_topk;       /* largest k a query may ask for (0 = 64) */
    int64_t memory_budget;  /* device bytes for queries in flight (0 = a quarter of free memory) */
    int64_t max_pending;    /* queries waiting for admission before ppr_submit returns PPR_EBUSY (0 = no limit) */
    int32_t chunk_sources, large_degree, warps_per_block; /* walker tuning (0 = defaults; the device loop
                               takes chunk_sources only) */
    int32_t sampler;        /* neighbour choice of every query, as ppr_run_args.sampler; with 1
                               the graph's alias tables are built by ppr_serve_start */
    int32_t refill_lanes;   /* as ppr_run_args.refill_lanes (0 = 1) */
    int32_t mode;           /* PPR_SERVE_DEVICE_LOOP (0) or PPR_SERVE_STREAMS (1) */
    int64_t idle_us;        /* device loop: idle time after which the resident kernel exits
                               (0 = 200,000 us); the next query launches it again */
} ppr_serve_cfg;

typedef struct {
    int64_t submit_ns, admit_ns, done_ns; /* steady-clock times of submission, admission, completion */
    uint64_t walks;
    int64_t sources;
    int64_t device_walk_ns;   /* device loop: from its first chunk taken to its last walk counted */
    int64_t device_reduce_ns; /* device loop: from its last walk counted to its last top-k row */
} ppr_query_stats;

typedef struct {
    int32_t mode;           /* the serving mode */
    uint32_t status;        /* device loop: exit reasons of its last launch (PPR_LOOP_*) */
    int64_t launches;       /* device loop launches so far */
    int64_t idle_exits;     /* launches that ended on the idle bound */
    int64_t in_flight;      /* queries admitted and not finished */
    int64_t completed;      /* queries finished */
    int32_t running;        /* the device loop is on the GPU now */
    /* device loop activity since serving started (each warp adds its counts about once a
       millisecond and when it exits): */
    uint64_t draws;         /* draws (walk steps) taken */
    uint64_t iterations;    /* walker-warp iterations that stepped at least one walk */
    uint64_t claims;        /* attempts of a walker warp to take a chunk of walks */
    uint64_t claim_misses;  /* attempts that found none */
    uint64_t sleeps;        /* waits of a walker warp with no walk and no chunk */
    uint64_t reduced;       /* sources reduced to their top-k */
    uint64_t cycles_claim, cycles_step, cycles_sleep, cycles_total; /* walker-warp SM clock cycles:
                               taking chunks, stepping walks, waiting, and in all */
    int32_t grid_blocks;    /* blocks of the device loop (8 warps each: 7 walk, 1 reduces) */
} ppr_serve_info;

/* Device loop exit reasons (ppr_serve_info.status). */
enum { PPR_LOOP_STOPPED = 1, PPR_LOOP_IDLE = 2, PPR_LOOP_SLOT_TIMEOUT = 4, PPR_LOOP_BUSY_TIMEOUT = 8 };

void ppr_serve_cfg_init(ppr_serve_cfg *cfg);

/* State of the server of ctx (PPR_EINVAL if serving is not started). */
int ppr_serve_get_info(ppr_ctx *ctx, ppr_serve_info *info);

/* Test hook (device loop; host side, no device fault): publishes a ring slot
 * that the host never wrote.  The loop's bounded wait for that slot's
 * descriptor (one second) runs out, the loop exits with
 * PPR_LOOP_SLOT_TIMEOUT, queries in flight fail with PPR_ECUDA and the server
 * accepts no more queries until ppr_serve_stop; the context stays usable. */
int ppr_debug_serve_publish_unwritten(ppr_ctx *ctx);

/* Starts serving graph g (plain graphs) on the context; one server per context. */
int ppr_serve_start(ppr_ctx *ctx, const ppr_graph *g, const ppr_serve_cfg *cfg);

/* Stops serving: queries not yet admitted are cancelled (their poll fails with
 * PPR_EINVAL); running queries finish first.  ppr_destroy stops it too. */
int ppr_serve_stop(ppr_ctx *ctx);

/*
 * Queues a query for `ns` source ids (host memory, copied; each in [0, n)).
 * Thread-safe.  *qid identifies it for ppr_poll.  Errors: PPR_EINVAL (bad
 * arguments, serving not started), PPR_ERANGE (larger than the memory budget),
 * PPR_EBUSY (max_pending reached, or stopping).
 */
int ppr_submit(ppr_ctx *ctx, const int32_t *srcs, int64_t ns, double alpha, uint32_t R, uint64_t seed, int32_t topk,
               uint64_t *qid);

/*
 * Waits up to timeout_ms (< 0: no deadline) for query qid.  On success writes
 * its top-k (ns * topk ids and counts, row i for srcs[i], as ppr_topk) into
 * idx / cnt (host memory, either may be NULL), fills *stats if non-NULL, and
 * forgets the query.  PPR_ETIMEOUT leaves it pending.  Thread-safe.
 */
int ppr_poll(ppr_ctx *ctx, uint64_t qid, int32_t *idx, uint32_t *cnt, int64_t timeout_ms, ppr_query_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* PPR_H */
