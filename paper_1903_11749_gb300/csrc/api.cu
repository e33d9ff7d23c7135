// api.cu -- the extern "C" entry points of libppr.so (declared in
// include/ppr.h): argument checks, ownership of device state, batching of a
// source range into device-sized launches, and the row/top-k/dense readers.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "ppr_host.h"
#include "scan.cuh"

#include <atomic>

namespace {
thread_local char g_err[512] = "";
std::atomic<long long> g_launches{0};
}

namespace ppr {

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return PPR_ENOMEM;
    return PPR_ECUDA;
}

// Device memory comes from the device's default stream-ordered pool, which
// the context sets to keep freed memory reserved: repeated runs reuse it
// without cudaMalloc/cudaFree round trips to the driver.
// Host-side fault injection (ppr_debug_fail_allocs): allocations left before
// every further one fails; negative = off.
static std::atomic<long long> g_allocs_left{-1};

int dev_alloc(void **p, size_t bytes, const char *what, cudaStream_t st)
{
    *p = nullptr;
    if (g_allocs_left.load(std::memory_order_relaxed) >= 0 && g_allocs_left.fetch_sub(1) <= 0) {
        g_allocs_left.store(0);
        set_error("cannot allocate %zu bytes of device memory for %s: injected failure", bytes, what);
        return PPR_ENOMEM;
    }
    cudaError_t e = cudaMallocAsync(p, bytes > 0 ? bytes : 1, st);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free allocation error
        *p = nullptr;
        set_error("cannot allocate %zu bytes of device memory for %s: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PPR_ENOMEM : PPR_ECUDA;
    }
    return PPR_OK;
}

void dev_free(void *p, cudaStream_t st)
{
    if (p) cudaFreeAsync(p, st);
}

// Row compaction: one warp per source copies its stored pairs to the
// compacted position given by the exclusive scan of the row sizes.
__global__ void k_compact_rows(int64_t S, uint32_t cap, const uint32_t *nnz, const uint64_t *off, const int32_t *cols,
                               const uint32_t *cnts, int32_t *ocol, uint32_t *ocnt)
{
    const uint32_t lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += warps) {
        const uint32_t c = nnz[s];
        const uint64_t o = off[s];
        for (uint32_t i = lane; i < c; i += 32) {
            ocol[o + i] = cols[(uint64_t)s * cap + i];
            ocnt[o + i] = cnts[(uint64_t)s * cap + i];
        }
    }
}

// Row starts of one batch made absolute: off[i] += *base, the entries of the
// batches before it (kept on the device, so the batch needs no host round trip).
__global__ void k_add_base(int64_t n, uint64_t *off, const unsigned long long *base)
{
    const uint64_t b = *base;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        off[i] += b;
}

// The running base after a batch: its last absolute row start.
__global__ void k_next_base(unsigned long long *base, const uint64_t *off_end) { *base = *off_end; }

__global__ void k_dense(int64_t S, int64_t n, uint32_t cap, const uint32_t *nnz, const int32_t *cols,
                        const uint32_t *cnts, uint32_t *out)
{
    const uint32_t lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += warps) {
        const uint32_t c = nnz[s];
        for (uint32_t i = lane; i < c; i += 32)
            out[(uint64_t)s * n + (uint32_t)cols[(uint64_t)s * cap + i]] = cnts[(uint64_t)s * cap + i];
    }
}

void ctx_retain(ppr_ctx *ctx)
{
    if (ctx) ctx->refs.fetch_add(1);
}

void ctx_release(ppr_ctx *ctx)
{
    if (!ctx || ctx->refs.fetch_sub(1) != 1) return;
    if (ctx->copy_stream || ctx->pinned) {
        cudaSetDevice(ctx->device);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        if (ctx->pinned) cudaFreeHost(ctx->pinned);
        cudaGetLastError();
    }
    delete ctx;
}
}  // namespace ppr

using namespace ppr;

static int set_device(const ppr_ctx *ctx)
{
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    // a sticky error means the context is lost; anything else is left over from
    // an unchecked call (a release path) and must not fail this one
    e = cudaGetLastError();
    if (e != cudaSuccess && cudaPeekAtLastError() != cudaSuccess) return cuda_fail(e, "device");
    return PPR_OK;
}

extern "C" {

int ppr_version(void) { return PPR_ABI_VERSION; }

uint32_t ppr_alpha_threshold(double alpha)
{
    if (!(alpha > 0.0) || !(alpha < 1.0)) return 0u;
    double t = alpha * 4294967296.0;  // exact: scaling by a power of two
    return (uint32_t)t;
}

void ppr_debug_fail_allocs(int64_t after) { g_allocs_left.store(after < 0 ? -1 : after); }

int ppr_walks_for_accuracy(double eps, double delta, double p_f, uint64_t *omega)
{
    if (!omega || !(eps > 0.0) || !(delta > 0.0) || !(delta <= 1.0) || !(p_f > 0.0) || !(p_f < 1.0)) {
        set_error("need eps > 0, 0 < delta <= 1, 0 < p_f < 1 and an output pointer");
        return PPR_EINVAL;
    }
    const double w = (2.0 + 2.0 * eps / 3.0) * std::log(2.0 / p_f) / (eps * eps * delta);
    if (!(w < 9007199254740992.0)) {
        set_error("omega = %g is beyond 2^53", w);
        return PPR_ERANGE;
    }
    *omega = (uint64_t)std::ceil(w);
    return PPR_OK;
}

const char *ppr_last_error(void) { return g_err; }

int64_t ppr_kernel_launches(void) { return (int64_t)g_launches.load(); }

int ppr_create(int device, ppr_ctx **out)
{
    if (!out) {
        set_error("out is NULL");
        return PPR_EINVAL;
    }
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        set_error("no CUDA device available: %s", e != cudaSuccess ? cudaGetErrorString(e) : "count is 0");
        return PPR_ECUDA;
    }
    if (device < 0 || device >= count) {
        set_error("device %d out of range [0, %d)", device, count);
        return PPR_EINVAL;
    }
    PPR_CUDA(cudaSetDevice(device));
    ppr_ctx *c = new (std::nothrow) ppr_ctx;
    if (!c) {
        set_error("host allocation failed");
        return PPR_ENOMEM;
    }
    c->device = device;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    c->sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxPersistingL2CacheSize, device);
    c->l2_persist_max = (size_t)v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxAccessPolicyWindowSize, device);
    c->l2_window_max = (size_t)v;
    cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, device);
    c->l2_bytes = (size_t)v;
    ppr::preload_run_kernels();
    {
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k_compact_rows);
        cudaFuncGetAttributes(&fa, k_dense);
        cudaFuncGetAttributes(&fa, k_add_base);
        cudaFuncGetAttributes(&fa, k_next_base);
        cudaGetLastError();
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = ~0ull;  // keep freed blocks reserved for reuse
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    *out = c;
    return PPR_OK;
}


void ppr_destroy(ppr_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->server) ppr_serve_stop(ctx);
    ctx_release(ctx);
}

int ppr_device_sms(const ppr_ctx *ctx) { return ctx ? ctx->sms : 0; }

static int load_common(ppr_ctx *ctx, int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                       const uint32_t *w, uint32_t flags, void *stream, ppr_graph *g)
{
    if (n < 1 || n > PPR_MAX_NODES) {
        set_error("n = %lld outside [1, %lld]", (long long)n, (long long)PPR_MAX_NODES);
        return n < 1 ? PPR_EINVAL : PPR_ERANGE;
    }
    if (m < 0 || m > PPR_MAX_EDGES) {
        set_error("m = %lld outside [0, %lld]", (long long)m, (long long)PPR_MAX_EDGES);
        return m < 0 ? PPR_EINVAL : PPR_ERANGE;
    }
    if (!row_ptr || (m > 0 && (!col || !w))) {
        set_error("row_ptr, col and w must be non-NULL");
        return PPR_EINVAL;
    }
    if (flags & ~(PPR_PTRS_DEVICE | PPR_RENUMBER | PPR_KEEP_IDS)) {
        set_error("unknown flags 0x%x", flags);
        return PPR_EINVAL;
    }
    if ((flags & PPR_RENUMBER) && (flags & PPR_KEEP_IDS)) {
        set_error("PPR_RENUMBER and PPR_KEEP_IDS exclude each other");
        return PPR_EINVAL;
    }
    if ((flags & PPR_RENUMBER) && g->instances > 0) {
        set_error("PPR_RENUMBER applies to plain graphs (batched instances keep their numbering)");
        return PPR_EINVAL;
    }
    int rc = set_device(ctx);
    if (rc) return rc;
    Range range("ppr_load_graph");
    g->ctx = ctx;
    ctx_retain(ctx);
    g->n = n;
    g->m = m;
    g->stream = (cudaStream_t)stream;
    // node records of 32 bytes: renumber when they would take more than twice the L2
    const bool renumber = g->instances == 0 && ((flags & PPR_RENUMBER) != 0 ||
                                                ((flags & PPR_KEEP_IDS) == 0 && (uint64_t)n * 32 > 2 * ctx->l2_bytes));
    return build_graph(ctx, n, m, row_ptr, col, w, (flags & PPR_PTRS_DEVICE) != 0, renumber, (cudaStream_t)stream, g);
}

int ppr_load_graph(ppr_ctx *ctx, int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                   const uint32_t *w, uint32_t flags, void *stream, ppr_graph **out)
{
    if (!ctx || !out) {
        set_error("ctx and out must be non-NULL");
        return PPR_EINVAL;
    }
    *out = nullptr;
    ppr_graph *g = new (std::nothrow) ppr_graph;
    if (!g) return PPR_ENOMEM;
    int rc = load_common(ctx, n, m, row_ptr, col, w, flags, stream, g);
    if (rc) {
        ppr_free_graph(g);
        return rc;
    }
    *out = g;
    return PPR_OK;
}

int ppr_load_graph_batch(ppr_ctx *ctx, int32_t count, const int64_t *node_off, int64_t m, const int64_t *row_ptr,
                         const int32_t *col, const uint32_t *w, uint32_t flags, void *stream, ppr_graph **out)
{
    if (!ctx || !out || !node_off) {
        set_error("ctx, node_off and out must be non-NULL");
        return PPR_EINVAL;
    }
    *out = nullptr;
    if (count < 1) {
        set_error("count must be >= 1");
        return PPR_EINVAL;
    }
    // node_off is always host memory (count + 1 values)
    if (node_off[0] != 0) {
        set_error("node_off[0] must be 0");
        return PPR_EINVAL;
    }
    for (int32_t i = 0; i < count; ++i)
        if (node_off[i + 1] <= node_off[i]) {
            set_error("every instance needs at least one node (node_off strictly increasing)");
            return PPR_EINVAL;
        }
    ppr_graph *g = new (std::nothrow) ppr_graph;
    if (!g) return PPR_ENOMEM;
    g->instances = count;
    g->node_off.assign(node_off, node_off + count + 1);
    int rc = load_common(ctx, node_off[count], m, row_ptr, col, w, flags, stream, g);
    if (rc) {
        ppr_free_graph(g);
        return rc;
    }
    *out = g;
    return PPR_OK;
}

int ppr_graph_get_info(const ppr_graph *g, ppr_graph_info *info)
{
    if (!g || !info) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    info->n = g->n;
    info->m = g->m;
    info->max_degree = g->max_degree;
    info->dangling = g->dangling;
    info->wide = g->wide ? 1 : 0;
    info->instances = g->instances;
    info->device_bytes = g->device_bytes;
    info->segment_nodes = g->seg.nodes;
    info->segment_entries = g->seg.entries_n;
    info->renumbered = g->order ? 1 : 0;
    info->reserved = 0;
    return PPR_OK;
}

void ppr_free_graph(ppr_graph *g)
{
    if (!g) return;
    if (g->ctx) {
        cudaSetDevice(g->ctx->device);
        cudaDeviceSynchronize();  // runs on any stream may still read the graph
    }
    dev_free(g->node, g->stream);
    dev_free(g->edges, g->stream);
    dev_free(g->sum, g->stream);
    dev_free(g->seg.node, g->stream);
    dev_free(g->seg.entries, g->stream);
    dev_free(g->d_node_off, g->stream);
    dev_free(g->order, g->stream);
    dev_free(g->rank, g->stream);
    dev_free(g->alias.node, g->stream);
    dev_free(g->alias.slots, g->stream);
    cudaGetLastError();  // a failed free must not surface in a later call
    ctx_release(g->ctx);
    delete g;
}

void ppr_run_args_init(ppr_run_args *a)
{
    if (!a) return;
    memset(a, 0, sizeof(*a));
    a->alpha = 0.15;
    a->R = 100;
    a->seed = 1;
    a->kernel = PPR_KERNEL_PERSISTENT;
}

static void result_release(ppr_result *r)
{
    if (!r) return;
    if (r->ctx) cudaSetDevice(r->ctx->device);
    dev_free(r->d_nnz, r->stream);
    dev_free(r->d_cols, r->stream);
    dev_free(r->d_cnts, r->stream);
    dev_free(r->d_topk_idx, r->stream);
    dev_free(r->d_topk_cnt, r->stream);
    dev_free(r->d_steps, r->stream);
    for (void *p : r->scratch) dev_free(p, r->stream);
    if (r->ev_start) cudaEventDestroy(r->ev_start);
    if (r->ev_walk_end) cudaEventDestroy(r->ev_walk_end);
    if (r->ev_done) cudaEventDestroy(r->ev_done);
    for (cudaEvent_t ev : r->walk_events) cudaEventDestroy(ev);
    cudaGetLastError();  // a failed free must not surface in a later call
    ctx_release(r->ctx);
    delete r;
}

}  // extern "C"

namespace ppr {
// Checks shared by every run entry point; count = number of sources (from the
// range, or of an explicit list).  Fills *plan.
int check_run(const ppr_graph *g, const ppr_run_args *a, int64_t count, bool list, RunPlan *plan)
{
    const uint32_t T = ppr_alpha_threshold(a->alpha);
    if (T == 0) {
        set_error("alpha = %g: need 0 < alpha < 1 and floor(alpha * 2^32) >= 1", a->alpha);
        return PPR_EINVAL;
    }
    if (a->R < 1) {
        set_error("R must be >= 1");
        return PPR_EINVAL;
    }
    if (a->R > PPR_MAX_R) {
        set_error("R = %u exceeds the limit %u", a->R, PPR_MAX_R);
        return PPR_ERANGE;
    }
    if (!list && (a->src_begin < 0 || a->src_end > g->n || a->src_begin >= a->src_end)) {
        set_error("source range [%lld, %lld) must be non-empty and inside [0, %lld)", (long long)a->src_begin,
                  (long long)a->src_end, (long long)g->n);
        return PPR_EINVAL;
    }
    if (list && count < 1) {
        set_error("the source list is empty");
        return PPR_EINVAL;
    }
    if (a->topk < 0 || (uint32_t)a->topk > PPR_MAX_R) {
        set_error("topk = %d outside [0, %u]", a->topk, PPR_MAX_R);
        return PPR_EINVAL;
    }
    if ((a->dangling != 0 && a->dangling != 1) || (a->segments != 0 && a->segments != 1) ||
        (a->kernel != PPR_KERNEL_PERSISTENT && a->kernel != PPR_KERNEL_PLAIN) || a->large_degree < 0 ||
        a->warps_per_block < 0 || a->warps_per_block > 32 || a->chunk_sources < 0 || a->max_batch_sources < 0 ||
        (a->stats != 0 && a->stats != 1) || (a->sampler != 0 && a->sampler != 1) ||
        (a->l2_persist != 0 && a->l2_persist != 1) || a->refill_lanes < 0 || a->refill_lanes > 32 ||
        a->step_loads < -1 || a->step_loads == 1 || a->step_loads > 16) {
        set_error("invalid mode or tuning argument");
        return PPR_EINVAL;
    }
    if (a->sampler == 1 && a->segments) {
        set_error("segment tables run with the prefix sampler only");
        return PPR_ENOTSUP;
    }
    if (g->instances > 0 && a->tag != 0) {
        set_error("batched graphs use the instance id as tag; tag must be 0");
        return PPR_EINVAL;
    }
    if (g->instances > 0 && list) {
        set_error("source lists are supported on plain graphs");
        return PPR_ENOTSUP;
    }
    if (a->chunk_sources > 0 && (uint64_t)a->chunk_sources * a->R > (1u << 20)) {
        set_error("chunk_sources * R too large");
        return PPR_ERANGE;
    }
    *plan = RunPlan{};
    plan->T = T;
    plan->R = a->R;
    plan->seed = a->seed;
    plan->tag = a->tag;
    plan->dangling = a->dangling;
    plan->segments = a->segments != 0;
    plan->kernel = a->kernel;
    plan->large_degree = a->large_degree;
    plan->warps_per_block = a->warps_per_block;
    plan->chunk_sources = a->chunk_sources;
    plan->refill_lanes = a->refill_lanes;
    plan->stats = a->stats != 0;
    plan->sampler = a->sampler;
    plan->l2_persist = a->l2_persist == 1;
    plan->step_loads = a->step_loads == 0 ? kDefaultStepLoads : (a->step_loads < 0 ? 0 : a->step_loads);
    return PPR_OK;
}
}  // namespace ppr

extern "C" {

// Device tables a run needs beyond the base layout (built once per graph).
static int prepare_tables(const ppr_graph *g, const RunPlan &plan, cudaStream_t st)
{
    int rc = PPR_OK;
    if (plan.segments) rc = build_segments(const_cast<ppr_graph *>(g), plan.T, st);
    if (!rc && plan.sampler == 1) rc = build_alias(const_cast<ppr_graph *>(g), st);
    return rc;
}

static uint32_t row_capacity(const ppr_graph *g, uint32_t R)
{
    int64_t n_local_max = g->n;
    if (g->instances > 0) {
        n_local_max = 0;
        for (int32_t i = 0; i < g->instances; ++i)
            n_local_max = std::max<int64_t>(n_local_max, g->node_off[i + 1] - g->node_off[i]);
    }
    return (uint32_t)std::min<int64_t>((int64_t)R, n_local_max);
}

// ppr_run / ppr_run_list: result-owned outputs, batches sized to memory.
static int run_common(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *a, const int32_t *list, int64_t count,
                      ppr_result **out)
{
    RunPlan plan;
    int rc = check_run(g, a, count, list != nullptr, &plan);
    if (rc) return rc;
    Range range(list ? "ppr_run_list" : "ppr_run");
    if (list) {
        for (int64_t i = 0; i < count; ++i)
            if (list[i] < 0 || list[i] >= g->n) {
                set_error("source %lld of the list (%d) is outside [0, %lld)", (long long)i, list[i], (long long)g->n);
                return PPR_EINVAL;
            }
    }
    rc = set_device(ctx);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)a->stream;
    if ((rc = prepare_tables(g, plan, st))) return rc;
    ppr_result *r = new (std::nothrow) ppr_result;
    if (!r) return PPR_ENOMEM;
    r->ctx = ctx;
    ctx_retain(ctx);
    r->g = g;
    r->stream = st;
    r->S = list ? count : a->src_end - a->src_begin;
    r->R = a->R;
    r->topk = a->topk;
    r->src_begin = list ? 0 : a->src_begin;
    r->cap = row_capacity(g, a->R);
    auto fail = [&](int code) {
        result_release(r);
        return code;
    };
    const size_t S = (size_t)r->S;
    if ((rc = dev_alloc((void **)&r->d_nnz, sizeof(uint32_t) * S, "row sizes", st))) return fail(rc);
    if ((rc = dev_alloc((void **)&r->d_cols, sizeof(int32_t) * S * r->cap, "row ids", st))) return fail(rc);
    if ((rc = dev_alloc((void **)&r->d_cnts, sizeof(uint32_t) * S * r->cap, "row counts", st))) return fail(rc);
    if (r->topk > 0) {
        if ((rc = dev_alloc((void **)&r->d_topk_idx, sizeof(int32_t) * S * r->topk, "top-k ids", st))) return fail(rc);
        if ((rc = dev_alloc((void **)&r->d_topk_cnt, sizeof(uint32_t) * S * r->topk, "top-k counts", st))) return fail(rc);
    }
    if ((rc = dev_alloc((void **)&r->d_steps, sizeof(unsigned long long) * 8, "counters", st))) return fail(rc);
    uint32_t *d_list = nullptr;
    if (list) {
        if ((rc = dev_alloc((void **)&d_list, sizeof(uint32_t) * S, "source list", st))) return fail(rc);
        r->scratch.push_back(d_list);
        cudaError_t e = cudaMemcpyAsync(d_list, list, sizeof(uint32_t) * S, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(cuda_fail(e, "source list upload"));
    }
    cudaError_t e = cudaEventCreate(&r->ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev_walk_end);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev_done);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaEventCreate"));

    // Batch size (the paper's per-pipeline walk budget, gamma <= alpha*M/(n*c),
    // Sec. 4.3, becomes a source batch sized to device memory): every walk of
    // a batch keeps its 4-byte endpoint in HBM until the batch is aggregated;
    // that scratch is bounded to a quarter of the free memory.
    int64_t batch = r->S;
    if (a->max_batch_sources > 0) batch = std::min<int64_t>(batch, a->max_batch_sources);
    {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        int64_t fit = (int64_t)(free_b / 4 / ((size_t)a->R * sizeof(uint32_t)));
        batch = std::max<int64_t>(1, std::min<int64_t>(batch, fit));
    }
    unsigned char *ws = nullptr;
    if ((rc = dev_alloc((void **)&ws, launch_workspace_bytes(g, plan, batch), "walk workspace", st))) return fail(rc);
    r->scratch.push_back(ws);
    if ((e = cudaMemsetAsync(r->d_steps, 0, sizeof(unsigned long long) * 8, st)) != cudaSuccess)
        return fail(cuda_fail(e, "memset"));
    if ((e = cudaEventRecord(r->ev_start, st)) != cudaSuccess) return fail(cuda_fail(e, "cudaEventRecord"));
    const Outputs o{r->d_nnz, r->d_cols, r->d_cnts, r->cap, r->d_topk_idx, r->d_topk_cnt, r->topk, r->d_steps};
    for (int64_t b = 0; b < r->S; b += batch) {
        const int64_t nb = std::min<int64_t>(r->S - b, batch);
        rc = launch_walks(ctx, g, plan, o, r->src_begin + b, nb, d_list ? d_list + b : nullptr, b, ws, st, r,
                          b > 0);
        if (rc) {
            cudaStreamSynchronize(st);
            return fail(rc);
        }
    }
    if ((e = cudaEventRecord(r->ev_walk_end, st)) != cudaSuccess) return fail(cuda_fail(e, "cudaEventRecord"));
    if ((e = cudaEventRecord(r->ev_done, st)) != cudaSuccess) return fail(cuda_fail(e, "cudaEventRecord"));
    *out = r;
    return PPR_OK;
}

int ppr_run(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *a, ppr_result **out)
{
    if (!ctx || !g || !a || !out) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    *out = nullptr;
    return run_common(ctx, g, a, nullptr, 0, out);
}

int ppr_run_list(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *a, const int32_t *sources, int64_t count,
                 ppr_result **out)
{
    if (!ctx || !g || !a || !out || !sources) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    *out = nullptr;
    return run_common(ctx, g, a, sources, count, out);
}

int ppr_run_to_host(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *a, int32_t parts, int64_t *row_ptr,
                    int32_t *col, uint32_t *cnt, int64_t cap, int64_t *nnz, int32_t *topk_idx, uint32_t *topk_cnt,
                    ppr_result_info *info)
{
    if (!ctx || !g || !a || !row_ptr || !col || !cnt || parts < 0) {
        set_error("NULL argument or parts < 0");
        return PPR_EINVAL;
    }
    if (a->topk > 0 && (!topk_idx || !topk_cnt)) {
        set_error("topk > 0 needs topk_idx and topk_cnt");
        return PPR_EINVAL;
    }
    RunPlan plan;
    int rc = check_run(g, a, 0, false, &plan);
    if (rc) return rc;
    if ((rc = set_device(ctx))) return rc;
    Range range("ppr_run_to_host");
    cudaStream_t st = (cudaStream_t)a->stream;
    if ((rc = prepare_tables(g, plan, st))) return rc;
    cudaError_t e = cudaSuccess;
    if (!ctx->copy_stream && (e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "copy stream");
    if (!ctx->pinned && (e = cudaHostAlloc((void **)&ctx->pinned, 4 * sizeof(unsigned long long), 0)) != cudaSuccess)
        return cuda_fail(e, "page-locked words");
    cudaStream_t cs = ctx->copy_stream;
    const int64_t S = a->src_end - a->src_begin;
    const uint32_t rcap = row_capacity(g, a->R);
    const int32_t k = a->topk;
    int64_t P = parts > 0 ? parts : std::min<int64_t>(8, std::max<int64_t>(1, (S + 131071) / 131072));
    P = std::min<int64_t>(P, S);
    int64_t B = (S + P - 1) / P;
    {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        // endpoints, two slots of rows (stored and compacted) and top-k per source
        const size_t per = (size_t)a->R * 4 + 2 * ((size_t)rcap * 16 + (size_t)k * 8 + 16);
        const int64_t fit = (int64_t)(free_b / 2 / per);
        B = std::max<int64_t>(1, std::min<int64_t>(B, fit));
    }
    P = (S + B - 1) / B;
    // batch starts: B sources each, and the last batch split into three
    // quarters and one, so the copies left after the last walk are short
    std::vector<int64_t> start;
    for (int64_t b = 0; b < S; b += B) start.push_back(b);
    if (P >= 2 && S - start.back() >= 4) start.push_back(S - (S - start.back()) / 4);
    start.push_back(S);
    P = (int64_t)start.size() - 1;
    const int64_t tiles = (B + kScanTile - 1) / kScanTile;
    struct Slot {
        uint32_t *nnz = nullptr;
        int32_t *cols = nullptr, *ccol = nullptr, *ti = nullptr;
        uint32_t *cnts = nullptr, *ccnt = nullptr, *tc = nullptr;
        uint64_t *off = nullptr, *tmp = nullptr;
        cudaEvent_t ready = nullptr, copied = nullptr;
    } slot[2];
    ppr_result *r = new (std::nothrow) ppr_result;  // owns the walker events and counters
    if (!r) return PPR_ENOMEM;
    r->ctx = ctx;
    ctx_retain(ctx);
    r->stream = st;
    unsigned char *ws = nullptr;
    auto finish = [&](int code) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(st);
        for (Slot &q : slot) {
            dev_free(q.nnz, st);
            dev_free(q.cols, st);
            dev_free(q.cnts, st);
            dev_free(q.ccol, st);
            dev_free(q.ccnt, st);
            dev_free(q.ti, st);
            dev_free(q.tc, st);
            dev_free(q.off, st);
            dev_free(q.tmp, st);
            if (q.ready) cudaEventDestroy(q.ready);
            if (q.copied) cudaEventDestroy(q.copied);
        }
        dev_free(ws, st);
        result_release(r);
        return code;
    };
    for (Slot &q : slot) {
        const size_t rows = (size_t)B * rcap;
        if ((rc = dev_alloc((void **)&q.nnz, sizeof(uint32_t) * B, "row sizes", st)) ||
            (rc = dev_alloc((void **)&q.cols, sizeof(int32_t) * rows, "row ids", st)) ||
            (rc = dev_alloc((void **)&q.cnts, sizeof(uint32_t) * rows, "row counts", st)) ||
            (rc = dev_alloc((void **)&q.ccol, sizeof(int32_t) * (rows + 1), "compacted ids", st)) ||
            (rc = dev_alloc((void **)&q.ccnt, sizeof(uint32_t) * (rows + 1), "compacted counts", st)) ||
            (rc = dev_alloc((void **)&q.off, sizeof(uint64_t) * (B + 1), "row offsets", st)) ||
            (rc = dev_alloc((void **)&q.tmp, sizeof(uint64_t) * (tiles + 2), "scan scratch", st)))
            return finish(rc);
        if (k > 0 && ((rc = dev_alloc((void **)&q.ti, sizeof(int32_t) * B * k, "top-k ids", st)) ||
                      (rc = dev_alloc((void **)&q.tc, sizeof(uint32_t) * B * k, "top-k counts", st))))
            return finish(rc);
        if ((e = cudaEventCreateWithFlags(&q.ready, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&q.copied, cudaEventDisableTiming)) != cudaSuccess)
            return finish(cuda_fail(e, "cudaEventCreate"));
    }
    // counters: [0..4] as ppr_run's, [7] the running row base of the batches so far
    if ((rc = dev_alloc((void **)&r->d_steps, sizeof(unsigned long long) * 8, "counters", st))) return finish(rc);
    if ((rc = dev_alloc((void **)&ws, launch_workspace_bytes(g, plan, B), "walk workspace", st))) return finish(rc);
    if ((e = cudaMemsetAsync(r->d_steps, 0, sizeof(unsigned long long) * 8, st)) != cudaSuccess)
        return finish(cuda_fail(e, "memset"));
    unsigned long long *d_base = r->d_steps + 7;
    const int cblocks = (int)std::min<int64_t>((B + 7) / 8, (int64_t)ctx->sms * 32);
    uint64_t base = 0;
    for (int64_t i = 0; i <= P; ++i) {
        if (i < P) {  // batch i: walk, reduce, compact on the run's stream
            Range batch_range("batch");
            Slot &q = slot[i & 1];
            const int64_t b0 = start[i], nb = start[i + 1] - b0;
            if (i >= 2 && (e = cudaStreamWaitEvent(st, q.copied, 0)) != cudaSuccess)
                return finish(cuda_fail(e, "cudaStreamWaitEvent"));
            const Outputs o{q.nnz, q.cols, q.cnts, rcap, q.ti, q.tc, k, r->d_steps};
            if ((rc = launch_walks(ctx, g, plan, o, a->src_begin + b0, nb, nullptr, 0, ws, st, r, i > 0)))
                return finish(rc);
            exclusive_scan_u32(q.nnz, nb, q.off, q.tmp, st);
            k_compact_rows<<<std::max(1, cblocks), 256, 0, st>>>(nb, rcap, q.nnz, q.off, q.cols, q.cnts, q.ccol, q.ccnt);
            note_launch();
            // row starts made absolute here, so the copy stream runs copies only:
            // a kernel there would wait for SMs behind the next batch's walker
            k_add_base<<<(int)std::min<int64_t>((nb + 256) / 256, (int64_t)ctx->sms * 8), 256, 0, st>>>(nb + 1, q.off,
                                                                                                      d_base);
            note_launch();
            k_next_base<<<1, 1, 0, st>>>(d_base, q.off + nb);
            note_launch();
            if ((e = cudaMemcpyAsync(&ctx->pinned[i & 1], q.off + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaEventRecord(q.ready, st)) != cudaSuccess)
                return finish(cuda_fail(e, "batch"));
        }
        if (i >= 1) {  // batch i - 1: its copies on the copy stream, overlapping batch i
            const int64_t j = i - 1;
            Slot &q = slot[j & 1];
            const int64_t b0 = start[j], nb = start[j + 1] - b0;
            if ((e = cudaEventSynchronize(q.ready)) != cudaSuccess) return finish(cuda_fail(e, "batch"));
            const uint64_t tot = ctx->pinned[j & 1] - base;  // the batch's last absolute row start, less the base
            if ((uint64_t)cap < base + tot) {
                set_error("capacity %lld < nnz (at least %llu)", (long long)cap, (unsigned long long)(base + tot));
                return finish(PPR_ERANGE);
            }
            const int64_t nrp = nb + (j == P - 1 ? 1 : 0);  // the last batch also writes row_ptr[S]
            e = cudaMemcpyAsync(row_ptr + b0, q.off, sizeof(int64_t) * nrp, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess && tot > 0)
                e = cudaMemcpyAsync(col + base, q.ccol, sizeof(int32_t) * tot, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess && tot > 0)
                e = cudaMemcpyAsync(cnt + base, q.ccnt, sizeof(uint32_t) * tot, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess && k > 0)
                e = cudaMemcpyAsync(topk_idx + b0 * k, q.ti, sizeof(int32_t) * nb * k, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess && k > 0)
                e = cudaMemcpyAsync(topk_cnt + b0 * k, q.tc, sizeof(uint32_t) * nb * k, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaEventRecord(q.copied, cs);
            if (e != cudaSuccess) return finish(cuda_fail(e, "output copies"));
            base += tot;
        }
    }
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return finish(cuda_fail(e, "run"));
    if (nnz) *nnz = (int64_t)base;
    unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
    if ((e = cudaMemcpy(c, r->d_steps, sizeof(c), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return finish(cuda_fail(e, "counters"));
    if (c[4]) {  // only a checked build sets it
        set_error("checked build: an index left its array (flags 0x%llx)", c[4]);
        return finish(PPR_ECUDA);
    }
    if (info) {
        float kms = 0.f, ms = 0.f;
        for (size_t t = 0; t + 1 < r->walk_events.size(); t += 2) {
            if (cudaEventElapsedTime(&ms, r->walk_events[t], r->walk_events[t + 1]) == cudaSuccess) kms += ms;
        }
        info->sources = S;
        info->R = a->R;
        info->topk = k;
        info->nnz = (int64_t)base;
        info->steps = c[0];
        info->walks = (uint64_t)S * a->R;
        info->kernel_ms = kms;
        info->sectors = c[2];
        info->run_ms = 0.f;
        info->model_sectors = c[5];
    }
    return finish(PPR_OK);
}

int ppr_workspace_size(const ppr_graph *g, const ppr_run_args *a, size_t *bytes)
{
    if (!g || !a || !bytes) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    RunPlan plan;
    int rc = check_run(g, a, 0, false, &plan);
    if (rc) return rc;
    *bytes = 256 + launch_workspace_bytes(g, plan, a->src_end - a->src_begin);
    return PPR_OK;
}

int ppr_run_into(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *a, void *workspace, size_t bytes,
                 uint32_t *nnz, int32_t *cols, uint32_t *cnts, uint32_t cap, int32_t *topk_idx, uint32_t *topk_cnt)
{
    if (!ctx || !g || !a || !workspace || !nnz || !cols || !cnts) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    RunPlan plan;
    int rc = check_run(g, a, 0, false, &plan);
    if (rc) return rc;
    if (a->kernel != PPR_KERNEL_PERSISTENT || a->stats) {
        set_error("ppr_run_into runs the persistent kernel without statistics");
        return PPR_EINVAL;
    }
    if (a->topk > 0 && (!topk_idx || !topk_cnt)) {
        set_error("top-k outputs missing");
        return PPR_EINVAL;
    }
    if (a->segments && !(g->seg.T == plan.T && g->seg.node)) {
        set_error("segment tables for this alpha are not built (a ppr_run with segments=1 builds them)");
        return PPR_ENOTSUP;
    }
    if (a->sampler == 1 && !g->alias.node) {
        set_error("alias tables are not built (a ppr_run with sampler=1 builds them)");
        return PPR_ENOTSUP;
    }
    if (cap < row_capacity(g, a->R)) {
        set_error("row capacity %u < min(R, n) = %u", cap, row_capacity(g, a->R));
        return PPR_EINVAL;
    }
    const int64_t S = a->src_end - a->src_begin;
    const size_t need = 256 + launch_workspace_bytes(g, plan, S);
    if (bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_error("workspace of %zu bytes at %p: need %zu bytes, 256-byte aligned", bytes, workspace, need);
        return PPR_EINVAL;
    }
    if ((rc = set_device(ctx))) return rc;
    cudaStream_t st = (cudaStream_t)a->stream;
    unsigned char *w = static_cast<unsigned char *>(workspace);
    cudaError_t e = cudaMemsetAsync(w, 0, 256, st);  // counters start at zero
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace counters)");
    const Outputs o{nnz, cols, cnts, cap, topk_idx, topk_cnt, a->topk, reinterpret_cast<unsigned long long *>(w)};
    return launch_walks(ctx, g, plan, o, a->src_begin, S, nullptr, 0, w + 256, st, nullptr);
}

// Times each candidate tuning on a sample of the run's sources (an evenly
// strided list) and keeps the fastest.  Results do not depend on the tuning.
int ppr_autotune(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *a, int64_t sample_sources, ppr_tuning *best)
{
    if (!ctx || !g || !a || !best) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    RunPlan plan;
    int rc = check_run(g, a, 0, false, &plan);
    if (rc) return rc;
    if ((rc = set_device(ctx))) return rc;
    cudaStream_t st = (cudaStream_t)a->stream;
    if ((rc = prepare_tables(g, plan, st))) return rc;
    const int64_t S_all = a->src_end - a->src_begin;
    const int64_t S = std::max<int64_t>(1, std::min<int64_t>(S_all, sample_sources > 0 ? sample_sources : 65536));
    // batched graphs keep their instance structure: tune on a contiguous range
    // (chunks follow instances); plain graphs on an evenly strided list
    const bool use_list = g->instances == 0;
    std::vector<uint32_t> list;
    if (use_list) {
        list.resize((size_t)S);
        for (int64_t i = 0; i < S; ++i) list[(size_t)i] = (uint32_t)(a->src_begin + i * S_all / S);
    }
    const uint32_t cap = row_capacity(g, a->R);
    const int32_t topk = a->topk;
    unsigned char *buf = nullptr;
    const size_t ws_bytes = launch_workspace_bytes(g, plan, S);
    const size_t out_bytes = (size_t)S * (4 + 8ull * cap + 8ull * topk) + 256 + sizeof(uint32_t) * S + 1024;
    if ((rc = dev_alloc((void **)&buf, ws_bytes + out_bytes + 256, "autotune buffers", st))) return rc;
    unsigned char *p = buf;
    auto take = [&](size_t n) {
        unsigned char *q = p;
        p += (n + 255) & ~(size_t)255;
        return q;
    };
    unsigned char *ws = take(ws_bytes);
    Outputs o;
    o.counters = reinterpret_cast<unsigned long long *>(take(256));
    o.nnz = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S));
    o.cols = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * S * cap));
    o.cnts = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S * cap));
    o.topk_idx = topk ? reinterpret_cast<int32_t *>(take(sizeof(int32_t) * S * topk)) : nullptr;
    o.topk_cnt = topk ? reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S * topk)) : nullptr;
    o.cap = cap;
    o.topk = topk;
    uint32_t *d_list = use_list ? reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S)) : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && use_list)
        e = cudaMemcpyAsync(d_list, list.data(), sizeof(uint32_t) * S, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        dev_free(buf, st);
        return cuda_fail(e, "autotune setup");
    }
    const int cs_base = std::max(1, (int)(400 / a->R));
    const int cs_cands[] = {std::max(1, cs_base / 4), std::max(1, cs_base / 2), cs_base, cs_base * 2, cs_base * 4};
    const int lg_cands[] = {0, 4096, 65536};
    const int wpb_cands[] = {8, 4};
    ppr_tuning bt{};
    bt.ms = -1.f;
    int tried = 0;
    for (int wpb : wpb_cands)
        for (int lg : lg_cands)
            for (int cs : cs_cands) {
                if ((uint64_t)cs * a->R > (1u << 20)) continue;
                RunPlan pl = plan;
                pl.kernel = PPR_KERNEL_PERSISTENT;
                pl.stats = false;
                pl.chunk_sources = cs;
                pl.large_degree = lg;
                pl.warps_per_block = wpb;
                if (launch_workspace_bytes(g, pl, S) > ws_bytes) continue;
                float ms_best = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaMemsetAsync(o.counters, 0, 256, st);
                    cudaEventRecord(e0, st);
                    rc = launch_walks(ctx, g, pl, o, use_list ? 0 : a->src_begin, S, d_list, 0, ws, st, nullptr);
                    cudaEventRecord(e1, st);
                    if (rc) break;
                    e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) {
                        rc = cuda_fail(e, "autotune run");
                        break;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_best = std::min(ms_best, ms);
                }
                if (rc) break;
                ++tried;
                if (bt.ms < 0 || ms_best < bt.ms) {
                    bt.chunk_sources = cs;
                    bt.large_degree = lg;
                    bt.warps_per_block = wpb;
                    bt.refill_lanes = plan.refill_lanes > 0 ? plan.refill_lanes : 1;
                    bt.ms = ms_best;
                }
            }
    // refill thresholds with the fastest launch shape
    const int rf_cands[] = {8, 16, 24, 32};
    for (int rf : rf_cands) {
        if (rc || bt.ms < 0) break;
        RunPlan pl = plan;
        pl.kernel = PPR_KERNEL_PERSISTENT;
        pl.stats = false;
        pl.chunk_sources = bt.chunk_sources;
        pl.large_degree = bt.large_degree;
        pl.warps_per_block = bt.warps_per_block;
        pl.refill_lanes = rf;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaMemsetAsync(o.counters, 0, 256, st);
            cudaEventRecord(e0, st);
            rc = launch_walks(ctx, g, pl, o, use_list ? 0 : a->src_begin, S, d_list, 0, ws, st, nullptr);
            cudaEventRecord(e1, st);
            if (rc) break;
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune run");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_best = std::min(ms_best, ms);
        }
        if (rc) break;
        ++tried;
        if (ms_best < bt.ms) {
            bt.refill_lanes = rf;
            bt.ms = ms_best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    dev_free(buf, st);
    if (rc) return rc;
    bt.candidates = tried;
    bt.sample_sources = S;
    *best = bt;
    return PPR_OK;
}

int ppr_wait(ppr_result *r, int64_t timeout_ms)
{
    if (!r) {
        set_error("NULL result");
        return PPR_EINVAL;
    }
    int rc = set_device(r->ctx);
    if (rc) return rc;
    if (r->waited) return PPR_OK;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(r->ev_done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "run");
        if (timeout_ms >= 0) {
            auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) {
                set_error("run not finished after %lld ms", (long long)timeout_ms);
                return PPR_ETIMEOUT;
            }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    unsigned long long cnt[6] = {0, 0, 0, 0, 0, 0};
    PPR_CUDA(cudaMemcpy(cnt, r->d_steps, sizeof(cnt), cudaMemcpyDeviceToHost));
    r->steps = cnt[0];
    r->sectors = cnt[2];
    r->model_sectors = cnt[5];
    if (cnt[4]) {  // only a checked build sets it
        set_error("checked build: an index left its array (flags 0x%llx: 1 node, 2 edge row, 4 segment table, "
                  "8 endpoint)", cnt[4]);
        return PPR_ECUDA;
    }
    float ms = 0.f;
    PPR_CUDA(cudaEventElapsedTime(&ms, r->ev_start, r->ev_walk_end));
    r->run_ms = ms;
    float kms = 0.f;
    for (size_t i = 0; i + 1 < r->walk_events.size(); i += 2) {
        PPR_CUDA(cudaEventElapsedTime(&ms, r->walk_events[i], r->walk_events[i + 1]));
        kms += ms;
    }
    r->kernel_ms = kms;
    r->waited = true;
    return PPR_OK;
}

static int need_done(const ppr_result *r)
{
    if (!r) {
        set_error("NULL result");
        return PPR_EINVAL;
    }
    if (!r->waited) {
        set_error("result not ready: call ppr_wait first");
        return PPR_EBUSY;
    }
    return set_device(r->ctx);
}

int ppr_result_get_info(const ppr_result *r, ppr_result_info *info)
{
    if (!r || !info) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    info->sources = r->S;
    info->R = r->R;
    info->topk = r->topk;
    info->nnz = r->nnz_total;
    info->steps = r->steps;
    info->walks = (uint64_t)r->S * r->R;
    info->kernel_ms = r->kernel_ms;
    info->run_ms = r->run_ms;
    info->sectors = r->sectors;
    info->model_sectors = r->model_sectors;
    return PPR_OK;
}

int ppr_sparse_rows(const ppr_result *rc_, int64_t *row_ptr, int32_t *col, uint32_t *cnt, int64_t cap, int64_t *nnz,
                    uint32_t flags)
{
    int rc = need_done(rc_);
    if (rc) return rc;
    Range range("ppr_sparse_rows");
    ppr_result *r = const_cast<ppr_result *>(rc_);
    const bool dev_out = (flags & PPR_PTRS_DEVICE) != 0;
    cudaStream_t st = r->stream;
    const int64_t S = r->S;
    int64_t tiles = (S + kScanTile - 1) / kScanTile;
    uint64_t *d_off = nullptr, *d_tmp = nullptr;
    if ((rc = dev_alloc((void **)&d_off, sizeof(uint64_t) * (S + 1), "row offsets", st))) return rc;
    if ((rc = dev_alloc((void **)&d_tmp, sizeof(uint64_t) * (tiles + 2), "scan scratch", st)))
        return dev_free(d_off, st), rc;
    int32_t *d_col = nullptr;
    uint32_t *d_cnt = nullptr;
    auto done = [&](int code) {
        dev_free(d_off, st);
        dev_free(d_tmp, st);
        if (!dev_out) {
            dev_free(d_col, st);
            dev_free(d_cnt, st);
        }
        return code;
    };
    exclusive_scan_u32(r->d_nnz, S, d_off, d_tmp, st);
    uint64_t total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, d_off + S, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "row scan"));
    r->nnz_total = (int64_t)total;
    if (nnz) *nnz = (int64_t)total;
    if (row_ptr) {
        e = cudaMemcpyAsync(row_ptr, d_off, sizeof(int64_t) * (S + 1),
                            dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return done(cuda_fail(e, "row_ptr copy"));
    }
    if (col || cnt) {
        if (!col || !cnt) {
            set_error("col and cnt must both be given");
            return done(PPR_EINVAL);
        }
        if (cap < (int64_t)total) {
            set_error("capacity %lld < nnz %llu", (long long)cap, (unsigned long long)total);
            return done(PPR_ERANGE);
        }
        if (dev_out) {
            d_col = col;
            d_cnt = cnt;
        } else {
            if ((rc = dev_alloc((void **)&d_col, sizeof(int32_t) * (total + 1), "compacted ids", st))) return done(rc);
            if ((rc = dev_alloc((void **)&d_cnt, sizeof(uint32_t) * (total + 1), "compacted counts", st))) return done(rc);
        }
        int blocks = (int)std::min<int64_t>((S + 7) / 8, (int64_t)r->ctx->sms * 32);
        if (blocks < 1) blocks = 1;
        k_compact_rows<<<blocks, 256, 0, st>>>(S, r->cap, r->d_nnz, d_off, r->d_cols, r->d_cnts, d_col, d_cnt);
        note_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess && !dev_out && total > 0) {
            e = cudaMemcpyAsync(col, d_col, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, d_cnt, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost, st);
        }
        if (e != cudaSuccess) return done(cuda_fail(e, "row compaction"));
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "sparse rows"));
    return done(PPR_OK);
}

int ppr_topk(const ppr_result *r, int32_t k, int32_t *idx, uint32_t *cnt, uint32_t flags)
{
    int rc = need_done(r);
    if (rc) return rc;
    if (k < 1 || k > r->topk) {
        set_error("k = %d outside [1, %d] (the run's topk)", k, r->topk);
        return PPR_EINVAL;
    }
    if (!idx || !cnt) {
        set_error("idx and cnt must be non-NULL");
        return PPR_EINVAL;
    }
    cudaMemcpyKind kind = (flags & PPR_PTRS_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    PPR_CUDA(cudaMemcpy2DAsync(idx, sizeof(int32_t) * k, r->d_topk_idx, sizeof(int32_t) * r->topk, sizeof(int32_t) * k,
                               (size_t)r->S, kind, r->stream));
    PPR_CUDA(cudaMemcpy2DAsync(cnt, sizeof(uint32_t) * k, r->d_topk_cnt, sizeof(uint32_t) * r->topk,
                               sizeof(uint32_t) * k, (size_t)r->S, kind, r->stream));
    PPR_CUDA(cudaStreamSynchronize(r->stream));
    return PPR_OK;
}

int ppr_dense(const ppr_result *r, uint32_t *out, uint32_t flags)
{
    int rc = need_done(r);
    if (rc) return rc;
    if (!out) {
        set_error("out is NULL");
        return PPR_EINVAL;
    }
    if (r->g->instances > 0) {
        set_error("dense output is defined for plain graphs only");
        return PPR_ENOTSUP;
    }
    const int64_t n = r->g->n;
    const size_t bytes = sizeof(uint32_t) * (size_t)r->S * (size_t)n;
    const bool dev_out = (flags & PPR_PTRS_DEVICE) != 0;
    uint32_t *d = out;
    if (!dev_out && (rc = dev_alloc((void **)&d, bytes, "dense counts", r->stream))) return rc;
    cudaError_t e = cudaMemsetAsync(d, 0, bytes, r->stream);
    int blocks = (int)std::min<int64_t>((r->S + 7) / 8, (int64_t)r->ctx->sms * 32);
    if (blocks < 1) blocks = 1;
    if (e == cudaSuccess) {
        k_dense<<<blocks, 256, 0, r->stream>>>(r->S, n, r->cap, r->d_nnz, r->d_cols, r->d_cnts, d);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !dev_out) e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (!dev_out) dev_free(d, r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "dense");
    return PPR_OK;
}

void ppr_free_result(ppr_result *r) { result_release(r); }

}  // extern "C"
