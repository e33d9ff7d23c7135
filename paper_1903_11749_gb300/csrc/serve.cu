// serve.cu -- multi-source PPR queries served by continuous batching.
//
// A scheduler thread per context admits queries in arrival order whenever a
// stream slot is free and the query's device memory (per-walk endpoints, rows,
// top-k) fits the budget left by the queries in flight; each admitted query
// runs the persistent walker on its own stream, so queries that arrive while
// others run start as soon as slots and memory free up and their work shares
// the GPU.  A finished query's top-k is copied to pinned memory on its stream;
// ppr_poll hands it to the caller.  Every host wait has a deadline; nothing
// spins on the device.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ppr_host.h"

namespace ppr {

using clock_t_ = std::chrono::steady_clock;

static int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(clock_t_::now().time_since_epoch()).count();
}

struct Query {
    uint64_t id = 0;
    std::vector<uint32_t> sources;
    RunPlan plan{};
    int32_t topk = 0;
    size_t bytes = 0;  // device memory while in flight
    enum State { Pending, Running, Done, Failed } state = Pending;
    int status = PPR_OK;
    std::string error;
    std::vector<int32_t> idx;
    std::vector<uint32_t> cnt;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    uint64_t walks = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::shared_ptr<Query> q;
    unsigned char *dev = nullptr;  // device block of the running query
    unsigned char *pin = nullptr;  // pinned staging: sources in, top-k out
    size_t pin_bytes = 0;
};

struct Server {
    ppr_ctx *ctx = nullptr;
    const ppr_graph *g = nullptr;
    ppr_serve_cfg cfg{};
    size_t budget = 0, in_use = 0;
    std::vector<Slot> slots;
    std::deque<std::shared_ptr<Query>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Query>> table;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::atomic<bool> stop{false};
    std::thread worker;
    uint64_t next_id = 1;
    uint64_t completed = 0;
};

static size_t query_bytes(const ppr_graph *g, const RunPlan &plan, int64_t S, int32_t topk, uint32_t cap)
{
    size_t b = 0;
    auto add = [&](size_t n) { b += (n + 255) & ~(size_t)255; };
    add(256);                                    // counters
    add(sizeof(uint32_t) * S);                   // source list
    add(sizeof(uint32_t) * S);                   // nnz
    add(sizeof(int32_t) * S * cap);              // row ids
    add(sizeof(uint32_t) * S * cap);             // row counts
    add(sizeof(int32_t) * S * topk);             // top-k ids
    add(sizeof(uint32_t) * S * topk);            // top-k counts
    add(launch_workspace_bytes(g, plan, S));     // endpoints
    return b;
}

// Starts query q on slot s (scheduler thread, lock held by caller not needed for the slot).
static int start_query(Server *sv, Slot &s, const std::shared_ptr<Query> &q)
{
    const int64_t S = (int64_t)q->sources.size();
    const uint32_t cap = (uint32_t)std::min<int64_t>((int64_t)q->plan.R, sv->g->n);
    int rc = dev_alloc((void **)&s.dev, q->bytes, "query buffers", s.stream);
    if (rc) return rc;
    unsigned char *p = s.dev;
    auto take = [&](size_t n) {
        unsigned char *r = p;
        p += (n + 255) & ~(size_t)255;
        return r;
    };
    Outputs o;
    o.counters = reinterpret_cast<unsigned long long *>(take(256));
    uint32_t *list = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S));
    o.nnz = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S));
    o.cols = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * S * cap));
    o.cnts = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S * cap));
    o.topk_idx = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * S * q->topk));
    o.topk_cnt = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * S * q->topk));
    o.cap = cap;
    o.topk = q->topk;
    unsigned char *ws = take(launch_workspace_bytes(sv->g, q->plan, S));
    // sources through the slot's pinned staging buffer
    const size_t src_b = sizeof(uint32_t) * S, out_b = sizeof(int32_t) * S * q->topk;
    std::memcpy(s.pin, q->sources.data(), src_b);
    cudaError_t e = cudaMemsetAsync(o.counters, 0, 256, s.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(list, s.pin, src_b, cudaMemcpyHostToDevice, s.stream);
    if (e != cudaSuccess) return cuda_fail(e, "query upload");
    rc = launch_walks(sv->ctx, sv->g, q->plan, o, 0, S, list, 0, ws, s.stream, nullptr);
    if (rc) return rc;
    e = cudaMemcpyAsync(s.pin, o.topk_idx, out_b, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.pin + out_b, o.topk_cnt, out_b, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
    if (e != cudaSuccess) return cuda_fail(e, "query download");
    return PPR_OK;
}

static void finish_slot(Server *sv, Slot &s, int status)
{
    std::shared_ptr<Query> q = s.q;
    const int64_t S = (int64_t)q->sources.size();
    if (status == PPR_OK) {
        const size_t out_b = sizeof(int32_t) * S * q->topk;
        q->idx.resize((size_t)S * q->topk);
        q->cnt.resize((size_t)S * q->topk);
        std::memcpy(q->idx.data(), s.pin, out_b);
        std::memcpy(q->cnt.data(), s.pin + out_b, out_b);
    }
    dev_free(s.dev, s.stream);
    s.dev = nullptr;
    s.q.reset();
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->in_use -= q->bytes;
    q->t_done = now_ns();
    q->status = status;
    q->state = status == PPR_OK ? Query::Done : Query::Failed;
    if (status != PPR_OK) q->error = ppr_last_error();
    ++sv->completed;
    sv->cv_done.notify_all();
}

static void scheduler(Server *sv)
{
    cudaSetDevice(sv->ctx->device);
    for (;;) {
        // retire finished queries
        bool busy = false;
        for (Slot &s : sv->slots) {
            if (!s.q) continue;
            cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaSuccess) finish_slot(sv, s, PPR_OK);
            else if (e != cudaErrorNotReady) finish_slot(sv, s, cuda_fail(e, "query"));
            else busy = true;
        }
        // admit in arrival order while a slot and the memory budget allow
        for (Slot &s : sv->slots) {
            if (s.q) continue;
            std::shared_ptr<Query> q;
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                if (sv->pending.empty()) break;
                std::shared_ptr<Query> f = sv->pending.front();
                if (sv->in_use + f->bytes > sv->budget && sv->in_use > 0) break;  // wait for memory
                sv->pending.pop_front();
                sv->in_use += f->bytes;
                f->state = Query::Running;
                f->t_admit = now_ns();
                q = f;
            }
            s.q = q;
            int rc = start_query(sv, s, q);
            if (rc) finish_slot(sv, s, rc);
            else busy = true;
        }
        std::unique_lock<std::mutex> lock(sv->mu);
        if (sv->stop && sv->pending.empty() && !busy) break;
        if (busy) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
            sv->cv_work.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace ppr

using namespace ppr;

extern "C" {

void ppr_serve_cfg_init(ppr_serve_cfg *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->streams = 4;
    c->max_sources = 100000;
}

int ppr_serve_start(ppr_ctx *ctx, const ppr_graph *g, const ppr_serve_cfg *cfg_in)
{
    if (!ctx || !g) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    if (ctx->server) {
        set_error("serving already started on this context");
        return PPR_EBUSY;
    }
    if (g->instances > 0) {
        set_error("serving runs on plain graphs");
        return PPR_ENOTSUP;
    }
    ppr_serve_cfg cfg;
    ppr_serve_cfg_init(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.streams < 1 || cfg.streams > 64 || cfg.max_sources < 1 || cfg.memory_budget < 0 || cfg.max_pending < 0 ||
        cfg.max_topk < 0 || cfg.max_topk > (int32_t)PPR_MAX_R || (cfg.sampler != 0 && cfg.sampler != 1) ||
        cfg.refill_lanes < 0 || cfg.refill_lanes > 32) {
        set_error("invalid serving configuration");
        return PPR_EINVAL;
    }
    if (cfg.max_topk == 0) cfg.max_topk = 64;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (cfg.sampler == 1) {
        const int rc = build_alias(const_cast<ppr_graph *>(g), g->stream);
        if (rc) return rc;
    }
    Server *sv = new (std::nothrow) Server;
    if (!sv) return PPR_ENOMEM;
    sv->ctx = ctx;
    sv->g = g;
    sv->cfg = cfg;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    sv->budget = cfg.memory_budget > 0 ? (size_t)cfg.memory_budget : free_b / 4;
    sv->slots.resize((size_t)cfg.streams);
    const size_t pin_b = std::max(sizeof(uint32_t) * (size_t)cfg.max_sources,
                                  2 * sizeof(int32_t) * (size_t)cfg.max_sources * (size_t)cfg.max_topk);
    for (Slot &s : sv->slots) {
        e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&s.pin, pin_b);
        if (e != cudaSuccess) {
            for (Slot &t : sv->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.done) cudaEventDestroy(t.done);
                if (t.pin) cudaFreeHost(t.pin);
            }
            delete sv;
            return cuda_fail(e, "serving set-up");
        }
        s.pin_bytes = pin_b;
    }
    sv->worker = std::thread(scheduler, sv);
    ctx->server = sv;
    return PPR_OK;
}

int ppr_serve_stop(ppr_ctx *ctx)
{
    if (!ctx || !ctx->server) {
        set_error("serving not started");
        return PPR_EINVAL;
    }
    Server *sv = ctx->server;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        // queries not yet admitted are cancelled; running ones finish
        for (auto &q : sv->pending) {
            q->state = Query::Failed;
            q->status = PPR_EINVAL;
            q->error = "cancelled: serving stopped";
        }
        sv->pending.clear();
        sv->stop = true;
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    sv->worker.join();
    for (Slot &s : sv->slots) {
        cudaStreamSynchronize(s.stream);
        cudaStreamDestroy(s.stream);
        cudaEventDestroy(s.done);
        cudaFreeHost(s.pin);
    }
    ctx->server = nullptr;
    delete sv;
    return PPR_OK;
}

int ppr_submit(ppr_ctx *ctx, const int32_t *srcs, int64_t ns, double alpha, uint32_t R, uint64_t seed, int32_t topk,
               uint64_t *qid)
{
    if (!ctx || !srcs || !qid) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    Server *sv = ctx->server;
    if (!sv) {
        set_error("serving not started");
        return PPR_EINVAL;
    }
    const uint32_t T = ppr_alpha_threshold(alpha);
    if (T == 0 || R < 1 || R > PPR_MAX_R || ns < 1 || ns > sv->cfg.max_sources || topk < 1 ||
        topk > sv->cfg.max_topk) {
        set_error("invalid query: alpha %g, R %u, %lld sources (max %lld), topk %d (max %d)", alpha, R, (long long)ns,
                  (long long)sv->cfg.max_sources, topk, sv->cfg.max_topk);
        return PPR_EINVAL;
    }
    auto q = std::make_shared<Query>();
    q->sources.resize((size_t)ns);
    for (int64_t i = 0; i < ns; ++i) {
        if (srcs[i] < 0 || srcs[i] >= sv->g->n) {
            set_error("query source %d outside [0, %lld)", srcs[i], (long long)sv->g->n);
            return PPR_EINVAL;
        }
        q->sources[(size_t)i] = (uint32_t)srcs[i];
    }
    q->plan.T = T;
    q->plan.R = R;
    q->plan.seed = seed;
    q->plan.tag = 0;
    q->plan.dangling = 0;
    q->plan.segments = false;
    q->plan.kernel = PPR_KERNEL_PERSISTENT;
    q->plan.large_degree = sv->cfg.large_degree;
    q->plan.warps_per_block = sv->cfg.warps_per_block;
    q->plan.refill_lanes = sv->cfg.refill_lanes;
    q->plan.chunk_sources = sv->cfg.chunk_sources;
    q->plan.sampler = sv->cfg.sampler;
    q->plan.stats = false;
    q->topk = topk;
    const uint32_t cap = (uint32_t)std::min<int64_t>((int64_t)R, sv->g->n);
    q->bytes = query_bytes(sv->g, q->plan, ns, topk, cap);
    q->walks = (uint64_t)ns * R;
    q->t_submit = now_ns();
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) {
        set_error("serving is stopping");
        return PPR_EBUSY;
    }
    if (q->bytes > sv->budget) {
        set_error("query needs %zu bytes of device memory; the serving budget is %zu", q->bytes, sv->budget);
        return PPR_ERANGE;
    }
    if (sv->cfg.max_pending > 0 && (int64_t)sv->pending.size() >= sv->cfg.max_pending) {
        set_error("%lld queries pending", (long long)sv->pending.size());
        return PPR_EBUSY;
    }
    q->id = sv->next_id++;
    sv->table[q->id] = q;
    sv->pending.push_back(q);
    *qid = q->id;
    sv->cv_work.notify_one();
    return PPR_OK;
}

int ppr_poll(ppr_ctx *ctx, uint64_t qid, int32_t *idx, uint32_t *cnt, int64_t timeout_ms, ppr_query_stats *stats)
{
    if (!ctx) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    Server *sv = ctx->server;
    if (!sv) {
        set_error("serving not started");
        return PPR_EINVAL;
    }
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->table.find(qid);
    if (it == sv->table.end()) {
        set_error("unknown query %llu", (unsigned long long)qid);
        return PPR_EINVAL;
    }
    std::shared_ptr<Query> q = it->second;
    auto ready = [&] { return q->state == Query::Done || q->state == Query::Failed; };
    if (timeout_ms < 0) sv->cv_done.wait(lock, ready);
    else if (!sv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) {
        set_error("query %llu not finished after %lld ms", (unsigned long long)qid, (long long)timeout_ms);
        return PPR_ETIMEOUT;
    }
    if (stats) {
        stats->submit_ns = q->t_submit;
        stats->admit_ns = q->t_admit;
        stats->done_ns = q->t_done;
        stats->walks = q->walks;
        stats->sources = (int64_t)q->sources.size();
    }
    if (q->state == Query::Failed) {
        set_error("%s", q->error.c_str());
        sv->table.erase(it);
        return q->status != PPR_OK ? q->status : PPR_ECUDA;
    }
    if (idx) std::memcpy(idx, q->idx.data(), sizeof(int32_t) * q->idx.size());
    if (cnt) std::memcpy(cnt, q->cnt.data(), sizeof(uint32_t) * q->cnt.size());
    sv->table.erase(it);
    return PPR_OK;
}

}  // extern "C"
