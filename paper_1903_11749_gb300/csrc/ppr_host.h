// ppr_host.h -- host-side objects behind the C ABI (not part of the ABI).
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/ppr.h"
#include "ppr_internal.cuh"

namespace ppr {

// Named range on the profiler timeline (NVTX) for the lifetime of the object.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

void set_error(const char *fmt, ...);
void note_launch();  // counts every kernel launch of the library (ppr_kernel_launches)
int cuda_fail(cudaError_t e, const char *what);

#define PPR_CUDA(call)                                                 \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::ppr::cuda_fail(e_, #call);     \
    } while (0)

// Stream-ordered device allocation (reports PPR_ENOMEM) and release.
int dev_alloc(void **p, size_t bytes, const char *what, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

struct AliasCache {
    AliasNode *node = nullptr; // node records pointing at alias slots
    AliasRec *slots = nullptr; // one per edge
};

struct SegCache {
    uint32_t T = 0;               // threshold the tables were built for (0 = none)
    void *node = nullptr;         // node records (the graph's type) with eligible nodes switched to their tables
    SegEntry *entries = nullptr;  // all tables
    int64_t nodes = 0, entries_n = 0;  // tables, and the entries they hold
    int64_t entries_cap = 0;           // entries allocated (tables sit at fixed slots, with gaps)
};

}  // namespace ppr

namespace ppr {
struct Server;
}

struct ppr_ctx {
    int device = 0;
    int sms = 0;
    size_t smem_optin = 0;
    ppr::Server *server = nullptr;  // serving state (ppr_serve_start)
    size_t l2_persist_max = 0;    // device limits for L2 access-policy windows
    size_t l2_window_max = 0;
    size_t l2_persist_set = 0;    // persisting set-aside this context asked for
    size_t l2_bytes = 0;          // L2 size (the layout's renumbering policy)
    cudaStream_t copy_stream = nullptr;  // output copies of ppr_run_to_host
    unsigned long long *pinned = nullptr;  // page-locked words for per-batch totals
    std::atomic<int> refs{1};  // the caller's handle plus every live graph and result
};

namespace ppr {
// A graph or result keeps its context alive: ppr_destroy only drops the
// caller's reference, so handles may be freed in any order.
void ctx_retain(ppr_ctx *ctx);
void ctx_release(ppr_ctx *ctx);
}  // namespace ppr

struct ppr_graph {
    ppr_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;  // stream the graph was built on
    int64_t n = 0, m = 0;
    int64_t max_degree = 0, dangling = 0;
    bool wide = false;
    void *node = nullptr;   // NodeRecN[n] (narrow layout) or NodeRec[n] (wide layout)
    void *edges = nullptr;  // EdgeN[m] or EdgeW[m]
    int64_t edge_records = 0;  // records the edge layout holds (blocked narrow rows: with padding)
    uint32_t *sum = nullptr;   // narrow layout: the blocked rows' summary levels (8 keys a sector), or
    int64_t sum_sectors = 0;   // null: each row's summary precedes its blocks in the edge array
    // where the walkers read summary sectors (the summary array or the edge array) and how many there are
    const uint32_t *sum_base() const { return sum ? sum : static_cast<const uint32_t *>(edges); }
    uint64_t sum_extent() const { return sum ? (uint64_t)sum_sectors : (uint64_t)edge_records / 4; }
    // internal numbering of the layout (renumber.cu), or null: caller ids
    int32_t *order = nullptr;  // [n] caller id of internal node i
    int32_t *rank = nullptr;   // [n] internal id of caller node v
    int64_t device_bytes_extra = 0;  // order and rank
    // block-diagonal instances
    int32_t instances = 0;
    std::vector<int64_t> node_off;  // host copy, count+1
    int64_t *d_node_off = nullptr;  // device copy
    ppr::SegCache seg;
    ppr::AliasCache alias;
    int64_t device_bytes = 0;
};

struct ppr_result {
    ppr_ctx *ctx = nullptr;
    const ppr_graph *g = nullptr;
    cudaStream_t stream = nullptr;
    int64_t S = 0;
    uint32_t R = 0;
    int32_t topk = 0;
    uint32_t cap = 0;
    int64_t src_begin = 0;
    uint32_t *d_nnz = nullptr;
    int32_t *d_cols = nullptr;
    uint32_t *d_cnts = nullptr;
    int32_t *d_topk_idx = nullptr;
    uint32_t *d_topk_cnt = nullptr;
    unsigned long long *d_steps = nullptr;  // counters: [0] steps, [1] work queue, [2] sectors, [3] chunks,
                                            // [4] checked-build flags, [5] flat-CSR model sectors
    cudaEvent_t ev_start = nullptr, ev_walk_end = nullptr, ev_done = nullptr;
    std::vector<cudaEvent_t> walk_events;  // (before, after) each walker launch
    bool waited = false;
    uint64_t steps = 0, sectors = 0, model_sectors = 0;
    float kernel_ms = 0.f;  // walker launches only
    float run_ms = 0.f;     // walkers, reductions and everything between
    int64_t nnz_total = -1;
    std::vector<void *> scratch;  // freed with the result
};

namespace ppr {

// graph.cu
int build_graph(ppr_ctx *ctx, int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                const uint32_t *w, bool device_ptrs, bool renumber, cudaStream_t st, ppr_graph *g);
// renumber.cu: order and rank of the in-degree numbering (see ppr_graph)
int renumber_by_indegree(ppr_ctx *ctx, int64_t n, int64_t m, const int32_t *d_col, cudaStream_t st, int32_t *order,
                         int32_t *rank, std::vector<void *> &tmp);
int build_segments(ppr_graph *g, uint32_t T, cudaStream_t st);
int build_alias(ppr_graph *g, cudaStream_t st);

// walk.cu
void preload_run_kernels();  // loads every kernel a run launches (once per device)
struct RunPlan {
    uint32_t T, R;
    uint64_t seed;
    uint32_t tag;
    int32_t dangling;
    bool segments;
    int32_t kernel;
    int32_t large_degree;
    int32_t warps_per_block;
    int32_t chunk_sources;
    int32_t refill_lanes;  // persistent kernel: idle lanes before a warp refills (0 = 1)
    bool stats;
    int32_t sampler;  // 0 first-prefix-above rule, 1 integer alias method
    bool l2_persist;  // walker launches keep the node records in L2 (access-policy window)
    int32_t step_loads;  // bounded step: dependent loads per lane per warp iteration (0 = unbounded)
};
constexpr int32_t kDefaultStepLoads = 6;
// Enqueues the walks of sources [s_begin, s_end) writing output rows from
// out_row0.  ends: S * R endpoint scratch for the plain kernel (else unused);
// queue: one device counter for the persistent kernel's work queue.
// Where a launch writes: rows (nnz / cols / cnts at row * cap), top-k, and
// the counters block: [0] steps, [1] work queue, [2] sectors, [3] chunk count.
struct Outputs {
    uint32_t *nnz;
    int32_t *cols;
    uint32_t *cnts;
    uint32_t cap;
    int32_t *topk_idx;
    uint32_t *topk_cnt;
    int32_t topk;
    unsigned long long *counters;
};

// Argument checks shared by every run entry point (api.cu); count = number of
// sources of an explicit list (list = true), else the range is checked.
// Fills *plan; returns a PPR_* status with the message set.
int check_run(const ppr_graph *g, const ppr_run_args *a, int64_t count, bool list, RunPlan *plan);

// Device workspace one launch of S sources needs (endpoints, chunk table).
size_t launch_workspace_bytes(const ppr_graph *g, const RunPlan &p, int64_t S);

// Enqueues walks and reduction for S sources: node s_begin + i, or
// src_list[i] (device) when given; rows go to out_row0 + i.  ws holds
// launch_workspace_bytes.  ev_owner: record walker-time events into it.
// The persistent walker's work queue (o.counters[1]) must be zero when the
// launch runs: callers zero the counters before their first launch and pass
// reset_queue for every later launch on the same counters.
int launch_walks(ppr_ctx *ctx, const ppr_graph *g, const RunPlan &p, const Outputs &o, int64_t s_begin, int64_t S,
                 const uint32_t *src_list, int64_t out_row0, unsigned char *ws, cudaStream_t st, ppr_result *ev_owner,
                 bool reset_queue = false);

}  // namespace ppr
