// walk.cu -- the batch walker kernels (one step of a walk: walk_step.cuh).
//
// k_walk_plain:      one thread per walk, endpoint to HBM (baseline).
// k_walk_persistent: persistent warps pull chunks of walks from a global
//                    queue and refill lanes as walks end (the paper's
//                    pipelines keep the cluster busy the same way); rows above
//                    a set degree may be searched by the whole warp.
// Both write one endpoint per walk to HBM; k_aggregate (aggregate.cuh) then
// turns each source's R endpoints into its count row and top-k.
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <mutex>

#include "ppr_host.h"
#include "scan.cuh"
#include "aggregate.cuh"
#include "walk_step.cuh"

namespace ppr {

__device__ __forceinline__ void warp_add(unsigned long long *dst, uint32_t v)
{
    unsigned long long s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, s);
}

template <bool STATS>
__device__ __forceinline__ void warp_add_tally(unsigned long long *dst, const Tally &t)
{
    warp_add(dst, t.steps);
    if (STATS) {
        warp_add(dst + 2, t.sectors);
        warp_add(dst + 5, t.model);
    }
}

// ------------------------------------------------------------ plain (K4) ----
#ifndef PPR_WALK_MINB
#define PPR_WALK_MINB 6  // resident 256-thread blocks per SM asked of ptxas (6: 40 registers, no spills)
#endif

template <class E, bool SEG, bool STATS, bool SPLIT = false>
__global__ void __launch_bounds__(256, PPR_WALK_MINB) k_walk_plain(KParams p)
{
    const E edges = make_edges<E>(p.edges);
    const uint64_t S = (uint64_t)(p.s_end - p.s_begin);
    const uint64_t total = S * p.R;
    Tally tl;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = t / p.R;
        const uint32_t j = (uint32_t)(t - i * p.R);
        const uint32_t src = p.src_list ? p.src_list[i] : (uint32_t)(p.s_begin + (int64_t)i);
        uint32_t ctr_base = 0, tag = p.tag;
        if (p.inst_off) {  // batched graph: the source's instance gives counter base and tag
            int32_t lo = 0, hi = p.instances;
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (p.inst_off[mid] <= (int64_t)src) lo = mid;
                else hi = mid;
            }
            ctr_base = (uint32_t)p.inst_off[lo];
            tag = (uint32_t)lo;
        }
        // the draw is keyed by the caller's source id; the walk starts (and
        // restarts) at its node of the layout
        const uint32_t s0 = p.rank ? (uint32_t)p.rank[src] : src;
        uint32_t k = 0, u = s0, end = 0;
        while (!walk_step<E, SEG, false, STATS, SPLIT>(p, StepKey{p.k0, p.k1, p.T}, edges, true, s0, src - ctr_base, j,
                                                        tag, k, u, end, tl)) {
        }
        p.ends[t] = end - ctr_base;
    }
    warp_add_tally<STATS>(p.steps, tl);
}

// ------------------------------------------------------- persistent (K5) ----
// Persistent warps.  Each warp pulls chunks of sources from a global queue
// (one atomic per chunk) and keeps all 32 lanes busy: a lane whose walk ends
// takes the next walk of the warp's chunk at once, so a warp never waits for
// the longest of 32 geometric walk lengths (the paper's pipelines keep the
// cluster busy the same way: new walks start while old ones finish).  Steps
// run in lockstep; a row longer than p.large can be searched by the whole
// warp (search_warp).  Endpoints go to the per-walk buffer, reduced per
// source by k_aggregate.  The walker uses no shared memory beyond the queue
// state, so L1 keeps its full size.
struct WarpQueue {
    uint32_t base, ctr_base, tag;  // current chunk: first position, counter base, tag
    uint32_t j0;                   // walk index (within source `base`) of the chunk's first walk
    uint32_t issued, total;
};

__device__ __forceinline__ uint32_t div_by_R(uint32_t w, uint64_t magic)
{
    return (uint32_t)(((uint64_t)w * magic) >> 40);  // exact for w < 2^20, R <= 4096
}

template <class E, bool SEG, bool STATS, bool BOUNDED = false, bool SPLIT = false>
__global__ void __launch_bounds__(256, PPR_WALK_MINB) k_walk_persistent(KParams p)
{
    __shared__ WarpQueue wq_all[8];
    __shared__ uint32_t ps_all[BOUNDED ? 8 * 256 : 1];  // bounded step: each lane's pending search
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpQueue &wq = wq_all[wid];
    const E edges = make_edges<E>(p.edges);
    if (lane == 0) {
        wq.issued = 0;
        wq.total = 0;
    }
    __syncwarp();
    bool queue_empty = false;
    bool active = false;
    uint32_t src = 0, sctr = 0, j = 0, k = 0, u = 0, tag = 0, ctr_base = 0;
    uint64_t slot = 0;  // endpoint index: (src - s_begin) * R + j
    bool pend = false;  // bounded step: this lane's draw has a search in progress
    Tally tl;

    for (;;) {
        uint32_t idle = __ballot_sync(0xffffffffu, !active);
        // refill once p.refill lanes are idle, then every idle lane
        if ((uint32_t)__popc(idle) < p.refill) idle = 0;
        while (idle && !queue_empty) {
            if (wq.issued == wq.total) {
                unsigned long long c = 0;
                if (lane == 0) c = atomicAdd(p.queue, 1ull);
                c = __shfl_sync(0xffffffffu, c, 0);
                const unsigned long long nch = p.nchunks_dev ? *p.nchunks_dev : p.nchunks;
                if (c >= nch) {
                    queue_empty = true;
                    break;
                }
                if (lane == 0) {
                    uint32_t nwalks;
                    if (p.chunks) {  // whole sources of one instance
                        const int4 d = p.chunks[c];
                        wq.base = (uint32_t)d.x;
                        wq.ctr_base = (uint32_t)p.inst_off[d.z];
                        wq.tag = (uint32_t)d.z;
                        wq.j0 = 0;
                        nwalks = (uint32_t)d.y * p.R;
                    } else {  // walks [c * CW, ...) of the whole launch
                        const uint64_t b = c * (uint64_t)p.CW;
                        const uint64_t i0 = b / p.R;
                        wq.base = (uint32_t)i0;
                        wq.j0 = (uint32_t)(b - i0 * p.R);
                        nwalks = (uint32_t)min((uint64_t)p.CW, p.walks - b);
                        wq.ctr_base = 0;
                        wq.tag = p.tag;
                    }
                    wq.issued = 0;
                    wq.total = nwalks;
                }
                __syncwarp();
            }
            const uint32_t issued = wq.issued;
            const uint32_t take = min(wq.total - issued, (uint32_t)__popc(idle));
            const uint32_t rank = __popc(idle & ((1u << lane) - 1));
            if (((idle >> lane) & 1) && rank < take) {
                const uint32_t w = wq.j0 + issued + rank;  // < 2^20: CW <= 2^19, j0 < R <= 4096
                const uint32_t i = div_by_R(w, p.r_magic);
                j = w - i * p.R;
                const uint32_t pos = wq.base + i;
                src = p.src_list ? p.src_list[pos] : (uint32_t)(p.s_begin + pos);
                ctr_base = wq.ctr_base;
                sctr = src - ctr_base;  // draws keyed by the caller's source id
                if (p.rank) src = (uint32_t)p.rank[src];  // start and restart node of the layout
                tag = wq.tag;
                slot = (uint64_t)pos * p.R + j;
                k = 0;
                u = src;
                active = true;
            }
            __syncwarp();
            if (lane == 0) wq.issued = issued + take;
            __syncwarp();
            idle = __ballot_sync(0xffffffffu, !active);
        }
        if (__ballot_sync(0xffffffffu, active) == 0) break;  // queue drained and every walk done

        uint32_t end = 0;
        bool ended;
        if constexpr (BOUNDED) {
            ended = active && walk_step_bounded<SEG, SPLIT>(p, StepKey{p.k0, p.k1, p.T}, edges, src, sctr, j, tag, k, u, end,
                                                     pend, PendRef{ps_all, blockDim.x, threadIdx.x}, tl);
        } else {
            ended = walk_step<E, SEG, true, STATS, SPLIT>(p, StepKey{p.k0, p.k1, p.T}, edges, active, src, sctr, j, tag, k, u,
                                                   end, tl);
        }
        if (ended) {
#ifdef PPR_CHECKED
            if (slot >= (uint64_t)(p.s_end - p.s_begin) * p.R) atomicOr(p.err, 8ull);
            else
#endif
            p.ends[slot] = end - ctr_base;
            active = false;
        }
    }
    warp_add_tally<STATS>(p.steps, tl);
}

// ------------------------------------------------------------- launcher ----

// Events around a walker launch, for the walker-only device time.
static int walker_event(ppr_result *r, cudaStream_t st)
{
    if (!r) return PPR_OK;  // allocation-free runs record no events
    cudaEvent_t ev;
    PPR_CUDA(cudaEventCreate(&ev));
    r->walk_events.push_back(ev);
    PPR_CUDA(cudaEventRecord(ev, st));
    return PPR_OK;
}

template <class E, bool SEG, bool STATS, bool BOUNDED = false, bool SPLIT = false>
static int launch_typed(ppr_ctx *ctx, const KParams &kp, const RunPlan &plan, int64_t S, cudaStream_t st,
                        ppr_result *r)
{
    int rc;
    if (plan.kernel == PPR_KERNEL_PLAIN) {
        uint64_t total = (uint64_t)S * kp.R;
        int blocks = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->sms * 64);
        if (blocks < 1) blocks = 1;
        if ((rc = walker_event(r, st))) return rc;
        k_walk_plain<E, SEG, STATS, SPLIT><<<blocks, 256, 0, st>>>(kp);
        note_launch();
        PPR_CUDA(cudaGetLastError());
        if ((rc = walker_event(r, st))) return rc;
        return launch_aggregate(ctx, AggParams{kp.ends, kp.R, kp.P2, S, kp.out_row0, kp.out, kp.order}, st);
    }
    // walkers per CTA: 32 * warps_per_block (4 or 8 warps; default 8)
    const int wpb = plan.warps_per_block == 4 ? 4 : 8;
    // resident blocks per SM: fixed for this kernel, device and block size,
    // so queried once (a host call per run shows in short runs)
    static std::atomic<int> occupancy[64][2];
    std::atomic<int> *occ = ctx->device >= 0 && ctx->device < 64 ? &occupancy[ctx->device][wpb == 8] : nullptr;
    int per_sm = occ ? occ->load(std::memory_order_relaxed) : 0;
    if (per_sm < 1) {
        PPR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_walk_persistent<E, SEG, STATS, BOUNDED, SPLIT>, 32 * wpb, 0));
        if (per_sm < 1) per_sm = 1;
        if (occ) occ->store(per_sm, std::memory_order_relaxed);
    }
    int64_t blocks = (int64_t)ctx->sms * per_sm;
    int64_t needed = ((int64_t)kp.nchunks + wpb - 1) / wpb;
    if (blocks > needed) blocks = std::max<int64_t>(needed, 1);
    if ((rc = walker_event(r, st))) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(32 * wpb);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (plan.l2_persist && ctx->l2_persist_max > 0 && ctx->l2_window_max > 0) {
        // node records persisting in L2: every step reads one, the rows'
        // records stream past them
        const size_t bytes = std::min((size_t)kp.n_nodes * sizeof(typename E::Node), ctx->l2_window_max);
        if (ctx->l2_persist_set < std::min(bytes, ctx->l2_persist_max)) {
            ctx->l2_persist_set = std::min(bytes, ctx->l2_persist_max);
            PPR_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, ctx->l2_persist_set));
        }
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = (void *)kp.node;
        attr[0].val.accessPolicyWindow.num_bytes = bytes;
        attr[0].val.accessPolicyWindow.hitRatio = std::min(1.0f, (float)ctx->l2_persist_set / (float)bytes);
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    PPR_CUDA(cudaLaunchKernelEx(&cfg, k_walk_persistent<E, SEG, STATS, BOUNDED, SPLIT>, kp));
    note_launch();
    PPR_CUDA(cudaGetLastError());
    if ((rc = walker_event(r, st))) return rc;
    return launch_aggregate(ctx, AggParams{kp.ends, kp.R, kp.P2, S, kp.out_row0, kp.out, kp.order}, st);
}

// Chunk table of a batched graph, built on the device: chunks of at most CS
// sources that never cross an instance boundary, with positions relative to
// s_begin; the count goes to *nchunks.
__global__ void k_chunk_count(int32_t count, const int64_t *node_off, int64_t s_begin, int64_t s_end, uint32_t CS,
                              uint32_t *cnt)
{
    for (int32_t gi = blockIdx.x * blockDim.x + threadIdx.x; gi < count; gi += gridDim.x * blockDim.x) {
        const int64_t a = max(node_off[gi], s_begin), b = min(node_off[gi + 1], s_end);
        cnt[gi] = b > a ? (uint32_t)((b - a + CS - 1) / CS) : 0u;
    }
}

__global__ void k_chunk_fill(int32_t count, const int64_t *node_off, int64_t s_begin, int64_t s_end, uint32_t CS,
                             const uint64_t *offs, int4 *chunks, unsigned long long *nchunks)
{
    for (int32_t gi = blockIdx.x * blockDim.x + threadIdx.x; gi < count; gi += gridDim.x * blockDim.x) {
        const int64_t a = max(node_off[gi], s_begin), b = min(node_off[gi + 1], s_end);
        uint64_t o = offs[gi];
        for (int64_t s = a; s < b; s += CS, ++o)
            chunks[o] = make_int4((int)(s - s_begin), (int)min((int64_t)CS, b - s), gi, 0);
        if (gi == count - 1) *nchunks = offs[count];
    }
}

// sources per chunk; a chunk holds at most 2^19 walks (walk indices within a
// chunk stay below 2^20 for the multiply-shift division by R)
static uint32_t chunk_sources(const RunPlan &plan)
{
    const uint32_t cs = plan.chunk_sources > 0 ? (uint32_t)plan.chunk_sources : std::max(1u, 400u / plan.R);
    return std::min(cs, std::max(1u, (1u << 19) / plan.R));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t launch_workspace_bytes(const ppr_graph *g, const RunPlan &plan, int64_t S)
{
    size_t b = align256((size_t)S * plan.R * sizeof(uint32_t));  // endpoints
    if (g->instances > 0 && plan.kernel == PPR_KERNEL_PERSISTENT) {
        const uint32_t CS = chunk_sources(plan);
        const int64_t cnt = g->instances;
        const int64_t tiles = (cnt + kScanTile - 1) / kScanTile;
        b += align256(sizeof(int4) * (size_t)((S + CS - 1) / CS + cnt + 1));  // chunk table
        b += align256(sizeof(uint32_t) * (size_t)cnt);                      // per-instance chunk counts
        b += align256(sizeof(uint64_t) * (size_t)(cnt + 1));                // their offsets
        b += align256(sizeof(uint64_t) * (size_t)(tiles + 2));              // scan scratch
    }
    return b;
}

// Every kernel a run can launch is loaded here, once per device.  With lazy
// module loading the first launch of a kernel may wait for the device to go
// idle; loaded up front, a run's launches stay asynchronous.
template <class E, bool SEG, bool STATS, bool SPLIT = false>
static void preload_walkers()
{
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, k_walk_plain<E, SEG, STATS, SPLIT>);
    cudaFuncGetAttributes(&a, k_walk_persistent<E, SEG, STATS, false, SPLIT>);
}

void preload_run_kernels()
{
    preload_walkers<NarrowEdges, false, false>();
    preload_walkers<NarrowEdges, true, false>();
    preload_walkers<NarrowEdges, false, true>();
    preload_walkers<NarrowEdges, true, true>();
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_walk_persistent<NarrowEdges, false, false, true>);
    cudaFuncGetAttributes(&fa, k_walk_persistent<NarrowEdges, true, false, true>);
    preload_walkers<NarrowEdges, false, false, true>();
    preload_walkers<NarrowEdges, true, false, true>();
    preload_walkers<NarrowEdges, false, true, true>();
    preload_walkers<NarrowEdges, true, true, true>();
    cudaFuncGetAttributes(&fa, k_walk_persistent<NarrowEdges, false, false, true, true>);
    cudaFuncGetAttributes(&fa, k_walk_persistent<NarrowEdges, true, false, true, true>);
    preload_walkers<WideEdges, false, false>();
    preload_walkers<WideEdges, true, false>();
    preload_walkers<WideEdges, false, true>();
    preload_walkers<WideEdges, true, true>();
    preload_walkers<AliasEdges, false, false>();
    preload_walkers<AliasEdges, false, true>();
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, k_aggregate<0>);
    cudaFuncGetAttributes(&a, k_aggregate<1>);
    cudaFuncGetAttributes(&a, k_aggregate<2>);
    cudaFuncGetAttributes(&a, k_aggregate<4>);
    cudaFuncGetAttributes(&a, k_aggregate<8>);
    cudaFuncGetAttributes(&a, k_aggregate<16>);
    cudaFuncGetAttributes(&a, k_aggregate<32>);
    cudaFuncGetAttributes(&a, k_chunk_count);
    cudaFuncGetAttributes(&a, k_chunk_fill);
    cudaFuncGetAttributes(&a, k_scan_tile_sums);
    cudaFuncGetAttributes(&a, k_scan_tile_offsets);
    cudaFuncGetAttributes(&a, k_scan_apply);
    cudaGetLastError();
}

// Narrow layout: SPLIT for a renumbered graph's layout (summary array,
// evict-first bottom blocks), else summaries before each row's blocks.
template <bool SPLIT>
static int launch_narrow(ppr_ctx *ctx, const KParams &kp, const RunPlan &plan, int64_t S, cudaStream_t st,
                         ppr_result *ev_owner)
{
    if (plan.stats)
        return plan.segments ? launch_typed<NarrowEdges, true, true, false, SPLIT>(ctx, kp, plan, S, st, ev_owner)
                             : launch_typed<NarrowEdges, false, true, false, SPLIT>(ctx, kp, plan, S, st, ev_owner);
    // the bounded step: persistent kernel, no cooperative search (statistics launches took the branch above)
    if (plan.step_loads > 0 && plan.kernel == PPR_KERNEL_PERSISTENT && kp.large == 0xffffffffu)
        return plan.segments ? launch_typed<NarrowEdges, true, false, true, SPLIT>(ctx, kp, plan, S, st, ev_owner)
                             : launch_typed<NarrowEdges, false, false, true, SPLIT>(ctx, kp, plan, S, st, ev_owner);
    return plan.segments ? launch_typed<NarrowEdges, true, false, false, SPLIT>(ctx, kp, plan, S, st, ev_owner)
                         : launch_typed<NarrowEdges, false, false, false, SPLIT>(ctx, kp, plan, S, st, ev_owner);
}

int launch_walks(ppr_ctx *ctx, const ppr_graph *g, const RunPlan &plan, const Outputs &o, int64_t s_begin, int64_t S,
                 const uint32_t *src_list, int64_t out_row0, unsigned char *ws, cudaStream_t st, ppr_result *ev_owner,
                 bool reset_queue)
{
    if (S <= 0) return PPR_OK;
    KParams kp{};
    kp.node = plan.segments ? g->seg.node : (plan.sampler == 1 ? g->alias.node : g->node);
    kp.edges = plan.sampler == 1 ? (const void *)g->alias.slots : g->edges;
    kp.seg = g->seg.entries;
    kp.R = plan.R;
    kp.T = plan.T;
    kp.k0 = (uint32_t)plan.seed;
    kp.k1 = (uint32_t)(plan.seed >> 32);
    kp.tag = plan.tag;
    kp.dangling = plan.dangling;
    kp.large = plan.large_degree > 0 ? (uint32_t)plan.large_degree : 0xffffffffu;  // 0: off
    kp.s_begin = s_begin;
    kp.s_end = s_begin + S;
    kp.src_list = src_list;
    kp.rank = g->rank;
    kp.order = g->order;
    kp.out_row0 = out_row0;
    kp.out.nnz = o.nnz;
    kp.out.cols = o.cols;
    kp.out.cnts = o.cnts;
    kp.out.topk_idx = o.topk_idx;
    kp.out.topk_cnt = o.topk_cnt;
    kp.out.cap = o.cap;
    kp.out.topk = o.topk;
    kp.steps = o.counters;
    kp.queue = o.counters + 1;
    uint32_t P2 = 1;
    while (P2 < plan.R) P2 <<= 1;
    kp.P2 = P2;
    kp.r_magic = ((1ull << 40) + plan.R - 1) / plan.R;
    kp.refill = plan.refill_lanes > 0 ? (uint32_t)std::min(plan.refill_lanes, 32) : 1u;
    kp.step_loads = (uint32_t)std::max(plan.step_loads, 0);
    kp.n_nodes = g->n;
    kp.n_records = plan.sampler == 1 ? (uint64_t)g->m : (uint64_t)g->edge_records;
    kp.sum = g->sum_base();
    kp.n_sum = g->sum_extent();
    kp.n_seg = (uint64_t)g->seg.entries_cap;
    kp.err = o.counters + 4;
    kp.ends = reinterpret_cast<uint32_t *>(ws);
    size_t off = align256((size_t)S * plan.R * sizeof(uint32_t));

    if (plan.kernel == PPR_KERNEL_PLAIN) {
        if (g->instances > 0) {
            kp.inst_off = g->d_node_off;
            kp.instances = g->instances;
        }
    } else {
        const uint32_t CS = chunk_sources(plan);
        kp.CS = CS;
        if (g->instances > 0) {
            const int64_t cnt = g->instances;
            int4 *chunks = reinterpret_cast<int4 *>(ws + off);
            off += align256(sizeof(int4) * (size_t)((S + CS - 1) / CS + cnt + 1));
            uint32_t *ccount = reinterpret_cast<uint32_t *>(ws + off);
            off += align256(sizeof(uint32_t) * (size_t)cnt);
            uint64_t *coffs = reinterpret_cast<uint64_t *>(ws + off);
            off += align256(sizeof(uint64_t) * (size_t)(cnt + 1));
            uint64_t *ctmp = reinterpret_cast<uint64_t *>(ws + off);
            const int cb = (int)std::min<int64_t>((cnt + 255) / 256, 1024);
            k_chunk_count<<<cb, 256, 0, st>>>((int32_t)cnt, g->d_node_off, s_begin, s_begin + S, CS, ccount);
            note_launch();
            exclusive_scan_u32(ccount, cnt, coffs, ctmp, st);
            k_chunk_fill<<<cb, 256, 0, st>>>((int32_t)cnt, g->d_node_off, s_begin, s_begin + S, CS, coffs, chunks,
                                             o.counters + 3);
            note_launch();
            PPR_CUDA(cudaGetLastError());
            kp.chunks = chunks;
            kp.inst_off = g->d_node_off;
            kp.nchunks_dev = o.counters + 3;
            kp.nchunks = (uint32_t)((S + CS - 1) / CS + cnt);  // upper bound, for the grid size
        } else {
            // walks per chunk: CS sources' worth, smaller when that leaves warps
            // idle (a small run still spreads over every resident warp)
            const uint64_t walks = (uint64_t)S * plan.R;
            const uint64_t warps = (uint64_t)ctx->sms * 48;
            uint64_t cw = std::min<uint64_t>((uint64_t)CS * plan.R, 1u << 19);
            if ((walks + cw - 1) / cw < warps) cw = std::max<uint64_t>(32, (walks + warps - 1) / warps);
            cw = std::min<uint64_t>(cw, 1u << 19);
            kp.CW = (uint32_t)cw;
            kp.walks = walks;
            kp.nchunks = (uint32_t)((walks + cw - 1) / cw);
        }
        if (reset_queue) PPR_CUDA(cudaMemsetAsync(kp.queue, 0, sizeof(unsigned long long), st));
    }
    if (plan.sampler == 1)
        return plan.stats ? launch_typed<AliasEdges, false, true>(ctx, kp, plan, S, st, ev_owner)
                          : launch_typed<AliasEdges, false, false>(ctx, kp, plan, S, st, ev_owner);
    if (g->wide) {
        if (plan.stats)
            return plan.segments ? launch_typed<WideEdges, true, true>(ctx, kp, plan, S, st, ev_owner)
                                 : launch_typed<WideEdges, false, true>(ctx, kp, plan, S, st, ev_owner);
        return plan.segments ? launch_typed<WideEdges, true, false>(ctx, kp, plan, S, st, ev_owner)
                             : launch_typed<WideEdges, false, false>(ctx, kp, plan, S, st, ev_owner);
    }
    return g->sum ? launch_narrow<true>(ctx, kp, plan, S, st, ev_owner)
                  : launch_narrow<false>(ctx, kp, plan, S, st, ev_owner);
}

// ------------------------------------------------ allocation-free run ----
// Scratch for ppr_run_noalloc: a fixed array in device memory that exists on
// every GPU where this library's kernels are loaded, for the life of the
// process.  Layout: 256-byte header (steps, queue, sectors counters), then
// one 4-byte endpoint per walk.
constexpr size_t kNoAllocBytes = 64ull << 20;
constexpr size_t kNoAllocHeader = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device addresses of g_noalloc_scratch, one per device, fetched on the first
// call for that device (the host-side symbol is only a stand-in).
static void *g_noalloc_ptr[64];
static std::mutex g_noalloc_mu;

static int noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= 64) {
        set_error("device %d out of range for the allocation-free entry point", device);
        return PPR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);  // device is current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[device] = ptr;
    }
    *out = static_cast<unsigned char *>(g_noalloc_ptr[device]);
    return PPR_OK;
}

}  // namespace ppr

using namespace ppr;

extern "C" int ppr_run_noalloc(ppr_ctx *ctx, const ppr_graph *g, const ppr_run_args *a, uint32_t *nnz, int32_t *cols,
                               uint32_t *cnts, uint32_t cap, int32_t *topk_idx, uint32_t *topk_cnt)
{
    if (!ctx || !g || !a || !nnz || !cols || !cnts) {
        set_error("NULL argument");
        return PPR_EINVAL;
    }
    // the checks every run entry point shares (ranges, modes, tuning limits)
    RunPlan plan;
    int rc = check_run(g, a, 0, false, &plan);
    if (rc) return rc;
    // and those of this entry point: one persistent launch into caller buffers
    if (a->topk > 0 && (!topk_idx || !topk_cnt)) {
        set_error("topk = %d needs the top-k outputs", a->topk);
        return PPR_EINVAL;
    }
    if (a->kernel != PPR_KERNEL_PERSISTENT || a->stats != 0) {
        set_error("invalid mode for the allocation-free run (persistent kernel, no statistics)");
        return PPR_EINVAL;
    }
    if (g->instances > 0) {
        set_error("the allocation-free run takes plain graphs only");
        return PPR_ENOTSUP;
    }
    if (plan.segments && !(g->seg.T == plan.T && g->seg.node)) {
        set_error("segment tables for this alpha are not built (a ppr_run with segments=1 builds them)");
        return PPR_ENOTSUP;
    }
    if (plan.sampler == 1 && !g->alias.node) {
        set_error("alias sampler: needs tables built by an earlier ppr_run with sampler=1");
        return PPR_ENOTSUP;
    }
    const uint32_t need_cap = (uint32_t)std::min<int64_t>((int64_t)a->R, g->n);
    if (cap < need_cap) {
        set_error("row capacity %u < min(R, n) = %u", cap, need_cap);
        return PPR_EINVAL;
    }
    const int64_t S = a->src_end - a->src_begin;
    const size_t need = kNoAllocHeader + (size_t)S * a->R * sizeof(uint32_t);
    if (need > kNoAllocBytes) {
        set_error("allocation-free run needs %zu bytes of scratch for %lld sources x %u walks; the fixed scratch "
                  "holds %zu (at most %zu walks per call)",
                  need, (long long)S, a->R, kNoAllocBytes, (kNoAllocBytes - kNoAllocHeader) / sizeof(uint32_t));
        return PPR_ERANGE;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    unsigned char *scratch = nullptr;
    rc = noalloc_scratch(ctx->device, &scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)a->stream;
    // the counters must start at zero on every call; endpoints are overwritten
    e = cudaMemsetAsync(scratch, 0, kNoAllocHeader, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch header)");

    plan.l2_persist = false;  // no device-limit change from the allocation-free path
    Outputs out{nnz, cols, cnts, cap, topk_idx, topk_cnt, a->topk, reinterpret_cast<unsigned long long *>(scratch)};
    return launch_walks(ctx, g, plan, out, a->src_begin, a->src_end - a->src_begin, nullptr, 0,
                        scratch + kNoAllocHeader, st, nullptr);
}
