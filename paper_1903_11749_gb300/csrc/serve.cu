// serve.cu -- multi-source PPR queries served by continuous batching.
//
// Device loop (PPR_SERVE_DEVICE_LOOP, the default).  One persistent kernel
// (k_serve_loop) stays resident and serves every query; the walks' state lives
// in its registers across queries.  The host admits queries in arrival order
// as device memory (an arena of memory_budget bytes) and one of kRing ring
// slots allow: it copies the query's sources to the device, writes the slot's
// descriptor and counters, and advances a tail counter in host-mapped memory.
// Seven of each block's eight warps walk: a warp takes a chunk of walks from
// the published queries (starting at its own query among those with chunks
// left, so each query gets a share of the warps as soon as it is published)
// and refills its lanes as walks end, a lane carrying walks of different
// queries at once, each with its own Philox key and stop threshold -- the
// paper's pipelines (Sec. 3, Algorithm 2) start new walks while old ones
// finish in the same way.  Finished walks are counted per query.  The eighth
// warp of each block aggregates: once all walks of a query are done it takes
// the query's sources one at a time (the per-source reduction of
// aggregate.cuh), writes each top-k row straight into pinned host memory and,
// after the last row, marks the query done in host-mapped memory, where the
// host's scheduler thread picks it up.  Every wait on the device is bounded in
// time (%globaltimer): a loop without work exits after idle_us and the host
// launches it again with the next query; a published slot whose descriptor
// does not appear within a second ends the loop with an error status, which
// fails the queries in flight.
//
// Streams (PPR_SERVE_STREAMS).  The host scheduler of earlier builds: each
// admitted query runs the persistent walker and the reduction on one of a few
// streams; a finished query's top-k is copied to pinned memory.
//
// Both modes give every query the rows of ppr_run_list over its sources
// (tag 0, dangling mode 0, no segment tables): the draw of walk j of source s
// at step k depends on (seed, s, j, k) alone.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ppr_host.h"
#include "walk_step.cuh"

namespace ppr {

using clock_t_ = std::chrono::steady_clock;

static int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(clock_t_::now().time_since_epoch()).count();
}

// ======================================================= device loop ====

constexpr int kRing = 64;            // queries in flight at most (ring slots)
constexpr int kLoopWarps = 8;        // per block: kLoopWarps - 1 walker warps, one aggregator
constexpr uint32_t kLoopMaxR = 1024; // largest R the loop's reduction takes
constexpr uint64_t kSlotWaitNs = 1000000000ull;   // bound on the wait for a published descriptor
constexpr uint64_t kBusyWaitNs = 120000000000ull;  // bound on an aggregator waiting for walks in flight

// Descriptor of a published query (device memory; the host writes it, then
// publishes).  seq1 = the query's sequence number + 1 (0: never written).
struct __align__(16) SDesc {
    const uint32_t *src;  // S source ids
    uint32_t *ends;       // S * R endpoints, walk g = pos * R + j at [g]
    int32_t *out_idx;     // S * topk, host-mapped
    uint32_t *out_cnt;
    uint64_t r_magic;     // ceil(2^40 / R): g / R by multiply-shift (exact for g < 2^40 / R)
    uint64_t seq1;
    uint32_t S, R, T, k0, k1, topk, cw, nchunks, walks, P2;
    uint32_t pad[2];
};

// Counters of a ring slot (device memory; the host writes them before
// publishing).  claim and agg hold the low 32 bits of (sequence number + 1)
// above the number of chunks / sources handed out so far: one load tells a
// warp whether the slot holds the query it looks for and whether work is
// left, and work is taken with one atomic add (no retries under contention);
// the tag of the word an add returns says whose work it took, so a warp with
// a stale view of the ring that lands on a reused slot takes work of the
// query that holds it now (never work that no one else will do).
struct __align__(64) SSlot {
    unsigned long long claim;       // chunks still to hand out
    unsigned long long agg;         // sources still to hand to aggregators
    unsigned long long walks_done;  // walks finished
    unsigned long long agg_done;    // sources reduced
    unsigned long long t_claim, t_walks, t_done;  // %globaltimer: first chunk taken, last walk counted, last row
    unsigned long long pad;
};

// Control block in host-mapped memory.
struct SCtl {
    unsigned long long tail;            // queries published (host)
    unsigned long long done[kRing];     // seq + 1 of the query finished in each slot (device)
    unsigned int stop;                  // host: end once no work is left
    unsigned int status;                // device: exit reasons (PPR_LOOP_*)
};

struct SGlob {  // device memory, persists across launches of the loop
    unsigned long long head;      // oldest query that may still have chunks to hand out
    unsigned long long agg_head;  // oldest query that may still have sources to reduce
    unsigned long long err;       // checked build: flags of indices that left their array
    // activity counters (ppr_serve_info)
    unsigned long long draws, iterations, claims, claim_misses, sleeps, reduced;
    unsigned long long cyc_claim, cyc_step, cyc_sleep, cyc_total;  // walker-warp clock cycles by activity
};

struct LoopParams {
    KParams kp;  // the graph layout (node, edges, n_nodes, n_records); dangling mode 0, no segments
    const SDesc *desc;
    SSlot *slot;
    SCtl *ctl;   // device view of the host-mapped control block
    SGlob *glob;
    uint32_t refill;
    uint32_t walker_warps;  // in the whole grid
    uint64_t idle_ns;
};

__device__ __forceinline__ uint64_t gtime_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The published tail, read from host memory without acquire semantics (an
// acquire would invalidate the SM's L1 under the walkers): the host writes a
// slot's descriptor and counters, waits for those copies, and only then
// advances the tail; the loop reads slots through L2 (ld.cg) after it has
// seen the tail, so it sees them written.
__device__ __forceinline__ unsigned long long ld_tail(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

// count += v with release semantics at device scope: the endpoint stores of
// every lane that synchronised with this one (__syncwarp) are visible in L2
// before the count is (no full fence: nothing is invalidated).  Returns the
// count before.
__device__ __forceinline__ unsigned long long add_release(unsigned long long *p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_volatile(const unsigned int *p) { return *(const volatile unsigned int *)p; }

__device__ __forceinline__ void flag_exit(const LoopParams &P, uint32_t why) { atomicOr(&P.ctl->status, why); }

// Relation of a tagged slot word to query id: 0 the slot holds id, 1 it holds
// a later query (id is finished), -1 it was not yet written for id.
__device__ __forceinline__ int tag_rel(unsigned long long w, uint64_t id)
{
    const int32_t d = (int32_t)((uint32_t)(w >> 32) - (uint32_t)(id + 1));
    return d == 0 ? 0 : (d > 0 ? 1 : -1);
}

// Lane 0: waits (bounded) until the word *w is written for query id; 1 when it
// is (or a later query holds it), -1 when the bound ran out (the loop then
// exits with PPR_LOOP_SLOT_TIMEOUT).  The host writes a slot before it
// publishes it, so only a slot published unwritten (the test hook) waits.
__device__ int await_slot(const LoopParams &P, const unsigned long long *w, uint64_t id)
{
    const uint64_t t0 = gtime_ns();
    while (tag_rel(__ldcg(w), id) < 0) {
        if (gtime_ns() - t0 > kSlotWaitNs) {
            flag_exit(P, PPR_LOOP_SLOT_TIMEOUT);
            return -1;
        }
        __nanosleep(1000);
    }
    return 1;
}

// Advance *head from h to h + 1 (another warp may have done it).
__device__ __forceinline__ void bump(unsigned long long *head, uint64_t h) { atomicCAS(head, h, h + 1); }

// The block's copy of the published tail (s[0]) and when it was last read
// from host memory (s[1]).  A warp that finds no work asks for a refresh; the
// host is read at most once per kTailReadNs per block (lane 0; the tail goes
// to every lane).
constexpr uint64_t kTailReadNs = 4000;
constexpr uint64_t kClaimRetryNs = 20000;  // a warp with walks running waits this long after a claim found nothing
__device__ __forceinline__ uint64_t block_tail(const LoopParams &P, unsigned long long *s, bool refresh)
{
    unsigned long long t = 0;
    if ((threadIdx.x & 31) == 0) {
        t = *(volatile unsigned long long *)&s[0];
        if (refresh) {
            const uint64_t now = gtime_ns();
            if (now - *(volatile unsigned long long *)&s[1] > kTailReadNs) {
                s[1] = now;
                const unsigned long long ht = ld_tail(&P.ctl->tail);
                if (ht > t) {
                    atomicMax(&s[0], ht);
                    t = ht;
                }
            }
        }
    }
    return __shfl_sync(0xffffffffu, t, 0);
}

// Work of one walker warp: a chunk of walks [g0, g0 + total) of query `id`.
struct WalkChunk {
    uint64_t id, magic;
    const uint32_t *src;
    uint32_t slot, g0, issued, total, R, T, k0, k1;
};

// Lane 0: fills *c with chunk ci of the query whose descriptor is in slot s
// (sequence number + 1 = tag), once that descriptor is in place (the host
// writes it before the slot's counters; bounded wait).  1, or -1 when the
// wait ran out.
__device__ int take_chunk(const LoopParams &P, uint32_t s, uint32_t tag, uint32_t ci, WalkChunk *c)
{
    const SDesc *d = P.desc + s;
    const uint64_t t0 = gtime_ns();
    while ((uint32_t)__ldcg(&d->seq1) != tag) {
        if (gtime_ns() - t0 > kSlotWaitNs) {
            flag_exit(P, PPR_LOOP_SLOT_TIMEOUT);
            return -1;
        }
        __nanosleep(500);
    }
    atomicCAS(&P.slot[s].t_claim, 0ull, (unsigned long long)gtime_ns());
    const uint32_t cw = __ldcg(&d->cw), walks = __ldcg(&d->walks);
    c->id = __ldcg(&d->seq1) - 1;
    c->slot = s;
    c->g0 = ci * cw;
    c->total = min(cw, walks - ci * cw);
    c->issued = 0;
    c->R = __ldcg(&d->R);
    c->T = __ldcg(&d->T);
    c->k0 = __ldcg(&d->k0);
    c->k1 = __ldcg(&d->k1);
    c->magic = __ldcg(&d->r_magic);
    c->src = reinterpret_cast<const uint32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&d->src)));
    return 1;
}

// Whole warp: hands out one chunk of some published query into *c (written by
// lane 0).  The lanes read the claim words of the queries in [head, tail) in
// parallel; among those with chunks left the warp takes the start-th (mod
// their number), so the walker warps share themselves out over the queries in
// flight, and takes the next chunk of it with one atomic add (no retries under
// contention).  The word's tag says which query the add landed on: if the
// slot was reused in the meantime, the warp takes the chunk of the query that
// now holds it.  Returns 1 (a chunk), 0 (none now), -1 (the loop must end: a
// published slot stayed unwritten).
__device__ int claim_chunk(const LoopParams &P, uint32_t start, WalkChunk *c, unsigned long long *s_tail)
{
    const uint32_t lane = threadIdx.x & 31;
    bool refresh = false;
    for (int attempt = 0; attempt < 3; ++attempt) {
        const uint64_t t = block_tail(P, s_tail, refresh);
        uint64_t h = __ldcg(&P.glob->head);
        if (t > kRing && h < t - kRing) h = t - kRing;  // ids below t - kRing are finished (their slots reused)
        const uint32_t n = h < t ? (uint32_t)(t - h < (uint64_t)kRing ? t - h : (uint64_t)kRing) : 0u;
        uint32_t ok[2];
        int unwritten = -1;  // window index of a slot published but not yet written
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const uint32_t i = r * 32 + lane;
            bool o = false;
            if (i < n) {
                const uint64_t id = h + i;
                const uint32_t s = (uint32_t)(id % kRing);
                const unsigned long long w = __ldcg(&P.slot[s].claim);
                const int rel = tag_rel(w, id);
                const bool left = rel == 0 && (uint32_t)w < __ldcg(&P.desc[s].nchunks);
                o = left;
                if (rel < 0) unwritten = (int)i;
                if (i == 0 && (rel > 0 || (rel == 0 && !left))) bump(&P.glob->head, h);
            }
            ok[r] = __ballot_sync(0xffffffffu, o);
        }
        const uint32_t um = __ballot_sync(0xffffffffu, unwritten >= 0);
        if (um) {
            const int ui = __shfl_sync(0xffffffffu, unwritten, __ffs(um) - 1);
            int r = 0;
            if (lane == 0) r = await_slot(P, &P.slot[(h + ui) % kRing].claim, h + ui);
            if (__shfl_sync(0xffffffffu, r, 0) < 0) return -1;
            continue;
        }
        const uint32_t cnt = __popc(ok[0]) + __popc(ok[1]);
        if (cnt == 0) {  // nothing in view: look once at the host's tail (rate-limited), then give up
            if (refresh) return 0;
            refresh = true;
            continue;
        }
        // the k-th query with chunks left
        uint32_t k = start % cnt, i;
        if (k < (uint32_t)__popc(ok[0])) {
            uint32_t m = ok[0];
            for (uint32_t q = 0; q < k; ++q) m &= m - 1;
            i = __ffs(m) - 1;
        } else {
            uint32_t m = ok[1];
            for (uint32_t q = __popc(ok[0]); q < k; ++q) m &= m - 1;
            i = 32 + __ffs(m) - 1;
        }
        int got = 0;
        if (lane == 0) {
            const uint32_t s = (uint32_t)((h + i) % kRing);
            const unsigned long long old = atomicAdd(&P.slot[s].claim, 1ull);
            const uint32_t tag = (uint32_t)(old >> 32), ci = (uint32_t)old;
            // the chunk exists if ci is below the chunk count of the query that holds the slot now
            const SDesc *d = P.desc + s;
            if (tag != 0) {
                const uint64_t t0 = gtime_ns();
                while ((uint32_t)__ldcg(&d->seq1) != tag && gtime_ns() - t0 < kSlotWaitNs) __nanosleep(500);
                if ((uint32_t)__ldcg(&d->seq1) == tag && ci < __ldcg(&d->nchunks)) got = take_chunk(P, s, tag, ci, c);
            }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got) return got;
    }
    return 0;
}

// Finished walks of query slot q: n more, after the writers' endpoint stores
// (the warp has synchronised; the add is a release).
__device__ __forceinline__ void count_walks(const LoopParams &P, uint32_t q, uint32_t n)
{
    const unsigned long long old = add_release(&P.slot[q].walks_done, (unsigned long long)n);
    if (old + n == __ldcg(&P.desc[q].walks)) P.slot[q].t_walks = gtime_ns();
}

template <class E, bool SPLIT>
__device__ void walker_warp(const LoopParams &P, WalkChunk &wc, uint32_t **ends_of, uint32_t gwarp,
                            unsigned long long *s_tail)
{
    const uint32_t lane = threadIdx.x & 31;
    const E edges = make_edges<E>(P.kp.edges);
    bool active = false;
    uint32_t q = 0, g = 0, src = 0, j = 0, k = 0, u = 0;
    uint32_t s0 = 0;  // the walk's start (and restart) node in the layout's numbering
    StepKey key{0, 0, 0};
    uint32_t pend_q = 0xffffffffu, pend_n = 0;  // uniform: walks of pend_q finished, not yet counted
    bool have = false;                          // uniform: wc holds walks left to issue
    uint64_t idle_t0 = 0, flush_t = gtime_ns(), claim_after = 0;
    uint32_t backoff = 256;
    uint32_t n_iter = 0, n_claim = 0, n_miss = 0, n_sleep = 0;  // activity, flushed to P.glob
    unsigned long long c_claim = 0, c_step = 0, c_sleep = 0;
    long long c_start = clock64();
    Tally tl;
    auto flush = [&]() {
        unsigned long long d = tl.steps;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) {
            const long long now = clock64();
            atomicAdd(&P.glob->draws, d);
            atomicAdd(&P.glob->iterations, (unsigned long long)n_iter);
            atomicAdd(&P.glob->claims, (unsigned long long)n_claim);
            atomicAdd(&P.glob->claim_misses, (unsigned long long)n_miss);
            atomicAdd(&P.glob->sleeps, (unsigned long long)n_sleep);
            atomicAdd(&P.glob->cyc_claim, c_claim);
            atomicAdd(&P.glob->cyc_step, c_step);
            atomicAdd(&P.glob->cyc_sleep, c_sleep);
            atomicAdd(&P.glob->cyc_total, (unsigned long long)(now - c_start));
            c_start = now;
        }
        tl.steps = 0;
        n_iter = n_claim = n_miss = n_sleep = 0;
        c_claim = c_step = c_sleep = 0;
    };
    for (;;) {
        uint32_t idle = __ballot_sync(0xffffffffu, !active);
        const bool all_idle = idle == 0xffffffffu;
        if ((uint32_t)__popc(idle) < P.refill) idle = 0;
        // after a claim found nothing, a warp with walks still running tries again only later
        if (!all_idle && !have && claim_after && gtime_ns() < claim_after) idle = 0;
        int status = 0;
        while (idle) {
            if (!have) {
                const long long c0 = clock64();
                const int r = claim_chunk(P, gwarp, &wc, s_tail);
                __syncwarp();
                c_claim += clock64() - c0;
                ++n_claim;
                n_miss += r <= 0;
                claim_after = (r == 0 && !all_idle) ? gtime_ns() + kClaimRetryNs : 0;
                if (r <= 0) {
                    status = r;
                    break;
                }
                have = true;
                if (lane == 0) ends_of[wc.slot] = const_cast<uint32_t *>(
                    reinterpret_cast<const uint32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&P.desc[wc.slot].ends))));
                if (wc.slot != pend_q) {  // count what is pending before switching
                    if (pend_n) {
                        __syncwarp();
                        if (lane == 0) count_walks(P, pend_q, pend_n);
                        pend_n = 0;
                    }
                    pend_q = wc.slot;
                }
                __syncwarp();
            }
            const uint32_t issued = wc.issued;
            const uint32_t take = min(wc.total - issued, (uint32_t)__popc(idle));
            const uint32_t rank = __popc(idle & ((1u << lane) - 1));
            if (((idle >> lane) & 1) && rank < take) {
                g = wc.g0 + issued + rank;
                const uint32_t pos = (uint32_t)(((uint64_t)g * wc.magic) >> 40);
                j = g - pos * wc.R;
                src = __ldcg(wc.src + pos);  // the caller's id keys the draws
                s0 = P.kp.rank ? (uint32_t)P.kp.rank[src] : src;
                q = wc.slot;
                key = StepKey{wc.k0, wc.k1, wc.T};
                k = 0;
                u = s0;
                active = true;
            }
            __syncwarp();
            if (lane == 0) wc.issued = issued + take;
            __syncwarp();
            if (issued + take == wc.total) have = false;
            idle = __ballot_sync(0xffffffffu, !active);
        }
        if (status < 0) break;  // a descriptor wait ran out: the loop ends
        if (__ballot_sync(0xffffffffu, active) == 0) {
            // no walk and no chunk: stop, or wait (bounded) for the next query
            if (ld_volatile(&P.ctl->stop)) {
                if (lane == 0) flag_exit(P, PPR_LOOP_STOPPED);
                break;
            }
            const uint64_t t = gtime_ns();
            if (idle_t0 == 0) idle_t0 = t;
            else if (t - idle_t0 > P.idle_ns) {
                if (lane == 0) flag_exit(P, PPR_LOOP_IDLE);
                break;
            }
            ++n_sleep;
            const long long c0 = clock64();
            __nanosleep(backoff);
            c_sleep += clock64() - c0;
            backoff = min(backoff * 2, 32768u);
            continue;
        }
        idle_t0 = 0;
        backoff = 256;
        if (++n_iter % 1024 == 0) {
            const uint64_t t = gtime_ns();
            if (t - flush_t > 1000000) {
                flush();
                flush_t = t;
            }
        }
        uint32_t end = 0;
        bool fin = false;
        const long long c0 = clock64();
        if (walk_step<E, false, false, false, SPLIT>(P.kp, key, edges, active, s0, src, j, 0, k, u, end, tl)) {
            ends_of[q][g] = end;
            active = false;
            fin = true;
        }
        __syncwarp();
        c_step += clock64() - c0;
        // completion counting: walks of pend_q add up in a register, others at once
        const uint32_t fin_m = __ballot_sync(0xffffffffu, fin);
        if (fin_m) {
            const uint32_t same = __ballot_sync(0xffffffffu, fin && q == pend_q);
            pend_n += __popc(same);
            const uint32_t other = fin_m & ~same;
            if (other) {
                __syncwarp();
                if ((other >> lane) & 1) {
                    const uint32_t m = __match_any_sync(other, q);
                    if (lane == (uint32_t)(__ffs(m) - 1)) count_walks(P, q, __popc(m));
                }
                __syncwarp();
            }
        }
        if (pend_n && __ballot_sync(0xffffffffu, active && q == pend_q) == 0 && !(have && wc.slot == pend_q)) {
            __syncwarp();
            if (lane == 0) count_walks(P, pend_q, pend_n);
            pend_n = 0;
        }
    }
    if (pend_n) {  // nothing active here: every walk of pend_q this warp ran is done
        __syncwarp();
        if (lane == 0) count_walks(P, pend_q, pend_n);
    }
    flush();
}

// Whole warp: hands out one source of the oldest query whose walks are all
// done.  Returns 1 (query id, slot, source i on every lane), 0 (none now),
// -1 (the loop must end); *in_flight tells whether published queries still
// have sources to hand out (ready or not).
__device__ int claim_source(const LoopParams &P, unsigned long long *s_tail, bool refresh, uint32_t max_R,
                            uint64_t &id_out, uint32_t &slot_out, uint32_t &i_out, uint32_t &n_out, bool &in_flight)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t t = block_tail(P, s_tail, refresh);
    uint64_t h = __ldcg(&P.glob->agg_head);
    if (t > kRing && h < t - kRing) h = t - kRing;
    const uint32_t n = h < t ? (uint32_t)(t - h < (uint64_t)kRing ? t - h : (uint64_t)kRing) : 0u;
    uint32_t ready[2], left = 0;
    int unwritten = -1;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const uint32_t i = r * 32 + lane;
        bool o = false;
        if (i < n) {
            const uint64_t id = h + i;
            const uint32_t s = (uint32_t)(id % kRing);
            const unsigned long long a = __ldcg(&P.slot[s].agg);
            const unsigned long long wd = __ldcg(&P.slot[s].walks_done);
            const uint32_t wk = __ldcg(&P.desc[s].walks);
            const uint32_t S = __ldcg(&P.desc[s].S);
            const int rel = tag_rel(a, id);
            const bool has = rel == 0 && (uint32_t)a < S;
            o = has && wd >= wk && __ldcg(&P.desc[s].R) <= max_R;
            left |= has;
            if (rel < 0) unwritten = (int)i;
            if (i == 0 && (rel > 0 || (rel == 0 && !has))) bump(&P.glob->agg_head, h);
        }
        ready[r] = __ballot_sync(0xffffffffu, o);
    }
    in_flight = __ballot_sync(0xffffffffu, left) != 0;
    const uint32_t um = __ballot_sync(0xffffffffu, unwritten >= 0);
    if (um) {
        const int ui = __shfl_sync(0xffffffffu, unwritten, __ffs(um) - 1);
        int r = 0;
        if (lane == 0) r = await_slot(P, &P.slot[(h + ui) % kRing].agg, h + ui);
        return __shfl_sync(0xffffffffu, r, 0) < 0 ? -1 : 0;
    }
    for (int r = 0; r < 2; ++r) {
        uint32_t m = ready[r];
        while (m) {  // oldest ready query first
            const uint32_t i = r * 32 + __ffs(m) - 1;
            m &= m - 1;
            int got = 0;
            uint32_t src_i = 0, take = 0, slot = 0;
            uint64_t qid = 0;
            if (lane == 0) {
                const uint32_t s = (uint32_t)((h + i) % kRing);
                const SDesc *d = P.desc + s;
                const uint32_t S = __ldcg(&d->S);
                // a batch of sources per claim: a few batches per aggregating warp of the loop
                const uint32_t batch = max(1u, min(32u, S / (4u * (P.walker_warps / (kLoopWarps - 1)))));
                const unsigned long long old = atomicAdd(&P.slot[s].agg, (unsigned long long)batch);
                const uint32_t tag = (uint32_t)(old >> 32), c = (uint32_t)old;
                // the sources are those of the query that holds the slot now (another one if it was reused)
                if (tag != 0 && (uint32_t)__ldcg(&d->seq1) == tag) {
                    const uint32_t S2 = __ldcg(&d->S);
                    if (c < S2) {
                        src_i = c;
                        take = min(batch, S2 - c);
                        slot = s;
                        qid = tag - 1;
                        got = 1;
                        // its walks may still be running if the slot was reused: wait for them (bounded)
                        const uint64_t t0 = gtime_ns();
                        while (__ldcg(&P.slot[s].walks_done) < __ldcg(&d->walks)) {
                            if (gtime_ns() - t0 > kBusyWaitNs) {
                                flag_exit(P, PPR_LOOP_BUSY_TIMEOUT);
                                got = -1;
                                break;
                            }
                            __nanosleep(1000);
                        }
                    }
                }
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            if (got < 0) return -1;
            if (got) {
                id_out = __shfl_sync(0xffffffffu, qid, 0);
                slot_out = __shfl_sync(0xffffffffu, slot, 0);
                i_out = __shfl_sync(0xffffffffu, src_i, 0);
                n_out = __shfl_sync(0xffffffffu, take, 0);
                return 1;
            }
        }
    }
    return 0;
}

// Reduction of source i of query slot s into its top-k row (host memory).
// smem: cap endpoints, then the reduction's scratch (3 * cap words); cap >= R.
__device__ void reduce_source(const LoopParams &P, uint32_t s, uint32_t i, uint32_t *smem, uint32_t cap)
{
    const uint32_t lane = threadIdx.x & 31;
    const SDesc *d = P.desc + s;
    const uint32_t R = __ldcg(&d->R), P2 = __ldcg(&d->P2), topk = __ldcg(&d->topk);
    const uint32_t *ends = reinterpret_cast<const uint32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&d->ends)));
    AggOut o{};
    o.topk_idx = reinterpret_cast<int32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&d->out_idx)));
    o.topk_cnt = reinterpret_cast<uint32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&d->out_cnt)));
    o.topk = (int32_t)topk;
    uint32_t *e = smem;  // the endpoints, read past L1 (the arena is reused by later queries)
    for (uint32_t r = lane; r < R; r += 32) e[r] = caller_id(P.kp.order, __ldcg(ends + (uint64_t)i * R + r));
    __syncwarp();
    uint32_t *scratch = smem + cap;
    switch (P2) {
    case 1: case 2: case 4: case 8: case 16: case 32: aggregate_source_reg<1>(e, R, scratch, o, i); break;
    case 64: aggregate_source_reg<2>(e, R, scratch, o, i); break;
    case 128: aggregate_source_reg<4>(e, R, scratch, o, i); break;
    default: {
        uint64_t *keys = reinterpret_cast<uint64_t *>(scratch);
        aggregate_source(e, R, reinterpret_cast<uint32_t *>(keys + P2), keys, o, i);
    }
    }
}

// After a warp has written source i's row: counts it; the last source of the
// query marks it done for the host.
__device__ void finish_source(const LoopParams &P, uint64_t id, uint32_t s, uint32_t n)
{
    __threadfence_system();  // these rows are in host memory before the count says so
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&P.glob->reduced, (unsigned long long)n);
        const unsigned long long old = atomicAdd(&P.slot[s].agg_done, (unsigned long long)n);
        if (old + n == __ldcg(&P.desc[s].S)) {
            P.slot[s].t_done = gtime_ns();
            __threadfence_system();
            st_release_sys(&P.ctl->done[s], id + 1);
        }
    }
}

__device__ void aggregator_warp(const LoopParams &P, uint32_t *smem, unsigned long long *s_tail)
{
    const uint32_t lane = threadIdx.x & 31;
    uint64_t idle_t0 = 0, busy_t0 = 0;
    uint32_t backoff = 256;
    bool refresh = true;
    for (;;) {
        uint64_t id = 0;
        uint32_t s = 0, i = 0, nb = 0;
        bool in_flight = false;
        const int r = claim_source(P, s_tail, refresh, kLoopMaxR, id, s, i, nb, in_flight);
        if (r < 0) break;
        if (r > 0) {
            for (uint32_t b = 0; b < nb; ++b) reduce_source(P, s, i + b, smem, kLoopMaxR);
            finish_source(P, id, s, nb);
            idle_t0 = busy_t0 = 0;
            backoff = 256;
            refresh = false;
            continue;
        }
        refresh = true;
        const uint64_t t = gtime_ns();
        if (!in_flight) {  // nothing published is left to reduce
            busy_t0 = 0;
            if (ld_volatile(&P.ctl->stop)) {
                if (lane == 0) flag_exit(P, PPR_LOOP_STOPPED);
                break;
            }
            if (idle_t0 == 0) idle_t0 = t;
            else if (t - idle_t0 > P.idle_ns) {
                if (lane == 0) flag_exit(P, PPR_LOOP_IDLE);
                break;
            }
        } else {  // queries whose walks are still running: wait for them (bounded)
            idle_t0 = 0;
            if (busy_t0 == 0) busy_t0 = t;
            else if (t - busy_t0 > kBusyWaitNs) {
                if (lane == 0) flag_exit(P, PPR_LOOP_BUSY_TIMEOUT);
                break;
            }
            if (ld_volatile(&P.ctl->status) & (PPR_LOOP_SLOT_TIMEOUT | PPR_LOOP_BUSY_TIMEOUT)) break;
        }
        __nanosleep(backoff);
        backoff = min(backoff * 2, 4096u);
    }
}

// SPLIT: the narrow layout of a renumbered graph (see search_blocked)
template <class E, bool SPLIT = false>
__global__ void __launch_bounds__(32 * kLoopWarps, 4) k_serve_loop(LoopParams P)
{
    __shared__ WalkChunk wc[kLoopWarps - 1];
    __shared__ uint32_t *ends_of[kRing];  // endpoint array of each slot, set by the warp that takes a chunk of it
    __shared__ __align__(16) uint32_t smem[kLoopMaxR + 3 * kLoopMaxR];  // the aggregator warp's endpoints and scratch
    __shared__ unsigned long long s_tail[2];  // the block's copy of the published tail, and when it was read
    if (threadIdx.x == 0) s_tail[0] = s_tail[1] = 0;
    __syncthreads();
    const uint32_t wid = threadIdx.x >> 5;
    if (wid == kLoopWarps - 1) {
        aggregator_warp(P, smem, s_tail);
        return;
    }
    walker_warp<E, SPLIT>(P, wc[wid], ends_of, blockIdx.x * (kLoopWarps - 1) + wid, s_tail);
}

// ============================================================ queries ====

struct Query {
    uint64_t id = 0;
    std::vector<uint32_t> sources;
    RunPlan plan{};
    int32_t topk = 0;
    size_t bytes = 0;  // device memory while in flight
    enum State { Pending, Running, Done, Failed } state = Pending;
    int status = PPR_OK;
    std::string error;
    std::vector<int32_t> idx;  // stream mode results
    std::vector<uint32_t> cnt;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    uint64_t walks = 0;
    // device loop
    uint64_t seq = 0;
    uint32_t slot = 0;
    size_t dev_off = 0, pin_off = 0, pin_bytes = 0;
    int64_t dev_walk_ns = 0, dev_reduce_ns = 0;
};

// First-fit allocator over one block of bytes (host-side bookkeeping).
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t &off)
    {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<size_t, size_t> free_;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

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
    std::deque<std::shared_ptr<Query>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Query>> table;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::atomic<bool> stop{false};
    std::thread worker;
    uint64_t next_id = 1;
    uint64_t completed = 0;
    // stream mode
    std::vector<Slot> slots;
    // device loop
    cudaStream_t loop_stream = nullptr, ctl_stream = nullptr;
    cudaEvent_t loop_done = nullptr;
    SCtl *ctl = nullptr, *ctl_dev = nullptr;  // host-mapped
    SDesc *d_desc = nullptr, *h_desc = nullptr;
    SSlot *d_slot = nullptr, *h_slot = nullptr;
    SGlob *d_glob = nullptr;
    unsigned char *arena = nullptr;  // device
    unsigned char *pin = nullptr;    // pinned, mapped
    size_t pin_size = 0;
    Arena dev_arena, pin_arena;      // guarded by mu
    std::shared_ptr<Query> ring[kRing];
    uint64_t published = 0;  // queries published so far (= the next sequence number)
    bool loop_running = false, failed = false;
    int64_t launches = 0, idle_exits = 0, in_flight = 0;
    uint32_t last_status = 0;
    uint32_t grid = 0;
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

// device loop: a query's device bytes (sources, endpoints) and pinned bytes (sources staged, top-k out)
static size_t loop_dev_bytes(int64_t S, uint32_t R) { return align256(4 * (size_t)S) + align256(4 * (size_t)S * R); }
static size_t loop_pin_bytes(int64_t S, int32_t k) { return align256(4 * (size_t)S) + 2 * align256(4 * (size_t)S * k); }

// ---------------------------------------------------------- stream mode ----

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

static void scheduler_streams(Server *sv)
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

// ---------------------------------------------------------- device loop ----

template <class E, bool SPLIT = false>
static int launch_loop_typed(Server *sv)
{
    const ppr_graph *g = sv->g;
    LoopParams P{};
    P.kp.node = sv->cfg.sampler == 1 ? (const void *)g->alias.node : g->node;
    P.kp.edges = sv->cfg.sampler == 1 ? (const void *)g->alias.slots : g->edges;
    P.kp.large = 0xffffffffu;
    P.kp.n_nodes = g->n;
    P.kp.rank = g->rank;
    P.kp.order = g->order;
    P.kp.n_records = sv->cfg.sampler == 1 ? (uint64_t)g->m : (uint64_t)g->edge_records;
    P.kp.sum = g->sum_base();
    P.kp.n_sum = g->sum_extent();
    P.kp.err = &sv->d_glob->err;
    P.desc = sv->d_desc;
    P.slot = sv->d_slot;
    P.ctl = sv->ctl_dev;
    P.glob = sv->d_glob;
    P.refill = sv->cfg.refill_lanes > 0 ? (uint32_t)std::min(sv->cfg.refill_lanes, 32) : 1u;
    P.idle_ns = (uint64_t)(sv->cfg.idle_us > 0 ? sv->cfg.idle_us : 200000) * 1000ull;
    if (!sv->grid) {
        int per_sm = 0;
        PPR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve_loop<E, SPLIT>, 32 * kLoopWarps, 0));
        sv->grid = (uint32_t)(sv->ctx->sms * std::max(per_sm, 1));
    }
    P.walker_warps = sv->grid * (kLoopWarps - 1);
    k_serve_loop<E, SPLIT><<<sv->grid, 32 * kLoopWarps, 0, sv->loop_stream>>>(P);
    note_launch();
    PPR_CUDA(cudaGetLastError());
    PPR_CUDA(cudaEventRecord(sv->loop_done, sv->loop_stream));
    return PPR_OK;
}

static int launch_loop(Server *sv)
{
    __atomic_store_n(&sv->ctl->status, 0u, __ATOMIC_RELEASE);
    int rc;
    if (sv->cfg.sampler == 1) rc = launch_loop_typed<AliasEdges>(sv);
    else if (sv->g->wide) rc = launch_loop_typed<WideEdges>(sv);
    else if (sv->g->sum) rc = launch_loop_typed<NarrowEdges, true>(sv);
    else rc = launch_loop_typed<NarrowEdges>(sv);
    if (rc == PPR_OK) {
        sv->loop_running = true;
        ++sv->launches;
    }
    return rc;
}

// Marks query q finished (lock held).
static void loop_finish(Server *sv, const std::shared_ptr<Query> &q, int status, const char *err)
{
    if (status == PPR_OK) {  // the device's own times of the query (its slot is not reused before this)
        SSlot c;
        if (cudaMemcpyAsync(&c, sv->d_slot + q->slot, sizeof(c), cudaMemcpyDeviceToHost, sv->ctl_stream) ==
                cudaSuccess &&
            cudaStreamSynchronize(sv->ctl_stream) == cudaSuccess) {
            q->dev_walk_ns = (int64_t)(c.t_walks - c.t_claim);
            q->dev_reduce_ns = (int64_t)(c.t_done - c.t_walks);
        }
        cudaGetLastError();
    }
    sv->dev_arena.release(q->dev_off, loop_dev_bytes((int64_t)q->sources.size(), q->plan.R));
    sv->ring[q->slot].reset();
    --sv->in_flight;
    q->t_done = now_ns();
    q->status = status;
    q->state = status == PPR_OK ? Query::Done : Query::Failed;
    if (status != PPR_OK) {
        q->error = err;
        sv->pin_arena.release(q->pin_off, q->pin_bytes);  // nothing to read back
        q->pin_bytes = 0;
    }
    ++sv->completed;
}

static void scheduler_loop(Server *sv)
{
    cudaSetDevice(sv->ctx->device);
    std::vector<std::shared_ptr<Query>> batch;
    for (;;) {
        bool progress = false;
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            // finished queries: their top-k rows are in pinned memory
            for (int s = 0; s < kRing; ++s) {
                const std::shared_ptr<Query> q = sv->ring[s];
                if (q && __atomic_load_n(&sv->ctl->done[s], __ATOMIC_ACQUIRE) == q->seq + 1) {
                    loop_finish(sv, q, PPR_OK, "");
                    progress = true;
                }
            }
            // the loop kernel ended: on its idle bound, or on an error
            if (sv->loop_running && cudaEventQuery(sv->loop_done) != cudaErrorNotReady) {
                sv->loop_running = false;
                const cudaError_t e = cudaEventQuery(sv->loop_done);
                sv->last_status = __atomic_load_n(&sv->ctl->status, __ATOMIC_ACQUIRE);
                if (sv->last_status & PPR_LOOP_IDLE) ++sv->idle_exits;
                if (e != cudaSuccess || (sv->last_status & (PPR_LOOP_SLOT_TIMEOUT | PPR_LOOP_BUSY_TIMEOUT))) {
                    sv->failed = true;
                    const char *why = e != cudaSuccess ? cudaGetErrorString(e)
                                      : (sv->last_status & PPR_LOOP_SLOT_TIMEOUT)
                                          ? "serving loop ended: a published ring slot was never written"
                                          : "serving loop ended: walks in flight did not finish in time";
                    for (int s = 0; s < kRing; ++s)
                        if (sv->ring[s]) loop_finish(sv, sv->ring[s], PPR_ECUDA, why);
                }
                progress = true;
            }
            // admit in arrival order while a ring slot and both arenas allow
            batch.clear();
            while (!sv->failed && !sv->pending.empty()) {
                const std::shared_ptr<Query> f = sv->pending.front();
                const uint32_t s = (uint32_t)(sv->published + batch.size()) % kRing;
                if (sv->ring[s]) break;
                const int64_t S = (int64_t)f->sources.size();
                size_t doff, poff;
                if (!sv->dev_arena.alloc(loop_dev_bytes(S, f->plan.R), doff)) break;  // wait for memory
                f->pin_bytes = loop_pin_bytes(S, f->topk);
                if (!sv->pin_arena.alloc(f->pin_bytes, poff)) {
                    sv->dev_arena.release(doff, loop_dev_bytes(S, f->plan.R));
                    break;
                }
                sv->pending.pop_front();
                f->dev_off = doff;
                f->pin_off = poff;
                f->slot = s;
                f->seq = sv->published + batch.size();
                sv->ring[s] = f;
                batch.push_back(f);
            }
        }
        if (!batch.empty()) {
            cudaError_t e = cudaSuccess;
            for (const auto &f : batch) {
                const int64_t S = (int64_t)f->sources.size();
                const uint32_t R = f->plan.R, k = (uint32_t)f->topk, s = f->slot;
                unsigned char *pin = sv->pin + f->pin_off;
                unsigned char *dev = sv->arena + f->dev_off;
                std::memcpy(pin, f->sources.data(), 4 * (size_t)S);
                SDesc &d = sv->h_desc[s];
                d.src = reinterpret_cast<const uint32_t *>(dev);
                d.ends = reinterpret_cast<uint32_t *>(dev + align256(4 * (size_t)S));
                int32_t *oi = reinterpret_cast<int32_t *>(pin + align256(4 * (size_t)S));
                uint32_t *oc = reinterpret_cast<uint32_t *>(pin + align256(4 * (size_t)S) + align256(4 * (size_t)S * k));
                void *oi_d = nullptr, *oc_d = nullptr;
                if (e == cudaSuccess) e = cudaHostGetDevicePointer(&oi_d, oi, 0);
                if (e == cudaSuccess) e = cudaHostGetDevicePointer(&oc_d, oc, 0);
                d.out_idx = static_cast<int32_t *>(oi_d);
                d.out_cnt = static_cast<uint32_t *>(oc_d);
                d.r_magic = ((1ull << 40) + R - 1) / R;
                d.seq1 = f->seq + 1;
                d.S = (uint32_t)S;
                d.R = R;
                d.T = f->plan.T;
                d.k0 = (uint32_t)f->plan.seed;
                d.k1 = (uint32_t)(f->plan.seed >> 32);
                d.topk = k;
                d.walks = (uint32_t)(S * R);
                uint32_t P2 = 1;
                while (P2 < R) P2 <<= 1;
                d.P2 = P2;
                // walks per chunk: about four chunks per walker warp for a large query
                const uint64_t ww = std::max<uint64_t>(1, 4ull * sv->grid * (kLoopWarps - 1));
                uint64_t cw = sv->cfg.chunk_sources > 0 ? (uint64_t)sv->cfg.chunk_sources * R : (d.walks + ww - 1) / ww;
                cw = std::min<uint64_t>(std::max<uint64_t>(cw, 32), 4096);
                d.cw = (uint32_t)cw;
                d.nchunks = (uint32_t)((d.walks + cw - 1) / cw);
                SSlot &c = sv->h_slot[s];
                const unsigned long long tag = (unsigned long long)(uint32_t)(f->seq + 1) << 32;
                c.claim = tag;  // chunks handed out so far (counts up)
                c.agg = tag;    // sources handed out so far (counts up)
                c.walks_done = 0;
                c.agg_done = 0;
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync((void *)d.src, pin, 4 * (size_t)S, cudaMemcpyHostToDevice, sv->ctl_stream);
                // the descriptor first: a warp whose claim lands on the new counters finds it in place
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(sv->d_desc + s, &d, sizeof(SDesc), cudaMemcpyHostToDevice, sv->ctl_stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(sv->d_slot + s, &c, sizeof(SSlot), cudaMemcpyHostToDevice, sv->ctl_stream);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(sv->ctl_stream);
            std::lock_guard<std::mutex> lock(sv->mu);
            if (e != cudaSuccess) {
                const int code = cuda_fail(e, "query upload");
                sv->failed = true;
                for (const auto &f : batch) loop_finish(sv, f, code, "query upload failed");
            } else {
                const int64_t t = now_ns();
                for (const auto &f : batch) {
                    f->state = Query::Running;
                    f->t_admit = t;
                    ++sv->in_flight;
                }
                sv->published += batch.size();
                __atomic_store_n(&sv->ctl->tail, (unsigned long long)sv->published, __ATOMIC_RELEASE);
            }
            progress = true;
        }
        std::unique_lock<std::mutex> lock(sv->mu);
        if (progress) sv->cv_done.notify_all();
        // the loop runs while queries are in flight (launched again after an idle exit)
        if (!sv->loop_running && !sv->failed && sv->in_flight > 0) {
            if (launch_loop(sv) != PPR_OK) {
                sv->failed = true;
                for (int s = 0; s < kRing; ++s)
                    if (sv->ring[s]) loop_finish(sv, sv->ring[s], PPR_ECUDA, "serving loop launch failed");
                sv->cv_done.notify_all();
            }
        }
        if (sv->stop && sv->pending.empty() && sv->in_flight == 0) break;
        if (sv->in_flight > 0 || !sv->pending.empty()) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(10));
        } else {
            sv->cv_work.wait_for(lock, std::chrono::milliseconds(2));
        }
    }
}

static void free_loop(Server *sv)
{
    if (sv->loop_stream) {
        // the loop ends on its stop flag once idle (bounded); wait for it
        __atomic_store_n(&sv->ctl->stop, 1u, __ATOMIC_RELEASE);
        cudaStreamSynchronize(sv->loop_stream);
    }
    if (sv->ctl_stream) cudaStreamSynchronize(sv->ctl_stream);
    cudaFree(sv->arena);
    cudaFree(sv->d_desc);
    cudaFree(sv->d_slot);
    cudaFree(sv->d_glob);
    if (sv->pin) cudaFreeHost(sv->pin);
    if (sv->ctl) cudaFreeHost(sv->ctl);
    if (sv->h_desc) cudaFreeHost(sv->h_desc);
    if (sv->h_slot) cudaFreeHost(sv->h_slot);
    if (sv->loop_done) cudaEventDestroy(sv->loop_done);
    if (sv->loop_stream) cudaStreamDestroy(sv->loop_stream);
    if (sv->ctl_stream) cudaStreamDestroy(sv->ctl_stream);
    cudaGetLastError();
}

static int start_loop(Server *sv)
{
    const ppr_serve_cfg &cfg = sv->cfg;
    cudaError_t e = cudaStreamCreateWithFlags(&sv->loop_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->ctl_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->loop_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->ctl, sizeof(SCtl), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&sv->ctl_dev, sv->ctl, 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->h_desc, sizeof(SDesc) * kRing, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->h_slot, sizeof(SSlot) * kRing, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sv->d_desc, sizeof(SDesc) * kRing);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sv->d_slot, sizeof(SSlot) * kRing);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sv->d_glob, sizeof(SGlob));
    if (e == cudaSuccess) e = cudaMalloc((void **)&sv->arena, sv->budget);
    // pinned output: room for several of the largest queries
    sv->pin_size = std::max<size_t>(64ull << 20, 4 * loop_pin_bytes(cfg.max_sources, cfg.max_topk));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->pin, sv->pin_size, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->d_desc, 0, sizeof(SDesc) * kRing, sv->ctl_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->d_slot, 0, sizeof(SSlot) * kRing, sv->ctl_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->d_glob, 0, sizeof(SGlob), sv->ctl_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->ctl_stream);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "serving set-up");
        free_loop(sv);
        return rc == PPR_ECUDA && e == cudaErrorMemoryAllocation ? PPR_ENOMEM : rc;
    }
    std::memset(sv->ctl, 0, sizeof(SCtl));
    std::memset(sv->h_desc, 0, sizeof(SDesc) * kRing);
    sv->dev_arena.reset(sv->budget);
    sv->pin_arena.reset(sv->pin_size);
    // the resident loop starts now (so the first query needs no launch)
    int rc = launch_loop(sv);
    if (rc) {
        free_loop(sv);
        return rc;
    }
    return PPR_OK;
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
    c->mode = PPR_SERVE_DEVICE_LOOP;
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
    if (cfg.streams < 1 || cfg.streams > 64 || cfg.max_sources < 1 || cfg.max_sources > (1 << 22) ||
        cfg.memory_budget < 0 || cfg.max_pending < 0 || cfg.max_topk < 0 || cfg.max_topk > (int32_t)PPR_MAX_R ||
        (cfg.sampler != 0 && cfg.sampler != 1) || cfg.refill_lanes < 0 || cfg.refill_lanes > 32 ||
        (cfg.mode != PPR_SERVE_DEVICE_LOOP && cfg.mode != PPR_SERVE_STREAMS) || cfg.idle_us < 0 ||
        cfg.chunk_sources < 0) {
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
    if (g->stream) {  // the graph (and its tables) are built before the loop reads them
        e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "graph build");
    }
    Server *sv = new (std::nothrow) Server;
    if (!sv) return PPR_ENOMEM;
    sv->ctx = ctx;
    sv->g = g;
    sv->cfg = cfg;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    sv->budget = cfg.memory_budget > 0 ? (size_t)cfg.memory_budget : free_b / 4;
    if (cfg.mode == PPR_SERVE_DEVICE_LOOP) {
        const int rc = start_loop(sv);
        if (rc) {
            delete sv;
            return rc;
        }
        sv->worker = std::thread(scheduler_loop, sv);
    } else {
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
        sv->worker = std::thread(scheduler_streams, sv);
    }
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
    int rc = PPR_OK;
    if (sv->cfg.mode == PPR_SERVE_DEVICE_LOOP) {
        if (sv->failed) {
            set_error("serving loop failed (exit status 0x%x)", sv->last_status);
            rc = PPR_ECUDA;
        }
        free_loop(sv);
    } else {
        for (Slot &s : sv->slots) {
            cudaStreamSynchronize(s.stream);
            cudaStreamDestroy(s.stream);
            cudaEventDestroy(s.done);
            cudaFreeHost(s.pin);
        }
    }
    ctx->server = nullptr;
    delete sv;
    return rc;
}

int ppr_serve_get_info(ppr_ctx *ctx, ppr_serve_info *info)
{
    if (!ctx || !info || !ctx->server) {
        set_error("serving not started");
        return PPR_EINVAL;
    }
    Server *sv = ctx->server;
    std::lock_guard<std::mutex> lock(sv->mu);
    std::memset(info, 0, sizeof(*info));
    info->mode = sv->cfg.mode;
    info->status = sv->loop_running ? __atomic_load_n(&sv->ctl->status, __ATOMIC_ACQUIRE) : sv->last_status;
    info->launches = sv->launches;
    info->idle_exits = sv->idle_exits;
    info->in_flight = sv->in_flight;
    info->completed = (int64_t)sv->completed;
    info->running = sv->loop_running ? 1 : 0;
    if (sv->cfg.mode == PPR_SERVE_DEVICE_LOOP) {
        SGlob gl;
        cudaError_t e = cudaMemcpyAsync(&gl, sv->d_glob, sizeof(gl), cudaMemcpyDeviceToHost, sv->ctl_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sv->ctl_stream);
        if (e != cudaSuccess) return cuda_fail(e, "serving counters");
        info->draws = gl.draws;
        info->iterations = gl.iterations;
        info->claims = gl.claims;
        info->claim_misses = gl.claim_misses;
        info->sleeps = gl.sleeps;
        info->reduced = gl.reduced;
        info->cycles_claim = gl.cyc_claim;
        info->cycles_step = gl.cyc_step;
        info->cycles_sleep = gl.cyc_sleep;
        info->cycles_total = gl.cyc_total;
        info->grid_blocks = (int32_t)sv->grid;
    }
    return PPR_OK;
}

int ppr_debug_serve_publish_unwritten(ppr_ctx *ctx)
{
    if (!ctx || !ctx->server || ctx->server->cfg.mode != PPR_SERVE_DEVICE_LOOP) {
        set_error("device-loop serving not started");
        return PPR_EINVAL;
    }
    Server *sv = ctx->server;
    std::lock_guard<std::mutex> lock(sv->mu);
    // the sequence number is used up without a descriptor, a query or a ring entry
    sv->published += 1;
    __atomic_store_n(&sv->ctl->tail, (unsigned long long)sv->published, __ATOMIC_RELEASE);
    if (!sv->loop_running && !sv->failed) {
        const int rc = launch_loop(sv);
        if (rc) return rc;
    }
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
    const bool loop = sv->cfg.mode == PPR_SERVE_DEVICE_LOOP;
    if (loop && (R > kLoopMaxR || (uint64_t)ns * R * R >= (1ull << 40))) {
        // walk g of a query maps to (g / R, g % R) by a multiply-shift exact for g < 2^40 / R
        set_error("the serving loop takes R <= %u and sources * R^2 < 2^40 (R = %u, %lld sources); the stream "
                  "mode takes any R", kLoopMaxR, R, (long long)ns);
        return PPR_ERANGE;
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
    q->plan.step_loads = kDefaultStepLoads;
    q->topk = topk;
    const uint32_t cap = (uint32_t)std::min<int64_t>((int64_t)R, sv->g->n);
    q->bytes = loop ? loop_dev_bytes(ns, R) : query_bytes(sv->g, q->plan, ns, topk, cap);
    q->walks = (uint64_t)ns * R;
    q->t_submit = now_ns();
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) {
        set_error("serving is stopping");
        return PPR_EBUSY;
    }
    if (sv->failed) {
        set_error("the serving loop failed (exit status 0x%x); stop and start serving again", sv->last_status);
        return PPR_ECUDA;
    }
    if (q->bytes > sv->budget || (loop && loop_pin_bytes(ns, topk) > sv->pin_size)) {
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
        stats->device_walk_ns = q->dev_walk_ns;
        stats->device_reduce_ns = q->dev_reduce_ns;
    }
    if (q->state == Query::Failed) {
        set_error("%s", q->error.c_str());
        sv->table.erase(it);
        return q->status != PPR_OK ? q->status : PPR_ECUDA;
    }
    const size_t n = q->sources.size() * (size_t)q->topk;
    if (sv->cfg.mode == PPR_SERVE_DEVICE_LOOP) {
        const int64_t S = (int64_t)q->sources.size();
        const unsigned char *pin = sv->pin + q->pin_off;
        if (idx) std::memcpy(idx, pin + align256(4 * (size_t)S), 4 * n);
        if (cnt) std::memcpy(cnt, pin + align256(4 * (size_t)S) + align256(4 * n), 4 * n);
        sv->pin_arena.release(q->pin_off, q->pin_bytes);
        q->pin_bytes = 0;
    } else {
        if (idx) std::memcpy(idx, q->idx.data(), sizeof(int32_t) * n);
        if (cnt) std::memcpy(cnt, q->cnt.data(), sizeof(uint32_t) * n);
    }
    sv->table.erase(it);
    return PPR_OK;
}

}  // extern "C"
