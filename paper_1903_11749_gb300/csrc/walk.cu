// walk.cu -- the walker kernels.
//
// One step (Sec. 2.1, Algorithm 2): draw Philox4x32-10 at counter
// (s_local, j, k, tag); at a node with out-edges take the first edge whose
// inclusive weight prefix exceeds floor(r64 * W_u / 2^64) and move to its
// target; at a node without out-edges restart at the source (or end the walk,
// dangling mode 1); then stop iff x2 < T.  At a node carrying a segment table
// (Algorithm 4, depth 3) the same draw selects one outcome: a terminated
// outcome ends the walk, an active one moves the walk and advances k by the
// outcome's length.
//
// k_walk_plain:      one thread per walk, endpoint to HBM (baseline), then
// k_aggregate:       one warp per source sorts its R endpoints into a row.
// k_walk_persistent: persistent warps pull source chunks from a global queue,
//                    refill lanes as walks end (the paper's pipelines keep
//                    the cluster busy the same way), search large rows with the
//                    whole warp, and aggregate a chunk in shared memory as soon
//                    as its last walk ends.
#include <algorithm>

#include "ppr_host.h"

namespace ppr {

struct KParams {
    const NodeRec *node;
    const void *edges;
    const SegEntry *seg;
    uint32_t k0, k1, T, R, tag;
    int32_t dangling;
    uint32_t large;
    int64_t s_begin, s_end;   // sources of this launch (global ids)
    int64_t out_row0;         // output row of s_begin
    uint32_t CS;              // sources per chunk
    uint32_t nchunks;
    const int4 *chunks;       // batched graphs: {base, nsrc, instance, 0}; else null
    const int64_t *inst_off;  // batched graphs: node_off
    AggOut out;
    uint32_t *ends;           // plain kernel: S * R endpoints
    unsigned long long *queue;
    unsigned long long *steps;    // [0] draws consumed, [2] algorithmic sectors (statistics launch)
    uint32_t slot_cap;        // walks per chunk slot (CS * R)
    uint32_t P2;              // next_pow2(R)
};

// One step of one walk.  Returns true when the walk has ended (end is set).
// With COOP, every lane of the warp calls it (inactive lanes with act=false)
// and rows longer than p.large are searched by the whole warp.
struct Tally {
    uint32_t steps = 0;
    uint32_t sectors = 0;
};

// STATS: count, per step, the 32-byte sectors a thread-serial bisection must
// touch (node record + distinct probe sectors); rows are then searched by
// bisection only, which returns the same edge as the cooperative search.
template <class E, bool SEG, bool COOP, bool STATS>
__device__ __forceinline__ bool walk_step(const KParams &p, const E &edges, bool act, uint32_t src, uint32_t sctr,
                                          uint32_t j, uint32_t tag, uint32_t &k, uint32_t &u, uint32_t &end,
                                          Tally &tl)
{
    uint4 x = make_uint4(0, 0, 0, 0);
    uint64_t w0 = 0, total = 0;
    if (act) {
        x = philox4x32_10(make_uint4(sctr, j, k, tag), p.k0, p.k1);
        NodeRec r = load_node(p.node, u);
        w0 = r.word0;
        total = r.total;
    }
    const uint32_t cnt = (uint32_t)(w0 >> 40) & kCountMask;
    const uint64_t beg = w0 & kBeginMask;
    const bool segf = SEG && (w0 >> 63);
    const uint64_t r64 = (uint64_t)x.x | ((uint64_t)x.y << 32);
    uint64_t xr = 0;
    if (act && (cnt > 1 || segf)) {
        if (segf || total >= (1ull << 32)) xr = mulhi64(r64, total);
        else xr = mulhi64_by32(x.x, x.y, (uint32_t)total);
    }
    uint32_t next = 0;
    bool big = false;
    if (COOP && !STATS) {
        big = act && !segf && cnt > p.large;
        uint32_t bigmask = __ballot_sync(0xffffffffu, big);
        const uint32_t lane = threadIdx.x & 31;
        while (bigmask) {
            const uint32_t L = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            const uint64_t lo = __shfl_sync(0xffffffffu, beg, L);
            const uint32_t n = __shfl_sync(0xffffffffu, cnt, L);
            const uint64_t xx = __shfl_sync(0xffffffffu, xr, L);
            auto rec = search_warp(edges, lo, n, xx);
            if (lane == L) next = E::target(rec);
        }
    }
    if (!act) return false;
    if (STATS) ++tl.sectors;  // the node record
    if (segf) {
        SegTable tab{p.seg};
        uint4 o = STATS ? search_serial_tally(tab, beg, cnt, xr, tl.sectors) : search_serial(tab, beg, cnt, xr);
        ++tl.steps;
        if ((o.w >> 8) == 0) {
            end = o.z;
            return true;
        }
        u = o.z;
        k += o.w & 0xffu;
        return false;
    }
    if (cnt == 0) {
        if (p.dangling == 1) {
            end = u;
            return true;
        }
        next = src;
    } else if (cnt == 1) {
        next = (uint32_t)total;  // single out-edge: target kept in the node record
    } else if (!big) {
        next = E::target(STATS ? search_serial_tally(edges, beg, cnt, xr, tl.sectors) : search_serial(edges, beg, cnt, xr));
    }
    ++tl.steps;
    ++k;
    u = next;
    if (x.z < p.T) {
        end = u;
        return true;
    }
    return false;
}

template <class E>
__device__ __forceinline__ E make_edges(const void *e);
template <>
__device__ __forceinline__ NarrowEdges make_edges<NarrowEdges>(const void *e)
{
    return NarrowEdges{(const EdgeN *)e};
}
template <>
__device__ __forceinline__ WideEdges make_edges<WideEdges>(const void *e)
{
    return WideEdges{(const EdgeW *)e};
}

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
    if (STATS) warp_add(dst + 2, t.sectors);
}

// ------------------------------------------------------------ plain (K4) ----
template <class E, bool SEG, bool STATS>
__global__ void __launch_bounds__(256) k_walk_plain(KParams p)
{
    const E edges = make_edges<E>(p.edges);
    const uint64_t S = (uint64_t)(p.s_end - p.s_begin);
    const uint64_t total = S * p.R;
    Tally tl;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = t / p.R;
        const uint32_t j = (uint32_t)(t - i * p.R);
        const uint32_t src = (uint32_t)(p.s_begin + (int64_t)i);
        uint32_t k = 0, u = src, end = 0;
        while (!walk_step<E, SEG, false, STATS>(p, edges, true, src, src, j, p.tag, k, u, end, tl)) {
        }
        p.ends[t] = end;
    }
    warp_add_tally<STATS>(p.steps, tl);
}

__global__ void __launch_bounds__(128) k_aggregate(KParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t *keys = reinterpret_cast<uint64_t *>(smem_raw) + (size_t)wid * p.P2;
    uint32_t *sortbuf = reinterpret_cast<uint32_t *>(reinterpret_cast<uint64_t *>(smem_raw) + (size_t)nw * p.P2) +
                        (size_t)wid * p.P2;
    const uint64_t S = (uint64_t)(p.s_end - p.s_begin);
    for (uint64_t i = (uint64_t)blockIdx.x * nw + wid; i < S; i += (uint64_t)gridDim.x * nw)
        aggregate_source(p.ends + i * p.R, p.R, sortbuf, keys, p.out, (uint64_t)p.out_row0 + i);
}

// ------------------------------------------------------- persistent (K5) ----
// Every lane runs its own walk as a small state machine that issues at most
// one 16-byte load per loop iteration:
//   NODE   load the node record of the tail u (the step's Philox draw is
//          computed while the load is in flight);
//   SEARCH one bisection probe of the row prefix (or of the segment table);
//   FINAL  load the chosen record when the last probe did not bring it.
// Lanes in different phases share each load instruction, so a lane deep in a
// long bisection does not hold back the others (a lockstep step would wait
// for the longest search of the warp every step).  Rows longer than
// p.large are searched by the whole warp (search_warp) at the start of an
// iteration.  Lanes that finish a walk are refilled from the warp's current
// chunk; a chunk's R-endpoint blocks are aggregated in shared memory as soon
// as its last walk ends, while the next chunk's walks are already running.
struct SlotState {
    uint32_t base, nsrc, total, issued, done, ctr_base, tag, live;
};

enum : uint32_t { kIdle = 0, kNode = 1, kSearch = 2, kFinal = 3, kCoop = 4, kResolved = 5 };

template <class E>
__device__ __forceinline__ const uint4 *block_of(const void *base, uint64_t idx)
{
    // 16-byte aligned block holding record idx
    return reinterpret_cast<const uint4 *>(base) + ((idx * sizeof(typename E::Rec)) >> 4);
}

template <class E>
__device__ __forceinline__ void rec_in_block(uint4 v, uint64_t idx, uint64_t &key, uint32_t &tgt, uint32_t &aux)
{
    if constexpr (sizeof(typename E::Rec) == 8) {
        const bool hi = (idx & 1) != 0;
        key = hi ? v.z : v.x;
        tgt = hi ? v.w : v.y;
        aux = 0;
    } else {
        key = (uint64_t)v.x | ((uint64_t)v.y << 32);
        tgt = v.z;
        aux = v.w;
    }
}

#ifndef PPR_WALK_MINB
#define PPR_WALK_MINB 1  // minimum resident 256-thread blocks per SM requested from ptxas
#endif

template <class E, bool SEG, bool STATS>
__global__ void __launch_bounds__(256, PPR_WALK_MINB) k_walk_persistent(KParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // per-warp shared memory: keys[P2] u64 | sortbuf[P2] u32 | slot ends [2][slot_cap] u32 | SlotState[2]
    const size_t per_warp = (size_t)p.P2 * 12 + (size_t)p.slot_cap * 8 + sizeof(SlotState) * 2;
    const size_t per_warp_al = (per_warp + 15) & ~(size_t)15;
    unsigned char *mine = smem_raw + per_warp_al * wid;
    uint64_t *keys = reinterpret_cast<uint64_t *>(mine);
    uint32_t *sortbuf = reinterpret_cast<uint32_t *>(mine + (size_t)p.P2 * 8);
    uint32_t *slot_ends = sortbuf + p.P2;
    SlotState *ss = reinterpret_cast<SlotState *>(slot_ends + 2 * (size_t)p.slot_cap);
    const E edges = make_edges<E>(p.edges);

    if (lane < 2) ss[lane].live = 0;
    __syncwarp();
    int cur = -1;
    bool queue_empty = false;
    uint32_t phase = kIdle;
    uint32_t slot = 0, widx = 0, src = 0, j = 0, k = 0, u = 0;
    uint32_t n = 0, x2 = 0;
    uint64_t lo = 0, x = 0;
    bool segw = false;
    Tally tl;
    uint64_t last_sec = ~0ull;  // statistics only

    for (;;) {
        // ---- refill idle lanes from the issuing slot, opening chunks as needed
        uint32_t idle = __ballot_sync(0xffffffffu, phase == kIdle);
        while (idle) {
            if (cur < 0 || ss[cur].issued == ss[cur].total) {
                if (queue_empty) break;
                const int fresh = cur < 0 ? 0 : (cur ^ 1);
                if (ss[fresh].live) break;  // older chunk still has walks in flight
                unsigned long long c = 0;
                if (lane == 0) c = atomicAdd(p.queue, 1ull);
                c = __shfl_sync(0xffffffffu, c, 0);
                if (c >= p.nchunks) {
                    queue_empty = true;
                    break;
                }
                if (lane == 0) {
                    SlotState s;
                    if (p.chunks) {
                        int4 d = p.chunks[c];
                        s.base = (uint32_t)d.x;
                        s.nsrc = (uint32_t)d.y;
                        s.ctr_base = (uint32_t)p.inst_off[d.z];
                        s.tag = (uint32_t)d.z;
                    } else {
                        int64_t b = p.s_begin + (int64_t)c * p.CS;
                        s.base = (uint32_t)b;
                        s.nsrc = (uint32_t)std::min<int64_t>((int64_t)p.CS, p.s_end - b);
                        s.ctr_base = 0;
                        s.tag = p.tag;
                    }
                    s.total = s.nsrc * p.R;
                    s.issued = 0;
                    s.done = 0;
                    s.live = 1;
                    ss[fresh] = s;
                }
                __syncwarp();
                cur = fresh;
            }
            const uint32_t issued = ss[cur].issued, total = ss[cur].total, base = ss[cur].base;
            const uint32_t take = min(total - issued, (uint32_t)__popc(idle));
            const uint32_t rank = __popc(idle & ((1u << lane) - 1));
            if (((idle >> lane) & 1) && rank < take) {
                widx = issued + rank;
                slot = (uint32_t)cur;
                const uint32_t i = widx / p.R;
                j = widx - i * p.R;
                src = base + i;
                k = 0;
                u = src;
                phase = kNode;
            }
            __syncwarp();
            if (lane == 0) ss[cur].issued = issued + take;
            __syncwarp();
            idle = __ballot_sync(0xffffffffu, phase == kIdle);
        }
        const uint32_t act_mask = __ballot_sync(0xffffffffu, phase != kIdle);
        if (act_mask == 0) {
            if (queue_empty && !ss[0].live && !ss[1].live) break;
        }

        // ---- rows above the cooperative threshold: searched by the whole warp
        if (!STATS) {
            uint32_t cm = __ballot_sync(0xffffffffu, phase == kCoop);
            while (cm) {
                const uint32_t L = __ffs(cm) - 1;
                cm &= cm - 1;
                const uint64_t l0 = __shfl_sync(0xffffffffu, lo, L);
                const uint32_t n0 = __shfl_sync(0xffffffffu, n, L);
                const uint64_t xx = __shfl_sync(0xffffffffu, x, L);
                auto rec = search_warp(edges, l0, n0, xx);
                if (lane == L) {
                    u = E::target(rec);  // the chosen edge's target; the step completes below
                    phase = kResolved;
                }
            }
        }

        // ---- one load per active lane
        uint64_t aidx = 0;
        if (phase == kNode) {
            aidx = u;
        } else if (phase == kSearch) {
            aidx = lo + (n >> 1) - 1;
        } else if (phase == kFinal) {
            aidx = lo;
        }
        const bool loads = phase == kNode || phase == kSearch || phase == kFinal;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (loads) {
            const uint4 *addr;
            if (phase == kNode) addr = reinterpret_cast<const uint4 *>(p.node) + aidx;
            else if (SEG && segw) addr = reinterpret_cast<const uint4 *>(p.seg) + aidx;
            else addr = block_of<E>(p.edges, aidx);
            v = __ldg(addr);
        }

        // Philox of the step a lane starts, overlapping the node-record load
        uint4 rnd = make_uint4(0, 0, 0, 0);
        if (phase == kNode) rnd = philox4x32_10(make_uint4(src - ss[slot].ctr_base, j, k, ss[slot].tag), p.k0, p.k1);

        bool step_done = false, fin = false;
        uint32_t next = 0, end = 0;
        if (phase == kNode) {
            const uint64_t w0 = (uint64_t)v.x | ((uint64_t)v.y << 32);
            const uint64_t total = (uint64_t)v.z | ((uint64_t)v.w << 32);
            const uint32_t cnt = (uint32_t)(w0 >> 40) & kCountMask;
            const bool segf = SEG && (w0 >> 63);
            x2 = rnd.z;
            if (STATS) {
                ++tl.sectors;
                last_sec = ~0ull;
            }
            if (cnt == 0) {
                if (p.dangling == 1) {
                    fin = true;
                    end = u;
                } else {
                    next = src;
                    step_done = true;
                }
            } else if (cnt == 1 && !segf) {
                next = (uint32_t)total;
                step_done = true;
            } else {
                const uint64_t r64 = (uint64_t)rnd.x | ((uint64_t)rnd.y << 32);
                x = (segf || total >= (1ull << 32)) ? mulhi64(r64, total) : mulhi64_by32(rnd.x, rnd.y, (uint32_t)total);
                lo = w0 & kBeginMask;
                n = cnt;
                segw = segf;
                phase = (!STATS && !segf && cnt > p.large) ? kCoop : (n > 1 ? kSearch : kFinal);
            }
        } else if (phase == kSearch) {
            uint64_t key;
            uint32_t tgt, aux;
            if (SEG && segw) rec_in_block<SegTable>(v, aidx, key, tgt, aux);
            else rec_in_block<E>(v, aidx, key, tgt, aux);
            if (STATS) {
                const uint64_t sec = (SEG && segw) ? ((reinterpret_cast<uint64_t>(p.seg) + aidx * 16) >> 5)
                                                   : ((reinterpret_cast<uint64_t>(p.edges) + aidx * sizeof(typename E::Rec)) >> 5);
                if (sec != last_sec) ++tl.sectors, last_sec = sec;
            }
            const uint32_t half = n >> 1;
            if (key <= x) {
                lo += half;
                n -= half;
            } else {
                n = half;
            }
            if (n == 1) {
                // the answer is lo; the 16-byte block just loaded may already hold it
                const bool in_block = (SEG && segw) ? (lo == aidx)
                                                    : (sizeof(typename E::Rec) == 8 ? ((lo >> 1) == (aidx >> 1)) : (lo == aidx));
                if (in_block) {  // (same sector as the probe: no new sector for the statistics)
                    uint64_t k2;
                    if (SEG && segw) rec_in_block<SegTable>(v, lo, k2, tgt, aux);
                    else rec_in_block<E>(v, lo, k2, tgt, aux);
                    if (SEG && segw) {
                        if ((aux >> 8) == 0) {
                            fin = true;
                            end = tgt;
                            ++tl.steps;
                        } else {
                            u = tgt;
                            k += aux & 0xffu;
                            ++tl.steps;
                            phase = kNode;
                        }
                    } else {
                        next = tgt;
                        step_done = true;
                    }
                } else {
                    phase = kFinal;
                }
            }
        } else if (phase == kFinal) {
            uint64_t key;
            uint32_t tgt, aux;
            if (SEG && segw) rec_in_block<SegTable>(v, aidx, key, tgt, aux);
            else rec_in_block<E>(v, aidx, key, tgt, aux);
            if (STATS) {
                const uint64_t sec = (SEG && segw) ? ((reinterpret_cast<uint64_t>(p.seg) + aidx * 16) >> 5)
                                                   : ((reinterpret_cast<uint64_t>(p.edges) + aidx * sizeof(typename E::Rec)) >> 5);
                if (sec != last_sec) ++tl.sectors, last_sec = sec;
            }
            if (SEG && segw) {
                ++tl.steps;
                if ((aux >> 8) == 0) {
                    fin = true;
                    end = tgt;
                } else {
                    u = tgt;
                    k += aux & 0xffu;
                    phase = kNode;
                }
            } else {
                next = tgt;
                step_done = true;
            }
        } else if (phase == kResolved) {
            next = u;  // chosen by the cooperative search
            step_done = true;
        }
        if (step_done) {
            ++tl.steps;
            ++k;
            u = next;
            if (x2 < p.T) {
                fin = true;
                end = u;
            } else {
                phase = kNode;
            }
        }
        if (fin) {
            slot_ends[(size_t)slot * p.slot_cap + widx] = end - ss[slot].ctr_base;
            phase = kIdle;
        }
        const uint32_t f0 = __ballot_sync(0xffffffffu, fin && slot == 0);
        const uint32_t f1 = __ballot_sync(0xffffffffu, fin && slot == 1);
        if ((f0 | f1) != 0) {
            __syncwarp();
            if (lane == 0) {
                ss[0].done += __popc(f0);
                ss[1].done += __popc(f1);
            }
            __syncwarp();
            // ---- aggregate finished chunks in shared memory
#pragma unroll
            for (int sI = 0; sI < 2; ++sI) {
                const SlotState s = ss[sI];
                if (s.live && s.done == s.total && s.issued == s.total) {
                    for (uint32_t i = 0; i < s.nsrc; ++i) {
                        const uint64_t row = (uint64_t)p.out_row0 + (uint64_t)((int64_t)(s.base + i) - p.s_begin);
                        aggregate_source(slot_ends + (size_t)sI * p.slot_cap + (size_t)i * p.R, p.R, sortbuf, keys,
                                         p.out, row);
                    }
                    __syncwarp();
                    if (lane == 0) ss[sI].live = 0;
                    __syncwarp();
                }
            }
        }
    }
    warp_add_tally<STATS>(p.steps, tl);
}

// ------------------------------------------------------------- launcher ----

template <class E, bool SEG, bool STATS>
static int launch_typed(ppr_ctx *ctx, const KParams &kp0, const RunPlan &plan, int64_t S, cudaStream_t st)
{
    KParams kp = kp0;
    if (plan.kernel == PPR_KERNEL_PLAIN) {
        uint64_t total = (uint64_t)S * kp.R;
        int blocks = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->sms * 64);
        if (blocks < 1) blocks = 1;
        k_walk_plain<E, SEG, STATS><<<blocks, 256, 0, st>>>(kp);
        PPR_CUDA(cudaGetLastError());
        const int aw = 4;
        size_t smem = (size_t)aw * kp.P2 * 12;
        if (smem > 48 * 1024) PPR_CUDA(cudaFuncSetAttribute(k_aggregate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int ablocks = (int)std::min<int64_t>((S + aw - 1) / aw, (int64_t)ctx->sms * 16);
        if (ablocks < 1) ablocks = 1;
        k_aggregate<<<ablocks, aw * 32, smem, st>>>(kp);
        PPR_CUDA(cudaGetLastError());
        return PPR_OK;
    }
    int wpb = plan.warps_per_block > 0 ? plan.warps_per_block : 8;
    const size_t per_warp = (size_t)kp.P2 * 12 + (size_t)kp.slot_cap * 8 + sizeof(SlotState) * 2;
    const size_t per_warp_al = (per_warp + 15) & ~(size_t)15;
    while (wpb > 1 && per_warp_al * wpb > ctx->smem_optin) wpb >>= 1;
    size_t smem = per_warp_al * wpb;
    if (smem > ctx->smem_optin) {
        set_error("persistent walker needs %zu bytes of shared memory per warp", per_warp_al);
        return PPR_ERANGE;
    }
    PPR_CUDA(cudaFuncSetAttribute(k_walk_persistent<E, SEG, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PPR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_persistent<E, SEG, STATS>, wpb * 32, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)ctx->sms * per_sm;
    int64_t needed = ((int64_t)kp.nchunks + wpb - 1) / wpb;
    if (blocks > needed) blocks = std::max<int64_t>(needed, 1);
    k_walk_persistent<E, SEG, STATS><<<(unsigned)blocks, wpb * 32, smem, st>>>(kp);
    PPR_CUDA(cudaGetLastError());
    return PPR_OK;
}

int launch_walks(ppr_ctx *ctx, const ppr_graph *g, const RunPlan &plan, ppr_result *r, int64_t s_begin,
                 int64_t s_end, int64_t out_row0, uint32_t *ends, unsigned long long *queue, cudaStream_t st)
{
    const int64_t S = s_end - s_begin;
    if (S <= 0) return PPR_OK;
    KParams kp{};
    kp.node = plan.segments ? g->seg.node : g->node;
    kp.edges = g->edges;
    kp.seg = g->seg.entries;
    kp.R = plan.R;
    kp.T = plan.T;
    kp.k0 = (uint32_t)plan.seed;
    kp.k1 = (uint32_t)(plan.seed >> 32);
    kp.tag = plan.tag;
    kp.dangling = plan.dangling;
    kp.large = plan.large_degree > 0 ? (uint32_t)plan.large_degree : 4096u;
    kp.s_begin = s_begin;
    kp.s_end = s_end;
    kp.out_row0 = out_row0;
    kp.out.nnz = r->d_nnz;
    kp.out.cols = r->d_cols;
    kp.out.cnts = r->d_cnts;
    kp.out.topk_idx = r->d_topk_idx;
    kp.out.topk_cnt = r->d_topk_cnt;
    kp.out.cap = r->cap;
    kp.out.topk = r->topk;
    kp.steps = r->d_steps;
    kp.queue = queue;
    kp.ends = ends;
    uint32_t P2 = 1;
    while (P2 < plan.R) P2 <<= 1;
    kp.P2 = P2;
    int rc;

    std::vector<int4> chunks;
    if (plan.kernel == PPR_KERNEL_PLAIN) {
        if (g->instances > 0) {
            set_error("the plain kernel runs plain graphs only");
            return PPR_ENOTSUP;
        }
    } else {
        uint32_t CS = plan.chunk_sources > 0 ? (uint32_t)plan.chunk_sources : std::max(1u, 512u / plan.R);
        kp.CS = CS;
        kp.slot_cap = CS * plan.R;
        if (g->instances > 0) {
            // chunks never cross an instance boundary
            const auto &off = g->node_off;
            for (int32_t gi = 0; gi < g->instances; ++gi) {
                int64_t a = std::max(off[gi], s_begin), b = std::min(off[gi + 1], s_end);
                for (int64_t s = a; s < b; s += CS)
                    chunks.push_back(make_int4((int)s, (int)std::min<int64_t>(CS, b - s), gi, 0));
            }
            kp.nchunks = (uint32_t)chunks.size();
            void *d = nullptr;
            if ((rc = dev_alloc(&d, sizeof(int4) * std::max<size_t>(chunks.size(), 1), "chunk table"))) return rc;
            r->scratch.push_back(d);
            PPR_CUDA(cudaMemcpyAsync(d, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, st));
            kp.chunks = (const int4 *)d;
            void *o = nullptr;
            if ((rc = dev_alloc(&o, sizeof(int64_t) * (g->instances + 1), "instance offsets"))) return rc;
            r->scratch.push_back(o);
            PPR_CUDA(cudaMemcpyAsync(o, off.data(), sizeof(int64_t) * (g->instances + 1), cudaMemcpyHostToDevice, st));
            kp.inst_off = (const int64_t *)o;
        } else {
            kp.nchunks = (uint32_t)((S + CS - 1) / CS);
        }
        PPR_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st));
    }
    if (plan.stats) {
        if (g->wide)
            return plan.segments ? launch_typed<WideEdges, true, true>(ctx, kp, plan, S, st)
                                 : launch_typed<WideEdges, false, true>(ctx, kp, plan, S, st);
        return plan.segments ? launch_typed<NarrowEdges, true, true>(ctx, kp, plan, S, st)
                             : launch_typed<NarrowEdges, false, true>(ctx, kp, plan, S, st);
    }
    if (g->wide)
        return plan.segments ? launch_typed<WideEdges, true, false>(ctx, kp, plan, S, st)
                             : launch_typed<WideEdges, false, false>(ctx, kp, plan, S, st);
    return plan.segments ? launch_typed<NarrowEdges, true, false>(ctx, kp, plan, S, st)
                         : launch_typed<NarrowEdges, false, false>(ctx, kp, plan, S, st);
}

}  // namespace ppr
