// walk_step.cuh -- one step of one walk (Sec. 2.1, Algorithm 2), shared by
// the batch walkers (walk.cu) and the serving loop (serve.cu).
//
// A step draws Philox4x32-10 at counter (s_local, j, k, tag); at a node with
// out-edges it takes the first edge whose inclusive weight prefix exceeds
// floor(r64 * W_u / 2^64) and moves to its target; at a node without
// out-edges it restarts at the source (or ends the walk, dangling mode 1);
// then it stops iff x2 < T.  At a node carrying a segment table (Algorithm 4,
// depth 3) the same draw selects one outcome: a terminated outcome ends the
// walk, an active one moves the walk and advances k by the outcome's length.
#pragma once
#include <type_traits>

#include "ppr_host.h"
#include "aggregate.cuh"

namespace ppr {

struct KParams {
    const void *node;         // NodeRecN (narrow layout) or NodeRec (wide layout, alias tables)
    const void *edges;
    const uint32_t *sum;      // narrow split layout: the summary array of the blocked rows
    const SegEntry *seg;
    uint32_t k0, k1, T, R, tag;
    int32_t dangling;
    uint32_t large;
    int64_t s_begin, s_end;   // sources of this launch (global ids)
    int64_t out_row0;         // output row of s_begin
    uint32_t CS;              // sources per chunk (batched graphs)
    uint32_t CW;              // walks per chunk (plain graphs; a chunk may start inside a source)
    uint32_t refill;          // idle lanes before a warp starts new walks (1..32)
    uint32_t step_loads;      // bounded step: dependent loads per lane per iteration (walk_step_bounded)
    uint64_t walks;           // S * R
    uint32_t nchunks;
    const unsigned long long *nchunks_dev;  // batched graphs: chunk count written on the device
    const int4 *chunks;       // batched graphs: {position, nsrc, instance, 0}; else null
    const uint32_t *src_list; // explicit sources (position -> node id); null: s_begin + position
    const int32_t *rank;      // renumbered layout: internal id of a caller node (the walk's start), else null
    const int32_t *order;     // renumbered layout: caller id of an internal node (endpoints), else null
    const int64_t *inst_off;  // batched graphs: node_off
    int32_t instances;
    AggOut out;
    uint32_t *ends;           // S * R endpoints (instance-local ids)
    unsigned long long *queue;
    unsigned long long *steps;    // [0] draws consumed, [2] layout sectors, [5] flat-CSR model sectors (statistics launch)
    uint32_t P2;              // next_pow2(R)
    uint64_t r_magic;         // ceil(2^40 / R): walk index -> source index by multiply-shift
    int64_t n_nodes;          // node records (for the L2 window and the checked build)
    uint64_t n_records;       // checked build: records of the edge layout walked (alias: slots)
    uint64_t n_sum;           // checked build: sectors of the summary array
    uint64_t n_seg;           // checked build: segment entries allocated
    unsigned long long *err;  // checked build: flags of indices that left their array
};

// Checked build (-DPPR_CHECKED): every node index and every row extent a step
// is about to read is tested against its array first; a bad one sets a flag
// in p.err (1 node, 2 edge row, 4 segment table, 8 endpoint slot) and ends the
// walk instead of reading, so the host reports the run as failed; nothing traps.
#ifdef PPR_CHECKED
#define PPR_CHECK(cond, flag)                                  \
    do {                                                       \
        if (!(cond)) {                                         \
            atomicOr(p.err, (unsigned long long)(flag));       \
            end = 0;                                           \
            return true;                                       \
        }                                                      \
    } while (0)
#else
#define PPR_CHECK(cond, flag) \
    do {                      \
    } while (0)
#endif

// One step of one walk.  Returns true when the walk has ended (end is set).
// With COOP, every lane of the warp calls it (inactive lanes with act=false)
// and rows longer than p.large are searched by the whole warp.
struct Tally {
    uint32_t steps = 0;
    uint32_t sectors = 0;
    uint32_t model = 0;  // the same draws on a flat CSR searched by bisection (statistics launch)
};

// 32-byte sectors a draw at a node of out-degree d costs on a flat CSR
// searched by bisection, without reuse: the row_ptr pair, max(1, ceil(log2 d) - 1)
// sectors of prefix probes (the last few probes share a sector), the col
// entry; a dangling node reads its row_ptr pair only.
__device__ __forceinline__ uint32_t flat_model_sectors(uint32_t d)
{
    if (d == 0) return 1;
    const uint32_t lg = d > 1 ? 32u - __clz(d - 1) : 0u;  // ceil(log2 d)
    return 2u + max(1u, lg > 0 ? lg - 1 : 0u);
}

// STATS: count, per step, the 32-byte sectors a thread-serial bisection must
// touch (node record + distinct probe sectors); rows are then searched by
// bisection only, which returns the same edge as the cooperative search.
// The draw of one walk: Philox key (seed) and stop threshold T.  Uniform over
// a launch of the batch kernels; per lane in the serving loop, whose lanes
// may carry walks of different queries.
struct StepKey {
    uint32_t k0, k1, T;
};

// SPLIT: the narrow layout of a renumbered graph (summaries in their own
// array, evict-first bottom blocks); see search_blocked.
template <class E, bool SEG, bool COOP, bool STATS, bool SPLIT = false>
__device__ __forceinline__ bool walk_step(const KParams &p, const StepKey &key, const E &edges, bool act, uint32_t src,
                                          uint32_t sctr, uint32_t j, uint32_t tag, uint32_t &k, uint32_t &u,
                                          uint32_t &end, Tally &tl)
{
    uint4 x = make_uint4(0, 0, 0, 0);
    NodeRec r{};
#ifdef PPR_CHECKED
    bool bad_node = false;
#endif
    if (act) {
#ifdef PPR_CHECKED
        if ((uint64_t)u >= (uint64_t)p.n_nodes) {
            atomicOr(p.err, 1ull);
            bad_node = true;
            u = 0;  // read a valid record; the walk ends at this step
        }
#endif
        r = E::load_node(p.node, u);  // issued before the draw: the record load overlaps Philox
        x = philox4x32_10(make_uint4(sctr, j, k, tag), key.k0, key.k1);
    }
    const uint64_t w0 = r.word0, total = r.total;
    const uint32_t cnt = (uint32_t)(w0 >> 40) & kCountMask;
    const uint64_t beg = w0 & kBeginMask;
    const bool segf = SEG && (w0 >> 63);
    const uint64_t r64 = (uint64_t)x.x | ((uint64_t)x.y << 32);
#ifdef PPR_CHECKED
    if (act && bad_node) {  // flagged above
        end = 0;
        return true;
    }
#endif
    if constexpr (std::is_same<E, AliasEdges>::value) {
        // integer alias method: slot j = floor(r*d / 2^64), y = floor(frac * W / 2^64)
        if (!act) return false;
        PPR_CHECK(cnt < 2 || beg + cnt <= p.n_records, 2);
        if (STATS) ++tl.sectors, ++tl.model;  // the node record
        uint32_t next;
        if (cnt == 0) {
            if (p.dangling == 1) {
                end = u;
                return true;
            }
            next = src;
        } else if (cnt == 1) {
            next = (uint32_t)beg;  // single out-edge: target kept in the record
        } else {
            const uint64_t j = __umul64hi(r64, (uint64_t)cnt);
            const uint64_t frac = r64 * (uint64_t)cnt;
            const uint4 rec = edges.load(beg + j);  // {thr, col, alias col, W}
            const uint64_t y = mulhi64_by32((uint32_t)frac, (uint32_t)(frac >> 32), rec.w);
            next = y < rec.x ? rec.y : rec.z;
            if (STATS) ++tl.sectors, ++tl.model;
        }
        ++tl.steps;
        ++k;
        u = next;
        if (x.z < key.T) {
            end = u;
            return true;
        }
        return false;
    }
    uint64_t xr = 0;
    if (act && (cnt > 1 || segf)) {
        // narrow rows hold the summary shape above bit 32 (W < 2^32 there)
        if (segf || sizeof(typename E::Rec) != 8) xr = mulhi64(r64, total);
        else xr = mulhi64_by32(x.x, x.y, (uint32_t)total);
    }
    uint32_t next = 0;
    bool big = false;
    if (COOP && !STATS && p.large != 0xffffffffu) {  // uniform: skipped whole when the path is off
        big = act && !segf && cnt > p.large;
        uint32_t bigmask = __ballot_sync(0xffffffffu, big);
        const uint32_t lane = threadIdx.x & 31;
        while (bigmask) {
            const uint32_t L = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            const uint32_t n = __shfl_sync(0xffffffffu, cnt, L);
            const uint64_t lo = E::edge_base(__shfl_sync(0xffffffffu, beg, L), n);
            const uint64_t xx = __shfl_sync(0xffffffffu, xr, L);
            auto rec = search_warp(edges, lo, n, xx);
            if (lane == L) next = E::target(rec);
        }
    }
    if (!act) return false;
    if (STATS) {
        ++tl.sectors;  // the node record
        tl.model += segf ? 1u + (cnt <= 2 ? 1u : 2u) : flat_model_sectors(cnt);
    }
    PPR_CHECK(!segf || beg + cnt <= p.n_seg, 4);
    PPR_CHECK(segf || cnt < 2 ||
                  beg + (sizeof(typename E::Rec) == 8 ? (uint64_t)blocked_row_records(cnt) : (uint64_t)cnt) <= p.n_records,
              2);
    PPR_CHECK(segf || cnt < 2 || sizeof(typename E::Rec) != 8 ||
                  (SPLIT ? (uint64_t)blocked_sum(total) + summary_sectors(cnt) <= p.n_sum
                         : blocked_sum(total) == summary_sectors(cnt) && 4ull * blocked_sum(total) <= beg),
              2);
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
        if constexpr (sizeof(typename E::Rec) == 8) {
            next = search_blocked<STATS, SPLIT>(edges.e, p.sum, beg, cnt, blocked_sum(total), blocked_levels(total),
                                                (uint32_t)xr, static_cast<const NodeRecN *>(p.node) + u, tl.sectors);
        } else {
            next = E::target(STATS ? search_serial_tally(edges, beg, cnt, xr, tl.sectors) : search_serial(edges, beg, cnt, xr));
        }
    }
    ++tl.steps;
    ++k;
    u = next;
    if (x.z < key.T) {
        end = u;
        return true;
    }
    return false;
}

// ------------------------------------------------------- bounded step ----
// The warp steps its lanes together, so with walk_step a warp iteration lasts
// as long as the deepest search among its lanes: on a power-law graph nearly
// every iteration has a lane at a hub.  walk_step_bounded gives each lane at
// most p.step_loads dependent loads per iteration (the node record counts as
// one); a search that needs more keeps its place in shared memory (the
// lane's PendSearch words) and resumes in the next iteration while the other
// lanes go on with new draws.  Draw, search rule and result are those of
// walk_step; only the schedule of the loads changes.
// Pending search of one lane: word i of lane t at ps[i * stride + t]
// (structure of arrays: no bank conflicts).  Rows: beg (w0, w1), d (w2),
// flags | levels left (w3), summary field S (w4), sector offset (w5),
// block b (w6), key x (w7).  Segment tables: bisection base (w0, w1), range n (w2), flags (w3),
// key (w6, w7).  Flags: bit 31 the draw stops at the found target, bit 30 a
// segment table.
struct PendRef {
    uint32_t *ps;
    uint32_t stride, t;
    __device__ __forceinline__ uint32_t &operator[](int i) const { return ps[i * stride + t]; }
};

template <bool SEG, bool SPLIT>
__device__ __forceinline__ bool walk_step_bounded(const KParams &p, const StepKey &key, const NarrowEdges &edges,
                                                  uint32_t src, uint32_t sctr, uint32_t j, uint32_t tag, uint32_t &k,
                                                  uint32_t &u, uint32_t &end, bool &pend, const PendRef &ps, Tally &tl)
{
    uint64_t beg = 0, sx = 0;
    uint32_t d = 0, S = 0, l = 0, off = 0, b = 0, x = 0, budget;
    bool stop = false, seg = false;
    if (!pend) {
#ifdef PPR_CHECKED
        if ((uint64_t)u >= (uint64_t)p.n_nodes) {
            atomicOr(p.err, 1ull);
            end = 0;
            return true;
        }
#endif
        const NodeRec r = NarrowEdges::load_node(p.node, u);  // overlaps Philox
        const uint4 xv = philox4x32_10(make_uint4(sctr, j, k, tag), key.k0, key.k1);
        const uint32_t cnt = (uint32_t)(r.word0 >> 40) & kCountMask;
        beg = r.word0 & kBeginMask;
        stop = xv.z < key.T;
        const uint64_t r64 = (uint64_t)xv.x | ((uint64_t)xv.y << 32);
        if (SEG && (r.word0 >> 63)) {
            PPR_CHECK(beg + cnt <= p.n_seg, 4);
            seg = true;
            sx = mulhi64(r64, r.total);
            d = cnt;  // bisection range
        } else if (cnt <= 1) {  // no search: restart (or end) at a dangling node, the single target otherwise
            if (cnt == 0) {
                if (p.dangling == 1) {  // the walk ends here without a step
                    end = u;
                    return true;
                }
                u = src;
            } else {
                u = (uint32_t)r.total;
            }
            ++tl.steps;
            ++k;
            if (stop) {
                end = u;
                return true;
            }
            return false;
        } else {
            PPR_CHECK(beg + (uint64_t)blocked_row_records(cnt) <= p.n_records, 2);
            PPR_CHECK(SPLIT ? (uint64_t)blocked_sum(r.total) + summary_sectors(cnt) <= p.n_sum
                            : blocked_sum(r.total) == summary_sectors(cnt) && 4ull * blocked_sum(r.total) <= beg,
                      2);
            d = cnt;
            S = blocked_sum(r.total);
            l = blocked_levels(r.total);
            x = (uint32_t)mulhi64_by32(xv.x, xv.y, (uint32_t)r.total);
            if (root_in_record(d, l)) {  // the top level is ranked from the record's own sector
                const uint4 kk = __ldg(reinterpret_cast<const uint4 *>(static_cast<const NodeRecN *>(p.node)[u].key));
                b = min(rank8(kk.x, kk.y, kk.z, kk.w, 0xffffffffu, 0xffffffffu, 0xffffffffu, x), (d - 1) >> (3 * l));
                off = 1;
                --l;
            }
        }
        budget = p.step_loads - 1;
    } else {
        const uint32_t fl = ps[3];
        stop = (fl >> 31) != 0;
        seg = SEG && ((fl >> 30) & 1u);
        beg = (uint64_t)ps[0] | ((uint64_t)ps[1] << 32);
        d = ps[2];
        if (seg) {
            sx = (uint64_t)ps[6] | ((uint64_t)ps[7] << 32);
        } else {
            l = fl & 0xfu;
            S = ps[4];
            off = ps[5];
            b = ps[6];
            x = ps[7];
        }
        budget = p.step_loads;
    }
    if (SEG && seg) {  // bisection of the outcome table (Algorithm 4), range [beg, beg + d)
        SegTable tab{p.seg};
        while (d > 1 && budget > 0) {
            const uint32_t half = d >> 1;
            if (SegTable::key(tab.load(beg + half - 1)) <= sx) {
                beg += half;
                d -= half;
            } else {
                d = half;
            }
            --budget;
        }
        if (budget > 0) {
            const uint4 o = tab.load(beg);
            pend = false;
            ++tl.steps;
            if ((o.w >> 8) == 0) {
                end = o.z;
                return true;
            }
            u = o.z;
            k += o.w & 0xffu;
            return false;
        }
        ps[0] = (uint32_t)beg;
        ps[1] = (uint32_t)(beg >> 32);
        ps[2] = d;
        ps[3] = (stop ? 0x80000000u : 0u) | 0x40000000u;
        ps[6] = (uint32_t)sx;
        ps[7] = (uint32_t)(sx >> 32);
        pend = true;
        return false;
    }
    // the row's search tree: levels l .. 1, then the 8-record block
    const unsigned char *base = summary_base<SPLIT>(edges.e, p.sum, beg, S);
    while (l >= 1 && budget > 0) {
        const Sector kv = ld_sector(base + 32ull * (off + b));
        const uint32_t c = rank8(kv.v[0], kv.v[1], kv.v[2], kv.v[3], kv.v[4], kv.v[5], kv.v[6], x);
        off += level_sectors(d, l);
        b = b * 8 + c;
        --l;
        --budget;
    }
    if (budget > 0) {
        const uint32_t len = min(8u, d - 8 * b);
        const unsigned char *q = reinterpret_cast<const unsigned char *>(edges.e + beg) + 64ull * b;
        const Sector r0 = ld_block_sector<SPLIT>(q);
        Sector r1;
        if (len > 4) r1 = ld_block_sector<SPLIT>(q + 32);
        else {
#pragma unroll
            for (int i = 0; i < 8; ++i) r1.v[i] = 0xffffffffu;
        }
        const uint32_t c = rank8(r0.v[0], r0.v[2], r0.v[4], r0.v[6], r1.v[0], r1.v[2], r1.v[4], x);
        const bool hiq = (c & 4u) != 0;
        const uint32_t h1 = hiq ? r1.v[1] : r0.v[1], h3 = hiq ? r1.v[3] : r0.v[3];
        const uint32_t h5 = hiq ? r1.v[5] : r0.v[5], h7 = hiq ? r1.v[7] : r0.v[7];
        const uint32_t lo = (c & 1u) ? h3 : h1, hi = (c & 1u) ? h7 : h5;
        pend = false;
        ++tl.steps;
        ++k;
        u = (c & 2u) ? hi : lo;
        if (stop) {
            end = u;
            return true;
        }
        return false;
    }
    ps[0] = (uint32_t)beg;
    ps[1] = (uint32_t)(beg >> 32);
    ps[2] = d;
    ps[3] = (stop ? 0x80000000u : 0u) | l;
    ps[4] = S;
    ps[5] = off;
    ps[6] = b;
    ps[7] = x;
    pend = true;
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
template <>
__device__ __forceinline__ AliasEdges make_edges<AliasEdges>(const void *e)
{
    return AliasEdges{(const AliasRec *)e};
}

}  // namespace ppr
