// ppr_internal.cuh -- device-side building blocks of libppr.so (sm_103a).
//
// Graph layout in HBM
//   NodeRec (16 B, one aligned half-sector per node; wide layout, alias tables)
//     word0 = begin (bits 0..39) | count (bits 40..62) | segment flag (bit 63)
//     word1 = W_u, the row's total weight (Sec. 2.1 routing denominator), or
//             the target id when the row has exactly one edge (no search), or
//             Q_v, the total fixed-point mass of a segment table (Algorithm 4);
//             narrow blocked rows keep W_u in bits 0..31, a summary field
//             (bits 32..59, see blocked_sum) and their level count L (bits
//             60..63) above it
//   NodeRecN (32 B, one sector per node; narrow layout): a NodeRec and the
//     first four keys of the row's top summary level when that level has at
//     most five keys (the fifth is W_u), so the step that reads the record
//     ranks the draw within the top level and skips that sector
//   plain rows:  begin/count index the edge-record array
//   segment rows: begin/count index the segment-entry array
//   EdgeN (8 B): {uint32 P, int32 col}  -- narrow layout, every W_u < 2^32
//   EdgeW (16 B): {uint64 P, int32 col, pad} -- wide layout (flat rows)
//
// Narrow rows are stored as static search trees ("blocked" rows).  A row with
// d >= 2 edges has its edge records in blocks of 8 in the edge array (the
// area rounded up to whole sectors, padding keys 0xFFFFFFFF) and, when d > 8,
// summary levels, top level first.  Two placements (the walkers' SPLIT
// template parameter):
//   split (renumbered graphs far larger than L2): the summaries sit in a
//     summary array that holds nothing else, so the summary sectors that
//     every draw at a node passes through share L2 lines and DRAM pages
//     instead of lying one per row between blocks that a draw reads once;
//     every row's blocks start on 64 bytes, so a full block is one fetch;
//   interleaved (otherwise): each row's area holds its summary, then its
//     blocks, starting on a 32-byte sector.
// Level 1 keeps the last prefix of every 8-record block, level l+1 the last
// key of every 8-key sector of level l, up to a top level of at most 8 keys
// (one sector).
// A search reads one sector per level and one 8-record block: the same edge
// as bisection of the flat prefix (the first P > x is unique), found with
// ceil(log8 d) + 1 dependent loads instead of ceil(log2 d) + 1.  The alias
// tree of the paper (Algorithm 3) splits large neighbour sets the same way so
// that a selection touches one small set per level; Lemma 1 is the analogous
// exactness argument.
//   SegEntry (16 B): {uint64 cum, uint32 node, uint32 mark_len}
//   P / cum are inclusive prefix sums within the row / table.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ppr {

constexpr uint64_t kBeginMask = (1ull << 40) - 1;
constexpr uint32_t kCountMask = (1u << 23) - 1;
constexpr uint64_t kSegFlag = 1ull << 63;

struct __align__(16) NodeRec {
    uint64_t word0;
    uint64_t total;
};

struct __align__(32) NodeRecN {
    uint64_t word0;
    uint64_t total;
    uint32_t key[4];  // top-level keys 0..3 (see root_in_record), else 0xFFFFFFFF
};

struct __align__(8) EdgeN {
    uint32_t P;
    int32_t col;
};

struct __align__(16) EdgeW {
    uint64_t P;
    int32_t col;
    uint32_t pad;
};

// Alias slot (integer Algorithm 1): edge j of the row is taken when the
// draw's y < thr, else its alias; both targets and the row total W (the slot
// capacity y is scaled to) are kept so that a step reads one record after
// an 8-byte node record.
struct __align__(16) AliasRec {
    uint32_t thr;
    int32_t col;
    int32_t alias_col;
    uint32_t W;
};

// Node record of the alias layout: first slot (bits 0..39) | degree (bits
// 40..62); a single-edge row keeps its target in the slot field.
struct __align__(8) AliasNode {
    uint64_t word;
};

struct __align__(16) SegEntry {
    uint64_t cum;
    uint32_t node;
    uint32_t mark_len;  // (active << 8) | len
};

__host__ __device__ inline uint64_t pack_word0(uint64_t begin, uint32_t count, bool seg)
{
    return (begin & kBeginMask) | ((uint64_t)(count & kCountMask) << 40) | (seg ? kSegFlag : 0ull);
}

// ceil(d / 2^s)
__host__ __device__ __forceinline__ uint32_t ceil_shift(uint32_t d, uint32_t s) { return (d + (1u << s) - 1) >> s; }

// Number of summary levels above a blocked row of d edges (0 for d <= 8).
__host__ __device__ __forceinline__ uint32_t tree_levels(uint32_t d)
{
    uint32_t L = 0;
    while (d > (1u << (3 * (L + 1)))) ++L;
    return L;
}

// Sectors of level l (1 <= l <= L): ceil(keys_l / 8) = ceil(d / 8^(l+1)).
__host__ __device__ __forceinline__ uint32_t level_sectors(uint32_t d, uint32_t l) { return ceil_shift(d, 3 * (l + 1)); }

__host__ __device__ __forceinline__ uint32_t summary_sectors(uint32_t d)
{
    uint32_t L = tree_levels(d), S = 0;
    for (uint32_t l = 1; l <= L; ++l) S += level_sectors(d, l);
    return S;
}

// 8-byte record slots a blocked row's blocks take (a one-edge row keeps its
// target in the node record and needs none), not counting its summary
// levels (summary_sectors) or the split layout's padding to 64 bytes.
__host__ __device__ __forceinline__ uint32_t blocked_row_records(uint32_t d)
{
    if (d <= 1) return 0;
    return 4 * ceil_shift(d, 2);
}

// A blocked row's record keeps, above W_u, a 28-bit summary field and its
// level count (4 bits).  The field is the row's first sector in the summary
// array on a split layout (renumbered graphs far larger than L2), and the
// number of summary sectors that precede the row's blocks in the edge array
// otherwise; the record's begin points at the blocks either way.
constexpr uint32_t kSumBits = 28;
constexpr uint64_t kSumSectorsMax = 1ull << kSumBits;
__host__ __device__ __forceinline__ uint32_t blocked_sum(uint64_t total) { return (uint32_t)(total >> 32) & (uint32_t)(kSumSectorsMax - 1); }
__host__ __device__ __forceinline__ uint32_t blocked_levels(uint64_t total) { return (uint32_t)(total >> 60); }

// ---------------------------------------------------------------- Philox ----
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// takes the 32x32->64 products of counter words 0 and 2 with two fixed
// multipliers, and the new words are (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
// the key advances by the golden-ratio and sqrt(3) Weyl increments between
// rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t lo0 = m0 * c.x, hi0 = __umulhi(m0, c.x);
        uint32_t lo1 = m1 * c.z, hi1 = __umulhi(m1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// floor(r * W / 2^64) for a 32-bit W, exactly, with two 32x32 products.
__device__ __forceinline__ uint64_t mulhi64_by32(uint32_t r_lo, uint32_t r_hi, uint32_t W)
{
    uint64_t a = (uint64_t)r_lo * W;
    uint64_t b = (uint64_t)r_hi * W + (a >> 32);
    return b >> 32;
}

__device__ __forceinline__ uint64_t mulhi64(uint64_t r, uint64_t W) { return __umul64hi(r, W); }

// ---------------------------------------------------------------- loads ----
__device__ __forceinline__ NodeRec load_node(const NodeRec *node, uint32_t u)
{
    uint4 v = __ldg(reinterpret_cast<const uint4 *>(node) + u);
    NodeRec r;
    r.word0 = (uint64_t)v.x | ((uint64_t)v.y << 32);
    r.total = (uint64_t)v.z | ((uint64_t)v.w << 32);
    return r;
}

// One 32-byte sector in a single 256-bit load (sm_100+ vector width).
struct Sector {
    uint32_t v[8];
};
__device__ __forceinline__ Sector ld_sector(const void *p)
{
    Sector s;
    asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]), "=r"(s.v[6]),
                   "=r"(s.v[7])
                 : "l"(p));
    return s;
}


// One 32-byte sector of a row's bottom block.  EF (layouts of graphs far
// larger than L2) loads it with an evict-first L2 policy: a bottom block
// serves the one draw that picked it and is rarely read again before it would
// leave L2, while node records and summary sectors are shared by every draw
// that passes the same node, so blocks should be the first to go.  On a graph
// about the size of L2 the blocks are reused (evict-first there cost the
// 2,048-graph batch 3 %), so they keep the normal policy.
template <bool EF>
__device__ __forceinline__ Sector ld_block_sector(const void *p)
{
    if constexpr (!EF) {
        return ld_sector(p);
    } else {
        uint64_t pol;
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
        Sector s;
        asm("ld.global.nc.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
            : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]), "=r"(s.v[6]),
              "=r"(s.v[7])
            : "l"(p), "l"(pol));
        return s;
    }
}

// A blocked row of d edges with L >= 1 summary levels keeps its top level's
// keys in the node record when that level has at most five keys
// (ceil(d / 8^L) <= 5): keys 0..3 in NodeRecN::key, the fifth being W_u.
__host__ __device__ __forceinline__ bool root_in_record(uint32_t d, uint32_t L)
{
    return L >= 1 && d <= (5u << (3 * L));
}

struct NarrowEdges {
    using Key = uint32_t;
    using Node = NodeRecN;
    // the record half of the sector; search_blocked reads the key half when
    // it needs it (then an L1 hit: the first load brought the whole sector)
    __device__ __forceinline__ static NodeRec load_node(const void *node, uint32_t u)
    {
        return ppr::load_node(reinterpret_cast<const NodeRec *>(static_cast<const NodeRecN *>(node) + u), 0);
    }
    const EdgeN *e;
    // record index of edge 0 of a row whose region starts at `begin`
    __host__ __device__ __forceinline__ static uint64_t edge_base(uint64_t begin, uint32_t)
    {
        return begin;  // the summary levels live in their own array
    }
    __device__ __forceinline__ uint2 load(uint64_t i) const
    {
        return __ldg(reinterpret_cast<const uint2 *>(e) + i);
    }
    __device__ __forceinline__ static uint64_t key(uint2 v) { return v.x; }
    __device__ __forceinline__ static uint32_t target(uint2 v) { return v.y; }
    using Rec = uint2;
};

struct WideEdges {
    using Node = NodeRec;
    __device__ __forceinline__ static NodeRec load_node(const void *node, uint32_t u)
    {
        return ppr::load_node(static_cast<const NodeRec *>(node), u);
    }
    const EdgeW *e;
    __host__ __device__ __forceinline__ static uint64_t edge_base(uint64_t begin, uint32_t) { return begin; }
    __device__ __forceinline__ uint4 load(uint64_t i) const
    {
        return __ldg(reinterpret_cast<const uint4 *>(e) + i);
    }
    __device__ __forceinline__ static uint64_t key(uint4 v) { return (uint64_t)v.x | ((uint64_t)v.y << 32); }
    __device__ __forceinline__ static uint32_t target(uint4 v) { return v.z; }
    using Rec = uint4;
};

// Alias layout: begin/count of a node record index its alias slots.
struct AliasEdges {
    using Node = AliasNode;
    __device__ __forceinline__ static NodeRec load_node(const void *node, uint32_t u)
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(node) + u);
        NodeRec r;
        r.word0 = (uint64_t)v.x | ((uint64_t)v.y << 32);
        r.total = 0;
        return r;
    }
    const AliasRec *e;
    __host__ __device__ __forceinline__ static uint64_t edge_base(uint64_t begin, uint32_t) { return begin; }
    __device__ __forceinline__ uint4 load(uint64_t i) const { return __ldg(reinterpret_cast<const uint4 *>(e) + i); }
    __device__ __forceinline__ static uint64_t key(uint4 v) { return v.x; }
    __device__ __forceinline__ static uint32_t target(uint4 v) { return v.y; }
    using Rec = uint4;
};

// Segment entries have the same 16-byte shape as wide edges: key = cum,
// target = node, and the fourth word carries mark_len.
struct SegTable {
    const SegEntry *e;
    __device__ __forceinline__ uint4 load(uint64_t i) const
    {
        return __ldg(reinterpret_cast<const uint4 *>(e) + i);
    }
    __device__ __forceinline__ static uint64_t key(uint4 v) { return (uint64_t)v.x | ((uint64_t)v.y << 32); }
    __device__ __forceinline__ static uint32_t target(uint4 v) { return v.z; }
    using Rec = uint4;
};

// Smallest index e in [lo, lo+n) with key(e) > x, given key(lo+n-1) > x.
// Thread-serial bisection; returns the record at e.
template <class E>
__device__ __forceinline__ typename E::Rec search_serial(const E &edges, uint64_t lo, uint32_t n, uint64_t x)
{
    while (n > 1) {
        uint32_t half = n >> 1;
        typename E::Rec v = edges.load(lo + half - 1);
        if (E::key(v) <= x) {
            lo += half;
            n -= half;
        } else {
            n = half;
        }
    }
    return edges.load(lo);
}

// The same bisection, also counting the distinct 32-byte sectors its probes
// touch (consecutive probes in one sector count once).  Used by the
// statistics launch that measures the algorithmic bytes of a run.
template <class E>
__device__ __forceinline__ typename E::Rec search_serial_tally(const E &edges, uint64_t lo, uint32_t n, uint64_t x,
                                                              uint32_t &sectors)
{
    const uint64_t base = reinterpret_cast<uint64_t>(edges.e);
    constexpr uint64_t rec = sizeof(typename E::Rec);
    uint64_t last = ~0ull;
    while (n > 1) {
        uint32_t half = n >> 1;
        uint64_t sec = (base + (lo + half - 1) * rec) >> 5;
        if (sec != last) ++sectors, last = sec;
        typename E::Rec v = edges.load(lo + half - 1);
        if (E::key(v) <= x) {
            lo += half;
            n -= half;
        } else {
            n = half;
        }
    }
    uint64_t sec = (base + lo * rec) >> 5;
    if (sec != last) ++sectors;
    return edges.load(lo);
}


// field: the row's summary field (below 2^28; see blocked_sum)
__host__ __device__ __forceinline__ uint64_t pack_blocked_total(uint64_t W, uint64_t field, uint32_t d)
{
    return W | (field << 32) | ((uint64_t)tree_levels(d) << 60);
}

// Number of the 8 keys k[0..7] that are <= x, for keys in ascending order with
// k[7] > x (a summary sector's last key is its parent's key, above x; missing
// keys are 0xFFFFFFFF): three comparisons of a binary search, 0..7.
__device__ __forceinline__ uint32_t rank8(uint32_t k0, uint32_t k1, uint32_t k2, uint32_t k3, uint32_t k4, uint32_t k5,
                                          uint32_t k6, uint32_t x)
{
    uint32_t c = k3 <= x ? 4u : 0u;
    c += (c ? k5 : k1) <= x ? 2u : 0u;
    const uint32_t kk = (c & 4u) ? ((c & 2u) ? k6 : k4) : ((c & 2u) ? k2 : k0);
    return c + (kk <= x ? 1u : 0u);
}

// First byte of a blocked row's summary (its top level): sector S of the
// summary array SUM (SPLIT), or the S sectors before the row's blocks.
template <bool SPLIT>
__device__ __forceinline__ const unsigned char *summary_base(const EdgeN *E, const uint32_t *SUM, uint64_t begin,
                                                             uint32_t S)
{
    if constexpr (SPLIT) return reinterpret_cast<const unsigned char *>(SUM + 8ull * S);
    else return reinterpret_cast<const unsigned char *>(E + begin) - 32ull * S;
}

// Search of a blocked narrow row (layout above) whose blocks start at record
// `begin` of E, with summary field S and L summary levels: the target of the
// first edge with P > x.  TALLY counts the 32-byte sectors read.
template <bool TALLY, bool SPLIT>
__device__ __forceinline__ uint32_t search_blocked(const EdgeN *E, const uint32_t *SUM, uint64_t begin, uint32_t d,
                                                   uint32_t S, uint32_t L, uint32_t x, const NodeRecN *rec,
                                                   uint32_t &sectors)
{
    const unsigned char *base = summary_base<SPLIT>(E, SUM, begin, S);  // the row's top level
    uint32_t b = 0, off = 0, l = L;
    if (root_in_record(d, L)) {  // the top level (one sector) is ranked from the node record
        const uint4 k = __ldg(reinterpret_cast<const uint4 *>(rec->key));
        b = min(rank8(k.x, k.y, k.z, k.w, 0xffffffffu, 0xffffffffu, 0xffffffffu, x), (d - 1) >> (3 * L));
        off = 1;
        --l;
    }
    for (; l >= 1; --l) {
        const Sector k = ld_sector(base + 32ull * (off + b));
        const uint32_t c = rank8(k.v[0], k.v[1], k.v[2], k.v[3], k.v[4], k.v[5], k.v[6], x);
        off += level_sectors(d, l);
        b = b * 8 + c;
        if (TALLY) ++sectors;
    }
    const uint32_t len = min(8u, d - 8 * b);
    const unsigned char *q = reinterpret_cast<const unsigned char *>(E + begin) + 64ull * b;  // block b: (P, col) pairs
    const Sector r0 = ld_block_sector<SPLIT>(q);
    Sector r1;
    if (len > 4) r1 = ld_block_sector<SPLIT>(q + 32);
    else {
#pragma unroll
        for (int i = 0; i < 8; ++i) r1.v[i] = 0xffffffffu;
    }
    if (TALLY) sectors += len > 4 ? 2 : 1;
    // record i holds (P, col) in words 2i, 2i+1 of r0 (i < 4) or r1 (i >= 4)
    const uint32_t c = rank8(r0.v[0], r0.v[2], r0.v[4], r0.v[6], r1.v[0], r1.v[2], r1.v[4], x);
    const Sector &h = (c & 4u) ? r1 : r0;
    const uint32_t lo = (c & 1u) ? h.v[3] : h.v[1], hi = (c & 1u) ? h.v[7] : h.v[5];
    return (c & 2u) ? hi : lo;
}

// Same result, computed by the whole warp for one lane's search (all 32 lanes
// must call it with the same arguments).  Each round splits the range into 32
// parts, every lane reads the last key of one part and a ballot locates the
// part holding the answer: ceil(log32 n) + 1 rounds instead of log2 n
// dependent loads.
template <class E>
__device__ __forceinline__ typename E::Rec search_warp(const E &edges, uint64_t lo, uint32_t n, uint64_t x)
{
    const uint32_t lane = threadIdx.x & 31;
    while (n > 32) {
        uint32_t end_i = (uint32_t)(((uint64_t)(lane + 1) * n) >> 5);  // part i = [i*n/32, (i+1)*n/32)
        uint32_t beg_i = (uint32_t)(((uint64_t)lane * n) >> 5);
        bool above = true;
        if (end_i > beg_i) above = E::key(edges.load(lo + end_i - 1)) > x;
        uint32_t mask = __ballot_sync(0xffffffffu, above);
        uint32_t f = __ffs(mask) - 1;  // mask != 0: the last part ends at n-1 whose key > x
        uint32_t nb = (uint32_t)(((uint64_t)f * n) >> 5);
        uint32_t ne = (uint32_t)(((uint64_t)(f + 1) * n) >> 5);
        lo += nb;
        n = ne - nb;
    }
    typename E::Rec v{};
    bool above = false;
    if (lane < n) {
        v = edges.load(lo + lane);
        above = E::key(v) > x;
    }
    uint32_t mask = __ballot_sync(0xffffffffu, above);
    uint32_t f = __ffs(mask) - 1;
    typename E::Rec r;
    if constexpr (sizeof(typename E::Rec) == 8) {
        r.x = __shfl_sync(0xffffffffu, v.x, f);
        r.y = __shfl_sync(0xffffffffu, v.y, f);
    } else {
        r.x = __shfl_sync(0xffffffffu, v.x, f);
        r.y = __shfl_sync(0xffffffffu, v.y, f);
        r.z = __shfl_sync(0xffffffffu, v.z, f);
        r.w = __shfl_sync(0xffffffffu, v.w, f);
    }
    return r;
}

// ----------------------------------------------------------- aggregation ----
// Per-source aggregation of R endpoints (Algorithm 2's final grouping of the
// terminated walks by (head, tail)), done by one warp in shared memory:
// bitonic sort of the endpoints, run-length counting, row write-out, then a
// second bitonic sort of (count desc, end asc) keys for the top-k.

__device__ __forceinline__ uint32_t next_pow2(uint32_t v)
{
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <class T>
__device__ __forceinline__ void warp_bitonic_sort(T *a, uint32_t n_pow2)
{
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = 2; k <= n_pow2; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < n_pow2; i += 32) {
                uint32_t l = i ^ j;
                if (l > i) {
                    T x = a[i], y = a[l];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace ppr
