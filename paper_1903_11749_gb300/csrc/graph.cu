// graph.cu -- device construction of the walk layout (node records, per-row
// inclusive weight prefixes) and of the depth-3 segment tables.
//
// Sec. 2.1 defines the routing probability r(s,t) = w(<s,t>) / sum_v w(<s,v>).
// The step rule realises it exactly over integers with the row's inclusive
// prefix P and total W_u: the next edge is the first e with P[e] > x for x
// uniform on [0, W_u).  Algorithm 4 ("big moves") precomputes, for small
// nodes, the distribution over short walk outcomes; here it is built with a
// fixed depth of 3 in 2^62 fixed point, one warp per node.
#include <cstdio>

#include "ppr_host.h"
#include "scan.cuh"

namespace ppr {

enum : uint32_t { kBadRowPtr = 1u, kBadCol = 2u, kBadWeight = 4u };

struct BuildStats {
    unsigned long long max_total;
    unsigned long long max_degree;
    unsigned long long dangling;
    unsigned int status;
};

// Instance of global node u in a block-diagonal graph (node_off has count+1
// entries); returns 0 for a plain graph.
__device__ __forceinline__ int32_t instance_of(const int64_t *node_off, int32_t count, int64_t u)
{
    int32_t lo = 0, hi = count;  // find last g with node_off[g] <= u
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (node_off[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Wide layout (some row total >= 2^32), two passes.
// Pass 1: one warp per row.  Validates the CSR, sums the row weights.
__global__ void k_rows_pass1(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                             const uint32_t *w, const int64_t *node_off, int32_t count, uint64_t *W,
                             BuildStats *st)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        int64_t a = row_ptr[u], b = row_ptr[u + 1];
        bool bad = a < 0 || b < a || b > m || (u == 0 && a != 0) || (u == n - 1 && b != m);
        if (bad) {
            if (lane == 0) atomicOr(&st->status, kBadRowPtr);
            if (lane == 0) W[u] = 0;
            continue;
        }
        int64_t lo_id = 0, hi_id = n;
        if (count > 0) {
            int32_t g = instance_of(node_off, count, u);
            lo_id = 0;
            hi_id = node_off[g + 1] - node_off[g];
        }
        uint64_t sum = 0;
        uint32_t flags = 0;
        for (int64_t e = a + lane; e < b; e += 32) {
            uint32_t we = w[e];
            int64_t c = col[e];
            if (we == 0) flags |= kBadWeight;
            if (c < lo_id || c >= hi_id) flags |= kBadCol;
            sum += we;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            flags |= __shfl_xor_sync(0xffffffffu, flags, o);
        }
        if (lane == 0) {
            W[u] = sum;
            if (flags) atomicOr(&st->status, flags);
            atomicMax(&st->max_total, (unsigned long long)sum);
            atomicMax(&st->max_degree, (unsigned long long)(b - a));
            if (b == a) atomicAdd(&st->dangling, 1ull);
        }
    }
}

// Pass 2: one warp per row.  Inclusive prefix of the row's weights (warp scan
// over 32-edge chunks with a carry) into the edge records; the node record.
template <bool WIDE>
__global__ void k_rows_pass2(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint32_t *w,
                             const int64_t *node_off, int32_t count, const uint64_t *W, NodeRec *node,
                             void *edges_v)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        int64_t a = row_ptr[u], b = row_ptr[u + 1];
        int64_t base_id = 0;
        if (count > 0) base_id = node_off[instance_of(node_off, count, u)];
        uint64_t carry = 0;
        for (int64_t e0 = a; e0 < b; e0 += 32) {
            int64_t e = e0 + lane;
            uint64_t v = e < b ? (uint64_t)w[e] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            uint64_t P = carry + v;
            if (e < b) {
                int32_t c = (int32_t)(col[e] + base_id);
                if (WIDE) {
                    EdgeW r;
                    r.P = P;
                    r.col = c;
                    r.pad = 0;
                    reinterpret_cast<EdgeW *>(edges_v)[e] = r;
                } else {
                    EdgeN r;
                    r.P = (uint32_t)P;
                    r.col = c;
                    reinterpret_cast<EdgeN *>(edges_v)[e] = r;
                }
            }
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) {
            NodeRec r;
            r.word0 = pack_word0((uint64_t)a, (uint32_t)(b - a), false);
            // a single out-edge needs no draw-to-edge search: keep its target inline
            r.total = (b - a == 1) ? (uint64_t)(uint32_t)(col[a] + base_id) : W[u];
            node[u] = r;
        }
    }
}

// ----------------------------------------------------- single-pass build ----
// The narrow (32-bit prefix) layout is built in one validating pass over the
// input: k_layout checks row_ptr and sizes every blocked row; after the scan
// of those sizes, k_build_small builds every row of at most 32 edges with one
// thread, and queues longer rows for k_build_mid (one warp per row, up to
// 1,024 edges) and k_build_big (one block per row, up to 8,192); longer rows
// are cut into tiles.  The limits keep every row within a few passes of its
// group, so no single long row leaves the GPU idle behind it.  A row total
// >= 2^32 sets kWide and the graph is rebuilt in the wide layout.
enum : uint32_t { kWide = 8u, kBigDegree = 16u };
constexpr uint32_t kSmallRow = 32, kMidRow = 1024, kHugeRow = 8192;
constexpr uint32_t kBuildTile = 8192;  // edges per tile block of a huge row (256 threads x 32)

struct LayoutStats {
    unsigned long long max_degree;
    unsigned long long dangling;
    unsigned int status;
    unsigned int n_mid, n_big, n_huge;
};

__device__ __forceinline__ void block_stats(LayoutStats *st, uint32_t deg_max, uint32_t dang, uint32_t flags)
{
    __shared__ uint32_t s_max, s_dang, s_flags;
    if (threadIdx.x == 0) {
        s_max = 0;
        s_dang = 0;
        s_flags = 0;
    }
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        deg_max = max(deg_max, __shfl_xor_sync(0xffffffffu, deg_max, o));
        dang += __shfl_xor_sync(0xffffffffu, dang, o);
        flags |= __shfl_xor_sync(0xffffffffu, flags, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&s_max, deg_max);
        atomicAdd(&s_dang, dang);
        atomicOr(&s_flags, flags);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_max) atomicMax(&st->max_degree, (unsigned long long)s_max);
        if (s_dang) atomicAdd(&st->dangling, (unsigned long long)s_dang);
        if (s_flags) atomicOr(&st->status, s_flags);
    }
}

// order: the caller's row of internal node u (renumbered layout), or null.
// sizes: the row's records in the edge array (its blocks, and with
// interleave its summary sectors before them); ssizes: its summary sectors.
__global__ void __launch_bounds__(256) k_layout(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *order,
                                                bool interleave, uint32_t *sizes, uint32_t *ssizes, LayoutStats *st,
                                                uint2 *huge, uint32_t huge_cap)
{
    uint32_t dmax = 0, dang = 0, flags = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = order ? (int64_t)order[u] : u;
        const int64_t a = row_ptr[o], b = row_ptr[o + 1];
        const bool bad = a < 0 || b < a || b > m || (o == 0 && a != 0) || (o == n - 1 && b != m);
        uint32_t sz = 0, ssz = 0;
        if (bad) {
            flags |= kBadRowPtr;
        } else if (b - a > PPR_MAX_DEGREE) {
            flags |= kBigDegree;
        } else {
            const uint32_t d = (uint32_t)(b - a);
            dmax = max(dmax, d);
            dang += d == 0;
            ssz = d >= 2 ? summary_sectors(d) : 0u;
            // split layout: every row's blocks start on 64 bytes (a full block is
            // one 64-byte DRAM fetch); otherwise on 32 bytes after the summary
            sz = interleave ? blocked_row_records(d) + 4 * ssz : (d <= 1 ? 0u : 8u * ceil_shift(d, 3));
            if (d > kHugeRow) {  // a valid row_ptr has at most m / kHugeRow of them
                const uint32_t k = atomicAdd(&st->n_huge, 1u);
                if (k < huge_cap) huge[k] = make_uint2((uint32_t)u, d);
            }
        }
        sizes[u] = sz;
        ssizes[u] = ssz;
    }
    block_stats(st, dmax, dang, flags);
}

struct BuildArgs {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col;
    const uint32_t *w;
    const int64_t *node_off;
    int32_t count;
    const uint64_t *region;   // first record of each row's area in E
    const uint64_t *sregion;  // first summary sector of each row in K, or null: summary at the start of the row's area
    NodeRecN *node;
    EdgeN *E;
    uint32_t *K;              // the summary array (8 keys a sector)
    LayoutStats *st;
    uint32_t *list;  // mid rows from the front, big rows from the back
    const int32_t *order;  // renumbered layout: caller row of internal node u, else null
    const int32_t *rank;   // renumbered layout: internal id of caller node v, else null
};

// First block record (reg) and first summary sector (sreg) of row u of degree
// d: separate arrays, or one area in E holding the summary, then the blocks.
__device__ __forceinline__ void row_regions(const BuildArgs &A, int64_t u, uint32_t d, uint64_t &reg, uint64_t &sreg)
{
    if (A.sregion) {
        reg = A.region[u];
        sreg = A.sregion[u];
    } else {
        sreg = A.region[u] / 4;  // areas start on a 32-byte sector
        reg = A.region[u] + (d >= 2 ? 4ull * summary_sectors(d) : 0ull);
    }
}

// Input row (caller numbering) of internal node u, and the internal id of a
// target the caller numbered c (c already checked to lie in [0, n)).
__device__ __forceinline__ int64_t in_row(const BuildArgs &A, int64_t u) { return A.order ? (int64_t)A.order[u] : u; }
__device__ __forceinline__ int64_t map_col(const BuildArgs &A, int64_t c) { return A.rank ? (int64_t)A.rank[c] : c; }

// u32 slot in the summary array of key i of level l of a blocked row (first
// summary sector sreg, degree d, L levels; the top level comes first)
__device__ __forceinline__ uint64_t key_slot(uint64_t sreg, uint32_t d, uint32_t L, uint32_t l, uint32_t i)
{
    uint32_t off = 0;
    for (uint32_t q = L; q > l; --q) off += level_sectors(d, q);
    return (sreg + off) * 8ull + i;
}

// Node record of a built row; a row whose top summary level fits the record
// (root_in_record) gets that level's first four keys, read back from the
// level the calling group has just written.
__device__ __forceinline__ void write_node(const BuildArgs &A, int64_t u, uint64_t reg, uint64_t sreg, uint32_t d,
                                           uint64_t W, uint32_t first_target)
{
    NodeRecN r;
    r.word0 = pack_word0(reg, d, false);
    // summary field: the first sector in the summary array (split layout), or
    // the number of summary sectors before the blocks (see blocked_sum)
    const uint64_t field = d <= 8 ? 0ull : (A.sregion ? sreg : (uint64_t)summary_sectors(d));
    r.total = d == 1 ? (uint64_t)first_target : (d == 0 ? 0ull : pack_blocked_total(W, field, d));
    const uint32_t L = d >= 2 ? tree_levels(d) : 0;
    const bool root = root_in_record(d, L);
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) r.key[i] = root ? A.K[key_slot(sreg, d, L, L, i)] : 0xffffffffu;
    A.node[u] = r;
}

__device__ __forceinline__ int64_t instance_base(const BuildArgs &A, int64_t u, int64_t &hi_id)
{
    if (A.count == 0) {
        hi_id = A.n;
        return 0;
    }
    const int32_t g = instance_of(A.node_off, A.count, u);
    hi_id = A.node_off[g + 1] - A.node_off[g];
    return A.node_off[g];
}

// summary levels 2..L from level 1 (already written), padding included;
// the calling group (warp or block) strides over keys with `rank`/`size`
__device__ void write_upper_levels(uint32_t *K, uint64_t sreg, uint32_t d, uint32_t L, uint32_t rank, uint32_t size,
                                   bool block)
{
    for (uint32_t l = 2; l <= L; ++l) {
        const uint32_t nl = ceil_shift(d, 3 * l), np = ceil_shift(d, 3 * (l - 1));
        for (uint32_t i = rank; i < 8 * level_sectors(d, l); i += size) {
            uint32_t kv = 0xffffffffu;
            if (i < nl) kv = K[key_slot(sreg, d, L, l - 1, min(8 * i + 8, np) - 1)];
            K[key_slot(sreg, d, L, l, i)] = kv;
        }
        if (block) __syncthreads();
        else __syncwarp();
    }
}

// Each thread of a row's group takes a run of kRun consecutive edges per pass:
// its kRun loads are independent, so a pass costs one memory latency for
// 32 * kRun (warp) or 512 * kRun (block) edges.
constexpr uint32_t kRun = 4;

struct EdgeRun {
    uint32_t w[kRun];
    int32_t c[kRun];
    uint64_t sum;
};

// Loads edges [i0, i0 + kRun) of row (a, d); missing ones read as weight 0.
__device__ __forceinline__ EdgeRun load_run(const BuildArgs &A, int64_t a, uint32_t d, uint32_t i0, int64_t hi_id,
                                            uint32_t &flags)
{
    EdgeRun r;
    r.sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < kRun; ++q) {
        const uint32_t i = i0 + q;
        r.w[q] = 0;
        r.c[q] = 0;
        if (i < d) {
            r.w[q] = A.w[a + i];
            r.c[q] = A.col[a + i];
        }
    }
#pragma unroll
    for (uint32_t q = 0; q < kRun; ++q) {
        if (i0 + q < d) {
            if (r.w[q] == 0) flags |= kBadWeight;
            if (r.c[q] < 0 || (int64_t)r.c[q] >= hi_id) flags |= kBadCol;
            else if (A.rank) r.c[q] = A.rank[r.c[q]];
        }
        r.sum += r.w[q];
    }
    return r;
}

// Writes the run's records (P after each edge, target) from the exclusive
// prefix P0, padding records past d included (a row's region is padded to a
// multiple of 4 records, and i0 is a multiple of 4), and its level-1 keys.
__device__ __forceinline__ void write_run(const BuildArgs &A, uint32_t *K, const EdgeRun &r, uint64_t P0, uint64_t sreg,
                                          uint64_t eb, uint32_t d, uint32_t L, uint32_t i0, int64_t base_id)
{
    if (i0 >= d) return;
    uint32_t v[8];
    uint64_t P = P0;
#pragma unroll
    for (uint32_t q = 0; q < kRun; ++q) {
        const uint32_t i = i0 + q;
        P += r.w[q];
        const bool in = i < d;
        v[2 * q] = in ? (uint32_t)P : 0xffffffffu;
        v[2 * q + 1] = in ? (uint32_t)(r.c[q] + base_id) : 0u;
        if (in && ((i & 7) == 7 || i == d - 1)) K[key_slot(sreg, d, L, 1, i >> 3)] = (uint32_t)P;
    }
    uint4 *dst = reinterpret_cast<uint4 *>(A.E + eb + i0);  // 32-byte aligned
    dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
    dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
}

__global__ void __launch_bounds__(256) k_build_small(BuildArgs A)
{
    uint32_t *K = A.K;
    uint32_t flags = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < A.n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = in_row(A, u);
        const int64_t a = A.row_ptr[o];
        const uint32_t d = (uint32_t)(A.row_ptr[o + 1] - a);
        if (d > kSmallRow) {
            if (d <= kMidRow) A.list[atomicAdd(&A.st->n_mid, 1u)] = (uint32_t)u;
            else if (d <= kHugeRow) A.list[A.n - 1 - atomicAdd(&A.st->n_big, 1u)] = (uint32_t)u;
            continue;  // rows above kHugeRow: tile kernels
        }
        int64_t hi_id;
        const int64_t base_id = instance_base(A, u, hi_id);
        uint64_t reg, sreg;
        row_regions(A, u, d, reg, sreg);
        const uint32_t L = tree_levels(d);  // 0 or 1 here
        const uint64_t eb = reg;
        uint64_t P = 0;
        uint32_t first = 0;
        for (uint32_t i = 0; i < d; ++i) {
            const uint32_t wi = A.w[a + i];
            int64_t c = A.col[a + i];
            if (wi == 0) flags |= kBadWeight;
            if (c < 0 || c >= hi_id) flags |= kBadCol;
            else c = map_col(A, c);
            P += wi;
            if (i == 0) first = (uint32_t)(c + base_id);
            if (d >= 2) {
                EdgeN r;
                r.P = (uint32_t)P;
                r.col = (int32_t)(c + base_id);
                A.E[eb + i] = r;
                if (L > 0 && ((i & 7) == 7 || i == d - 1)) K[key_slot(sreg, d, L, 1, i >> 3)] = (uint32_t)P;
            }
        }
        if (P >= (1ull << 32)) flags |= kWide;
        if (d >= 2) {
            for (uint32_t i = d; i < 4 * ceil_shift(d, 2); ++i) {
                EdgeN r;
                r.P = 0xffffffffu;
                r.col = 0;
                A.E[eb + i] = r;
            }
            if (L > 0)
                for (uint32_t i = ceil_shift(d, 3); i < 8 * level_sectors(d, 1); ++i) K[key_slot(sreg, d, L, 1, i)] = 0xffffffffu;
        }
        write_node(A, u, reg, sreg, d, P, first);
    }
    block_stats(A.st, 0, 0, flags);
}

__global__ void __launch_bounds__(256) k_build_mid(BuildArgs A)
{
    uint32_t *K = A.K;
    const uint32_t lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t flags = 0;
    const uint32_t nmid = A.st->n_mid;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nmid; t += warps) {
        const int64_t u = A.list[t];
        const int64_t o = in_row(A, u);
        const int64_t a = A.row_ptr[o];
        const uint32_t d = (uint32_t)(A.row_ptr[o + 1] - a);
        int64_t hi_id;
        const int64_t base_id = instance_base(A, u, hi_id);
        uint64_t reg, sreg;
        row_regions(A, u, d, reg, sreg);
        const uint32_t L = tree_levels(d);
        const uint64_t eb = reg;
        uint64_t carry = 0;
        for (uint32_t e0 = 0; e0 < d; e0 += 32 * kRun) {
            const uint32_t i0 = e0 + lane * kRun;
            const EdgeRun r = load_run(A, a, d, i0, hi_id, flags);
            uint64_t v = r.sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            write_run(A, K, r, carry + v - r.sum, sreg, eb, d, L, i0, base_id);
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (carry >= (1ull << 32)) flags |= kWide;
        for (uint32_t i = ceil_shift(d, 3) + lane; i < 8 * level_sectors(d, 1); i += 32)
            K[key_slot(sreg, d, L, 1, i)] = 0xffffffffu;
        __syncwarp();
        write_upper_levels(K, sreg, d, L, lane, 32, false);
        if (lane == 0) write_node(A, u, reg, sreg, d, carry, 0);
    }
    block_stats(A.st, 0, 0, flags);
}

__global__ void __launch_bounds__(512) k_build_big(BuildArgs A)
{
    __shared__ uint64_t s_warp[16];
    uint32_t *K = A.K;
    const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    uint32_t flags = 0;
    const uint32_t nbig = A.st->n_big;
    for (uint32_t t = blockIdx.x; t < nbig; t += gridDim.x) {
        const int64_t u = A.list[A.n - 1 - t];
        const int64_t o = in_row(A, u);
        const int64_t a = A.row_ptr[o];
        const uint32_t d = (uint32_t)(A.row_ptr[o + 1] - a);
        int64_t hi_id;
        const int64_t base_id = instance_base(A, u, hi_id);
        uint64_t reg, sreg;
        row_regions(A, u, d, reg, sreg);
        const uint32_t L = tree_levels(d);
        const uint64_t eb = reg;
        uint64_t carry = 0;
        for (uint32_t e0 = 0; e0 < d; e0 += blockDim.x * kRun) {
            const uint32_t i0 = e0 + tid * kRun;
            const EdgeRun r = load_run(A, a, d, i0, hi_id, flags);
            uint64_t v = r.sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (lane == 31) s_warp[wid] = v;
            __syncthreads();
            uint64_t before = 0, chunk = 0;
            for (uint32_t q = 0; q < nw; ++q) {
                if (q < wid) before += s_warp[q];
                chunk += s_warp[q];
            }
            write_run(A, K, r, carry + before + v - r.sum, sreg, eb, d, L, i0, base_id);
            carry += chunk;
            __syncthreads();
        }
        if (carry >= (1ull << 32)) flags |= kWide;
        for (uint32_t i = ceil_shift(d, 3) + tid; i < 8 * level_sectors(d, 1); i += blockDim.x)
            K[key_slot(sreg, d, L, 1, i)] = 0xffffffffu;
        __syncthreads();
        write_upper_levels(K, sreg, d, L, tid, blockDim.x, true);
        if (tid == 0) write_node(A, u, reg, sreg, d, carry, 0);
        __syncthreads();
    }
    // one status word per block
    __shared__ uint32_t s_flags;
    if (tid == 0) s_flags = 0;
    __syncthreads();
    if (flags) atomicOr(&s_flags, flags);
    __syncthreads();
    if (tid == 0 && s_flags) atomicOr(&A.st->status, s_flags);
}

// Rows above kHugeRow edges are built by tiles of kBuildTile edges, one block
// each, so a hub row does not leave one block working while the GPU idles:
// tile weight totals, a scan of each row's tiles, tile writes of the prefix
// records and level-1 keys, then one block per row for the padding, the upper
// summary levels and the node record.
struct BuildTiles {
    BuildArgs A;
    const uint4 *rows;   // (node, degree, first tile, tiles)
    const uint2 *tiles;  // (row index, first edge of the tile)
    uint64_t *tile_sum;  // per tile: weight total, then its exclusive offset in the row
    uint64_t *row_total; // per row: W
    uint32_t nrows;
};

__device__ __forceinline__ uint64_t block_sum_u64(uint64_t v, uint64_t *s)  // 256 threads
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    uint64_t t = 0;
    for (int q = 0; q < 8; ++q) t += s[q];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256) k_build_tile_totals(BuildTiles T)
{
    __shared__ uint64_t s[8];
    const BuildArgs &A = T.A;
    const uint2 tl = T.tiles[blockIdx.x];
    const uint4 rw = T.rows[tl.x];
    const int64_t a = A.row_ptr[in_row(A, rw.x)];
    int64_t hi_id;
    instance_base(A, rw.x, hi_id);
    const uint32_t end = min(tl.y + kBuildTile, rw.y);
    const uint32_t lo = min(tl.y + threadIdx.x * 32, end), hi = min(lo + 32, end);
    uint64_t sum = 0;
    uint32_t flags = 0;
    for (uint32_t i = lo; i < hi; ++i) {
        const uint32_t wi = A.w[a + i];
        const int64_t c = A.col[a + i];
        if (wi == 0) flags |= kBadWeight;
        if (c < 0 || c >= hi_id) flags |= kBadCol;
        sum += wi;
    }
    if (flags) atomicOr(&A.st->status, flags);
    const uint64_t t = block_sum_u64(sum, s);
    if (threadIdx.x == 0) T.tile_sum[blockIdx.x] = t;
}

__global__ void k_build_tile_scan(BuildTiles T)
{
    const uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= T.nrows) return;
    const uint32_t lane = threadIdx.x & 31;
    const uint4 rw = T.rows[r];
    uint64_t carry = 0;
    for (uint32_t t0 = 0; t0 < rw.w; t0 += 32) {
        const uint32_t t = t0 + lane;
        uint64_t v = t < rw.w ? T.tile_sum[rw.z + t] : 0ull;
        const uint64_t own = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (t < rw.w) T.tile_sum[rw.z + t] = carry + v - own;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) {
        T.row_total[r] = carry;
        if (carry >= (1ull << 32)) atomicOr(&T.A.st->status, kWide);
    }
}

__global__ void __launch_bounds__(256) k_build_tile_write(BuildTiles T)
{
    __shared__ uint64_t s[8];
    const BuildArgs &A = T.A;
    uint32_t *K = A.K;
    const uint2 tl = T.tiles[blockIdx.x];
    const uint4 rw = T.rows[tl.x];
    const uint32_t d = rw.y;
    const int64_t a = A.row_ptr[in_row(A, rw.x)];
    int64_t hi_id;
    const int64_t base_id = instance_base(A, rw.x, hi_id);
    uint64_t reg, sreg;
    row_regions(A, rw.x, d, reg, sreg);
    const uint32_t L = tree_levels(d);
    const uint64_t eb = reg;
    const uint32_t end = min(tl.y + kBuildTile, d);
    const uint32_t lo = min(tl.y + threadIdx.x * 32, end), hi = min(lo + 32, end);
    uint64_t own = 0;
    for (uint32_t i = lo; i < hi; ++i) own += A.w[a + i];
    // exclusive offset of this thread's run within the tile
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t v = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s[wid] = v;
    __syncthreads();
    uint64_t before = 0;
    for (uint32_t q = 0; q < wid; ++q) before += s[q];
    uint64_t P = T.tile_sum[blockIdx.x] + before + v - own;
    for (uint32_t i = lo; i < hi; ++i) {
        P += A.w[a + i];
        const int64_t c = A.col[a + i];  // checked by k_build_tile_totals (the build fails if it is out of range)
        EdgeN r;
        r.P = (uint32_t)P;
        r.col = (int32_t)((c >= 0 && c < hi_id ? map_col(A, c) : c) + base_id);
        A.E[eb + i] = r;
        if ((i & 7) == 7 || i == d - 1) K[key_slot(sreg, d, L, 1, i >> 3)] = (uint32_t)P;
    }
}

__global__ void __launch_bounds__(512) k_build_tile_finish(BuildTiles T)
{
    const BuildArgs &A = T.A;
    uint32_t *K = A.K;
    const uint4 rw = T.rows[blockIdx.x];
    const uint32_t d = rw.y, tid = threadIdx.x;
    uint64_t reg, sreg;
    row_regions(A, rw.x, d, reg, sreg);
    const uint32_t L = tree_levels(d);
    const uint64_t eb = reg;
    for (uint32_t i = d + tid; i < 4 * ceil_shift(d, 2); i += blockDim.x) {
        EdgeN r;
        r.P = 0xffffffffu;
        r.col = 0;
        A.E[eb + i] = r;
    }
    for (uint32_t i = ceil_shift(d, 3) + tid; i < 8 * level_sectors(d, 1); i += blockDim.x)
        K[key_slot(sreg, d, L, 1, i)] = 0xffffffffu;
    __syncthreads();
    write_upper_levels(K, sreg, d, L, tid, blockDim.x, true);
    if (tid == 0) write_node(A, rw.x, reg, sreg, d, T.row_total[blockIdx.x], 0);
}

// Narrow layout in one pass.  Returns PPR_OK, an error, or 1 when a row total
// reaches 2^32 (the caller then builds the wide layout).
static int build_narrow(ppr_ctx *ctx, int64_t n, int64_t m, const int64_t *d_rp, const int32_t *d_col,
                        const uint32_t *d_w, const int64_t *d_off, cudaStream_t st, ppr_graph *g,
                        std::vector<void *> &tmp)
{
    int rc;
    uint32_t *d_sizes, *d_ssizes;
    uint64_t *d_region, *d_sregion, *d_scan;
    LayoutStats *d_ls;
    uint32_t *d_list;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if ((rc = dev_alloc((void **)&d_sizes, sizeof(uint32_t) * n, "row sizes", st))) return rc;
    tmp.push_back(d_sizes);
    if ((rc = dev_alloc((void **)&d_region, sizeof(uint64_t) * (n + 1), "row regions", st))) return rc;
    tmp.push_back(d_region);
    if ((rc = dev_alloc((void **)&d_ssizes, sizeof(uint32_t) * n, "summary sizes", st))) return rc;
    tmp.push_back(d_ssizes);
    if ((rc = dev_alloc((void **)&d_sregion, sizeof(uint64_t) * (n + 1), "summary regions", st))) return rc;
    tmp.push_back(d_sregion);
    if ((rc = dev_alloc((void **)&d_scan, sizeof(uint64_t) * (tiles + 2), "scan scratch", st))) return rc;
    tmp.push_back(d_scan);
    if ((rc = dev_alloc((void **)&d_ls, sizeof(LayoutStats), "layout stats", st))) return rc;
    tmp.push_back(d_ls);
    if ((rc = dev_alloc((void **)&d_list, sizeof(uint32_t) * n, "long-row list", st))) return rc;
    tmp.push_back(d_list);
    const uint32_t huge_cap = (uint32_t)(m / kHugeRow + 1);
    uint2 *d_huge;
    if ((rc = dev_alloc((void **)&d_huge, sizeof(uint2) * huge_cap, "huge-row list", st))) return rc;
    tmp.push_back(d_huge);
    cudaError_t e = cudaMemsetAsync(d_ls, 0, sizeof(LayoutStats), st);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    const int tblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->sms * 16));
    // Summary levels in an array of their own on a renumbered layout (graphs
    // far larger than L2: the summaries every draw passes through then pack
    // L2 lines instead of sharing them with blocks a draw reads once); at the
    // start of each row's area, before its blocks, otherwise (the summary
    // sector of a small row shares a DRAM page with its blocks).  The record's
    // 28-bit summary offset bounds the shared area: 2 m + 4 n records cover
    // every row's blocks and summary.
    const bool interleave = g->order == nullptr && (uint64_t)(2 * m + 4 * n) / 4 < kSumSectorsMax;
    k_layout<<<tblocks, 256, 0, st>>>(n, m, d_rp, g->order, interleave, d_sizes, d_ssizes, d_ls, d_huge, huge_cap);
    note_launch();
    exclusive_scan_u32(d_sizes, n, d_region, d_scan, st);
    if (!interleave) exclusive_scan_u32(d_ssizes, n, d_sregion, d_scan, st);  // same scratch, in stream order
    LayoutStats hs;
    uint64_t slots = 0, sum_sectors = 0;
    e = cudaMemcpyAsync(&hs, d_ls, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&slots, d_region + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !interleave)
        e = cudaMemcpyAsync(&sum_sectors, d_sregion + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "graph layout");
    if (hs.status & kBadRowPtr) {
        set_error("row_ptr must start at 0, be non-decreasing and end at m");
        return PPR_EINVAL;
    }
    if (hs.status & kBigDegree) {
        set_error("an out-degree exceeds the limit %lld", (long long)PPR_MAX_DEGREE);
        return PPR_ERANGE;
    }
    if (slots > kBeginMask) {
        set_error("edge layout needs %llu record slots, beyond 2^40", (unsigned long long)slots);
        return PPR_ERANGE;
    }
    if (sum_sectors >= kSumSectorsMax) {
        set_error("the rows' search-tree summaries need %llu sectors, beyond 2^28", (unsigned long long)sum_sectors);
        return PPR_ERANGE;
    }
    g->max_degree = (int64_t)hs.max_degree;
    g->dangling = (int64_t)hs.dangling;
    if ((rc = dev_alloc((void **)&g->node, sizeof(NodeRecN) * n, "node records", st))) return rc;
    const size_t edge_bytes = (size_t)(slots > 0 ? slots : 2) * sizeof(EdgeN);
    if ((rc = dev_alloc(&g->edges, edge_bytes, "edge records", st))) return rc;
    g->edge_records = (int64_t)slots;
    size_t sum_bytes = 0;
    if (!interleave) {
        sum_bytes = (size_t)(sum_sectors > 0 ? sum_sectors : 1) * 32;
        if ((rc = dev_alloc((void **)&g->sum, sum_bytes, "row summaries", st))) return rc;
        g->sum_sectors = (int64_t)sum_sectors;
    }
    g->device_bytes = (int64_t)(sizeof(NodeRecN) * n + edge_bytes + sum_bytes);
    BuildArgs A{n, d_rp, d_col, d_w, d_off, g->instances, d_region, interleave ? nullptr : d_sregion,
                static_cast<NodeRecN *>(g->node), (EdgeN *)g->edges,
                interleave ? reinterpret_cast<uint32_t *>(g->edges) : g->sum, d_ls, d_list, g->order, g->rank};
    k_build_small<<<tblocks, 256, 0, st>>>(A);
    note_launch();
    k_build_mid<<<ctx->sms * 8, 256, 0, st>>>(A);
    note_launch();
    k_build_big<<<ctx->sms * 3, 512, 0, st>>>(A);  // three resident 512-thread blocks per SM (39 registers)
    note_launch();
    std::vector<uint4> hrows;  // host tables must outlive their uploads (synchronised below)
    std::vector<uint2> htiles;
    if (hs.n_huge > 0) {
        const uint32_t nh = std::min(hs.n_huge, huge_cap);
        std::vector<uint2> hl(nh);
        e = cudaMemcpyAsync(hl.data(), d_huge, sizeof(uint2) * nh, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "huge rows");
        for (uint32_t r = 0; r < nh; ++r) {
            const uint32_t d = hl[r].y, nt = (d + kBuildTile - 1) / kBuildTile;
            hrows.push_back(make_uint4(hl[r].x, d, (uint32_t)htiles.size(), nt));
            for (uint32_t t = 0; t < nt; ++t) htiles.push_back(make_uint2(r, t * kBuildTile));
        }
        const uint32_t nt = (uint32_t)htiles.size();
        uint4 *d_rows;
        uint2 *d_tiles;
        uint64_t *d_tsum, *d_rtot;
        if ((rc = dev_alloc((void **)&d_rows, sizeof(uint4) * nh, "huge rows", st))) return rc;
        tmp.push_back(d_rows);
        if ((rc = dev_alloc((void **)&d_tiles, sizeof(uint2) * nt, "tile table", st))) return rc;
        tmp.push_back(d_tiles);
        if ((rc = dev_alloc((void **)&d_tsum, sizeof(uint64_t) * nt, "tile sums", st))) return rc;
        tmp.push_back(d_tsum);
        if ((rc = dev_alloc((void **)&d_rtot, sizeof(uint64_t) * nh, "row totals", st))) return rc;
        tmp.push_back(d_rtot);
        e = cudaMemcpyAsync(d_rows, hrows.data(), sizeof(uint4) * nh, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_tiles, htiles.data(), sizeof(uint2) * nt, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "tile table upload");
        BuildTiles T{A, d_rows, d_tiles, d_tsum, d_rtot, nh};
        k_build_tile_totals<<<nt, 256, 0, st>>>(T);
        note_launch();
        k_build_tile_scan<<<(nh + 7) / 8, 256, 0, st>>>(T);
        note_launch();
        k_build_tile_write<<<nt, 256, 0, st>>>(T);
        note_launch();
        k_build_tile_finish<<<nh, 512, 0, st>>>(T);
        note_launch();
    }
    e = cudaMemcpyAsync(&hs, d_ls, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "graph build");
    if (hs.status & kBadCol) {
        set_error("an edge target is outside [0, n) (of its instance)");
        return PPR_EINVAL;
    }
    if (hs.status & kBadWeight) {
        set_error("edge weights must be >= 1 (w(e) > 0, Sec. 2.1)");
        return PPR_EINVAL;
    }
    if (hs.status & kWide) {
        dev_free(g->node, st);
        dev_free(g->edges, st);
        dev_free(g->sum, st);
        g->node = nullptr;
        g->edges = nullptr;
        g->sum = nullptr;
        g->sum_sectors = 0;
        return 1;
    }
    return PPR_OK;
}

int build_graph(ppr_ctx *ctx, int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                const uint32_t *w, bool device_ptrs, bool renumber, cudaStream_t st, ppr_graph *g)
{
    const int64_t *d_rp = row_ptr;
    const int32_t *d_col = col;
    const uint32_t *d_w = w;
    std::vector<void *> tmp;
    auto cleanup = [&]() {
        for (void *p : tmp) dev_free(p, st);
        tmp.clear();
    };
    int rc;
    if (!device_ptrs) {
        void *p;
        if ((rc = dev_alloc(&p, sizeof(int64_t) * (n + 1), "row_ptr copy", st))) return cleanup(), rc;
        tmp.push_back(p);
        d_rp = (const int64_t *)p;
        if (m > 0) {
            if ((rc = dev_alloc(&p, sizeof(int32_t) * m, "col copy", st))) return cleanup(), rc;
            tmp.push_back(p);
            d_col = (const int32_t *)p;
            if ((rc = dev_alloc(&p, sizeof(uint32_t) * m, "w copy", st))) return cleanup(), rc;
            tmp.push_back(p);
            d_w = (const uint32_t *)p;
        }
        cudaError_t e = cudaMemcpyAsync((void *)d_rp, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && m > 0)
            e = cudaMemcpyAsync((void *)d_col, col, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && m > 0)
            e = cudaMemcpyAsync((void *)d_w, w, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cleanup(), cuda_fail(e, "graph upload");
    }
    int64_t *d_off = nullptr;
    if (g->instances > 0) {  // kept with the graph: the walker reads instance offsets
        if ((rc = dev_alloc((void **)&g->d_node_off, sizeof(int64_t) * (g->instances + 1), "node_off", st)))
            return cleanup(), rc;
        d_off = g->d_node_off;
        cudaError_t e = cudaMemcpyAsync(d_off, g->node_off.data(), sizeof(int64_t) * (g->instances + 1),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cleanup(), cuda_fail(e, "node_off upload");
    }
    if (renumber && g->instances == 0) {
        if ((rc = dev_alloc((void **)&g->order, sizeof(int32_t) * n, "node order", st)) ||
            (rc = dev_alloc((void **)&g->rank, sizeof(int32_t) * n, "node rank", st)) ||
            (rc = renumber_by_indegree(ctx, n, m, d_col, st, g->order, g->rank, tmp)))
            return cleanup(), rc;
        g->device_bytes_extra = (int64_t)(2 * sizeof(int32_t) * n);
    }
    rc = build_narrow(ctx, n, m, d_rp, d_col, d_w, d_off, st, g, tmp);
    if (rc != 1) {
        if (rc == PPR_OK) g->device_bytes += g->device_bytes_extra;
        cleanup();
        return rc;
    }
    // the wide layout keeps the caller's numbering
    dev_free(g->order, st);
    dev_free(g->rank, st);
    g->order = g->rank = nullptr;
    g->device_bytes_extra = 0;
    // some row total reaches 2^32: 64-bit prefixes in flat rows
    void *p;
    if ((rc = dev_alloc(&p, sizeof(uint64_t) * n, "row totals", st))) return cleanup(), rc;
    tmp.push_back(p);
    uint64_t *d_W = (uint64_t *)p;
    if ((rc = dev_alloc(&p, sizeof(BuildStats), "build stats", st))) return cleanup(), rc;
    tmp.push_back(p);
    BuildStats *d_st = (BuildStats *)p;
    cudaError_t e = cudaMemsetAsync(d_st, 0, sizeof(BuildStats), st);
    if (e != cudaSuccess) return cleanup(), cuda_fail(e, "memset");

    const int threads = 256;
    int64_t want_blocks = (n + 7) / 8;
    int blocks = (int)std::min<int64_t>(want_blocks, (int64_t)ctx->sms * 64);
    if (blocks < 1) blocks = 1;
    k_rows_pass1<<<blocks, threads, 0, st>>>(n, m, d_rp, d_col, d_w, d_off, g->instances, d_W, d_st);
    note_launch();
    BuildStats hs;
    e = cudaMemcpyAsync(&hs, d_st, sizeof(BuildStats), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(), cuda_fail(e, "graph validation");
    if (hs.status & kBadRowPtr) {
        set_error("row_ptr must start at 0, be non-decreasing and end at m");
        return cleanup(), PPR_EINVAL;
    }
    if (hs.status & kBadCol) {
        set_error("an edge target is outside [0, n) (of its instance)");
        return cleanup(), PPR_EINVAL;
    }
    if (hs.status & kBadWeight) {
        set_error("edge weights must be >= 1 (w(e) > 0, Sec. 2.1)");
        return cleanup(), PPR_EINVAL;
    }
    if ((int64_t)hs.max_degree > PPR_MAX_DEGREE) {
        set_error("out-degree %llu exceeds the limit %lld", hs.max_degree, (long long)PPR_MAX_DEGREE);
        return cleanup(), PPR_ERANGE;
    }
    g->wide = true;
    g->max_degree = (int64_t)hs.max_degree;
    g->dangling = (int64_t)hs.dangling;
    if ((rc = dev_alloc((void **)&g->node, sizeof(NodeRec) * n, "node records", st))) return cleanup(), rc;
    {
        size_t edge_bytes = (size_t)m * sizeof(EdgeW);
        if ((rc = dev_alloc(&g->edges, edge_bytes > 0 ? edge_bytes : 16, "edge records", st))) return cleanup(), rc;
        g->edge_records = m;
        g->device_bytes = (int64_t)(sizeof(NodeRec) * n + edge_bytes);
        k_rows_pass2<true><<<blocks, threads, 0, st>>>(n, d_rp, d_col, d_w, d_off, g->instances, d_W,
                                                       static_cast<NodeRec *>(g->node), g->edges);
        note_launch();
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "graph build");
    return PPR_OK;
}

// ------------------------------------------------------------ segments ----

constexpr int kSegMaxDeg = 8;
constexpr int kSegMaxOut = 64;

__device__ __forceinline__ uint64_t mul_shift32(uint64_t q, uint32_t f)
{
    // floor(q * f / 2^32), q < 2^63
    uint64_t lo = q * (uint64_t)f;
    uint64_t hi = __umul64hi(q, (uint64_t)f);
    return (hi << 32) | (lo >> 32);
}

__device__ __forceinline__ uint64_t mul_div(uint64_t q, uint64_t num, uint64_t den)
{
    unsigned __int128 p = (unsigned __int128)q * num;
    return (uint64_t)(p / den);
}

template <class E>
struct RowView {
    const typename E::Node *node;
    E edges;
    __device__ __forceinline__ uint32_t deg(uint32_t u) const { return (uint32_t)(node[u].word0 >> 40) & kCountMask; }
    __device__ __forceinline__ uint64_t begin(uint32_t u) const { return node[u].word0 & kBeginMask; }
    // row total = last inclusive prefix (the node record holds the target of a
    // single-edge row instead of its total)
    __device__ __forceinline__ uint64_t total(uint32_t u) const
    {
        uint32_t d = deg(u);
        if (d == 1) return 1;  // with wt = 1 above: the single edge has ratio 1
        return d ? E::key(edges.load(E::edge_base(begin(u), d) + d - 1)) : 0ull;
    }
    // weight and target of the i-th edge of u
    __device__ __forceinline__ void edge(uint32_t u, uint32_t i, uint64_t &wt, uint32_t &tgt) const
    {
        const uint32_t d = deg(u);
        if (d == 1) {  // target kept in the node record; weight ratio is 1
            wt = 1;
            tgt = (uint32_t)node[u].total;
            return;
        }
        uint64_t b = E::edge_base(begin(u), d);
        auto r = edges.load(b + i);
        uint64_t prev = i > 0 ? E::key(edges.load(b + i - 1)) : 0ull;
        wt = E::key(r) - prev;
        tgt = E::target(r);
    }
};

// Segment tables in two passes.  k_seg_scan (every node; a warp takes 32 at a
// time) copies the plain record into the segment record array, tests the
// depth-1 shape of all 32 nodes at once (degree <= 8 of the node and of its
// targets), then for each candidate left the depth-2 shape, and counts the
// raw contributions the path enumeration will make; eligible nodes are listed
// by that count (one reservation per warp and tier), with min(raw, 64)
// entries each, whose scan gives every listed node a fixed slot range.
// k_seg_fill (one warp per listed node) enumerates the paths once, level by
// level, sums equal outcomes in a shared-memory hash table, drops zero
// masses, rejects a node with more than 64 outcomes, puts the rest in
// canonical order (terminated before active, then node, then length) by
// ranking, and writes the table at the node's slot.  A table's place in the
// entry array is free (its record holds begin and count; a shorter table
// leaves a gap), so only its content is fixed.

constexpr unsigned long long kSegEmpty = ~0ull;  // free hash slot (an outcome key's node field is below 2^31)
constexpr uint32_t kSegSmallRaw = 128;  // raw contributions up to which the small table (256 slots) serves
constexpr int kSegLargeSlots = 2048;    // the largest raw count is 8 * (1 + 8 * (1 + 2 * 8)) = 1,096

struct SegCounters {
    unsigned int listed[2];       // nodes listed: [0] small table, [1] large table
    unsigned long long bound;     // sum over listed nodes of min(raw, 64): entries to allocate
    unsigned long long used;      // entries written
    unsigned long long tables;    // nodes given a table
};

// Path enumeration by level: depth-1 targets, then the pairs (i1, i2).
struct SegStage {
    unsigned long long s1_q[kSegMaxDeg], s1_W[kSegMaxDeg];
    unsigned long long s2_q[kSegMaxDeg * kSegMaxDeg], s2_W[kSegMaxDeg * kSegMaxDeg];
    uint32_t s1_node[kSegMaxDeg], s1_deg[kSegMaxDeg];
    uint32_t s2_node[kSegMaxDeg * kSegMaxDeg], s2_deg[kSegMaxDeg * kSegMaxDeg], s2_pre[kSegMaxDeg * kSegMaxDeg + 1];
};

// Compacted, then ranked outcomes; so: the keys with the caller's node ids
// (ranking on a renumbered layout).
struct SegRank {
    unsigned long long sk[kSegMaxOut], sq[kSegMaxOut], so[kSegMaxOut];
};

// Hash table of one warp: more slots than the tier's largest raw count, so it never fills.
template <int SLOTS>
struct SegHash {
    unsigned long long key[SLOTS];
    unsigned long long val[SLOTS];
    uint16_t used[SLOTS];          // claimed slots, in claim order
    union {  // one node at a time: the enumeration's staging, then the ranking's outcomes
        SegStage e;
        SegRank r;
    } u;
    unsigned int count;
    unsigned int full;  // a probe found no slot (cannot happen when the scan's count is right): no table
};

// list: listed nodes, small tier from the front, large from the back;
// lbound[list position]: min(raw contributions, 64), the entries the node's
// table may take (its slot range in the entry array comes from a scan of these).
template <class E>
__global__ void __launch_bounds__(256) k_seg_scan(RowView<E> G, int64_t n, typename E::Node *seg_node, uint32_t *list,
                                                  uint32_t *lbound, SegCounters *ct)
{
    const uint32_t lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // each warp takes 32 consecutive nodes (coalesced record copy and degree
    // test), then examines the candidates among them one by one with all lanes
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const int64_t vl = base + lane;
        uint32_t dl = 0;
        bool c = false;
        if (vl < n) {
            const typename E::Node r = G.node[vl];
            seg_node[vl] = r;  // plain record unless a table replaces it
            dl = (uint32_t)(r.word0 >> 40) & kCountMask;
            // depth 1, every lane its own node at once (most candidates have
            // a neighbour above the limit): the row's targets, then their degrees
            c = dl >= 1 && dl <= (uint32_t)kSegMaxDeg;
            if (c) {
                uint32_t tg[kSegMaxDeg];
                const uint64_t eb = E::edge_base(r.word0 & kBeginMask, dl);
#pragma unroll
                for (uint32_t i = 0; i < (uint32_t)kSegMaxDeg; ++i)
                    tg[i] = i >= dl ? 0u : (dl == 1 ? (uint32_t)r.total : E::target(G.edges.load(eb + i)));
#pragma unroll
                for (uint32_t i = 0; i < (uint32_t)kSegMaxDeg; ++i)
                    if (i < dl && G.deg(tg[i]) > (uint32_t)kSegMaxDeg) c = false;
            }
        }
        uint32_t cand = __ballot_sync(0xffffffffu, c);
        uint32_t listed_mask[2] = {0u, 0u}, my_bound = 0;  // this group's listed nodes (lane = node), per tier
        while (cand) {
            const uint32_t src_lane = __ffs(cand) - 1;
            cand &= cand - 1;
            const uint32_t v = (uint32_t)(base + src_lane);
            const uint32_t d1 = __shfl_sync(0xffffffffu, dl, src_lane);
            bool ok = true;
            uint32_t raw = 0;
            for (uint32_t p = lane; p < d1 * kSegMaxDeg; p += 32) {
                const uint32_t i1 = p / kSegMaxDeg, i2 = p % kSegMaxDeg;
                uint64_t wt;
                uint32_t a;
                G.edge(v, i1, wt, a);
                const uint32_t da = G.deg(a);
                if (da > (uint32_t)kSegMaxDeg) {
                    ok = false;
                    continue;
                }
                if (i2 == 0) raw += 1 + (da == 0);  // (a, terminated), and (a, active, 1) at a dead end
                if (i2 < da) {
                    uint32_t b;
                    G.edge(a, i2, wt, b);
                    const uint32_t db = G.deg(b);
                    if (db > (uint32_t)kSegMaxDeg) ok = false;
                    else raw += 1 + (db == 0) + 2 * db;  // (b, terminated), dead end, both outcomes at each c
                }
            }
            if (!__all_sync(0xffffffffu, ok)) continue;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) raw += __shfl_xor_sync(0xffffffffu, raw, o);
            listed_mask[raw <= kSegSmallRaw ? 0 : 1] |= 1u << src_lane;
            if (lane == src_lane) my_bound = min(raw, (uint32_t)kSegMaxOut);
        }
        // one reservation per tier for the group's listed nodes (not one
        // atomic per node: every warp would queue on the same counters)
        uint32_t res[2] = {0u, 0u};
        unsigned long long bsum = my_bound;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
        if (lane == 0) {
            if (listed_mask[0]) res[0] = atomicAdd(&ct->listed[0], (uint32_t)__popc(listed_mask[0]));
            if (listed_mask[1]) res[1] = atomicAdd(&ct->listed[1], (uint32_t)__popc(listed_mask[1]));
            if (bsum) atomicAdd(&ct->bound, bsum);
        }
        res[0] = __shfl_sync(0xffffffffu, res[0], 0);
        res[1] = __shfl_sync(0xffffffffu, res[1], 0);
#pragma unroll
        for (int tier = 0; tier < 2; ++tier) {
            if ((listed_mask[tier] >> lane) & 1u) {
                const uint32_t k = res[tier] + __popc(listed_mask[tier] & ((1u << lane) - 1));
                const int64_t pos = tier ? n - 1 - k : k;  // small tier from the front, large from the back
                list[pos] = (uint32_t)vl;
                lbound[pos] = my_bound;
            }
        }
    }
}

template <int SLOTS>
__device__ __forceinline__ void seg_insert(SegHash<SLOTS> *h, uint32_t node, uint32_t active, uint32_t len, uint64_t q)
{
    const unsigned long long key = ((unsigned long long)active << 63) | ((unsigned long long)node << 8) | len;
    uint32_t s = (node * 0x9E3779B1u ^ (len << 29) ^ (active << 31)) & (SLOTS - 1);
    for (uint32_t probe = 0; probe < (uint32_t)SLOTS; ++probe) {
        const unsigned long long prev = atomicCAS(&h->key[s], kSegEmpty, key);
        if (prev == kSegEmpty) h->used[atomicAdd(&h->count, 1u)] = (uint16_t)s;  // each claim takes a new slot
        if (prev == kSegEmpty || prev == key) {
            atomicAdd(&h->val[s], (unsigned long long)q);
            return;
        }
        s = (s + 1) & (SLOTS - 1);
    }
    h->full = 1;
}

// Tables of the nodes of one tier of `list`; SLOTS is above the tier's
// largest raw count.  Each warp's hash table is cleared once and restored
// slot by slot after each node.
// An outcome key with its node field replaced by the caller's id of that node.
__device__ __forceinline__ unsigned long long seg_key_caller(unsigned long long k, const int32_t *order)
{
    const uint32_t node = (uint32_t)((k >> 8) & 0x7fffffffull);
    return (k & ~(0x7fffffffull << 8)) | ((unsigned long long)(uint32_t)order[node] << 8);
}

// order: the renumbered layout's order array (the canonical order ranks
// outcomes by the caller's node ids), or null.
// slot: first entry of the table of list position pos (exclusive scan of
// lbound), so a table is written without a shared counter.
template <class E, int SLOTS, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_seg_fill(RowView<E> G, uint32_t T, const uint32_t *list, int tier,
                                                         int64_t n, SegCounters *ct, SegEntry *ent,
                                                         typename E::Node *seg_node, const int32_t *order,
                                                         const uint64_t *slot)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SegHash<SLOTS> *h = reinterpret_cast<SegHash<SLOTS> *>(smem_raw) + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31, below = (1u << lane) - 1;
    for (uint32_t i = lane; i < (uint32_t)SLOTS; i += 32) {
        h->key[i] = kSegEmpty;
        h->val[i] = 0;
    }
    if (lane == 0) {
        h->count = 0;
        h->full = 0;
    }
    __syncwarp();
    const uint32_t listed = ct->listed[tier];
    const uint32_t cont = (uint32_t)(0x100000000ull - T);  // 2^32 - T, T >= 1
    const int64_t warps = (int64_t)gridDim.x * WARPS;
    unsigned long long w_used = 0, w_tables = 0;  // this warp's tables and their entries
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < listed; t += warps) {
        const uint32_t v = list[tier ? n - 1 - t : t];
        const uint32_t d1 = G.deg(v);
        const uint64_t Wv = G.total(v);
        // all paths of length 1, 2, 3, level by level (the paper's masses in
        // 2^62 fixed point, the same arithmetic as the oracle's): the d1 edges
        // of v, then the pairs (i1, i2), then the triples, each level's
        // targets, masses and row totals staged in shared memory so that a
        // level costs one round of dependent loads for all its paths
        if (lane < d1) {
            uint64_t w1;
            uint32_t a;
            G.edge(v, lane, w1, a);
            const uint64_t q1 = mul_div(1ull << 62, w1, Wv);
            const uint32_t da = G.deg(a);
            seg_insert(h, a, 0, 0, mul_shift32(q1, T));
            if (da == 0) seg_insert(h, a, 1, 1, mul_shift32(q1, cont));
            h->u.e.s1_node[lane] = a;
            h->u.e.s1_deg[lane] = da;
            h->u.e.s1_q[lane] = mul_shift32(q1, cont);  // the mass that continues past a
            h->u.e.s1_W[lane] = da ? G.total(a) : 1ull;
        }
        __syncwarp();
        const uint32_t np = d1 * kSegMaxDeg;  // pair slots (i1, i2), i2 < deg(a_i1) valid
        for (uint32_t p = lane; p < np; p += 32) {
            const uint32_t i1 = p / kSegMaxDeg, i2 = p % kSegMaxDeg;
            uint32_t db = 0;
            if (i2 < h->u.e.s1_deg[i1]) {
                uint64_t w2;
                uint32_t b;
                G.edge(h->u.e.s1_node[i1], i2, w2, b);
                const uint64_t q2 = mul_div(h->u.e.s1_q[i1], w2, h->u.e.s1_W[i1]);
                db = G.deg(b);
                seg_insert(h, b, 0, 0, mul_shift32(q2, T));
                if (db == 0) seg_insert(h, b, 1, 2, mul_shift32(q2, cont));
                h->u.e.s2_node[p] = b;
                h->u.e.s2_q[p] = mul_shift32(q2, cont);
                h->u.e.s2_W[p] = db ? G.total(b) : 1ull;
            }
            h->u.e.s2_deg[p] = db;
        }
        __syncwarp();
        // triples packed: pair p owns [pre[p], pre[p + 1])
        uint32_t n3 = 0;  // triples
        for (uint32_t p0 = 0; p0 < np; p0 += 32) {
            uint32_t x = p0 + lane < np ? h->u.e.s2_deg[p0 + lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (p0 + lane < np) h->u.e.s2_pre[p0 + lane + 1] = n3 + x;
            n3 += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) h->u.e.s2_pre[0] = 0;
        __syncwarp();
        for (uint32_t t3 = lane; t3 < n3; t3 += 32) {
            uint32_t lo = 0, hi = np;  // the pair p with pre[p] <= t3 < pre[p + 1]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (h->u.e.s2_pre[mid] <= t3) lo = mid;
                else hi = mid;
            }
            uint64_t w3;
            uint32_t c;
            G.edge(h->u.e.s2_node[lo], t3 - h->u.e.s2_pre[lo], w3, c);
            const uint64_t q3 = mul_div(h->u.e.s2_q[lo], w3, h->u.e.s2_W[lo]);
            seg_insert(h, c, 0, 0, mul_shift32(q3, T));
            seg_insert(h, c, 1, 3, mul_shift32(q3, cont));
        }
        __syncwarp();
        // outcomes of nonzero mass, compacted (the first 64 kept); slots restored
        const uint32_t D = h->count;
        uint32_t K = 0;
        for (uint32_t i0 = 0; i0 < D; i0 += 32) {
            const uint32_t i = i0 + lane;
            unsigned long long k = 0, q = 0;
            if (i < D) {
                const uint32_t s = h->used[i];
                k = h->key[s];
                q = h->val[s];
                h->key[s] = kSegEmpty;
                h->val[s] = 0;
            }
            const bool nzero = i < D && q > 0;
            const uint32_t m = __ballot_sync(0xffffffffu, nzero);
            const uint32_t pos = K + __popc(m & below);
            if (nzero && pos < (uint32_t)kSegMaxOut) {
                h->u.r.sk[pos] = k;
                h->u.r.sq[pos] = q;
            }
            K += __popc(m);
        }
        const bool full = h->full != 0;
        __syncwarp();
        if (lane == 0) {
            h->count = 0;
            h->full = 0;
        }
        if (K == 0 || K > (uint32_t)kSegMaxOut || full) {  // no table: the plain record stays
            __syncwarp();
            continue;
        }
        // canonical order: rank of each key among the K distinct keys (node
        // ids as the caller numbers them)
        unsigned long long mk[2], mq[2], mo[2];
        uint32_t rk[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t i = (uint32_t)e * 32 + lane;
            mk[e] = i < K ? h->u.r.sk[i] : ~0ull;
            mq[e] = i < K ? h->u.r.sq[i] : 0ull;
            mo[e] = (order && i < K) ? seg_key_caller(mk[e], order) : mk[e];
            if (order && i < K) h->u.r.so[i] = mo[e];
        }
        __syncwarp();
        const unsigned long long *cmp = order ? h->u.r.so : h->u.r.sk;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            uint32_t r = 0;
            for (uint32_t j = 0; j < K; ++j) r += cmp[j] < mo[e];
            rk[e] = r;
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if ((uint32_t)e * 32 + lane < K) {
                h->u.r.sk[rk[e]] = mk[e];
                h->u.r.sq[rk[e]] = mq[e];
            }
        __syncwarp();
        // inclusive prefix of the masses in that order
        unsigned long long cum[2];
        unsigned long long carry = 0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t i = (uint32_t)e * 32 + lane;
            unsigned long long x = i < K ? h->u.r.sq[i] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            cum[e] = carry + x;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        const unsigned long long base = slot[tier ? n - 1 - t : t];
        w_used += K;
        ++w_tables;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t i = (uint32_t)e * 32 + lane;
            if (i < K) {
                const unsigned long long k = h->u.r.sk[i];
                SegEntry se;
                se.cum = cum[e];
                se.node = (uint32_t)((k >> 8) & 0x7fffffffull);
                se.mark_len = ((uint32_t)(k >> 63) << 8) | (uint32_t)(k & 0xff);
                ent[base + i] = se;
            }
        }
        if (lane == 0) {
            typename E::Node r = G.node[v];  // a NodeRecN keeps its (unused) top-level keys
            r.word0 = pack_word0(base, K, true);
            r.total = carry;  // Q_v, the table's total mass
            seg_node[v] = r;
        }
        __syncwarp();
    }
    if (lane == 0 && w_tables) {
        atomicAdd(&ct->used, w_used);
        atomicAdd(&ct->tables, w_tables);
    }
}

template <class E>
static int seg_build_typed(ppr_graph *g, uint32_t T, cudaStream_t st, const RowView<E> &G, uint32_t *list,
                           SegCounters *d_ct)
{
    const int64_t n = g->n;
    typename E::Node *seg_node = static_cast<typename E::Node *>(g->seg.node);
    uint32_t *lbound = nullptr;
    uint64_t *slot = nullptr, *scan_tmp = nullptr;
    auto done = [&](int code) {
        dev_free(lbound, st);
        dev_free(slot, st);
        dev_free(scan_tmp, st);
        return code;
    };
    int rc;
    if ((rc = dev_alloc((void **)&lbound, sizeof(uint32_t) * n, "segment bounds", st)) ||
        (rc = dev_alloc((void **)&slot, sizeof(uint64_t) * (n + 1), "segment slots", st)) ||
        (rc = dev_alloc((void **)&scan_tmp, sizeof(uint64_t) * ((n + kScanTile - 1) / kScanTile + 2), "scan scratch",
                        st)))
        return done(rc);
    cudaError_t e = cudaMemsetAsync(lbound, 0, sizeof(uint32_t) * n, st);  // unlisted positions take no entries
    if (e != cudaSuccess) return done(cuda_fail(e, "memset"));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g->ctx->sms * 16));
    k_seg_scan<E><<<blocks, 256, 0, st>>>(G, n, seg_node, list, lbound, d_ct);
    note_launch();
    exclusive_scan_u32(lbound, n, slot, scan_tmp, st);  // each listed node's slot range in the entry array
    SegCounters hc;
    e = cudaMemcpyAsync(&hc, d_ct, sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "segment scan"));
    if ((rc = dev_alloc((void **)&g->seg.entries, sizeof(SegEntry) * (hc.bound > 0 ? hc.bound : 1), "segment tables",
                        st)))
        return done(rc);
    if (hc.listed[0]) {
        constexpr int W = 8;
        const size_t smem = sizeof(SegHash<2 * kSegSmallRaw>) * W;
        e = cudaFuncSetAttribute(k_seg_fill<E, 2 * kSegSmallRaw, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return done(cuda_fail(e, "cudaFuncSetAttribute(k_seg_fill)"));
        const int fb = (int)std::min<int64_t>((hc.listed[0] + W - 1) / W, (int64_t)g->ctx->sms * 16);
        k_seg_fill<E, 2 * kSegSmallRaw, W><<<fb, 32 * W, smem, st>>>(G, T, list, 0, n, d_ct, g->seg.entries, seg_node,
                                                                     g->order, slot);
        note_launch();
    }
    if (hc.listed[1]) {
        constexpr int W = 2;
        const size_t smem = sizeof(SegHash<kSegLargeSlots>) * W;
        e = cudaFuncSetAttribute(k_seg_fill<E, kSegLargeSlots, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return done(cuda_fail(e, "cudaFuncSetAttribute(k_seg_fill)"));
        const int fb = (int)std::min<int64_t>((hc.listed[1] + W - 1) / W, (int64_t)g->ctx->sms * 8);
        k_seg_fill<E, kSegLargeSlots, W><<<fb, 32 * W, smem, st>>>(G, T, list, 1, n, d_ct, g->seg.entries, seg_node,
                                                                   g->order, slot);
        note_launch();
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, d_ct, sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "segment build"));
    g->seg.nodes = (int64_t)hc.tables;
    g->seg.entries_n = (int64_t)hc.used;
    g->seg.entries_cap = (int64_t)hc.bound;
    g->device_bytes += (int64_t)(sizeof(typename E::Node) * n + sizeof(SegEntry) * hc.bound);
    return done(PPR_OK);
}

int build_segments(ppr_graph *g, uint32_t T, cudaStream_t st)
{
    if (g->seg.T == T && g->seg.node) return PPR_OK;
    Range range("segment tables");
    dev_free(g->seg.node, st);
    dev_free(g->seg.entries, st);
    g->seg = SegCache{};
    const int64_t n = g->n;
    uint32_t *list = nullptr;
    SegCounters *d_ct = nullptr;
    int rc;
    auto done = [&](int code) {
        dev_free(list, st);
        dev_free(d_ct, st);
        if (code != PPR_OK) {
            cudaStreamSynchronize(st);
            dev_free(g->seg.node, st);
            dev_free(g->seg.entries, st);
            g->seg = SegCache{};
        }
        return code;
    };
    const size_t node_bytes = g->wide ? sizeof(NodeRec) : sizeof(NodeRecN);
    if ((rc = dev_alloc((void **)&list, sizeof(uint32_t) * n, "segment node list", st)) ||
        (rc = dev_alloc((void **)&d_ct, sizeof(SegCounters), "segment counters", st)) ||
        (rc = dev_alloc((void **)&g->seg.node, node_bytes * n, "segment node records", st)))
        return done(rc);
    cudaError_t e = cudaMemsetAsync(d_ct, 0, sizeof(SegCounters), st);
    if (e != cudaSuccess) return done(cuda_fail(e, "memset"));
    if (g->wide) {
        RowView<WideEdges> G{static_cast<const NodeRec *>(g->node), WideEdges{(const EdgeW *)g->edges}};
        rc = seg_build_typed(g, T, st, G, list, d_ct);
    } else {
        RowView<NarrowEdges> G{static_cast<const NodeRecN *>(g->node), NarrowEdges{(const EdgeN *)g->edges}};
        rc = seg_build_typed(g, T, st, G, list, d_ct);
    }
    if (rc != PPR_OK) return done(rc);
    g->seg.T = T;
    return done(PPR_OK);
}

// --------------------------------------------------------- alias tables ----
// Integer Algorithm 1 per row: p_e = d * w_e against a slot capacity of W.
// The pairing order (free in Algorithm 1): y is the first edge of S^l in
// ascending order; x is the edge that has just dropped into S^s if there is
// one, else the next edge of the initial S^s in ascending order.  In that
// order the whole table is a closed form of two running sums -- D_i over the
// small edges of W - p, E_j over the large edges of p - W:
//   small edge i: thr = p, alias = large edge min{j : E_j > D_(i-1)}
//   large edge j (not the last): thr = W - (D_q - E_j) with q = min{q : D_q >= E_j},
//                                alias = large edge j + 1
//   last large edge, edges with p = W: thr = W, alias = itself.
// Rows of at most 32 edges run the pairing rounds serially, one thread per
// row; longer rows compute the closed form: one warp per row with the row in
// shared memory (up to 512 edges), one warp (up to 1,024) or block (up to
// 8,192) per row with scratch in global memory (alias_row_group), and tiles
// of blocks above that.  The limits keep each row's merge to a few dozen
// dependent probes per thread, so no long row is left running alone.

constexpr uint32_t kAliasInline = 32, kAliasSerial = 512, kAliasMid = 1024, kAliasHuge = 8192;
constexpr uint32_t kAliasMaxHuge = 65536;  // rows taken by the tile path; more go to the block tier
constexpr uint32_t kTileEdges = 8192;     // edges per tile block (256 threads x 32)

struct AliasArgs {
    int64_t n;
    const NodeRecN *node;  // the narrow layout's records (begin, count, W)
    const EdgeN *edges;
    const uint64_t *off;  // first slot of each row (exclusive scan of degrees)
    AliasNode *anode;
    AliasRec *slots;
    uint2 *ic;            // per slot of a long row: (edge, col) of the small edges from the front,
                          // of the large edges from the back
    uint64_t *sum;        // their running sums D_i / E_j
    uint32_t *list;       // rows per tier: [0, n) one thread, [n, 2n) one warp, [2n, 3n) one block
    uint32_t *counts;     // rows in each list; [3] rows offered to the tile path
    uint2 *huge;          // tile-path rows (node, degree), kAliasMaxHuge entries
};

template <class N>
__device__ __forceinline__ uint32_t row_degree(const N &r) { return (uint32_t)(r.word0 >> 40) & kCountMask; }

// The pairing rounds of one row, serially (row of d >= 2 edges, slots from o).
__device__ void alias_row_serial(const AliasArgs &A, const NodeRecN &nr, uint32_t d, uint64_t o)
{
    const uint64_t W = nr.total & 0xffffffffull;
    const uint64_t eb = NarrowEdges::edge_base(nr.word0 & kBeginMask, d);
    auto pw = [&](uint32_t i) -> uint64_t {
        const uint32_t hi = A.edges[eb + i].P, lo = i ? A.edges[eb + i - 1].P : 0u;
        return (uint64_t)d * (hi - lo);
    };
    for (uint32_t i = 0; i < d; ++i) {
        const int32_t c = A.edges[eb + i].col;
        A.slots[o + i] = AliasRec{(uint32_t)W, c, c, (uint32_t)W};
    }
    auto next_small = [&](uint32_t i) { while (i < d && pw(i) >= W) ++i; return i; };
    auto next_large = [&](uint32_t j) { while (j < d && pw(j) <= W) ++j; return j; };
    uint32_t i = next_small(0), j = next_large(0);
    if (j >= d) return;
    uint64_t py = pw(j);  // remaining p of the current large edge
    for (uint32_t guard = 0; guard < 2 * d; ++guard) {
        if (py > W) {  // x = next small edge, y = j
            if (i >= d) break;
            const uint64_t px = pw(i);
            A.slots[o + i].thr = (uint32_t)px;
            A.slots[o + i].alias_col = A.edges[eb + j].col;
            py -= W - px;
            i = next_small(i + 1);
        } else {  // j leaves S^l; if it dropped below W it is the next x
            const uint32_t j2 = next_large(j + 1);
            if (j2 >= d) break;  // py == W here: the last large edge
            if (py < W) {
                A.slots[o + j].thr = (uint32_t)py;
                A.slots[o + j].alias_col = A.edges[eb + j2].col;
            }
            py = pw(j2) - (W - py);
            j = j2;
        }
    }
}

// Node records of the alias layout for every row; rows of at most 32 edges
// are built here, longer ones are listed for their tier.
__global__ void __launch_bounds__(256) k_alias_small(AliasArgs A)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < A.n; u += (int64_t)gridDim.x * blockDim.x) {
        const NodeRecN nr = A.node[u];
        const uint32_t d = row_degree(nr);
        const uint64_t o = A.off[u];
        // first slot and degree; a single-edge row keeps its target instead
        A.anode[u] = AliasNode{pack_word0(d == 1 ? (nr.total & 0xffffffffull) : o, d, false)};
        if (d < 2) continue;
        if (d > kAliasInline) {
            if (d > kAliasHuge) {
                const uint32_t k = atomicAdd(&A.counts[3], 1u);
                if (k < kAliasMaxHuge) {
                    A.huge[k] = make_uint2((uint32_t)u, d);
                    continue;
                }
            }
            const uint32_t tier = d <= kAliasSerial ? 0 : (d <= kAliasMid ? 1 : 2);
            A.list[(int64_t)tier * A.n + atomicAdd(&A.counts[tier], 1u)] = (uint32_t)u;
            continue;
        }
        alias_row_serial(A, nr, d, o);
    }
}

// Rows of 33..512 edges, one warp per row, the row staged in shared memory:
// a coalesced pass classifies the edges, ranks them with ballots and forms
// the running sums D and E with warp scans; each lane then merges a
// contiguous share of the small (and of the large) edges against the other
// sequence, as alias_row_group does, with every probe in shared memory.
constexpr int kSmemWarps = 4;
struct RowSmem {
    int32_t col[kAliasSerial];
    uint16_t idx[kAliasSerial];  // edge of each small (from the front) and large (from the back) entry
    uint64_t sum[kAliasSerial];  // D_i / E_j
};

__global__ void __launch_bounds__(32 * kSmemWarps) k_alias_serial(AliasArgs A)
{
    __shared__ RowSmem sm_all[kSmemWarps];
    RowSmem &sm = sm_all[threadIdx.x >> 5];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t rows = A.counts[0];
    const uint32_t warps = gridDim.x * kSmemWarps;
    for (uint32_t t = blockIdx.x * kSmemWarps + (threadIdx.x >> 5); t < rows; t += warps) {
        const uint32_t u = A.list[t];
        const NodeRecN nr = A.node[u];
        const uint32_t d = row_degree(nr);  // 33..512
        const uint64_t o = A.off[u];
        const uint64_t W = nr.total & 0xffffffffull;
        const uint64_t eb = NarrowEdges::edge_base(nr.word0 & kBeginMask, d);
        uint32_t ns = 0, nl = 0;
        uint64_t Dc = 0, Ec = 0;
        for (uint32_t e0 = 0; e0 < d; e0 += 32) {
            const uint32_t i = e0 + lane;
            uint64_t p = 0;
            int32_t c = 0;
            if (i < d) {
                const EdgeN rec = A.edges[eb + i];
                const uint32_t lo = i ? A.edges[eb + i - 1].P : 0u;
                p = (uint64_t)d * (rec.P - lo);
                c = rec.col;
                sm.col[i] = c;
                A.slots[o + i] = AliasRec{(uint32_t)W, c, c, (uint32_t)W};
            }
            const bool isS = i < d && p < W, isL = i < d && p > W;
            const uint32_t bs = __ballot_sync(0xffffffffu, isS), bl = __ballot_sync(0xffffffffu, isL);
            const uint32_t lt = (1u << lane) - 1;
            uint64_t dv = isS ? W - p : 0ull, ev = isL ? p - W : 0ull;
#pragma unroll
            for (int q = 1; q < 32; q <<= 1) {
                const uint64_t yd = __shfl_up_sync(0xffffffffu, dv, q), ye = __shfl_up_sync(0xffffffffu, ev, q);
                if (lane >= (uint32_t)q) {
                    dv += yd;
                    ev += ye;
                }
            }
            if (isS) {
                const uint32_t k = ns + __popc(bs & lt);
                sm.idx[k] = (uint16_t)i;
                sm.sum[k] = Dc + dv;
            } else if (isL) {
                const uint32_t k = d - 1 - (nl + __popc(bl & lt));
                sm.idx[k] = (uint16_t)i;
                sm.sum[k] = Ec + ev;
            }
            ns += __popc(bs);
            nl += __popc(bl);
            Dc += __shfl_sync(0xffffffffu, dv, 31);
            Ec += __shfl_sync(0xffffffffu, ev, 31);
        }
        __syncwarp();
        const uint32_t a = ns, b = nl;
        if (a > 0 && b > 0 && a + b <= d) {
            auto E = [&](uint32_t j) { return sm.sum[d - 1 - j]; };
            auto D = [&](uint32_t q) { return sm.sum[q]; };
            // small edges t: donor = first large j with E_j > D_(t-1)
            const uint32_t shs = (a + 31) / 32, t0 = min(lane * shs, a), t1 = min(t0 + shs, a);
            if (t0 < t1) {
                uint64_t prev = t0 ? D(t0 - 1) : 0ull;
                uint32_t jl = 0, jh = b - 1;
                while (jl < jh) {
                    const uint32_t mid = (jl + jh) >> 1;
                    if (E(mid) > prev) jh = mid;
                    else jl = mid + 1;
                }
                uint32_t j = jl;
                for (uint32_t tt = t0; tt < t1; ++tt) {
                    while (j + 1 < b && E(j) <= prev) ++j;
                    const uint64_t Dt = D(tt);
                    const uint32_t e = sm.idx[tt];
                    A.slots[o + e].thr = (uint32_t)(W - (Dt - prev));
                    A.slots[o + e].alias_col = sm.col[sm.idx[d - 1 - j]];
                    prev = Dt;
                }
            }
            // large edges j (not the last): q = first small with D_q >= E_j
            const uint32_t nlm = b - 1, shl = (nlm + 31) / 32;
            const uint32_t j0 = min(lane * shl, nlm), j1 = min(j0 + shl, nlm);
            if (j0 < j1) {
                uint64_t Ej = E(j0);
                uint32_t ql = 0, qh = a - 1;
                while (ql < qh) {
                    const uint32_t mid = (ql + qh) >> 1;
                    if (D(mid) >= Ej) qh = mid;
                    else ql = mid + 1;
                }
                uint32_t q = ql;
                for (uint32_t j = j0; j < j1; ++j) {
                    Ej = E(j);
                    while (q + 1 < a && D(q) < Ej) ++q;
                    const uint64_t th = W - (D(q) - Ej);
                    if (th < W) {
                        const uint32_t e = sm.idx[d - 1 - j];
                        A.slots[o + e].thr = (uint32_t)th;
                        A.slots[o + e].alias_col = sm.col[sm.idx[d - 2 - j]];
                    }
                }
            }
        }
        __syncwarp();  // the next row reuses the warp's shared memory
    }
}

// Inclusive scan of three u64 values over a warp (NT = 32) or a block; `tot`
// receives the group totals.  Block form: s holds 3 * (NT / 32) words.
template <int NT>
__device__ __forceinline__ void group_scan3(uint64_t v[3], uint64_t tot[3], uint64_t *s)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, v[k], o);
            if (lane >= o) v[k] += y;
        }
    }
    if constexpr (NT == 32) {
#pragma unroll
        for (int k = 0; k < 3; ++k) tot[k] = __shfl_sync(0xffffffffu, v[k], 31);
    } else {
        constexpr int NW = NT / 32;
        if (lane == 31)
            for (int k = 0; k < 3; ++k) s[k * NW + wid] = v[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint64_t before = 0, all = 0;
            for (int q = 0; q < NW; ++q) {
                const uint64_t t = s[k * NW + q];
                before += q < (int)wid ? t : 0ull;
                all += t;
            }
            v[k] += before;
            tot[k] = all;
        }
        __syncthreads();
    }
}

template <int NT>
__device__ __forceinline__ void group_sync()
{
    if constexpr (NT == 32) __syncwarp();
    else __syncthreads();
}

// Closed-form alias table of one row of d > 32 edges by a group of NT threads
// (rank = thread index within the group).  Each thread owns a contiguous run
// of about d / NT edges: it totals its run, one group scan gives the run's
// starting ranks and sums, and a second walk over the run writes the small
// and large edges with their running sums to scratch.  The partners are then
// a merge of the two sorted sequences D and E: each thread takes a contiguous
// share of the small (and of the large) edges, finds its first partner by
// bisection and advances linearly from there.
template <int NT>
__device__ void alias_row_group(const AliasArgs &A, int64_t u, uint32_t rank, uint64_t *s)
{
    const NodeRecN nr = A.node[u];
    const uint32_t d = row_degree(nr);
    const uint64_t o = A.off[u];
    const uint64_t W = nr.total & 0xffffffffull;
    const uint64_t eb = NarrowEdges::edge_base(nr.word0 & kBeginMask, d);
    const uint32_t run = (d + NT - 1) / NT;
    const uint32_t lo = min(rank * run, d), hi = min(lo + run, d);
    // totals of this thread's run
    uint64_t v[3] = {0, 0, 0};  // small | large << 32 counts, sum of W - p, sum of p - W
    {
        uint32_t prevP = lo ? A.edges[eb + lo - 1].P : 0u;
        for (uint32_t i0 = lo; i0 < hi; i0 += 8) {
            uint32_t Pv[8];  // eight loads in flight before their use
#pragma unroll
            for (int q = 0; q < 8; ++q) Pv[q] = i0 + q < hi ? A.edges[eb + i0 + q].P : 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (i0 + q >= hi) break;
                const uint64_t p = (uint64_t)d * (Pv[q] - prevP);
                prevP = Pv[q];
                if (p < W) {
                    v[0] += 1;
                    v[1] += W - p;
                } else if (p > W) {
                    v[0] += 1ull << 32;
                    v[2] += p - W;
                }
            }
        }
    }
    const uint64_t own[3] = {v[0], v[1], v[2]};
    uint64_t tot[3];
    group_scan3<NT>(v, tot, s);
    uint64_t ks = (v[0] - own[0]) & 0xffffffffull, kl = (v[0] - own[0]) >> 32;
    uint64_t Dr = v[1] - own[1], Er = v[2] - own[2];
    {
        uint32_t prevP = lo ? A.edges[eb + lo - 1].P : 0u;
        for (uint32_t i0 = lo; i0 < hi; i0 += 8) {
            EdgeN rv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (i0 + q < hi) rv[q] = A.edges[eb + i0 + q];
                else rv[q] = EdgeN{0u, 0};
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t i = i0 + q;
                if (i >= hi) break;
                const EdgeN rec = rv[q];
                const uint64_t p = (uint64_t)d * (rec.P - prevP);
                prevP = rec.P;
                A.slots[o + i] = AliasRec{(uint32_t)W, rec.col, rec.col, (uint32_t)W};
                if (p < W && ks < d) {
                    Dr += W - p;
                    A.ic[o + ks] = make_uint2(i, (uint32_t)rec.col);
                    A.sum[o + ks] = Dr;
                    ++ks;
                } else if (p > W && kl < d) {
                    Er += p - W;
                    A.ic[o + d - 1 - kl] = make_uint2(i, (uint32_t)rec.col);
                    A.sum[o + d - 1 - kl] = Er;
                    ++kl;
                }
            }
        }
    }
    group_sync<NT>();
    const uint32_t a = (uint32_t)(tot[0] & 0xffffffffull), b = (uint32_t)(tot[0] >> 32);
    if (a == 0 || b == 0 || (uint64_t)a + b > d) return;  // every p equals W (the sums force a > 0 iff b > 0)
    auto E = [&](uint32_t j) { return A.sum[o + d - 1 - j]; };
    auto D = [&](uint32_t q) { return A.sum[o + q]; };
    auto large_col = [&](uint32_t j) { return (int32_t)A.ic[o + d - 1 - j].y; };
    // small edges t in [t0, t1): donor = first large j with E_j > D_(t-1)
    {
        const uint32_t share = (a + NT - 1) / NT;
        const uint32_t t0 = min(rank * share, a), t1 = min(t0 + share, a);
        if (t0 < t1) {
            uint64_t prev = t0 ? D(t0 - 1) : 0ull;
            uint32_t jl = 0, jh = b - 1;
            while (jl < jh) {
                const uint32_t mid = (jl + jh) >> 1;
                if (E(mid) > prev) jh = mid;
                else jl = mid + 1;
            }
            uint32_t j = jl;
            for (uint32_t t = t0; t < t1; ++t) {
                while (j + 1 < b && E(j) <= prev) ++j;
                const uint64_t Dt = D(t);
                const uint32_t e = A.ic[o + t].x;
                A.slots[o + e].thr = (uint32_t)(W - (Dt - prev));
                A.slots[o + e].alias_col = large_col(j);
                prev = Dt;
            }
        }
    }
    // large edges j in [j0, j1) (not the last): q = first small with D_q >= E_j
    {
        const uint32_t nl = b - 1, share = (nl + NT - 1) / NT;
        const uint32_t j0 = min(rank * share, nl), j1 = min(j0 + share, nl);
        if (j0 < j1) {
            uint64_t Ej = E(j0);
            uint32_t ql = 0, qh = a - 1;
            while (ql < qh) {
                const uint32_t mid = (ql + qh) >> 1;
                if (D(mid) >= Ej) qh = mid;
                else ql = mid + 1;
            }
            uint32_t q = ql;
            for (uint32_t j = j0; j < j1; ++j) {
                Ej = E(j);
                while (q + 1 < a && D(q) < Ej) ++q;
                const uint64_t th = W - (D(q) - Ej);
                if (th < W) {
                    const uint32_t e = A.ic[o + d - 1 - j].x;
                    A.slots[o + e].thr = (uint32_t)th;
                    A.slots[o + e].alias_col = large_col(j + 1);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_alias_mid(AliasArgs A)
{
    const uint32_t lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t rows = A.counts[1];
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < rows; t += warps)
        alias_row_group<32>(A, A.list[A.n + t], lane, nullptr);
}

__global__ void __launch_bounds__(512) k_alias_big(AliasArgs A)
{
    __shared__ uint64_t s[3 * 16];
    const uint32_t rows = A.counts[2];
    for (uint32_t t = blockIdx.x; t < rows; t += gridDim.x) {
        alias_row_group<512>(A, A.list[2 * A.n + t], threadIdx.x, s);
        __syncthreads();
    }
}

// ------------------------------------------------ alias tables: tile path ----
// Rows above kAliasHuge edges are cut into tiles of kTileEdges edges, one
// block per tile, so a hub does not leave one block working while the GPU
// idles: (1) every tile totals its small/large counts and running-sum parts,
// (2) one warp per row scans its tiles' totals, (3) every tile writes its
// small and large edges with their running sums to scratch, (4) merge chunks
// of kTileEdges small (or large) edges each find their partners as in
// alias_row_group.

struct HugeRow {
    uint32_t u, d;
    uint32_t tile0, ntiles;  // tiles of the row in the tile table
    uint32_t chunk0;         // first merge chunk (2 * ntiles chunks: small edges, then large edges)
};

struct TileVal {
    uint64_t cnt, D, E;  // small | large << 32 counts, sum of W - p, sum of p - W
};

struct TileArgs {
    AliasArgs A;
    const HugeRow *rows;
    uint32_t nrows;
    const uint2 *tiles;      // (row index, first edge of the tile within the row)
    TileVal *tile_val;       // per tile: its totals, then (after the row scan) its exclusive offsets
    ulonglong2 *row_ab;      // per row: small count, large count
};

// Per-thread run of up to 32 edges of a tile: fills the three totals.
__device__ __forceinline__ void tile_run_totals(const AliasArgs &A, uint64_t eb, uint32_t d, uint64_t W, uint32_t lo,
                                                uint32_t hi, uint64_t v[3])
{
    uint32_t prevP = lo ? A.edges[eb + lo - 1].P : 0u;
    for (uint32_t i0 = lo; i0 < hi; i0 += 8) {
        uint32_t Pv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) Pv[q] = i0 + q < hi ? A.edges[eb + i0 + q].P : 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (i0 + q >= hi) break;
            const uint64_t p = (uint64_t)d * (Pv[q] - prevP);
            prevP = Pv[q];
            if (p < W) {
                v[0] += 1;
                v[1] += W - p;
            } else if (p > W) {
                v[0] += 1ull << 32;
                v[2] += p - W;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_alias_tile_totals(TileArgs T)
{
    __shared__ uint64_t s[3 * 8];
    const AliasArgs &A = T.A;
    const uint2 tl = T.tiles[blockIdx.x];
    const HugeRow hr = T.rows[tl.x];
    const NodeRecN nr = A.node[hr.u];
    const uint64_t W = nr.total & 0xffffffffull;
    const uint64_t eb = NarrowEdges::edge_base(nr.word0 & kBeginMask, hr.d);
    const uint32_t end = min(tl.y + kTileEdges, hr.d);
    const uint32_t lo = min(tl.y + threadIdx.x * 32, end), hi = min(lo + 32, end);
    uint64_t v[3] = {0, 0, 0};
    tile_run_totals(A, eb, hr.d, W, lo, hi, v);
    uint64_t tot[3];
    group_scan3<256>(v, tot, s);
    if (threadIdx.x == 0) T.tile_val[blockIdx.x] = TileVal{tot[0], tot[1], tot[2]};
}

// One warp per row: exclusive scan of its tiles' totals (in place), row counts.
__global__ void k_alias_tile_scan(TileArgs T)
{
    const uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= T.nrows) return;
    const uint32_t lane = threadIdx.x & 31;
    const HugeRow hr = T.rows[r];
    uint64_t carry[3] = {0, 0, 0};
    for (uint32_t t0 = 0; t0 < hr.ntiles; t0 += 32) {
        const uint32_t t = t0 + lane;
        TileVal tv{0, 0, 0};
        if (t < hr.ntiles) tv = T.tile_val[hr.tile0 + t];
        uint64_t v[3] = {tv.cnt, tv.D, tv.E}, tot[3];
        const uint64_t own[3] = {v[0], v[1], v[2]};
        group_scan3<32>(v, tot, nullptr);
        if (t < hr.ntiles)
            T.tile_val[hr.tile0 + t] = TileVal{carry[0] + v[0] - own[0], carry[1] + v[1] - own[1],
                                               carry[2] + v[2] - own[2]};
        for (int k = 0; k < 3; ++k) carry[k] += tot[k];
    }
    if (lane == 0) T.row_ab[r] = make_ulonglong2(carry[0] & 0xffffffffull, carry[0] >> 32);
}

__global__ void __launch_bounds__(256) k_alias_tile_write(TileArgs T)
{
    __shared__ uint64_t s[3 * 8];
    const AliasArgs &A = T.A;
    const uint2 tl = T.tiles[blockIdx.x];
    const HugeRow hr = T.rows[tl.x];
    const uint32_t d = hr.d;
    const NodeRecN nr = A.node[hr.u];
    const uint64_t W = nr.total & 0xffffffffull;
    const uint64_t eb = NarrowEdges::edge_base(nr.word0 & kBeginMask, d);
    const uint64_t o = A.off[hr.u];
    const uint32_t end = min(tl.y + kTileEdges, d);
    const uint32_t lo = min(tl.y + threadIdx.x * 32, end), hi = min(lo + 32, end);
    uint64_t v[3] = {0, 0, 0};
    tile_run_totals(A, eb, d, W, lo, hi, v);
    const uint64_t own[3] = {v[0], v[1], v[2]};
    uint64_t tot[3];
    group_scan3<256>(v, tot, s);
    const TileVal base = T.tile_val[blockIdx.x];  // the tile's exclusive offsets within the row
    uint64_t ks = (base.cnt & 0xffffffffull) + ((v[0] - own[0]) & 0xffffffffull);
    uint64_t kl = (base.cnt >> 32) + ((v[0] - own[0]) >> 32);
    uint64_t Dr = base.D + v[1] - own[1], Er = base.E + v[2] - own[2];
    uint32_t prevP = lo ? A.edges[eb + lo - 1].P : 0u;
    for (uint32_t i = lo; i < hi; ++i) {
        const EdgeN rec = A.edges[eb + i];
        const uint64_t p = (uint64_t)d * (rec.P - prevP);
        prevP = rec.P;
        A.slots[o + i] = AliasRec{(uint32_t)W, rec.col, rec.col, (uint32_t)W};
        if (p < W && ks < d) {
            Dr += W - p;
            A.ic[o + ks] = make_uint2(i, (uint32_t)rec.col);
            A.sum[o + ks] = Dr;
            ++ks;
        } else if (p > W && kl < d) {
            Er += p - W;
            A.ic[o + d - 1 - kl] = make_uint2(i, (uint32_t)rec.col);
            A.sum[o + d - 1 - kl] = Er;
            ++kl;
        }
    }
}

// Merge chunk c of a row: chunks [0, ntiles) cover small edges
// [c * kTileEdges, ...), chunks [ntiles, 2 ntiles) cover large edges (the
// last large edge keeps thr = W).  Each thread takes 32 consecutive ones.
__global__ void __launch_bounds__(256) k_alias_tile_merge(TileArgs T)
{
    const AliasArgs &A = T.A;
    uint32_t lo = 0, hi = T.nrows;  // row of this chunk: last row with chunk0 <= blockIdx.x
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (T.rows[mid].chunk0 <= blockIdx.x) lo = mid;
        else hi = mid;
    }
    const HugeRow hr = T.rows[lo];
    const uint32_t c = blockIdx.x - hr.chunk0;
    if (c >= 2 * hr.ntiles) return;
    const ulonglong2 ab = T.row_ab[lo];
    const uint32_t a = (uint32_t)ab.x, b = (uint32_t)ab.y, d = hr.d;
    if (a == 0 || b == 0 || (uint64_t)a + b > d) return;
    const NodeRecN nr = A.node[hr.u];
    const uint64_t W = nr.total & 0xffffffffull;
    const uint64_t o = A.off[hr.u];
    auto E = [&](uint32_t j) { return A.sum[o + d - 1 - j]; };
    auto D = [&](uint32_t q) { return A.sum[o + q]; };
    if (c < hr.ntiles) {  // small edges t in [t0, t1): donor = first large j with E_j > D_(t-1)
        const uint32_t t0 = min(c * kTileEdges + threadIdx.x * 32, a), t1 = min(t0 + 32, min((c + 1) * kTileEdges, a));
        if (t0 >= t1) return;
        uint64_t prev = t0 ? D(t0 - 1) : 0ull;
        uint32_t jl = 0, jh = b - 1;
        while (jl < jh) {
            const uint32_t mid = (jl + jh) >> 1;
            if (E(mid) > prev) jh = mid;
            else jl = mid + 1;
        }
        uint32_t j = jl;
        for (uint32_t t = t0; t < t1; ++t) {
            while (j + 1 < b && E(j) <= prev) ++j;
            const uint64_t Dt = D(t);
            const uint32_t e = A.ic[o + t].x;
            A.slots[o + e].thr = (uint32_t)(W - (Dt - prev));
            A.slots[o + e].alias_col = (int32_t)A.ic[o + d - 1 - j].y;
            prev = Dt;
        }
    } else {  // large edges j in [j0, j1), not the last: q = first small with D_q >= E_j
        const uint32_t cl = c - hr.ntiles, nl = b - 1;
        const uint32_t j0 = min(cl * kTileEdges + threadIdx.x * 32, nl), j1 = min(j0 + 32, min((cl + 1) * kTileEdges, nl));
        if (j0 >= j1) return;
        uint64_t Ej = E(j0);
        uint32_t ql = 0, qh = a - 1;
        while (ql < qh) {
            const uint32_t mid = (ql + qh) >> 1;
            if (D(mid) >= Ej) qh = mid;
            else ql = mid + 1;
        }
        uint32_t q = ql;
        for (uint32_t j = j0; j < j1; ++j) {
            Ej = E(j);
            while (q + 1 < a && D(q) < Ej) ++q;
            const uint64_t th = W - (D(q) - Ej);
            if (th < W) {
                const uint32_t e = A.ic[o + d - 1 - j].x;
                A.slots[o + e].thr = (uint32_t)th;
                A.slots[o + e].alias_col = (int32_t)A.ic[o + d - 2 - j].y;
            }
        }
    }
}

__global__ void k_alias_degrees(int64_t n, const NodeRecN *node, uint32_t *deg)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        deg[u] = row_degree(node[u]);
}

int build_alias(ppr_graph *g, cudaStream_t st)
{
    if (g->alias.node) return PPR_OK;
    Range range("alias tables");
    if (g->wide) {
        set_error("the alias sampler needs every row total below 2^32");
        return PPR_ENOTSUP;
    }
    const int64_t n = g->n, m = std::max<int64_t>(g->m, 1);
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    uint32_t *deg = nullptr, *list = nullptr, *counts = nullptr;
    uint2 *ic = nullptr, *huge = nullptr, *d_tiles = nullptr;
    uint64_t *off = nullptr, *tmp = nullptr, *sum = nullptr;
    HugeRow *d_rows = nullptr;
    TileVal *tile_val = nullptr;
    ulonglong2 *row_ab = nullptr;
    int rc;
    auto cleanup = [&]() {
        dev_free(deg, st);
        dev_free(off, st);
        dev_free(tmp, st);
        dev_free(ic, st);
        dev_free(sum, st);
        dev_free(list, st);
        dev_free(counts, st);
        dev_free(huge, st);
        dev_free(d_rows, st);
        dev_free(d_tiles, st);
        dev_free(tile_val, st);
        dev_free(row_ab, st);
    };
    auto fail = [&](int code) {
        cudaStreamSynchronize(st);
        cleanup();
        dev_free(g->alias.node, st);
        dev_free(g->alias.slots, st);
        g->alias.node = nullptr;
        g->alias.slots = nullptr;
        return code;
    };
    if ((rc = dev_alloc((void **)&deg, sizeof(uint32_t) * n, "alias degrees", st)) ||
        (rc = dev_alloc((void **)&off, sizeof(uint64_t) * (n + 1), "alias offsets", st)) ||
        (rc = dev_alloc((void **)&tmp, sizeof(uint64_t) * (tiles + 2), "scan scratch", st)) ||
        (rc = dev_alloc((void **)&ic, sizeof(uint2) * m, "alias scratch", st)) ||
        (rc = dev_alloc((void **)&sum, sizeof(uint64_t) * m, "alias scratch", st)) ||
        (rc = dev_alloc((void **)&list, sizeof(uint32_t) * 3 * n, "long-row lists", st)) ||
        (rc = dev_alloc((void **)&counts, sizeof(uint32_t) * 4, "long-row counts", st)) ||
        (rc = dev_alloc((void **)&huge, sizeof(uint2) * kAliasMaxHuge, "tile-path rows", st)))
        return cleanup(), rc;
    if ((rc = dev_alloc((void **)&g->alias.node, sizeof(AliasNode) * n, "alias node records", st))) return cleanup(), rc;
    if ((rc = dev_alloc((void **)&g->alias.slots, sizeof(AliasRec) * m, "alias slots", st))) return fail(rc);
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * 4, st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "memset"));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g->ctx->sms * 16));
    k_alias_degrees<<<blocks, 256, 0, st>>>(n, static_cast<const NodeRecN *>(g->node), deg);
    note_launch();
    exclusive_scan_u32(deg, n, off, tmp, st);
    AliasArgs A{n, static_cast<const NodeRecN *>(g->node), (const EdgeN *)g->edges, off, g->alias.node, g->alias.slots, ic,
                sum, list, counts, huge};
    k_alias_small<<<blocks, 256, 0, st>>>(A);
    note_launch();
    // rows for the tile path: their count and degrees decide the tile grid
    uint32_t hc[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "alias build"));
    const uint32_t nh = std::min(hc[3], kAliasMaxHuge);
    if (nh > 0) {
        std::vector<uint2> hl(nh);
        e = cudaMemcpy(hl.data(), huge, sizeof(uint2) * nh, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(cuda_fail(e, "alias build"));
        std::vector<HugeRow> rows(nh);
        std::vector<uint2> tl;
        uint32_t chunks = 0;
        for (uint32_t r = 0; r < nh; ++r) {
            const uint32_t d = hl[r].y, nt = (d + kTileEdges - 1) / kTileEdges;
            rows[r] = HugeRow{hl[r].x, d, (uint32_t)tl.size(), nt, chunks};
            for (uint32_t t = 0; t < nt; ++t) tl.push_back(make_uint2(r, t * kTileEdges));
            chunks += 2 * nt;
        }
        const uint32_t nt = (uint32_t)tl.size();
        if ((rc = dev_alloc((void **)&d_rows, sizeof(HugeRow) * nh, "tile-path rows", st)) ||
            (rc = dev_alloc((void **)&d_tiles, sizeof(uint2) * nt, "tile table", st)) ||
            (rc = dev_alloc((void **)&tile_val, sizeof(TileVal) * nt, "tile totals", st)) ||
            (rc = dev_alloc((void **)&row_ab, sizeof(ulonglong2) * nh, "tile-path counts", st)))
            return fail(rc);
        e = cudaMemcpyAsync(d_rows, rows.data(), sizeof(HugeRow) * nh, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_tiles, tl.data(), sizeof(uint2) * nt, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(cuda_fail(e, "tile table upload"));
        TileArgs T{A, d_rows, nh, d_tiles, tile_val, row_ab};
        k_alias_tile_totals<<<nt, 256, 0, st>>>(T);
        note_launch();
        k_alias_tile_scan<<<(nh + 7) / 8, 256, 0, st>>>(T);
        note_launch();
        k_alias_tile_write<<<nt, 256, 0, st>>>(T);
        note_launch();
        k_alias_tile_merge<<<chunks, 256, 0, st>>>(T);
        note_launch();
        // the host vectors must outlive the asynchronous uploads
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(cuda_fail(e, "alias build"));
    }
    if (hc[0]) {
        k_alias_serial<<<g->ctx->sms * 16, 32 * kSmemWarps, 0, st>>>(A);
        note_launch();
    }
    if (hc[1]) {
        k_alias_mid<<<g->ctx->sms * 8, 256, 0, st>>>(A);
        note_launch();
    }
    if (hc[2]) {
        k_alias_big<<<(int)std::min<uint32_t>(hc[2], (uint32_t)g->ctx->sms * 2), 512, 0, st>>>(A);
        note_launch();
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "alias build"));
    cleanup();
    g->device_bytes += (int64_t)(sizeof(AliasNode) * n + sizeof(AliasRec) * m);
    return PPR_OK;
}

}  // namespace ppr
