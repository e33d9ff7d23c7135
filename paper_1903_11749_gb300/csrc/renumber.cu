// renumber.cu -- the walk layout's own node numbering for graphs far larger
// than L2.
//
// A walk with restart from every node visits node v at a rate proportional
// to its PageRank (Sec. 2.1: the walks of all sources together follow the
// random surfer with teleport alpha), which on a power-law graph is led by
// its in-degree.  The layout numbers nodes in descending order of in-degree
// (counted on every fourth edge; eight classes per power of two, ties in
// input order), so the records and rows of the most visited nodes sit
// together at the front of their arrays: their 32-byte sectors share
// 128-byte L2 lines and DRAM pages instead of being spread over gigabytes.  The numbering is internal: sources, result
// rows and top-k use the caller's ids, and the draw of a walk is keyed by the
// caller's source id, so every count is the same with and without it.
//   order[i]: caller id of internal node i;  rank[v]: internal id of caller node v.
#include "ppr_host.h"
#include "scan.cuh"

namespace ppr {

constexpr int kRnBuckets = 1 + 32 * 8;  // in-degree 0, then 8 classes per power of two
constexpr int kRnTile = 1024;           // nodes per warp tile of the counting sort

// In-degree of every node, counted on every kRnEvery-th edge (the ordering
// needs the classes of the well-visited nodes, whose counts a quarter of the
// edges already fixes to within a class or two; the atomics, not the read,
// set this kernel's time).  Edges whose target lies outside [0, n) are
// skipped (the layout build reports them).  Equal targets within a warp are
// summed first, so a hub takes one atomic per warp and not one per edge.
constexpr int64_t kRnEvery = 4;

__global__ void __launch_bounds__(256) k_rn_indegree(int64_t n, int64_t m, const int32_t *col, uint32_t *indeg)
{
    const uint32_t lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t ms = (m + kRnEvery - 1) / kRnEvery;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ms; base += stride) {
        const int64_t e = (base + threadIdx.x) * kRnEvery;
        int32_t c = -1;
        if (e < m) c = col[e];
        const bool ok = c >= 0 && (int64_t)c < n;
        const uint32_t key = ok ? (uint32_t)c : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        if (ok && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&indeg[c], (uint32_t)__popc(peers));
    }
}

// Class of an in-degree: 0 for none, else 1 + 8 * floor(log2 c) + the three
// bits after the leading one.  Placed in descending class order.
__device__ __forceinline__ uint32_t rn_slot(uint32_t c)
{
    if (c == 0) return kRnBuckets - 1;
    const uint32_t lg = 31u - __clz(c);
    const uint32_t frac = lg >= 3 ? (c >> (lg - 3)) & 7u : (c << (3 - lg)) & 7u;
    return (uint32_t)(kRnBuckets - 1) - (1u + 8u * lg + frac);
}

// Per-tile class counts, class-major: hist[slot * tiles + tile].
__global__ void __launch_bounds__(256) k_rn_hist(int64_t n, const uint32_t *indeg, uint32_t *hist, int64_t tiles)
{
    __shared__ uint32_t h[8][kRnBuckets];
    const uint32_t wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * 8 + wid;
    for (uint32_t i = lane; i < (uint32_t)kRnBuckets; i += 32) h[wid][i] = 0;
    __syncwarp();
    if (tile < tiles) {
        for (uint32_t r = 0; r < (uint32_t)kRnTile; r += 32) {
            const int64_t v = tile * kRnTile + r + lane;
            if (v < n) atomicAdd(&h[wid][rn_slot(indeg[v])], 1u);
        }
        __syncwarp();
        for (uint32_t i = lane; i < (uint32_t)kRnBuckets; i += 32) hist[(int64_t)i * tiles + tile] = h[wid][i];
    }
}

// Stable scatter: node v of tile t goes to off[slot * tiles + t] plus the
// number of earlier nodes of the tile in its class.
__global__ void __launch_bounds__(256) k_rn_scatter(int64_t n, const uint32_t *indeg, const uint64_t *off,
                                                    int64_t tiles, int32_t *order, int32_t *rank)
{
    __shared__ uint32_t seen[8][kRnBuckets];
    const uint32_t wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * 8 + wid;
    for (uint32_t i = lane; i < (uint32_t)kRnBuckets; i += 32) seen[wid][i] = 0;
    __syncwarp();
    if (tile >= tiles) return;
    for (uint32_t r = 0; r < (uint32_t)kRnTile; r += 32) {
        const int64_t v = tile * kRnTile + r + lane;
        const uint32_t s = v < n ? rn_slot(indeg[v]) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, s);
        const uint32_t before = __popc(peers & ((1u << lane) - 1));
        uint32_t base = 0;
        if (v < n) base = seen[wid][s];
        __syncwarp();
        if (v < n) {
            const int64_t pos = (int64_t)off[(int64_t)s * tiles + tile] + base + before;
            order[pos] = (int32_t)v;
            rank[v] = (int32_t)pos;
            if (before == 0) seen[wid][s] = base + __popc(peers);
        }
        __syncwarp();
    }
}

// order and rank (n int32 each, device) for the CSR col[0..m); scratch goes
// to tmp (freed by the caller).  Enqueued on st.
int renumber_by_indegree(ppr_ctx *ctx, int64_t n, int64_t m, const int32_t *d_col, cudaStream_t st, int32_t *order,
                         int32_t *rank, std::vector<void *> &tmp)
{
    Range range("renumber");
    int rc;
    const int64_t tiles = (n + kRnTile - 1) / kRnTile;
    const int64_t cells = tiles * kRnBuckets;
    uint32_t *indeg, *hist;
    uint64_t *off, *scan_tmp;
    if ((rc = dev_alloc((void **)&indeg, sizeof(uint32_t) * n, "in-degrees", st))) return rc;
    tmp.push_back(indeg);
    if ((rc = dev_alloc((void **)&hist, sizeof(uint32_t) * cells, "class counts", st))) return rc;
    tmp.push_back(hist);
    if ((rc = dev_alloc((void **)&off, sizeof(uint64_t) * (cells + 1), "class offsets", st))) return rc;
    tmp.push_back(off);
    if ((rc = dev_alloc((void **)&scan_tmp, sizeof(uint64_t) * ((cells + kScanTile - 1) / kScanTile + 2), "scan scratch",
                        st)))
        return rc;
    tmp.push_back(scan_tmp);
    PPR_CUDA(cudaMemsetAsync(indeg, 0, sizeof(uint32_t) * n, st));
    if (m > 0) {
        const int64_t ms = (m + kRnEvery - 1) / kRnEvery;
        const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((ms + 255) / 256, (int64_t)ctx->sms * 32));
        k_rn_indegree<<<eb, 256, 0, st>>>(n, m, d_col, indeg);
        note_launch();
    }
    const int tb = (int)((tiles + 7) / 8);
    k_rn_hist<<<tb, 256, 0, st>>>(n, indeg, hist, tiles);
    note_launch();
    exclusive_scan_u32(hist, cells, off, scan_tmp, st);
    k_rn_scatter<<<tb, 256, 0, st>>>(n, indeg, off, tiles, order, rank);
    note_launch();
    PPR_CUDA(cudaGetLastError());
    return PPR_OK;
}

}  // namespace ppr
