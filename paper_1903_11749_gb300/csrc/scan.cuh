// scan.cuh -- exclusive prefix sum of uint32 counts into uint64 offsets, three
// passes: per-tile sums, one-block scan of the tile sums, per-tile scan with
// the tile's offset.  Used for segment-table offsets and compacted rows.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ppr {

void note_launch();

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline uint64_t block_exclusive_scan(uint64_t v, uint64_t *warp_tot, uint64_t *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive warp totals
        if (lane == nw - 1) *total = t;
    }
    __syncthreads();
    uint64_t before = wid > 0 ? warp_tot[wid - 1] : 0;
    uint64_t r = before + x - v;
    __syncthreads();
    return r;
}

static __global__ void k_scan_tile_sums(const uint32_t *in, int64_t n, uint64_t *tile_sums)
{
    __shared__ uint64_t wt[32];
    __shared__ uint64_t tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    block_exclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// One block scans `tiles` sums in place (exclusive), looping over chunks.
static __global__ void k_scan_tile_offsets(uint64_t *tile_sums, int64_t tiles, uint64_t *grand_total)
{
    __shared__ uint64_t wt[32];
    __shared__ uint64_t tot;
    uint64_t carry = 0;
    for (int64_t b = 0; b < tiles; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        uint64_t v = i < tiles ? tile_sums[i] : 0;
        uint64_t ex = block_exclusive_scan(v, wt, &tot);
        if (i < tiles) tile_sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

static __global__ void k_scan_apply(const uint32_t *in, int64_t n, const uint64_t *tile_off, uint64_t *out)
{
    __shared__ uint64_t wt[32];
    __shared__ uint64_t tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    uint64_t ex = block_exclusive_scan(s, wt, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (n > 0 && base <= n - 1 && n - 1 < base + kScanItems) out[n] = ex;  // holder of element n-1 writes the total
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.  tmp needs
// ceil(n / kScanTile) + 1 uint64.  Enqueued on st.
inline void exclusive_scan_u32(const uint32_t *in, int64_t n, uint64_t *out, uint64_t *tmp, cudaStream_t st)
{
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
        return;
    }
    k_scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp);
    note_launch();
    k_scan_tile_offsets<<<1, 1024, 0, st>>>(tmp, tiles, tmp + tiles);
    note_launch();
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp, out);
    note_launch();
}

}  // namespace ppr
