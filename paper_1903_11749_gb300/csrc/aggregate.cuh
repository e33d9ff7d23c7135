// aggregate.cuh -- endpoint aggregation of libppr.so (sm_103a): the R walk
// endpoints of each source become its sparse count row (end ids ascending,
// counts summing to R; pi_hat(s, t) = count / R, Sec. 2.2) and its top-k
// (count descending, then id ascending).  One warp per source; included by
// walk.cu, whose walker writes the endpoints this reads.
#pragma once
#include "ppr_host.h"

namespace ppr {

struct AggOut {
    uint32_t *nnz;       // [S], or null: no rows (top-k only)
    int32_t *cols;       // [S * cap], or null with cnts
    uint32_t *cnts;      // [S * cap]
    int32_t *topk_idx;   // [S * topk]
    uint32_t *topk_cnt;  // [S * topk]
    uint32_t cap;
    int32_t topk;
};

// Caller id of an endpoint the walker wrote in the layout's numbering
// (order: the renumbered layout's order array, else null).
__device__ __forceinline__ uint32_t caller_id(const int32_t *order, uint32_t v)
{
    return order ? (uint32_t)order[v] : v;
}

// ends: the R endpoints of one source (shared memory).  sortbuf: next_pow2(R)
// uint32 and keys: next_pow2(R) uint64 of per-warp shared scratch.  Writes
// row `out_row` of the outputs.  All 32 lanes call it.
__device__ inline void aggregate_source(const uint32_t *ends, uint32_t R, uint32_t *sortbuf, uint64_t *keys,
                                        const AggOut &o, uint64_t out_row, const int32_t *order = nullptr)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t P2 = next_pow2(R);
    for (uint32_t i = lane; i < P2; i += 32) sortbuf[i] = i < R ? caller_id(order, ends[i]) : 0xffffffffu;
    __syncwarp();
    warp_bitonic_sort(sortbuf, P2);
    // One run per distinct endpoint.  A run is found at its last element;
    // its first element comes from a lower-bound search of the sorted buffer.
    const uint64_t rbase = out_row * o.cap;
    uint32_t nrun = 0;
    for (uint32_t base = 0; base < R; base += 32) {
        uint32_t i = base + lane;
        uint32_t v = i < R ? sortbuf[i] : 0u;
        bool tail = i < R && (i == R - 1 || sortbuf[i + 1] != v);
        uint32_t m = __ballot_sync(0xffffffffu, tail);
        if (tail) {
            uint32_t r = nrun + __popc(m & ((1u << lane) - 1));
            uint32_t lo = 0, hi = i;
            while (lo < hi) {
                uint32_t mid = (lo + hi) >> 1;
                if (sortbuf[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            uint32_t c = i - lo + 1;
            if (o.cols) {
                o.cols[rbase + r] = (int32_t)v;
                o.cnts[rbase + r] = c;
            }
            if (o.topk > 0) keys[r] = ((uint64_t)(~c) << 32) | v;
        }
        nrun += __popc(m);
    }
    if (lane == 0 && o.nnz) o.nnz[out_row] = nrun;
    if (o.topk > 0) {
        uint32_t K2 = next_pow2(nrun);
        for (uint32_t i = nrun + lane; i < K2; i += 32) keys[i] = ~0ull;
        __syncwarp();
        warp_bitonic_sort(keys, K2);
        const uint64_t tb = out_row * (uint64_t)o.topk;
        for (uint32_t i = lane; i < (uint32_t)o.topk; i += 32) {
            if (i < nrun) {
                uint64_t k = keys[i];
                o.topk_idx[tb + i] = (int32_t)(uint32_t)k;
                o.topk_cnt[tb + i] = ~(uint32_t)(k >> 32);
            } else {
                o.topk_idx[tb + i] = -1;
                o.topk_cnt[tb + i] = 0;
            }
        }
    }
    __syncwarp();
}

// Register-resident variant for next_pow2(R) = 32 * E <= 1024: the sorted
// block lives in registers in striped order (element i = e * 32 + lane), a
// bitonic network runs on shuffles (partner distance < 32) and in-register
// exchanges (distance >= 32).  Runs are found from neighbour values; the
// top-k sorts 32-bit keys (R - count) << 12 | run, whose order is count
// descending then end id ascending because runs are numbered in id order.
template <int E>
__device__ __forceinline__ void warp_sort_reg(uint32_t (&v)[E])
{
    const uint32_t lane = threadIdx.x & 31;
    constexpr int N = 32 * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int f = e ^ (j >> 5);
                    if (f > e) {
                        const bool up = (((uint32_t)e * 32 + lane) & (uint32_t)k) == 0;
                        const uint32_t a = v[e], b = v[f];
                        const bool sw = (a > b) == up;
                        v[e] = sw ? b : a;
                        v[f] = sw ? a : b;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, v[e], j);
                    const bool up = (((uint32_t)e * 32 + lane) & (uint32_t)k) == 0;
                    const bool lower = (lane & (uint32_t)j) == 0;
                    v[e] = (lower == up) ? min(v[e], o) : max(v[e], o);
                }
            }
        }
    }
}

// Top-K of one row without sorting every run, for K <= 32 and K < nrun:
// kv holds the keys (R - count) << 12 | run of runs e * 32 + lane (0xFFFFFFFF
// past nrun), and the answer is the K smallest keys in ascending order.  The
// count rank q = key >> 12 of the K-th smallest key is found by bisection
// over [0, R - 1] with ballot counts; every key with q below it is taken (fewer
// than K, sorted in one register per lane), then the first keys with q equal
// to it in run order (= ascending key, as runs are numbered in id order)
// fill the remaining places.  cbuf: 32 uint32 of per-warp shared memory.
template <int E>
__device__ __forceinline__ void topk_select_reg(const uint32_t (&kv)[E], uint32_t K, uint32_t R,
                                                const uint32_t *run_id, uint32_t *cbuf, const AggOut &o, uint64_t tb)
{
    const uint32_t lane = threadIdx.x & 31, below = (1u << lane) - 1;
    auto count_le = [&](uint32_t t) {
        uint32_t c = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) c += __popc(__ballot_sync(0xffffffffu, (kv[e] >> 12) <= t));
        return c;
    };
    // smallest t with count_le(t) >= K; count_le(R - 1) = nrun > K.  Most rows
    // have fewer than K runs of count >= 2, so t = R - 1 is tried first.
    uint32_t lo = 0, hi = R - 1;
    if (R >= 2 && count_le(R - 2) < K) lo = R - 1;
    else hi = R >= 2 ? R - 2 : 0;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (count_le(mid) >= K) hi = mid;
        else lo = mid + 1;
    }
    const uint32_t t = lo;
    uint32_t nlt = 0;  // keys below t, gathered into cbuf in run order
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const bool lt = (kv[e] >> 12) < t;
        const uint32_t ml = __ballot_sync(0xffffffffu, lt);
        if (lt) cbuf[nlt + __popc(ml & below)] = kv[e];
        nlt += __popc(ml);
    }
    __syncwarp();
    // nlt < K places for the keys below t, sorted; then K - nlt keys equal to t
    uint32_t v[1] = {lane < nlt ? cbuf[lane] : 0xffffffffu};
    warp_sort_reg<1>(v);
    if (lane < nlt) {
        o.topk_idx[tb + lane] = (int32_t)run_id[v[0] & 0xfffu];
        o.topk_cnt[tb + lane] = R - (v[0] >> 12);
    }
    uint32_t seen = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const bool eq = (kv[e] >> 12) == t;
        const uint32_t me = __ballot_sync(0xffffffffu, eq);
        const uint32_t pos = nlt + seen + __popc(me & below);
        if (eq && pos < K) {
            o.topk_idx[tb + pos] = (int32_t)run_id[kv[e] & 0xfffu];
            o.topk_cnt[tb + pos] = R - t;
        }
        seen += __popc(me);
    }
}

// The whole row in top-k order (K >= nrun): kv as in topk_select_reg.  Runs
// counted once come last (count 1 is the smallest) and already in run order,
// so only the runs counted twice or more are sorted -- in one register per
// lane when at most 32 of them (always when R <= 65) -- and the rest are
// placed by ballot prefix counts.  Returns false (nothing written) when more
// than 32 runs repeat; the caller then sorts every key.
template <int E>
__device__ __forceinline__ bool topk_all_reg(const uint32_t (&kv)[E], uint32_t nrun, uint32_t K, uint32_t R,
                                             const uint32_t *run_id, uint32_t *cbuf, const AggOut &o, uint64_t tb)
{
    const uint32_t lane = threadIdx.x & 31, below = (1u << lane) - 1;
    const uint32_t t1 = (R - 1) << 12;  // keys from here on: count 1 (or no run)
    uint32_t nm = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) nm += __popc(__ballot_sync(0xffffffffu, kv[e] < t1));
    if (nm > 32) return false;
    uint32_t seen = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const bool rep = kv[e] < t1;
        const uint32_t mr = __ballot_sync(0xffffffffu, rep);
        if (rep) cbuf[seen + __popc(mr & below)] = kv[e];
        seen += __popc(mr);
    }
    __syncwarp();
    uint32_t v[1] = {lane < nm ? cbuf[lane] : 0xffffffffu};
    warp_sort_reg<1>(v);
    if (lane < nm && lane < K) {
        o.topk_idx[tb + lane] = (int32_t)run_id[v[0] & 0xfffu];
        o.topk_cnt[tb + lane] = R - (v[0] >> 12);
    }
    uint32_t ones = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)e * 32 + lane;
        const bool one = i < nrun && kv[e] >= t1;
        const uint32_t m1 = __ballot_sync(0xffffffffu, one);
        const uint32_t pos = nm + ones + __popc(m1 & below);
        if (one && pos < K) {
            o.topk_idx[tb + pos] = (int32_t)run_id[kv[e] & 0xfffu];
            o.topk_cnt[tb + pos] = 1;
        }
        ones += __popc(m1);
    }
    for (uint32_t i = nrun + lane; i < K; i += 32) {
        o.topk_idx[tb + i] = -1;
        o.topk_cnt[tb + i] = 0;
    }
    return true;
}

// scratch: 3 * R uint32 of per-warp shared memory
template <int E>
__device__ inline void aggregate_source_reg(const uint32_t *ends, uint32_t R, uint32_t *scratch, const AggOut &o,
                                            uint64_t out_row, const int32_t *order = nullptr)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t *start_pos = scratch, *run_id = scratch + R, *kbuf = scratch + 2 * R;
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)e * 32 + lane;
        v[e] = i < R ? ends[i] : 0xffffffffu;
    }
    const uint64_t rbase = out_row * o.cap;
    // A row whose R endpoints are all one node (a dangling source, whose walks
    // restart where they began: 4-6 % of the sources of the R-MAT graphs) is
    // one run of count R; it skips the sort.
    const uint32_t v0 = __shfl_sync(0xffffffffu, v[0], 0);
    bool same = true;
#pragma unroll
    for (int e = 0; e < E; ++e) same = same && ((uint32_t)e * 32 + lane >= R || v[e] == v0);
    if (__all_sync(0xffffffffu, same)) {
        const int32_t id = (int32_t)caller_id(order, v0);
        if (lane == 0) {
            if (o.cols) {
                o.cols[rbase] = id;
                o.cnts[rbase] = R;
            }
            if (o.nnz) o.nnz[out_row] = 1;
        }
        const uint64_t tb = out_row * (uint64_t)o.topk;
        for (uint32_t i = lane; i < (uint32_t)max(o.topk, 0); i += 32) {
            o.topk_idx[tb + i] = i == 0 ? id : -1;
            o.topk_cnt[tb + i] = i == 0 ? R : 0u;
        }
        __syncwarp();
        return;
    }
    if (order) {
#pragma unroll
        for (int e = 0; e < E; ++e)
            if ((uint32_t)e * 32 + lane < R) v[e] = (uint32_t)order[v[e]];
    }
    warp_sort_reg<E>(v);
    uint32_t nrun = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)e * 32 + lane;
        const uint32_t pu = __shfl_up_sync(0xffffffffu, v[e], 1);
        const uint32_t pe = __shfl_sync(0xffffffffu, v[e > 0 ? e - 1 : 0], 31);
        const uint32_t nd = __shfl_down_sync(0xffffffffu, v[e], 1);
        const uint32_t ne = __shfl_sync(0xffffffffu, v[e + 1 < E ? e + 1 : e], 0);
        const uint32_t prev = lane == 0 ? pe : pu;
        const uint32_t next = lane == 31 ? ne : nd;
        const bool valid = i < R;
        const bool head = valid && (i == 0 || prev != v[e]);
        const bool tail = valid && (i == R - 1 || next != v[e]);
        const uint32_t hb = __ballot_sync(0xffffffffu, head);
        const uint32_t run = nrun + __popc(hb & ((2u << lane) - 1)) - 1;  // run of element i
        if (head) {
            start_pos[run] = i;
            run_id[run] = v[e];
        }
        __syncwarp();
        if (tail) {
            const uint32_t c = i - start_pos[run] + 1;
            if (o.cols) {
                o.cols[rbase + run] = (int32_t)v[e];
                o.cnts[rbase + run] = c;
            }
            kbuf[run] = ((R - c) << 12) | run;
        }
        nrun += __popc(hb);
    }
    if (lane == 0 && o.nnz) o.nnz[out_row] = nrun;
    if (o.topk > 0) {
        __syncwarp();
        uint32_t kv[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t i = (uint32_t)e * 32 + lane;
            kv[e] = i < nrun ? kbuf[i] : 0xffffffffu;
        }
        const uint64_t tb = out_row * (uint64_t)o.topk;
        const uint32_t K = (uint32_t)o.topk;
        if (E > 1 && K <= 32 && K < nrun) {
            topk_select_reg<E>(kv, K, R, run_id, start_pos, o, tb);
        } else if (E > 1 && E <= 8 && K >= nrun && topk_all_reg<E>(kv, nrun, K, R, run_id, start_pos, o, tb)) {
            // the whole row, in top-k order (R <= 256)
        } else {
            warp_sort_reg<E>(kv);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint32_t i = (uint32_t)e * 32 + lane;
                if (i < K) {
                    if (i < nrun) {
                        o.topk_idx[tb + i] = (int32_t)run_id[kv[e] & 0xfffu];
                        o.topk_cnt[tb + i] = R - (kv[e] >> 12);
                    } else {
                        o.topk_idx[tb + i] = -1;
                        o.topk_cnt[tb + i] = 0;
                    }
                }
            }
            // k may exceed the sorted block (k > next_pow2(R) >= nnz): pad the rest
            for (uint32_t i = 32u * E + lane; i < K; i += 32) {
                o.topk_idx[tb + i] = -1;
                o.topk_cnt[tb + i] = 0;
            }
        }
    }
    __syncwarp();
}

// Launch parameters of k_aggregate: S sources, R endpoints each, source-major.
struct AggParams {
    const uint32_t *ends;
    uint32_t R, P2;     // P2 = next_pow2(R)
    int64_t S;
    int64_t out_row0;   // output row of the first source
    AggOut out;
    const int32_t *order;  // renumbered layout: caller id of an internal node, else null
};

// E > 0: register-resident reduction for next_pow2(R) = 32 * E; E = 0:
// shared-memory reduction (any R).  Four warps per block, 12 * P2 bytes of
// shared scratch per warp.
template <int E>
__global__ void __launch_bounds__(128) k_aggregate(AggParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned char *scratch = smem_raw + (size_t)wid * p.P2 * 12;
    const uint64_t S = (uint64_t)p.S;
    for (uint64_t i = (uint64_t)blockIdx.x * nw + wid; i < S; i += (uint64_t)gridDim.x * nw) {
        if constexpr (E > 0) {
            aggregate_source_reg<E>(p.ends + i * p.R, p.R, reinterpret_cast<uint32_t *>(scratch), p.out,
                                    (uint64_t)p.out_row0 + i, p.order);
        } else {
            uint64_t *keys = reinterpret_cast<uint64_t *>(scratch);
            aggregate_source(p.ends + i * p.R, p.R, reinterpret_cast<uint32_t *>(keys + p.P2), keys, p.out,
                             (uint64_t)p.out_row0 + i, p.order);
        }
    }
}

template <int E>
static int launch_aggregate_e(ppr_ctx *ctx, const AggParams &ap, cudaStream_t st)
{
    const int aw = 4;
    size_t smem = (size_t)aw * ap.P2 * 12;
    if (smem > 48 * 1024)
        PPR_CUDA(cudaFuncSetAttribute(k_aggregate<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int ablocks = (int)std::min<int64_t>((ap.S + aw - 1) / aw, (int64_t)ctx->sms * 16);
    if (ablocks < 1) ablocks = 1;
    k_aggregate<E><<<ablocks, aw * 32, smem, st>>>(ap);
    note_launch();
    PPR_CUDA(cudaGetLastError());
    return PPR_OK;
}

static int launch_aggregate(ppr_ctx *ctx, const AggParams &ap, cudaStream_t st)
{
    switch (ap.P2) {
    case 1: case 2: case 4: case 8: case 16: case 32: return launch_aggregate_e<1>(ctx, ap, st);
    case 64: return launch_aggregate_e<2>(ctx, ap, st);
    case 128: return launch_aggregate_e<4>(ctx, ap, st);
    case 256: return launch_aggregate_e<8>(ctx, ap, st);
    case 512: return launch_aggregate_e<16>(ctx, ap, st);
    case 1024: return launch_aggregate_e<32>(ctx, ap, st);
    default: return launch_aggregate_e<0>(ctx, ap, st);
    }
}

}  // namespace ppr
