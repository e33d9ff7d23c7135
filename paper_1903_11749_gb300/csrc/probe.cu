// probe.cu -- measurement probes beside the walk path.
//
// ppr_probe_philox:  the device's Philox4x32-10 words for a run of counters
//                    (the generator every walk step draws from), for a
//                    bit-for-bit comparison with an independent host one.
// ppr_probe_rate:    the practical ceilings a walk step is measured against:
//   kind 0 (chains): chains of dependent random 32-byte sector reads over a
//                    device buffer, one 256-bit load per read; the next
//                    address depends on the loaded value, as a walk's next
//                    node does (uniform addresses: no hot nodes).
//   kind 1 (philox): Philox4x32-10 draws per second with no memory traffic.
//   kind 2 (gather): independent random 32-byte sector reads, four in
//                    flight per thread: the random-access bandwidth of the
//                    memory system for sector-sized reads.
#include <algorithm>
#include <chrono>

#include "ppr_host.h"

namespace ppr {

__global__ void k_probe_philox(uint4 c0, uint32_t k0, uint32_t k1, int64_t count, uint4 *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint4 c = c0;
        c.x += (uint32_t)i;  // counter word 0 advances (mod 2^32)
        out[i] = philox4x32_10(c, k0, k1);
    }
}

// splitmix-style finaliser for the probe's addresses (not a walk draw)
__device__ __forceinline__ uint64_t probe_mix(uint64_t z)
{
    z ^= z >> 31;
    z *= 0x7fb5d329728ea185ull;
    z ^= z >> 27;
    z *= 0x81dadef4bc2dd44dull;
    return z ^ (z >> 33);
}

__global__ void k_probe_fill(uint32_t *buf, int64_t words)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
        buf[i] = (uint32_t)probe_mix((uint64_t)i);
}

__global__ void __launch_bounds__(256, 6) k_probe_gather(const uint32_t *buf, uint64_t sectors, int32_t steps,
                                                         unsigned long long *sink)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t h = probe_mix(tid + 1);
    uint32_t acc = 0;
    for (int32_t s = 0; s < steps; ++s) {
        const uint64_t idx = __umul64hi(h, sectors);  // uniform in [0, sectors)
        const Sector v = ld_sector(buf + 8 * idx);
        acc ^= v.v[0] ^ v.v[7];
        h = probe_mix(h ^ v.v[3]);  // the next address depends on the loaded sector
    }
    if (acc == 0x9e3779b9u) atomicAdd(sink, 1ull);  // keeps the loads live
}

__global__ void __launch_bounds__(256, 6) k_probe_gather_indep(const uint32_t *buf, uint64_t sectors, int32_t rounds,
                                                               unsigned long long *sink)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int32_t s = 0; s < rounds; ++s) {
        Sector v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint64_t h = probe_mix((tid << 24) ^ ((uint64_t)s << 2) ^ (uint64_t)q);
            v[q] = ld_sector(buf + 8 * __umul64hi(h, sectors));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc ^= v[q].v[2 * q];
    }
    if (acc == 0x9e3779b9u) atomicAdd(sink, 1ull);
}

__global__ void __launch_bounds__(256, 6) k_probe_philox_rate(uint32_t k0, uint32_t k1, int32_t per_thread,
                                                              unsigned long long *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int32_t j = 0; j < per_thread; ++j) {
        const uint4 x = philox4x32_10(make_uint4(tid, (uint32_t)j, 0u, 0u), k0, k1);
        acc ^= x.x ^ x.y ^ x.z;
    }
    if (acc == 0x9e3779b9u) atomicAdd(sink, 1ull);
}

}  // namespace ppr

using namespace ppr;

extern "C" int ppr_probe_philox(ppr_ctx *ctx, uint64_t seed, const uint32_t counter[4], int64_t count, uint32_t *out)
{
    if (!ctx || !counter || !out || count < 1 || count > (1ll << 28)) {
        set_error("need a context, a counter, an output and 1 <= count <= 2^28");
        return PPR_EINVAL;
    }
    PPR_CUDA(cudaSetDevice(ctx->device));
    uint4 *d = nullptr;
    int rc;
    if ((rc = dev_alloc((void **)&d, sizeof(uint4) * count, "probe words", nullptr))) return rc;
    const uint4 c0 = make_uint4(counter[0], counter[1], counter[2], counter[3]);
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)ctx->sms * 16);
    k_probe_philox<<<blocks, 256>>>(c0, (uint32_t)seed, (uint32_t)(seed >> 32), count, d);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(uint4) * count, cudaMemcpyDeviceToHost);
    dev_free(d, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "philox probe");
    return PPR_OK;
}

extern "C" int ppr_probe_rate(ppr_ctx *ctx, int32_t kind, int64_t bytes, double *per_second, float *ms)
{
    const bool mem = kind == 0 || kind == 2;
    if (!ctx || !per_second || kind < 0 || kind > 2 || (mem && (bytes < (1 << 20) || bytes > (1ll << 40)))) {
        set_error("kind 0 (chains) or 2 (gather) with 1 MiB <= bytes <= 2^40, or 1 (philox); and an output");
        return PPR_EINVAL;
    }
    PPR_CUDA(cudaSetDevice(ctx->device));
    int rc;
    unsigned long long *sink = nullptr;
    uint32_t *buf = nullptr;
    if ((rc = dev_alloc((void **)&sink, sizeof(unsigned long long), "probe sink", nullptr))) return rc;
    const int blocks = ctx->sms * 6;  // one resident wave of 256-thread blocks, as the walker
    const double threads = (double)blocks * 256;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double units = 0;
    const uint64_t sectors = (uint64_t)bytes / 32;
    if (e == cudaSuccess && mem) {
        if ((rc = dev_alloc((void **)&buf, sectors * 32, "probe buffer", nullptr))) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            dev_free(sink, nullptr);
            return rc;
        }
        k_probe_fill<<<ctx->sms * 16, 256>>>(buf, (int64_t)sectors * 8);
        note_launch();
        const int32_t steps = 256;
        if (kind == 0) {
            k_probe_gather<<<blocks, 256>>>(buf, sectors, 16, sink);  // warm-up
            note_launch();
            e = cudaEventRecord(e0);
            k_probe_gather<<<blocks, 256>>>(buf, sectors, steps, sink);
        } else {
            k_probe_gather_indep<<<blocks, 256>>>(buf, sectors, 2, sink);
            note_launch();
            e = cudaEventRecord(e0);
            k_probe_gather_indep<<<blocks, 256>>>(buf, sectors, steps / 4, sink);
        }
        note_launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        units = threads * steps;
    } else if (e == cudaSuccess) {
        const int32_t per = 512;
        k_probe_philox_rate<<<blocks, 256>>>(1u, 2u, 8, sink);
        note_launch();
        e = cudaEventRecord(e0);
        k_probe_philox_rate<<<blocks, 256>>>(1u, 2u, per, sink);
        note_launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        units = threads * per;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(buf, nullptr);
    dev_free(sink, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "rate probe");
    *per_second = units / (t * 1e-3);
    if (ms) *ms = t;
    return PPR_OK;
}
