// Random-gather probe: the empirical ceiling for the index gathers of the search path.
// Each thread reads `per_thread` granules of `granule` bytes (32, 64 or 128) at uniformly
// random granule-aligned offsets of a device buffer, `inflight` of them in flight at a time,
// and folds them into one word so the loads stay live.  Offsets come from a splitmix64 hash
// of (seed, thread, iteration) (Steele, Lea and Flood 2014).  Measurement only: it reads the
// caller's buffer and writes one word per thread to `sink`.
#include "fm_internal.cuh"

namespace fm {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int G, int U>
__global__ void __launch_bounds__(256) k_probe_gather(const uint8_t *__restrict__ buf,
                                                       uint64_t n_granules, uint32_t per_thread,
                                                       uint64_t seed, uint32_t *__restrict__ sink) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint32_t i = 0; i < per_thread; i += U) {
        uint4 v[U][2 * (G / 32)];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t h = mix64(seed + 0x9E3779B97F4A7C15ull * (t * per_thread + i + u + 1));
            const uint8_t *p = buf + __umul64hi(h, n_granules) * G;   // uniform in [0, n)
#pragma unroll
            for (int s = 0; s < G / 32; ++s) ldg256(p + 32 * s, v[u][2 * s], v[u][2 * s + 1]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int s = 0; s < 2 * (G / 32); ++s) acc ^= v[u][s].x ^ v[u][s].y ^ v[u][s].z ^ v[u][s].w;
    }
    sink[t] = acc;
}

}  // namespace
}  // namespace fm

using namespace fm;

template <int G>
static void launch_probe(uint32_t inflight, unsigned grid, cudaStream_t st, const uint8_t *buf,
                         uint64_t ng, uint32_t per, uint64_t seed, uint32_t *sink) {
    switch (inflight) {
        case 1: k_probe_gather<G, 1><<<grid, 256, 0, st>>>(buf, ng, per, seed, sink); break;
        case 2: k_probe_gather<G, 2><<<grid, 256, 0, st>>>(buf, ng, per, seed, sink); break;
        case 8: k_probe_gather<G, 8><<<grid, 256, 0, st>>>(buf, ng, per, seed, sink); break;
        default: k_probe_gather<G, 4><<<grid, 256, 0, st>>>(buf, ng, per, seed, sink); break;
    }
}

extern "C" int fm_probe_gather(const void *buf, uint64_t bytes, uint32_t granule,
                               uint32_t threads, uint32_t per_thread, uint32_t inflight,
                               uint64_t seed, uint32_t *sink, void *stream) {
    if (!buf || !sink || (granule != 32 && granule != 64 && granule != 128) || bytes < granule ||
        ((uintptr_t)buf & 31) || threads % 256 ||
        (inflight != 1 && inflight != 2 && inflight != 4 && inflight != 8) ||
        per_thread % inflight)
        return set_global_error(FM_EINVAL, "fm_probe_gather: bad argument");
    const uint64_t ng = bytes / granule;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned grid = threads / 256;
    const uint8_t *b = (const uint8_t *)buf;
    switch (granule) {
        case 32: launch_probe<32>(inflight, grid, st, b, ng, per_thread, seed, sink); break;
        case 64: launch_probe<64>(inflight, grid, st, b, ng, per_thread, seed, sink); break;
        default: launch_probe<128>(inflight, grid, st, b, ng, per_thread, seed, sink); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_global_error(FM_ECUDA, cudaGetErrorString(e));
    return FM_OK;
}
