// Random-gather probe for bench.py (a measurement aid, not part of libshm.so): the memory traffic of
// an uncorrelated query batch without its arithmetic.  Per item q: read 12 B of input, gather one
// aligned block of `block_bytes` (16..64) at a hashed position in `table`, write 28 B.  The bench
// times it beside the random planet query to show what the memory system sustains for that access
// pattern.  Built by bench_probe/__init__.py into bench_probe/_build/libgather_probe.so.
#include <cuda_runtime.h>
#include <stdint.h>

// Four items per thread per round, all four gathers issued before any is consumed, so that each
// thread keeps four independent misses in flight (the probe should not be latency-limited where
// the query kernel is not).
__device__ __forceinline__ int64_t probe_block(float a, float b, float c, int64_t n_blocks)
{
    uint64_t h = ((uint64_t)__float_as_uint(a) << 32) ^ __float_as_uint(b) ^ ((uint64_t)__float_as_uint(c) << 17);
    h ^= h >> 33; h *= 0xff51afd7ed558ccdull; h ^= h >> 33; h *= 0xc4ceb9fe1a85ec53ull; h ^= h >> 33;
    return (int64_t)(h % (uint64_t)n_blocks);
}

__global__ void __launch_bounds__(512) k_gather_probe(const float4* __restrict__ table, int64_t n_blocks, int block_v4,
                                                      int64_t Q, const float* __restrict__ in, float* __restrict__ out)
{
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q0 < Q; q0 += U * stride) {
        int64_t blk[U];
        float acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t q = q0 + u * stride;
            blk[u] = -1;
            acc[u] = 0.0f;
            if (q < Q) blk[u] = probe_block(__ldg(in + 3 * q), __ldg(in + 3 * q + 1), __ldg(in + 3 * q + 2), n_blocks);
        }
        float4 t[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v)
                t[u][v] = (blk[u] >= 0 && v < block_v4) ? __ldg(table + blk[u] * block_v4 + v) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t q = q0 + u * stride;
            if (q >= Q) continue;
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u] += t[u][v].x + t[u][v].y + t[u][v].z + t[u][v].w;
            out[7 * q] = acc[u];
            for (int k = 1; k < 7; ++k) out[7 * q + k] = acc[u] * (float)k;
        }
    }
}

// Returns 0 on success, 1 for an invalid argument, 4 for a CUDA error (the status codes of shm.h).
extern "C" int gather_probe(const void* table, int64_t table_bytes, int32_t block_bytes, int64_t Q, const float* in,
                            float* out, cudaStream_t s)
{
    if (!table || Q < 0 || (Q > 0 && (!in || !out))) return 1;
    if (block_bytes < 16 || block_bytes > 64 || block_bytes % 16 != 0 || ((uintptr_t)table & 15u) != 0 ||
        table_bytes < block_bytes)
        return 1;
    if (Q == 0) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 4;
    const int v4 = block_bytes / 16;
    const int64_t n_blocks = table_bytes / block_bytes;
    int64_t blocks = (Q + 511) / 512;
    const int64_t cap = (int64_t)sms * 4;
    if (blocks > cap) blocks = cap;
    k_gather_probe<<<(unsigned)blocks, 512, 0, s>>>(reinterpret_cast<const float4*>(table), n_blocks, v4, Q, in, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

