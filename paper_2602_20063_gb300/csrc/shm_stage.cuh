// Shared-memory staging of one glyph's table for the per-glyph segment kernels (forward query,
// reverse pass): one thread issues cp.async.bulk copies completing on an mbarrier, every thread
// waits on it with a time limit.
#pragma once
#include "shm_internal.h"

namespace shm {
namespace stage {

constexpr uint64_t WAIT_NS = 1000000000ull;   // 1 s
constexpr uint64_t DRAIN_NS = 100000000ull;   // 100 ms
constexpr uint32_t BULK_PIECE = 32768;        // bytes per cp.async.bulk
constexpr int TABLE_OFFSET = 128;             // mbarrier first, table 128-byte aligned

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint64_t limit)
{
    if (bar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!bar_try_wait(bar, parity))
        if (gtimer() - t0 > limit) return false;
    return true;
}

// Thread 0 of the CTA: initialise the barrier (once per kernel).
__device__ __forceinline__ void init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Thread 0: copy `bytes` (a multiple of 16, 16-byte aligned source) into shared memory at dst,
// completing on `bar`.  Earlier generic-proxy reads of the destination are ordered before it.
__device__ __forceinline__ void issue(uint32_t bar, uint32_t dst, const unsigned char* src, uint32_t bytes)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    for (uint32_t off = 0; off < bytes; off += BULK_PIECE) {
        const uint32_t n = min(BULK_PIECE, bytes - off);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(dst + off), "l"(src + off), "r"(n), "r"(bar)
                     : "memory");
    }
}

template <int DT>
__device__ __forceinline__ float4 rec(const unsigned char* table, int r)
{
    if (DT == SHM_F32) return reinterpret_cast<const float4*>(table)[r];
    const uint2 v = reinterpret_cast<const uint2*>(table)[r];
    return DT == SHM_F16 ? h4_to_f4(v) : b4_to_f4(v);
}

// The 2x2 footprint of cell (i, j) on face f from a staged texel table of padded width P.
template <int DT>
__device__ __forceinline__ Corners corners(const unsigned char* table, int P, int f, int i, int j)
{
    const int r = (f * P + j) * P + i;
    Corners c;
    c.c00 = rec<DT>(table, r);
    c.c10 = rec<DT>(table, r + 1);
    c.c01 = rec<DT>(table, r + P);
    c.c11 = rec<DT>(table, r + P + 1);
    return c;
}

}  // namespace stage
}  // namespace shm
