// Forward query kernel skeleton: direction -> face/uv -> 2x2 texel fetch -> Hermite value + chart
// gradient -> S^2 gradient -> normal (arXiv 2602.20063, §3.2-§3.4).
//
// One thread per query; warps cover 32 consecutive queries so direction loads and output stores
// stay coalesced; for CSR segments one binary search per warp and chunk finds the glyph of the
// warp's first query and each lane then walks forward.
// The path is bound by HBM bandwidth: 12 B of direction, 4 corner records (64 B f32 / 32 B
// 16-bit) and 28 B of outputs per query against ~250 flops.
//
// The skeleton is shared with the value-only reconstruction baselines (RECON >= 0, shm_recon.cu),
// which replace the 2x2 Hermite footprint by their own and keep the work distribution, glyph
// lookup and I/O path, so that measured differences come from the footprint and arithmetic.
#pragma once
#include "shm_internal.h"

namespace shm {

// Launch shapes (threads per CTA, rounds per CTA chunk): a CTA takes BLOCK * IT consecutive
// queries.  Shape 0 is the default; shm_tune_query times the others on a caller's batch and
// records the fastest per (path, dtype, layout) for later calls.
struct QShape {
    int block, it;
};
constexpr int N_QSHAPES = 4;
constexpr QShape QSHAPES[N_QSHAPES] = {{512, 8}, {256, 16}, {1024, 4}, {256, 8}};

// Work is handed out per CTA in contiguous chunks (4,096 queries by default), so that for per-glyph query
// segments a CTA serves whole glyphs and the glyph's table stays in that SM's L1 (two CTAs per SM
// keep two tables of up to ~110 KB resident) instead of being pulled into several SMs.
//
// VEC (all of dirs / grad / normal 16-byte aligned): for a full warp round (32 queries) the 384 B
// of directions are read with 24 128-bit loads and the 384 B of gradients and of normals are
// written with 24 128-bit stores, re-distributed through a 384-byte per-warp shared buffer, so a
// warp issues 1 + 4 + 3 global memory instructions per round instead of 3 + 4 + 7 (the load/store
// queue, not DRAM, limited the random-access case).  Partial rounds use scalar accesses.
// The Hermite query keeps <= 64 registers (1,024 resident threads per SM); the 16-tap baselines
// need more than 64 registers: one resident CTA of 512 per SM for them.
template <int RECON, int QBLOCK>
struct QueryOccupancy {
    static constexpr int min_blocks = (RECON >= SHM_RECON_BICUBIC) ? 1 : (QBLOCK >= 1024 ? 1 : 1024 / QBLOCK);
};

template <int DT, int LAYOUT, bool VEC, int RECON, int QBLOCK = 512, int QIT = 8>
__global__ void __launch_bounds__(QBLOCK, (QueryOccupancy<RECON, QBLOCK>::min_blocks)) k_query_fwd(QueryArgs a)
{
    __shared__ __align__(16) float sbuf[QBLOCK / 32][96];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* wb = sbuf[warp];
    const int64_t CH = (int64_t)QBLOCK * QIT;
    const int G = a.L.n_glyphs;
    uint32_t status = 0;
    const float qnan = __int_as_float(0x7fc00000);
    const float4* dirs4 = reinterpret_cast<const float4*>(a.dirs);

    for (int64_t c0 = (int64_t)blockIdx.x * CH; c0 < a.Q; c0 += (int64_t)gridDim.x * CH) {
        // glyph of this lane's first query and the end of its segment (one search per warp and chunk)
        int g = 0;
        int64_t seg_end = INT64_MAX;
        const int64_t qw0 = c0 + warp * 32;
        if (a.seg) {
            int g0 = 0;
            long long e0 = 0;
            if (lane == 0 && qw0 < a.Q) {
                g0 = (qw0 < __ldg(a.seg)) ? -1 : seg_find(a.seg, G, qw0);
                e0 = (g0 >= 0 && g0 < G) ? __ldg(a.seg + g0 + 1) : 0;
            }
            g = __shfl_sync(0xffffffffu, g0, 0);
            seg_end = __shfl_sync(0xffffffffu, e0, 0);
        }
        // direction of the first round: vector (full round) or scalar
        float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
        float n0 = 0.f, n1 = 0.f, n2 = 0.f;
        if (VEC && qw0 + 32 <= a.Q) {
            if (lane < 24) pv = __ldg(dirs4 + (3 * qw0) / 4 + lane);
        } else if (qw0 + lane < a.Q) {
            const int64_t q = qw0 + lane;
            n0 = __ldcs(a.dirs + 3 * q); n1 = __ldcs(a.dirs + 3 * q + 1); n2 = __ldcs(a.dirs + 3 * q + 2);
        }
#pragma unroll 1
        for (int it = 0; it < QIT; ++it) {
            const int64_t qw = qw0 + (int64_t)it * QBLOCK;
            if (qw >= a.Q) break;
            const bool full = VEC && (qw + 32 <= a.Q);
            const int64_t q = qw + lane;
            float d0, d1, d2;
            if (full) {
                // re-distribute the warp's 24 float4 of directions: lane L takes floats 3L..3L+2
                if (lane < 24) reinterpret_cast<float4*>(wb)[lane] = pv;
                __syncwarp();
                d0 = wb[3 * lane]; d1 = wb[3 * lane + 1]; d2 = wb[3 * lane + 2];
                __syncwarp();
            } else {
                if (q >= a.Q) break;
                d0 = n0; d1 = n1; d2 = n2;
            }
            // prefetch the next round's directions: the latency overlaps the table fetch below
            if (it + 1 < QIT) {
                const int64_t qn = qw + QBLOCK;
                if (VEC && qn + 32 <= a.Q) {
                    if (lane < 24) pv = __ldg(dirs4 + (3 * qn) / 4 + lane);
                } else if (qn + lane < a.Q) {
                    n0 = __ldcs(a.dirs + 3 * (qn + lane));
                    n1 = __ldcs(a.dirs + 3 * (qn + lane) + 1);
                    n2 = __ldcs(a.dirs + 3 * (qn + lane) + 2);
                }
            }
            int gq = 0;
            if (a.glyph) {
                gq = __ldg(a.glyph + q);
            } else if (a.seg) {
                if (q >= seg_end || g < 0) {
                    if (g < 0 && q >= __ldg(a.seg)) g = 0;
                    while (g >= 0 && g < G && q >= __ldg(a.seg + g + 1)) ++g;
                    seg_end = (g >= 0 && g < G) ? __ldg(a.seg + g + 1) : INT64_MAX;
                }
                gq = g;
            }
            bool valid = true;
            if (gq < 0 || gq >= G) { valid = false; status |= SHM_DEV_BOUNDS; }
            QueryResult r;
            Chart c;
            if (valid) {
                const GlyphRef Gr = glyph_ref(a.L, gq);
                if constexpr (RECON < 0) valid = query_one<DT, LAYOUT>(a.L, Gr, d0, d1, d2, r, c);
                else valid = recon_one<RECON, DT>(a.L, Gr, d0, d1, d2, r, c);
                if (!valid) status |= SHM_DEV_NONFINITE;
            }
            if (!valid) {
                r.R = r.Ru = r.Rv = qnan;
                r.grad = Vec3{qnan, qnan, qnan};
                r.f = r.i = r.j = -1;
            }
            const Vec3 n = (a.normal && valid) ? surface_normal(d0, d1, d2, r.R, r.grad) : Vec3{qnan, qnan, qnan};
            if (a.R) __stcs(a.R + q, r.R);
            if (full) {
                if (a.grad) {
                    wb[3 * lane] = r.grad.x; wb[3 * lane + 1] = r.grad.y; wb[3 * lane + 2] = r.grad.z;
                    __syncwarp();
                    if (lane < 24) __stcs(reinterpret_cast<float4*>(a.grad) + (3 * qw) / 4 + lane, reinterpret_cast<const float4*>(wb)[lane]);
                    __syncwarp();
                }
                if (a.normal) {
                    wb[3 * lane] = n.x; wb[3 * lane + 1] = n.y; wb[3 * lane + 2] = n.z;
                    __syncwarp();
                    if (lane < 24) __stcs(reinterpret_cast<float4*>(a.normal) + (3 * qw) / 4 + lane, reinterpret_cast<const float4*>(wb)[lane]);
                    __syncwarp();
                }
            } else {
                if (a.grad) {
                    a.grad[3 * q] = r.grad.x;
                    a.grad[3 * q + 1] = r.grad.y;
                    a.grad[3 * q + 2] = r.grad.z;
                }
                if (a.normal) {
                    a.normal[3 * q] = n.x;
                    a.normal[3 * q + 1] = n.y;
                    a.normal[3 * q + 2] = n.z;
                }
            }
            if (a.chart) {
                a.chart[2 * q] = r.Ru;
                a.chart[2 * q + 1] = r.Rv;
            }
            if (a.fij) {
                a.fij[3 * q] = r.f;
                a.fij[3 * q + 1] = r.i;
                a.fij[3 * q + 2] = r.j;
            }
        }
    }
    report_status(a.dev_status, status);
}

template <int DT, int LAYOUT, bool VEC, int RECON, int QBLOCK, int QIT>
cudaError_t launch_fwd_v(const QueryArgs& a, cudaStream_t s)
{
    // one persistent wave: SMs x resident blocks per SM
    static int resident = 0;
    if (resident == 0) {
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_query_fwd<DT, LAYOUT, VEC, RECON, QBLOCK, QIT>, QBLOCK,
                                                          0) != cudaSuccess ||
            r < 1)
            r = QueryOccupancy<RECON, QBLOCK>::min_blocks;
        resident = r;
    }
    int64_t blocks = (a.Q + (int64_t)QBLOCK * QIT - 1) / ((int64_t)QBLOCK * QIT);
    const int64_t cap = (int64_t)sm_count() * resident;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_query_fwd<DT, LAYOUT, VEC, RECON, QBLOCK, QIT><<<(unsigned)blocks, QBLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// The vector I/O path measured 4 % faster on uniform random queries of one large table and 7 %
// slower on per-glyph CSR segments (GB300, 2^28 planet queries / 2^26 glyph-field queries), so it
// is used when there are no segments and the buffers are 16-byte aligned.
template <int DT, int LAYOUT, int RECON, int QBLOCK = 512, int QIT = 8>
cudaError_t launch_fwd_t(const QueryArgs& a, cudaStream_t s)
{
    const auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    if (!a.seg && al16(a.dirs) && al16(a.grad) && al16(a.normal))
        return launch_fwd_v<DT, LAYOUT, true, RECON, QBLOCK, QIT>(a, s);
    return launch_fwd_v<DT, LAYOUT, false, RECON, QBLOCK, QIT>(a, s);
}

}  // namespace shm
