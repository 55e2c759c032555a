// Forward query kernel: direction -> face/uv -> 2x2 texel fetch -> Hermite value + chart
// gradient -> S^2 gradient -> normal (arXiv 2602.20063, §3.2-§3.4).
//
// One thread per query.  Work is handed out in warp-contiguous chunks of 32*QCHUNK queries so
// that direction loads and output stores stay coalesced and, for CSR segments, one binary
// search per chunk finds the glyph of the chunk's first query; each lane then walks forward.
// The path is bound by HBM bandwidth: 12 B of direction, 4 corner records (64 B f32 / 32 B
// 16-bit) and 28 B of outputs per query against ~250 flops.
#include "shm_internal.h"

namespace shm {

constexpr int QCHUNK = 8;
constexpr int QBLOCK = 256;
constexpr int QMINBLOCKS = 5;  // <= 51 registers: 40 resident warps per SM

template <int DT, int LAYOUT>
__global__ void __launch_bounds__(QBLOCK, QMINBLOCKS) k_query_fwd(QueryArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * QBLOCK + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * QBLOCK) >> 5;
    const int64_t chunk = 32 * QCHUNK;
    const int G = a.L.n_glyphs;
    uint32_t status = 0;
    const float qnan = __int_as_float(0x7fc00000);

    for (int64_t c0 = warp0 * chunk; c0 < a.Q; c0 += nwarps * chunk) {
        // glyph of the chunk's first query and the end of its segment (one search per chunk)
        int g = 0;
        int64_t seg_end = INT64_MAX;
        if (a.seg) {
            int g0 = 0;
            long long e0 = 0;
            if (lane == 0) {
                g0 = (c0 < __ldg(a.seg)) ? -1 : seg_find(a.seg, G, c0);
                e0 = (g0 >= 0 && g0 < G) ? __ldg(a.seg + g0 + 1) : 0;
            }
            g = __shfl_sync(0xffffffffu, g0, 0);
            seg_end = __shfl_sync(0xffffffffu, e0, 0);
        }
        int64_t q = c0 + lane;
        float n0 = 0.f, n1 = 0.f, n2 = 0.f;
        if (q < a.Q) { n0 = __ldg(a.dirs + 3 * q); n1 = __ldg(a.dirs + 3 * q + 1); n2 = __ldg(a.dirs + 3 * q + 2); }
#pragma unroll 1
        for (int it = 0; it < QCHUNK; ++it, q += 32) {
            if (q >= a.Q) break;
            const float d0 = n0, d1 = n1, d2 = n2;
            // prefetch the next direction of this lane: its latency overlaps the table fetch below
            if (it + 1 < QCHUNK && q + 32 < a.Q) {
                n0 = __ldg(a.dirs + 3 * (q + 32));
                n1 = __ldg(a.dirs + 3 * (q + 32) + 1);
                n2 = __ldg(a.dirs + 3 * (q + 32) + 2);
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
                valid = query_one<DT, LAYOUT>(a.L, Gr, d0, d1, d2, r, c);
                if (!valid) status |= SHM_DEV_NONFINITE;
            }
            if (!valid) {
                r.R = r.Ru = r.Rv = qnan;
                r.grad = Vec3{qnan, qnan, qnan};
                r.f = r.i = r.j = -1;
            }
            if (a.R) a.R[q] = r.R;
            if (a.grad) {
                a.grad[3 * q] = r.grad.x;
                a.grad[3 * q + 1] = r.grad.y;
                a.grad[3 * q + 2] = r.grad.z;
            }
            if (a.normal) {
                const Vec3 n = valid ? surface_normal(d0, d1, d2, r.R, r.grad) : Vec3{qnan, qnan, qnan};
                a.normal[3 * q] = n.x;
                a.normal[3 * q + 1] = n.y;
                a.normal[3 * q + 2] = n.z;
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

template <int DT, int LAYOUT>
static cudaError_t launch_fwd_t(const QueryArgs& a, cudaStream_t s)
{
    // one persistent wave: SMs x resident blocks per SM
    static int resident = 0;
    if (resident == 0) {
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_query_fwd<DT, LAYOUT>, QBLOCK, 0) != cudaSuccess || r < 1)
            r = QMINBLOCKS;
        resident = r;
    }
    const int64_t chunks = (a.Q + 32 * QCHUNK - 1) / (32 * QCHUNK);
    int64_t blocks = (chunks + (QBLOCK / 32) - 1) / (QBLOCK / 32);
    const int64_t cap = (int64_t)sm_count() * resident;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_query_fwd<DT, LAYOUT><<<(unsigned)blocks, QBLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_query_fwd(const QueryArgs& a, cudaStream_t s)
{
    if (a.Q == 0) return cudaSuccess;
    const int dt = a.L.dtype, ly = a.L.layout;
    if (ly == SHM_LAYOUT_TEXEL) {
        if (dt == SHM_F32) return launch_fwd_t<SHM_F32, SHM_LAYOUT_TEXEL>(a, s);
        if (dt == SHM_F16) return launch_fwd_t<SHM_F16, SHM_LAYOUT_TEXEL>(a, s);
        return launch_fwd_t<SHM_BF16, SHM_LAYOUT_TEXEL>(a, s);
    }
    if (dt == SHM_F32) return launch_fwd_t<SHM_F32, SHM_LAYOUT_CELL>(a, s);
    if (dt == SHM_F16) return launch_fwd_t<SHM_F16, SHM_LAYOUT_CELL>(a, s);
    return launch_fwd_t<SHM_BF16, SHM_LAYOUT_CELL>(a, s);
}

}  // namespace shm
