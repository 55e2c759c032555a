// Deterministic reverse pass of the query (SHM_BWD_DETERMINISTIC; not in the paper): dL/dtable comes
// out bit-identical from run to run and independent of the launch shape, by a segmented reduction in
// a fixed order instead of atomic accumulation.
//
// Needs per-glyph query segments: one CTA owns a glyph (and so its dL/dtable slab) and walks the
// glyph's queries in chunks of DBLOCK.  Per chunk:
//   1. every thread runs the reverse math of its query (shm_bwd.cuh), writes d/ddirs, and keeps the
//      cell (record index of corner (0,0)) as a sort key and (s, t, g_r, g_rs, g_rt) in shared memory;
//   2. a bitonic sort of (cell, query) keys groups the chunk's queries by cell, in query order
//      (keys in registers; partners within a warp by shuffles, across warps through shared memory);
//   3. the first thread of each cell's run sums the corner weights of the run's queries in that order;
//   4. four passes, one per corner (aa, bb), add those sums to the slab with one vector reduction
//      (red.global.add.v4.f32) per cell: within one pass distinct cells reach distinct records, and
//      the passes are separated by CTA barriers, so every record receives its contributions one at
//      a time in a fixed order.
// Chunks run in order inside the CTA, glyphs are disjoint, so the whole result is fixed.  Chunks of
// 256 queries and four CTAs per SM (footprints read through L1/L2): with whole tables staged in
// shared memory only two 1,024-thread CTAs fit per SM, which measured 5.7 ms against 4.7 ms on the
// 2^26-query glyph field.  Sort keys are 32-bit (one shuffle per exchange) when every record index
// of a uniform pool fits in 24 bits (N <= 1670), else 64-bit.
#include "shm_bwd.cuh"

namespace shm {

namespace {

constexpr int DBLOCK = 256;
constexpr int DBITS = 8;   // log2(DBLOCK): query slot in the low bits of the sort key
constexpr int DMINB = 4;   // CTAs per SM
// Shared memory: two key buffers [DBLOCK] of KT, then the payload [5][DBLOCK] f32.
template <class KT>
constexpr uint32_t det_smem() { return 2 * DBLOCK * sizeof(KT) + 5 * DBLOCK * 4; }

template <class KT>
struct DetEmit {
    KT key;
    float* pay;  // [5][DBLOCK]: s, t, g_r, g_rs, g_rt
    int slot;
    __device__ __forceinline__ void operator()(int64_t rec, float s, float t, float g_r, float g_rs, float g_rt)
    {
        key = ((KT)rec << DBITS) | (KT)slot;
        pay[slot] = s;
        pay[DBLOCK + slot] = t;
        pay[2 * DBLOCK + slot] = g_r;
        pay[3 * DBLOCK + slot] = g_rs;
        pay[4 * DBLOCK + slot] = g_rt;
    }
};

__device__ __forceinline__ uint64_t shfl_xor_key(uint64_t v, int m)
{
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint32_t shfl_xor_key(uint32_t v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// Ascending bitonic sort of the DBLOCK keys held one per thread (thread tid holds position tid).
// Compare-exchange partners tid ^ j: by shuffles for j < 32, through shared memory otherwise, with
// two buffers used in turn so that one barrier per shared stage suffices.  Returns the key at
// position tid; the sorted keys are also left in `out` (one of the two buffers) after a barrier.
template <class KT>
__device__ __forceinline__ KT bitonic_sort(KT x, KT* buf0, KT* buf1, KT*& out, int tid)
{
    int flip = 0;
    for (int k = 2; k <= DBLOCK; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            KT y;
            if (j >= 32) {
                KT* b = flip ? buf1 : buf0;
                flip ^= 1;
                b[tid] = x;
                __syncthreads();
                y = b[tid ^ j];
            } else {
                y = shfl_xor_key(x, j);
            }
            const bool up = (tid & k) == 0, lower = (tid & j) == 0;
            x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
        }
    // the buffer not written by the last shared stage is free: every thread has passed that stage's barrier
    out = flip ? buf1 : buf0;
    out[tid] = x;
    __syncthreads();
    return x;
}

template <int DT, int LAYOUT, class KT>
__global__ void __launch_bounds__(DBLOCK, DMINB) k_query_bwd_det(BackwardArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr KT NO_KEY = ~(KT)0;
    unsigned char* fixed = smem;
    KT* kbuf0 = reinterpret_cast<KT*>(fixed);
    KT* kbuf1 = kbuf0 + DBLOCK;
    float* pay = reinterpret_cast<float*>(fixed + 2 * DBLOCK * sizeof(KT));
    const int tid = threadIdx.x;
    const int G = a.L.n_glyphs;
    uint32_t status = 0;
    float loss_unused = 0.0f;
    const float qnan = __int_as_float(0x7fc00000);
    {
        // queries outside every segment: NaN d/ddirs and SHM_DEV_BOUNDS
        const int64_t lo = min(max(__ldg(a.seg), (int64_t)0), a.Q);
        const int64_t hi = min(max(__ldg(a.seg + G), lo), a.Q);
        const int64_t stride = (int64_t)gridDim.x * DBLOCK;
        for (int part = 0; part < 2; ++part) {
            const int64_t b = part ? hi : 0, e = part ? a.Q : lo;
            for (int64_t q = b + (int64_t)blockIdx.x * DBLOCK + tid; q < e; q += stride) {
                status |= SHM_DEV_BOUNDS;
                if (a.ddirs) { a.ddirs[3 * q] = qnan; a.ddirs[3 * q + 1] = qnan; a.ddirs[3 * q + 2] = qnan; }
            }
        }
    }
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t s0 = min(max(__ldg(a.seg + g), (int64_t)0), a.Q);
        const int64_t s1 = min(max(__ldg(a.seg + g + 1), s0), a.Q);
        if (s1 <= s0) continue;  // block-uniform
        const GlyphRef Gr = glyph_ref(a.L, g);
        const int P = Gr.N + 2;
        float4* dbase = reinterpret_cast<float4*>(a.dlut) + glyph_ref(a.D, g).base;
        // the next chunk's direction is loaded while this chunk computes, sorts and adds
        float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
        if (s0 + tid < s1) {
            n0 = __ldcs(a.dirs + 3 * (s0 + tid));
            n1 = __ldcs(a.dirs + 3 * (s0 + tid) + 1);
            n2 = __ldcs(a.dirs + 3 * (s0 + tid) + 2);
        }
        for (int64_t c0 = s0; c0 < s1; c0 += DBLOCK) {
            // 1. reverse math per query; key and payload into shared memory
            const int64_t q = c0 + tid;
            const float d0 = n0, d1 = n1, d2 = n2;
            if (q + DBLOCK < s1) {
                n0 = __ldcs(a.dirs + 3 * (q + DBLOCK));
                n1 = __ldcs(a.dirs + 3 * (q + DBLOCK) + 1);
                n2 = __ldcs(a.dirs + 3 * (q + DBLOCK) + 2);
            }
            DetEmit<KT> emit{NO_KEY, pay, tid};
            if (q < s1) {
                const PreUp up(a, q);  // issued before the chart, used after the forward recompute
                float3 dd = make_float3(qnan, qnan, qnan);
                Chart c;
                if (chart_of(d0, d1, d2, c)) {
                    auto fetch = [&a, &Gr](int f, int i, int j) { return fetch_corners<DT, LAYOUT>(a.L.data, Gr, f, i, j); };
                    bwd_query<false>(a, up, Gr, c, d0, d1, d2, fetch, emit, dd, loss_unused);
                } else {
                    status |= SHM_DEV_NONFINITE;
                }
                if (a.ddirs) { __stcs(a.ddirs + 3 * q, dd.x); __stcs(a.ddirs + 3 * q + 1, dd.y); __stcs(a.ddirs + 3 * q + 2, dd.z); }
            }
            // 2. group by cell, queries in order within a cell (the payload writes are ordered before
            //    the reads of step 3 by the sort's barriers)
            KT* key;
            const KT k = bitonic_sort<KT>(emit.key, kbuf0, kbuf1, key, tid);
            // 3. the first slot of each cell's run sums the run in query order
            const KT cell = k >> DBITS;
            const bool head = (k != NO_KEY) && (tid == 0 || (key[tid - 1] >> DBITS) != cell);
            float4 acc[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[m] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (head) {
                for (int r = tid; r < DBLOCK; ++r) {
                    const KT kr = key[r];
                    if (kr == NO_KEY || (kr >> DBITS) != cell) break;
                    const int src = (int)(kr & (DBLOCK - 1));
                    float4 w[4];
                    corner_weights(pay[src], pay[DBLOCK + src], pay[2 * DBLOCK + src], pay[3 * DBLOCK + src],
                                   pay[4 * DBLOCK + src], w);
#pragma unroll
                    for (int m = 0; m < 4; ++m) acc[m] = padd4(acc[m], w[m]);
                }
            }
            // 4. one pass per corner: distinct cells touch distinct records within a pass, so each
            //    record receives at most one vector reduction per pass, and the CTA barrier between
            //    passes orders a record's reductions from one pass before those of the next (the
            //    same adds, in the same order, as a read-add-write, without waiting for the read)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (head) atomicAdd(dbase + (int64_t)cell + (m >> 1) * P + (m & 1), acc[m]);
                __syncthreads();
            }
        }
    }
    report_status(a.dev_status, status);
}

template <int DT, int LAYOUT, class KT>
cudaError_t launch_det_k(const BackwardArgs& a, cudaStream_t s)
{
    const int smem = (int)det_smem<KT>();
    cudaError_t e = ensure_dynamic_smem((const void*)k_query_bwd_det<DT, LAYOUT, KT>, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (int64_t)sm_count() * DMINB;
    if (blocks > a.L.n_glyphs) blocks = a.L.n_glyphs;
    if (blocks < 1) blocks = 1;
    k_query_bwd_det<DT, LAYOUT, KT><<<(unsigned)blocks, DBLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int DT, int LAYOUT>
cudaError_t launch_det_t(const BackwardArgs& a, cudaStream_t s)
{
    // the gradient table is float32 texel layout: record indices below 6 (N + 2)^2 per glyph
    const bool narrow = a.D.N_uniform > 0 && 6LL * (a.D.N_uniform + 2) * (a.D.N_uniform + 2) < (1LL << (32 - DBITS));
    return narrow ? launch_det_k<DT, LAYOUT, uint32_t>(a, s) : launch_det_k<DT, LAYOUT, uint64_t>(a, s);
}

}  // namespace

cudaError_t launch_query_bwd_det(const BackwardArgs& a, cudaStream_t s)
{
    if (a.Q == 0) return cudaSuccess;
    const int dt = a.L.dtype;
    if (a.L.layout == SHM_LAYOUT_TEXEL) {
        if (dt == SHM_F32) return launch_det_t<SHM_F32, SHM_LAYOUT_TEXEL>(a, s);
        if (dt == SHM_F16) return launch_det_t<SHM_F16, SHM_LAYOUT_TEXEL>(a, s);
        return launch_det_t<SHM_BF16, SHM_LAYOUT_TEXEL>(a, s);
    }
    if (dt == SHM_F32) return launch_det_t<SHM_F32, SHM_LAYOUT_CELL>(a, s);
    if (dt == SHM_F16) return launch_det_t<SHM_F16, SHM_LAYOUT_CELL>(a, s);
    return launch_det_t<SHM_BF16, SHM_LAYOUT_CELL>(a, s);
}

}  // namespace shm
