// Reverse pass of the query with atomic accumulation (the per-query math is in shm_bwd.cuh): every
// corner record's float4 of gradients is added with one vector reduction (red.global.add.v4.f32),
// two lanes of a warp adding the two adjacent records of a footprint row in the same instruction,
// so the summation order, hence the last bits of dL/dtable, depends on scheduling.
// Per-glyph segments on small uniform tables take k_query_bwd_staged: the table is staged in shared
// memory as in the forward.  (Accumulating each glyph's gradients in a shared-memory slab with
// shared float atomics instead measured 4.8 ms against 3.3 ms for the global vector atomics on the
// 2^26-query glyph field: sixteen scattered 4-byte shared atomics per query cost more than four
// 16-byte L2 ones.)
#include "shm_bwd.cuh"
#include "shm_stage.cuh"

namespace shm {

// One query's cell and upstream values, kept for the paired reductions after its reverse pass.
struct CaptureEmit {
    int64_t base = 0;  // the glyph's first record in the gradient table
    int P = 0;         // the glyph's padded table width
    int64_t rec = -1;  // record of corner (0,0) in the gradient table; -1: no contribution
    float s = 0.0f, t = 0.0f, g_r = 0.0f, g_rs = 0.0f, g_rt = 0.0f;
    __device__ __forceinline__ void operator()(int64_t r, float s_, float t_, float gr, float grs, float grt)
    {
        rec = base + r;
        s = s_;
        t = t_;
        g_r = gr;
        g_rs = grs;
        g_rt = grt;
    }
};

__device__ __forceinline__ float4 shfl_xor_f4(float4 v, int m)
{
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m),
                       __shfl_xor_sync(0xffffffffu, v.z, m), __shfl_xor_sync(0xffffffffu, v.w, m));
}

// The corner reductions of a warp's queries (every lane calls it), in pairs of lanes: lanes 2k and
// 2k + 1 add the two adjacent records (i, j), (i+1, j) of one query's footprint row in the same
// instruction, 32 contiguous bytes, so each vector-reduction instruction reaches the L2 as about 16
// requests instead of 32 scattered ones (glyph field: reverse pass 2.23 -> 2.01 ms).  Four
// instructions per lane as before; the partner's weights and cell come by shuffles.
__device__ __forceinline__ void paired_reds(float4* dl, const CaptureEmit& e, int lane)
{
    float4 w[4];
    if (e.rec >= 0) {
        corner_weights(e.s, e.t, e.g_r, e.g_rs, e.g_rt, w);
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) w[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool even = (lane & 1) == 0;
    const int64_t prec = ((int64_t)__shfl_xor_sync(0xffffffffu, (int)(e.rec >> 32), 1) << 32) |
                         (uint32_t)__shfl_xor_sync(0xffffffffu, (int)(uint32_t)e.rec, 1);
    const int pP = __shfl_xor_sync(0xffffffffu, e.P, 1);
    // each lane passes the partner the weights the partner writes: even lanes their (i+1) records,
    // odd lanes their (i) records, for rows j and j + 1
    const float4 r0 = shfl_xor_f4(even ? w[1] : w[0], 1);
    const float4 r1 = shfl_xor_f4(even ? w[3] : w[2], 1);
    const int64_t qa = even ? e.rec : prec, qb = even ? prec : e.rec;  // the even and the odd lane's cells
    const int Pa = even ? e.P : pP, Pb = even ? pP : e.P;
    const int da = even ? 0 : 1;
    if (qa >= 0) {
        atomicAdd(dl + qa + da, even ? w[0] : r0);
        atomicAdd(dl + qa + Pa + da, even ? w[2] : r1);
    }
    if (qb >= 0) {
        atomicAdd(dl + qb + da, even ? r0 : w[1]);
        atomicAdd(dl + qb + Pb + da, even ? r1 : w[3]);
    }
}

constexpr int BCHUNK = 4;
constexpr int BBLOCK = 256;

template <int DT, int LAYOUT, bool FIT>
__global__ void __launch_bounds__(BBLOCK, 4) k_query_bwd(BackwardArgs a)
{
    float loss_acc = 0.0f;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * BBLOCK + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * BBLOCK) >> 5;
    const int64_t chunk = 32 * BCHUNK;
    const int G = a.L.n_glyphs;
    uint32_t status = 0;
    const float qnan = __int_as_float(0x7fc00000);

    for (int64_t c0 = warp0 * chunk; c0 < a.Q; c0 += nwarps * chunk) {
        int g = 0;
        if (a.seg) {
            int g0 = 0;
            if (lane == 0) g0 = (c0 < __ldg(a.seg)) ? -1 : seg_find(a.seg, G, c0);
            g = __shfl_sync(0xffffffffu, g0, 0);
        }
#pragma unroll 1
        for (int it = 0; it < BCHUNK; ++it) {
            const int64_t q = c0 + it * 32 + lane;
            if (c0 + it * 32 >= a.Q) break;  // warp-uniform: the paired reductions need every lane
            CaptureEmit sink;
            if (q < a.Q) {
                int gq = 0;
                if (a.glyph) {
                    gq = __ldg(a.glyph + q);
                } else if (a.seg) {
                    if (g < 0 && q >= __ldg(a.seg)) g = 0;
                    while (g >= 0 && g < G && q >= __ldg(a.seg + g + 1)) ++g;
                    gq = g;
                }
                float3 dd = make_float3(qnan, qnan, qnan);
                const float d0 = __ldcs(a.dirs + 3 * q), d1 = __ldcs(a.dirs + 3 * q + 1), d2 = __ldcs(a.dirs + 3 * q + 2);
                Chart c;
                bool ok = (gq >= 0 && gq < G);
                if (!ok) status |= SHM_DEV_BOUNDS;
                if (ok && !chart_of(d0, d1, d2, c)) { ok = false; status |= SHM_DEV_NONFINITE; }
                if (ok) {
                    const GlyphRef Gr = glyph_ref(a.L, gq);
                    sink.base = glyph_ref(a.D, gq).base;
                    sink.P = Gr.N + 2;
                    auto fetch = [&a, &Gr](int f, int i, int j) { return fetch_corners<DT, LAYOUT>(a.L.data, Gr, f, i, j); };
                    if constexpr (FIT) bwd_query<FIT>(a, PreFit(a, q), Gr, c, d0, d1, d2, fetch, sink, dd, loss_acc);
                    else bwd_query<FIT>(a, GlobalUp{a, q}, Gr, c, d0, d1, d2, fetch, sink, dd, loss_acc);
                }
                if (a.ddirs) {
                    __stcs(a.ddirs + 3 * q, dd.x);
                    __stcs(a.ddirs + 3 * q + 1, dd.y);
                    __stcs(a.ddirs + 3 * q + 2, dd.z);
                }
            }
            paired_reds(reinterpret_cast<float4*>(a.dlut), sink, lane);
        }
    }
    if (FIT) {
        for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
        if ((threadIdx.x & 31) == 0 && a.loss) atomicAdd(a.loss, loss_acc);
    }
    report_status(a.dev_status, status);
}

// Per-glyph segments on tables that fit in shared memory: one CTA per glyph stages the table (as
// the forward does) and answers the footprint reads from it; the gradient atomics of a glyph then
// all come from one SM within a short window, so its dL/dtable slab stays in L2 while it is hit.
constexpr int SBB = 512;

template <int DT, bool FIT>
__global__ void __launch_bounds__(SBB, 2) k_query_bwd_staged(BackwardArgs a, uint32_t table_bytes)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(smem);
    const unsigned char* table = smem + stage::TABLE_OFFSET;
    const int tid = threadIdx.x;
    const int G = a.L.n_glyphs, N = a.L.N_uniform, P = N + 2;
    uint32_t status = 0;
    float loss_acc = 0.0f;
    const float qnan = __int_as_float(0x7fc00000);
    {
        const int64_t lo = min(max(__ldg(a.seg), (int64_t)0), a.Q);
        const int64_t hi = min(max(__ldg(a.seg + G), lo), a.Q);
        const int64_t stride = (int64_t)gridDim.x * SBB;
        for (int part = 0; part < 2; ++part) {
            const int64_t b = part ? hi : 0, e = part ? a.Q : lo;
            for (int64_t q = b + (int64_t)blockIdx.x * SBB + tid; q < e; q += stride) {
                status |= SHM_DEV_BOUNDS;
                if (a.ddirs) { a.ddirs[3 * q] = qnan; a.ddirs[3 * q + 1] = qnan; a.ddirs[3 * q + 2] = qnan; }
            }
        }
    }
    if (tid == 0) {
        stage::init(bar);
        s_abort = 0;
    }
    __syncthreads();
    auto fetch = [table, P](int f, int i, int j) { return stage::corners<DT>(table, P, f, i, j); };
    uint32_t phase = 0;
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t s0 = min(max(__ldg(a.seg + g), (int64_t)0), a.Q);
        const int64_t s1 = min(max(__ldg(a.seg + g + 1), s0), a.Q);
        if (s1 <= s0) continue;  // block-uniform
        if (tid == 0)
            stage::issue(bar, bar + stage::TABLE_OFFSET,
                         reinterpret_cast<const unsigned char*>(a.L.data) + (size_t)g * table_bytes, table_bytes);
        if (!stage::bar_wait(bar, phase, stage::WAIT_NS)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            status |= SHM_DEV_TIMEOUT;
            if (tid == 0) stage::bar_wait(bar, phase, stage::DRAIN_NS);
            break;
        }
        phase ^= 1;
        const GlyphRef Gr = glyph_ref(a.L, g);
        const int64_t dbase = glyph_ref(a.D, g).base;
        // warp-uniform trip count: the paired reductions need every lane of the warp
        for (int64_t qw = s0 + (tid & ~31); qw < s1; qw += SBB) {
            const int64_t q = qw + (tid & 31);
            CaptureEmit sink;
            sink.base = dbase;
            sink.P = P;
            if (q < s1) {
                float3 dd = make_float3(qnan, qnan, qnan);
                const float d0 = __ldcs(a.dirs + 3 * q), d1 = __ldcs(a.dirs + 3 * q + 1), d2 = __ldcs(a.dirs + 3 * q + 2);
                Chart c;
                if constexpr (FIT) {
                    const PreFit up(a, q);
                    if (chart_of(d0, d1, d2, c)) bwd_query<FIT>(a, up, Gr, c, d0, d1, d2, fetch, sink, dd, loss_acc);
                    else status |= SHM_DEV_NONFINITE;
                } else {
                    const PreUp up(a, q);  // issued before the chart, used after the forward recompute
                    if (chart_of(d0, d1, d2, c)) bwd_query<FIT>(a, up, Gr, c, d0, d1, d2, fetch, sink, dd, loss_acc);
                    else status |= SHM_DEV_NONFINITE;
                }
                if (a.ddirs) { __stcs(a.ddirs + 3 * q, dd.x); __stcs(a.ddirs + 3 * q + 1, dd.y); __stcs(a.ddirs + 3 * q + 2, dd.z); }
            }
            paired_reds(reinterpret_cast<float4*>(a.dlut), sink, tid & 31);
        }
        __syncthreads();  // every read of this table is done before the next copy lands
    }
    if (FIT) {
        for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
        if ((tid & 31) == 0 && a.loss) atomicAdd(a.loss, loss_acc);
    }
    report_status(a.dev_status, status);
}

template <int DT, bool FIT>
static cudaError_t launch_bwd_staged_ft(const BackwardArgs& a, uint32_t table_bytes, cudaStream_t s)
{
    const int smem = stage::TABLE_OFFSET + (int)table_bytes;
    cudaError_t e = ensure_dynamic_smem((const void*)k_query_bwd_staged<DT, FIT>, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (int64_t)sm_count() * 2;
    if (blocks > a.L.n_glyphs) blocks = a.L.n_glyphs;
    k_query_bwd_staged<DT, FIT><<<(unsigned)blocks, SBB, smem, s>>>(a, table_bytes);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t launch_bwd_staged(const BackwardArgs& a, uint32_t table_bytes, cudaStream_t s)
{
    return a.fit ? launch_bwd_staged_ft<DT, true>(a, table_bytes, s) : launch_bwd_staged_ft<DT, false>(a, table_bytes, s);
}

template <int DT, int LAYOUT>
static cudaError_t launch_bwd_t(const BackwardArgs& a, cudaStream_t s)
{
    const int64_t chunks = (a.Q + 32 * BCHUNK - 1) / (32 * BCHUNK);
    int64_t blocks = (chunks + (BBLOCK / 32) - 1) / (BBLOCK / 32);
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (a.fit) k_query_bwd<DT, LAYOUT, true><<<(unsigned)blocks, BBLOCK, 0, s>>>(a);
    else k_query_bwd<DT, LAYOUT, false><<<(unsigned)blocks, BBLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_query_bwd(const BackwardArgs& a, cudaStream_t s)
{
    if (a.Q == 0) return cudaSuccess;
    const int dt = a.L.dtype, ly = a.L.layout;
    // per-glyph segments on small uniform tables: stage each glyph's table in shared memory
    if (a.seg && !a.glyph && a.L.N_uniform > 0 && a.D.N_uniform == a.L.N_uniform && ly == SHM_LAYOUT_TEXEL) {
        const int64_t P = (int64_t)a.L.N_uniform + 2;
        const int64_t bytes = 6 * P * P * (dt == SHM_F32 ? 16 : 8);
        if (bytes <= STAGED_TABLE_MAX_BYTES) {
            if (dt == SHM_F32) return launch_bwd_staged<SHM_F32>(a, (uint32_t)bytes, s);
            if (dt == SHM_F16) return launch_bwd_staged<SHM_F16>(a, (uint32_t)bytes, s);
            return launch_bwd_staged<SHM_BF16>(a, (uint32_t)bytes, s);
        }
    }
    if (ly == SHM_LAYOUT_TEXEL) {
        if (dt == SHM_F32) return launch_bwd_t<SHM_F32, SHM_LAYOUT_TEXEL>(a, s);
        if (dt == SHM_F16) return launch_bwd_t<SHM_F16, SHM_LAYOUT_TEXEL>(a, s);
        return launch_bwd_t<SHM_BF16, SHM_LAYOUT_TEXEL>(a, s);
    }
    if (dt == SHM_F32) return launch_bwd_t<SHM_F32, SHM_LAYOUT_CELL>(a, s);
    if (dt == SHM_F16) return launch_bwd_t<SHM_F16, SHM_LAYOUT_CELL>(a, s);
    return launch_bwd_t<SHM_BF16, SHM_LAYOUT_CELL>(a, s);
}

}  // namespace shm

namespace shm {

// Adam (Kingma & Ba, 2015) with bias correction; optionally zeroes the gradient for the next step.
__device__ __forceinline__ void adam_one(float& p, float& g, float& m, float& v, float lr, float b1, float b2,
                                         float eps, float c1, float c2, int zero_grad)
{
    const float gi = g;
    const float mi = b1 * m + (1.0f - b1) * gi;
    const float vi = b2 * v + (1.0f - b2) * gi * gi;
    m = mi;
    v = vi;
    p -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    if (zero_grad) g = 0.0f;
}

// VEC4: all four arrays 16-byte aligned; 128-bit loads and stores over n/4 quadruples, then the tail.
template <bool VEC4>
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                                              float c1, float c2, int zero_grad)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (VEC4) {
        const int64_t n4 = n / 4;
        float4 *p4 = reinterpret_cast<float4*>(p), *g4 = reinterpret_cast<float4*>(g);
        float4 *m4 = reinterpret_cast<float4*>(m), *v4 = reinterpret_cast<float4*>(v);
        for (int64_t i = tid; i < n4; i += stride) {
            float4 P = p4[i], Gq = g4[i], M = m4[i], V = v4[i];
            adam_one(P.x, Gq.x, M.x, V.x, lr, b1, b2, eps, c1, c2, zero_grad);
            adam_one(P.y, Gq.y, M.y, V.y, lr, b1, b2, eps, c1, c2, zero_grad);
            adam_one(P.z, Gq.z, M.z, V.z, lr, b1, b2, eps, c1, c2, zero_grad);
            adam_one(P.w, Gq.w, M.w, V.w, lr, b1, b2, eps, c1, c2, zero_grad);
            p4[i] = P;
            m4[i] = M;
            v4[i] = V;
            if (zero_grad) g4[i] = Gq;
        }
        done = n4 * 4;
    }
    for (int64_t i = done + tid; i < n; i += stride) adam_one(p[i], g[i], m[i], v[i], lr, b1, b2, eps, c1, c2, zero_grad);
}

cudaError_t launch_adam(float* param, float* grad, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                        float eps, int step, int zero_grad, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const float c1 = 1.0f - (float)pow((double)beta1, (double)step);
    const float c2 = 1.0f - (float)pow((double)beta2, (double)step);
    const bool vec = (((uintptr_t)param | (uintptr_t)grad | (uintptr_t)m | (uintptr_t)v) & 15u) == 0;
    int64_t blocks = (n / (vec ? 4 : 1) + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (vec) k_adam<true><<<(unsigned)blocks, 256, 0, s>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2, zero_grad);
    else k_adam<false><<<(unsigned)blocks, 256, 0, s>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2, zero_grad);
    return cudaGetLastError();
}

}  // namespace shm
