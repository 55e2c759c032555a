// Reverse mode of the query (the paper has no adjoint; this makes tables fittable under autograd).
//
// Per query the forward is recomputed and the upstream gradients (gR, ggrad, gnormal) are pulled
// back through, in reverse order:
//   normal  n = m/|m|, m = R w - grad:       gm = (gn - n (n.gn))/|m|;  gR += gm.w;  gw = R gm;
//                                            ggrad -= gm
//   grad    = (rho/2)[R_u b + R_v c - (x R_u + y R_v) a]  (the §3.4 Cramer solution in closed form)
//                                            -> gR_u, gR_v and the chart-coordinate terms gx, gy
//   Hermite r, r_s, r_t are linear in the 16 stored scalars (§3.3): each corner record receives
//           float4 weights, added with one vector atomic per corner (red.global.add.v4.f32);
//           s, t move with the direction: gs, gt from the second derivatives of the patch
//   chart   x = d_k1/|d_k|, y = d_k2/|d_k|, s = (x+1)N/2 + 1/2 - i:  gd from gx + gs N/2, gy + gt N/2
//   w = d/|d|                               gd += (gw - w (w.gw))/|d|
// Face and cell indices are piecewise constant, so they carry no derivative.
// Per-glyph segments on small uniform tables take k_query_bwd_staged: the table is staged in shared
// memory as in the forward.  (Accumulating each glyph's gradients in a shared-memory slab with
// shared float atomics instead measured 4.8 ms against 3.3 ms for the global vector atomics on the
// 2^26-query glyph field: sixteen scattered 4-byte shared atomics per query cost more than four
// 16-byte L2 ones.)
#include "shm_stage.cuh"

namespace shm {

constexpr int BCHUNK = 4;
constexpr int BBLOCK = 256;

struct Herm2 {
    float H1, h0d, h1d, dH1, dh0d, dh1d, ddH1, ddh0d, ddh1d;
};

__device__ __forceinline__ Herm2 herm2(float s)
{
    Herm2 h;
    const float s2 = s * s, om = 1.0f - s;
    h.H1 = s2 * (3.0f - 2.0f * s);
    h.h0d = s * om * om;
    h.h1d = s2 * (s - 1.0f);
    h.dH1 = 6.0f * s * om;
    h.dh0d = om * (1.0f - 3.0f * s);
    h.dh1d = s * (3.0f * s - 2.0f);
    h.ddH1 = 6.0f - 12.0f * s;
    h.ddh0d = 6.0f * s - 4.0f;
    h.ddh1d = 6.0f * s - 2.0f;
    return h;
}

// One query's reverse pass on glyph table Gr: the 2x2 footprint comes from `fetch(f, i, j)`,
// corner-record gradients go to `sink(record, float4)` (record index within the glyph's texel
// table), the direction gradient to dd.
template <bool FIT, class Fetch, class Sink>
__device__ __forceinline__ void bwd_query(const BackwardArgs& a, int64_t q, const GlyphRef& Gr, const Chart& c,
                                          float d0, float d1, float d2, const Fetch& fetch, Sink& sink, float3& dd,
                                          float& loss_acc)
{
    const int N = Gr.N;
    int i, j;
    float s, t;
    cell_of(pick3(c.k1, d0, d1, d2), c.m, c.im, N, i, s);
    cell_of(pick3(c.k2, d0, d1, d2), c.m, c.im, N, j, t);
    const Corners cr = fetch(c.f, i, j);
    const Herm2 A = herm2(s), B = herm2(t);
    // --- forward (difference form) with second derivatives
    const float d0r = cr.c10.x - cr.c00.x, d1r = cr.c11.x - cr.c01.x;
    const float e0 = cr.c10.z - cr.c00.z, e1 = cr.c11.z - cr.c01.z;
    const float p0 = cr.c00.x + A.H1 * d0r + A.h0d * cr.c00.y + A.h1d * cr.c10.y;
    const float p1 = cr.c01.x + A.H1 * d1r + A.h0d * cr.c01.y + A.h1d * cr.c11.y;
    const float q0 = cr.c00.z + A.H1 * e0 + A.h0d * cr.c00.w + A.h1d * cr.c10.w;
    const float q1 = cr.c01.z + A.H1 * e1 + A.h0d * cr.c01.w + A.h1d * cr.c11.w;
    const float ps0 = A.dH1 * d0r + A.dh0d * cr.c00.y + A.dh1d * cr.c10.y;
    const float ps1 = A.dH1 * d1r + A.dh0d * cr.c01.y + A.dh1d * cr.c11.y;
    const float qs0 = A.dH1 * e0 + A.dh0d * cr.c00.w + A.dh1d * cr.c10.w;
    const float qs1 = A.dH1 * e1 + A.dh0d * cr.c01.w + A.dh1d * cr.c11.w;
    const float pss0 = A.ddH1 * d0r + A.ddh0d * cr.c00.y + A.ddh1d * cr.c10.y;
    const float pss1 = A.ddH1 * d1r + A.ddh0d * cr.c01.y + A.ddh1d * cr.c11.y;
    const float qss0 = A.ddH1 * e0 + A.ddh0d * cr.c00.w + A.ddh1d * cr.c10.w;
    const float qss1 = A.ddH1 * e1 + A.ddh0d * cr.c01.w + A.ddh1d * cr.c11.w;
    const float dp = p1 - p0;
    const float r = p0 + B.H1 * dp + B.h0d * q0 + B.h1d * q1;
    const float rs = ps0 + B.H1 * (ps1 - ps0) + B.h0d * qs0 + B.h1d * qs1;
    const float rt = B.dH1 * dp + B.dh0d * q0 + B.dh1d * q1;
    const float rss = pss0 + B.H1 * (pss1 - pss0) + B.h0d * qss0 + B.h1d * qss1;
    const float rst = B.dH1 * (ps1 - ps0) + B.dh0d * qs0 + B.dh1d * qs1;
    const float rtt = B.ddH1 * dp + B.ddh0d * q0 + B.ddh1d * q1;
    const float Nf = (float)N;
    const float R = Gr.r0 + r, Ru = Nf * rs, Rv = Nf * rt;
    const float x = c.x, y = c.y;
    const float rho = sqrtf(fmaf(x, x, fmaf(y, y, 1.0f)));
    // tangent-frame components (a, b, c) = (sigma e_k, e_k1, e_k2)
    const float Va = -(x * Ru + y * Rv), Vb = Ru, Vc = Rv;
    const float il = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    const float wk = pick3(c.k, d0, d1, d2) * il * c.sigma;  // w . a
    const float w1 = pick3(c.k1, d0, d1, d2) * il;            // w . b
    const float w2 = pick3(c.k2, d0, d1, d2) * il;            // w . c
    const float Ga = 0.5f * rho * Va, Gb = 0.5f * rho * Vb, Gc = 0.5f * rho * Vc;
    const float ma = R * wk - Ga, mb = R * w1 - Gb, mc = R * w2 - Gc;
    const float iml = rsqrtf(ma * ma + mb * mb + mc * mc);
    const float na = ma * iml, nb = mb * iml, nc = mc * iml;
    // upstream in the (a, b, c) frame
    float gRu_in = a.gR ? __ldg(a.gR + q) : 0.0f;
    float gGa = 0.f, gGb = 0.f, gGc = 0.f, gna = 0.f, gnb = 0.f, gnc = 0.f;
    if (FIT) {
        // L_q = w_v (R - R_t)^2 + w_n |n - n_t|^2: upstream dL/dR, dL/dn in the frame
        const float eR = R - __ldg(a.R_target + q);
        const float t0 = __ldg(a.n_target + 3 * q), t1 = __ldg(a.n_target + 3 * q + 1),
                    t2 = __ldg(a.n_target + 3 * q + 2);
        const float ea = na - pick3(c.k, t0, t1, t2) * c.sigma, eb = nb - pick3(c.k1, t0, t1, t2),
                    ec = nc - pick3(c.k2, t0, t1, t2);
        loss_acc += a.w_value * eR * eR + a.w_normal * (ea * ea + eb * eb + ec * ec);
        gRu_in = 2.0f * a.w_value * eR;
        gna = 2.0f * a.w_normal * ea;
        gnb = 2.0f * a.w_normal * eb;
        gnc = 2.0f * a.w_normal * ec;
    }
    if (!FIT && a.ggrad) {
        const float gx0 = __ldg(a.ggrad + 3 * q), gx1 = __ldg(a.ggrad + 3 * q + 1), gx2 = __ldg(a.ggrad + 3 * q + 2);
        gGa = pick3(c.k, gx0, gx1, gx2) * c.sigma;
        gGb = pick3(c.k1, gx0, gx1, gx2);
        gGc = pick3(c.k2, gx0, gx1, gx2);
    }
    if (!FIT && a.gnormal) {
        const float gx0 = __ldg(a.gnormal + 3 * q), gx1 = __ldg(a.gnormal + 3 * q + 1), gx2 = __ldg(a.gnormal + 3 * q + 2);
        gna = pick3(c.k, gx0, gx1, gx2) * c.sigma;
        gnb = pick3(c.k1, gx0, gx1, gx2);
        gnc = pick3(c.k2, gx0, gx1, gx2);
    }
    // --- reverse
    const float ndg = na * gna + nb * gnb + nc * gnc;
    const float gma = (gna - na * ndg) * iml, gmb = (gnb - nb * ndg) * iml, gmc = (gnc - nc * ndg) * iml;
    const float gRt = gRu_in + gma * wk + gmb * w1 + gmc * w2;
    const float gwa = R * gma, gwb = R * gmb, gwc = R * gmc;
    const float tGa = gGa - gma, tGb = gGb - gmb, tGc = gGc - gmc;
    const float gVa = 0.5f * rho * tGa, gVb = 0.5f * rho * tGb, gVc = 0.5f * rho * tGc;
    const float grho = 0.5f * (Va * tGa + Vb * tGb + Vc * tGc);
    const float gRu = gVb - x * gVa;
    const float gRv = gVc - y * gVa;
    const float gx = -Ru * gVa + grho * x / rho;
    const float gy = -Rv * gVa + grho * y / rho;
    const float g_r = gRt, g_rs = Nf * gRu, g_rt = Nf * gRv;
    // table: corner weights (value / d/ds / d/dt combined), one float4 per corner
    {
        const float H0s = 1.0f - A.H1, dH0s = -A.dH1, H0t = 1.0f - B.H1, dH0t = -B.dH1;
        const float al0 = g_r * H0s + g_rs * dH0s, al1 = g_r * A.H1 + g_rs * A.dH1;
        const float ad0 = g_r * A.h0d + g_rs * A.dh0d, ad1 = g_r * A.h1d + g_rs * A.dh1d;
        const float be0 = g_rt * H0s, be1 = g_rt * A.H1, bd0 = g_rt * A.h0d, bd1 = g_rt * A.h1d;
        const float Ht[2] = {H0t, B.H1}, dHt[2] = {dH0t, B.dH1}, hdt[2] = {B.h0d, B.h1d}, dhdt[2] = {B.dh0d, B.dh1d};
        const float al[2] = {al0, al1}, ad[2] = {ad0, ad1}, be[2] = {be0, be1}, bd[2] = {bd0, bd1};
        const int P = N + 2;
        const int rec = (c.f * P + j) * P + i;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int aa = 0; aa < 2; ++aa) {
                float4 wv;
                wv.x = al[aa] * Ht[bb] + be[aa] * dHt[bb];
                wv.y = ad[aa] * Ht[bb] + bd[aa] * dHt[bb];
                wv.z = al[aa] * hdt[bb] + be[aa] * dhdt[bb];
                wv.w = ad[aa] * hdt[bb] + bd[aa] * dhdt[bb];
                sink(rec + bb * P + aa, wv);
            }
    }
    if (a.ddirs) {
        const float gs = g_r * rs + g_rs * rss + g_rt * rst;
        const float gt = g_r * rt + g_rs * rst + g_rt * rtt;
        const float gxx = gx + gs * 0.5f * Nf, gyy = gy + gt * 0.5f * Nf;
        // chart coordinates -> d (frame components; a-component carries sigma)
        float dA = -(x * gxx + y * gyy) / c.m;  // along a = sigma e_k
        float dB = gxx / c.m, dC = gyy / c.m;
        // w = d/|d|
        const float wdg = wk * gwa + w1 * gwb + w2 * gwc;
        dA += (gwa - wk * wdg) * il;
        dB += (gwb - w1 * wdg) * il;
        dC += (gwc - w2 * wdg) * il;
        // back to Cartesian (a = sigma e_k): component c.k gets dA sigma, c.k1 dB, c.k2 dC
        const float sA = dA * c.sigma;
        dd = make_float3(c.k == 0 ? sA : (c.k1 == 0 ? dB : dC), c.k == 1 ? sA : (c.k1 == 1 ? dB : dC),
                         c.k == 2 ? sA : (c.k1 == 2 ? dB : dC));
    }
}

template <int DT, int LAYOUT, bool FIT>
__global__ void __launch_bounds__(BBLOCK, 3) k_query_bwd(BackwardArgs a)
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
            if (q >= a.Q) break;
            int gq = 0;
            if (a.glyph) {
                gq = __ldg(a.glyph + q);
            } else if (a.seg) {
                if (g < 0 && q >= __ldg(a.seg)) g = 0;
                while (g >= 0 && g < G && q >= __ldg(a.seg + g + 1)) ++g;
                gq = g;
            }
            float3 dd = make_float3(qnan, qnan, qnan);
            const float d0 = __ldg(a.dirs + 3 * q), d1 = __ldg(a.dirs + 3 * q + 1), d2 = __ldg(a.dirs + 3 * q + 2);
            Chart c;
            bool ok = (gq >= 0 && gq < G);
            if (!ok) status |= SHM_DEV_BOUNDS;
            if (ok && !chart_of(d0, d1, d2, c)) { ok = false; status |= SHM_DEV_NONFINITE; }
            if (ok) {
                const GlyphRef Gr = glyph_ref(a.L, gq);
                const GlyphRef Gd = glyph_ref(a.D, gq);
                float4* dbase = reinterpret_cast<float4*>(a.dlut) + Gd.base;
                auto sink = [dbase](int rec, float4 wv) { atomicAdd(dbase + rec, wv); };
                auto fetch = [&a, &Gr](int f, int i, int j) { return fetch_corners<DT, LAYOUT>(a.L.data, Gr, f, i, j); };
                bwd_query<FIT>(a, q, Gr, c, d0, d1, d2, fetch, sink, dd, loss_acc);
            }
            if (a.ddirs) {
                a.ddirs[3 * q] = dd.x;
                a.ddirs[3 * q + 1] = dd.y;
                a.ddirs[3 * q + 2] = dd.z;
            }
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
        float4* dbase = reinterpret_cast<float4*>(a.dlut) + glyph_ref(a.D, g).base;
        auto sink = [dbase](int rec, float4 wv) { atomicAdd(dbase + rec, wv); };
        for (int64_t q = s0 + tid; q < s1; q += SBB) {
            float3 dd = make_float3(qnan, qnan, qnan);
            const float d0 = __ldg(a.dirs + 3 * q), d1 = __ldg(a.dirs + 3 * q + 1), d2 = __ldg(a.dirs + 3 * q + 2);
            Chart c;
            if (chart_of(d0, d1, d2, c)) bwd_query<FIT>(a, q, Gr, c, d0, d1, d2, fetch, sink, dd, loss_acc);
            else status |= SHM_DEV_NONFINITE;
            if (a.ddirs) { a.ddirs[3 * q] = dd.x; a.ddirs[3 * q + 1] = dd.y; a.ddirs[3 * q + 2] = dd.z; }
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
    static int configured = -1;
    if (configured != smem) {
        cudaError_t e = cudaFuncSetAttribute(k_query_bwd_staged<DT, FIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
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
