// Device building blocks of the Spherical Hermite Map hot path (arXiv 2602.20063), sm_103a.
//
//   chart   §3.2: direction -> axis k, face f, chart coordinates, cell (i, j), local (s, t)
//   fetch   §3.3: the 2x2 texel footprint of one cell, any record dtype / layout
//   hermite §3.3: value and chart derivatives by tensor-product cubic Hermite interpolation
//   grad    §3.4: S^2 gradient from chart derivatives, normal
//
// Everything is float32.  Two numerical choices differ from a literal transcription:
//   * the cell coordinate x = uN + 1/2 is formed from a double-float quotient
//     q = d_{k+1}/|d_k| (hi + lo) so that s, t carry ~1e-8 absolute error even at N = 2048,
//     where a plain float x = uN + 1/2 would lose ~1e-4 of a cell;
//   * the 1-D Hermite sums are evaluated in difference form H0 f0 + H1 f1 = f0 + H1 (f1 - f0),
//     so the large common value of neighbouring texels cancels exactly before it is scaled
//     by N in the chart derivative.
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/shm.h"

namespace shm {

// ------------------------------------------------------------------------------------------
// Table addressing
struct LutView {
    const void* data;
    const int32_t* N;
    const int64_t* offset;
    const float* r0;
    int32_t n_glyphs;
    int32_t N_uniform;
    int32_t dtype;
    int32_t layout;
};

__host__ __device__ __forceinline__ int64_t records_per_glyph(int N, int layout)
{
    const int64_t P = (layout == SHM_LAYOUT_CELL) ? (int64_t)N + 1
                      : (layout == SHM_LAYOUT_VALUE) ? (int64_t)N + 4 : (int64_t)N + 2;
    return 6 * P * P;
}

struct GlyphRef {
    int N;
    int64_t base;  // first record
    float r0;
};

__device__ __forceinline__ GlyphRef glyph_ref(const LutView& L, int g)
{
    GlyphRef r;
    if (L.N_uniform > 0) {
        r.N = L.N_uniform;
        r.base = (int64_t)g * records_per_glyph(L.N_uniform, L.layout);
    } else {
        r.N = __ldg(L.N + g);
        r.base = __ldg(L.offset + g);
    }
    r.r0 = L.r0 ? __ldg(L.r0 + g) : 0.0f;
    return r;
}

// ------------------------------------------------------------------------------------------
// Chart (§3.2)
struct Chart {
    int k, k1, k2;   // dominant axis and the two chart axes
    float sigma;     // sign of d_k
    float m;         // |d_k|
    float im;        // 1/|d_k| (round to nearest)
    float x, y;      // chart coordinates 2u-1 = d_k1/|d_k|, 2v-1 = d_k2/|d_k|
    int f;           // face 2k + (d_k < 0)
};

__device__ __forceinline__ float pick3(int c, float a0, float a1, float a2)
{
    return c == 0 ? a0 : (c == 1 ? a1 : a2);
}

// Returns false for zero / non-finite directions.  Besides the face it keeps 1/|d_k| so the
// cell coordinates need no further division.
__device__ __forceinline__ bool chart_of(float d0, float d1, float d2, Chart& c)
{
    const float a0 = fabsf(d0), a1 = fabsf(d1), a2 = fabsf(d2);
    int k = 0;
    float m = a0;
    if (a1 > m) { k = 1; m = a1; }
    if (a2 > m) { k = 2; m = a2; }
    if (!(m > 0.0f) || !(m <= 3.402823466e38f) || !(a0 == a0) || !(a1 == a1) || !(a2 == a2))
        return false;
    c.k = k;
    c.k1 = (k == 2) ? 0 : k + 1;
    c.k2 = (k == 0) ? 2 : k - 1;
    const float dk = pick3(k, d0, d1, d2);
    c.sigma = (dk < 0.0f) ? -1.0f : 1.0f;
    c.f = 2 * k + (dk < 0.0f ? 1 : 0);
    c.m = m;
    c.im = __frcp_rn(m);
    c.x = pick3(c.k1, d0, d1, d2) * c.im;
    c.y = pick3(c.k2, d0, d1, d2) * c.im;
    return true;
}

// Cell index and local coordinate along one chart axis: x = uN + 1/2 = q N/2 + (N+1)/2 with
// q = num/m, i = clamp(floor(x), 0, N), s = x - i, in double-float arithmetic: q = q0 + q1 with
// q0 = num * (1/m) and q1 = fma(-q0, m, num) * (1/m) (the residual is exact), carried through
// X = q N/2 with its exact product error, so s is correct to ~1e-8 of a cell for any N < 2^20.
__device__ __forceinline__ void cell_of(float num, float m, float im, int N, int& i, float& s)
{
    const float q = num * im;
    const float ql = fmaf(-q, m, num) * im;
    const float hN = 0.5f * (float)N;
    const float X = __fmul_rn(q, hN);
    const float Xl = fmaf(q, hN, -X) + ql * hN;  // product error + low part of q
    const float c = 0.5f * (float)(N + 1);
    float fl = floorf(__fadd_rn(X, c));
    float sv = __fadd_rn(__fsub_rn(X, fl - c), Xl);
    if (sv < 0.0f) { fl -= 1.0f; sv += 1.0f; }
    else if (sv >= 1.0f) { fl += 1.0f; sv -= 1.0f; }
    if (fl < 0.0f) { fl = 0.0f; }
    if (fl > (float)N) { fl = (float)N; }
    i = (int)fl;
    s = sv;
}

// ------------------------------------------------------------------------------------------
// Record fetch: the four corners (i,j) (i+1,j) (i,j+1) (i+1,j+1) as float4 (r, ru h, rv h, ruv h^2)
struct Corners {
    float4 c00, c10, c01, c11;
};

__device__ __forceinline__ float4 h4_to_f4(uint2 v)
{
    const __half2 a = *reinterpret_cast<const __half2*>(&v.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&v.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

__device__ __forceinline__ float4 b4_to_f4(uint2 v)
{
    // bf16 -> f32 is exact: the bf16 bits are the top half of the f32 bits
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                       __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
}

template <int DT>
__device__ __forceinline__ float4 load_rec(const void* base, int64_t rec)
{
    if (DT == SHM_F32) {
        return __ldg(reinterpret_cast<const float4*>(base) + rec);
    } else {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + rec);
        return DT == SHM_F16 ? h4_to_f4(v) : b4_to_f4(v);
    }
}

// 256-bit read-only load (sm_100+): 32 contiguous, 32-byte aligned bytes.
__device__ __forceinline__ void ldg256(const void* p, float4& a, float4& b)
{
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

template <int DT, int LAYOUT>
__device__ __forceinline__ Corners fetch_corners(const void* data, const GlyphRef& G, int f, int i, int j)
{
    Corners c;
    if (LAYOUT == SHM_LAYOUT_TEXEL) {
        const int64_t P = G.N + 2;
        const int64_t r = G.base + ((int64_t)f * P + j) * P + i;
        c.c00 = load_rec<DT>(data, r);
        c.c10 = load_rec<DT>(data, r + 1);
        c.c01 = load_rec<DT>(data, r + P);
        c.c11 = load_rec<DT>(data, r + P + 1);
    } else {
        // a cell record is one aligned block (64 B f32, 32 B 16-bit): 256-bit loads
        const int64_t P = G.N + 1;
        const int64_t cell = G.base + ((int64_t)f * P + j) * P + i;
        if (DT == SHM_F32) {
            const float* p = reinterpret_cast<const float*>(data) + cell * 16;
            ldg256(p, c.c00, c.c10);
            ldg256(p + 8, c.c01, c.c11);
        } else {
            float4 lo, hi;
            ldg256(reinterpret_cast<const uint16_t*>(data) + cell * 16, lo, hi);
            const uint2 r0 = make_uint2(__float_as_uint(lo.x), __float_as_uint(lo.y));
            const uint2 r1 = make_uint2(__float_as_uint(lo.z), __float_as_uint(lo.w));
            const uint2 r2 = make_uint2(__float_as_uint(hi.x), __float_as_uint(hi.y));
            const uint2 r3 = make_uint2(__float_as_uint(hi.z), __float_as_uint(hi.w));
            if (DT == SHM_F16) {
                c.c00 = h4_to_f4(r0); c.c10 = h4_to_f4(r1); c.c01 = h4_to_f4(r2); c.c11 = h4_to_f4(r3);
            } else {
                c.c00 = b4_to_f4(r0); c.c10 = b4_to_f4(r1); c.c01 = b4_to_f4(r2); c.c11 = b4_to_f4(r3);
            }
        }
    }
    return c;
}

// ------------------------------------------------------------------------------------------
// Paired float32 arithmetic (sm_100+): one instruction for the two lanes of a float2, each lane
// rounded as the scalar operation (fma: one rounding).  Frees issue slots where two independent
// lanes run the same operation; a broadcast operand (bc) costs nothing extra.
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.0f), a); }  // a - b, one rounding
__device__ __forceinline__ float4 padd4(float4 a, float4 b)
{
    const float2 lo = padd(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 hi = padd(make_float2(a.z, a.w), make_float2(b.z, b.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// ------------------------------------------------------------------------------------------
// 1-D cubic Hermite basis (§3.3) with H0 = 1 - H1 used implicitly (difference form)
struct Herm {
    float H1, h0d, h1d;     // H1, H0d, H1d
    float dH1, dh0d, dh1d;  // derivatives; dH0 = -dH1
};

__device__ __forceinline__ Herm herm(float s)
{
    Herm h;
    const float s2 = s * s;
    const float om = 1.0f - s;
    h.H1 = s2 * (3.0f - 2.0f * s);
    h.h0d = s * om * om;
    h.h1d = s2 * (s - 1.0f);
    h.dH1 = 6.0f * s * om;
    h.dh0d = om * (1.0f - 3.0f * s);
    h.dh1d = s * (3.0f * s - 2.0f);
    return h;
}

struct HermOut {
    float r, rs, rt;  // value and d/ds, d/dt
};

// Tensor-product Hermite value and first derivatives from the four corner records.  The rows along
// s are formed as (value, d/ds) pairs and interpolated along t as pairs (paired float32 arithmetic,
// the same operations in the same order as the scalar form).
__device__ __forceinline__ HermOut hermite2(const Corners& c, float s, float t)
{
    const Herm a = herm(s), b = herm(t);
    const float2 aH1 = make_float2(a.H1, a.dH1), ah0 = make_float2(a.h0d, a.dh0d), ah1 = make_float2(a.h1d, a.dh1d);
    // rows along s: value row p_b and v-derivative row q_b (Hermite of r_v h with r_uv h^2), each
    // with its s-derivative: P_b = (p_b, ps_b), Q_b = (q_b, qs_b)
    const float d0 = c.c10.x - c.c00.x, d1 = c.c11.x - c.c01.x;
    const float e0 = c.c10.z - c.c00.z, e1 = c.c11.z - c.c01.z;
    const float2 P0 = pfma(ah1, bc(c.c10.y), pfma(ah0, bc(c.c00.y), pfma(aH1, bc(d0), make_float2(c.c00.x, 0.0f))));
    const float2 P1 = pfma(ah1, bc(c.c11.y), pfma(ah0, bc(c.c01.y), pfma(aH1, bc(d1), make_float2(c.c01.x, 0.0f))));
    const float2 Q0 = pfma(ah1, bc(c.c10.w), pfma(ah0, bc(c.c00.w), pfma(aH1, bc(e0), make_float2(c.c00.z, 0.0f))));
    const float2 Q1 = pfma(ah1, bc(c.c11.w), pfma(ah0, bc(c.c01.w), pfma(aH1, bc(e1), make_float2(c.c01.z, 0.0f))));
    const float2 DP = psub(P1, P0);
    const float2 Rr = pfma(bc(b.h1d), Q1, pfma(bc(b.h0d), Q0, pfma(bc(b.H1), DP, P0)));  // (r, r_s)
    HermOut o;
    o.r = Rr.x;
    o.rs = Rr.y;
    o.rt = b.dH1 * DP.x + b.dh0d * Q0.x + b.dh1d * Q1.x;
    return o;
}

// The value alone (same operations as hermite2's r), for callers that need no derivative.
__device__ __forceinline__ float hermite_value(const Corners& c, float s, float t)
{
    const Herm a = herm(s), b = herm(t);
    const float d0 = c.c10.x - c.c00.x, d1 = c.c11.x - c.c01.x;
    const float e0 = c.c10.z - c.c00.z, e1 = c.c11.z - c.c01.z;
    const float p0 = c.c00.x + a.H1 * d0 + a.h0d * c.c00.y + a.h1d * c.c10.y;
    const float p1 = c.c01.x + a.H1 * d1 + a.h0d * c.c01.y + a.h1d * c.c11.y;
    const float q0 = c.c00.z + a.H1 * e0 + a.h0d * c.c00.w + a.h1d * c.c10.w;
    const float q1 = c.c01.z + a.H1 * e1 + a.h0d * c.c01.w + a.h1d * c.c11.w;
    const float dp = p1 - p0;
    return p0 + b.H1 * dp + b.h0d * q0 + b.h1d * q1;
}

// ------------------------------------------------------------------------------------------
// §3.4: the Cramer solution of G [alpha beta]^T = [R_u R_v]^T in closed form.  With
// w~ = a + x b + y c, rho = |w~|, e1 = (2/rho)(I - w w^T) b, e2 = (2/rho)(I - w w^T) c, the
// tangent vector (rho/2) [R_u b + R_v c - (x R_u + y R_v) a] satisfies grad.e1 = R_u,
// grad.e2 = R_v and grad.w = 0, so it is alpha e1 + beta e2 (det G = 16/rho^6 > 0, no clamp).
struct Vec3 {
    float x, y, z;
};

__device__ __forceinline__ Vec3 s2_gradient(const Chart& c, float Ru, float Rv)
{
    const float rho = sqrtf(fmaf(c.x, c.x, fmaf(c.y, c.y, 1.0f)));
    const float h = 0.5f * rho;
    const float gk = -h * c.sigma * fmaf(c.x, Ru, c.y * Rv);
    const float g1 = h * Ru;
    const float g2 = h * Rv;
    // scatter (k, k1, k2) -> (0, 1, 2)
    Vec3 g;
    g.x = (c.k == 0) ? gk : (c.k1 == 0 ? g1 : g2);
    g.y = (c.k == 1) ? gk : (c.k1 == 1 ? g1 : g2);
    g.z = (c.k == 2) ? gk : (c.k1 == 2 ? g1 : g2);
    return g;
}

__device__ __forceinline__ Vec3 surface_normal(float d0, float d1, float d2, float R, const Vec3& g)
{
    const float il = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    const float mx = fmaf(R * d0, il, -g.x), my = fmaf(R * d1, il, -g.y), mz = fmaf(R * d2, il, -g.z);
    const float im = rsqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
    return Vec3{mx * im, my * im, mz * im};
}

// One full query on one glyph: returns false (and leaves outputs unset) for invalid directions.
struct QueryResult {
    float R, Ru, Rv;
    Vec3 grad;
    int f, i, j;
};

template <int DT, int LAYOUT>
__device__ __forceinline__ bool query_one(const LutView& L, const GlyphRef& G, float d0, float d1, float d2,
                                          QueryResult& out, Chart& c)
{
    if (!chart_of(d0, d1, d2, c)) return false;
    int i, j;
    float s, t;
    cell_of(pick3(c.k1, d0, d1, d2), c.m, c.im, G.N, i, s);
    cell_of(pick3(c.k2, d0, d1, d2), c.m, c.im, G.N, j, t);
    const Corners cr = fetch_corners<DT, LAYOUT>(L.data, G, c.f, i, j);
    const HermOut h = hermite2(cr, s, t);
    out.R = G.r0 + h.r;
    out.Ru = (float)G.N * h.rs;
    out.Rv = (float)G.N * h.rt;
    out.grad = s2_gradient(c, out.Ru, out.Rv);
    out.f = c.f;
    out.i = i;
    out.j = j;
    return true;
}

// ------------------------------------------------------------------------------------------
// Value-only reconstruction baselines (§4.2, §4.5) on a SHM_LAYOUT_VALUE table: one scalar per
// texel, [6][N+4][N+4], entry (ii, jj) = texel (ii-1, jj-1), texel i at x = uN + 1/2 = i.
template <int DT>
__device__ __forceinline__ float load_val(const void* base, int64_t idx)
{
    if (DT == SHM_F32) return __ldg(reinterpret_cast<const float*>(base) + idx);
    if (DT == SHM_F16) return __half2float(__ldg(reinterpret_cast<const __half*>(base) + idx));
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(base) + idx));
}

template <int DT>
struct ValueFace {
    const void* data;
    int64_t base;  // entry (0, 0) of the face = texel (-1, -1)
    int S;
    __device__ __forceinline__ float operator()(int i, int j) const
    {
        return load_val<DT>(data, base + (int64_t)(j + 1) * S + (i + 1));
    }
};

// Catmull-Rom weights of taps i-1 .. i+2 at local coordinate s, and their s-derivatives.
__device__ __forceinline__ void catmull_rom(float s, float w[4], float dw[4])
{
    const float s2 = s * s, s3 = s2 * s;
    w[0] = 0.5f * (-s3 + 2.0f * s2 - s);
    w[1] = 0.5f * (3.0f * s3 - 5.0f * s2 + 2.0f);
    w[2] = 0.5f * (-3.0f * s3 + 4.0f * s2 + s);
    w[3] = 0.5f * (s3 - s2);
    dw[0] = 0.5f * (-3.0f * s2 + 4.0f * s - 1.0f);
    dw[1] = 0.5f * (9.0f * s2 - 10.0f * s);
    dw[2] = 0.5f * (-9.0f * s2 + 8.0f * s + 1.0f);
    dw[3] = 0.5f * (3.0f * s2 - 2.0f * s);
}

// Uniform cubic B-spline weights of taps i-1 .. i+2 (any s: the cell's polynomial).
__device__ __forceinline__ void bspline3(float s, float w[4])
{
    const float r = 1.0f - s, s2 = s * s, s3 = s2 * s;
    w[0] = r * r * r * (1.0f / 6.0f);
    w[1] = (3.0f * s3 - 6.0f * s2 + 4.0f) * (1.0f / 6.0f);
    w[2] = (-3.0f * s3 + 3.0f * s2 + 3.0f * s + 1.0f) * (1.0f / 6.0f);
    w[3] = s3 * (1.0f / 6.0f);
}

template <int DT>
__device__ __forceinline__ float tensor16(const ValueFace<DT>& V, int i, int j, const float wu[4], const float wv[4])
{
    float acc = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float row = 0.0f;
#pragma unroll
        for (int a = 0; a < 4; ++a) row = fmaf(wu[a], V(i - 1 + a, j - 1 + b), row);
        acc = fmaf(wv[b], row, acc);
    }
    return acc;
}

template <int DT>
__device__ __forceinline__ float bilinear_at(const ValueFace<DT>& V, int i, int j, float s, float t)
{
    const float a = V(i, j), b = V(i + 1, j), c = V(i, j + 1), d = V(i + 1, j + 1);
    const float lo = fmaf(s, b - a, a), hi = fmaf(s, d - c, c);
    return fmaf(t, hi - lo, lo);
}

// Cubic B-spline value at cell (k, l) shifted by (di, dj) texels, the cell clamped to [0, N]
// and the local coordinate carried along.
template <int DT>
__device__ __forceinline__ float bspline_at(const ValueFace<DT>& V, int N, int i, int j, float s, float t)
{
    const int ic = min(max(i, 0), N), jc = min(max(j, 0), N);
    float wu[4], wv[4];
    bspline3(s + (float)(i - ic), wu);
    bspline3(t + (float)(j - jc), wv);
    return tensor16(V, ic, jc, wu, wv);
}

template <int METHOD, int DT>
__device__ __forceinline__ bool recon_one(const LutView& L, const GlyphRef& G, float d0, float d1, float d2,
                                          QueryResult& out, Chart& c)
{
    if (!chart_of(d0, d1, d2, c)) return false;
    const int N = G.N;
    int i, j;
    float s, t;
    cell_of(pick3(c.k1, d0, d1, d2), c.m, c.im, N, i, s);
    cell_of(pick3(c.k2, d0, d1, d2), c.m, c.im, N, j, t);
    const int S = N + 4;
    const ValueFace<DT> V{L.data, G.base + (int64_t)c.f * S * S, S};
    const float hN = 0.5f * (float)N;
    float r, Ru = 0.0f, Rv = 0.0f;
    if (METHOD == SHM_RECON_NEAREST) {
        i = min(max(i + (s >= 0.5f ? 1 : 0), 1), N);
        j = min(max(j + (t >= 0.5f ? 1 : 0), 1), N);
        r = V(i, j);
    } else if (METHOD == SHM_RECON_BILINEAR) {
        r = bilinear_at(V, i, j, s, t);
        Ru = (bilinear_at(V, i + 1, j, s, t) - bilinear_at(V, i - 1, j, s, t)) * hN;
        Rv = (bilinear_at(V, i, j + 1, s, t) - bilinear_at(V, i, j - 1, s, t)) * hN;
    } else if (METHOD == SHM_RECON_BICUBIC) {
        float wu[4], dwu[4], wv[4], dwv[4];
        catmull_rom(s, wu, dwu);
        catmull_rom(t, wv, dwv);
        float acc = 0.0f, au = 0.0f, av = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float row = 0.0f, drow = 0.0f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float v = V(i - 1 + a, j - 1 + b);
                row = fmaf(wu[a], v, row);
                drow = fmaf(dwu[a], v, drow);
            }
            acc = fmaf(wv[b], row, acc);
            au = fmaf(wv[b], drow, au);
            av = fmaf(dwv[b], row, av);
        }
        r = acc;
        Ru = (float)N * au;
        Rv = (float)N * av;
    } else {
        r = bspline_at(V, N, i, j, s, t);
        Ru = (bspline_at(V, N, i + 1, j, s, t) - bspline_at(V, N, i - 1, j, s, t)) * hN;
        Rv = (bspline_at(V, N, i, j + 1, s, t) - bspline_at(V, N, i, j - 1, s, t)) * hN;
    }
    out.R = G.r0 + r;
    out.Ru = Ru;
    out.Rv = Rv;
    out.grad = s2_gradient(c, Ru, Rv);
    out.f = c.f;
    out.i = i;
    out.j = j;
    return true;
}

// ------------------------------------------------------------------------------------------
// Generic record store / load for any dtype and layout.
__device__ __forceinline__ uint2 f4_to_h4(float4 v)
{
    const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}

__device__ __forceinline__ uint2 f4_to_b4(float4 v)
{
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}

__device__ __forceinline__ void store_rec(void* data, int dtype, int64_t rec, float4 v)
{
    if (dtype == SHM_F32) reinterpret_cast<float4*>(data)[rec] = v;
    else if (dtype == SHM_F16) reinterpret_cast<uint2*>(data)[rec] = f4_to_h4(v);
    else reinterpret_cast<uint2*>(data)[rec] = f4_to_b4(v);
}

__device__ __forceinline__ void store_val(void* data, int dtype, int64_t idx, float v)
{
    if (dtype == SHM_F32) reinterpret_cast<float*>(data)[idx] = v;
    else if (dtype == SHM_F16) reinterpret_cast<__half*>(data)[idx] = __float2half_rn(v);
    else reinterpret_cast<__nv_bfloat16*>(data)[idx] = __float2bfloat16_rn(v);
}

__device__ __forceinline__ float4 load_rec_any(const void* data, int dtype, int64_t rec)
{
    if (dtype == SHM_F32) return load_rec<SHM_F32>(data, rec);
    if (dtype == SHM_F16) return load_rec<SHM_F16>(data, rec);
    return load_rec<SHM_BF16>(data, rec);
}

// Store texel (i, j) of face f: one record (texel layout) or up to four cell corners.
__device__ __forceinline__ void store_texel(void* data, int dtype, int layout, const GlyphRef& G, int f, int j,
                                            int i, float4 v)
{
    if (layout == SHM_LAYOUT_TEXEL) {
        const int64_t P = G.N + 2;
        store_rec(data, dtype, G.base + ((int64_t)f * P + j) * P + i, v);
    } else {
        const int64_t P = G.N + 1;
        for (int cj = j - 1; cj <= j; ++cj) {
            if (cj < 0 || cj > G.N) continue;
            for (int ci = i - 1; ci <= i; ++ci) {
                if (ci < 0 || ci > G.N) continue;
                const int corner = (j - cj) * 2 + (i - ci);
                store_rec(data, dtype, (G.base + ((int64_t)f * P + cj) * P + ci) * 4 + corner, v);
            }
        }
    }
}

__device__ __forceinline__ float4 load_texel(const void* data, int dtype, int layout, const GlyphRef& G, int f,
                                             int j, int i)
{
    if (layout == SHM_LAYOUT_TEXEL) {
        const int64_t P = G.N + 2;
        return load_rec_any(data, dtype, G.base + ((int64_t)f * P + j) * P + i);
    }
    const int64_t P = G.N + 1;
    const int ci = min(i, G.N), cj = min(j, G.N);
    return load_rec_any(data, dtype, (G.base + ((int64_t)f * P + cj) * P + ci) * 4 + (j - cj) * 2 + (i - ci));
}

}  // namespace shm
