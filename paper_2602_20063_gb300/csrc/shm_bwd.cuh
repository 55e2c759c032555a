// Reverse mode of one query (the paper has no adjoint; this makes tables fittable under autograd),
// shared by the atomic reverse passes (shm_query_bwd.cu) and the deterministic one
// (shm_query_bwd_det.cu).
//
// Per query the forward is recomputed and the upstream gradients (gR, ggrad, gnormal) are pulled
// back through, in reverse order:
//   normal  n = m/|m|, m = R w - grad:       gm = (gn - n (n.gn))/|m|;  gR += gm.w;  gw = R gm;
//                                            ggrad -= gm
//   grad    = (rho/2)[R_u b + R_v c - (x R_u + y R_v) a]  (the §3.4 Cramer solution in closed form)
//                                            -> gR_u, gR_v and the chart-coordinate terms gx, gy
//   Hermite r, r_s, r_t are linear in the 16 stored scalars (§3.3): each corner record receives a
//           float4 of weights (corner_weights), handed to the caller's emitter with the cell;
//           s, t move with the direction: gs, gt from the second derivatives of the patch
//   chart   x = d_k1/|d_k|, y = d_k2/|d_k|, s = (x+1)N/2 + 1/2 - i:  gd from gx + gs N/2, gy + gt N/2
//   w = d/|d|                               gd += (gw - w (w.gw))/|d|
// Face and cell indices are piecewise constant, so they carry no derivative.
//
// Where two independent lanes run the same operation the arithmetic is written on float2 pairs (the
// t-interpolation of a quantity and of its s-derivative; the b and c components of a tangent-frame
// vector; the corner weights' Hermite factors of s and t and the (x, y) and (z, w) halves of each
// weight record): sm_100+ executes __ffma2_rn / __fmul2_rn / __fadd2_rn as one instruction for both
// lanes, each lane rounded as the scalar operation, which frees issue slots in this
// instruction-bound pass.  The forward's Hermite factors and s-rows stay scalar: paired, their
// constant operands and pair alignment pushed the kernels past 64 registers into spills.
#pragma once
#include "shm_internal.h"

namespace shm {

// Cubic Hermite factors (§3.3) at s (.x) and t (.y), with H0 = 1 - H1 used implicitly (difference
// form), and their first derivatives (for the corner weights).
struct Herm2P {
    float2 H1, h0d, h1d, dH1, dh0d, dh1d;
};

__device__ __forceinline__ Herm2P herm2p(float2 u)
{
    Herm2P h;
    const float2 u2 = pmul(u, u);
    const float2 om = pfma(u, bc(-1.0f), bc(1.0f));  // 1 - u
    const float2 uom = pmul(u, om);
    h.H1 = pmul(u2, pfma(u, bc(-2.0f), bc(3.0f)));
    h.h0d = pmul(uom, om);
    h.h1d = pmul(u2, padd(u, bc(-1.0f)));
    h.dH1 = pmul(bc(6.0f), uom);
    h.dh0d = pmul(om, pfma(u, bc(-3.0f), bc(1.0f)));
    h.dh1d = pmul(u, pfma(u, bc(3.0f), bc(-2.0f)));
    return h;
}

// The same factors at one coordinate, with the second derivatives (the forward recompute).
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

// Weights of the four corner records (index bb * 2 + aa) for upstream (g_r, g_rs, g_rt) on the
// value and its two chart derivatives at (s, t): each record's (r, r_u h, r_v h, r_uv h^2) weights.
__device__ __forceinline__ void corner_weights(float s, float t, float g_r, float g_rs, float g_rt, float4 (&w)[4])
{
    const Herm2P h = herm2p(make_float2(s, t));
    const float2 H0 = pfma(h.H1, bc(-1.0f), bc(1.0f));  // (H0(s), H0(t))
    // per corner column aa: (al, ad) weigh the record's (r, r_u h) rows against the t factors,
    // (be, bd) against their t derivatives
    const float2 AL0 = make_float2(fmaf(g_rs, -h.dH1.x, g_r * H0.x), fmaf(g_rs, h.dh0d.x, g_r * h.h0d.x));
    const float2 AL1 = make_float2(fmaf(g_rs, h.dH1.x, g_r * h.H1.x), fmaf(g_rs, h.dh1d.x, g_r * h.h1d.x));
    const float2 BE0 = pmul(bc(g_rt), make_float2(H0.x, h.h0d.x));
    const float2 BE1 = pmul(bc(g_rt), make_float2(h.H1.x, h.h1d.x));
    const float Ht[2] = {H0.y, h.H1.y}, dHt[2] = {-h.dH1.y, h.dH1.y};
    const float hdt[2] = {h.h0d.y, h.h1d.y}, dhdt[2] = {h.dh0d.y, h.dh1d.y};
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
        const float2 x0 = pfma(BE0, bc(dHt[bb]), pmul(AL0, bc(Ht[bb])));
        const float2 z0 = pfma(BE0, bc(dhdt[bb]), pmul(AL0, bc(hdt[bb])));
        const float2 x1 = pfma(BE1, bc(dHt[bb]), pmul(AL1, bc(Ht[bb])));
        const float2 z1 = pfma(BE1, bc(dhdt[bb]), pmul(AL1, bc(hdt[bb])));
        w[bb * 2] = make_float4(x0.x, x0.y, z0.x, z0.y);
        w[bb * 2 + 1] = make_float4(x1.x, x1.y, z1.x, z1.y);
    }
}

// Upstream values of query q read from global memory where bwd_query uses them (streaming loads).
struct GlobalUp {
    const BackwardArgs& a;
    int64_t q;
    __device__ __forceinline__ float gR() const { return __ldcs(a.gR + q); }
    __device__ __forceinline__ float ggrad(int k) const { return __ldcs(a.ggrad + 3 * q + k); }
    __device__ __forceinline__ float gnormal(int k) const { return __ldcs(a.gnormal + 3 * q + k); }
    __device__ __forceinline__ float R_target() const { return __ldcs(a.R_target + q); }
    __device__ __forceinline__ float n_target(int k) const { return __ldcs(a.n_target + 3 * q + k); }
};

// Upstream values loaded before the query's forward recompute (the arrays bwd_query reads: gR,
// ggrad, gnormal; zero where absent), so that their latency overlaps it.
struct PreUp {
    float r, g0, g1, g2, n0, n1, n2;
    __device__ __forceinline__ PreUp(const BackwardArgs& a, int64_t q)
    {
        r = a.gR ? __ldcs(a.gR + q) : 0.0f;
        g0 = g1 = g2 = n0 = n1 = n2 = 0.0f;
        if (a.ggrad) { g0 = __ldcs(a.ggrad + 3 * q); g1 = __ldcs(a.ggrad + 3 * q + 1); g2 = __ldcs(a.ggrad + 3 * q + 2); }
        if (a.gnormal) { n0 = __ldcs(a.gnormal + 3 * q); n1 = __ldcs(a.gnormal + 3 * q + 1); n2 = __ldcs(a.gnormal + 3 * q + 2); }
    }
    __device__ __forceinline__ float gR() const { return r; }
    __device__ __forceinline__ float ggrad(int k) const { return k == 0 ? g0 : (k == 1 ? g1 : g2); }
    __device__ __forceinline__ float gnormal(int k) const { return k == 0 ? n0 : (k == 1 ? n1 : n2); }
    __device__ __forceinline__ float R_target() const { return 0.0f; }  // not used without the fit loss
    __device__ __forceinline__ float n_target(int) const { return 0.0f; }
};

// Fit targets loaded before the query's forward recompute (R_target, n_target), so that their
// latency overlaps it.
struct PreFit {
    float rt, t0, t1, t2;
    __device__ __forceinline__ PreFit(const BackwardArgs& a, int64_t q)
    {
        rt = __ldcs(a.R_target + q);
        t0 = __ldcs(a.n_target + 3 * q);
        t1 = __ldcs(a.n_target + 3 * q + 1);
        t2 = __ldcs(a.n_target + 3 * q + 2);
    }
    __device__ __forceinline__ float gR() const { return 0.0f; }  // not used by the fit loss
    __device__ __forceinline__ float ggrad(int) const { return 0.0f; }
    __device__ __forceinline__ float gnormal(int) const { return 0.0f; }
    __device__ __forceinline__ float R_target() const { return rt; }
    __device__ __forceinline__ float n_target(int k) const { return k == 0 ? t0 : (k == 1 ? t1 : t2); }
};

// One query's reverse pass on glyph table Gr: the 2x2 footprint comes from `fetch(f, i, j)`;
// `emit(rec, s, t, g_r, g_rs, g_rt)` receives the cell (record index of its corner (0,0) within the
// glyph's texel table), the cell coordinates and the upstream values of r, r_s, r_t, from which
// corner_weights gives the four record gradients; the direction gradient goes to dd.  `up`
// supplies the upstream values (GlobalUp, PreUp or PreFit).
template <bool FIT, class Up, class Fetch, class Emit>
__device__ __forceinline__ void bwd_query(const BackwardArgs& a, const Up& up, const GlyphRef& Gr, const Chart& c,
                                          float d0, float d1, float d2, const Fetch& fetch, Emit& emit, float3& dd,
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
    // along t: (r, r_s) and (r_t, r_st) as pairs; r_ss and r_tt apart
    const float2 P0 = make_float2(p0, ps0), Q0 = make_float2(q0, qs0), Q1 = make_float2(q1, qs1);
    const float2 DP = psub(make_float2(p1, ps1), P0);
    const float2 Rr = pfma(bc(B.h1d), Q1, pfma(bc(B.h0d), Q0, pfma(bc(B.H1), DP, P0)));  // (r, r_s)
    const float2 Rt = pfma(bc(B.dh1d), Q1, pfma(bc(B.dh0d), Q0, pmul(bc(B.dH1), DP)));   // (r_t, r_st)
    const float r = Rr.x, rs = Rr.y, rt = Rt.x, rst = Rt.y, dp = DP.x;
    const float rss = pss0 + B.H1 * (pss1 - pss0) + B.h0d * qss0 + B.h1d * qss1;
    const float rtt = B.ddH1 * dp + B.ddh0d * q0 + B.ddh1d * q1;
    const float Nf = (float)N;
    const float R = Gr.r0 + r;
    const float2 Ruv = pmul(bc(Nf), make_float2(rs, rt));  // (R_u, R_v) = tangent components (b, c) of V
    const float x = c.x, y = c.y;
    const float2 xy = make_float2(x, y);
    const float rho2 = fmaf(x, x, fmaf(y, y, 1.0f));
    const float irho = rsqrtf(rho2), rho = rho2 * irho;  // reciprocal square root: no division below
    const float hr = 0.5f * rho;
    // tangent-frame components (a, b, c) = (sigma e_k, e_k1, e_k2); (b, c) as pairs
    const float Va = -(x * Ruv.x + y * Ruv.y);
    const float il = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    const float wk = pick3(c.k, d0, d1, d2) * il * c.sigma;                       // w . a
    const float2 w12 = pmul(bc(il), make_float2(pick3(c.k1, d0, d1, d2), pick3(c.k2, d0, d1, d2)));  // w . b, w . c
    const float Ga = hr * Va;
    const float2 G12n = pmul(bc(-hr), Ruv);  // -(G_b, G_c)
    const float ma = R * wk - Ga;
    const float2 m12 = pfma(bc(R), w12, G12n);
    const float iml = rsqrtf(ma * ma + m12.x * m12.x + m12.y * m12.y);
    const float na = ma * iml;
    const float2 n12 = pmul(bc(iml), m12);
    // upstream in the (a, b, c) frame
    float gRu_in = a.gR ? up.gR() : 0.0f;
    float gGa = 0.f, gna = 0.f;
    float2 gG12 = make_float2(0.f, 0.f), gn12 = make_float2(0.f, 0.f);
    if (FIT) {
        // L_q = w_v (R - R_t)^2 + w_n |n - n_t|^2: upstream dL/dR, dL/dn in the frame
        const float eR = R - up.R_target();
        const float t0 = up.n_target(0), t1 = up.n_target(1), t2 = up.n_target(2);
        const float ea = na - pick3(c.k, t0, t1, t2) * c.sigma;
        const float2 e12 = psub(n12, make_float2(pick3(c.k1, t0, t1, t2), pick3(c.k2, t0, t1, t2)));
        loss_acc += a.w_value * eR * eR + a.w_normal * (ea * ea + e12.x * e12.x + e12.y * e12.y);
        gRu_in = 2.0f * a.w_value * eR;
        const float wn2 = 2.0f * a.w_normal;
        gna = wn2 * ea;
        gn12 = pmul(bc(wn2), e12);
    }
    if (!FIT && a.ggrad) {
        const float gx0 = up.ggrad(0), gx1 = up.ggrad(1), gx2 = up.ggrad(2);
        gGa = pick3(c.k, gx0, gx1, gx2) * c.sigma;
        gG12 = make_float2(pick3(c.k1, gx0, gx1, gx2), pick3(c.k2, gx0, gx1, gx2));
    }
    if (!FIT && a.gnormal) {
        const float gx0 = up.gnormal(0), gx1 = up.gnormal(1), gx2 = up.gnormal(2);
        gna = pick3(c.k, gx0, gx1, gx2) * c.sigma;
        gn12 = make_float2(pick3(c.k1, gx0, gx1, gx2), pick3(c.k2, gx0, gx1, gx2));
    }
    // --- reverse
    const float ndg = na * gna + n12.x * gn12.x + n12.y * gn12.y;
    const float gma = (gna - na * ndg) * iml;
    const float2 gm12 = pmul(bc(iml), pfma(n12, bc(-ndg), gn12));
    const float gRt = gRu_in + gma * wk + gm12.x * w12.x + gm12.y * w12.y;
    const float gwa = R * gma;
    const float2 gw12 = pmul(bc(R), gm12);
    const float tGa = gGa - gma;
    const float2 tG12 = psub(gG12, gm12);
    const float gVa = hr * tGa;
    const float2 gV12 = pmul(bc(hr), tG12);
    const float grho = 0.5f * (Va * tGa + Ruv.x * tG12.x + Ruv.y * tG12.y);
    const float2 gRuv = pfma(xy, bc(-gVa), gV12);                          // (gR_u, gR_v)
    const float2 gxy = pfma(xy, bc(grho * irho), pmul(Ruv, bc(-gVa)));    // (gx, gy)
    const float g_r = gRt;
    const float2 g_st = pmul(bc(Nf), gRuv);                                // (g_rs, g_rt)
    // table: the cell's corner weights go to the emitter (record index of corner (0,0) within the
    // glyph's texel table; corner (aa, bb) is record rec + bb P + aa)
    emit(((int64_t)c.f * (N + 2) + j) * (N + 2) + i, s, t, g_r, g_st.x, g_st.y);
    if (a.ddirs) {
        // (gs, gt) = g_r (r_s, r_t) + g_rs (r_ss, r_st) + g_rt (r_st, r_tt)
        const float2 gst = pfma(bc(g_st.y), make_float2(rst, rtt),
                                pfma(bc(g_st.x), make_float2(rss, rst), pmul(bc(g_r), make_float2(rs, rt))));
        const float2 gxxyy = pfma(gst, bc(0.5f * Nf), gxy);
        // chart coordinates -> d (frame components; a-component carries sigma)
        float dA = -(x * gxxyy.x + y * gxxyy.y) * c.im;  // along a = sigma e_k (c.im = 1/|d_k|)
        float2 dBC = pmul(gxxyy, bc(c.im));
        // w = d/|d|
        const float wdg = wk * gwa + w12.x * gw12.x + w12.y * gw12.y;
        dA += (gwa - wk * wdg) * il;
        dBC = pfma(pfma(w12, bc(-wdg), gw12), bc(il), dBC);
        // back to Cartesian (a = sigma e_k): component c.k gets dA sigma, c.k1 dB, c.k2 dC
        const float sA = dA * c.sigma;
        const float dB = dBC.x, dC = dBC.y;
        dd = make_float3(c.k == 0 ? sA : (c.k1 == 0 ? dB : dC), c.k == 1 ? sA : (c.k1 == 1 ? dB : dC),
                         c.k == 2 ? sA : (c.k1 == 2 ? dB : dC));
    }
}

}  // namespace shm
