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
#pragma once
#include "shm_internal.h"

namespace shm {

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
// value and its two chart derivatives: each record's (r, r_u h, r_v h, r_uv h^2) weights.
__device__ __forceinline__ void corner_weights(const Herm2& A, const Herm2& B, float g_r, float g_rs, float g_rt,
                                               float4 (&w)[4])
{
    const float H0s = 1.0f - A.H1, dH0s = -A.dH1, H0t = 1.0f - B.H1, dH0t = -B.dH1;
    const float al[2] = {g_r * H0s + g_rs * dH0s, g_r * A.H1 + g_rs * A.dH1};
    const float ad[2] = {g_r * A.h0d + g_rs * A.dh0d, g_r * A.h1d + g_rs * A.dh1d};
    const float be[2] = {g_rt * H0s, g_rt * A.H1}, bd[2] = {g_rt * A.h0d, g_rt * A.h1d};
    const float Ht[2] = {H0t, B.H1}, dHt[2] = {dH0t, B.dH1}, hdt[2] = {B.h0d, B.h1d}, dhdt[2] = {B.dh0d, B.dh1d};
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int aa = 0; aa < 2; ++aa) {
            float4 wv;
            wv.x = al[aa] * Ht[bb] + be[aa] * dHt[bb];
            wv.y = ad[aa] * Ht[bb] + bd[aa] * dHt[bb];
            wv.z = al[aa] * hdt[bb] + be[aa] * dhdt[bb];
            wv.w = ad[aa] * hdt[bb] + bd[aa] * dhdt[bb];
            w[bb * 2 + aa] = wv;
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
// `emit(rec, A, B, s, t, g_r, g_rs, g_rt)` receives the cell (record index of its corner (0,0)
// within the glyph's texel table), the Hermite factors at (s, t) and the upstream values of
// r, r_s, r_t, from which corner_weights gives the four record gradients; the direction gradient
// goes to dd.  `up` supplies the upstream values (GlobalUp or PreUp).
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
    const float rho2 = fmaf(x, x, fmaf(y, y, 1.0f));
    const float irho = rsqrtf(rho2), rho = rho2 * irho;  // reciprocal square root: no division below
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
    float gRu_in = a.gR ? up.gR() : 0.0f;
    float gGa = 0.f, gGb = 0.f, gGc = 0.f, gna = 0.f, gnb = 0.f, gnc = 0.f;
    if (FIT) {
        // L_q = w_v (R - R_t)^2 + w_n |n - n_t|^2: upstream dL/dR, dL/dn in the frame
        const float eR = R - up.R_target();
        const float t0 = up.n_target(0), t1 = up.n_target(1), t2 = up.n_target(2);
        const float ea = na - pick3(c.k, t0, t1, t2) * c.sigma, eb = nb - pick3(c.k1, t0, t1, t2),
                    ec = nc - pick3(c.k2, t0, t1, t2);
        loss_acc += a.w_value * eR * eR + a.w_normal * (ea * ea + eb * eb + ec * ec);
        gRu_in = 2.0f * a.w_value * eR;
        gna = 2.0f * a.w_normal * ea;
        gnb = 2.0f * a.w_normal * eb;
        gnc = 2.0f * a.w_normal * ec;
    }
    if (!FIT && a.ggrad) {
        const float gx0 = up.ggrad(0), gx1 = up.ggrad(1), gx2 = up.ggrad(2);
        gGa = pick3(c.k, gx0, gx1, gx2) * c.sigma;
        gGb = pick3(c.k1, gx0, gx1, gx2);
        gGc = pick3(c.k2, gx0, gx1, gx2);
    }
    if (!FIT && a.gnormal) {
        const float gx0 = up.gnormal(0), gx1 = up.gnormal(1), gx2 = up.gnormal(2);
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
    const float gx = -Ru * gVa + grho * x * irho;
    const float gy = -Rv * gVa + grho * y * irho;
    const float g_r = gRt, g_rs = Nf * gRu, g_rt = Nf * gRv;
    // table: the cell's corner weights go to the emitter (record index of corner (0,0) within the
    // glyph's texel table; corner (aa, bb) is record rec + bb P + aa)
    emit(((int64_t)c.f * (N + 2) + j) * (N + 2) + i, A, B, s, t, g_r, g_rs, g_rt);
    if (a.ddirs) {
        const float gs = g_r * rs + g_rs * rss + g_rt * rst;
        const float gt = g_r * rt + g_rs * rst + g_rt * rtt;
        const float gxx = gx + gs * 0.5f * Nf, gyy = gy + gt * 0.5f * Nf;
        // chart coordinates -> d (frame components; a-component carries sigma)
        float dA = -(x * gxx + y * gyy) * c.im;  // along a = sigma e_k (c.im = 1/|d_k|)
        float dB = gxx * c.im, dC = gyy * c.im;
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

}  // namespace shm
