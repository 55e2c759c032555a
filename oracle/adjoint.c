/*
 * Oracle (test infrastructure only): reverse-mode derivative of the query and of the SH bake.
 * The paper has no adjoint; this is the hand-derived transpose of the forward steps in query.c,
 * taken in reverse order, in float64:
 *
 *   forward                                   reverse
 *   w = d/|d|                                 gd += (gw - w (w.gw))/|d|
 *   m = |d_k| (sign sigma), x = d_k1/m,       gd_k1 += gx'/m, gd_k2 += gy'/m,
 *     y = d_k2/m, u = (x+1)/2, v = (y+1)/2      gd_k  -= sigma (x gx' + y gy')/m
 *   s = uN + 1/2 - i,  t = vN + 1/2 - j       gx' = gx + gs N/2,  gy' = gy + gt N/2
 *   (r, r_s, r_t) = Hermite(s, t; 16 scalars) d(16 scalars) += weights; gs, gt from 2nd derivatives
 *   R = r0 + r, R_u = N r_s, R_v = N r_t
 *   grad = (rho/2)[R_u b + R_v c - (x R_u + y R_v) a],  rho = sqrt(1 + x^2 + y^2)
 *   n = (R w - grad)/|R w - grad|             gm = (gn - n (n.gn))/|R w - grad|
 *
 * The gradient line is the closed form of the §3.4 Cramer solution (both give the unique
 * tangent vector with grad.e1 = R_u and grad.e2 = R_v; the tests check that they agree).
 * The face and cell indices are piecewise constant in d, so they carry no derivative; at face
 * and cell boundaries (a set of measure zero) the one-sided derivative of the chosen cell is
 * returned.  The whole file is pinned by central finite differences of query.c and by the
 * dot-product test <J x, y> = <x, J^T y>.
 */
#include <math.h>
#include <string.h>
#include <stdlib.h>
#include "oracle.h"

void shmo_query_vjp_one(const double* glut, int N, double r0, const double d[3],
                        double gR, const double gG[3], const double gn[3],
                        double* dglut, double dd[3])
{
    int P = N + 2;
    /* ---- forward, keeping intermediates */
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double w[3] = {d[0] / len, d[1] / len, d[2] / len};
    double u, v;
    int f = shmo_face_uv(d, &u, &v);
    int k = f / 2, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    double sigma = (f % 2) ? -1.0 : 1.0;
    double m = fabs(d[k]);
    double x = 2.0 * u - 1.0, y = 2.0 * v - 1.0;
    int i, j;
    double s, t;
    shmo_cell(N, u, &i, &s);
    shmo_cell(N, v, &j, &t);
    const double* face = glut + (size_t)f * P * P * 4;
    double h6[6];
    shmo_hermite_eval(face, N, i, j, s, t, h6);
    double R = r0 + h6[0], Ru = (double)N * h6[1], Rv = (double)N * h6[2];
    double a[3], b[3], c[3];
    shmo_face_frame(f, a, b, c);
    double rho = sqrt(1.0 + x * x + y * y);
    double V[3], G[3];
    for (int q = 0; q < 3; ++q) {
        V[q] = Ru * b[q] + Rv * c[q] - (x * Ru + y * Rv) * a[q];
        G[q] = 0.5 * rho * V[q];
    }
    double mv[3];
    for (int q = 0; q < 3; ++q) mv[q] = R * w[q] - G[q];
    double ml = sqrt(mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]);
    double n[3] = {mv[0] / ml, mv[1] / ml, mv[2] / ml};

    /* ---- reverse */
    double ndotg = n[0] * gn[0] + n[1] * gn[1] + n[2] * gn[2];
    double gm[3];
    for (int q = 0; q < 3; ++q) gm[q] = (gn[q] - n[q] * ndotg) / ml;
    double gRt = gR + gm[0] * w[0] + gm[1] * w[1] + gm[2] * w[2];
    double gw[3], gGt[3];
    for (int q = 0; q < 3; ++q) {
        gw[q] = R * gm[q];
        gGt[q] = gG[q] - gm[q];
    }
    double gV[3];
    for (int q = 0; q < 3; ++q) gV[q] = 0.5 * rho * gGt[q];
    double grho = 0.5 * (V[0] * gGt[0] + V[1] * gGt[1] + V[2] * gGt[2]);
    double gVa = gV[0] * a[0] + gV[1] * a[1] + gV[2] * a[2];
    double gVb = gV[0] * b[0] + gV[1] * b[1] + gV[2] * b[2];
    double gVc = gV[0] * c[0] + gV[1] * c[1] + gV[2] * c[2];
    double gRu = gVb - x * gVa;
    double gRv = gVc - y * gVa;
    double gx = -Ru * gVa + grho * x / rho;
    double gy = -Rv * gVa + grho * y / rho;
    /* R = r0 + r, R_u = N r_s, R_v = N r_t */
    double g_r = gRt, g_rs = (double)N * gRu, g_rt = (double)N * gRv;
    /* 16 stored scalars: the query is linear in them */
    if (dglut) {
        double W[3][4][4];
        shmo_hermite_weights(s, t, W);
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                int corner = bb * 2 + aa;
                double* p = dglut + ((size_t)f * P * P + (size_t)(j + bb) * P + (size_t)(i + aa)) * 4;
                for (int ch = 0; ch < 4; ++ch)
                    p[ch] += g_r * W[0][corner][ch] + g_rs * W[1][corner][ch] + g_rt * W[2][corner][ch];
            }
    }
    if (dd) {
        double gs = g_r * h6[1] + g_rs * h6[3] + g_rt * h6[4];
        double gt = g_r * h6[2] + g_rs * h6[4] + g_rt * h6[5];
        double gxx = gx + gs * (double)N / 2.0;
        double gyy = gy + gt * (double)N / 2.0;
        double gd[3] = {0.0, 0.0, 0.0};
        gd[k1] += gxx / m;
        gd[k2] += gyy / m;
        gd[k] -= sigma * (x * gxx + y * gyy) / m;
        double wdotg = w[0] * gw[0] + w[1] * gw[1] + w[2] * gw[2];
        for (int q = 0; q < 3; ++q) gd[q] += (gw[q] - w[q] * wdotg) / len;
        for (int q = 0; q < 3; ++q) dd[q] = gd[q];
    }
}

void shmo_query_vjp_batch(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                          int64_t Q, const float* dirs, const int32_t* glyph,
                          const double* gR, const double* gG, const double* gn,
                          double* dpool, double* ddirs)
{
    const double zero3[3] = {0.0, 0.0, 0.0};
    for (int64_t q = 0; q < Q; ++q) {
        int g = glyph ? glyph[q] : 0;
        double d[3] = {dirs[3 * q], dirs[3 * q + 1], dirs[3 * q + 2]};
        double dd[3];
        shmo_query_vjp_one(pool + (size_t)off[g] * 4, Ns[g], r0 ? r0[g] : 0.0, d,
                           gR ? gR[q] : 0.0, gG ? gG + 3 * q : zero3, gn ? gn + 3 * q : zero3,
                           dpool ? dpool + (size_t)off[g] * 4 : NULL, ddirs ? dd : NULL);
        if (ddirs) for (int k = 0; k < 3; ++k) ddirs[3 * q + k] = dd[k];
    }
}

/* The SH bake is linear in the coefficients, lut = sum_k c_k B_k, so dL/dc_k = <dL/dlut, B_k>. */
void shmo_bake_sh_vjp(int N, int L, const double* dlut, double* dcoeffs)
{
    int P = N + 2, K = shmo_sh_count(L);
    double h = 1.0 / (double)N;
    double* Yk = (double*)malloc(sizeof(double) * 4 * (size_t)K);
    for (int k = 0; k < K; ++k) dcoeffs[k] = 0.0;
    for (int f = 0; f < 6; ++f)
        for (int j = 0; j < P; ++j)
            for (int i = 0; i < P; ++i) {
                shmo_sh_chart_basis(L, f, shmo_texel_centre(i, N), shmo_texel_centre(j, N), Yk);
                const double* g = dlut + (((size_t)f * P + j) * P + i) * 4;
                for (int k = 0; k < K; ++k)
                    dcoeffs[k] += g[0] * Yk[4 * k] + g[1] * Yk[4 * k + 1] * h +
                                  g[2] * Yk[4 * k + 2] * h + g[3] * Yk[4 * k + 3] * h * h;
            }
    free(Yk);
}
