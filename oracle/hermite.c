/*
 * Oracle (test infrastructure only): §3.3 (reconstruction and derivative extraction).
 *
 * 1-D cubic Hermite basis (§3.3):  H0 = 2s^3 - 3s^2 + 1,  H1 = -2s^3 + 3s^2,
 *                                   H0d = s^3 - 2s^2 + s,  H1d = s^3 - s^2.
 * 2-D reconstruction: r(s,t) = sum over the four corners (a,b) in {0,1}^2 of
 *   H_a(s)H_b(t) r_ab + H^d_a(s)H_b(t) (r_u h)_ab + H_a(s)H^d_b(t) (r_v h)_ab
 *   + H^d_a(s)H^d_b(t) (r_uv h^2)_ab,
 * where corner a indexes texel column i (a=0) / i+1 (a=1) along u and b indexes row j / j+1
 * along v.  Chart derivatives: r_u = (1/h) d r/ds, r_v = (1/h) d r/dt, the paper's elided
 * terms completed by the product rule.  Second derivatives (used only by the adjoint) follow
 * the same pattern with H''.
 *
 * Cell location (§3.2 with cell-centred texels u_i = (i-1/2)/N): x = u N + 1/2,
 * i = clamp(floor(x), 0, N), s = x - i, so the corners are texels i and i+1 of the padded face.
 */
#include <math.h>
#include "oracle.h"

void shmo_hermite_basis(double s, double H[4], double dH[4], double ddH[4])
{
    double s2 = s * s, s3 = s2 * s;
    H[0] = 2.0 * s3 - 3.0 * s2 + 1.0;
    H[1] = -2.0 * s3 + 3.0 * s2;
    H[2] = s3 - 2.0 * s2 + s;
    H[3] = s3 - s2;
    dH[0] = 6.0 * s2 - 6.0 * s;
    dH[1] = -6.0 * s2 + 6.0 * s;
    dH[2] = 3.0 * s2 - 4.0 * s + 1.0;
    dH[3] = 3.0 * s2 - 2.0 * s;
    ddH[0] = 12.0 * s - 6.0;
    ddH[1] = -12.0 * s + 6.0;
    ddH[2] = 6.0 * s - 4.0;
    ddH[3] = 6.0 * s - 2.0;
}

void shmo_cell(int N, double u, int* i, double* s)
{
    double x = u * (double)N + 0.5;
    double fl = floor(x);
    if (fl < 0.0) fl = 0.0;
    if (fl > (double)N) fl = (double)N;
    *i = (int)fl;
    *s = x - fl;
}

/* Basis index: value functions H_a at 0..1, derivative functions H^d_a at 2..3. */
static void corner_basis(const double H[4], int a, double* val, double* der)
{
    *val = H[a];
    *der = H[2 + a];
}

void shmo_hermite_weights(double s, double t, double w[3][4][4])
{
    double Hs[4], dHs[4], ddHs[4], Ht[4], dHt[4], ddHt[4];
    shmo_hermite_basis(s, Hs, dHs, ddHs);
    shmo_hermite_basis(t, Ht, dHt, ddHt);
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 2; ++a) {
            int corner = b * 2 + a;
            double hs, hsd, hs1, hsd1, ht, htd, ht1, htd1;
            corner_basis(Hs, a, &hs, &hsd);
            corner_basis(dHs, a, &hs1, &hsd1);
            corner_basis(Ht, b, &ht, &htd);
            corner_basis(dHt, b, &ht1, &htd1);
            /* value */
            w[0][corner][0] = hs * ht;
            w[0][corner][1] = hsd * ht;
            w[0][corner][2] = hs * htd;
            w[0][corner][3] = hsd * htd;
            /* d/ds */
            w[1][corner][0] = hs1 * ht;
            w[1][corner][1] = hsd1 * ht;
            w[1][corner][2] = hs1 * htd;
            w[1][corner][3] = hsd1 * htd;
            /* d/dt */
            w[2][corner][0] = hs * ht1;
            w[2][corner][1] = hsd * ht1;
            w[2][corner][2] = hs * htd1;
            w[2][corner][3] = hsd * htd1;
        }
    }
}

void shmo_hermite_eval(const double* face, int N, int i, int j, double s, double t, double out[6])
{
    int P = N + 2;
    double Hs[4], dHs[4], ddHs[4], Ht[4], dHt[4], ddHt[4];
    shmo_hermite_basis(s, Hs, dHs, ddHs);
    shmo_hermite_basis(t, Ht, dHt, ddHt);
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 2; ++a) {
            const double* p = face + ((size_t)(j + b) * P + (size_t)(i + a)) * 4;
            /* s-direction factors (value / first / second derivative of the basis) */
            double v0 = Hs[a], vd = Hs[2 + a];
            double d0 = dHs[a], dd = dHs[2 + a];
            double e0 = ddHs[a], ed = ddHs[2 + a];
            /* t-direction factors */
            double w0 = Ht[b], wd = Ht[2 + b];
            double x0 = dHt[b], xd = dHt[2 + b];
            double y0 = ddHt[b], yd = ddHt[2 + b];
            out[0] += v0 * w0 * p[0] + vd * w0 * p[1] + v0 * wd * p[2] + vd * wd * p[3];
            out[1] += d0 * w0 * p[0] + dd * w0 * p[1] + d0 * wd * p[2] + dd * wd * p[3];
            out[2] += v0 * x0 * p[0] + vd * x0 * p[1] + v0 * xd * p[2] + vd * xd * p[3];
            out[3] += e0 * w0 * p[0] + ed * w0 * p[1] + e0 * wd * p[2] + ed * wd * p[3];
            out[4] += d0 * x0 * p[0] + dd * x0 * p[1] + d0 * xd * p[2] + dd * xd * p[3];
            out[5] += v0 * y0 * p[0] + vd * y0 * p[1] + v0 * yd * p[2] + vd * yd * p[3];
        }
    }
}
