/*
 * Oracle (test infrastructure only): cubemap chart, tangents, metric and normal in float64.
 *
 * §3.2: a direction maps to one of six faces with local (u,v) in [0,1]^2.  The paper prints
 * no face table, so this file fixes one (any fixed table is correct because gutters are baked
 * by evaluation in each face's own chart, §3.2):
 *   axis k = argmax_k |w_k| (ties -> lowest k), sign sigma = +1 iff w_k >= 0 (so -0 counts as +),
 *   face f = 2k + (sigma < 0); frame a_f = sigma e_k, b_f = e_{(k+1)%3}, c_f = e_{(k+2)%3};
 *   unnormalised direction w~(u,v) = a_f + (2u-1) b_f + (2v-1) c_f.
 * §3.2 texel centres: padded (N+2)^2 per face, interior 1..N, h = 1/N; the paper does not say
 * where centres lie; the cell-centred reading u_i = (i - 1/2)/N is used (gutter i=0 at -h/2).
 * §3.4: tangents by differentiating the normalised cubemap direction, metric tensor G, Cramer's
 * rule, clamped det G, normal n.
 */
#include <math.h>
#include "oracle.h"

int shmo_face_uv(const double w[3], double* u, double* v)
{
    int k = 0;
    double m = fabs(w[0]);
    if (fabs(w[1]) > m) { k = 1; m = fabs(w[1]); }
    if (fabs(w[2]) > m) { k = 2; m = fabs(w[2]); }
    int f = 2 * k + (w[k] < 0.0 ? 1 : 0);
    /* w~ = w / |w_k| puts the face plane at distance 1: u = (w~ . b_f + 1)/2, v likewise. */
    *u = (w[(k + 1) % 3] / m + 1.0) / 2.0;
    *v = (w[(k + 2) % 3] / m + 1.0) / 2.0;
    return f;
}

void shmo_face_frame(int f, double a[3], double b[3], double c[3])
{
    int k = f / 2;
    for (int q = 0; q < 3; ++q) a[q] = b[q] = c[q] = 0.0;
    a[k] = (f % 2) ? -1.0 : 1.0;
    b[(k + 1) % 3] = 1.0;
    c[(k + 2) % 3] = 1.0;
}

void shmo_dir_tilde(int f, double u, double v, double wt[3])
{
    double a[3], b[3], c[3];
    shmo_face_frame(f, a, b, c);
    for (int q = 0; q < 3; ++q) wt[q] = a[q] + (2.0 * u - 1.0) * b[q] + (2.0 * v - 1.0) * c[q];
}

double shmo_texel_centre(int i, int N)
{
    return ((double)i - 0.5) / (double)N;
}

/* §3.4, tangent equation: d w / d xi = (I - w w^T) / |w~| * d w~ / d xi, with d w~/du = 2 b_f and
 * d w~/dv = 2 c_f constant per face. */
void shmo_tangents(int f, double u, double v, double e1[3], double e2[3])
{
    double a[3], b[3], c[3], wt[3], w[3];
    shmo_face_frame(f, a, b, c);
    shmo_dir_tilde(f, u, v, wt);
    double rho = sqrt(wt[0] * wt[0] + wt[1] * wt[1] + wt[2] * wt[2]);
    for (int q = 0; q < 3; ++q) w[q] = wt[q] / rho;
    double dwu[3], dwv[3];
    for (int q = 0; q < 3; ++q) { dwu[q] = 2.0 * b[q]; dwv[q] = 2.0 * c[q]; }
    double wu = w[0] * dwu[0] + w[1] * dwu[1] + w[2] * dwu[2];
    double wv = w[0] * dwv[0] + w[1] * dwv[1] + w[2] * dwv[2];
    for (int q = 0; q < 3; ++q) {
        e1[q] = (dwu[q] - w[q] * wu) / rho;
        e2[q] = (dwv[q] - w[q] * wv) / rho;
    }
}

/* §3.4: g11 = e1.e1, g12 = e1.e2, g22 = e2.e2. */
void shmo_metric(int f, double u, double v, double G[3])
{
    double e1[3], e2[3];
    shmo_tangents(f, u, v, e1, e2);
    G[0] = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    G[1] = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    G[2] = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
}

/* §3.4: grad_{S^2} R = alpha e1 + beta e2 with G [alpha beta]^T = [R_u R_v]^T, solved by Cramer's
 * rule; det G is clamped from below before inversion (the paper gives no threshold: 1e-12). */
void shmo_s2_gradient(int f, double u, double v, double Ru, double Rv, double grad[3])
{
    double e1[3], e2[3];
    shmo_tangents(f, u, v, e1, e2);
    double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    double det = g11 * g22 - g12 * g12;
    if (det < 1e-12) det = 1e-12;
    double alpha = (g22 * Ru - g12 * Rv) / det;
    double beta = (g11 * Rv - g12 * Ru) / det;
    for (int q = 0; q < 3; ++q) grad[q] = alpha * e1[q] + beta * e2[q];
}

/* §3.4: n = (R w - grad R) / |R w - grad R|. */
void shmo_normal(const double w[3], double R, const double grad[3], double n[3])
{
    double m[3];
    for (int q = 0; q < 3; ++q) m[q] = R * w[q] - grad[q];
    double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    for (int q = 0; q < 3; ++q) n[q] = m[q] / len;
}
