/*
 * Oracle (test infrastructure only): real spherical harmonics with exact chart derivatives.
 *
 * §3.3 (analytic SH derivatives): r(w) = sum_{l,m} c_l^m Y_l^m(w); derivatives of the SH
 * expansion are exact, and are converted to face-chart (u,v) derivatives by the chain rule.
 * The paper fixes neither normalisation, phase nor indexing.  Reading used here:
 *   orthonormal real SH on S^2, coefficient index k = l*l + l + m, no Condon-Shortley phase,
 *   Y_l^0  = K_l0 Qbar_l^0(z),
 *   Y_l^m  = sqrt(2) K_lm Qbar_l^m(z) C_m(x,y),   Y_l^-m = sqrt(2) K_lm Qbar_l^m(z) S_m(x,y)  (m>0),
 *   K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),  C_m + i S_m = (x + i y)^m,
 *   Qbar_l^m(z) = d^m P_l / dz^m  (the associated Legendre function divided by sin^m theta),
 * so every Y is a polynomial in the Cartesian components (x, y, z) of the unit direction.
 * The chart derivatives r_u, r_v and the mixed r_uv are obtained exactly, with no step size,
 * by evaluating that polynomial on hyper-dual numbers (Fike & Alonso, AIAA 2011-886) carried
 * through w~(u,v) = a + (2u-1) b + (2v-1) c and the normalisation w = w~/|w~|.  The paper only
 * says "analytic derivatives + chain rule" for r_uv; the hyper-dual route is this reading.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

static shmo_hd hd_const(double a) { shmo_hd r = {a, 0.0, 0.0, 0.0}; return r; }
static shmo_hd hd_add(shmo_hd x, shmo_hd y) { shmo_hd r = {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; return r; }
static shmo_hd hd_sub(shmo_hd x, shmo_hd y) { shmo_hd r = {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; return r; }
static shmo_hd hd_scale(shmo_hd x, double k) { shmo_hd r = {k * x.a, k * x.b, k * x.c, k * x.d}; return r; }
static shmo_hd hd_mul(shmo_hd x, shmo_hd y)
{
    shmo_hd r = {x.a * y.a,
                 x.a * y.b + x.b * y.a,
                 x.a * y.c + x.c * y.a,
                 x.a * y.d + x.b * y.c + x.c * y.b + x.d * y.a};
    return r;
}
/* f(x) for a scalar function with value f, derivative df, second derivative d2f at x.a */
static shmo_hd hd_apply(shmo_hd x, double f, double df, double d2f)
{
    shmo_hd r = {f, df * x.b, df * x.c, df * x.d + d2f * x.b * x.c};
    return r;
}
static shmo_hd hd_rsqrt(shmo_hd x)
{
    double f = 1.0 / sqrt(x.a);
    return hd_apply(x, f, -0.5 * f / x.a, 0.75 * f / (x.a * x.a));
}

int shmo_sh_count(int L) { return (L + 1) * (L + 1); }

static double norm_K(int l, int m)
{
    /* (l-m)!/(l+m)! as a product, then K_lm */
    double ratio = 1.0;
    for (int q = l - m + 1; q <= l + m; ++q) ratio /= (double)q;
    return sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio);
}

void shmo_sh_basis_hd(int L, shmo_hd x, shmo_hd y, shmo_hd z, shmo_hd* Y)
{
    shmo_hd* C = (shmo_hd*)malloc(sizeof(shmo_hd) * (size_t)(L + 1));
    shmo_hd* S = (shmo_hd*)malloc(sizeof(shmo_hd) * (size_t)(L + 1));
    shmo_hd* Qb = (shmo_hd*)malloc(sizeof(shmo_hd) * (size_t)(L + 1));
    C[0] = hd_const(1.0);
    S[0] = hd_const(0.0);
    for (int m = 1; m <= L; ++m) {
        /* (x + i y)^m = (x + i y)(C_{m-1} + i S_{m-1}) */
        C[m] = hd_sub(hd_mul(x, C[m - 1]), hd_mul(y, S[m - 1]));
        S[m] = hd_add(hd_mul(x, S[m - 1]), hd_mul(y, C[m - 1]));
    }
    for (int m = 0; m <= L; ++m) {
        /* Qbar_m^m = (2m-1)!!;  Qbar_{m+1}^m = (2m+1) z Qbar_m^m;
         * (l-m) Qbar_l^m = (2l-1) z Qbar_{l-1}^m - (l+m-1) Qbar_{l-2}^m. */
        double dfact = 1.0;
        for (int q = 1; q <= m; ++q) dfact *= (double)(2 * q - 1);
        for (int l = m; l <= L; ++l) {
            if (l == m) {
                Qb[l] = hd_const(dfact);
            } else if (l == m + 1) {
                Qb[l] = hd_scale(hd_mul(z, Qb[l - 1]), (double)(2 * m + 1));
            } else {
                shmo_hd t1 = hd_scale(hd_mul(z, Qb[l - 1]), (double)(2 * l - 1));
                shmo_hd t2 = hd_scale(Qb[l - 2], (double)(l + m - 1));
                Qb[l] = hd_scale(hd_sub(t1, t2), 1.0 / (double)(l - m));
            }
            double K = norm_K(l, m);
            if (m == 0) {
                Y[l * l + l] = hd_scale(Qb[l], K);
            } else {
                Y[l * l + l + m] = hd_scale(hd_mul(Qb[l], C[m]), sqrt(2.0) * K);
                Y[l * l + l - m] = hd_scale(hd_mul(Qb[l], S[m]), sqrt(2.0) * K);
            }
        }
    }
    free(C);
    free(S);
    free(Qb);
}

void shmo_sh_basis(int L, const double w[3], double* Y)
{
    int K = shmo_sh_count(L);
    shmo_hd* Yh = (shmo_hd*)malloc(sizeof(shmo_hd) * (size_t)K);
    double len = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    shmo_sh_basis_hd(L, hd_const(w[0] / len), hd_const(w[1] / len), hd_const(w[2] / len), Yh);
    for (int k = 0; k < K; ++k) Y[k] = Yh[k].a;
    free(Yh);
}

/* Per basis function k: (Y_k, dY_k/du, dY_k/dv, d2Y_k/dudv) of Y_k(w~(u,v)/|w~(u,v)|) on face f,
 * exactly (hyper-dual in (u, v)).  out is [K][4]. */
void shmo_sh_chart_basis(int L, int f, double u, double v, double* out)
{
    double a[3], b[3], c[3];
    shmo_face_frame(f, a, b, c);
    shmo_hd U = {u, 1.0, 0.0, 0.0};
    shmo_hd V = {v, 0.0, 1.0, 0.0};
    shmo_hd xu = hd_sub(hd_scale(U, 2.0), hd_const(1.0));
    shmo_hd yv = hd_sub(hd_scale(V, 2.0), hd_const(1.0));
    shmo_hd wt[3];
    for (int q = 0; q < 3; ++q)
        wt[q] = hd_add(hd_add(hd_const(a[q]), hd_scale(xu, b[q])), hd_scale(yv, c[q]));
    shmo_hd rho2 = hd_add(hd_add(hd_mul(wt[0], wt[0]), hd_mul(wt[1], wt[1])), hd_mul(wt[2], wt[2]));
    shmo_hd inv = hd_rsqrt(rho2);
    shmo_hd w[3];
    for (int q = 0; q < 3; ++q) w[q] = hd_mul(wt[q], inv);
    int K = shmo_sh_count(L);
    shmo_hd* Y = (shmo_hd*)malloc(sizeof(shmo_hd) * (size_t)K);
    shmo_sh_basis_hd(L, w[0], w[1], w[2], Y);
    for (int k = 0; k < K; ++k) {
        out[4 * k + 0] = Y[k].a;
        out[4 * k + 1] = Y[k].b;
        out[4 * k + 2] = Y[k].c;
        out[4 * k + 3] = Y[k].d;
    }
    free(Y);
}

/* r, r_u, r_v, r_uv of r(w~(u,v)/|w~(u,v)|) = sum_k c_k Y_k on face f, exactly. */
void shmo_sh_chart(int L, const double* coeffs, int f, double u, double v, double out[4])
{
    int K = shmo_sh_count(L);
    double* Yk = (double*)malloc(sizeof(double) * 4 * (size_t)K);
    shmo_sh_chart_basis(L, f, u, v, Yk);
    for (int q = 0; q < 4; ++q) out[q] = 0.0;
    for (int k = 0; k < K; ++k)
        for (int q = 0; q < 4; ++q) out[q] += coeffs[k] * Yk[4 * k + q];
    free(Yk);
}

/* Direct SH value and S^2 gradient at w: chart derivatives on w's own face, then the metric
 * solve of §3.4 (grad lies in the tangent plane and is independent of the chart used). */
void shmo_sh_value_grad(int L, const double* coeffs, const double w[3], double* r, double grad[3])
{
    double u, v, out[4];
    int f = shmo_face_uv(w, &u, &v);
    shmo_sh_chart(L, coeffs, f, u, v, out);
    *r = out[0];
    if (grad) shmo_s2_gradient(f, u, v, out[1], out[2], grad);
}

void shmo_sh_eval_batch(int L, const double* coeffs, int64_t Q, const float* dirs,
                        const int32_t* glyph, double* R, double* grad, double* normal, int nthreads)
{
    int K = shmo_sh_count(L);
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (int64_t q = 0; q < Q; ++q) {
        double d[3] = {dirs[3 * q], dirs[3 * q + 1], dirs[3 * q + 2]};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double w[3] = {d[0] / len, d[1] / len, d[2] / len};
        const double* c = coeffs + (size_t)(glyph ? glyph[q] : 0) * (size_t)K;
        double r, g[3];
        shmo_sh_value_grad(L, c, w, &r, g);
        if (R) R[q] = r;
        if (grad) for (int k = 0; k < 3; ++k) grad[3 * q + k] = g[k];
        if (normal) {
            double n[3];
            shmo_normal(w, r, g, n);
            for (int k = 0; k < 3; ++k) normal[3 * q + k] = n[k];
        }
    }
}
