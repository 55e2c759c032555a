/*
 * Oracle (test infrastructure only): Algorithm 1 (the per-face bake), §3.3.
 *
 * For every stored texel centre (u_i, v_j) of the padded (N+2)^2 face, gutter included, the
 * record (r, r_u h, r_v h, r_uv h^2) with h = 1/N is stored (Eq. hermite_storage).  Gutter
 * texels are filled by evaluating the function at their own centres in the face's own chart,
 * never by copying or reflecting (§3.2).  Two derivative modes (§3.3):
 *   analytic SH   exact chart derivatives of the SH expansion (sh.c, hyper-dual);
 *   finite diff.  central differences in (u,v) on a sample grid that carries a one-texel
 *                 bake-time margin beyond the gutter (the paper allows a margin or one-sided
 *                 stencils; the margin is this reading):
 *                 r_u h = (r[i+1] - r[i-1]) / 2,  r_v h = (r[j+1] - r[j-1]) / 2,
 *                 r_uv h^2 = (r[i+1,j+1] - r[i+1,j-1] - r[i-1,j+1] + r[i-1,j-1]) / 4.
 * Sample grids are [6][N+4][N+4] with entry (jj, ii) at texel index (ii-1, jj-1), i.e. centres
 * u = (ii - 3/2)/N.  A value offset r0 may be subtracted from channel 0 (r0 + stored = r).
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

void shmo_bake_sh(int N, int L, const double* coeffs, double* lut)
{
    int P = N + 2;
    double h = 1.0 / (double)N;
    for (int f = 0; f < 6; ++f)
        for (int j = 0; j < P; ++j)
            for (int i = 0; i < P; ++i) {
                double out[4];
                shmo_sh_chart(L, coeffs, f, shmo_texel_centre(i, N), shmo_texel_centre(j, N), out);
                double* rec = lut + (((size_t)f * P + j) * P + i) * 4;
                rec[0] = out[0];
                rec[1] = out[1] * h;
                rec[2] = out[2] * h;
                rec[3] = out[3] * h * h;
            }
}

/* B[k][f][j][i][ch]: the record of the k-th basis function alone, i.e. the bake is the linear
 * map lut = sum_k c_k B[k]. */
void shmo_sh_basis_records(int N, int L, double* B)
{
    int K = shmo_sh_count(L);
    size_t T = (size_t)6 * (N + 2) * (N + 2);
    double* e = (double*)calloc((size_t)K, sizeof(double));
    for (int k = 0; k < K; ++k) {
        e[k] = 1.0;
        shmo_bake_sh(N, L, e, B + (size_t)k * T * 4);
        e[k] = 0.0;
    }
    free(e);
}

void shmo_bake_fd(int N, const double* samples, double r0, double* lut)
{
    int P = N + 2, S = N + 4;
    for (int f = 0; f < 6; ++f) {
        const double* g = samples + (size_t)f * S * S;
        for (int j = 0; j < P; ++j)
            for (int i = 0; i < P; ++i) {
                /* texel (i, j) sits at sample (i+1, j+1) */
#define SMP(di, dj) g[(size_t)(j + 1 + (dj)) * S + (size_t)(i + 1 + (di))]
                double* rec = lut + (((size_t)f * P + j) * P + i) * 4;
                rec[0] = SMP(0, 0) - r0;
                rec[1] = (SMP(1, 0) - SMP(-1, 0)) / 2.0;
                rec[2] = (SMP(0, 1) - SMP(0, -1)) / 2.0;
                rec[3] = (SMP(1, 1) - SMP(1, -1) - SMP(-1, 1) + SMP(-1, -1)) / 4.0;
#undef SMP
            }
    }
}

static void sample_dir(int f, int ii, int jj, int N, double w[3])
{
    double wt[3];
    shmo_dir_tilde(f, shmo_texel_centre(ii - 1, N), shmo_texel_centre(jj - 1, N), wt);
    double len = sqrt(wt[0] * wt[0] + wt[1] * wt[1] + wt[2] * wt[2]);
    for (int q = 0; q < 3; ++q) w[q] = wt[q] / len;
}

void shmo_sample_grid_bumps(int N, int nb, const double* mu, const double* amp, const double* width,
                            double* samples)
{
    int S = N + 4;
    for (int f = 0; f < 6; ++f)
        for (int jj = 0; jj < S; ++jj)
            for (int ii = 0; ii < S; ++ii) {
                double w[3];
                sample_dir(f, ii, jj, N, w);
                samples[((size_t)f * S + jj) * S + ii] = shmo_bumps(w, nb, mu, amp, width);
            }
}

/* Planet heightfield samples h(w) = amplitude * fBm(w); the radius is R0 + h with R0 carried as
 * the table's value offset (§4.10: R = R0 + h). */
void shmo_sample_grid_fbm(int N, int octaves, const uint32_t* keys, double base_freq,
                          double lacunarity, double gain, double amplitude, double* samples)
{
    int S = N + 4;
    for (int f = 0; f < 6; ++f)
        for (int jj = 0; jj < S; ++jj)
            for (int ii = 0; ii < S; ++ii) {
                double w[3];
                sample_dir(f, ii, jj, N, w);
                samples[((size_t)f * S + jj) * S + ii] =
                    amplitude * shmo_fbm(w, octaves, keys, base_freq, lacunarity, gain);
            }
}

/* Upper bound of |interpolated r| over the sphere for one glyph table.  On one cell the value
 * weights H_a(s)H_b(t) are non-negative and sum to 1, and sum_a |H^d_a(s)| = s(1-s) <= 1/4, so
 * |r| <= max|r0 + r_ab| + (max|r_u h| + max|r_v h|)/4 + max|r_uv h^2|/16 with the maxima over the
 * cell's four corners; the bound is the largest such cell bound.  Used as the bounding-sphere
 * radius R_max of §3.1 (the paper says only "a bounding sphere"). */
double shmo_lut_bound(const double* glut, int N, double r0)
{
    int P = N + 2;
    double best = 0.0;
    for (int f = 0; f < 6; ++f)
        for (int j = 0; j <= N; ++j)
            for (int i = 0; i <= N; ++i) {
                double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        const double* p = glut + (((size_t)f * P + (j + b)) * P + (i + a)) * 4;
                        if (fabs(r0 + p[0]) > m0) m0 = fabs(r0 + p[0]);
                        if (fabs(p[1]) > m1) m1 = fabs(p[1]);
                        if (fabs(p[2]) > m2) m2 = fabs(p[2]);
                        if (fabs(p[3]) > m3) m3 = fabs(p[3]);
                    }
                double cb = m0 + (m1 + m2) / 4.0 + m3 / 16.0;
                if (cb > best) best = cb;
            }
    return best;
}
