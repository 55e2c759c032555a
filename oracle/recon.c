/*
 * Oracle (test infrastructure only): value-only reconstruction baselines on the same padded
 * cubemap chart (§4.2 Table psnr_value, §4.5 Table cost_extended), in float64.
 *
 * Value table: one scalar per texel with a two-texel gutter, [6][N+4][N+4], entry (ii, jj) =
 * texel (ii-1, jj-1) of the face, texel i at u_i = (i - 1/2)/N, i = -1 .. N+2, every entry
 * evaluated at its own centre in the face's chart (the gutter rule of Algorithm 1, widened
 * because a 4 x 4 footprint needs texels i-1 .. i+2).  The grid coincides with the sample grid
 * of the finite-difference bake.  x = uN + 1/2 puts texel i at x = i.
 *
 * Methods:
 *   nearest       the interior texel whose square contains (u, v); no gradient (R_u = R_v = 0)
 *   bilinear+FD   tensor linear interpolation in (x, y); chart derivatives by central
 *                 differences of the bilinear value at u +- h, v +- h, h = 1/N (4 more lookups)
 *   bicubic       16-tap tensor Catmull-Rom (interpolating, Keys a = -1/2) with the analytic
 *                 chart gradient of the same polynomial
 *   fast bicubic  the tensor cubic B-spline that GPU Gems 2 (ch. 20) evaluates with 4 bilinear
 *                 fetches, written here as its 16-tap definition; chart derivatives by central
 *                 differences of its value at u +- h, v +- h
 * The chart derivatives then go through the same S^2 gradient and normal as the Hermite query.
 * Cell index clamps keep each footprint inside the table: [-1, N+1] for the 2-tap rule and
 * [0, N] for the 4-tap rules (the local coordinate then extends the nearest cell's polynomial).
 */
#include <math.h>
#include "oracle.h"

static double vt(const double* face, int N, int i, int j)
{
    const int S = N + 4;
    return face[(size_t)(j + 1) * S + (size_t)(i + 1)];
}

static void cell_clamped(int N, double u, int lo, int hi, int* i, double* s)
{
    double x = u * N + 0.5;
    int k = (int)floor(x);
    if (k < lo) k = lo;
    if (k > hi) k = hi;
    *i = k;
    *s = x - k;
}

/* Catmull-Rom weights of taps i-1, i, i+1, i+2 and their s-derivatives */
void shmo_catmull_rom(double s, double w[4], double dw[4])
{
    double s2 = s * s, s3 = s2 * s;
    w[0] = 0.5 * (-s3 + 2.0 * s2 - s);
    w[1] = 0.5 * (3.0 * s3 - 5.0 * s2 + 2.0);
    w[2] = 0.5 * (-3.0 * s3 + 4.0 * s2 + s);
    w[3] = 0.5 * (s3 - s2);
    dw[0] = 0.5 * (-3.0 * s2 + 4.0 * s - 1.0);
    dw[1] = 0.5 * (9.0 * s2 - 10.0 * s);
    dw[2] = 0.5 * (-9.0 * s2 + 8.0 * s + 1.0);
    dw[3] = 0.5 * (3.0 * s2 - 2.0 * s);
}

/* uniform cubic B-spline weights of taps i-1, i, i+1, i+2 */
void shmo_bspline3(double s, double w[4])
{
    double r = 1.0 - s;
    w[0] = r * r * r / 6.0;
    w[1] = (3.0 * s * s * s - 6.0 * s * s + 4.0) / 6.0;
    w[2] = (-3.0 * s * s * s + 3.0 * s * s + 3.0 * s + 1.0) / 6.0;
    w[3] = s * s * s / 6.0;
}

static double bilinear(const double* face, int N, double u, double v)
{
    int i, j;
    double s, t;
    cell_clamped(N, u, -1, N + 1, &i, &s);
    cell_clamped(N, v, -1, N + 1, &j, &t);
    return (1.0 - s) * (1.0 - t) * vt(face, N, i, j) + s * (1.0 - t) * vt(face, N, i + 1, j) +
           (1.0 - s) * t * vt(face, N, i, j + 1) + s * t * vt(face, N, i + 1, j + 1);
}

static double tensor4(const double* face, int N, int i, int j, const double wu[4], const double wv[4])
{
    double acc = 0.0;
    for (int b = 0; b < 4; ++b) {
        double row = 0.0;
        for (int a = 0; a < 4; ++a) row += wu[a] * vt(face, N, i - 1 + a, j - 1 + b);
        acc += wv[b] * row;
    }
    return acc;
}

static double bspline_value(const double* face, int N, double u, double v)
{
    int i, j;
    double s, t, wu[4], wv[4];
    cell_clamped(N, u, 0, N, &i, &s);
    cell_clamped(N, v, 0, N, &j, &t);
    shmo_bspline3(s, wu);
    shmo_bspline3(t, wv);
    return tensor4(face, N, i, j, wu, wv);
}

void shmo_recon_one(int method, const double* grid, int N, double r0, const double d[3], shmo_query_out* o)
{
    const int S = N + 4;
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double w[3] = {d[0] / len, d[1] / len, d[2] / len};
    o->face = shmo_face_uv(d, &o->u, &o->v);
    const double* face = grid + (size_t)o->face * S * S;
    const double h = 1.0 / N;
    double r = 0.0, ru = 0.0, rv = 0.0;
    o->s = o->t = 0.0;
    switch (method) {
    case SHMO_RECON_NEAREST: {
        int i = (int)floor(o->u * N) + 1, j = (int)floor(o->v * N) + 1;
        if (i < 1) i = 1;
        if (i > N) i = N;
        if (j < 1) j = 1;
        if (j > N) j = N;
        o->i = i;
        o->j = j;
        r = vt(face, N, i, j);
        break;
    }
    case SHMO_RECON_BILINEAR:
        cell_clamped(N, o->u, -1, N + 1, &o->i, &o->s);
        cell_clamped(N, o->v, -1, N + 1, &o->j, &o->t);
        r = bilinear(face, N, o->u, o->v);
        ru = (bilinear(face, N, o->u + h, o->v) - bilinear(face, N, o->u - h, o->v)) / (2.0 * h);
        rv = (bilinear(face, N, o->u, o->v + h) - bilinear(face, N, o->u, o->v - h)) / (2.0 * h);
        break;
    case SHMO_RECON_BICUBIC: {
        double wu[4], dwu[4], wv[4], dwv[4];
        cell_clamped(N, o->u, 0, N, &o->i, &o->s);
        cell_clamped(N, o->v, 0, N, &o->j, &o->t);
        shmo_catmull_rom(o->s, wu, dwu);
        shmo_catmull_rom(o->t, wv, dwv);
        r = tensor4(face, N, o->i, o->j, wu, wv);
        ru = N * tensor4(face, N, o->i, o->j, dwu, wv);  /* dx/du = N */
        rv = N * tensor4(face, N, o->i, o->j, wu, dwv);
        break;
    }
    default: /* SHMO_RECON_FAST_BICUBIC */
        cell_clamped(N, o->u, 0, N, &o->i, &o->s);
        cell_clamped(N, o->v, 0, N, &o->j, &o->t);
        r = bspline_value(face, N, o->u, o->v);
        ru = (bspline_value(face, N, o->u + h, o->v) - bspline_value(face, N, o->u - h, o->v)) / (2.0 * h);
        rv = (bspline_value(face, N, o->u, o->v + h) - bspline_value(face, N, o->u, o->v - h)) / (2.0 * h);
        break;
    }
    o->R = r0 + r;
    o->Ru = ru;
    o->Rv = rv;
    shmo_s2_gradient(o->face, o->u, o->v, ru, rv, o->grad);
    shmo_normal(w, o->R, o->grad, o->normal);
}

void shmo_recon_batch(int method, const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                      int64_t Q, const float* dirs, const int32_t* glyph, double* R, double* grad, double* normal,
                      double* chart, int32_t* fij, int nthreads)
{
#pragma omp parallel for schedule(static, 1024) num_threads(nthreads)
    for (int64_t q = 0; q < Q; ++q) {
        int g = glyph ? glyph[q] : 0;
        double d[3] = {dirs[3 * q], dirs[3 * q + 1], dirs[3 * q + 2]};
        shmo_query_out o;
        shmo_recon_one(method, pool + off[g], Ns[g], r0 ? r0[g] : 0.0, d, &o);
        if (R) R[q] = o.R;
        if (grad) for (int k = 0; k < 3; ++k) grad[3 * q + k] = o.grad[k];
        if (normal) for (int k = 0; k < 3; ++k) normal[3 * q + k] = o.normal[k];
        if (chart) { chart[2 * q] = o.Ru; chart[2 * q + 1] = o.Rv; }
        if (fij) { fij[3 * q] = o.face; fij[3 * q + 1] = o.i; fij[3 * q + 2] = o.j; }
    }
}

/* Value table of an SH function: r at every texel centre of the two-texel-gutter grid. */
void shmo_value_grid_sh(int N, int L, const double* coeffs, double* grid)
{
    int S = N + 4;
    for (int f = 0; f < 6; ++f)
        for (int jj = 0; jj < S; ++jj)
            for (int ii = 0; ii < S; ++ii) {
                double wt[3], g[3], r;
                shmo_dir_tilde(f, shmo_texel_centre(ii - 1, N), shmo_texel_centre(jj - 1, N), wt);
                double len = sqrt(wt[0] * wt[0] + wt[1] * wt[1] + wt[2] * wt[2]);
                double w[3] = {wt[0] / len, wt[1] / len, wt[2] / len};
                shmo_sh_value_grad(L, coeffs, w, &r, g);
                grid[((size_t)f * S + jj) * S + ii] = r;
            }
}
