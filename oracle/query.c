/*
 * Oracle (test infrastructure only): one Spherical Hermite Map query in float64.
 *
 * Steps, in the paper's order:
 *   §3.2  direction -> face f and chart (u, v)                        (chart.c)
 *   §3.2  cell (i, j) and local (s, t) between cell-centred texels     (hermite.c)
 *   §3.3  2x2 texel fetch, Hermite value r and chart derivatives       (hermite.c)
 *         R = r0 + r,  R_u = (1/h) dr/ds,  R_v = (1/h) dr/dt
 *   §3.4  tangents e1, e2, metric G, Cramer solve -> grad_{S^2} R      (chart.c)
 *   §3.4  normal n = (R w - grad R)/|R w - grad R|                      (chart.c)
 * The face is chosen from the raw input components (exact comparisons); w = d/|d| is used for
 * the normal.  Queries of the raw function r (scale 1, no |r|); the signed-function rule of
 * §3.1/§3.4 is applied by the ray caster.
 */
#include <math.h>
#include "oracle.h"

void shmo_query_one(const double* glut, int N, double r0, const double d[3], shmo_query_out* o)
{
    int P = N + 2;
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double w[3] = {d[0] / len, d[1] / len, d[2] / len};
    o->face = shmo_face_uv(d, &o->u, &o->v);
    shmo_cell(N, o->u, &o->i, &o->s);
    shmo_cell(N, o->v, &o->j, &o->t);
    double out[6];
    shmo_hermite_eval(glut + (size_t)o->face * P * P * 4, N, o->i, o->j, o->s, o->t, out);
    o->R = r0 + out[0];
    o->Ru = (double)N * out[1];
    o->Rv = (double)N * out[2];
    shmo_s2_gradient(o->face, o->u, o->v, o->Ru, o->Rv, o->grad);
    shmo_normal(w, o->R, o->grad, o->normal);
}

void shmo_query_batch(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                      int64_t Q, const float* dirs, const int32_t* glyph,
                      double* R, double* grad, double* normal, double* chart, int32_t* fij,
                      int nthreads)
{
#pragma omp parallel for schedule(static, 1024) num_threads(nthreads)
    for (int64_t q = 0; q < Q; ++q) {
        int g = glyph ? glyph[q] : 0;
        double d[3] = {dirs[3 * q], dirs[3 * q + 1], dirs[3 * q + 2]};
        shmo_query_out o;
        shmo_query_one(pool + (size_t)off[g] * 4, Ns[g], r0 ? r0[g] : 0.0, d, &o);
        if (R) R[q] = o.R;
        if (grad) for (int k = 0; k < 3; ++k) grad[3 * q + k] = o.grad[k];
        if (normal) for (int k = 0; k < 3; ++k) normal[3 * q + k] = o.normal[k];
        if (chart) { chart[2 * q] = o.Ru; chart[2 * q + 1] = o.Rv; }
        if (fij) { fij[3 * q] = o.face; fij[3 * q + 1] = o.i; fij[3 * q + 2] = o.j; }
    }
}
