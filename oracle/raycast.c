/*
 * Oracle (test infrastructure only): §3.1 (surface model and ray casting) in float64.
 *
 * Surface x(w) = c + R(w) w with R = s |r| (s > 0 the object scale); implicit
 * F(x) = |x - c| - R(w), w = (x - c)/|x - c|.  Per pixel a view ray p(t) = o + t d is cast;
 * a bounding sphere of radius R_max gives the entry interval [t_min, t_max]; the hit is refined
 * by bisection followed by Newton-Raphson on F(p(t)) = 0.  The paper does not say how the
 * bisection bracket is formed (F >= 0 at both ends of the sphere chord), so this reading is used:
 *   1. march: F at t_k = t_min + (t_max - t_min) k / M, k = 0..M; the first k with F(t_k) < 0
 *      brackets [t_{k-1}, t_k] (F(t_min) < 0 -> hit at t_min); no sign change -> miss;
 *   2. `bisect` halvings keeping F(lo) >= 0 > F(hi);
 *   3. `newton` steps from the bracket midpoint with F' = d . grad F,
 *      grad F(x) = w - grad_{S^2} R / |x - c| (grad_{S^2} R = s sign(r) grad_{S^2} r, sign(0)=+1);
 *      a step that leaves [lo, hi] or meets F' = 0 ends the iteration.
 * The nearest hit over all objects is kept (every object is tested, so the result does not
 * depend on traversal order).  Shading (§4.4 names none): Blinn-Phong with ambient + kd
 * max(n.l, 0) + ks max(n.h, 0)^shininess, white albedo, light direction `light`.
 * `margin` = min |F(t_k)| over all march samples of the pixel: pixels with a small margin may
 * legitimately resolve a different root under a different rounding of F.
 * With prm->recon >= 0 the surface is the value-only baseline reconstruction of recon.c on value
 * grids instead of the Hermite query, everything else unchanged (§4.5 equal-storage renders).
 *
 * Camera: d = normalise(fwd + x_ndc tan(fov_y/2) (W/H) right + y_ndc tan(fov_y/2) up) with
 * x_ndc = 2(px + 1/2)/W - 1 and y_ndc = 1 - 2(py + 1/2)/H.
 *
 * Refinement allocation by projected size (§3.1: more refinement iterations for glyphs that are
 * large on screen; the paper gives no rule).  Reading: projected radius p = R_max (H/2) /
 * (|c - o| tan(fov_y/2)) pixels; bisection steps = the fewest b in [bisect_min, bisect] with
 * M 2^b >= 128 p, i.e. the marched bracket 2 R_max / M shrinks below 1/64 pixel (b = bisect if
 * none does); Newton steps = newton if p >= 64 pixels, else newton_min.  p decides integers, so it is
 * formed in float32, operation by operation in the order written (the device does the same).
 */
#include <math.h>
#include "oracle.h"

typedef struct {
    const double* pool;
    const int64_t* off;
    const int32_t* Ns;
    const double* r0;
    int recon;
} lut_ref;

/* R and its S^2 gradient at direction x of glyph g: the Hermite query (§3.3-§3.4), or for the
 * equal-storage comparison (§4.5) a value-only baseline reconstruction of the glyph's value grid. */
static void eval_surface(const lut_ref* L, int g, const double x[3], shmo_query_out* qo)
{
    double r0 = L->r0 ? L->r0[g] : 0.0;
    if (L->recon >= 0) shmo_recon_one(L->recon, L->pool + (size_t)L->off[g], L->Ns[g], r0, x, qo);
    else shmo_query_one(L->pool + (size_t)L->off[g] * 4, L->Ns[g], r0, x, qo);
}

/* F(p(t)) and dF/dt for one object. */
static void surface_F(const lut_ref* L, int g, double scale, const double c[3], const double o[3],
                      const double d[3], double t, double* F, double* dF, shmo_query_out* qo)
{
    double x[3] = {o[0] + t * d[0] - c[0], o[1] + t * d[1] - c[1], o[2] + t * d[2] - c[2]};
    double dist = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    eval_surface(L, g, x, qo);
    double sg = (qo->R >= 0.0) ? 1.0 : -1.0;
    double R = scale * fabs(qo->R);
    *F = dist - R;
    if (dF) {
        double w[3] = {x[0] / dist, x[1] / dist, x[2] / dist};
        double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
        double dg = d[0] * qo->grad[0] + d[1] * qo->grad[1] + d[2] * qo->grad[2];
        *dF = dw - scale * sg * dg / dist;
    }
}

void shmo_lod_steps(const shmo_camera* cam, const shmo_raycast_params* prm, const double centre[3], double rmax,
                    int* bisect, int* newton, float* p_px)
{
    *bisect = prm->bisect;
    *newton = prm->newton;
    if (!prm->lod) { if (p_px) *p_px = NAN; return; }
    float dx = (float)centre[0] - (float)cam->eye[0];
    float dy = (float)centre[1] - (float)cam->eye[1];
    float dz = (float)centre[2] - (float)cam->eye[2];
    float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    float D = sqrtf((xx + yy) + zz);
    float num = (float)rmax * (0.5f * (float)cam->H);
    float den = D * (float)cam->tan_half_fov_y;
    float p = num / den;
    float need = 128.0f * p;
    for (int b = prm->bisect_min; b <= prm->bisect; ++b) {
        if ((float)prm->march * ldexpf(1.0f, b) >= need) { *bisect = b; break; }
    }
    *newton = (p >= 64.0f) ? prm->newton : prm->newton_min;
    if (p_px) *p_px = p;
}

void shmo_raycast_pixel(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                        int n_obj, const double* centre, const double* scale, const double* rmax,
                        const int32_t* glyph, const shmo_camera* cam, const shmo_raycast_params* prm,
                        int px, int py, double rgba[4], double* depth, double normal[3],
                        int32_t* obj_id, double* margin)
{
    lut_ref L = {pool, off, Ns, r0, prm->recon};
    double aspect = (double)cam->W / (double)cam->H;
    double xn = (2.0 * (px + 0.5) / cam->W - 1.0) * cam->tan_half_fov_y * aspect;
    double yn = (1.0 - 2.0 * (py + 0.5) / cam->H) * cam->tan_half_fov_y;
    double d[3];
    for (int q = 0; q < 3; ++q) d[q] = cam->fwd[q] + xn * cam->right[q] + yn * cam->up[q];
    double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int q = 0; q < 3; ++q) d[q] /= dl;
    const double* o = cam->eye;

    double best_t = INFINITY, mg = INFINITY;
    int best = -1;
    for (int ob = 0; ob < n_obj; ++ob) {
        const double* c = centre + 3 * ob;
        double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
        double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
        double cc = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - rmax[ob] * rmax[ob];
        double disc = b * b - cc;
        if (disc < 0.0) continue;
        double sq = sqrt(disc);
        double t0 = -b - sq, t1 = -b + sq;
        if (t1 <= 0.0) continue;
        if (t0 < 0.0) t0 = 0.0;
        int n_bisect, n_newton;
        shmo_lod_steps(cam, prm, c, rmax[ob], &n_bisect, &n_newton, NULL);
        shmo_query_out qo;
        double F, dF;
        double lo = t0, hi = t0, thit = NAN;
        surface_F(&L, glyph[ob], scale[ob], c, o, d, t0, &F, NULL, &qo);
        if (fabs(F) < mg) mg = fabs(F);
        if (F < 0.0) {
            thit = t0;
        } else {
            int found = 0;
            for (int k = 1; k <= prm->march; ++k) {
                double tk = t0 + (t1 - t0) * (double)k / (double)prm->march;
                surface_F(&L, glyph[ob], scale[ob], c, o, d, tk, &F, NULL, &qo);
                if (fabs(F) < mg) mg = fabs(F);
                if (F < 0.0) {
                    lo = t0 + (t1 - t0) * (double)(k - 1) / (double)prm->march;
                    hi = tk;
                    found = 1;
                    break;
                }
            }
            if (!found) continue;
            for (int it = 0; it < n_bisect; ++it) {
                double mid = 0.5 * (lo + hi);
                surface_F(&L, glyph[ob], scale[ob], c, o, d, mid, &F, NULL, &qo);
                if (F < 0.0) hi = mid; else lo = mid;
            }
            double t = 0.5 * (lo + hi);
            for (int it = 0; it < n_newton; ++it) {
                surface_F(&L, glyph[ob], scale[ob], c, o, d, t, &F, &dF, &qo);
                if (dF == 0.0) break;
                double tn = t - F / dF;
                if (!(tn >= lo && tn <= hi)) break;
                t = tn;
            }
            thit = t;
        }
        if (thit < best_t) {
            best_t = thit;
            best = ob;
        }
    }
    *margin = mg;
    *obj_id = best;
    if (best < 0) {
        *depth = INFINITY;
        for (int q = 0; q < 4; ++q) rgba[q] = 0.0;
        for (int q = 0; q < 3; ++q) normal[q] = 0.0;
        return;
    }
    /* normal of the signed-function surface at the hit (§3.4 with grad R = s sign(r) grad r) */
    const double* c = centre + 3 * best;
    double x[3] = {o[0] + best_t * d[0] - c[0], o[1] + best_t * d[1] - c[1], o[2] + best_t * d[2] - c[2]};
    double dist = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double w[3] = {x[0] / dist, x[1] / dist, x[2] / dist};
    shmo_query_out qo;
    eval_surface(&L, glyph[best], x, &qo);
    double sg = (qo.R >= 0.0) ? 1.0 : -1.0;
    double R = scale[best] * fabs(qo.R);
    double gr[3] = {scale[best] * sg * qo.grad[0], scale[best] * sg * qo.grad[1], scale[best] * sg * qo.grad[2]};
    shmo_normal(w, R, gr, normal);
    *depth = best_t;
    double l[3] = {prm->light[0], prm->light[1], prm->light[2]};
    double ll = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    for (int q = 0; q < 3; ++q) l[q] /= ll;
    double hv[3] = {l[0] - d[0], l[1] - d[1], l[2] - d[2]};
    double hl = sqrt(hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2]);
    for (int q = 0; q < 3; ++q) hv[q] /= hl;
    double ndl = normal[0] * l[0] + normal[1] * l[1] + normal[2] * l[2];
    double ndh = normal[0] * hv[0] + normal[1] * hv[1] + normal[2] * hv[2];
    double I = prm->ambient + prm->kd * (ndl > 0.0 ? ndl : 0.0) +
               prm->ks * (ndh > 0.0 ? pow(ndh, prm->shininess) : 0.0);
    rgba[0] = rgba[1] = rgba[2] = I;
    rgba[3] = 1.0;
}

void shmo_raycast_image(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                        int n_obj, const double* centre, const double* scale, const double* rmax,
                        const int32_t* glyph, const shmo_camera* cam, const shmo_raycast_params* prm,
                        int64_t n_px, const int32_t* px, const int32_t* py,
                        double* rgba, double* depth, double* normal, int32_t* obj_id,
                        double* margin, int nthreads)
{
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (int64_t q = 0; q < n_px; ++q) {
        shmo_raycast_pixel(pool, off, Ns, r0, n_obj, centre, scale, rmax, glyph, cam, prm,
                           px[q], py[q], rgba + 4 * q, depth + q, normal + 3 * q, obj_id + q,
                           margin + q);
    }
}
