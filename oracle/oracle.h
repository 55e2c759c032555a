/*
 * FP64 CPU oracle for Spherical Hermite Maps (Abouagour & Garyfallidis, arXiv 2602.20063).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library against the
 * paper; only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Every function follows the paper step by step in float64, in the paper's notation:
 *   chart.c       §3.2 padded cubemap parameterization; §3.4 tangents, metric G, Cramer, normal
 *   hermite.c     §3.3 Hermite basis, 2-D reconstruction, derivative extraction
 *   sh.c          §3.3 real spherical harmonics and their exact derivatives (hyper-dual numbers)
 *   bake.c        Algorithm 1 (per-face bake): analytic-SH and finite-difference derivative channels
 *   procedural.c  §4.9/§4.10 synthetic radial functions (Gaussian bumps, value-noise fBm)
 *   query.c       the per-direction query: direction -> face/uv -> 2x2 texels -> R, grad, normal
 *   adjoint.c     reverse-mode derivative of the query and of the SH bake (not in the paper)
 *   raycast.c     §3.1 ray / star-shaped-surface intersection with bisection + Newton
 *   mip.c         §4.7 derivative-consistent and naive mip levels
 *   recon.c       §4.2/§4.5 value-only baselines: nearest, bilinear+FD, Catmull-Rom, B-spline
 *
 * Storage: one glyph's table is [6][P][P][4] float64 with P = N+2, texel (i, j) of face f at
 * ((f*P + j)*P + i)*4, channels (r, r_u h, r_v h, r_uv h^2) with h = 1/N (Eq. hermite_storage).
 * A pool of glyphs concatenates such tables; off[g] is the first texel of glyph g.
 * Stored channel 0 may carry an offset: the represented radius is r0[g] + stored value.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py (closed forms,
 * invariants, library special functions, brute force) except where a header comment says
 * "parity unpinned".
 */
#ifndef SHM_ORACLE_H
#define SHM_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------- hyper-dual numbers a + b e1 + c e2 + d e1 e2, e1^2 = e2^2 = 0 (Fike & Alonso 2011) */
typedef struct { double a, b, c, d; } shmo_hd;

/* ---------- chart.c */
int    shmo_face_uv(const double w[3], double* u, double* v);
void   shmo_face_frame(int f, double a[3], double b[3], double c[3]);
void   shmo_dir_tilde(int f, double u, double v, double wt[3]);
double shmo_texel_centre(int i, int N);
void   shmo_tangents(int f, double u, double v, double e1[3], double e2[3]);
void   shmo_metric(int f, double u, double v, double G[3]);  /* g11, g12, g22 */
void   shmo_s2_gradient(int f, double u, double v, double Ru, double Rv, double grad[3]);
void   shmo_normal(const double w[3], double R, const double grad[3], double n[3]);

/* ---------- hermite.c */
void shmo_hermite_basis(double s, double H[4], double dH[4], double ddH[4]);
void shmo_cell(int N, double u, int* i, double* s);
/* out: r, dr/ds, dr/dt, d2r/ds2, d2r/dsdt, d2r/dt2 at local (s,t) of cell (i,j) of one face */
void shmo_hermite_eval(const double* face, int N, int i, int j, double s, double t, double out[6]);
/* Per-corner weights of the 16 stored scalars: w[k][corner ab][ch], k = value, d/ds, d/dt. */
void shmo_hermite_weights(double s, double t, double w[3][4][4]);

/* ---------- sh.c */
int  shmo_sh_count(int L);
void shmo_sh_basis_hd(int L, shmo_hd x, shmo_hd y, shmo_hd z, shmo_hd* Y);
void shmo_sh_basis(int L, const double w[3], double* Y);
void shmo_sh_chart_basis(int L, int f, double u, double v, double* out);
void shmo_sh_chart(int L, const double* coeffs, int f, double u, double v, double out[4]);
void shmo_sh_value_grad(int L, const double* coeffs, const double w[3], double* r, double grad[3]);
void shmo_sh_eval_batch(int L, const double* coeffs, int64_t Q, const float* dirs,
                        const int32_t* glyph, double* R, double* grad, double* normal, int nthreads);

/* ---------- bake.c */
void shmo_bake_sh(int N, int L, const double* coeffs, double* lut);
void shmo_sh_basis_records(int N, int L, double* B);
void shmo_bake_fd(int N, const double* samples, double r0, double* lut);
void shmo_sample_grid_bumps(int N, int nb, const double* mu, const double* amp, const double* width,
                            double* samples);
void shmo_sample_grid_fbm(int N, int octaves, const uint32_t* keys, double base_freq,
                          double lacunarity, double gain, double amplitude, double* samples);
double shmo_lut_bound(const double* glut, int N, double r0);

/* ---------- procedural.c */
double shmo_bumps(const double w[3], int nb, const double* mu, const double* amp, const double* width);
double shmo_value_noise(const double p[3], const uint32_t key[3]);
double shmo_fbm(const double w[3], int octaves, const uint32_t* keys, double base_freq,
                double lacunarity, double gain);
void   shmo_pcg3d(uint32_t v[3]);

/* ---------- query.c */
typedef struct {
    int face, i, j;
    double u, v, s, t;
    double R, Ru, Rv;
    double grad[3], normal[3];
} shmo_query_out;
void shmo_query_one(const double* glut, int N, double r0, const double d[3], shmo_query_out* o);
void shmo_query_batch(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                      int64_t Q, const float* dirs, const int32_t* glyph,
                      double* R, double* grad, double* normal, double* chart, int32_t* fij,
                      int nthreads);

/* ---------- adjoint.c */
void shmo_query_vjp_one(const double* glut, int N, double r0, const double d[3],
                        double gR, const double gG[3], const double gn[3],
                        double* dglut, double dd[3]);
void shmo_query_vjp_batch(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                          int64_t Q, const float* dirs, const int32_t* glyph,
                          const double* gR, const double* gG, const double* gn,
                          double* dpool, double* ddirs);
void shmo_bake_sh_vjp(int N, int L, const double* dlut, double* dcoeffs);

/* ---------- recon.c */
enum { SHMO_RECON_NEAREST = 0, SHMO_RECON_BILINEAR = 1, SHMO_RECON_BICUBIC = 2, SHMO_RECON_FAST_BICUBIC = 3 };
void shmo_catmull_rom(double s, double w[4], double dw[4]);
void shmo_bspline3(double s, double w[4]);
void shmo_recon_one(int method, const double* grid, int N, double r0, const double d[3], shmo_query_out* o);
void shmo_recon_batch(int method, const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                      int64_t Q, const float* dirs, const int32_t* glyph, double* R, double* grad, double* normal,
                      double* chart, int32_t* fij, int nthreads);
void shmo_value_grid_sh(int N, int L, const double* coeffs, double* grid);

/* ---------- mip.c */
void shmo_mip_samples(const double* fine, int Nf, double r0, double* samples);
void shmo_mip_naive(const double* fine, int Nf, double* coarse);

/* ---------- raycast.c */
typedef struct {
    double eye[3], fwd[3], right[3], up[3];
    double tan_half_fov_y;
    int W, H;
} shmo_camera;
typedef struct {
    int march, bisect, newton;
    double ambient, kd, ks, shininess;
    double light[3];
    int lod, bisect_min, newton_min; /* projected-size refinement allocation (§3.1); lod = 0: fixed */
    int recon; /* -1: Hermite tables (pool in records, §3.3); else a SHMO_RECON_* value-only baseline on
                  value grids (pool in scalars, §4.5 equal-storage comparison) */
} shmo_raycast_params;
void shmo_lod_steps(const shmo_camera* cam, const shmo_raycast_params* prm, const double centre[3], double rmax,
                    int* bisect, int* newton, float* p_px);
void shmo_raycast_pixel(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                        int n_obj, const double* centre, const double* scale, const double* rmax,
                        const int32_t* glyph, const shmo_camera* cam, const shmo_raycast_params* prm,
                        int px, int py, double rgba[4], double* depth, double normal[3],
                        int32_t* obj_id, double* margin);
void shmo_raycast_image(const double* pool, const int64_t* off, const int32_t* Ns, const double* r0,
                        int n_obj, const double* centre, const double* scale, const double* rmax,
                        const int32_t* glyph, const shmo_camera* cam, const shmo_raycast_params* prm,
                        int64_t n_px, const int32_t* px, const int32_t* py,
                        double* rgba, double* depth, double* normal, int32_t* obj_id,
                        double* margin, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
