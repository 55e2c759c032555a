/*
 * shm.h -- C ABI of the GB300 (sm_103a) Spherical Hermite Map library, libshm.so.
 *
 * Spherical Hermite Maps (Abouagour & Garyfallidis, arXiv 2602.20063) store, per texel of a
 * padded cubemap, a radial function's value and scaled chart derivatives
 * (r, r_u h, r_v h, r_uv h^2), h = 1/N (§3.3, Eq. hermite_storage), and reconstruct value and
 * gradient together from a 2x2 texel footprint by bicubic Hermite interpolation (§3.3), from
 * which the S^2 gradient and the surface normal follow (§3.4).
 *
 * Conventions (every entry point):
 *   - All array pointers are DEVICE pointers owned by the caller, unless a comment says host.
 *     The library allocates no device memory and keeps no state between calls, except the
 *     static workspace of shm_raycast_noalloc and the launch-shape table of shm_tune_query
 *     (both described there).
 *   - Per-query buffers of shm_query, shm_query_recon, shm_tune_query, shm_query_backward and
 *     shm_fit_backward (directions, glyph ids, segments, outputs, upstream gradients, targets,
 *     loss, dev_status) may instead be page-locked host memory (cudaHostAlloc / cudaHostRegister):
 *     the kernels read and write it directly over the host link through its device alias, so no
 *     staging copy is needed.  Pageable host memory there gives SHM_ERR_INVALID_ARG.  Tables,
 *     coefficients and workspaces are device memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *     The returned status covers host-side argument validation and launch errors only.
 *   - Conditions found on the device never trap: they are OR-ed into *dev_status (device
 *     int32, may be NULL) as SHM_DEV_* bits and the affected outputs are NaN.
 *   - Directions need not be unit length; zero or non-finite directions give NaN outputs
 *     and SHM_DEV_NONFINITE.
 *   - Chart (paper §3.2 leaves it open): axis k = argmax |w_k| (ties -> lowest k),
 *     face f = 2k + (w_k < 0), b_f = e_{(k+1)%3}, c_f = e_{(k+2)%3}, u = (w_{k+1}/|w_k| + 1)/2,
 *     v = (w_{k+2}/|w_k| + 1)/2; texel centres u_i = (i - 1/2)/N for i = 0..N+1 (gutter at 0 and
 *     N+1, §3.2).  Face table [f][j][i], channel innermost.
 */
#ifndef SHM_H
#define SHM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* shm_stream; /* same type as cudaStream_t */

typedef enum {
    SHM_OK = 0,
    SHM_ERR_INVALID_ARG = 1, /* a pointer, size or enum argument is invalid */
    SHM_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. a dtype/layout pair) */
    SHM_ERR_WORKSPACE = 3,   /* workspace missing or smaller than the *_workspace_bytes figure */
    SHM_ERR_CUDA = 4,        /* a CUDA launch or runtime call failed */
    SHM_ERR_TIMEOUT = 5      /* reserved for bounded device waits */
} shm_status;

/* Bits OR-ed into *dev_status by device code. */
#define SHM_DEV_NONFINITE 1 /* zero / non-finite direction or non-finite coefficient met */
#define SHM_DEV_BOUNDS 2    /* glyph / object index out of range; that item was skipped (NaN) */
#define SHM_DEV_TIMEOUT 4   /* a bounded device wait gave up */

typedef enum { SHM_F32 = 0, SHM_F16 = 1, SHM_BF16 = 2 } shm_dtype;

/* Record layout of a table pool.
 *   SHM_LAYOUT_TEXEL: one record per texel, [6][P][P] records per glyph, P = N+2 (the paper's
 *                     RGBA face texture).  Record = 4 channels (16 B f32, 8 B 16-bit).
 *   SHM_LAYOUT_CELL:  one record per interpolation cell, [6][N+1][N+1] records per glyph; a
 *                     cell record holds its 2x2 corner texels (i,j),(i+1,j),(i,j+1),(i+1,j+1)
 *                     back to back (64 B f32, 32 B 16-bit), so a query reads one aligned
 *                     64 B / 32 B block.  Same values, 4x the bytes of the texel layout. */
/*   SHM_LAYOUT_VALUE: a value-only table for the reconstruction baselines of shm_query_recon
 *                     (§4.2, §4.5): one scalar per texel (4 B f32, 2 B 16-bit), [6][N+4][N+4]
 *                     per glyph with a two-texel gutter, entry (ii, jj) = texel (ii-1, jj-1),
 *                     i = -1 .. N+2, each evaluated at its own centre in the face's chart (a
 *                     4 x 4 footprint needs texels i-1 .. i+2).  Not accepted by shm_query. */
typedef enum { SHM_LAYOUT_TEXEL = 0, SHM_LAYOUT_CELL = 1, SHM_LAYOUT_VALUE = 2 } shm_layout;

/* A pool of per-glyph tables.  Represented radius = r0[g] + stored channel 0.
 * If N_uniform > 0 every glyph has interior resolution N_uniform and glyph g starts at record
 * g * shm_records_per_glyph(N_uniform, layout); N and offset may then be NULL.  Otherwise N[g]
 * and offset[g] (in records of `layout`) describe glyph g. */
typedef struct {
    int32_t n_glyphs;
    int32_t dtype;        /* shm_dtype */
    int32_t layout;       /* shm_layout */
    int32_t N_uniform;    /* > 0: uniform resolution; 0: per-glyph N[] / offset[] */
    const int32_t* N;     /* device [n_glyphs] interior resolution, N >= 1 */
    const int64_t* offset;/* device [n_glyphs] first record of each glyph */
    const float* r0;      /* device [n_glyphs] value offset, or NULL (= 0) */
    void* data;           /* device record pool, 16-byte aligned (32-byte for SHM_LAYOUT_CELL) */
} shm_lut;

/* ---------------------------------------------------------------- sizes (host only) */

/* Records one glyph of resolution N occupies in `layout`: 6(N+2)^2, 6(N+1)^2 or 6(N+4)^2. */
int64_t shm_records_per_glyph(int32_t N, int32_t layout);

/* Bytes of one record: 4 channels x 4 B (f32) or 2 B (16-bit), x 4 for the cell layout, one
 * channel for the value layout. */
int64_t shm_record_bytes(int32_t dtype, int32_t layout);

/* Host: fills offset_host[G] (records) for the per-glyph resolutions N_host[G] and returns
 * the pool size in bytes in *bytes.  Either output may be NULL. */
shm_status shm_lut_layout(int32_t G, const int32_t* N_host, int32_t dtype, int32_t layout,
                          int64_t* offset_host, int64_t* bytes);

/* ---------------------------------------------------------------- query (§3.2-§3.4) */

/* Evaluates Q queries.  Query q reads direction dirs[q] (float32 [Q][3], AoS) on glyph
 *   glyph[q]                       if glyph != NULL (int32 [Q]);
 *   g with seg[g] <= q < seg[g+1]  if seg != NULL (int64 [n_glyphs+1], CSR, non-decreasing);
 *   0                              otherwise.
 * Per query (§3.2 chart and cell, §3.3 Hermite reconstruction and derivative extraction,
 * §3.4 metric-tensor transport and normal):
 *   R        = r0 + r(s,t)                                  -> R[q]            (float32 [Q])
 *   R_u, R_v = (1/h) dr/ds, (1/h) dr/dt                     -> chart[2q..2q+1] (float32 [Q][2])
 *   grad     = alpha e1 + beta e2 with G [alpha beta] = [R_u R_v] (§3.4) -> grad[3q..] ([Q][3])
 *   normal   = (R w - grad) / |R w - grad|, w = d/|d|       -> normal[3q..]    ([Q][3])
 *   fij      = (face, i, j) of the 2x2 footprint            -> fij[3q..]       (int32 [Q][3])
 * Any output pointer may be NULL to skip it.  Inputs are read-only; outputs are overwritten.
 * Returns SHM_ERR_INVALID_ARG for a NULL lut/dirs, Q < 0, or an invalid dtype/layout. */
shm_status shm_query(const shm_lut* lut, int64_t Q, const float* dirs, const int32_t* glyph,
                     const int64_t* seg, float* R, float* grad, float* normal, float* chart,
                     int32_t* fij, int32_t* dev_status, shm_stream stream);

/* Launch-shape autotuning of shm_query (no counterpart in the paper).  Times every launch shape
 * of the kernel that shm_query would use for these arguments -- for per-glyph segments on small
 * uniform tables the shared-memory staged kernel (threads per CTA 512 / 1,024 / 256), otherwise
 * the per-query kernel ((threads per CTA, rounds per CTA chunk) = (512, 8), (256, 16), (1024, 4),
 * (256, 8)) -- `reps` times each on `stream` (writing the outputs), and records the fastest for
 * the current device, that path, dtype and layout; later shm_query calls use it.  Results do not
 * depend on the shape (same arithmetic per query).  Synchronises `stream`; not for use while a
 * CUDA graph is being captured.  *chosen (host, may be NULL) receives the shape index,
 * times_ms (host [SHM_TUNE_MAX_SHAPES], may be NULL) the mean time per shape (-1 = not tried).
 * The table is process-wide; shm_tune_reset() restores the defaults (shape 0). */
#define SHM_TUNE_MAX_SHAPES 4
shm_status shm_tune_query(const shm_lut* lut, int64_t Q, const float* dirs, const int32_t* glyph,
                          const int64_t* seg, float* R, float* grad, float* normal, int32_t reps,
                          int32_t* chosen, float* times_ms, shm_stream stream);
shm_status shm_tune_reset(void);

/* Binned query of one large table in random order (no counterpart in the paper, whose fragment
 * shader reads each footprint through the texture cache; the workload is the procedural planet of
 * §4.10 queried at uniformly random directions).  Same per-query results as shm_query with
 * glyph = seg = NULL (every query on glyph 0): R [Q], grad [Q][3], normal [Q][3] and the chart
 * derivatives chart [Q][2] (R_u, R_v), each may be NULL, in query order, bit-identical to
 * shm_query's.  Work: the queries are partitioned by the table region their 2x2 footprint reads
 * -- face and band of cell rows, a band holding about band_bytes of records (0 = 32 MiB) -- the
 * query runs over the partitioned batch so that the bands in flight stay resident in L2, and the
 * results return to query order.  The partition is stable and computed on the device; nothing is
 * synchronised with the host.
 *   - lut: any dtype, texel or cell layout, uniform resolution (N_uniform > 0, else
 *     SHM_ERR_UNSUPPORTED); only glyph 0 is read.
 *   - ws: device workspace of at least shm_query_binned_workspace_bytes(lut, Q, band_bytes)
 *     (about 25 B per query: the partitioned directions, intermediate R / R_u / R_v, one bin byte
 *     per query and per-tile counts), else SHM_ERR_WORKSPACE.  Its contents need no clearing and
 *     are scratch after the call; two calls that overlap on the GPU must not share it.
 *   - dirs and the outputs follow shm_query's rules (device or page-locked host memory); the
 *     directions are read three times, so device memory is the fast case.
 *   - band_bytes < 0 or Q < 0: SHM_ERR_INVALID_ARG. */
int64_t shm_query_binned_workspace_bytes(const shm_lut* lut, int64_t Q, int64_t band_bytes);
/* Bins (6 faces x bands) the partition uses for (lut, band_bytes); *band_rows (host, may be NULL)
 * receives the cell rows per band.  -1 for an unsupported table. */
int32_t shm_query_binned_bins(const shm_lut* lut, int64_t band_bytes, int32_t* band_rows);
shm_status shm_query_binned(const shm_lut* lut, int64_t Q, const float* dirs, float* R, float* grad,
                            float* normal, float* chart, int64_t band_bytes, void* ws, size_t ws_bytes,
                            int32_t* dev_status, shm_stream stream);

/* Value-only reconstruction baselines (§4.2 Table psnr_value, §4.5 Table cost_extended) on a
 * SHM_LAYOUT_VALUE table, with the chart, glyph selection, outputs and status rules of shm_query.
 * With x = uN + 1/2 (texel i at x = i) and (i, s) the cell of x as in shm_query:
 *   SHM_RECON_NEAREST       value of the interior texel whose square holds (u, v); R_u = R_v = 0
 *   SHM_RECON_BILINEAR      bilinear value; R_u, R_v by central differences of the bilinear value
 *                           one texel to either side (u +- h, v +- h), 5 bilinear lookups in all
 *   SHM_RECON_BICUBIC       16-tap Catmull-Rom (interpolating) value and its analytic gradient
 *   SHM_RECON_FAST_BICUBIC  cubic B-spline, the filter of the 4-bilinear-fetch "fast bicubic"
 *                           (GPU Gems 2 ch. 20), evaluated from its 16 taps; R_u, R_v by central
 *                           differences of the B-spline value at u +- h, v +- h
 * Cell indices of the shifted lookups are clamped to [-1, N+1] (2-tap) or [0, N] (4-tap), the
 * local coordinate then extending the nearest cell's polynomial.  The gradient and normal then
 * follow §3.4 exactly as in shm_query.  SHM_ERR_INVALID_ARG for a table that is not
 * SHM_LAYOUT_VALUE or an unknown method. */
typedef enum {
    SHM_RECON_NEAREST = 0,
    SHM_RECON_BILINEAR = 1,
    SHM_RECON_BICUBIC = 2,
    SHM_RECON_FAST_BICUBIC = 3
} shm_recon;

shm_status shm_query_recon(const shm_lut* lut, int32_t method, int64_t Q, const float* dirs,
                           const int32_t* glyph, const int64_t* seg, float* R, float* grad, float* normal,
                           float* chart, int32_t* fij, int32_t* dev_status, shm_stream stream);

/* ---------------------------------------------------------------- bake (Algorithm 1) */

typedef enum {
    SHM_SRC_SH = 0,      /* real SH coefficients; analytic derivatives (§3.3) */
    SHM_SRC_SAMPLES = 1, /* sampled values on a margin grid; central differences (§3.3) */
    SHM_SRC_BUMPS = 2,   /* R = 1 + sum_k a_k exp(-|w - mu_k|^2 / (2 w_k^2)), central differences */
    SHM_SRC_FBM = 3      /* h = amplitude * fBm(value noise), central differences (§4.10) */
} shm_source_kind;

/* Source of a bake.  All arrays device.
 *   SH:      coeffs [G][(L+1)^2] float32, index l*l + l + m (orthonormal real SH, no
 *            Condon-Shortley phase); basis from shm_sh_basis for (N_uniform, L).  SH sources
 *            need a uniform-N pool.
 *   SAMPLES: samples float32, glyph g's grid [6][N+4][N+4] at sample_offset[g] (floats);
 *            grid entry (jj, ii) is the value at texel centre (ii-1, jj-1) (one-texel bake
 *            margin around the padded face, §3.3).
 *   BUMPS:   bump_offset [G+1] (CSR), mu [B][3] unit vectors, amp [B], width [B] (radians).
 *   FBM:     keys [octaves][3] uint32 lattice keys; R = r0 + amplitude * sum_o gain^o
 *            noise(w base_freq lacunarity^o) (PCG3D-hashed value noise, quintic fade).
 * The stored channel 0 is the function minus r0[g] (r0 may be NULL = 0). */
typedef struct {
    int32_t kind;
    int32_t L;
    const float* coeffs;
    const float* basis;
    const float* samples;
    const int64_t* sample_offset;
    const int64_t* bump_offset;
    const float* mu;
    const float* amp;
    const float* width;
    int32_t octaves;
    const uint32_t* keys;
    float base_freq, lacunarity, gain, amplitude;
    int32_t* dev_status; /* optional device status word (SHM_DEV_TIMEOUT from the tensor-core bake) */
} shm_source;

/* Bytes of the SH bake basis for resolution N and degree L (host): K = (L+1)^2, M = 4*6(N+2)^2
 * table scalars per glyph, Kp = K rounded up to a multiple of 32, M16 = M rounded up to a multiple
 * of 16; 4 * (K*M + 2*M*Kp + 2*M16*Kp). */
int64_t shm_sh_basis_bytes(int32_t N, int32_t L);

/* Fills `basis` (device, shm_sh_basis_bytes) with every real SH function's record
 * (Y, Y_u h, Y_v h, Y_uv h^2) at every stored texel of the padded cubemap, from analytic
 * derivatives converted to the chart by the chain rule (§3.3, Algorithm 1).  The bake of
 * coefficients c is then lut = sum_k c_k basis_k.  Layout (float32): full [K][M] (row k =
 * basis_k's table, texel-major, channel innermost), then hi [M][Kp] and lo [M][Kp] with
 * hi = tf32(full^T), lo = tf32(full^T - hi), zero for k >= K (operands of the tensor-core bake),
 * then hiS and loS [M16/16][Kp][16], the same split untransposed in slabs of 16 columns (operands
 * of the tensor-core adjoint of shm_build_lut_backward, one contiguous 64-byte-swizzled tile per
 * slab): entry (k, c) at (c/16)*16*Kp + 16k + 4(((c%16)/4) XOR ((k/2)%4)) + c%4, zero for k >= K
 * and c >= M.  Compute once per (N, L) and reuse. */
shm_status shm_sh_basis(int32_t N, int32_t L, float* basis, shm_stream stream);

/* Workspace bytes that select the tensor-core engine of shm_build_lut for (lut, src): for SH
 * sources 2 * n_glyphs * Kp * 4 (tf32 hi/lo split of the coefficients); 0 for other sources. */
int64_t shm_build_workspace_bytes(const shm_lut* lut, const shm_source* src);

/* Writes every record of every glyph of `lut` (any dtype/layout) from `src` (Algorithm 1:
 * gutter texels evaluated at their own centres, derivative channels in each face's chart).
 * A SHM_LAYOUT_VALUE table receives the value at every texel centre of its two-texel gutter
 * grid: SH sources by direct evaluation (float32 CUDA cores; ws ignored), sampled sources copy
 * their margin grid, which is that same grid.
 * SH sources: with ws != NULL and ws_bytes >= shm_build_workspace_bytes the contraction runs on
 * the tensor cores (tcgen05, 3xTF32 split, float32-grade accuracy); with ws == NULL on the
 * float32 CUDA cores.  A non-NULL ws smaller than required returns SHM_ERR_WORKSPACE. */
shm_status shm_build_lut(const shm_lut* lut, const shm_source* src, void* ws, size_t ws_bytes,
                         shm_stream stream);

/* Re-encodes table `src` into `dst` (same glyphs and resolutions; any dtype/layout pair).
 * 16-bit stores round to nearest even.  dst channel 0 = src r0 + src channel 0 - dst r0. */
shm_status shm_pack_lut(const shm_lut* src, const shm_lut* dst, shm_stream stream);

/* Per-glyph bound R_max >= |r0 + interpolated r| over the sphere (for ray bracketing, §3.1):
 * max|r0 + r| + (max|r_u h| + max|r_v h|)/4 + max|r_uv h^2|/16 over the glyph's texels.
 * rmax: device float32 [n_glyphs]. */
shm_status shm_lut_bounds(const shm_lut* lut, float* rmax, shm_stream stream);

/* Derivative-consistent mip level (§4.7, Table lod): writes every record of `coarse` from
 * `fine`, glyph by glyph, with coarse N = fine N / 2 (fine N even).  The coarse value sample of
 * coarse texel (i, j) -- gutter ring and one-texel bake margin included -- is the mean of the fine
 * interpolant (shm_query's R) at the centres of fine texels 2i-1, 2i by 2j-1, 2j (directions
 * outside the face are served by the neighbouring face); the derivative channels follow by central
 * differences of those samples, as the finite-difference bake of shm_build_lut.  Any dtype/layout
 * on either side; 16-bit stores round to nearest even; coarse channel 0 is relative to the coarse
 * r0.  The tables must not overlap.  Uniform resolutions are checked here (SHM_ERR_INVALID_ARG);
 * with per-glyph arrays a glyph whose resolutions do not pair gets NaN records and SHM_DEV_BOUNDS
 * in *dev_status (device int32, may be NULL). */
shm_status shm_build_mip(const shm_lut* fine, const shm_lut* coarse, int32_t* dev_status, shm_stream stream);

/* ---------------------------------------------------------------- adjoint (not in the paper) */

/* Flags of shm_query_backward and shm_build_lut_backward. */
#define SHM_BWD_DETERMINISTIC 1u /* fixed summation order: dlut bit-identical from run to run */
#define SHM_BWD_CUDA_CORES 2u    /* shm_build_lut_backward: the float32 CUDA-core contraction */

/* Reverse mode of shm_query.  Upstream gradients gR [Q], ggrad [Q][3], gnormal [Q][3] (each
 * may be NULL = 0).  Accumulates (+=) dL/d(stored record) into dlut, a float32 TEXEL-layout
 * table with the same glyphs and resolutions as lut (any lut dtype/layout is read; a mismatch
 * gives SHM_ERR_INVALID_ARG), and writes (=) dL/d(dirs) into ddirs [Q][3] if not NULL.
 * flags = 0: atomic accumulation; the summation order, hence the last bits of dlut, may vary from
 * run to run.  flags = SHM_BWD_DETERMINISTIC: one CTA per glyph sorts each chunk of the glyph's
 * queries by cell and adds the per-cell sums in a fixed order, so dlut is bit-identical from run
 * to run and for any launch shape; needs CSR segments (glyph = NULL, seg != NULL, else
 * SHM_ERR_UNSUPPORTED) and parallelises over glyphs, so it suits many-glyph batches.  Other flag
 * bits: SHM_ERR_INVALID_ARG. */
shm_status shm_query_backward(const shm_lut* lut, int64_t Q, const float* dirs,
                              const int32_t* glyph, const int64_t* seg, const float* gR,
                              const float* ggrad, const float* gnormal, const shm_lut* dlut,
                              float* ddirs, uint32_t flags, int32_t* dev_status, shm_stream stream);

/* Reverse mode of the SH bake (Algorithm 1 is linear in the coefficients): dcoeffs[g][k] (=) sum
 * over texels and channels of dlut[g] * basis_k.  dlut: float32 texel layout, uniform N, 16-byte
 * aligned; basis from shm_sh_basis(N, L).
 * Default engine: the tensor cores (tcgen05, kind::tf32 with the 3xTF32 split of both operands,
 * the MMA sums drained into float32 registers every 256 texel scalars, float32-grade accuracy); for
 * few glyphs the CTAs of a thread-block cluster split the texel sum and add their partial sums in a
 * fixed rank order through distributed shared memory, so the result is bit-identical from run to
 * run with or without SHM_BWD_DETERMINISTIC.  It applies for K padded to 32 up to 128 (L <= 10);
 * otherwise, or with SHM_BWD_CUDA_CORES, the float32 CUDA-core contraction runs: flags = 0 splits the sum over
 * texels across CTAs and combines with atomics when there are few (glyph, k) tiles;
 * SHM_BWD_DETERMINISTIC makes one thread sum each entry in a fixed order.  A bounded wait of the
 * tensor-core kernel that expires (1 s) leaves dcoeffs unspecified (no status word here). */
shm_status shm_build_lut_backward(const shm_lut* dlut, int32_t L, const float* basis,
                                  float* dcoeffs, uint32_t flags, shm_stream stream);

/* Fused fit loss and adjoint (not in the paper; fits tables to targets).  Per query the forward
 * of shm_query is recomputed and L_q = w_value (R - R_target)^2 + w_normal |n - n_target|^2 is
 * formed; sum_q L_q is added (+=) to *loss (device float, may be NULL) and dL/d(stored record) is
 * accumulated (+=) into dlut (float32 texel layout, same glyphs and resolutions as lut).
 * R_target [Q], n_target [Q][3] float32.  Same glyph selection as shm_query. */
shm_status shm_fit_backward(const shm_lut* lut, int64_t Q, const float* dirs, const int32_t* glyph,
                            const int64_t* seg, const float* R_target, const float* n_target,
                            float w_value, float w_normal, const shm_lut* dlut, float* loss,
                            int32_t* dev_status, shm_stream stream);

/* One Adam step (Kingma & Ba 2015) over n float32 parameters with bias correction at step `step`
 * (>= 1): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).
 * zero_grad != 0 also sets grad to 0 for the next accumulation. */
shm_status shm_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                         float beta2, float eps, int32_t step, int32_t zero_grad, shm_stream stream);

/* ---------------------------------------------------------------- direct SH (ground truth) */

/* Direct evaluation of r(w) = sum c_lm Y_lm(w) with its S^2 gradient and normal (no table),
 * same glyph selection as shm_query.  coeffs [G][(L+1)^2] float32. */
shm_status shm_sh_eval(int32_t L, int32_t n_glyphs, const float* coeffs, int64_t Q,
                       const float* dirs, const int32_t* glyph, const int64_t* seg, float* R,
                       float* grad, float* normal, int32_t* dev_status, shm_stream stream);

/* ---------------------------------------------------------------- ray casting (§3.1) */

typedef struct {
    float eye[3], fwd[3], right[3], up[3]; /* orthonormal camera frame */
    float tan_half_fov_y;
    int32_t W, H;
} shm_camera;

typedef struct {
    int32_t march;  /* uniform F samples over the bounding-sphere chord (>= 1) */
    int32_t bisect; /* bisection steps after the first sign change (the maximum when lod != 0) */
    int32_t newton; /* Newton-Raphson steps after bisection (the maximum when lod != 0) */
    float ambient, kd, ks, shininess;
    float light[3];
    /* Refinement by projected size (§3.1: more iterations for glyphs large on screen; the paper
     * gives no rule).  lod != 0: per object, p = R_max (H/2) / (|c - eye| tan(fov_y/2)) pixels,
     * computed in float32 in that order without fused operations; bisection steps = the fewest b
     * in [bisect_min, bisect] with march * 2^b >= 128 p (the marched bracket 2 R_max / march
     * falls below 1/64 pixel; bisect if none does); Newton steps = newton if p >= 64, else
     * newton_min.  lod == 0: bisect and newton for every object. */
    int32_t lod;
    int32_t bisect_min;
    int32_t newton_min;
    /* Value-only tables (SHM_LAYOUT_VALUE) only: the SHM_RECON_* baseline that reconstructs the
     * surface and its gradient instead of the Hermite query (the equal-storage comparison renders of
     * §4.5); ignored for Hermite tables. */
    int32_t recon;
} shm_raycast_params;

typedef struct {
    float centre[3];
    float scale;  /* s > 0: R = s |r| */
    float rmax;   /* bounding-sphere radius (scale * shm_lut_bounds) */
    int32_t glyph;
} shm_object;

/* Workspace bytes shm_raycast needs for n_obj objects on a W x H image (host). */
int64_t shm_raycast_workspace_bytes(int32_t n_obj, int32_t W, int32_t H);

/* Ray casts star-shaped objects x(w) = c + s|r(w)| w (§3.1): per pixel ray p(t) = o + t d
 * with d = normalise(fwd + x_ndc tan(fov/2)(W/H) right + y_ndc tan(fov/2) up),
 * x_ndc = 2(px+1/2)/W - 1, y_ndc = 1 - 2(py+1/2)/H; per object the bounding-sphere chord
 * [t_min, t_max] is sampled `march` times, the first sample with F < 0 brackets the root of
 * F(x) = |x - c| - R(w), which is refined by `bisect` bisection and `newton` Newton steps;
 * the nearest hit is shaded Blinn-Phong with the analytic normal (§3.4, signed rule
 * grad R = s sign(r) grad r).  A SHM_LAYOUT_VALUE table is ray cast through the baseline
 * reconstruction prm->recon instead (its value and gradient, §4.5; SHM_ERR_INVALID_ARG for an
 * unknown method).  Outputs (row-major, may be NULL): rgba [H][W][4],
 * depth [H][W] (t, +inf on a miss), normal [H][W][3], obj_id [H][W] (-1 on a miss).
 * objs: device [n_obj]; cam, prm: HOST structs. */
shm_status shm_raycast(const shm_lut* lut, const shm_object* objs, int32_t n_obj,
                       const shm_camera* cam, const shm_raycast_params* prm, float* rgba,
                       float* depth, float* normal, int32_t* obj_id, void* ws, size_t ws_bytes,
                       int32_t* dev_status, shm_stream stream);

/* Capacity of the device-resident workspace used by shm_raycast_noalloc, in bytes. */
#define SHM_RAYCAST_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* shm_raycast without a caller workspace.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory when they ray cast, such as a renderer embedded
 * in a host application that owns the GPU memory budget through its own pool, or a real-time frame
 * loop where cudaMalloc / cudaFree would synchronise the device and stall the frame.
 *   - The workspace is a static device array of SHM_RAYCAST_NOALLOC_SCRATCH_BYTES (16 MiB) inside
 *     libshm.so; every GPU that loads the library holds it until the process exits.  Calls whose
 *     shm_raycast_workspace_bytes(n_obj, W, H) exceeds it return SHM_ERR_WORKSPACE and launch
 *     nothing (512 objects at 1920x1080 fit).
 *   - The first call on a device looks up the array's device address (with that device current)
 *     and caches it per device index for the life of the process; make that first call before any
 *     stream capture on the device.  A cudaDeviceReset of that device invalidates the cached
 *     address: do not call this entry point again in that process after such a reset.
 *   - All calls share the one array, which keeps the previous call's contents (the counters that
 *     must start at zero are cleared on `stream` by every call).  Calls that overlap on the GPU,
 *     for example on two streams, race on it: serialise them.
 *   - No device memory is allocated or freed.  Results equal shm_raycast's. */
shm_status shm_raycast_noalloc(const shm_lut* lut, const shm_object* objs, int32_t n_obj,
                               const shm_camera* cam, const shm_raycast_params* prm, float* rgba,
                               float* depth, float* normal, int32_t* obj_id, int32_t* dev_status,
                               shm_stream stream);

/* ---------------------------------------------------------------- L2 hint (not in the paper) */

/* L2 fetch granularity of the calling thread's current device context (a CUDA context limit,
 * released with the context; no device setting outlives the process): the largest block the L2
 * fetches from HBM for a miss.  Uncorrelated footprint reads (random directions into an out-of-L2
 * table) use 16-32 B of each fetch; smaller fetches keep more distinct table pieces in L2.  The
 * limit is a hint that applies to every kernel launched afterwards in the context, including other
 * libraries'.  bytes = -1 only reads the current value; 0..128 sets it.  *previous (host, may be
 * NULL) receives the value before the call.  SHM_ERR_UNSUPPORTED if the device rejects the limit. */
shm_status shm_l2_fetch_granularity(int32_t bytes, int32_t* previous);

/* ---------------------------------------------------------------- misc */

const char* shm_status_string(shm_status s);
int32_t shm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SHM_H */
