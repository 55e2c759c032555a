// Ray casting of star-shaped objects x(w) = c + s|r(w)| w through their Hermite tables
// (arXiv 2602.20063, §3.1; shading normals §3.4).
//
// The paper renders billboards through a raster pipeline; here there is no raster stage:
//   k_rank_objects  orders objects front to back by |c - eye| - R_max (rank by counting, keys
//                   staged in shared memory 256 at a time);
//   k_bin_tiles     one warp per 16x16 pixel tile walks the ordered objects 32 at a time and keeps,
//                   in order (ballot compaction), those whose conservative screen rectangle (from
//                   the bounding sphere) covers it;
//   k_raycast       persistent warps take 8x4-pixel blocks of a tile from an atomic counter (no
//                   waits, no CTA barriers: a warp moves on as soon as its own pixels are done); per pixel and
//                   candidate object: bounding-sphere chord [t_min, t_max] -> `march` samples of
//                   F(x) = |x - c| - R(w), spaced (t_max - t_min)/march apart -> first sign change ->
//                   `bisect` halvings (march and bisection on the value alone) -> `newton`
//                   Newton steps with F' = d.(w - grad_{S^2}R/|x - c|) -> nearest hit -> normal
//                   n = (R w - grad R)/|R w - grad R| with grad R = s sign(r) grad r -> Blinn-Phong.
// Workspace: 64-byte header {uint32 tile counter, uint32 pad, uint64 surface queries evaluated},
// then ranks [n_obj], ordered ids [n_obj], per-tile counts [tiles], per-tile lists [tiles][n_obj].
#include <math.h>

#include <mutex>

#include "shm_internal.h"

namespace shm {

constexpr int RT = 16;  // tile edge in pixels

struct WsLayout {
    int64_t rank_off, order_off, count_off, list_off, total;
};

__host__ __device__ __forceinline__ WsLayout ws_layout(int n_obj, int W, int H)
{
    const int64_t tiles = (int64_t)((W + RT - 1) / RT) * ((H + RT - 1) / RT);
    WsLayout w;
    w.rank_off = 64;
    w.order_off = w.rank_off + 4LL * n_obj;
    w.count_off = w.order_off + 4LL * n_obj;
    w.list_off = w.count_off + 4LL * tiles;
    w.list_off = (w.list_off + 15) / 16 * 16;
    w.total = w.list_off + 4LL * tiles * n_obj;
    return w;
}

int64_t raycast_workspace_bytes(int n_obj, int W, int H) { return ws_layout(n_obj, W, H).total; }

__device__ __forceinline__ float depth_key(const shm_object& o, const shm_camera& cam)
{
    const float dx = o.centre[0] - cam.eye[0], dy = o.centre[1] - cam.eye[1], dz = o.centre[2] - cam.eye[2];
    return sqrtf(dx * dx + dy * dy + dz * dz) - o.rmax;
}

constexpr int RANK_BLOCK = 256;

// NaN keys sort last (treated as +inf, ties by index), so ranks stay a permutation of 0..n-1.
__device__ __forceinline__ float rank_key(const shm_object& o, const shm_camera& cam)
{
    const float k = depth_key(o, cam);
    return (k == k) ? k : __int_as_float(0x7f800000);
}

__global__ void __launch_bounds__(RANK_BLOCK) k_rank_objects(const shm_object* __restrict__ objs, int n, shm_camera cam,
                                                             int32_t* order)
{
    __shared__ float kt[RANK_BLOCK];
    const int i = blockIdx.x * RANK_BLOCK + threadIdx.x;
    const float ki = i < n ? rank_key(objs[i], cam) : 0.0f;
    int rank = 0;
    for (int j0 = 0; j0 < n; j0 += RANK_BLOCK) {
        __syncthreads();
        if (j0 + (int)threadIdx.x < n) kt[threadIdx.x] = rank_key(objs[j0 + threadIdx.x], cam);
        __syncthreads();
        const int m = min(RANK_BLOCK, n - j0);
        for (int jj = 0; jj < m; ++jj) {
            const float kj = kt[jj];
            rank += (kj < ki) || (kj == ki && j0 + jj < i);
        }
    }
    if (i < n) order[rank] = i;
}

// Conservative pixel rectangle of a sphere (centre c, radius r): for every point p of the
// sphere, (p.right)/(p.fwd) and (p.up)/(p.fwd) lie in the box of the extreme ratios.
__device__ __forceinline__ bool sphere_rect(const shm_object& o, const shm_camera& cam, int& x0, int& x1, int& y0,
                                            int& y1)
{
    const float dx = o.centre[0] - cam.eye[0], dy = o.centre[1] - cam.eye[1], dz = o.centre[2] - cam.eye[2];
    const float cz = dx * cam.fwd[0] + dy * cam.fwd[1] + dz * cam.fwd[2];
    const float cx = dx * cam.right[0] + dy * cam.right[1] + dz * cam.right[2];
    const float cy = dx * cam.up[0] + dy * cam.up[1] + dz * cam.up[2];
    const float r = o.rmax * 1.001f + 1e-6f;
    if (cz + r <= 0.0f) return false;  // entirely behind the camera
    if (cz - r <= 1e-6f) {             // straddles the eye plane: cover the screen
        x0 = 0; y0 = 0; x1 = cam.W - 1; y1 = cam.H - 1;
        return true;
    }
    const float zn = cz - r, zf = cz + r;
    const float xa = cx - r, xb = cx + r, ya = cy - r, yb = cy + r;
    const float xmin = xa < 0.0f ? xa / zn : xa / zf, xmax = xb > 0.0f ? xb / zn : xb / zf;
    const float ymin = ya < 0.0f ? ya / zn : ya / zf, ymax = yb > 0.0f ? yb / zn : yb / zf;
    const float sx = 1.0f / (cam.tan_half_fov_y * ((float)cam.W / (float)cam.H)), sy = 1.0f / cam.tan_half_fov_y;
    // px + 1/2 = (x_ndc + 1) W/2, py + 1/2 = (1 - y_ndc) H/2
    const float fx0 = (xmin * sx + 1.0f) * 0.5f * cam.W - 0.5f, fx1 = (xmax * sx + 1.0f) * 0.5f * cam.W - 0.5f;
    const float fy0 = (1.0f - ymax * sy) * 0.5f * cam.H - 0.5f, fy1 = (1.0f - ymin * sy) * 0.5f * cam.H - 0.5f;
    if (fx1 < -1.0f || fy1 < -1.0f || fx0 > cam.W || fy0 > cam.H) return false;
    x0 = max(0, (int)floorf(fx0) - 1);
    x1 = min(cam.W - 1, (int)ceilf(fx1) + 1);
    y0 = max(0, (int)floorf(fy0) - 1);
    y1 = min(cam.H - 1, (int)ceilf(fy1) + 1);
    return x0 <= x1 && y0 <= y1;
}

__global__ void __launch_bounds__(256) k_bin_tiles(const shm_object* __restrict__ objs, int n, shm_camera cam,
                                                    const int32_t* __restrict__ order, int32_t* counts, int32_t* lists)
{
    const int tx_n = (cam.W + RT - 1) / RT, ty_n = (cam.H + RT - 1) / RT;
    const int tile = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (tile >= tx_n * ty_n) return;  // warp-uniform
    const int tx = tile % tx_n, ty = tile / tx_n;
    const int px0 = tx * RT, px1 = min(cam.W - 1, px0 + RT - 1), py0 = ty * RT, py1 = min(cam.H - 1, py0 + RT - 1);
    int cnt = 0;
    int32_t* out = lists + (int64_t)tile * n;
    for (int q0 = 0; q0 < n; q0 += 32) {
        const int q = q0 + lane;
        int id = -1;
        bool hit = false;
        if (q < n) {
            id = __ldg(order + q);
            if (id >= 0 && id < n) {
                const shm_object o = objs[id];
                int x0, x1, y0, y1;
                hit = sphere_rect(o, cam, x0, x1, y0, y1) && !(x1 < px0 || x0 > px1 || y1 < py0 || y0 > py1);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) out[cnt + __popc(m & ((1u << lane) - 1u))] = id;
        cnt += __popc(m);
    }
    if (lane == 0) counts[tile] = cnt;
}

struct Surf {
    float F, dF;
    float R, sgn;
    Vec3 grad;
};

// R and its S^2 gradient at direction x: the Hermite query (RECON < 0, §3.3-§3.4), or a value-only
// baseline reconstruction of a SHM_LAYOUT_VALUE table (RECON = SHM_RECON_*, the equal-storage
// renders of §4.5).
template <int DT, int LAYOUT, int RECON>
__device__ __forceinline__ bool eval_surface(const LutView& L, const GlyphRef& G, float x0, float x1, float x2,
                                             QueryResult& qr, Chart& ch)
{
    if constexpr (RECON < 0) return query_one<DT, LAYOUT>(L, G, x0, x1, x2, qr, ch);
    else return recon_one<RECON, DT>(L, G, x0, x1, x2, qr, ch);
}

template <int DT, int LAYOUT, int RECON>
__device__ __forceinline__ bool surface_F(const LutView& L, const GlyphRef& G, float scale, const float* c, const float* o,
                                          const Vec3& d, float t, Surf& S)
{
    const float x0 = o[0] + t * d.x - c[0], x1 = o[1] + t * d.y - c[1], x2 = o[2] + t * d.z - c[2];
    QueryResult qr;
    Chart ch;
    if (!eval_surface<DT, LAYOUT, RECON>(L, G, x0, x1, x2, qr, ch)) return false;
    const float dist = sqrtf(x0 * x0 + x1 * x1 + x2 * x2);
    S.sgn = qr.R >= 0.0f ? 1.0f : -1.0f;
    S.R = scale * fabsf(qr.R);
    S.F = dist - S.R;
    S.grad = Vec3{scale * S.sgn * qr.grad.x, scale * S.sgn * qr.grad.y, scale * S.sgn * qr.grad.z};
    const float id = 1.0f / dist;
    const float dw = (d.x * x0 + d.y * x1 + d.z * x2) * id;
    const float dg = d.x * S.grad.x + d.y * S.grad.y + d.z * S.grad.z;
    S.dF = dw - dg * id;
    return true;
}

// F alone at t (march and bisection need only its sign): chart, cell, footprint and the Hermite
// value, no derivatives.  Same value as surface_F's S.F.  (Value-only baselines: their full
// reconstruction, whose value is the same.)
template <int DT, int LAYOUT, int RECON>
__device__ __forceinline__ bool surface_value(const LutView& L, const GlyphRef& G, float scale, const float* c,
                                              const float* o, const Vec3& d, float t, float& F)
{
    const float x0 = o[0] + t * d.x - c[0], x1 = o[1] + t * d.y - c[1], x2 = o[2] + t * d.z - c[2];
    if constexpr (RECON >= 0) {
        QueryResult qr;
        Chart ch;
        if (!eval_surface<DT, LAYOUT, RECON>(L, G, x0, x1, x2, qr, ch)) return false;
        F = sqrtf(x0 * x0 + x1 * x1 + x2 * x2) - scale * fabsf(qr.R);
        return true;
    }
    Chart ch;
    if (!chart_of(x0, x1, x2, ch)) return false;
    int i, j;
    float s, tt;
    cell_of(pick3(ch.k1, x0, x1, x2), ch.m, ch.im, G.N, i, s);
    cell_of(pick3(ch.k2, x0, x1, x2), ch.m, ch.im, G.N, j, tt);
    const float R = G.r0 + hermite_value(fetch_corners<DT, LAYOUT>(L.data, G, ch.f, i, j), s, tt);
    F = sqrtf(x0 * x0 + x1 * x1 + x2 * x2) - scale * fabsf(R);
    return true;
}

// F alone for the march and the bisection, leaner than surface_value: the chart from an
// approximate reciprocal and the cell and local coordinate in plain float32 (x = u N/2 + N/2 + 1/2;
// the double-float cell_of matters for exact cell indices at large N, not for the sign of F), and
// |x| from a reciprocal square root.  F differs from surface_value's by a few float32 roundings, far
// inside the march's sign decisions; the Newton steps and the shading normal use surface_F.
// (A lean F and dF for the Newton steps as well measured slower: 0.433 against 0.417 ms for rank,
// bin and ray cast of the 512-object impostor frame.)
template <int DT, int LAYOUT>
__device__ __forceinline__ bool ray_value(const LutView& L, const GlyphRef& G, float scale, const float* c,
                                          const float* o, const Vec3& d, float t, float& F)
{
    const float x0 = o[0] + t * d.x - c[0], x1 = o[1] + t * d.y - c[1], x2 = o[2] + t * d.z - c[2];
    const float a0 = fabsf(x0), a1 = fabsf(x1), a2 = fabsf(x2);
    int k = 0;
    float m = a0;
    if (a1 > m) { k = 1; m = a1; }
    if (a2 > m) { k = 2; m = a2; }
    const float sum = a0 + a1 + a2;
    if (!(m > 0.0f) || !(m <= 3.402823466e38f) || !(sum == sum)) return false;
    const int k1 = (k == 2) ? 0 : k + 1, k2 = (k == 0) ? 2 : k - 1;
    const float dk = pick3(k, x0, x1, x2);
    const int f = 2 * k + (dk < 0.0f ? 1 : 0);
    const float im = __fdividef(1.0f, m);
    const float Nf = (float)G.N, hN = 0.5f * Nf, off = hN + 0.5f;
    const float X = fmaf(pick3(k1, x0, x1, x2) * im, hN, off), Y = fmaf(pick3(k2, x0, x1, x2) * im, hN, off);
    const float fi = fminf(fmaxf(floorf(X), 0.0f), Nf), fj = fminf(fmaxf(floorf(Y), 0.0f), Nf);
    const float R = G.r0 + hermite_value(fetch_corners<DT, LAYOUT>(L.data, G, f, (int)fi, (int)fj), X - fi, Y - fj);
    const float r2 = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
    F = r2 * rsqrtf(r2) - scale * fabsf(R);
    return true;
}

// The march and bisection evaluation: ray_value on Hermite tables, the baseline's full
// reconstruction on value tables.
template <int DT, int LAYOUT, int RECON>
__device__ __forceinline__ bool march_value(const LutView& L, const GlyphRef& G, float scale, const float* c,
                                            const float* o, const Vec3& d, float t, float& F)
{
    if constexpr (RECON < 0) return ray_value<DT, LAYOUT>(L, G, scale, c, o, d, t, F);
    else return surface_value<DT, LAYOUT, RECON>(L, G, scale, c, o, d, t, F);
}

// Refinement steps of one object by its projected radius (see shm_raycast_params).  The radius
// decides integers, so it is formed with round-to-nearest intrinsics (no contraction into FMA),
// operation by operation as written.
__device__ __forceinline__ void lod_steps(const shm_raycast_params& prm, const shm_camera& cam, const shm_object& ob,
                                          int& bisect, int& newton)
{
    bisect = prm.bisect;
    newton = prm.newton;
    if (!prm.lod) return;
    const float dx = __fsub_rn(ob.centre[0], cam.eye[0]);
    const float dy = __fsub_rn(ob.centre[1], cam.eye[1]);
    const float dz = __fsub_rn(ob.centre[2], cam.eye[2]);
    const float D = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
    const float p = __fdiv_rn(__fmul_rn(ob.rmax, 0.5f * (float)cam.H), __fmul_rn(D, cam.tan_half_fov_y));
    const float need = 128.0f * p;
    for (int b = prm.bisect_min; b <= prm.bisect; ++b) {
        if ((float)prm.march * __int_as_float((127 + b) << 23) >= need) {  // march * 2^b, exact
            bisect = b;
            break;
        }
    }
    newton = (p >= 64.0f) ? prm.newton : prm.newton_min;
}

template <int DT, int LAYOUT, int RECON>
__global__ void __launch_bounds__(RT * RT) k_raycast(LutView L, const shm_object* __restrict__ objs, int n, shm_camera cam,
                                                    shm_raycast_params prm, const int32_t* __restrict__ counts,
                                                    const int32_t* __restrict__ lists, uint32_t* tile_counter,
                                                    unsigned long long* query_counter, float* rgba, float* depth,
                                                    float* normal, int32_t* obj_id, int32_t* dev_status)
{
    const int tx_n = (cam.W + RT - 1) / RT, ty_n = (cam.H + RT - 1) / RT;
    const int nunits = tx_n * ty_n * (RT / 2);  // a unit = an 8x4-pixel block of a tile = one warp
    const int lane = threadIdx.x & 31;
    const float qnan = __int_as_float(0x7fc00000);
    uint32_t status = 0;
    unsigned long long nq = 0;
    float lx = prm.light[0], ly = prm.light[1], lz = prm.light[2];
    {
        const float il = rsqrtf(lx * lx + ly * ly + lz * lz);
        lx *= il; ly *= il; lz *= il;
    }
    const float aspect = (float)cam.W / (float)cam.H;
    const float inv_march = 1.0f / (float)prm.march;
    for (;;) {
        int unit = 0;
        if (lane == 0) unit = (int)atomicAdd(tile_counter, 1u);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= nunits) break;  // warp-uniform
        const int tile = unit / (RT / 2), blk = unit % (RT / 2);  // blocks: 2 across, 4 down a tile
        const int px = (tile % tx_n) * RT + (blk & 1) * 8 + (lane & 7), py = (tile / tx_n) * RT + (blk >> 1) * 4 + (lane >> 3);
        if (px >= cam.W || py >= cam.H) continue;
        const float xn = (2.0f * (px + 0.5f) / cam.W - 1.0f) * cam.tan_half_fov_y * aspect;
        const float yn = (1.0f - 2.0f * (py + 0.5f) / cam.H) * cam.tan_half_fov_y;
        Vec3 d{cam.fwd[0] + xn * cam.right[0] + yn * cam.up[0], cam.fwd[1] + xn * cam.right[1] + yn * cam.up[1],
               cam.fwd[2] + xn * cam.right[2] + yn * cam.up[2]};
        {
            const float il = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            d.x *= il; d.y *= il; d.z *= il;
        }
        const float* o = cam.eye;
        float best_t = __int_as_float(0x7f800000);
        int best = -1;
        const int cnt = __ldg(counts + tile);
        const int32_t* lst = lists + (int64_t)tile * n;
        for (int q = 0; q < cnt; ++q) {
            const int id = __ldg(lst + q);
            const shm_object ob = objs[id];
            if (ob.glyph < 0 || ob.glyph >= L.n_glyphs) { status |= SHM_DEV_BOUNDS; continue; }
            const float ocx = o[0] - ob.centre[0], ocy = o[1] - ob.centre[1], ocz = o[2] - ob.centre[2];
            const float b = ocx * d.x + ocy * d.y + ocz * d.z;
            const float cc = ocx * ocx + ocy * ocy + ocz * ocz - ob.rmax * ob.rmax;
            const float disc = b * b - cc;
            if (disc < 0.0f) continue;
            const float sq = sqrtf(disc);
            float t0 = -b - sq;
            const float t1 = -b + sq;
            if (t1 <= 0.0f) continue;
            if (t0 < 0.0f) t0 = 0.0f;
            if (t0 >= best_t) continue;
            int n_bisect, n_newton;
            lod_steps(prm, cam, ob, n_bisect, n_newton);
            const GlyphRef G = glyph_ref(L, ob.glyph);
            Surf S;
            float thit = qnan;
            float F;
            if (!march_value<DT, LAYOUT, RECON>(L, G, ob.scale, ob.centre, o, d, t0, F)) { status |= SHM_DEV_NONFINITE; continue; }
            ++nq;
            if (F < 0.0f) {
                thit = t0;
            } else {
                float lo = t0, hi = t0;
                bool found = false;
                const float span = t1 - t0;
                float kf = 0.0f;
                for (int k = 1; k <= prm.march; ++k) {
                    kf += 1.0f;
                    const float tk = fmaf(span, kf * inv_march, t0);
                    march_value<DT, LAYOUT, RECON>(L, G, ob.scale, ob.centre, o, d, tk, F);
                    ++nq;
                    if (F < 0.0f) {
                        hi = tk;
                        found = true;
                        break;
                    }
                    lo = tk;
                }
                if (!found) continue;
                for (int it = 0; it < n_bisect; ++it) {
                    const float mid = 0.5f * (lo + hi);
                    march_value<DT, LAYOUT, RECON>(L, G, ob.scale, ob.centre, o, d, mid, F);
                    ++nq;
                    if (F < 0.0f) hi = mid; else lo = mid;
                }
                float t = 0.5f * (lo + hi);
                for (int it = 0; it < n_newton; ++it) {
                    surface_F<DT, LAYOUT, RECON>(L, G, ob.scale, ob.centre, o, d, t, S);
                    ++nq;
                    if (S.dF == 0.0f) break;
                    const float tn = t - S.F / S.dF;
                    if (!(tn >= lo && tn <= hi)) break;
                    t = tn;
                }
                thit = t;
            }
            if (thit < best_t) {
                best_t = thit;
                best = id;
            }
        }
        const int64_t pix = (int64_t)py * cam.W + px;
        if (best < 0) {
            if (rgba) { rgba[4 * pix] = 0.f; rgba[4 * pix + 1] = 0.f; rgba[4 * pix + 2] = 0.f; rgba[4 * pix + 3] = 0.f; }
            if (depth) depth[pix] = __int_as_float(0x7f800000);
            if (normal) { normal[3 * pix] = 0.f; normal[3 * pix + 1] = 0.f; normal[3 * pix + 2] = 0.f; }
            if (obj_id) obj_id[pix] = -1;
            continue;
        }
        const shm_object ob = objs[best];
        const GlyphRef G = glyph_ref(L, ob.glyph);
        Surf S;
        surface_F<DT, LAYOUT, RECON>(L, G, ob.scale, ob.centre, o, d, best_t, S);
        ++nq;
        const float x0 = o[0] + best_t * d.x - ob.centre[0], x1 = o[1] + best_t * d.y - ob.centre[1],
                    x2 = o[2] + best_t * d.z - ob.centre[2];
        const Vec3 n = surface_normal(x0, x1, x2, S.R, S.grad);
        float hx = lx - d.x, hy = ly - d.y, hz = lz - d.z;
        const float ih = rsqrtf(hx * hx + hy * hy + hz * hz);
        hx *= ih; hy *= ih; hz *= ih;
        const float ndl = n.x * lx + n.y * ly + n.z * lz;
        const float ndh = n.x * hx + n.y * hy + n.z * hz;
        const float I = prm.ambient + prm.kd * fmaxf(ndl, 0.0f) + prm.ks * (ndh > 0.0f ? powf(ndh, prm.shininess) : 0.0f);
        if (rgba) { rgba[4 * pix] = I; rgba[4 * pix + 1] = I; rgba[4 * pix + 2] = I; rgba[4 * pix + 3] = 1.0f; }
        if (depth) depth[pix] = best_t;
        if (normal) { normal[3 * pix] = n.x; normal[3 * pix + 1] = n.y; normal[3 * pix + 2] = n.z; }
        if (obj_id) obj_id[pix] = best;
    }
    for (int off = 16; off > 0; off >>= 1) nq += __shfl_xor_sync(0xffffffffu, nq, off);
    if ((threadIdx.x & 31) == 0 && nq) atomicAdd(query_counter, nq);
    report_status(dev_status, status);
}

cudaError_t launch_raycast(const LutView& L, const shm_object* objs, int n_obj, const shm_camera& cam,
                           const shm_raycast_params& prm, float* rgba, float* depth, float* normal, int32_t* obj_id,
                           void* ws, size_t ws_bytes, int32_t* dev_status, cudaStream_t s)
{
    (void)ws_bytes;
    const WsLayout w = ws_layout(n_obj, cam.W, cam.H);
    char* base = (char*)ws;
    int32_t* order = (int32_t*)(base + w.order_off);
    int32_t* counts = (int32_t*)(base + w.count_off);
    int32_t* lists = (int32_t*)(base + w.list_off);
    const int tiles = ((cam.W + RT - 1) / RT) * ((cam.H + RT - 1) / RT);
    cudaError_t e = cudaMemsetAsync(base, 0, 64, s);
    if (e != cudaSuccess) return e;
    if (n_obj > 0) {
        e = cudaMemsetAsync(order, 0xff, 4LL * n_obj, s);
        if (e != cudaSuccess) return e;
        k_rank_objects<<<(n_obj + RANK_BLOCK - 1) / RANK_BLOCK, RANK_BLOCK, 0, s>>>(objs, n_obj, cam, order);
        k_bin_tiles<<<(unsigned)(((int64_t)tiles * 32 + 255) / 256), 256, 0, s>>>(objs, n_obj, cam, order, counts, lists);
    } else {
        e = cudaMemsetAsync(counts, 0, 4LL * tiles, s);
        if (e != cudaSuccess) return e;
    }
    int blocks = sm_count() * 4;
    if (blocks > tiles) blocks = tiles;
    uint32_t* tile_counter = (uint32_t*)base;
    unsigned long long* qc = (unsigned long long*)(base + 8);
#define SHM_RC(DT, LY)                                                                                         \
    k_raycast<DT, LY, -1><<<blocks, RT * RT, 0, s>>>(L, objs, n_obj, cam, prm, counts, lists, tile_counter, qc,   \
                                                     rgba, depth, normal, obj_id, dev_status)
#define SHM_RV(DT, M)                                                                                          \
    k_raycast<DT, SHM_LAYOUT_VALUE, M><<<blocks, RT * RT, 0, s>>>(L, objs, n_obj, cam, prm, counts, lists,      \
                                                                  tile_counter, qc, rgba, depth, normal, obj_id, \
                                                                  dev_status)
#define SHM_RV_DT(M)                                 \
    if (L.dtype == SHM_F32) SHM_RV(SHM_F32, M);      \
    else if (L.dtype == SHM_F16) SHM_RV(SHM_F16, M); \
    else SHM_RV(SHM_BF16, M)
    if (L.layout == SHM_LAYOUT_VALUE) {
        switch (prm.recon) {
        case SHM_RECON_NEAREST: SHM_RV_DT(SHM_RECON_NEAREST); break;
        case SHM_RECON_BILINEAR: SHM_RV_DT(SHM_RECON_BILINEAR); break;
        case SHM_RECON_BICUBIC: SHM_RV_DT(SHM_RECON_BICUBIC); break;
        default: SHM_RV_DT(SHM_RECON_FAST_BICUBIC); break;
        }
    } else if (L.layout == SHM_LAYOUT_TEXEL) {
        if (L.dtype == SHM_F32) SHM_RC(SHM_F32, SHM_LAYOUT_TEXEL);
        else if (L.dtype == SHM_F16) SHM_RC(SHM_F16, SHM_LAYOUT_TEXEL);
        else SHM_RC(SHM_BF16, SHM_LAYOUT_TEXEL);
    } else {
        if (L.dtype == SHM_F32) SHM_RC(SHM_F32, SHM_LAYOUT_CELL);
        else if (L.dtype == SHM_F16) SHM_RC(SHM_F16, SHM_LAYOUT_CELL);
        else SHM_RC(SHM_BF16, SHM_LAYOUT_CELL);
    }
#undef SHM_RC
#undef SHM_RV
#undef SHM_RV_DT
    return cudaGetLastError();
}

}  // namespace shm

// ------------------------------------------------------------------------------------------
// Allocation-free variant of shm_raycast (no counterpart in the paper).
//
// Some callers cannot allocate device memory at the point where they ray cast: a renderer
// running inside a host application that owns the GPU memory budget through its own pool, or a
// real-time frame loop in which a cudaMalloc / cudaFree would synchronise the device and stall the
// frame.  For them the workspace lives in this file-scope device array instead of a caller buffer.
// Every GPU that loads libshm.so holds the array until the process exits.
static __device__ __align__(256) unsigned char g_raycast_scratch[SHM_RAYCAST_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_raycast_scratch for the current device.  In host code the array's name is
// only a host-side stand-in, so the address is looked up once per device (with that device
// current) and cached per device index.  A cudaDeviceReset unloads the module and leaves the cached
// address stale; the header tells callers not to use this entry point after one.
void* raycast_scratch_address(shm_status* st)
{
    static std::mutex mu;
    static void* cache[256] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        *st = SHM_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_raycast_scratch) != cudaSuccess || !p) {
            *st = SHM_ERR_CUDA;
            return nullptr;
        }
        cache[dev] = p;
    }
    *st = SHM_OK;
    return cache[dev];
}

}  // namespace

extern "C" shm_status shm_raycast_noalloc(const shm_lut* lut, const shm_object* objs, int32_t n_obj,
                                          const shm_camera* cam, const shm_raycast_params* prm, float* rgba,
                                          float* depth, float* normal, int32_t* obj_id, int32_t* dev_status,
                                          shm_stream stream)
{
    if (!cam || n_obj < 0 || cam->W <= 0 || cam->H <= 0 || cam->W > 65536 || cam->H > 65536)
        return SHM_ERR_INVALID_ARG;
    if (shm::raycast_workspace_bytes(n_obj, cam->W, cam->H) > (int64_t)SHM_RAYCAST_NOALLOC_SCRATCH_BYTES)
        return SHM_ERR_WORKSPACE;
    shm_status st = SHM_OK;
    void* ws = raycast_scratch_address(&st);
    if (st != SHM_OK) return st;
    return shm_raycast(lut, objs, n_obj, cam, prm, rgba, depth, normal, obj_id, ws,
                       (size_t)SHM_RAYCAST_NOALLOC_SCRATCH_BYTES, dev_status, stream);
}
