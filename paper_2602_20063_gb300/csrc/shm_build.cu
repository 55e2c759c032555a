// Bake kernels (arXiv 2602.20063, Algorithm 1 and §3.3):
//
//   k_sh_basis      per stored texel (gutter included) and SH function Y_k the record
//                   (Y, Y_u h, Y_v h, Y_uv h^2): Y and its Cartesian gradient / Hessian from the
//                   polynomial form of the real SH, carried to the face chart by the chain rule
//                   r_u = grad Y . dw/du,  r_uv = (dw/du)^T H (dw/dv) + grad Y . d2w/dudv.
//   k_sh_gemm       lut[g][t][ch] = sum_k c[g][k] basis[k][t][ch] - r0[g] (ch 0): the bake of many
//                   glyphs as one [G x K] x [K x 4T] contraction (SIMT float32 reference engine).
//   k_sh_gemm_bwd   dc[g][k] = sum_{t,ch} dlut[g][t][ch] basis[k][t][ch].
//   k_fd_face       central differences on a sample grid with a one-texel bake margin, from
//                   stored samples, Gaussian bumps or value-noise fBm evaluated in the kernel
//                   (per face or 64 x 64 region, samples in shared memory); k_value_build stores
//                   the samples themselves for value-only tables.
//   k_pack          re-encode a table into another dtype / layout.
//   k_bounds        per-glyph bound of |interpolated r| for ray bracketing (§3.1).
//   k_sh_eval       direct SH value, S^2 gradient and normal (ground truth, no table).
//
// SH convention: orthonormal real SH, index l*l + l + m, no Condon-Shortley phase,
// Y_l0 = P~_l^0(z), Y_lm = sqrt2 P~_l^m(z) Re (x+iy)^m, Y_l-m = sqrt2 P~_l^m(z) Im (x+iy)^m, where
// P~_l^m = K_lm d^m P_l/dz^m comes from the normalised recurrences
//   P~_0^0 = 1/sqrt(4 pi),  P~_m^m = sqrt((2m+1)/(2m)) P~_{m-1}^{m-1},  P~_{m+1}^m = sqrt(2m+3) z P~_m^m,
//   P~_l^m = a_lm (z P~_{l-1}^m - b_lm P~_{l-2}^m),  a_lm = sqrt((4l^2-1)/(l^2-m^2)),
//   b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
// and K_lm d^{m+1}P_l/dz^{m+1} = sqrt((l-m)(l+m+1)) P~_l^{m+1} (no overflow for any L).
#include "shm_internal.h"

namespace shm {

constexpr int SH_LMAX = 20;

// ------------------------------------------------------------------------------------------
// Normalised associated Legendre table T[l(l+1)/2 + m], 0 <= m <= l <= L, in Qbar form.
__device__ __forceinline__ void legendre_table(int L, float z, float* T)
{
    T[0] = 0.28209479177387814f;  // 1/sqrt(4 pi)
    for (int m = 0; m <= L; ++m) {
        const int im = m * (m + 1) / 2 + m;
        if (m > 0) {
            const int ip = (m - 1) * m / 2 + (m - 1);
            T[im] = T[ip] * sqrtf((2.0f * m + 1.0f) / (2.0f * m));
        }
        if (m + 1 <= L) T[(m + 1) * (m + 2) / 2 + m] = sqrtf(2.0f * m + 3.0f) * z * T[im];
        for (int l = m + 2; l <= L; ++l) {
            const float l2 = (float)(l * l), m2 = (float)(m * m), lm1 = (float)((l - 1) * (l - 1));
            const float a = sqrtf((4.0f * l2 - 1.0f) / (l2 - m2));
            const float b = sqrtf((lm1 - m2) / (4.0f * lm1 - 1.0f));
            T[l * (l + 1) / 2 + m] = a * (z * T[(l - 1) * l / 2 + m] - b * T[(l - 2) * (l - 1) / 2 + m]);
        }
    }
}

__device__ __forceinline__ float tab(const float* T, int l, int m)
{
    return (m <= l) ? T[l * (l + 1) / 2 + m] : 0.0f;
}

// Value, Cartesian gradient and Hessian (xx, xy, yy, xz, yz, zz) of Y_lm at the unit vector w.
struct YDer {
    float v, gx, gy, gz, hxx, hxy, hyy, hxz, hyz, hzz;
};

// A = C_m (cosine part) or S_m (sine part) of (x + iy)^m, with derivatives from
// d/dx (x+iy)^m = m (x+iy)^{m-1},  d/dy (x+iy)^m = i m (x+iy)^{m-1}.
__device__ __forceinline__ YDer ylm_derivs(const float* T, int l, int m, bool sine, const float* C, const float* S)
{
    YDer y;
    const float q0 = tab(T, l, m);
    const float f1 = sqrtf((float)((l - m) * (l + m + 1)));
    const float q1 = f1 * tab(T, l, m + 1);
    const float q2 = f1 * sqrtf((float)max(0, (l - m - 1) * (l + m + 2))) * tab(T, l, m + 2);
    float A, Ax, Ay, Axx, Axy, Ayy;
    if (m == 0) {
        A = 1.0f; Ax = Ay = Axx = Axy = Ayy = 0.0f;
    } else if (!sine) {
        A = C[m];
        Ax = m * C[m - 1];
        Ay = -m * S[m - 1];
        const float mm = (float)(m * (m - 1));
        Axx = m >= 2 ? mm * C[m - 2] : 0.0f;
        Axy = m >= 2 ? -mm * S[m - 2] : 0.0f;
        Ayy = -Axx;
    } else {
        A = S[m];
        Ax = m * S[m - 1];
        Ay = m * C[m - 1];
        const float mm = (float)(m * (m - 1));
        Axx = m >= 2 ? mm * S[m - 2] : 0.0f;
        Axy = m >= 2 ? mm * C[m - 2] : 0.0f;
        Ayy = -Axx;
    }
    const float sc = (m == 0) ? 1.0f : 1.41421356237309515f;
    y.v = sc * q0 * A;
    y.gx = sc * q0 * Ax;
    y.gy = sc * q0 * Ay;
    y.gz = sc * q1 * A;
    y.hxx = sc * q0 * Axx;
    y.hxy = sc * q0 * Axy;
    y.hyy = sc * q0 * Ayy;
    y.hxz = sc * q1 * Ax;
    y.hyz = sc * q1 * Ay;
    y.hzz = sc * q2 * A;
    return y;
}

__device__ __forceinline__ void cs_table(int L, float x, float y, float* C, float* S)
{
    C[0] = 1.0f;
    S[0] = 0.0f;
    for (int m = 1; m <= L; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
}

// Unit vector of chart axis `axis` (0..2) with sign.
__device__ __forceinline__ Vec3 axis_vec(int axis, float sgn)
{
    return Vec3{axis == 0 ? sgn : 0.0f, axis == 1 ? sgn : 0.0f, axis == 2 ? sgn : 0.0f};
}

__device__ __forceinline__ float dot3(const Vec3& a, const Vec3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Direction of texel-centre chart coordinates (X, Y) = (2u-1, 2v-1) on face f, with the
// tangents e1 = dw/du, e2 = dw/dv and the mixed second derivative W = d2w/dudv.
struct TexelFrame {
    Vec3 w, e1, e2, W;
};

__device__ __forceinline__ TexelFrame texel_frame(int f, float X, float Y)
{
    const int k = f >> 1;
    const float sg = (f & 1) ? -1.0f : 1.0f;
    const Vec3 a = axis_vec(k, sg), b = axis_vec((k + 1) % 3, 1.0f), c = axis_vec((k + 2) % 3, 1.0f);
    const Vec3 wt{a.x + X * b.x + Y * c.x, a.y + X * b.y + Y * c.y, a.z + X * b.z + Y * c.z};
    const float rho2 = 1.0f + X * X + Y * Y;
    const float rho = sqrtf(rho2);
    const float ir = 1.0f / rho;
    TexelFrame T;
    T.w = Vec3{wt.x * ir, wt.y * ir, wt.z * ir};
    // e1 = (2/rho)(b - w (w.b)), w.b = X/rho; e2 likewise with c, Y
    const float wb = X * ir, wc = Y * ir;
    T.e1 = Vec3{2.0f * ir * (b.x - T.w.x * wb), 2.0f * ir * (b.y - T.w.y * wb), 2.0f * ir * (b.z - T.w.z * wb)};
    T.e2 = Vec3{2.0f * ir * (c.x - T.w.x * wc), 2.0f * ir * (c.y - T.w.y * wc), 2.0f * ir * (c.z - T.w.z * wc)};
    // W = (4/rho^3)(-Y b - X c) + (12 X Y / rho^5) w~
    const float i3 = 4.0f * ir * ir * ir, i5 = 12.0f * X * Y * ir * ir * ir * ir * ir;
    T.W = Vec3{i3 * (-Y * b.x - X * c.x) + i5 * wt.x, i3 * (-Y * b.y - X * c.y) + i5 * wt.y,
               i3 * (-Y * b.z - X * c.z) + i5 * wt.z};
    return T;
}

__global__ void __launch_bounds__(128) k_sh_basis(int N, int L, float* __restrict__ basis)
{
    const int P = N + 2;
    const int T = 6 * P * P;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int f = t / (P * P), rem = t % (P * P), j = rem / P, i = rem % P;
    // texel centre u_i = (i - 1/2)/N -> 2u - 1 = (2i - 1 - N)/N
    const float X = (float)(2 * i - 1 - N) / (float)N;
    const float Y = (float)(2 * j - 1 - N) / (float)N;
    const TexelFrame F = texel_frame(f, X, Y);
    float Tl[(SH_LMAX + 1) * (SH_LMAX + 2) / 2];
    float C[SH_LMAX + 1], S[SH_LMAX + 1];
    legendre_table(L, F.w.z, Tl);
    cs_table(L, F.w.x, F.w.y, C, S);
    const float h = 1.0f / (float)N;
    for (int l = 0; l <= L; ++l) {
        for (int mm = -l; mm <= l; ++mm) {
            const int m = mm < 0 ? -mm : mm;
            const YDer y = ylm_derivs(Tl, l, m, mm < 0, C, S);
            const float ru = y.gx * F.e1.x + y.gy * F.e1.y + y.gz * F.e1.z;
            const float rv = y.gx * F.e2.x + y.gy * F.e2.y + y.gz * F.e2.z;
            const float e1He2 = y.hxx * F.e1.x * F.e2.x + y.hyy * F.e1.y * F.e2.y + y.hzz * F.e1.z * F.e2.z +
                                y.hxy * (F.e1.x * F.e2.y + F.e1.y * F.e2.x) +
                                y.hxz * (F.e1.x * F.e2.z + F.e1.z * F.e2.x) +
                                y.hyz * (F.e1.y * F.e2.z + F.e1.z * F.e2.y);
            const float ruv = e1He2 + y.gx * F.W.x + y.gy * F.W.y + y.gz * F.W.z;
            const int k = l * l + l + mm;
            reinterpret_cast<float4*>(basis)[(int64_t)k * T + t] = make_float4(y.v, ru * h, rv * h, ruv * h * h);
        }
    }
}

cudaError_t launch_sh_basis(int N, int L, float* basis, cudaStream_t s)
{
    const int T = 6 * (N + 2) * (N + 2);
    k_sh_basis<<<(T + 127) / 128, 128, 0, s>>>(N, L, basis);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// SIMT bake contraction: tile of 32 glyphs x 64 texels (x 4 channels), K in chunks of 16.
constexpr int GT_G = 32, GT_T = 64, GT_K = 16;

__global__ void __launch_bounds__(256) k_sh_gemm(LutView out, void* data, int K, const float* __restrict__ coeffs,
                                                 const float* __restrict__ basis)
{
    __shared__ __align__(16) float Cs[GT_K][GT_G];
    __shared__ __align__(16) float4 Bs[GT_K][GT_T];
    const int N = out.N_uniform;
    const int T = 6 * (N + 2) * (N + 2);
    const int G = out.n_glyphs;
    const int g0 = blockIdx.y * GT_G, t0 = blockIdx.x * GT_T;
    const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
    float4 acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4* B4 = reinterpret_cast<const float4*>(basis);
    for (int k0 = 0; k0 < K; k0 += GT_K) {
        for (int e = tid; e < GT_K * GT_G; e += 256) {
            const int kk = e % GT_K, gg = e / GT_K;
            const int g = g0 + gg, k = k0 + kk;
            Cs[kk][gg] = (g < G && k < K) ? __ldg(coeffs + (int64_t)g * K + k) : 0.0f;
        }
        for (int e = tid; e < GT_K * GT_T; e += 256) {
            const int kk = e / GT_T, tt = e % GT_T;
            const int k = k0 + kk, t = t0 + tt;
            Bs[kk][tt] = (k < K && t < T) ? __ldg(B4 + (int64_t)k * T + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GT_K; ++kk) {
            const float4 b = Bs[kk][tx];
            const float4 ca = *reinterpret_cast<const float4*>(&Cs[kk][ty * 8]);
            const float4 cb = *reinterpret_cast<const float4*>(&Cs[kk][ty * 8 + 4]);
            const float cv[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                acc[r].x = fmaf(cv[r], b.x, acc[r].x);
                acc[r].y = fmaf(cv[r], b.y, acc[r].y);
                acc[r].z = fmaf(cv[r], b.z, acc[r].z);
                acc[r].w = fmaf(cv[r], b.w, acc[r].w);
            }
        }
        __syncthreads();
    }
    const int t = t0 + tx;
    if (t >= T) return;
    const int P = N + 2;
    const int f = t / (P * P), rem = t % (P * P), j = rem / P, i = rem % P;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int g = g0 + ty * 8 + r;
        if (g >= G) break;
        const GlyphRef Gr = glyph_ref(out, g);
        float4 v = acc[r];
        v.x -= Gr.r0;
        store_texel(data, out.dtype, out.layout, Gr, f, j, i, v);
    }
}

cudaError_t launch_sh_build(const LutView& out, void* data, int L, const float* coeffs, const float* basis,
                            cudaStream_t s)
{
    const int N = out.N_uniform;
    const int T = 6 * (N + 2) * (N + 2);
    const int K = (L + 1) * (L + 1);
    dim3 grid((T + GT_T - 1) / GT_T, (out.n_glyphs + GT_G - 1) / GT_G);
    k_sh_gemm<<<grid, 256, 0, s>>>(out, data, K, coeffs, basis);
    return cudaGetLastError();
}

// dc[g][k] = sum_r dlut[g][r] basis[k][r], r over 4T scalars.  Tile 64 glyphs x 32 k, the
// reduction split over blockIdx.z and combined with atomics into a zeroed dcoeffs (one split, so
// a fixed summation order, when the result must be deterministic).
constexpr int BG = 64, BK = 32, BR = 32;

__global__ void __launch_bounds__(256) k_sh_gemm_bwd(int R4, int G, int K, const float* __restrict__ dlut,
                                                     const float* __restrict__ basis, float* __restrict__ dc,
                                                     int r_per_split)
{
    __shared__ __align__(16) float Ds[BR][BG];
    __shared__ __align__(16) float Bs[BR][BK];
    const int g0 = blockIdx.x * BG, k0 = blockIdx.y * BK;
    const int rb = blockIdx.z * r_per_split, re = min(R4, rb + r_per_split);
    const int tid = threadIdx.x, tg = tid & 15, tk = tid >> 4;  // 4 glyphs x 2 k per thread
    float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int r0 = rb; r0 < re; r0 += BR) {
        for (int e = tid; e < BR * BG; e += 256) {
            const int rr = e % BR, gg = e / BR;
            const int g = g0 + gg, r = r0 + rr;
            Ds[rr][gg] = (g < G && r < re) ? __ldg(dlut + (int64_t)g * R4 + r) : 0.0f;
        }
        for (int e = tid; e < BR * BK; e += 256) {
            const int rr = e % BR, kk = e / BR;
            const int k = k0 + kk, r = r0 + rr;
            Bs[rr][kk] = (k < K && r < re) ? __ldg(basis + (int64_t)k * R4 + r) : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < BR; ++rr) {
            const float4 d = *reinterpret_cast<const float4*>(&Ds[rr][tg * 4]);
            const float2 b = *reinterpret_cast<const float2*>(&Bs[rr][tk * 2]);
            const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                acc[a][0] = fmaf(dv[a], b.x, acc[a][0]);
                acc[a][1] = fmaf(dv[a], b.y, acc[a][1]);
            }
        }
        __syncthreads();
    }
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 2; ++c) {
            const int g = g0 + tg * 4 + a, k = k0 + tk * 2 + c;
            if (g < G && k < K) atomicAdd(dc + (int64_t)g * K + k, acc[a][c]);
        }
}

cudaError_t launch_sh_build_bwd(int N, int G, int L, const float* dlut, const float* basis, float* dcoeffs, bool det,
                                cudaStream_t s)
{
    const int K = (L + 1) * (L + 1);
    const int R4 = 4 * 6 * (N + 2) * (N + 2);
    cudaError_t e = cudaMemsetAsync(dcoeffs, 0, sizeof(float) * (size_t)G * K, s);
    if (e != cudaSuccess) return e;
    const int gx = (G + BG - 1) / BG, ky = (K + BK - 1) / BK;
    int splits = det ? 1 : (sm_count() * 4 + gx * ky - 1) / (gx * ky);
    const int max_splits = (R4 + BR - 1) / BR;
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    int per = (R4 + splits - 1) / splits;
    per = (per + BR - 1) / BR * BR;
    splits = (R4 + per - 1) / per;
    k_sh_gemm_bwd<<<dim3(gx, ky, splits), 256, 0, s>>>(R4, G, K, dlut, basis, dcoeffs, per);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Procedural sources (radial depth-map impostors §4.9, procedural planets §4.10).
__device__ __forceinline__ void pcg3d(uint32_t& x, uint32_t& y, uint32_t& z)
{
    x = x * 1664525u + 1013904223u;
    y = y * 1664525u + 1013904223u;
    z = z * 1664525u + 1013904223u;
    x += y * z;
    y += z * x;
    z += x * y;
    x ^= x >> 16;
    y ^= y >> 16;
    z ^= z >> 16;
    x += y * z;
    y += z * x;
    z += x * y;
}

__device__ __forceinline__ float lattice_value(int ix, int iy, int iz, uint32_t k0, uint32_t k1, uint32_t k2)
{
    uint32_t x = (uint32_t)ix + k0, y = (uint32_t)iy + k1, z = (uint32_t)iz + k2;
    pcg3d(x, y, z);
    return (float)(x >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

__device__ __forceinline__ float quintic(float t) { return t * t * t * (t * (t * 6.0f - 15.0f) + 10.0f); }

__device__ float value_noise(float px, float py, float pz, uint32_t k0, uint32_t k1, uint32_t k2)
{
    const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    const float wx = quintic(px - fx), wy = quintic(py - fy), wz = quintic(pz - fz);
    float c[2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy) {
            const float v0 = lattice_value(ix, iy + dy, iz + dz, k0, k1, k2);
            const float v1 = lattice_value(ix + 1, iy + dy, iz + dz, k0, k1, k2);
            c[dz][dy] = v0 + wx * (v1 - v0);
        }
    const float e0 = c[0][0] + wy * (c[0][1] - c[0][0]);
    const float e1 = c[1][0] + wy * (c[1][1] - c[1][0]);
    return e0 + wz * (e1 - e0);
}

__device__ float fbm(const Vec3& w, const shm_source& src)
{
    float sum = 0.0f, freq = src.base_freq, amp = 1.0f;
    for (int o = 0; o < src.octaves; ++o) {
        const uint32_t* key = src.keys + 3 * o;
        sum = fmaf(amp, value_noise(w.x * freq, w.y * freq, w.z * freq, __ldg(key), __ldg(key + 1), __ldg(key + 2)), sum);
        freq *= src.lacunarity;
        amp *= src.gain;
    }
    return src.amplitude * sum;
}

// value_noise with the lattice values read from a table of the box [x0, x0+nx) x [y0, ...) x
// [z0, ...) (same corners and interpolation, so the same result).
__device__ __forceinline__ float value_noise_box(float px, float py, float pz, const float* T, int x0, int y0, int z0,
                                                 int nx, int ny, int nz)
{
    const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
    const float wx = quintic(px - fx), wy = quintic(py - fy), wz = quintic(pz - fz);
    // the corner stays inside the box (the callers' box is padded; the clamps only guard it)
    const int nxy = nx * ny;
    const int bx = min(max((int)fx - x0, 0), nx - 2), by = min(max((int)fy - y0, 0), ny - 2);
    const int bz = min(max((int)fz - z0, 0), nz - 2);
    const float* b = T + bz * nxy + by * nx + bx;
    float c[2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy) {
            const float* r = b + dz * nxy + dy * nx;
            const float v0 = r[0], v1 = r[1];
            c[dz][dy] = v0 + wx * (v1 - v0);
        }
    const float e0 = c[0][0] + wy * (c[0][1] - c[0][0]);
    const float e1 = c[1][0] + wy * (c[1][1] - c[1][0]);
    return e0 + wz * (e1 - e0);
}

// value_noise_box at two points at once (.x and .y): the same operations lane by lane (so the same
// values), the fade and the trilinear interpolation on float2 pairs, the box corners per lane.
__device__ __forceinline__ float2 quintic2(float2 t)
{
    return pmul(pmul(pmul(t, t), t), pfma(t, pfma(t, bc(6.0f), bc(-15.0f)), bc(10.0f)));
}

__device__ __forceinline__ float2 value_noise_box2(float2 px, float2 py, float2 pz, const float* T, int x0, int y0,
                                                   int z0, int nx, int ny, int nz)
{
    const float2 fx = make_float2(floorf(px.x), floorf(px.y)), fy = make_float2(floorf(py.x), floorf(py.y));
    const float2 fz = make_float2(floorf(pz.x), floorf(pz.y));
    const float2 wx = quintic2(psub(px, fx)), wy = quintic2(psub(py, fy)), wz = quintic2(psub(pz, fz));
    const int nxy = nx * ny;
    const float* b[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int bx = min(max((int)(l ? fx.y : fx.x) - x0, 0), nx - 2);
        const int by = min(max((int)(l ? fy.y : fy.x) - y0, 0), ny - 2);
        const int bz = min(max((int)(l ? fz.y : fz.x) - z0, 0), nz - 2);
        b[l] = T + bz * nxy + by * nx + bx;
    }
    float2 c[2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int o = dz * nxy + dy * nx;
            const float2 v0 = make_float2(b[0][o], b[1][o]), v1 = make_float2(b[0][o + 1], b[1][o + 1]);
            c[dz][dy] = pfma(wx, psub(v1, v0), v0);
        }
    const float2 e0 = pfma(wy, psub(c[0][1], c[0][0]), c[0][0]);
    const float2 e1 = pfma(wy, psub(c[1][1], c[1][0]), c[1][0]);
    return pfma(wz, psub(e1, e0), e0);
}

// ------------------------------------------------------------------------------------------
// Sampled sources: value tables (k_value_build) and finite-difference records (k_fd_face).
constexpr int FS = 18, MAX_BUMPS_SMEM = 128;
constexpr int FBM_CACHE = 4096;  // lattice values of the octaves' boxes per CTA (16 KB)
constexpr int FBM_MAX_OCT = 16;  // octaves whose boxes may be cached

// Gaussian bumps of one glyph, staged in shared memory: centre and amplitude as one float4 (a
// broadcast 16-byte read), and the exponent factor with log2(e) folded in, so that
//   a exp(-|w - mu|^2 / (2 width^2)) = a exp2(|w - mu|^2 k),  k = -log2(e) / (2 width^2),
// with 2^x from the PTX ex2.approx.ftz instruction (relative error about 2^-22; results below the
// float32 normal range flush to zero, far below the sum's rounding error).
struct BumpSmem {
    float4 m[MAX_BUMPS_SMEM];
    float k[MAX_BUMPS_SMEM];
};

__device__ __forceinline__ void stage_bumps(BumpSmem& B, const shm_source& src, int64_t bc, int nb)
{
    for (int e = threadIdx.x; e < nb; e += blockDim.x) {
        B.m[e] = make_float4(__ldg(src.mu + 3 * (bc + e)), __ldg(src.mu + 3 * (bc + e) + 1),
                             __ldg(src.mu + 3 * (bc + e) + 2), __ldg(src.amp + bc + e));
        const float wd = __ldg(src.width + bc + e);
        B.k[e] = -0.72134752044448170f / (wd * wd);  // 0.5 log2(e)
    }
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float bump_sum(const BumpSmem& B, int nb, const Vec3& w, float sum)
{
#pragma unroll 4
    for (int q = 0; q < nb; ++q) {
        const float4 m = B.m[q];
        const float dx = w.x - m.x, dy = w.y - m.y, dz = w.z - m.z;
        sum = fmaf(m.w, ex2_approx((dx * dx + dy * dy + dz * dz) * B.k[q]), sum);
    }
    return sum;
}

// bump_sum at two sample directions at once: the same operations lane by lane (so the same sums),
// with each bump's parameters read once and the arithmetic on float2 pairs (one instruction for
// both samples); the two exp2 evaluations stay scalar.
__device__ __forceinline__ float2 bump_sum2(const BumpSmem& B, int nb, const Vec3& wa, const Vec3& wb, float2 sum)
{
    const float2 wx = make_float2(wa.x, wb.x), wy = make_float2(wa.y, wb.y), wz = make_float2(wa.z, wb.z);
#pragma unroll 4
    for (int q = 0; q < nb; ++q) {
        const float4 m = B.m[q];
        const float2 dx = psub(wx, bc(m.x)), dy = psub(wy, bc(m.y)), dz = psub(wz, bc(m.z));
        const float2 e = pmul(pfma(dz, dz, pfma(dy, dy, pmul(dx, dx))), bc(B.k[q]));
        sum = pfma(bc(m.w), make_float2(ex2_approx(e.x), ex2_approx(e.y)), sum);
    }
    return sum;
}

// Value tables (SHM_LAYOUT_VALUE) of sampled sources: the table is the margin sample grid itself,
// so 18 x 18 tiles of samples are evaluated and stored (plus the value offset), no differences.
template <class Map>
__global__ void __launch_bounds__(256) k_value_build(LutView out, void* data, shm_source src, const __grid_constant__ Map map)
{
    __shared__ BumpSmem bump;
    int tile;
    const int g = map_block(map, tile), f = blockIdx.y;
    const GlyphRef Gr = glyph_ref(out, g);
    const int N = Gr.N, S = N + 4;
    const int tiles = (S + FS - 1) / FS;
    if (tile >= tiles * tiles) return;
    const int i0 = (tile % tiles) * FS, j0 = (tile / tiles) * FS;
    const int tid = threadIdx.x;
    const int k = f >> 1;
    const float sg = (f & 1) ? -1.0f : 1.0f;
    const Vec3 a = axis_vec(k, sg), bb = axis_vec((k + 1) % 3, 1.0f), cc = axis_vec((k + 2) % 3, 1.0f);

    // Two sample slots per thread (18 x 18 = 324 samples, 256 threads).  Sample-grid index
    // (ii, jj) holds texel (ii-1, jj-1) at u = (ii - 3/2)/N, i.e. 2u - 1 = (2 ii - 3 - N)/N.
    float acc[2] = {0.f, 0.f};
    Vec3 w[2];
    bool live[2];
    for (int r = 0; r < 2; ++r) {
        const int e = tid + r * 256;
        const int ii = i0 + (e % FS), jj = j0 + (e / FS);
        live[r] = (e < FS * FS) && ii < S && jj < S;
        const float X = (float)(2 * ii - 3 - N) / (float)N;
        const float Y = (float)(2 * jj - 3 - N) / (float)N;
        const float ir = rsqrtf(1.0f + X * X + Y * Y);
        w[r] = Vec3{(a.x + X * bb.x + Y * cc.x) * ir, (a.y + X * bb.y + Y * cc.y) * ir,
                    (a.z + X * bb.z + Y * cc.z) * ir};
        if (!live[r]) continue;
        if (src.kind == SHM_SRC_SAMPLES)
            acc[r] = __ldg(src.samples + __ldg(src.sample_offset + g) + ((int64_t)f * S + jj) * S + ii) - Gr.r0;
        else if (src.kind == SHM_SRC_FBM)
            acc[r] = fbm(w[r], src);
    }
    // Bumps: the sum without the leading 1 is kept in the samples (stored = sum + 1 - r0).
    float base = 0.0f;
    if (src.kind == SHM_SRC_BUMPS) {
        base = 1.0f - Gr.r0;
        const int64_t b_lo = __ldg(src.bump_offset + g), b_hi = __ldg(src.bump_offset + g + 1);
        for (int64_t bc = b_lo; bc < b_hi; bc += MAX_BUMPS_SMEM) {
            const int nb = (int)min((int64_t)MAX_BUMPS_SMEM, b_hi - bc);
            __syncthreads();
            stage_bumps(bump, src, bc, nb);
            __syncthreads();
            for (int r = 0; r < 2; ++r)
                if (live[r]) acc[r] = bump_sum(bump, nb, w[r], acc[r]);
        }
    }
    for (int r = 0; r < 2; ++r) {
        if (!live[r]) continue;
        const int e = tid + r * 256;
        const int ii = i0 + (e % FS), jj = j0 + (e / FS);
        store_val(data, out.dtype, Gr.base + ((int64_t)f * S + jj) * S + ii, acc[r] + base);
    }
}

// Region variant: one CTA per (glyph, face, T x T texel region) evaluates the region's
// (T+2)^2 margin samples once into shared memory, then forms its records.  For tables up to
// N = FACE_N_MAX the region is the whole padded face (no sample is evaluated twice; a 16x16 tile
// needs 18x18 samples, up to 3.2x the face's count at N = 16); larger tables use 64x64 regions
// (6 % re-evaluation at the region borders).  Pools of uneven N cap the region at FACE_SPLIT_T
// texels: a face of N = 128 then takes four CTAs, so the largest faces no longer set the launch's
// tail, and the smaller shared-memory footprint lets five CTAs share an SM instead of three.
// Uniform pools split each face into 2 x 2 equal regions once a whole face's samples would need
// more than FACE_SPLIT_SMEM bytes, i.e. fewer CTAs per SM than the register limit of five allows
// (512 bump objects: N = 128 0.944 vs 0.982 ms, N = 144 1.171 vs 1.340 ms; N <= 96 stays whole,
// where splitting measured -1 % to +1 %).  The sample directions and values are those of the
// value tables (k_value_build).
constexpr int FACE_N_MAX = 144;   // (N+4)^2 floats <= 87.6 KB
constexpr int REGION_T = 64;      // region edge for larger tables: 66^2 floats = 17.4 KB
constexpr int FACE_SPLIT_T = 66;  // uneven pools: N <= 64 faces stay whole, N = 128 faces split 2 x 2
constexpr int FACE_SPLIT_SMEM = 45 * 1024;

// FBM: the fBm source (its lattice cache is only allocated in that instantiation); otherwise stored
// samples or Gaussian bumps.
template <bool FBM, class Map>
__global__ void __launch_bounds__(256) k_fd_face(LutView out, void* data, shm_source src, int T,
                                                 const __grid_constant__ Map map)
{
    extern __shared__ float Sf[];  // [T+2][T+2]
    int region;
    const int g = map_block(map, region), f = blockIdx.y;
    const GlyphRef Gr = glyph_ref(out, g);
    const int N = Gr.N, P = N + 2;
    const int nr = (P + T - 1) / T;
    if (region >= nr * nr) return;
    const int i0 = (region % nr) * T, j0 = (region / nr) * T;  // first texel of the region
    const int ti = min(T, P - i0), tj = min(T, P - j0);      // texels in the region
    const int Si = ti + 2, Sj = tj + 2;                       // samples: texels i0-1 .. i0+ti
    const int tid = threadIdx.x;
    const int k = f >> 1;
    const float sg = (f & 1) ? -1.0f : 1.0f;
    const Vec3 a = axis_vec(k, sg), bb = axis_vec((k + 1) % 3, 1.0f), cc = axis_vec((k + 2) % 3, 1.0f);
    // sample-grid index (ii, jj) of the face (texel (ii-1, jj-1)); local sample (li, lj) = (ii-i0, jj-j0)
    auto dir = [&](int ii, int jj) {
        const float X = (float)(2 * ii - 3 - N) / (float)N;
        const float Y = (float)(2 * jj - 3 - N) / (float)N;
        const float ir = rsqrtf(1.0f + X * X + Y * Y);
        return Vec3{(a.x + X * bb.x + Y * cc.x) * ir, (a.y + X * bb.y + Y * cc.y) * ir,
                    (a.z + X * bb.z + Y * cc.z) * ir};
    };
    const int S = N + 4;
    float base = 0.0f;
    if constexpr (FBM) {
        // fBm over the region with the lattice values in shared memory: the corners an octave of
        // frequency f needs lie in the box [floor(f wmin), floor(f wmax) + 1] per axis (floor(f w)
        // is monotone in w), padded by one lattice step on each side; the boxes of all octaves that
        // fit are hashed once, the others are hashed per sample.  Chart coordinates X, Y of the
        // region's columns and rows are divided once.
        __shared__ float cache[FBM_CACHE];
        __shared__ float s_w[8][6];
        __shared__ float s_xy[2 * (REGION_T + 2)];
        __shared__ int s_box[FBM_MAX_OCT][8];  // x0, y0, z0, nx, ny, nz, cache offset, boxed
        const bool xy_tab = (Si <= REGION_T + 2 && Sj <= REGION_T + 2);  // block-uniform
        if (xy_tab) {
            for (int e = tid; e < Si + Sj; e += 256) {
                const int g2 = (e < Si) ? 2 * (i0 + e) : 2 * (j0 + e - Si);
                s_xy[e] = (float)(g2 - 3 - N) / (float)N;
            }
            __syncthreads();
        }
        auto wdir = [&](int li, int lj) {
            if (!xy_tab) return dir(i0 + li, j0 + lj);
            const float X = s_xy[li], Y = s_xy[Si + lj];
            const float ir = rsqrtf(1.0f + X * X + Y * Y);
            return Vec3{(a.x + X * bb.x + Y * cc.x) * ir, (a.y + X * bb.y + Y * cc.y) * ir,
                        (a.z + X * bb.z + Y * cc.z) * ir};
        };
        float lo[3] = {3.0f, 3.0f, 3.0f}, hi[3] = {-3.0f, -3.0f, -3.0f};
        for (int e = tid; e < Si * Sj; e += 256) {
            const Vec3 w = wdir(e % Si, e / Si);
            lo[0] = fminf(lo[0], w.x); lo[1] = fminf(lo[1], w.y); lo[2] = fminf(lo[2], w.z);
            hi[0] = fmaxf(hi[0], w.x); hi[1] = fmaxf(hi[1], w.y); hi[2] = fmaxf(hi[2], w.z);
        }
        for (int o = 16; o > 0; o >>= 1)
            for (int a3 = 0; a3 < 3; ++a3) {
                lo[a3] = fminf(lo[a3], __shfl_xor_sync(0xffffffffu, lo[a3], o));
                hi[a3] = fmaxf(hi[a3], __shfl_xor_sync(0xffffffffu, hi[a3], o));
            }
        if ((tid & 31) == 0)
            for (int a3 = 0; a3 < 3; ++a3) { s_w[tid >> 5][a3] = lo[a3]; s_w[tid >> 5][3 + a3] = hi[a3]; }
        __syncthreads();
        const int octaves = min(src.octaves, FBM_MAX_OCT);
        if (tid == 0) {
            for (int a3 = 0; a3 < 3; ++a3) {
                lo[a3] = s_w[0][a3];
                hi[a3] = s_w[0][3 + a3];
                for (int wp = 1; wp < 8; ++wp) { lo[a3] = fminf(lo[a3], s_w[wp][a3]); hi[a3] = fmaxf(hi[a3], s_w[wp][3 + a3]); }
            }
            float freq = src.base_freq;
            int used = 0;
            for (int o = 0; o < octaves; ++o) {
                int* bx = s_box[o];
                bx[0] = (int)floorf(lo[0] * freq) - 1;
                bx[1] = (int)floorf(lo[1] * freq) - 1;
                bx[2] = (int)floorf(lo[2] * freq) - 1;
                bx[3] = (int)floorf(hi[0] * freq) - bx[0] + 3;
                bx[4] = (int)floorf(hi[1] * freq) - bx[1] + 3;
                bx[5] = (int)floorf(hi[2] * freq) - bx[2] + 3;
                const int64_t n = (int64_t)bx[3] * bx[4] * bx[5];
                bx[6] = used;
                bx[7] = (used + n <= FBM_CACHE) ? 1 : 0;
                if (bx[7]) used += (int)n;
                freq *= src.lacunarity;
            }
        }
        __syncthreads();
        for (int o = 0; o < octaves; ++o) {
            const int* bx = s_box[o];
            if (!bx[7]) continue;  // block-uniform
            const int nx = bx[3], ny = bx[4], n = nx * ny * bx[5];
            const uint32_t k0 = __ldg(src.keys + 3 * o), k1 = __ldg(src.keys + 3 * o + 1), k2 = __ldg(src.keys + 3 * o + 2);
            for (int idx = tid; idx < n; idx += 256) {
                const int ix = idx % nx, iy = (idx / nx) % ny, iz = idx / (nx * ny);
                cache[bx[6] + idx] = lattice_value(bx[0] + ix, bx[1] + iy, bx[2] + iz, k0, k1, k2);
            }
        }
        __syncthreads();
        // two samples per thread at a time (e and e + 256), the last odd one alone: per octave the
        // box parameters are read once for both and the cached lattice is interpolated on pairs
        for (int e = tid; e < Si * Sj; e += 512) {
            const int e2 = e + 256;
            if (e2 < Si * Sj) {
                const Vec3 wa = wdir(e % Si, e / Si), wb = wdir(e2 % Si, e2 / Si);
                float2 sum = make_float2(0.0f, 0.0f);
                float freq = src.base_freq, amp = 1.0f;
                for (int o = 0; o < src.octaves; ++o) {
                    const float2 px = pmul(make_float2(wa.x, wb.x), bc(freq));
                    const float2 py = pmul(make_float2(wa.y, wb.y), bc(freq));
                    const float2 pz = pmul(make_float2(wa.z, wb.z), bc(freq));
                    float2 v;
                    if (o < FBM_MAX_OCT && s_box[o][7]) {
                        const int* bx = s_box[o];
                        v = value_noise_box2(px, py, pz, cache + bx[6], bx[0], bx[1], bx[2], bx[3], bx[4], bx[5]);
                    } else {
                        const uint32_t* key = src.keys + 3 * o;
                        const uint32_t k0 = __ldg(key), k1 = __ldg(key + 1), k2 = __ldg(key + 2);
                        v = make_float2(value_noise(px.x, py.x, pz.x, k0, k1, k2), value_noise(px.y, py.y, pz.y, k0, k1, k2));
                    }
                    sum = pfma(bc(amp), v, sum);
                    freq *= src.lacunarity;
                    amp *= src.gain;
                }
                Sf[e] = src.amplitude * sum.x;
                Sf[e2] = src.amplitude * sum.y;
            } else {
                const Vec3 w = wdir(e % Si, e / Si);
                float sum = 0.0f, freq = src.base_freq, amp = 1.0f;
                for (int o = 0; o < src.octaves; ++o) {
                    const float px = w.x * freq, py = w.y * freq, pz = w.z * freq;
                    float v;
                    if (o < FBM_MAX_OCT && s_box[o][7]) {
                        const int* bx = s_box[o];
                        v = value_noise_box(px, py, pz, cache + bx[6], bx[0], bx[1], bx[2], bx[3], bx[4], bx[5]);
                    } else {
                        const uint32_t* key = src.keys + 3 * o;
                        v = value_noise(px, py, pz, __ldg(key), __ldg(key + 1), __ldg(key + 2));
                    }
                    sum = fmaf(amp, v, sum);
                    freq *= src.lacunarity;
                    amp *= src.gain;
                }
                Sf[e] = src.amplitude * sum;
            }
        }
    } else {
        __shared__ BumpSmem bump;
        for (int e = tid; e < Si * Sj; e += 256) {
            const int ii = i0 + e % Si, jj = j0 + e / Si;
            float v = 0.0f;
            if (src.kind == SHM_SRC_SAMPLES)
                v = __ldg(src.samples + __ldg(src.sample_offset + g) + ((int64_t)f * S + jj) * S + ii) - Gr.r0;
            Sf[e] = v;
        }
        if (src.kind == SHM_SRC_BUMPS) {
            base = 1.0f - Gr.r0;
            const int64_t b_lo = __ldg(src.bump_offset + g), b_hi = __ldg(src.bump_offset + g + 1);
            for (int64_t bc = b_lo; bc < b_hi; bc += MAX_BUMPS_SMEM) {
                const int nb = (int)min((int64_t)MAX_BUMPS_SMEM, b_hi - bc);
                __syncthreads();
                stage_bumps(bump, src, bc, nb);
                __syncthreads();
                // two samples per thread at a time (e and e + 256), the last odd one alone
                for (int e = tid; e < Si * Sj; e += 512) {
                    const int e2 = e + 256;
                    if (e2 < Si * Sj) {
                        const float2 v = bump_sum2(bump, nb, dir(i0 + e % Si, j0 + e / Si), dir(i0 + e2 % Si, j0 + e2 / Si),
                                                   make_float2(Sf[e], Sf[e2]));
                        Sf[e] = v.x;
                        Sf[e2] = v.y;
                    } else {
                        Sf[e] = bump_sum(bump, nb, dir(i0 + e % Si, j0 + e / Si), Sf[e]);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < ti * tj; e += 256) {
        const int li = e % ti, lj = e / ti;
        const float* c = Sf + (lj + 1) * Si + (li + 1);  // texel (i0+li, j0+lj) is local sample (li+1, lj+1)
        float4 v;
        v.x = c[0] + base;
        v.y = 0.5f * (c[1] - c[-1]);
        v.z = 0.5f * (c[Si] - c[-Si]);
        v.w = 0.25f * ((c[Si + 1] - c[-Si + 1]) - (c[Si - 1] - c[-Si - 1]));
        store_texel(data, out.dtype, out.layout, Gr, f, j0 + lj, i0 + li, v);
    }
}

static int64_t value_tiles(int N)
{
    const int64_t t = (N + 4 + FS - 1) / FS;
    return t * t;
}

cudaError_t launch_fd_build(const LutView& out, void* data, const shm_source& src, const Sizes& sz, cudaStream_t s)
{
    if (out.layout == SHM_LAYOUT_VALUE)
        return for_each_glyph_chunk(sz, value_tiles, [&](unsigned bx, unsigned bz, const auto& map) {
            k_value_build<std::decay_t<decltype(map)>><<<dim3(bx, 6, bz), 256, 0, s>>>(out, data, src, map);
        });
    {
        int T = (sz.max_N <= FACE_N_MAX) ? sz.max_N + 2 : REGION_T;
        if (sz.N_uniform == 0 && T > FACE_SPLIT_T) T = FACE_SPLIT_T;
        if (sz.N_uniform > 0 && T <= FACE_N_MAX + 2 && (T + 2) * (T + 2) * (int)sizeof(float) > FACE_SPLIT_SMEM)
            T = (T + 1) / 2;
        const int smem = (T + 2) * (T + 2) * (int)sizeof(float);
        const int mi = sz.N_uniform > 0 ? 0 : 1, fi = src.kind == SHM_SRC_FBM ? 1 : 0;
        {
            const void* fn = fi ? (mi == 0 ? (const void*)k_fd_face<true, UniformMap> : (const void*)k_fd_face<true, TileMap>)
                                : (mi == 0 ? (const void*)k_fd_face<false, UniformMap> : (const void*)k_fd_face<false, TileMap>);
            cudaError_t e = ensure_dynamic_smem(fn, smem);
            if (e != cudaSuccess) return e;
        }
        auto regions = [T](int N) {
            const int64_t r = (N + 2 + T - 1) / T;
            return r * r;
        };
        return for_each_glyph_chunk(sz, regions, [&](unsigned bx, unsigned bz, const auto& map) {
            using M = std::decay_t<decltype(map)>;
            if (fi) k_fd_face<true, M><<<dim3(bx, 6, bz), 256, smem, s>>>(out, data, src, T, map);
            else k_fd_face<false, M><<<dim3(bx, 6, bz), 256, smem, s>>>(out, data, src, T, map);
        });
    }
}

// ------------------------------------------------------------------------------------------
// Value table of SH glyphs (SHM_LAYOUT_VALUE): r at every texel centre of the two-texel-gutter
// grid.  One thread per grid entry: the K basis values of its direction are formed once and
// applied to SH_VALUE_GLYPHS glyphs (blockIdx.y picks the glyph group).
constexpr int SH_VALUE_GLYPHS = 32;

__global__ void __launch_bounds__(128) k_sh_value(LutView out, void* data, int L, const float* __restrict__ coeffs)
{
    const int N = out.N_uniform, S = N + 4;
    const int64_t T = 6LL * S * S;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= T) return;
    const int f = (int)(e / ((int64_t)S * S)), rem = (int)(e % ((int64_t)S * S)), jj = rem / S, ii = rem % S;
    // texel (ii-1, jj-1): 2u - 1 = (2(ii-1) - 1 - N)/N
    const float X = (float)(2 * ii - 3 - N) / (float)N, Y = (float)(2 * jj - 3 - N) / (float)N;
    const TexelFrame fr = texel_frame(f, X, Y);
    const int K = (L + 1) * (L + 1);
    float Tl[(SH_LMAX + 1) * (SH_LMAX + 2) / 2];
    float C[SH_LMAX + 1], Sn[SH_LMAX + 1];
    legendre_table(L, fr.w.z, Tl);
    cs_table(L, fr.w.x, fr.w.y, C, Sn);
    const int g0 = blockIdx.y * SH_VALUE_GLYPHS, g1 = min(out.n_glyphs, g0 + SH_VALUE_GLYPHS);
    float acc[SH_VALUE_GLYPHS];
#pragma unroll
    for (int q = 0; q < SH_VALUE_GLYPHS; ++q) acc[q] = 0.0f;
    for (int l = 0; l <= L; ++l)
        for (int mm = -l; mm <= l; ++mm) {
            const int m = mm < 0 ? -mm : mm;
            const float y = ylm_derivs(Tl, l, m, mm < 0, C, Sn).v;
            const int k = l * l + l + mm;
#pragma unroll
            for (int q = 0; q < SH_VALUE_GLYPHS; ++q)
                if (g0 + q < g1) acc[q] = fmaf(__ldg(coeffs + (int64_t)(g0 + q) * K + k), y, acc[q]);
        }
    for (int q = 0; q < SH_VALUE_GLYPHS && g0 + q < g1; ++q) {
        const GlyphRef G = glyph_ref(out, g0 + q);
        store_val(data, out.dtype, G.base + e, acc[q] - G.r0);
    }
}

cudaError_t launch_sh_value(const LutView& out, void* data, int L, const float* coeffs, cudaStream_t s)
{
    const int S = out.N_uniform + 4;
    const int64_t T = 6LL * S * S;
    const unsigned gy = (unsigned)((out.n_glyphs + SH_VALUE_GLYPHS - 1) / SH_VALUE_GLYPHS);
    if (gy > 65535u) return cudaErrorInvalidConfiguration;
    k_sh_value<<<dim3((unsigned)((T + 127) / 128), gy), 128, 0, s>>>(out, data, L, coeffs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Pack: one thread per destination record.
constexpr int PACK_PER_BLOCK = 1024;

template <class Map>
__global__ void __launch_bounds__(256) k_pack(LutView src, LutView dst, void* ddata, const __grid_constant__ Map map)
{
    int blk;
    const int g = map_block(map, blk);
    const GlyphRef Gs = glyph_ref(src, g), Gd = glyph_ref(dst, g);
    const int N = Gd.N;
    const int64_t nrec = records_per_glyph(N, dst.layout);
    const int64_t r_end = min(nrec, (int64_t)(blk + 1) * PACK_PER_BLOCK);
    for (int64_t r = (int64_t)blk * PACK_PER_BLOCK + threadIdx.x; r < r_end; r += blockDim.x) {
        const float dr0 = Gs.r0 - Gd.r0;
        if (dst.layout == SHM_LAYOUT_TEXEL) {
            const int P = N + 2;
            const int f = (int)(r / ((int64_t)P * P)), rem = (int)(r % ((int64_t)P * P)), j = rem / P, i = rem % P;
            float4 v = load_texel(src.data, src.dtype, src.layout, Gs, f, j, i);
            v.x += dr0;
            store_rec(ddata, dst.dtype, Gd.base + r, v);
        } else {
            const int P = N + 1;
            const int f = (int)(r / ((int64_t)P * P)), rem = (int)(r % ((int64_t)P * P)), j = rem / P, i = rem % P;
            for (int corner = 0; corner < 4; ++corner) {
                float4 v = load_texel(src.data, src.dtype, src.layout, Gs, f, j + (corner >> 1), i + (corner & 1));
                v.x += dr0;
                store_rec(ddata, dst.dtype, (Gd.base + r) * 4 + corner, v);
            }
        }
    }
}

cudaError_t launch_pack(const LutView& src, const LutView& dst, void* dst_data, const Sizes& sz, cudaStream_t s)
{
    const int layout = dst.layout;
    auto blocks = [layout](int N) { return (records_per_glyph(N, layout) + PACK_PER_BLOCK - 1) / PACK_PER_BLOCK; };
    return for_each_glyph_chunk(sz, blocks, [&](unsigned bx, unsigned bz, const auto& map) {
        k_pack<<<dim3(bx, 1, bz), 256, 0, s>>>(src, dst, dst_data, map);
    });
}

// ------------------------------------------------------------------------------------------
// Bounds: per cell, |r| <= max|r0 + r_ab| + (max|r_u h| + max|r_v h|)/4 + max|r_uv h^2|/16 over the
// cell's four corners (value weights are >= 0 and sum to 1; sum_a |H^d_a| = s(1-s) <= 1/4).
constexpr int BOUNDS_PER_BLOCK = 2048;

template <int DT, int LAYOUT>
__device__ __forceinline__ float cell_bound(const LutView& L, const GlyphRef& G, int f, int i, int j)
{
    const Corners cr = fetch_corners<DT, LAYOUT>(L.data, G, f, i, j);
    const float4 v[4] = {cr.c00, cr.c10, cr.c01, cr.c11};
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        m0 = fmaxf(m0, fabsf(G.r0 + v[k].x));
        m1 = fmaxf(m1, fabsf(v[k].y));
        m2 = fmaxf(m2, fabsf(v[k].z));
        m3 = fmaxf(m3, fabsf(v[k].w));
    }
    return m0 + 0.25f * (m1 + m2) + 0.0625f * m3;
}

template <int DT, int LAYOUT, class Map>
__global__ void __launch_bounds__(256) k_bounds(LutView L, float* rmax, const __grid_constant__ Map map)
{
    __shared__ float warp_best[8];
    int blk;
    const int g = map_block(map, blk);
    const GlyphRef G = glyph_ref(L, g);
    const int N = G.N, P = N + 1;
    const int64_t ncell = 6LL * P * P;
    const int64_t c_end = min(ncell, (int64_t)(blk + 1) * BOUNDS_PER_BLOCK);
    float best = 0.0f;
    if (ncell <= 0x7fffffff) {  // 32-bit cell arithmetic (N < 18,900)
        const uint32_t PP = (uint32_t)P * (uint32_t)P;
        for (uint32_t c = (uint32_t)blk * BOUNDS_PER_BLOCK + threadIdx.x; c < (uint32_t)c_end; c += blockDim.x) {
            const uint32_t f = c / PP, rem = c - f * PP, j = rem / (uint32_t)P, i = rem - j * (uint32_t)P;
            best = fmaxf(best, cell_bound<DT, LAYOUT>(L, G, (int)f, (int)i, (int)j));
        }
    } else {
        for (int64_t c = (int64_t)blk * BOUNDS_PER_BLOCK + threadIdx.x; c < c_end; c += blockDim.x) {
            const int f = (int)(c / ((int64_t)P * P)), rem = (int)(c % ((int64_t)P * P)), j = rem / P, i = rem % P;
            best = fmaxf(best, cell_bound<DT, LAYOUT>(L, G, f, i, j));
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) warp_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) best = fmaxf(best, warp_best[w]);
        // non-negative floats order like their bit patterns
        atomicMax(reinterpret_cast<int*>(rmax + g), __float_as_int(best));
    }
}

cudaError_t launch_bounds(const LutView& L, float* rmax, const Sizes& sz, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(rmax, 0, sizeof(float) * (size_t)L.n_glyphs, s);
    if (e != cudaSuccess) return e;
    auto blocks = [](int N) { return (6LL * (N + 1) * (N + 1) + BOUNDS_PER_BLOCK - 1) / BOUNDS_PER_BLOCK; };
    return for_each_glyph_chunk(sz, blocks, [&](unsigned bx, unsigned bz, const auto& map) {
        using M = std::decay_t<decltype(map)>;
        const dim3 grid(bx, 1, bz);
        if (L.layout == SHM_LAYOUT_TEXEL) {
            if (L.dtype == SHM_F32) k_bounds<SHM_F32, SHM_LAYOUT_TEXEL, M><<<grid, 256, 0, s>>>(L, rmax, map);
            else if (L.dtype == SHM_F16) k_bounds<SHM_F16, SHM_LAYOUT_TEXEL, M><<<grid, 256, 0, s>>>(L, rmax, map);
            else k_bounds<SHM_BF16, SHM_LAYOUT_TEXEL, M><<<grid, 256, 0, s>>>(L, rmax, map);
        } else {
            if (L.dtype == SHM_F32) k_bounds<SHM_F32, SHM_LAYOUT_CELL, M><<<grid, 256, 0, s>>>(L, rmax, map);
            else if (L.dtype == SHM_F16) k_bounds<SHM_F16, SHM_LAYOUT_CELL, M><<<grid, 256, 0, s>>>(L, rmax, map);
            else k_bounds<SHM_BF16, SHM_LAYOUT_CELL, M><<<grid, 256, 0, s>>>(L, rmax, map);
        }
    });
}

// ------------------------------------------------------------------------------------------
// Direct SH: r = sum_k c_k Y_k(w), Euclidean gradient of the polynomial projected onto the tangent
// plane gives grad_{S^2} r, then the §3.4 normal.
__global__ void __launch_bounds__(128) k_sh_eval(int L, int G, const float* __restrict__ coeffs, int64_t Q,
                                                 const float* __restrict__ dirs, const int32_t* __restrict__ glyph,
                                                 const int64_t* __restrict__ seg, float* R, float* grad,
                                                 float* normal, int32_t* dev_status)
{
    const int K = (L + 1) * (L + 1);
    uint32_t status = 0;
    const float qnan = __int_as_float(0x7fc00000);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
        int g = 0;
        if (glyph) g = __ldg(glyph + q);
        else if (seg) g = (q < __ldg(seg)) ? -1 : seg_find(seg, G, q);
        const float d0 = __ldg(dirs + 3 * q), d1 = __ldg(dirs + 3 * q + 1), d2 = __ldg(dirs + 3 * q + 2);
        const float n2 = d0 * d0 + d1 * d1 + d2 * d2;
        bool ok = (g >= 0 && g < G);
        if (!ok) status |= SHM_DEV_BOUNDS;
        if (ok && !(n2 > 0.0f && n2 <= 3.0e38f)) { ok = false; status |= SHM_DEV_NONFINITE; }
        float r = qnan;
        Vec3 gs{qnan, qnan, qnan}, nn{qnan, qnan, qnan};
        if (ok) {
            const float il = rsqrtf(n2);
            const Vec3 w{d0 * il, d1 * il, d2 * il};
            float Tl[(SH_LMAX + 1) * (SH_LMAX + 2) / 2];
            float C[SH_LMAX + 1], S[SH_LMAX + 1];
            legendre_table(L, w.z, Tl);
            cs_table(L, w.x, w.y, C, S);
            const float* c = coeffs + (int64_t)g * K;
            float rv = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
            for (int l = 0; l <= L; ++l)
                for (int mm = -l; mm <= l; ++mm) {
                    const int m = mm < 0 ? -mm : mm;
                    const YDer y = ylm_derivs(Tl, l, m, mm < 0, C, S);
                    const float ck = __ldg(c + l * l + l + mm);
                    rv = fmaf(ck, y.v, rv);
                    gx = fmaf(ck, y.gx, gx);
                    gy = fmaf(ck, y.gy, gy);
                    gz = fmaf(ck, y.gz, gz);
                }
            const float wg = w.x * gx + w.y * gy + w.z * gz;
            r = rv;
            gs = Vec3{gx - w.x * wg, gy - w.y * wg, gz - w.z * wg};
            nn = surface_normal(d0, d1, d2, r, gs);
        }
        if (R) R[q] = r;
        if (grad) { grad[3 * q] = gs.x; grad[3 * q + 1] = gs.y; grad[3 * q + 2] = gs.z; }
        if (normal) { normal[3 * q] = nn.x; normal[3 * q + 1] = nn.y; normal[3 * q + 2] = nn.z; }
    }
    report_status(dev_status, status);
}

cudaError_t launch_sh_eval(int L, int G, const float* coeffs, int64_t Q, const float* dirs, const int32_t* glyph,
                           const int64_t* seg, float* R, float* grad, float* normal, int32_t* dev_status,
                           cudaStream_t s)
{
    if (Q == 0) return cudaSuccess;
    int64_t blocks = (Q + 127) / 128;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    k_sh_eval<<<(unsigned)blocks, 128, 0, s>>>(L, G, coeffs, Q, dirs, glyph, seg, R, grad, normal, dev_status);
    return cudaGetLastError();
}

}  // namespace shm
