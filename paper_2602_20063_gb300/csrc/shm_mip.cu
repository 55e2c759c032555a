// Derivative-consistent mip level (§4.7, Table lod) of a Spherical Hermite Map.
//
// A coarse table of resolution Nc = Nf/2 on the same cell-centred chart is baked from the fine
// table: the scalar field is filtered, then the derivative channels are recomputed from the
// filtered values by central differences in (u, v) (box-filtering the stored derivative channels
// the way hardware mipmapping treats RGBA breaks their meaning as scaled chart derivatives).
// Filter: the coarse sample at coarse texel ic is the mean of the fine interpolant at the centres
// of the fine texels 2ic-1 and 2ic along each axis (they straddle the coarse centre symmetrically).
// Child directions outside the face, on the gutter ring and the one-texel bake margin, are
// ordinary queries that land on the neighbouring face, so the seam treatment of the fine level is
// inherited.  Inside the face a child sits exactly on a fine texel centre, where the interpolant
// equals the stored value (§3.3): the four children of an interior coarse texel are the corners of
// fine cell (2ic-1, 2jc-1), read with one footprint fetch and no interpolation.
//
// One CTA per (16 x 16 coarse-texel tile, face, glyph): 18 x 18 margin samples (4 fine queries
// each, value only) into shared memory, then one record per thread, stored in any dtype/layout.
#include "shm_internal.h"

namespace shm {

namespace {

constexpr int MT = 16, MS = MT + 2;

template <int DT, int LAYOUT, class Map>
__global__ void __launch_bounds__(256) k_mip(LutView fine, LutView coarse, void* cdata, int32_t* dev_status,
                                             const __grid_constant__ Map map)
{
    __shared__ float Sm[MS][MS];
    int tile;
    const int g = map_block(map, tile), f = blockIdx.y;
    const GlyphRef Gc = glyph_ref(coarse, g), Gf = glyph_ref(fine, g);
    const int Nc = Gc.N, Nf = Gf.N, P = Nc + 2, S = Nc + 4;
    const int tiles = (P + MT - 1) / MT;
    if (tile >= tiles * tiles) return;
    const int i0 = (tile % tiles) * MT, j0 = (tile / tiles) * MT;
    const int tid = threadIdx.x;
    const bool paired = (Nf == 2 * Nc);
    if (!paired && tid == 0 && tile == 0 && f == 0 && dev_status) atomicOr(dev_status, SHM_DEV_BOUNDS);

    const int k = f >> 1, k1 = (k + 1) % 3;
    const float sg = (f & 1) ? -1.0f : 1.0f;
    const float dr0 = Gf.r0 - Gc.r0;
    for (int e = tid; e < MS * MS; e += 256) {
        const int ii = i0 + (e % MS), jj = j0 + (e / MS);
        float acc = 0.0f;
        const int ic = ii - 1, jc = jj - 1;
        if (paired && ii < S && jj < S && ic >= 1 && ic <= Nc && jc >= 1 && jc <= Nc) {
            const Corners cr = fetch_corners<DT, LAYOUT>(fine.data, Gf, f, 2 * ic - 1, 2 * jc - 1);
            acc = 0.25f * (((cr.c00.x + cr.c10.x) + cr.c01.x) + cr.c11.x) + dr0;
        } else if (paired && ii < S && jj < S) {
            // sample (ii, jj) is coarse texel (ii-1, jj-1); its children are fine texels
            // 2(ii-1)-1+a, a in {0, 1}, at 2u-1 = (2 i_f - 1 - Nf)/Nf
            for (int b = 0; b < 2; ++b) {
                const int jf = 2 * jj - 3 + b;
                const float Y = __fdiv_rn((float)(2 * jf - 1 - Nf), (float)Nf);
                for (int a = 0; a < 2; ++a) {
                    const int i_f = 2 * ii - 3 + a;
                    const float X = __fdiv_rn((float)(2 * i_f - 1 - Nf), (float)Nf);
                    // direction a + X b + Y c of face f (axis k with sign sg; b = e_k1, c = e_k2)
                    const float d0 = (k == 0) ? sg : (k1 == 0 ? X : Y);
                    const float d1 = (k == 1) ? sg : (k1 == 1 ? X : Y);
                    const float d2 = (k == 2) ? sg : (k1 == 2 ? X : Y);
                    Chart c;
                    chart_of(d0, d1, d2, c);  // |d| >= 1: always a valid direction
                    int i, j;
                    float s, t;
                    cell_of(pick3(c.k1, d0, d1, d2), c.m, c.im, Nf, i, s);
                    cell_of(pick3(c.k2, d0, d1, d2), c.m, c.im, Nf, j, t);
                    const Corners cr = fetch_corners<DT, LAYOUT>(fine.data, Gf, c.f, i, j);
                    acc += hermite2(cr, s, t).r;
                }
            }
            acc = 0.25f * acc + dr0;
        }
        Sm[e / MS][e % MS] = acc;
    }
    __syncthreads();
    const int ti = tid % MT, tj = tid / MT;
    const int i = i0 + ti, j = j0 + tj;
    if (i >= P || j >= P) return;
    const int si = ti + 1, sj = tj + 1;
    float4 v;
    if (paired) {
        v.x = Sm[sj][si];
        v.y = 0.5f * (Sm[sj][si + 1] - Sm[sj][si - 1]);
        v.z = 0.5f * (Sm[sj + 1][si] - Sm[sj - 1][si]);
        v.w = 0.25f * ((Sm[sj + 1][si + 1] - Sm[sj - 1][si + 1]) - (Sm[sj + 1][si - 1] - Sm[sj - 1][si - 1]));
    } else {
        v = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                        __int_as_float(0x7fc00000));
    }
    store_texel(cdata, coarse.dtype, coarse.layout, Gc, f, j, i, v);
}

template <int DT, int LAYOUT>
cudaError_t launch_mip_t(const LutView& fine, const LutView& coarse, void* cdata, int32_t* st, const Sizes& sz,
                         cudaStream_t s)
{
    auto tiles = [](int Nc) {
        const int64_t t = (Nc + 2 + MT - 1) / MT;
        return t * t;
    };
    return for_each_glyph_chunk(sz, tiles, [&](unsigned bx, unsigned bz, const auto& map) {
        k_mip<DT, LAYOUT><<<dim3(bx, 6, bz), 256, 0, s>>>(fine, coarse, cdata, st, map);
    });
}

}  // namespace

cudaError_t launch_mip(const LutView& fine, const LutView& coarse, void* cdata, int32_t* dev_status,
                       const Sizes& coarse_sz, cudaStream_t s)
{
    const bool cell = fine.layout == SHM_LAYOUT_CELL;
    const Sizes& z = coarse_sz;
    switch (fine.dtype) {
    case SHM_F32:
        return cell ? launch_mip_t<SHM_F32, SHM_LAYOUT_CELL>(fine, coarse, cdata, dev_status, z, s)
                    : launch_mip_t<SHM_F32, SHM_LAYOUT_TEXEL>(fine, coarse, cdata, dev_status, z, s);
    case SHM_F16:
        return cell ? launch_mip_t<SHM_F16, SHM_LAYOUT_CELL>(fine, coarse, cdata, dev_status, z, s)
                    : launch_mip_t<SHM_F16, SHM_LAYOUT_TEXEL>(fine, coarse, cdata, dev_status, z, s);
    default:
        return cell ? launch_mip_t<SHM_BF16, SHM_LAYOUT_CELL>(fine, coarse, cdata, dev_status, z, s)
                    : launch_mip_t<SHM_BF16, SHM_LAYOUT_TEXEL>(fine, coarse, cdata, dev_status, z, s);
    }
}

}  // namespace shm
