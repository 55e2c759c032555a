// Internal launch interfaces between the C-ABI layer (shm_api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <type_traits>
#include <vector>

#include "../../include/shm.h"
#include "shm_device.cuh"

namespace shm {

// ------------------------------------------------------------------------------------------
// Per-glyph block grids.  A pool with per-glyph resolutions would need max-N-sized grids per
// glyph, most of whose blocks exit at once (512 glyphs of N in {16..128}: ~60 % empty blocks).
// Instead the host, which reads the resolutions anyway, passes a prefix of per-glyph block counts
// by value (a __grid_constant__ kernel parameter of up to ~8 KB), and each block finds its glyph
// by a block-uniform binary search; the grid is exactly the work.  Uniform pools keep a
// (blocks, faces, glyphs) grid.
struct Sizes {
    int G;
    int N_uniform;              // > 0: every glyph has this N
    const int32_t* N_host;      // otherwise: host copy of the per-glyph N
    int max_N;
};

constexpr int TILEMAP_MAX = 2000;

struct UniformMap {
    int32_t g0;
};

struct TileMap {
    int32_t g0, n;
    int32_t cum[TILEMAP_MAX + 1];  // cum[k]: first block of glyph g0 + k; cum[n]: blocks in this launch
};

__device__ __forceinline__ int map_block(const UniformMap& m, int& local)
{
    local = blockIdx.x;
    return m.g0 + blockIdx.z;
}

__device__ __forceinline__ int map_block(const TileMap& m, int& local)
{
    const int b = blockIdx.x;
    int lo = 0, hi = m.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (m.cum[mid] <= b) lo = mid;
        else hi = mid;
    }
    local = b - m.cum[lo];
    return m.g0 + lo;
}

// Calls launch(grid_x, grid_z, map) once per chunk of glyphs, with blocks_of(N) blocks per glyph
// along x.  Glyphs with zero blocks are skipped by the search (equal prefixes).
template <class BlocksOf, class Launch>
cudaError_t for_each_glyph_chunk(const Sizes& sz, BlocksOf blocks_of, Launch launch)
{
    if (sz.N_uniform > 0) {
        const int64_t b = blocks_of(sz.N_uniform);
        if (b <= 0) return cudaSuccess;
        if (b > 0x7fffffff) return cudaErrorInvalidConfiguration;
        for (int g0 = 0; g0 < sz.G; g0 += 65535)
            launch((unsigned)b, (unsigned)(sz.G - g0 < 65535 ? sz.G - g0 : 65535), UniformMap{g0});
        return cudaGetLastError();
    }
    std::unique_ptr<TileMap> m(new TileMap);
    for (int g0 = 0; g0 < sz.G;) {
        m->g0 = g0;
        m->cum[0] = 0;
        int n = 0;
        int64_t total = 0;
        while (g0 + n < sz.G && n < TILEMAP_MAX) {
            const int64_t b = blocks_of(sz.N_host[g0 + n]);
            if (n > 0 && total + b > 0x7fffffff) break;
            if (b > 0x7fffffff) return cudaErrorInvalidConfiguration;
            total += b;
            m->cum[++n] = (int32_t)total;
        }
        m->n = n;
        if (total > 0) launch((unsigned)total, 1u, *m);
        g0 += n;
    }
    return cudaGetLastError();
}

struct QueryArgs {
    LutView L;
    int64_t Q;
    const float* dirs;
    const int32_t* glyph;
    const int64_t* seg;
    float* R;
    float* grad;
    float* normal;
    float* chart;
    int32_t* fij;
    int32_t* dev_status;
};

struct BackwardArgs {
    LutView L;       // table read by the forward
    LutView D;       // float32 texel-layout gradient table (written with atomics)
    float* dlut;     // D.data, writable
    int64_t Q;
    const float* dirs;
    const int32_t* glyph;
    const int64_t* seg;
    const float* gR;
    const float* ggrad;
    const float* gnormal;
    float* ddirs;
    int32_t* dev_status;
    // fused fit loss (fit != 0): upstream gradients from L = sum_q w_v (R - R_t)^2 + w_n |n - n_t|^2
    int fit;
    const float* R_target;
    const float* n_target;
    float w_value, w_normal;
    float* loss;  // accumulated (+=) sum of the per-query losses
};

int sm_count();

// Raises kernel fn's dynamic shared-memory limit to at least `bytes` on the calling thread's
// current device.  The attribute belongs to the device's context, so it is tracked per (kernel,
// device); thread-safe.
cudaError_t ensure_dynamic_smem(const void* fn, int bytes);

cudaError_t launch_query_fwd(const QueryArgs& a, cudaStream_t s);
cudaError_t launch_query_bwd_det(const BackwardArgs& a, cudaStream_t s);
// Glyph tables up to this size are staged whole in shared memory by the segment query (two CTAs
// of 512 threads per SM: (232,448 - 2 x 1 KB reserved) / 2 minus the barrier block).
constexpr int64_t STAGED_TABLE_MAX_BYTES = 114688;
cudaError_t launch_query_staged(const QueryArgs& a, int shape, cudaStream_t s);
int staged_shapes();
// Launch shapes and the per-device tuning table (shm_query.cu).
bool query_is_staged(const QueryArgs& a);
int query_shapes(const QueryArgs& a);
cudaError_t launch_query_shape(const QueryArgs& a, int shape, cudaStream_t s);
int tuned_query_shape(const QueryArgs& a);
void set_tuned_query_shape(const QueryArgs& a, int shape);
void reset_tuned_shapes();
// Binned query of one large table (shm_query_binned.cu): partition by (face, band of cell rows)
// so that the bands in flight stay in L2, query in partitioned order, restore query order.
constexpr int64_t BINNED_DEFAULT_BAND_BYTES = 32ll << 20;
int64_t binned_workspace_bytes(const LutView& L, int64_t Q, int64_t band_bytes);
int binned_bins(const LutView& L, int64_t band_bytes, int* band_rows);
cudaError_t launch_query_binned(const QueryArgs& a, int64_t band_bytes, void* ws, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_query_bwd(const BackwardArgs& a, cudaStream_t s);
cudaError_t launch_adam(float* param, float* grad, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                        float eps, int step, int zero_grad, cudaStream_t s);

cudaError_t launch_sh_basis(int N, int L, float* basis, cudaStream_t s);
cudaError_t launch_basis_split(int N, int L, float* basis, cudaStream_t s);
cudaError_t launch_sh_build_tc(const LutView& out, void* data, int L, const float* coeffs, const float* basis,
                               void* ws, cudaStream_t s, int32_t* dev_status);
int sh_kpad(int L);
int64_t sh_build_workspace_bytes(int G, int L);
cudaError_t launch_sh_build(const LutView& out, void* data, int L, const float* coeffs, const float* basis,
                            cudaStream_t s);
cudaError_t launch_sh_build_bwd(int N, int G, int L, const float* dlut, const float* basis, float* dcoeffs, bool det,
                                cudaStream_t s);
cudaError_t launch_sh_build_bwd_tc(int N, int G, int L, const float* dlut, const float* basis, float* dcoeffs,
                                   int32_t* dev_status, cudaStream_t s);
cudaError_t launch_basis_split_t(int N, int L, float* basis, cudaStream_t s);
cudaError_t launch_sh_value(const LutView& out, void* data, int L, const float* coeffs, cudaStream_t s);
cudaError_t launch_query_recon(const QueryArgs& a, int method, cudaStream_t s);
cudaError_t launch_fd_build(const LutView& out, void* data, const shm_source& src, const Sizes& sz, cudaStream_t s);
cudaError_t launch_pack(const LutView& src, const LutView& dst, void* dst_data, const Sizes& sz, cudaStream_t s);
cudaError_t launch_bounds(const LutView& L, float* rmax, const Sizes& sz, cudaStream_t s);
cudaError_t launch_mip(const LutView& fine, const LutView& coarse, void* cdata, int32_t* dev_status,
                       const Sizes& coarse_sz, cudaStream_t s);
cudaError_t launch_sh_eval(int L, int G, const float* coeffs, int64_t Q, const float* dirs, const int32_t* glyph,
                           const int64_t* seg, float* R, float* grad, float* normal, int32_t* dev_status,
                           cudaStream_t s);
cudaError_t launch_raycast(const LutView& L, const shm_object* objs, int n_obj, const shm_camera& cam,
                           const shm_raycast_params& prm, float* rgba, float* depth, float* normal,
                           int32_t* obj_id, void* ws, size_t ws_bytes, int32_t* dev_status, cudaStream_t s);
int64_t raycast_workspace_bytes(int n_obj, int W, int H);

// Warp-aggregated OR of device status bits.
__device__ __forceinline__ void report_status(int32_t* dev_status, uint32_t bits)
{
    const uint32_t any = __reduce_or_sync(0xffffffffu, bits);
    if (dev_status && any && (threadIdx.x & 31) == 0) atomicOr(dev_status, (int)any);
}

// Largest g in [0, G] with seg[g] <= q (q >= seg[0] assumed; g == G means q is past the end).
__device__ __forceinline__ int seg_find(const int64_t* seg, int G, int64_t q)
{
    int lo = 0, hi = G + 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(seg + mid) <= q) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace shm
