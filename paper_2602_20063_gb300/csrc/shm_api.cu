// C-ABI entry points of libshm.so (declared in include/shm.h): host-side validation, dispatch
// to the kernel launchers, CUDA error mapping.  No device memory is allocated here.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <vector>

#include "shm_internal.h"

namespace shm {

cudaError_t ensure_dynamic_smem(const void* fn, int bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> set;  // (kernel, device) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int& cur = set[{fn, dev}];
    if (cur >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

static bool valid_dtype(int d) { return d == SHM_F32 || d == SHM_F16 || d == SHM_BF16; }
static bool valid_layout(int l) { return l == SHM_LAYOUT_TEXEL || l == SHM_LAYOUT_CELL || l == SHM_LAYOUT_VALUE; }
static bool hermite_layout(int l) { return l == SHM_LAYOUT_TEXEL || l == SHM_LAYOUT_CELL; }

static shm_status check_lut(const shm_lut* L)
{
    if (!L || !L->data || L->n_glyphs <= 0) return SHM_ERR_INVALID_ARG;
    if (!valid_dtype(L->dtype) || !valid_layout(L->layout)) return SHM_ERR_INVALID_ARG;
    if (L->N_uniform < 0) return SHM_ERR_INVALID_ARG;
    if (L->N_uniform == 0 && (!L->N || !L->offset)) return SHM_ERR_INVALID_ARG;
    if (L->N_uniform > (1 << 20)) return SHM_ERR_INVALID_ARG;
    if (((uintptr_t)L->data & 15u) != 0) return SHM_ERR_INVALID_ARG;
    // cell records are read with 256-bit loads: the pool must be 32-byte aligned
    if (L->layout == SHM_LAYOUT_CELL && ((uintptr_t)L->data & 31u) != 0) return SHM_ERR_INVALID_ARG;
    return SHM_OK;
}

static LutView view(const shm_lut* L)
{
    LutView v;
    v.data = L->data;
    v.N = L->N;
    v.offset = L->offset;
    v.r0 = L->r0;
    v.n_glyphs = L->n_glyphs;
    v.N_uniform = L->N_uniform;
    v.dtype = L->dtype;
    v.layout = L->layout;
    return v;
}

static shm_status map_cuda(cudaError_t e) { return e == cudaSuccess ? SHM_OK : SHM_ERR_CUDA; }

// Per-query input and output buffers may live in device memory or in page-locked host memory
// (cudaHostAlloc / cudaHostRegister): the kernels then read and write the host buffer directly over
// the host link, through the pointer's device alias.  Pageable host memory is rejected, so that no
// kernel ever dereferences an address the device cannot reach.
template <class T>
static shm_status io_ptr(T*& p)
{
    if (!p) return SHM_OK;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, (const void*)p) != cudaSuccess) {
        (void)cudaGetLastError();
        return SHM_ERR_INVALID_ARG;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return SHM_OK;
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        p = static_cast<T*>(at.devicePointer);
        return SHM_OK;
    }
    return SHM_ERR_INVALID_ARG;
}

// The gradient table of a reverse pass must have the table's glyphs and resolutions (its records
// are addressed with the table's N).  Per-glyph resolutions are compared on the host.
static shm_status same_resolutions(const shm_lut* a, const shm_lut* b, cudaStream_t s)
{
    if (a->n_glyphs != b->n_glyphs) return SHM_ERR_INVALID_ARG;
    if (a->N_uniform > 0 || b->N_uniform > 0) return a->N_uniform == b->N_uniform ? SHM_OK : SHM_ERR_INVALID_ARG;
    if (a->N == b->N) return SHM_OK;
    // per-glyph arrays are compared on the host, which needs a synchronisation: not possible while
    // the stream is being captured into a graph, where the check is skipped
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return SHM_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SHM_OK;
    std::vector<int32_t> na(a->n_glyphs), nb(b->n_glyphs);
    if (cudaMemcpyAsync(na.data(), a->N, sizeof(int32_t) * na.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(nb.data(), b->N, sizeof(int32_t) * nb.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SHM_ERR_CUDA;
    return na == nb ? SHM_OK : SHM_ERR_INVALID_ARG;
}

static shm_status resolve_io(QueryArgs& a)
{
    shm_status st = SHM_OK;
    for (shm_status e : {io_ptr(a.dirs), io_ptr(a.glyph), io_ptr(a.seg), io_ptr(a.R), io_ptr(a.grad),
                         io_ptr(a.normal), io_ptr(a.chart), io_ptr(a.fij), io_ptr(a.dev_status)})
        if (e != SHM_OK) st = e;
    return st;
}

static shm_status resolve_io(BackwardArgs& a)
{
    shm_status st = SHM_OK;
    for (shm_status e : {io_ptr(a.dirs), io_ptr(a.glyph), io_ptr(a.seg), io_ptr(a.gR), io_ptr(a.ggrad),
                         io_ptr(a.gnormal), io_ptr(a.ddirs), io_ptr(a.dev_status), io_ptr(a.R_target),
                         io_ptr(a.n_target), io_ptr(a.loss)})
        if (e != SHM_OK) st = e;
    return st;
}

// Glyph resolutions for the launch grids: uniform N, or the per-glyph array read from the device
// (one synchronous copy on `stream`; callers with N_uniform avoid it).
static Sizes sizes_of(const shm_lut* L, cudaStream_t s, shm_status* st, std::vector<int32_t>& buf)
{
    *st = SHM_OK;
    Sizes z{L->n_glyphs, L->N_uniform, nullptr, L->N_uniform};
    if (L->N_uniform > 0) return z;
    buf.resize((size_t)L->n_glyphs);
    if (cudaMemcpyAsync(buf.data(), L->N, sizeof(int32_t) * buf.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        *st = SHM_ERR_CUDA;
        return z;
    }
    int mx = 0;
    for (int32_t n : buf) {
        if (n < 1 || n > (1 << 20)) { *st = SHM_ERR_INVALID_ARG; return z; }
        if (n > mx) mx = n;
    }
    z.N_host = buf.data();
    z.max_N = mx;
    return z;
}

}  // namespace shm

using namespace shm;

extern "C" {

int64_t shm_records_per_glyph(int32_t N, int32_t layout)
{
    if (N < 1 || !valid_layout(layout)) return -1;
    return records_per_glyph(N, layout);
}

int64_t shm_record_bytes(int32_t dtype, int32_t layout)
{
    if (!valid_dtype(dtype) || !valid_layout(layout)) return -1;
    const int64_t b = (dtype == SHM_F32) ? 16 : 8;
    if (layout == SHM_LAYOUT_VALUE) return b / 4;
    return layout == SHM_LAYOUT_CELL ? 4 * b : b;
}

shm_status shm_lut_layout(int32_t G, const int32_t* N_host, int32_t dtype, int32_t layout, int64_t* offset_host,
                          int64_t* bytes)
{
    if (G <= 0 || !N_host || !valid_dtype(dtype) || !valid_layout(layout)) return SHM_ERR_INVALID_ARG;
    int64_t off = 0;
    for (int g = 0; g < G; ++g) {
        if (N_host[g] < 1 || N_host[g] > (1 << 20)) return SHM_ERR_INVALID_ARG;
        if (offset_host) offset_host[g] = off;
        off += records_per_glyph(N_host[g], layout);
    }
    if (bytes) *bytes = off * shm_record_bytes(dtype, layout);
    return SHM_OK;
}

shm_status shm_query(const shm_lut* lut, int64_t Q, const float* dirs, const int32_t* glyph, const int64_t* seg,
                     float* R, float* grad, float* normal, float* chart, int32_t* fij, int32_t* dev_status,
                     shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!hermite_layout(lut->layout)) return SHM_ERR_UNSUPPORTED;
    if (Q < 0 || (Q > 0 && !dirs)) return SHM_ERR_INVALID_ARG;
    QueryArgs a;
    a.L = view(lut);
    a.Q = Q;
    a.dirs = dirs;
    a.glyph = glyph;
    a.seg = glyph ? nullptr : seg;
    a.R = R;
    a.grad = grad;
    a.normal = normal;
    a.chart = chart;
    a.fij = fij;
    a.dev_status = dev_status;
    if ((st = resolve_io(a)) != SHM_OK) return st;
    return map_cuda(launch_query_fwd(a, (cudaStream_t)stream));
}

shm_status shm_tune_query(const shm_lut* lut, int64_t Q, const float* dirs, const int32_t* glyph, const int64_t* seg,
                          float* R, float* grad, float* normal, int32_t reps, int32_t* chosen, float* times_ms,
                          shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!hermite_layout(lut->layout)) return SHM_ERR_UNSUPPORTED;
    if (Q <= 0 || !dirs || reps < 1 || reps > 1000) return SHM_ERR_INVALID_ARG;
    QueryArgs a;
    a.L = view(lut);
    a.Q = Q;
    a.dirs = dirs;
    a.glyph = glyph;
    a.seg = glyph ? nullptr : seg;
    a.R = R;
    a.grad = grad;
    a.normal = normal;
    a.chart = nullptr;
    a.fij = nullptr;
    a.dev_status = nullptr;
    if ((st = resolve_io(a)) != SHM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = query_shapes(a);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SHM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SHM_ERR_CUDA; }
    int best = 0;
    float best_ms = 0.0f;
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < SHM_TUNE_MAX_SHAPES && times_ms; ++k) times_ms[k] = -1.0f;
    for (int k = 0; k < n && err == cudaSuccess; ++k) {
        err = launch_query_shape(a, k, s);  // warm-up (first-use attributes, caches)
        if (err == cudaSuccess) err = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && err == cudaSuccess; ++r) err = launch_query_shape(a, k, s);
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) break;
        ms /= (float)reps;
        if (times_ms && k < SHM_TUNE_MAX_SHAPES) times_ms[k] = ms;
        if (k == 0 || ms < best_ms) { best = k; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return SHM_ERR_CUDA;
    set_tuned_query_shape(a, best);
    if (chosen) *chosen = best;
    return SHM_OK;
}

shm_status shm_tune_reset(void)
{
    reset_tuned_shapes();
    return SHM_OK;
}

int64_t shm_query_binned_workspace_bytes(const shm_lut* lut, int64_t Q, int64_t band_bytes)
{
    if (check_lut(lut) != SHM_OK || !hermite_layout(lut->layout) || lut->N_uniform <= 0 || Q < 0 || band_bytes < 0)
        return -1;
    return binned_workspace_bytes(view(lut), Q, band_bytes);
}

int32_t shm_query_binned_bins(const shm_lut* lut, int64_t band_bytes, int32_t* band_rows)
{
    if (check_lut(lut) != SHM_OK || !hermite_layout(lut->layout) || lut->N_uniform <= 0 || band_bytes < 0) return -1;
    int rows = 0;
    const int B = binned_bins(view(lut), band_bytes, &rows);
    if (band_rows) *band_rows = rows;
    return B;
}

shm_status shm_query_binned(const shm_lut* lut, int64_t Q, const float* dirs, float* R, float* grad, float* normal,
                            float* chart, int64_t band_bytes, void* ws, size_t ws_bytes, int32_t* dev_status,
                            shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!hermite_layout(lut->layout)) return SHM_ERR_UNSUPPORTED;
    if (lut->N_uniform <= 0) return SHM_ERR_UNSUPPORTED;
    if (Q < 0 || (Q > 0 && !dirs) || band_bytes < 0) return SHM_ERR_INVALID_ARG;
    const int64_t need = binned_workspace_bytes(view(lut), Q, band_bytes);
    if (need < 0) return SHM_ERR_INVALID_ARG;
    if (Q > 0 && (!ws || (int64_t)ws_bytes < need)) return SHM_ERR_WORKSPACE;
    if (((uintptr_t)ws & 255u) != 0) return SHM_ERR_INVALID_ARG;
    QueryArgs a;
    a.L = view(lut);
    a.Q = Q;
    a.dirs = dirs;
    a.glyph = nullptr;
    a.seg = nullptr;
    a.R = R;
    a.grad = grad;
    a.normal = normal;
    a.chart = chart;
    a.fij = nullptr;
    a.dev_status = dev_status;
    if ((st = resolve_io(a)) != SHM_OK) return st;
    return map_cuda(launch_query_binned(a, band_bytes, ws, ws_bytes, (cudaStream_t)stream));
}

shm_status shm_query_recon(const shm_lut* lut, int32_t method, int64_t Q, const float* dirs, const int32_t* glyph,
                           const int64_t* seg, float* R, float* grad, float* normal, float* chart, int32_t* fij,
                           int32_t* dev_status, shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (lut->layout != SHM_LAYOUT_VALUE) return SHM_ERR_INVALID_ARG;
    if (method < SHM_RECON_NEAREST || method > SHM_RECON_FAST_BICUBIC) return SHM_ERR_INVALID_ARG;
    if (Q < 0 || (Q > 0 && !dirs)) return SHM_ERR_INVALID_ARG;
    QueryArgs a;
    a.L = view(lut);
    a.Q = Q;
    a.dirs = dirs;
    a.glyph = glyph;
    a.seg = glyph ? nullptr : seg;
    a.R = R;
    a.grad = grad;
    a.normal = normal;
    a.chart = chart;
    a.fij = fij;
    a.dev_status = dev_status;
    if ((st = resolve_io(a)) != SHM_OK) return st;
    return map_cuda(launch_query_recon(a, method, (cudaStream_t)stream));
}

shm_status shm_l2_fetch_granularity(int32_t bytes, int32_t* previous)
{
    if (bytes < -1 || bytes > 128) return SHM_ERR_INVALID_ARG;
    size_t cur = 0;
    cudaError_t e = cudaDeviceGetLimit(&cur, cudaLimitMaxL2FetchGranularity);
    if (e == cudaErrorUnsupportedLimit) return SHM_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return SHM_ERR_CUDA;
    if (previous) *previous = (int32_t)cur;
    if (bytes < 0) return SHM_OK;
    e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes);
    if (e == cudaErrorUnsupportedLimit) return SHM_ERR_UNSUPPORTED;
    return e == cudaSuccess ? SHM_OK : SHM_ERR_CUDA;
}

int64_t shm_sh_basis_bytes(int32_t N, int32_t L)
{
    if (N < 1 || L < 0 || L > 20) return -1;
    const int64_t K = (int64_t)(L + 1) * (L + 1), M = 4LL * 6 * (N + 2) * (N + 2), Kp = sh_kpad(L);
    const int64_t M16 = (M + 15) / 16 * 16;  // the adjoint's slabs cover M rounded up to 16 columns
    return (K * M + 2 * M * Kp + 2 * M16 * Kp) * (int64_t)sizeof(float);
}

shm_status shm_sh_basis(int32_t N, int32_t L, float* basis, shm_stream stream)
{
    if (N < 1 || N > (1 << 14) || L < 0 || L > 20 || !basis) return SHM_ERR_INVALID_ARG;
    cudaError_t e = launch_sh_basis(N, L, basis, (cudaStream_t)stream);
    if (e != cudaSuccess) return SHM_ERR_CUDA;
    e = launch_basis_split(N, L, basis, (cudaStream_t)stream);
    if (e != cudaSuccess) return SHM_ERR_CUDA;
    return map_cuda(launch_basis_split_t(N, L, basis, (cudaStream_t)stream));
}

int64_t shm_build_workspace_bytes(const shm_lut* lut, const shm_source* src)
{
    if (!lut || !src || lut->n_glyphs <= 0) return -1;
    if (src->kind != SHM_SRC_SH) return 0;
    if (src->L < 0 || src->L > 20) return -1;
    return sh_build_workspace_bytes(lut->n_glyphs, src->L);
}

shm_status shm_build_lut(const shm_lut* lut, const shm_source* src, void* ws, size_t ws_bytes, shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!src) return SHM_ERR_INVALID_ARG;
    const LutView v = view(lut);
    cudaStream_t s = (cudaStream_t)stream;
    switch (src->kind) {
    case SHM_SRC_SH:
        if (lut->N_uniform <= 0) return SHM_ERR_UNSUPPORTED;
        if (lut->layout == SHM_LAYOUT_VALUE) {
            if (src->L < 0 || src->L > 20 || !src->coeffs) return SHM_ERR_INVALID_ARG;
            return map_cuda(launch_sh_value(v, lut->data, src->L, src->coeffs, s));
        }
        if (src->L < 0 || src->L > 20 || !src->coeffs || !src->basis) return SHM_ERR_INVALID_ARG;
        if (ws) {
            if ((int64_t)ws_bytes < sh_build_workspace_bytes(lut->n_glyphs, src->L) || ((uintptr_t)ws & 15u))
                return SHM_ERR_WORKSPACE;
            return map_cuda(launch_sh_build_tc(v, lut->data, src->L, src->coeffs, src->basis, ws, s, src->dev_status));
        }
        return map_cuda(launch_sh_build(v, lut->data, src->L, src->coeffs, src->basis, s));
    case SHM_SRC_SAMPLES:
    case SHM_SRC_BUMPS:
    case SHM_SRC_FBM: {
        if (src->kind == SHM_SRC_SAMPLES && (!src->samples || !src->sample_offset)) return SHM_ERR_INVALID_ARG;
        if (src->kind == SHM_SRC_BUMPS && (!src->bump_offset || !src->mu || !src->amp || !src->width))
            return SHM_ERR_INVALID_ARG;
        if (src->kind == SHM_SRC_FBM && (src->octaves < 0 || src->octaves > 32 || (src->octaves > 0 && !src->keys)))
            return SHM_ERR_INVALID_ARG;
        std::vector<int32_t> buf;
        const Sizes z = sizes_of(lut, s, &st, buf);
        if (st != SHM_OK) return st;
        return map_cuda(launch_fd_build(v, lut->data, *src, z, s));
    }
    default:
        return SHM_ERR_INVALID_ARG;
    }
}

shm_status shm_pack_lut(const shm_lut* src, const shm_lut* dst, shm_stream stream)
{
    shm_status st = check_lut(src);
    if (st != SHM_OK) return st;
    if (!hermite_layout(src->layout) || !hermite_layout(dst->layout)) return SHM_ERR_UNSUPPORTED;
    st = check_lut(dst);
    if (st != SHM_OK) return st;
    if (src->n_glyphs != dst->n_glyphs) return SHM_ERR_INVALID_ARG;
    if ((src->N_uniform > 0) != (dst->N_uniform > 0)) return SHM_ERR_INVALID_ARG;
    if (src->N_uniform > 0 && src->N_uniform != dst->N_uniform) return SHM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> buf;
    const Sizes z = sizes_of(dst, s, &st, buf);
    if (st != SHM_OK) return st;
    return map_cuda(launch_pack(view(src), view(dst), dst->data, z, s));
}

shm_status shm_lut_bounds(const shm_lut* lut, float* rmax, shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!hermite_layout(lut->layout)) return SHM_ERR_UNSUPPORTED;
    if (!rmax) return SHM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> buf;
    const Sizes z = sizes_of(lut, s, &st, buf);
    if (st != SHM_OK) return st;
    return map_cuda(launch_bounds(view(lut), rmax, z, s));
}

shm_status shm_build_mip(const shm_lut* fine, const shm_lut* coarse, int32_t* dev_status, shm_stream stream)
{
    shm_status st = check_lut(fine);
    if (st != SHM_OK) return st;
    if (!hermite_layout(fine->layout)) return SHM_ERR_UNSUPPORTED;
    st = check_lut(coarse);
    if (st != SHM_OK) return st;
    if (!hermite_layout(coarse->layout)) return SHM_ERR_UNSUPPORTED;
    if (fine->n_glyphs != coarse->n_glyphs) return SHM_ERR_INVALID_ARG;
    if ((fine->N_uniform > 0) != (coarse->N_uniform > 0)) return SHM_ERR_INVALID_ARG;
    if (fine->N_uniform > 0 && (fine->N_uniform % 2 != 0 || coarse->N_uniform * 2 != fine->N_uniform))
        return SHM_ERR_INVALID_ARG;
    if (fine->data == coarse->data) return SHM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> buf;
    const Sizes z = sizes_of(coarse, s, &st, buf);
    if (st != SHM_OK) return st;
    return map_cuda(launch_mip(view(fine), view(coarse), coarse->data, dev_status, z, s));
}

shm_status shm_query_backward(const shm_lut* lut, int64_t Q, const float* dirs, const int32_t* glyph,
                              const int64_t* seg, const float* gR, const float* ggrad, const float* gnormal,
                              const shm_lut* dlut, float* ddirs, uint32_t flags, int32_t* dev_status,
                              shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!hermite_layout(lut->layout)) return SHM_ERR_UNSUPPORTED;
    st = check_lut(dlut);
    if (st != SHM_OK) return st;
    if (dlut->dtype != SHM_F32 || dlut->layout != SHM_LAYOUT_TEXEL) return SHM_ERR_UNSUPPORTED;
    if ((flags & ~(uint32_t)SHM_BWD_DETERMINISTIC) != 0) return SHM_ERR_INVALID_ARG;
    if (Q < 0 || (Q > 0 && !dirs)) return SHM_ERR_INVALID_ARG;
    const bool det = (flags & SHM_BWD_DETERMINISTIC) != 0;
    if (det && (glyph || !seg)) return SHM_ERR_UNSUPPORTED;
    if ((st = same_resolutions(lut, dlut, (cudaStream_t)stream)) != SHM_OK) return st;
    BackwardArgs a;
    a.L = view(lut);
    a.D = view(dlut);
    a.dlut = (float*)dlut->data;
    a.Q = Q;
    a.dirs = dirs;
    a.glyph = glyph;
    a.seg = glyph ? nullptr : seg;
    a.gR = gR;
    a.ggrad = ggrad;
    a.gnormal = gnormal;
    a.ddirs = ddirs;
    a.dev_status = dev_status;
    a.fit = 0;
    a.R_target = a.n_target = nullptr;
    a.w_value = a.w_normal = 0.0f;
    a.loss = nullptr;
    if ((st = resolve_io(a)) != SHM_OK) return st;
    return map_cuda(det ? launch_query_bwd_det(a, (cudaStream_t)stream) : launch_query_bwd(a, (cudaStream_t)stream));
}

shm_status shm_fit_backward(const shm_lut* lut, int64_t Q, const float* dirs, const int32_t* glyph,
                            const int64_t* seg, const float* R_target, const float* n_target, float w_value,
                            float w_normal, const shm_lut* dlut, float* loss, int32_t* dev_status, shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!hermite_layout(lut->layout)) return SHM_ERR_UNSUPPORTED;
    st = check_lut(dlut);
    if (st != SHM_OK) return st;
    if (dlut->dtype != SHM_F32 || dlut->layout != SHM_LAYOUT_TEXEL) return SHM_ERR_UNSUPPORTED;
    if (Q < 0 || (Q > 0 && (!dirs || !R_target || !n_target))) return SHM_ERR_INVALID_ARG;
    if ((st = same_resolutions(lut, dlut, (cudaStream_t)stream)) != SHM_OK) return st;
    BackwardArgs a;
    a.L = view(lut);
    a.D = view(dlut);
    a.dlut = (float*)dlut->data;
    a.Q = Q;
    a.dirs = dirs;
    a.glyph = glyph;
    a.seg = glyph ? nullptr : seg;
    a.gR = a.ggrad = a.gnormal = nullptr;
    a.ddirs = nullptr;
    a.dev_status = dev_status;
    a.fit = 1;
    a.R_target = R_target;
    a.n_target = n_target;
    a.w_value = w_value;
    a.w_normal = w_normal;
    a.loss = loss;
    if ((st = resolve_io(a)) != SHM_OK) return st;
    return map_cuda(launch_query_bwd(a, (cudaStream_t)stream));
}

shm_status shm_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                         float eps, int32_t step, int32_t zero_grad, shm_stream stream)
{
    if (n < 0 || (n > 0 && (!param || !grad || !m || !v)) || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return SHM_ERR_INVALID_ARG;
    return map_cuda(launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, zero_grad, (cudaStream_t)stream));
}

shm_status shm_build_lut_backward(const shm_lut* dlut, int32_t L, const float* basis, float* dcoeffs,
                                  uint32_t flags, shm_stream stream)
{
    shm_status st = check_lut(dlut);
    if (st != SHM_OK) return st;
    if (dlut->dtype != SHM_F32 || dlut->layout != SHM_LAYOUT_TEXEL || dlut->N_uniform <= 0)
        return SHM_ERR_UNSUPPORTED;
    if (L < 0 || L > 20 || !basis || !dcoeffs) return SHM_ERR_INVALID_ARG;
    if ((flags & ~(uint32_t)(SHM_BWD_DETERMINISTIC | SHM_BWD_CUDA_CORES)) != 0) return SHM_ERR_INVALID_ARG;
    if (((uintptr_t)dlut->data & 15u) != 0 || ((uintptr_t)basis & 15u) != 0) return SHM_ERR_INVALID_ARG;
    if (!(flags & SHM_BWD_CUDA_CORES)) {
        const cudaError_t e = launch_sh_build_bwd_tc(dlut->N_uniform, dlut->n_glyphs, L, (const float*)dlut->data,
                                                     basis, dcoeffs, nullptr, (cudaStream_t)stream);
        if (e != cudaErrorNotSupported) return map_cuda(e);
        (void)cudaGetLastError();
    }
    return map_cuda(launch_sh_build_bwd(dlut->N_uniform, dlut->n_glyphs, L, (const float*)dlut->data, basis, dcoeffs,
                                        (flags & SHM_BWD_DETERMINISTIC) != 0, (cudaStream_t)stream));
}

shm_status shm_sh_eval(int32_t L, int32_t n_glyphs, const float* coeffs, int64_t Q, const float* dirs,
                       const int32_t* glyph, const int64_t* seg, float* R, float* grad, float* normal,
                       int32_t* dev_status, shm_stream stream)
{
    if (L < 0 || L > 20 || n_glyphs <= 0 || !coeffs || Q < 0 || (Q > 0 && !dirs)) return SHM_ERR_INVALID_ARG;
    return map_cuda(launch_sh_eval(L, n_glyphs, coeffs, Q, dirs, glyph, glyph ? nullptr : seg, R, grad, normal,
                                   dev_status, (cudaStream_t)stream));
}

int64_t shm_raycast_workspace_bytes(int32_t n_obj, int32_t W, int32_t H)
{
    if (n_obj < 0 || W <= 0 || H <= 0) return -1;
    return raycast_workspace_bytes(n_obj, W, H);
}

shm_status shm_raycast(const shm_lut* lut, const shm_object* objs, int32_t n_obj, const shm_camera* cam,
                       const shm_raycast_params* prm, float* rgba, float* depth, float* normal, int32_t* obj_id,
                       void* ws, size_t ws_bytes, int32_t* dev_status, shm_stream stream)
{
    shm_status st = check_lut(lut);
    if (st != SHM_OK) return st;
    if (!cam || !prm || n_obj < 0 || (n_obj > 0 && !objs)) return SHM_ERR_INVALID_ARG;
    if (lut->layout == SHM_LAYOUT_VALUE && (prm->recon < SHM_RECON_NEAREST || prm->recon > SHM_RECON_FAST_BICUBIC))
        return SHM_ERR_INVALID_ARG;
    if (cam->W <= 0 || cam->H <= 0 || cam->W > 65536 || cam->H > 65536) return SHM_ERR_INVALID_ARG;
    if (prm->march < 1 || prm->march > 4096 || prm->bisect < 0 || prm->bisect > 64 || prm->newton < 0 ||
        prm->newton > 64 ||
        (prm->lod && (prm->bisect_min < 0 || prm->bisect_min > prm->bisect || prm->newton_min < 0 ||
                      prm->newton_min > prm->newton)))
        return SHM_ERR_INVALID_ARG;
    const int64_t need = raycast_workspace_bytes(n_obj, cam->W, cam->H);
    if (need > 0 && (!ws || (int64_t)ws_bytes < need)) return SHM_ERR_WORKSPACE;
    return map_cuda(launch_raycast(view(lut), objs, n_obj, *cam, *prm, rgba, depth, normal, obj_id, ws, ws_bytes,
                                   dev_status, (cudaStream_t)stream));
}

const char* shm_status_string(shm_status s)
{
    switch (s) {
    case SHM_OK: return "ok";
    case SHM_ERR_INVALID_ARG: return "invalid argument";
    case SHM_ERR_UNSUPPORTED: return "unsupported dtype/layout/source combination";
    case SHM_ERR_WORKSPACE: return "workspace missing or too small";
    case SHM_ERR_CUDA: return "CUDA launch or runtime error";
    case SHM_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
    }
}

int32_t shm_version(void) { return 1; }

}  // extern "C"
