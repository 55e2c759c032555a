// Hermite query dispatch (§3.2-§3.4): dtype x layout x launch-shape instances of the query kernel
// skeleton, or the shared-memory staged kernel (shm_query_staged.cu) for per-glyph segments on
// small tables.  The launch shape comes from the per-device table that shm_tune_query fills.
#include <atomic>

#include "shm_query_kernel.cuh"

namespace shm {

namespace {

constexpr int MAX_DEV = 64;
// [device][path: 0 unstaged, 1 staged][dtype][layout] -> shape index (0 = default)
std::atomic<int> g_shape[MAX_DEV][2][3][2];

int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return -1;
    return dev;
}

template <int DT, int LAYOUT>
cudaError_t launch_unstaged_shape(const QueryArgs& a, int shape, cudaStream_t s)
{
    switch (shape) {
    case 1: return launch_fwd_t<DT, LAYOUT, -1, QSHAPES[1].block, QSHAPES[1].it>(a, s);
    case 2: return launch_fwd_t<DT, LAYOUT, -1, QSHAPES[2].block, QSHAPES[2].it>(a, s);
    case 3: return launch_fwd_t<DT, LAYOUT, -1, QSHAPES[3].block, QSHAPES[3].it>(a, s);
    default: return launch_fwd_t<DT, LAYOUT, -1, QSHAPES[0].block, QSHAPES[0].it>(a, s);
    }
}

}  // namespace

bool query_is_staged(const QueryArgs& a)
{
    if (!a.seg || a.glyph || a.L.N_uniform <= 0 || a.L.layout != SHM_LAYOUT_TEXEL) return false;
    const int64_t P = (int64_t)a.L.N_uniform + 2;
    return 6 * P * P * (a.L.dtype == SHM_F32 ? 16 : 8) <= STAGED_TABLE_MAX_BYTES;
}

int query_shapes(const QueryArgs& a) { return query_is_staged(a) ? staged_shapes() : N_QSHAPES; }

cudaError_t launch_query_shape(const QueryArgs& a, int shape, cudaStream_t s)
{
    if (a.Q == 0) return cudaSuccess;
    if (query_is_staged(a)) return launch_query_staged(a, shape, s);
    const int dt = a.L.dtype, ly = a.L.layout;
    if (ly == SHM_LAYOUT_TEXEL) {
        if (dt == SHM_F32) return launch_unstaged_shape<SHM_F32, SHM_LAYOUT_TEXEL>(a, shape, s);
        if (dt == SHM_F16) return launch_unstaged_shape<SHM_F16, SHM_LAYOUT_TEXEL>(a, shape, s);
        return launch_unstaged_shape<SHM_BF16, SHM_LAYOUT_TEXEL>(a, shape, s);
    }
    if (dt == SHM_F32) return launch_unstaged_shape<SHM_F32, SHM_LAYOUT_CELL>(a, shape, s);
    if (dt == SHM_F16) return launch_unstaged_shape<SHM_F16, SHM_LAYOUT_CELL>(a, shape, s);
    return launch_unstaged_shape<SHM_BF16, SHM_LAYOUT_CELL>(a, shape, s);
}

int tuned_query_shape(const QueryArgs& a)
{
    const int dev = current_device();
    if (dev < 0) return 0;
    return g_shape[dev][query_is_staged(a) ? 1 : 0][a.L.dtype][a.L.layout].load(std::memory_order_relaxed);
}

void set_tuned_query_shape(const QueryArgs& a, int shape)
{
    const int dev = current_device();
    if (dev >= 0) g_shape[dev][query_is_staged(a) ? 1 : 0][a.L.dtype][a.L.layout].store(shape, std::memory_order_relaxed);
}

void reset_tuned_shapes()
{
    for (auto& d : g_shape)
        for (auto& p : d)
            for (auto& t : p)
                for (auto& l : t) l.store(0, std::memory_order_relaxed);
}

cudaError_t launch_query_fwd(const QueryArgs& a, cudaStream_t s) { return launch_query_shape(a, tuned_query_shape(a), s); }

}  // namespace shm
