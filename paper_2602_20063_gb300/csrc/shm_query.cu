// Hermite query dispatch (§3.2-§3.4): dtype x layout instances of the query kernel skeleton, or
// the shared-memory staged kernel (shm_query_staged.cu) for per-glyph segments on small tables.
#include "shm_query_kernel.cuh"

namespace shm {

cudaError_t launch_query_fwd(const QueryArgs& a, cudaStream_t s)
{
    if (a.Q == 0) return cudaSuccess;
    const int dt = a.L.dtype, ly = a.L.layout;
    // per-glyph segments on small uniform tables: stage each glyph's table in shared memory
    if (a.seg && !a.glyph && a.L.N_uniform > 0 && ly == SHM_LAYOUT_TEXEL) {
        const int64_t P = (int64_t)a.L.N_uniform + 2;
        if (6 * P * P * (dt == SHM_F32 ? 16 : 8) <= STAGED_TABLE_MAX_BYTES) return launch_query_staged(a, s);
    }
    if (ly == SHM_LAYOUT_TEXEL) {
        if (dt == SHM_F32) return launch_fwd_t<SHM_F32, SHM_LAYOUT_TEXEL, -1>(a, s);
        if (dt == SHM_F16) return launch_fwd_t<SHM_F16, SHM_LAYOUT_TEXEL, -1>(a, s);
        return launch_fwd_t<SHM_BF16, SHM_LAYOUT_TEXEL, -1>(a, s);
    }
    if (dt == SHM_F32) return launch_fwd_t<SHM_F32, SHM_LAYOUT_CELL, -1>(a, s);
    if (dt == SHM_F16) return launch_fwd_t<SHM_F16, SHM_LAYOUT_CELL, -1>(a, s);
    return launch_fwd_t<SHM_BF16, SHM_LAYOUT_CELL, -1>(a, s);
}

}  // namespace shm
