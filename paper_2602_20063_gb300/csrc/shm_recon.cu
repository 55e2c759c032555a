// Value-only reconstruction baselines (§4.2 Table psnr_value, §4.5 Table cost_extended):
// nearest, bilinear + finite-difference gradient, 16-tap Catmull-Rom with analytic gradient and
// the cubic B-spline of the 4-bilinear-fetch "fast bicubic", on a SHM_LAYOUT_VALUE table, run
// through the same query kernel skeleton as the Hermite query.
#include "shm_query_kernel.cuh"

namespace shm {

template <int RECON>
static cudaError_t launch_recon_m(const QueryArgs& a, cudaStream_t s)
{
    if (a.L.dtype == SHM_F32) return launch_fwd_t<SHM_F32, SHM_LAYOUT_VALUE, RECON>(a, s);
    if (a.L.dtype == SHM_F16) return launch_fwd_t<SHM_F16, SHM_LAYOUT_VALUE, RECON>(a, s);
    return launch_fwd_t<SHM_BF16, SHM_LAYOUT_VALUE, RECON>(a, s);
}

cudaError_t launch_query_recon(const QueryArgs& a, int method, cudaStream_t s)
{
    if (a.Q == 0) return cudaSuccess;
    switch (method) {
    case SHM_RECON_NEAREST: return launch_recon_m<SHM_RECON_NEAREST>(a, s);
    case SHM_RECON_BILINEAR: return launch_recon_m<SHM_RECON_BILINEAR>(a, s);
    case SHM_RECON_BICUBIC: return launch_recon_m<SHM_RECON_BICUBIC>(a, s);
    default: return launch_recon_m<SHM_RECON_FAST_BICUBIC>(a, s);
    }
}

}  // namespace shm
