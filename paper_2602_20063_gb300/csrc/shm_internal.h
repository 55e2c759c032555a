// Internal launch interfaces between the C-ABI layer (shm_api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/shm.h"
#include "shm_device.cuh"

namespace shm {

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

cudaError_t launch_query_fwd(const QueryArgs& a, cudaStream_t s);
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
cudaError_t launch_sh_build_bwd(int N, int G, int L, const float* dlut, const float* basis, float* dcoeffs,
                                cudaStream_t s);
cudaError_t launch_fd_build(const LutView& out, void* data, const shm_source& src, int max_N, cudaStream_t s);
cudaError_t launch_pack(const LutView& src, const LutView& dst, void* dst_data, int max_N, cudaStream_t s);
cudaError_t launch_bounds(const LutView& L, float* rmax, int max_N, cudaStream_t s);
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
