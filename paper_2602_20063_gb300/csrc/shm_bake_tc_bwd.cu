// Tensor-core adjoint of the SH bake (sm_103a): see the comment at the top of namespace bwd.
#include "shm_tc.cuh"

namespace shm {
namespace tc {
// ------------------------------------------------------------------------------------------
// Adjoint of the bake on the tensor cores.  The bake is linear in the coefficients (Algorithm 1:
// table = sum_k c_k basis_k), so its reverse mode is the transposed contraction
//     dcoeffs[g][k] = sum_c dlut[g][c] basis[k][c]                     (c over the 4T table scalars)
// with a CTA's group of up to 128 glyphs on the MMA M side (rows beyond the group hold stale data and
// are never stored; see plan() for the group size) and the coefficients on N (K padded to
// Kp <= 128).  Operands:
//   A = dlut tiles [R glyphs x 16 c], loaded raw by TMA (64-byte swizzle) and split in place by
//       six converter warps into tf32 hi = x truncated (overwriting the raw tile) and
//       lo = tf32_rna(x - hi);
//   B = the transposed tf32 split of the basis, hiS / loS (part of shm_sh_basis's buffer), stored as
//       one contiguous [Kp][16 c] slab per stage with its rows already in the 64-byte swizzled order
//       that a tensor load would produce, so each stage's B tile is one plain bulk copy (a tensor
//       load of [Kp][16] from a [Kp][4T] array would be Kp separate 64-byte pieces).
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi (3xTF32, as the forward bake), in two MMAs per K step: B_hi
// and B_lo lie back to back in a stage, so A_hi [B_hi; B_lo] is one MMA of N = 2 Kp whose columns
// [0, Kp) take A_hi B_hi and [Kp, 2 Kp) A_hi B_lo, and A_lo B_hi adds into [0, Kp); the drain warps
// add both halves (TMEM: two buffers of 2 Kp columns).  Two MMA instructions instead of three per
// K step at the same tensor work: 0.962 -> 0.870 ms on the glyph field, the MMA issuer being one of
// the two roles that set the pace; the split, the other, runs on six warps (0.870 -> 0.853 ms).
// Accuracy: the error of the tensor cores' float32 accumulation grew with the length of the sum
// kept in one TMEM accumulator (measured: 4.6e-5 of the largest entry after 434 stages, against
// 7.9e-6 for a plain float32 sum).  So the MMAs accumulate CH stages at a time into one of two
// TMEM buffers, and four drain warps add each finished chunk into float32 registers (one glyph row
// per thread, Kp values) while the MMAs fill the other buffer.
// Latency: seven 28 KB stages, and the producer prefetches dlut into L2 in boxes of 1 KB per glyph
// row (16 stages), two boxes ahead of the shared-memory loads: the rows of a tile lie 4T x 4 B apart,
// so 64-byte pieces per row and stage would reach DRAM as scattered small requests.
// The c range may be split over the S CTAs of a thread-block cluster (small glyph counts); at the
// end every CTA writes its register sums to shared memory and each CTA sums a slice of them over
// the cluster's ranks in rank order through distributed shared memory, so the result does not
// depend on timing (deterministic, no atomics, no workspace).
//   warp 0 lane 0: TMA producer   warp 1: TMEM allocation, lane 0 issues the MMAs
//   warps 4-7: drain (TMEM lane quadrant = warp % 4) and epilogue   warps 2-3, 8-11: tf32 split
// Every mbarrier wait is bounded (1 s) and raises SHM_DEV_TIMEOUT on expiry; the cluster barriers
// are reached by every thread of every CTA the same number of times, aborted or not.
namespace bwd {

constexpr int MG = 128;                       // glyph rows (MMA M)
constexpr uint32_t A_TILE = MG * KC * 4;      // 8 KB
constexpr int KPMAX = 128;                    // register sums per drain thread
constexpr int CH = 16;                        // stages per TMEM chunk
constexpr int PFW = 16;                       // stages per L2 prefetch box (256 c: 1 KB of each glyph row)
constexpr int PFA = 2;                        // prefetch boxes ahead of the shared-memory loads
constexpr int THREADS = 384;
constexpr int SPLIT_T = 192;                  // tf32-split threads: warps 2-3 and 8-11
constexpr uint32_t STAGE_CAP = 196 * 1024;    // shared memory for the stages (and the partials after them)
constexpr uint32_t BAR_BYTES = 1024;
constexpr int MAXSTAGE = 8;

struct Args {
    const float* hiS;  // basis slabs, [NC][Kp][16] each, rows pre-swizzled
    const float* loS;
    int M4;        // table scalars per glyph (4T), the reduction length
    int G, K, Kp;
    int R;         // glyph rows per group (<= MG; the MMA's rows beyond R are never stored)
    int groups;
    int S;         // CTAs per cluster (splits of the c range)
    int NC;        // stages over the whole c range
    int nstage;    // pipeline depth
    uint32_t b_bytes, stage_bytes;
    float* dcoeffs;
    int32_t* dev_status;
};

// Plain bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared memory,
// completing on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// tf32 by truncation (the low 13 mantissa bits cleared): one logic operation where the rounding
// conversion is a slower instruction; the remainder x - hi is exact and carries what was cut off.
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ float ld_dsmem(uint32_t local_addr, uint32_t rank)
{
    uint32_t remote;
    float v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
    return v;
}

__device__ __forceinline__ void tma_prefetch_l2(const CUtensorMap* map, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(x),
                 "r"(y)
                 : "memory");
}

__device__ __forceinline__ uint32_t idesc(int NB)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(MG >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32_n(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
    k_sh_gemm_bwd_tc(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mApf, Args a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* bars = smem;
    uint8_t* stages = smem + BAR_BYTES;
    // barriers: full / conv / empty per stage (MAXSTAGE each at most), chunk full / empty per TMEM
    // buffer, the drain barrier
    const uint32_t full0 = smem_u32(bars), conv0 = full0 + 8 * MAXSTAGE, empty0 = conv0 + 8 * MAXSTAGE,
                   cfull0 = empty0 + 8 * MAXSTAGE, cempty0 = cfull0 + 16, drain = cempty0 + 16;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 512);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 520);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int g_base = (blockIdx.x / a.S) * a.R;
    const int c0 = (int)(((int64_t)a.NC * rank) / a.S), c1 = (int)(((int64_t)a.NC * (rank + 1)) / a.S);
    const int nst = c1 - c0;
    const int nchunk = (nst + CH - 1) / CH;
    const uint32_t ID = idesc(a.Kp), ID2 = idesc(2 * a.Kp);

    auto stA = [&](int st) { return stages + (size_t)st * a.stage_bytes; };
    auto stAlo = [&](int st) { return stages + (size_t)st * a.stage_bytes + A_TILE; };
    auto stBh = [&](int st) { return stages + (size_t)st * a.stage_bytes + 2 * A_TILE; };
    auto stBl = [&](int st) { return stages + (size_t)st * a.stage_bytes + 2 * A_TILE + a.b_bytes; };

    if (threadIdx.x == 0) {
        for (int st = 0; st < a.nstage; ++st) {
            mbar_init(full0 + 8 * st, 1);
            mbar_init(conv0 + 8 * st, SPLIT_T);
            mbar_init(empty0 + 8 * st, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(cfull0 + 8 * b, 1);
            mbar_init(cempty0 + 8 * b, 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;
    float acc[KPMAX];  // drain warps: the glyph row's running sums
#pragma unroll
    for (int i = 0; i < KPMAX; ++i) acc[i] = 0.0f;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- TMA producer
        for (int p = 0; p < PFA && p * PFW < nst; ++p) tma_prefetch_l2(&mApf, (c0 + p * PFW) * KC, g_base);
        int it = 0;
        for (; it < nst; ++it) {
            const int st = it % a.nstage;
            const uint32_t ph = (uint32_t)(it / a.nstage) & 1;
            if (!mbar_wait(empty0 + 8 * st, ph ^ 1, abort_flag, WAIT_LIMIT_NS)) break;
            if (it % PFW == 0 && it + PFA * PFW < nst) tma_prefetch_l2(&mApf, (c0 + it + PFA * PFW) * KC, g_base);
            const uint32_t fb = full0 + 8 * st;
            const int c = (c0 + it) * KC;
            mbar_expect_tx(fb, (uint32_t)a.R * KC * 4 + 2 * a.b_bytes);
            tma_load_2d(smem_u32(stA(st)), &mA, c, g_base, fb);
            const size_t slab = (size_t)(c0 + it) * a.Kp * KC;
            bulk_load(smem_u32(stBh(st)), a.hiS + slab, a.b_bytes, fb);
            bulk_load(smem_u32(stBl(st)), a.loS + slab, a.b_bytes, fb);
        }
        if (it < nst) {
            // aborted: the last load issued into each stage must land before the shared memory is reused
            for (int k = 1; k <= a.nstage && k <= it; ++k) {
                const int last = it - k;
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(full0 + 8 * (last % a.nstage), (uint32_t)(last / a.nstage) & 1) &&
                       globaltimer() - t0 < DRAIN_LIMIT_NS) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        bool ok = true, any = false;
        int it = 0;
        for (int j = 0; j < nchunk && ok; ++j) {
            const int b = j & 1;
            if (!mbar_wait(cempty0 + 8 * b, ((uint32_t)(j >> 1) & 1) ^ 1, abort_flag, WAIT_LIMIT_NS)) { ok = false; break; }
            fence_after();
            const uint32_t d = tmem + (uint32_t)(b * 2 * a.Kp);
            const int jend = min(nst, (j + 1) * CH);
            for (; it < jend; ++it) {
                const int st = it % a.nstage;
                const uint32_t ph = (uint32_t)(it / a.nstage) & 1;
                if (!mbar_wait(conv0 + 8 * st, ph, abort_flag, WAIT_LIMIT_NS)) { ok = false; break; }
                fence_after();
                const uint32_t ah = smem_u32(stA(st)), al = smem_u32(stAlo(st));
                const uint32_t bh = smem_u32(stBh(st));
#pragma unroll
                for (int kk = 0; kk < KC / 8; ++kk) {
                    const uint32_t o = kk * 32;
                    // columns [0, Kp): A_hi B_hi (+ A_lo B_hi below); [Kp, 2 Kp): A_hi B_lo, one MMA of
                    // N = 2 Kp over the stage's B_hi and B_lo slabs, which lie back to back
                    mma_tf32_n(d, sdesc(ah + o), sdesc(bh + o), ID2, (it != j * CH || kk != 0) ? 1u : 0u);
                    mma_tf32_n(d, sdesc(al + o), sdesc(bh + o), ID, 1);
                }
                any = true;
                mma_commit(empty0 + 8 * st);
            }
            if (ok) mma_commit(cfull0 + 8 * b);
        }
        if (!ok && any) {
            mma_commit(drain);
            const uint64_t t0 = globaltimer();
            while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < DRAIN_LIMIT_NS) {
            }
        }
    } else if (warp >= 8 || warp == 2 || warp == 3) {
        // ---------------------------------------------------------------- tf32 split of each stage
        const int t = warp >= 8 ? threadIdx.x - 256 : threadIdx.x + 64;  // warps 8-11: 0-127, warps 2-3: 128-191
        constexpr int n4 = (int)(A_TILE / 16);
        for (int it = 0; it < nst; ++it) {
            const int st = it % a.nstage;
            const uint32_t ph = (uint32_t)(it / a.nstage) & 1;
            if (!mbar_wait(full0 + 8 * st, ph, abort_flag, WAIT_LIMIT_NS)) break;
            float4* hi = reinterpret_cast<float4*>(stA(st));
            float4* lo = reinterpret_cast<float4*>(stAlo(st));
#pragma unroll
            for (int i = t; i < n4; i += SPLIT_T) {
                const float4 x = hi[i];
                float4 h, l;
                h.x = tf32_trunc(x.x); h.y = tf32_trunc(x.y); h.z = tf32_trunc(x.z); h.w = tf32_trunc(x.w);
                l.x = tf32_rna(x.x - h.x); l.y = tf32_rna(x.y - h.y); l.z = tf32_rna(x.z - h.z); l.w = tf32_rna(x.w - h.w);
                hi[i] = h;
                lo[i] = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(conv0 + 8 * st);
        }
    } else if (warp >= 4) {
        // ---------------------------------------------------------------- drain: chunk sums -> registers
        const int wq = warp & 3;
        for (int j = 0; j < nchunk; ++j) {
            const int b = j & 1;
            if (!mbar_wait(cfull0 + 8 * b, (uint32_t)(j >> 1) & 1, abort_flag, WAIT_LIMIT_NS)) break;
            fence_after();
#pragma unroll
            for (int cc = 0; cc < KPMAX; cc += 32) {
                if (cc < a.Kp) {
                    uint32_t r[32];
                    const uint32_t t0 = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(b * 2 * a.Kp + cc);
                    tmem_ld32(t0, r);  // A_hi B_hi + A_lo B_hi
#pragma unroll
                    for (int i = 0; i < 32; ++i) acc[cc + i] += __uint_as_float(r[i]);
                    tmem_ld32(t0 + (uint32_t)a.Kp, r);  // A_hi B_lo
#pragma unroll
                    for (int i = 0; i < 32; ++i) acc[cc + i] += __uint_as_float(r[i]);
                }
            }
            fence_before();
            mbar_arrive(cempty0 + 8 * b);
        }
    }
    __syncthreads();
    // ---------------------------------------------------------------- epilogue: cluster reduction
    const bool aborted = *abort_flag != 0;
    float* P = reinterpret_cast<float*>(stages);  // [128][Kp + 1] partial sums of this CTA
    const int PS = a.Kp + 1;
    if (warp >= 4 && warp < 8 && !aborted) {
        const int row = 32 * (warp & 3) + lane;
#pragma unroll
        for (int i = 0; i < KPMAX; ++i)
            if (i < a.Kp) P[row * PS + i] = acc[i];
    }
    cluster_sync();
    const uint32_t P_s = smem_u32(P);
    const int E = a.R * a.K;
    const int e0 = (int)(((int64_t)E * rank) / a.S), e1 = (int)(((int64_t)E * (rank + 1)) / a.S);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int row = e / a.K, k = e - row * a.K;
        const int g = g_base + row;
        float sum = 0.0f;
        for (int rr = 0; rr < a.S; ++rr) sum += ld_dsmem(P_s + 4u * (uint32_t)(row * PS + k), (uint32_t)rr);
        if (g < a.G && !aborted) a.dcoeffs[(int64_t)g * a.K + k] = sum;
    }
    cluster_sync();
    if (threadIdx.x == 0 && aborted && a.dev_status) atomicOr(a.dev_status, SHM_DEV_TIMEOUT);
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

// tf32 split of the basis into the adjoint's slabs: entry (k, c) of slab s = c / 16 at
// s*16*Kp + 16k + 4((c%16)/4 XOR (k/2)%4) + c%4 (16-byte chunks swizzled within each 64-byte row as
// the 64-byte swizzle places them); hi = tf32(full[k][c]), lo = tf32(full - hi); rows k >= K and
// columns c >= M4 of the last slab zero.
__global__ void k_split_basis_t(const float* __restrict__ full, int K, int Kp, int64_t M4, float* __restrict__ hiS,
                                float* __restrict__ loS)
{
    const int64_t NC = (M4 + KC - 1) / KC;
    const int64_t n = NC * Kp * KC;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slab = e / ((int64_t)Kp * KC);
        const int r = (int)(e - slab * Kp * KC);
        const int k = r / KC, q = r % KC;            // row and position within the stored row
        const int cc = (((q >> 2) ^ ((k >> 1) & 3)) << 2) | (q & 3);  // logical column within the slab
        const int64_t c = slab * KC + cc;
        const float v = (k < K && c < M4) ? __ldg(full + (int64_t)k * M4 + c) : 0.0f;
        const float h = tf32_rna(v);
        hiS[e] = h;
        loS[e] = tf32_rna(v - h);
    }
}

// 2-D map over a row-major [rows][M4] f32 array, boxes of [box_rows][box_c]: the operand loads use
// box_c = 16 with the 64-byte swizzle of the MMA descriptors; the L2 prefetch boxes are unswizzled.
static bool make_map_c(CUtensorMap* m, const float* base, int rows, int M4, int box_rows, int box_c = KC,
                       bool swizzle = true)
{
    EncodeFn enc = encode_fn();
    if (!enc || ((uintptr_t)base & 15u) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)M4, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)M4 * 4};
    const cuuint32_t box[2] = {(cuuint32_t)box_c, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Plan of the tensor-core adjoint for (G, K, Kp, M4) on `sms` SMs; false when it does not apply
// (the CUDA-core kernel is used then).  Glyph groups of R <= 128 rows: with at least 64 glyphs per
// SM, R is chosen so that the groups fill whole waves of the SMs (16,384 glyphs on 152 SMs: 108
// rows, 152 CTAs, where 128-row groups would leave 24 SMs idle); below that, 128-row groups whose c
// range is split over the CTAs of a cluster.
static bool plan(int G, int K, int Kp, int M4, int sms, int max_cluster, Args* out)
{
    Args a{};
    a.M4 = M4; a.G = G; a.K = K; a.Kp = Kp;
    if (Kp > KPMAX || Kp % 16 != 0) return false;
    a.R = MG;
    if ((int64_t)G >= 64LL * sms) {
        const int64_t waves = ((int64_t)G + (int64_t)MG * sms - 1) / ((int64_t)MG * sms);
        a.R = (int)(((int64_t)G + waves * sms - 1) / (waves * sms));
    }
    const int groups = (G + a.R - 1) / a.R;
    a.groups = groups;
    a.S = sms / groups;
    if (a.S > max_cluster) a.S = max_cluster;
    if (a.S < 1) a.S = 1;
    a.NC = (M4 + KC - 1) / KC;
    if (a.S > a.NC) a.S = a.NC;
    a.b_bytes = (uint32_t)Kp * KC * 4;
    a.stage_bytes = 2 * A_TILE + 2 * a.b_bytes;
    a.nstage = (int)(STAGE_CAP / a.stage_bytes);
    if (a.nstage > MAXSTAGE) a.nstage = MAXSTAGE;
    if (a.nstage < 2) return false;
    if ((uint64_t)MG * (Kp + 1) * 4 > (uint64_t)a.nstage * a.stage_bytes) return false;  // partials fit
    *out = a;
    return true;
}

}  // namespace bwd
}  // namespace tc

// basis: [K][M] full, hi [M][Kp], lo [M][Kp], then the adjoint's slabs hiS and loS [NC][Kp][16]
cudaError_t launch_basis_split_t(int N, int L, float* basis, cudaStream_t s)
{
    const int K = (L + 1) * (L + 1), Kp = sh_kpad(L);
    const int64_t M = 4LL * 6 * (N + 2) * (N + 2);
    const int64_t slabs = (M + tc::KC - 1) / tc::KC * tc::KC * Kp;
    float* hiS = basis + (int64_t)K * M + 2 * M * Kp;
    float* loS = hiS + slabs;
    tc::bwd::k_split_basis_t<<<(unsigned)((slabs + 255) / 256 < 65535 * 8 ? (slabs + 255) / 256 : 65535 * 8), 256, 0,
                               s>>>(basis, K, Kp, M, hiS, loS);
    return cudaGetLastError();
}

// Tensor-core adjoint of the SH bake; returns cudaErrorNotSupported when its plan does not apply
// (the caller then runs the CUDA-core kernel).
cudaError_t launch_sh_build_bwd_tc(int N, int G, int L, const float* dlut, const float* basis, float* dcoeffs,
                                   int32_t* dev_status, cudaStream_t s)
{
    using namespace tc::bwd;
    const int K = (L + 1) * (L + 1), Kp = sh_kpad(L);
    const int M4 = 4 * 6 * (N + 2) * (N + 2);
    const float* hiS = basis + (int64_t)K * M4 + 2LL * M4 * Kp;
    const float* loS = hiS + ((int64_t)M4 + tc::KC - 1) / tc::KC * tc::KC * Kp;
    cudaError_t e = ensure_dynamic_smem((const void*)k_sh_gemm_bwd_tc, (int)(1024 + BAR_BYTES + STAGE_CAP));
    if (e != cudaSuccess) return e;
    // clusters of up to 16 CTAs where the device allows them, else the portable 8
    static int max_cluster = 0;
    if (max_cluster == 0) {
        max_cluster = 8;
        if (cudaFuncSetAttribute((const void*)k_sh_gemm_bwd_tc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(16, 1, 1);
            q.blockDim = dim3(THREADS, 1, 1);
            q.dynamicSmemBytes = 1024 + BAR_BYTES + STAGE_CAP;
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = 16;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            q.attrs = &at;
            q.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_sh_gemm_bwd_tc, &q) == cudaSuccess && n > 0)
                max_cluster = 16;
        }
        (void)cudaGetLastError();
    }
    Args a;
    if (!plan(G, K, Kp, M4, sm_count(), max_cluster, &a)) return cudaErrorNotSupported;
    CUtensorMap mA, mApf;
    if (((uintptr_t)hiS & 15u) != 0 || !make_map_c(&mA, dlut, G, M4, a.R) ||
        !make_map_c(&mApf, dlut, G, M4, a.R, PFW * tc::KC, false))
        return cudaErrorNotSupported;
    a.hiS = hiS;
    a.loS = loS;
    a.dcoeffs = dcoeffs;
    a.dev_status = dev_status;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.groups * a.S), 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = 1024 + BAR_BYTES + (size_t)a.nstage * a.stage_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)a.S;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sh_gemm_bwd_tc, mA, mApf, a);
}
}  // namespace shm
