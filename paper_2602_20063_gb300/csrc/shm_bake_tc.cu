// Tensor-core SH bake (arXiv 2602.20063, Algorithm 1 with analytic SH derivatives, §3.3) on the
// 5th-generation tensor cores of sm_103a: tcgen05.mma with TMEM accumulators, operands staged by
// TMA into 128-byte-swizzled shared memory.
//
// The bake of G glyphs is the contraction
//     table[g][c] = sum_k coeff[g][k] basis[c][k]            (c = texel * 4 + channel, 4T columns)
// computed transposed, D[c][g] = A[c][:] . B[g][:], so that TMEM lane = table column and TMEM column =
// glyph: each epilogue thread owns one table column and a warp's 32 lanes store 32 consecutive
// floats of one glyph's table (coalesced 128 B).
//
// Precision: kind::tf32 multiplies 10-bit-mantissa operands.  To stay at float32 accuracy both
// operands are split x = x_hi + x_lo (x_hi = tf32(x), x_lo = tf32(x - x_hi), round to nearest) and
//     D = A_hi B_hi + A_hi B_lo + A_lo B_hi      (the 3xTF32 scheme of Ootomo & Yokota, 2022),
// leaving a relative error ~2^-21 per product, below the float32 accumulation error of K terms.
//
// Schedule: persistent CTAs (one per SM, 256 threads), tiles of 128 columns x 256 glyphs, K in
// chunks of 16 (64 B rows, 64-byte swizzle), 3 smem stages of 48 KB so TMA runs chunks ahead of
// the MMAs, 2 TMEM accumulators of 256 columns (512 columns, the whole TMEM) so the epilogue of
// one tile overlaps the MMAs of the next.  CTA b takes tiles b, b + grid, ..., with the glyph tile
// varying fastest, so the CTAs running together share column tiles of the basis (1.3 % faster than
// column tiles fastest; contiguous runs of tiles per CTA were 11 % slower).
//   warp 0 lane 0: TMA producer        warp 1: TMEM allocation; lane 0 issues the MMAs
//   warps 4-7: epilogue (TMEM lane quadrant = warp % 4), table writes
// Epilogue of the float32 texel table: per 32 glyphs the four warps transpose their TMEM rows into
// a [32 glyphs][128 columns] shared box (four boxes in flight) and one thread writes it with a TMA
// tensor store (512 B contiguous per glyph row).  Plain per-thread stores, 128 B per warp
// instruction to 32 different table rows, ran the memory write path at ~9 B/clk/SM and left the
// tensor pipe idle 70 % of the time.  Other dtypes / layouts keep per-thread stores.
// Every mbarrier wait is bounded (1 s); on expiry the CTA raises SHM_DEV_TIMEOUT, drains its own
// copies and MMAs with bounded waits, frees TMEM and returns.
#include "shm_tc.cuh"

namespace shm {
namespace tc {

constexpr int TM = 128;  // table columns per tile (MMA M)
constexpr int TN = 256;  // glyphs per tile (MMA N)
constexpr int NSTAGE = 3;
constexpr uint32_t A_BYTES = TM * KC * 4;
constexpr uint32_t B_BYTES = TN * KC * 4;
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int OG = 32;                                // glyphs per output store box
constexpr uint32_t OUT_BYTES = OG * TM * 4;           // one [32 glyphs][128 columns] f32 box, 16 KB
constexpr uint32_t BAR_BYTES = 256;
constexpr int NOUT = 4;                               // output boxes in flight per CTA
constexpr uint32_t SMEM_BYTES = NSTAGE * STAGE_BYTES + NOUT * OUT_BYTES + BAR_BYTES + 1024;
// kind::tf32 instruction descriptor: D f32, A and B tf32, both K-major, N = 256, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

struct Args {
    int M;                // table columns, 4T
    int G;                // glyphs
    int Kp;               // padded K (multiple of 32)
    int K;                // SH terms (K steps of 8 wholly beyond K are all zero and skipped)
    float* out;           // f32 texel table [G][M] when direct
    LutView view;         // output table (any dtype / layout) for the generic epilogue
    void* data;
    int direct;           // 1: f32 texel layout, uniform N, write out[g*M + c]
    int32_t* dev_status;
};

// at most NOUT - 1 stores may still be reading their shared boxes
__device__ __forceinline__ void bulk_wait_read_free() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(NOUT - 1) : "memory"); }
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// AND of `ok` over the 128 epilogue threads (named barrier 1): all leave or all stay.
__device__ __forceinline__ bool epi_all(bool ok)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)ok)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}

__global__ void __launch_bounds__(256, 1)
    k_sh_gemm_tc(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                 const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                 const __grid_constant__ CUtensorMap mOut, Args a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* obuf = reinterpret_cast<float*>(smem + NSTAGE * STAGE_BYTES);  // NOUT x [OG][TM]
    uint8_t* bars = smem + NSTAGE * STAGE_BYTES + NOUT * OUT_BYTES;
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * NSTAGE, tfull0 = empty0 + 8 * NSTAGE,
                   tempty0 = tfull0 + 16, drain = tempty0 + 16;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 128);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 136);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_m = (a.M + TM - 1) / TM, num_n = (a.G + TN - 1) / TN;
    const int tiles = num_m * num_n;
    const int NC = a.Kp / KC;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(tfull0 + 8 * q, 1);
            mbar_init(tempty0 + 8 * q, 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- TMA producer
        uint32_t it = 0;  // chunks issued so far
        bool ok = true;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
            const int nt = t % num_n, mt = t / num_n;
            for (int c = 0; c < NC; ++c, ++it) {
                const int s = it % NSTAGE;
                const uint32_t ph = (it / NSTAGE) & 1;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1, abort_flag, WAIT_LIMIT_NS)) { ok = false; break; }
                uint8_t* st = smem + s * STAGE_BYTES;
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, STAGE_BYTES);
                tma_load_2d(smem_u32(st), &mAh, c * KC, mt * TM, fb);
                tma_load_2d(smem_u32(st + A_BYTES), &mAl, c * KC, mt * TM, fb);
                tma_load_2d(smem_u32(st + 2 * A_BYTES), &mBh, c * KC, nt * TN, fb);
                tma_load_2d(smem_u32(st + 2 * A_BYTES + B_BYTES), &mBl, c * KC, nt * TN, fb);
            }
        }
        if (!ok) {
            // drain: the last load issued into each stage must land before the CTA exits
            for (uint32_t k = 1; k <= NSTAGE && k <= it; ++k) {
                const uint32_t last = it - k;  // the last chunk issued into stage last % NSTAGE
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(full0 + 8 * (last % NSTAGE), (last / NSTAGE) & 1) &&
                       globaltimer() - t0 < DRAIN_LIMIT_NS) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        uint32_t it = 0, j = 0;
        bool ok = true, any = false;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++j) {
            const uint32_t acc = j & 1, aph = (j >> 1) & 1;
            if (!mbar_wait(tempty0 + 8 * acc, aph ^ 1, abort_flag, WAIT_LIMIT_NS)) { ok = false; break; }
            fence_after();
            const uint32_t d = tmem + acc * TN;
            for (int c = 0; c < NC; ++c, ++it) {
                const int s = it % NSTAGE;
                const uint32_t ph = (it / NSTAGE) & 1;
                if (!mbar_wait(full0 + 8 * s, ph, abort_flag, WAIT_LIMIT_NS)) { ok = false; break; }
                fence_after();
                const uint32_t ah = smem_u32(smem + s * STAGE_BYTES), al = ah + A_BYTES;
                const uint32_t bh = ah + 2 * A_BYTES, bl = bh + B_BYTES;
#pragma unroll
                for (int kk = 0; kk < KC / 8; ++kk) {
                    if (c * KC + kk * 8 >= a.K) break;  // zero padding only (K >= 1: the first step always runs)
                    const uint32_t o = kk * 32;  // 8 tf32 = 32 B along K inside the 64-byte swizzle row
                    mma_tf32(d, sdesc(ah + o), sdesc(bh + o), (c | kk) != 0);
                    mma_tf32(d, sdesc(ah + o), sdesc(bl + o), 1);
                    mma_tf32(d, sdesc(al + o), sdesc(bh + o), 1);
                }
                any = true;
                mma_commit(empty0 + 8 * s);
            }
            if (!ok) break;
            mma_commit(tfull0 + 8 * acc);
        }
        if (!ok && any) {
            mma_commit(drain);
            const uint64_t t0 = globaltimer();
            while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < DRAIN_LIMIT_NS) {
            }
        }
    } else if (warp >= 4) {
        // ---------------------------------------------------------------- epilogue
        const int q = warp & 3;
        const int row = 32 * q + lane;
        const bool issuer = (warp == 4 && lane == 0);
        uint32_t j = 0, box = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
            const int nt = t % num_n, mt = t / num_n;
            const uint32_t acc = j & 1, aph = (j >> 1) & 1;
            const bool ok = mbar_wait(tfull0 + 8 * acc, aph, abort_flag, WAIT_LIMIT_NS);
            if (a.direct) {
                if (!epi_all(ok)) break;
            } else if (!ok) {
                break;
            }
            fence_after();
            const int col = mt * TM + row;
            const bool col_ok = col < a.M;
            const int ch = col & 3;
            for (int n0 = 0; n0 < TN; n0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + acc * TN + n0, r);
                if (n0 + 32 == TN) {
                    // the accumulator is in registers: the next tile's MMAs may start
                    fence_before();
                    mbar_arrive(tempty0 + 8 * acc);
                }
                const int g0 = nt * TN + n0;
                if (a.direct) {
                    if (g0 >= a.G) continue;  // block-uniform: whole box beyond the last glyph
                    float* buf = obuf + (box % NOUT) * (OG * TM);
                    if (issuer) bulk_wait_read_free();  // the store issued NOUT boxes ago has read `buf`
                    epi_bar();
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        float v = __uint_as_float(r[i]);
                        if (ch == 0 && a.view.r0 && g0 + i < a.G) v -= __ldg(a.view.r0 + g0 + i);
                        buf[i * TM + row] = v;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    epi_bar();
                    if (issuer) {
                        tma_store_2d(&mOut, smem_u32(buf), mt * TM, g0);  // clipped at M columns, G rows
                        bulk_commit();
                    }
                    ++box;
                } else {
                    // gather the four channels of a texel into the lane holding channel 0
                    const int P = a.view.N_uniform + 2;
                    const int tex = col >> 2;
                    const int f = tex / (P * P), rem = tex % (P * P), jj = rem / P, ii = rem % P;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float v0 = __uint_as_float(r[i]);
                        const float v1 = __shfl_down_sync(0xffffffffu, v0, 1);
                        const float v2 = __shfl_down_sync(0xffffffffu, v0, 2);
                        const float v3 = __shfl_down_sync(0xffffffffu, v0, 3);
                        const int g = g0 + i;
                        if (ch == 0 && g < a.G && col_ok) {
                            const GlyphRef Gr = glyph_ref(a.view, g);
                            store_texel(a.data, a.view.dtype, a.view.layout, Gr, f, jj, ii,
                                        make_float4(v0 - Gr.r0, v1, v2, v3));
                        }
                    }
                }
            }
        }
        if (issuer) bulk_wait_all();
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag && a.dev_status) atomicOr(a.dev_status, SHM_DEV_TIMEOUT);
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// rows x K float32 (row stride ld_in) -> hi, lo [rows][Kp] (zero padded)
__global__ void k_split_rows(const float* __restrict__ in, int rows, int K, int64_t ld_in, int64_t col_stride,
                             int Kp, float* __restrict__ hi, float* __restrict__ lo)
{
    const int64_t n = (int64_t)rows * Kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Kp;
        const int k = (int)(e % Kp);
        const float v = (k < K) ? __ldg(in + r * col_stride + (int64_t)k * ld_in) : 0.0f;
        const float h = tf32_rna(v);
        hi[e] = h;
        lo[e] = tf32_rna(v - h);
    }
}

static bool make_map(CUtensorMap* m, const float* base, int rows, int Kp, int box_rows)
{
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
    const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output table as a 2-D tensor [G rows][M columns] f32 (row pitch M * 4 B, a multiple of 16 since
// M = 4 * 6 (N+2)^2), stored in boxes of [OG glyphs][TM columns] without swizzle.
static bool make_out_map(CUtensorMap* m, float* base, int G, int M)
{
    EncodeFn enc = encode_fn();
    if (!enc || ((uintptr_t)base & 15u) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)G};
    const cuuint64_t strides[1] = {(cuuint64_t)M * 4};
    const cuuint32_t box[2] = {(cuuint32_t)TM, (cuuint32_t)OG};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


}  // namespace tc

// K padded to a multiple of 32 (a multiple of the stage K; the layout is part of shm_sh_basis's contract)
int sh_kpad(int L) { return (((L + 1) * (L + 1) + 31) / 32) * 32; }

int64_t sh_build_workspace_bytes(int G, int L) { return 2LL * G * sh_kpad(L) * (int64_t)sizeof(float); }

// basis: [K][M] float32 (full), followed by hi [M][Kp] and lo [M][Kp]
cudaError_t launch_basis_split(int N, int L, float* basis, cudaStream_t s)
{
    const int K = (L + 1) * (L + 1), Kp = sh_kpad(L), M = 4 * 6 * (N + 2) * (N + 2);
    float* hi = basis + (int64_t)K * M;
    float* lo = hi + (int64_t)M * Kp;
    const int64_t n = (int64_t)M * Kp;
    tc::k_split_rows<<<(unsigned)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8), 256, 0, s>>>(
        basis, M, K, (int64_t)M, 1, Kp, hi, lo);
    return cudaGetLastError();
}

cudaError_t launch_sh_build_tc(const LutView& out, void* data, int L, const float* coeffs, const float* basis,
                               void* ws, cudaStream_t s, int32_t* dev_status)
{
    const int N = out.N_uniform, G = out.n_glyphs;
    const int K = (L + 1) * (L + 1), Kp = sh_kpad(L), M = 4 * 6 * (N + 2) * (N + 2);
    float* chi = reinterpret_cast<float*>(ws);
    float* clo = chi + (int64_t)G * Kp;
    const int64_t n = (int64_t)G * Kp;
    tc::k_split_rows<<<(unsigned)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8), 256, 0, s>>>(
        coeffs, G, K, 1, (int64_t)K, Kp, chi, clo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float* bhi = basis + (int64_t)K * M;
    const float* blo = bhi + (int64_t)M * Kp;
    CUtensorMap mAh, mAl, mBh, mBl, mOut;
    if (!tc::make_map(&mAh, bhi, M, Kp, tc::TM) || !tc::make_map(&mAl, blo, M, Kp, tc::TM) ||
        !tc::make_map(&mBh, chi, G, Kp, tc::TN) || !tc::make_map(&mBl, clo, G, Kp, tc::TN))
        return cudaErrorInvalidValue;
    const bool direct = (out.dtype == SHM_F32 && out.layout == SHM_LAYOUT_TEXEL);
    if (direct) {
        if (!tc::make_out_map(&mOut, reinterpret_cast<float*>(data), G, M)) return cudaErrorInvalidValue;
    } else {
        mOut = mAh;  // unused by the generic epilogue
    }
    tc::Args a;
    a.M = M;
    a.G = G;
    a.Kp = Kp;
    a.K = K;
    a.view = out;
    a.data = data;
    a.out = reinterpret_cast<float*>(data);
    a.direct = direct ? 1 : 0;
    a.dev_status = dev_status;
    e = ensure_dynamic_smem((const void*)tc::k_sh_gemm_tc, (int)tc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int tiles = ((M + tc::TM - 1) / tc::TM) * ((G + tc::TN - 1) / tc::TN);
    int grid = sm_count();
    if (grid > tiles) grid = tiles;
    tc::k_sh_gemm_tc<<<grid, 256, tc::SMEM_BYTES, s>>>(mAh, mAl, mBh, mBl, mOut, a);
    return cudaGetLastError();
}


}  // namespace shm
