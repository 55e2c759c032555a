// Staged query (§3.2-§3.4) for per-glyph query segments on tables that fit in shared memory.
//
// With CSR segments every glyph's queries are contiguous, so a CTA can take a whole glyph: one
// bulk copy (cp.async.bulk, completion on an mbarrier) brings the glyph's padded table into shared
// memory, then the CTA answers all of that glyph's queries from it.  The table is read from HBM
// once, the 2x2 footprints become shared-memory reads, and HBM sees only the bulk copy and the
// coalesced direction / output streams (for N = 32, f32: 111 KB + 4,096 x 40 B per glyph), instead
// of texel reads that miss L1 about half of the time.  Two CTAs per SM overlap one CTA's copy with
// the other's queries.
//
// Results are bit-identical to k_query_fwd (same device functions on the same values).  Directions
// and outputs are touched once, so they are loaded and stored with the streaming cache hint
// (__ldcs / __stcs: evict first) and leave L2 to the tables.
// The wait for the copy is bounded (1 s); on expiry the CTA raises SHM_DEV_TIMEOUT, waits up to
// 100 ms more for its copy to land and returns without touching the outputs of that glyph.
#include "shm_stage.cuh"

namespace shm {

namespace {

// Launch shapes of the staged kernel: threads per CTA (shape 0 = 512, the default; 1 = 1,024;
// 2 = 256), with <= 64 registers so that 1,024 threads per SM fit; how many CTAs actually share
// an SM is set by the table's shared-memory footprint.
constexpr int N_SSHAPES = 3;
constexpr int SSHAPES[N_SSHAPES] = {512, 1024, 256};

// STD: the usual output set (R, gradient and normal; no chart derivatives, no cell indices), so the
// per-query output checks drop out of the loop.
template <int DT, int SBLOCK, bool STD>
__global__ void __launch_bounds__(SBLOCK, 1024 / SBLOCK) k_query_staged(QueryArgs a, uint32_t table_bytes)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(smem);
    const unsigned char* table = smem + stage::TABLE_OFFSET;
    const uint32_t table_s = bar + stage::TABLE_OFFSET;
    const int tid = threadIdx.x;
    const int G = a.L.n_glyphs, N = a.L.N_uniform, P = N + 2;
    const float qnan = __int_as_float(0x7fc00000);
    uint32_t status = 0;

    // queries outside every segment: NaN and SHM_DEV_BOUNDS, as in the unstaged kernel
    {
        const int64_t lo = min(max(__ldg(a.seg), (int64_t)0), a.Q);
        const int64_t hi = min(max(__ldg(a.seg + G), lo), a.Q);
        const int64_t stride = (int64_t)gridDim.x * SBLOCK;
        for (int part = 0; part < 2; ++part) {
            const int64_t b = part ? hi : 0, e = part ? a.Q : lo;
            for (int64_t q = b + (int64_t)blockIdx.x * SBLOCK + tid; q < e; q += stride) {
                status |= SHM_DEV_BOUNDS;
                if (a.R) a.R[q] = qnan;
                if (a.grad) { a.grad[3 * q] = qnan; a.grad[3 * q + 1] = qnan; a.grad[3 * q + 2] = qnan; }
                if (a.normal) { a.normal[3 * q] = qnan; a.normal[3 * q + 1] = qnan; a.normal[3 * q + 2] = qnan; }
                if (a.chart) { a.chart[2 * q] = qnan; a.chart[2 * q + 1] = qnan; }
                if (a.fij) { a.fij[3 * q] = -1; a.fij[3 * q + 1] = -1; a.fij[3 * q + 2] = -1; }
            }
        }
    }

    if (tid == 0) {
        stage::init(bar);
        s_abort = 0;
    }
    __syncthreads();

    uint32_t phase = 0;
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t s0 = min(max(__ldg(a.seg + g), (int64_t)0), a.Q);
        const int64_t s1 = min(max(__ldg(a.seg + g + 1), s0), a.Q);
        if (s1 <= s0) continue;  // block-uniform
        if (tid == 0)
            stage::issue(bar, table_s, reinterpret_cast<const unsigned char*>(a.L.data) + (size_t)g * table_bytes,
                         table_bytes);
        // first direction of this thread while the copy runs
        int64_t q = s0 + tid;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (q < s1) { d0 = __ldcs(a.dirs + 3 * q); d1 = __ldcs(a.dirs + 3 * q + 1); d2 = __ldcs(a.dirs + 3 * q + 2); }
        if (!stage::bar_wait(bar, phase, stage::WAIT_NS)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            status |= SHM_DEV_TIMEOUT;
            if (tid == 0) stage::bar_wait(bar, phase, stage::DRAIN_NS);
            break;
        }
        phase ^= 1;
        const float r0 = a.L.r0 ? __ldg(a.L.r0 + g) : 0.0f;
        for (; q < s1; q += SBLOCK) {
            const int64_t qn = q + SBLOCK;
            float n0 = 0.f, n1 = 0.f, n2 = 0.f;
            if (qn < s1) { n0 = __ldcs(a.dirs + 3 * qn); n1 = __ldcs(a.dirs + 3 * qn + 1); n2 = __ldcs(a.dirs + 3 * qn + 2); }
            Chart c;
            float R = qnan, Ru = qnan, Rv = qnan;
            Vec3 grad{qnan, qnan, qnan}, nrm{qnan, qnan, qnan};
            int f = -1, i = -1, j = -1;
            if (chart_of(d0, d1, d2, c)) {
                float s, t;
                cell_of(pick3(c.k1, d0, d1, d2), c.m, c.im, N, i, s);
                cell_of(pick3(c.k2, d0, d1, d2), c.m, c.im, N, j, t);
                const Corners cr = stage::corners<DT>(table, P, c.f, i, j);
                const HermOut h = hermite2(cr, s, t);
                R = r0 + h.r;
                Ru = (float)N * h.rs;
                Rv = (float)N * h.rt;
                grad = s2_gradient(c, Ru, Rv);
                if (STD || a.normal) nrm = surface_normal(d0, d1, d2, R, grad);
                f = c.f;
            } else {
                status |= SHM_DEV_NONFINITE;
            }
            if (STD || a.R) __stcs(a.R + q, R);
            if (STD || a.grad) { __stcs(a.grad + 3 * q, grad.x); __stcs(a.grad + 3 * q + 1, grad.y); __stcs(a.grad + 3 * q + 2, grad.z); }
            if (STD || a.normal) { __stcs(a.normal + 3 * q, nrm.x); __stcs(a.normal + 3 * q + 1, nrm.y); __stcs(a.normal + 3 * q + 2, nrm.z); }
            if (!STD && a.chart) { a.chart[2 * q] = Ru; a.chart[2 * q + 1] = Rv; }
            if (!STD && a.fij) { a.fij[3 * q] = f; a.fij[3 * q + 1] = i; a.fij[3 * q + 2] = j; }
            d0 = n0; d1 = n1; d2 = n2;
        }
        __syncthreads();  // every read of this table is done before the next copy lands
    }
    report_status(a.dev_status, status);
}

template <int DT, int SBLOCK, bool STD>
cudaError_t launch_staged_o(const QueryArgs& a, uint32_t table_bytes, cudaStream_t s)
{
    const int smem = stage::TABLE_OFFSET + (int)table_bytes;
    cudaError_t e = ensure_dynamic_smem((const void*)k_query_staged<DT, SBLOCK, STD>, smem);
    if (e != cudaSuccess) return e;
    int resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_query_staged<DT, SBLOCK, STD>, SBLOCK, smem) !=
            cudaSuccess ||
        resident < 1)
        resident = 1;
    int64_t blocks = (int64_t)sm_count() * resident;
    if (blocks > a.L.n_glyphs) blocks = a.L.n_glyphs;
    if (blocks < 1) blocks = 1;
    k_query_staged<DT, SBLOCK, STD><<<(unsigned)blocks, SBLOCK, smem, s>>>(a, table_bytes);
    return cudaGetLastError();
}

template <int DT, int SBLOCK>
cudaError_t launch_staged_t(const QueryArgs& a, uint32_t table_bytes, cudaStream_t s)
{
    const bool std_outputs = a.R && a.grad && a.normal && !a.chart && !a.fij;
    return std_outputs ? launch_staged_o<DT, SBLOCK, true>(a, table_bytes, s)
                       : launch_staged_o<DT, SBLOCK, false>(a, table_bytes, s);
}

template <int DT>
cudaError_t launch_staged_shape(const QueryArgs& a, uint32_t table_bytes, int shape, cudaStream_t s)
{
    switch (shape) {
    case 1: return launch_staged_t<DT, SSHAPES[1]>(a, table_bytes, s);
    case 2: return launch_staged_t<DT, SSHAPES[2]>(a, table_bytes, s);
    default: return launch_staged_t<DT, SSHAPES[0]>(a, table_bytes, s);
    }
}

}  // namespace

int staged_shapes() { return N_SSHAPES; }

cudaError_t launch_query_staged(const QueryArgs& a, int shape, cudaStream_t s)
{
    const int64_t P = (int64_t)a.L.N_uniform + 2;
    const int64_t rb = (a.L.dtype == SHM_F32) ? 16 : 8;
    const uint32_t table_bytes = (uint32_t)(6 * P * P * rb);
    if (a.L.dtype == SHM_F32) return launch_staged_shape<SHM_F32>(a, table_bytes, shape, s);
    if (a.L.dtype == SHM_F16) return launch_staged_shape<SHM_F16>(a, table_bytes, shape, s);
    return launch_staged_shape<SHM_BF16>(a, table_bytes, shape, s);
}

}  // namespace shm
