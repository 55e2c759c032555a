// Binned query (§3.2-§3.4) for one table larger than L2 queried in random order (the procedural
// planet of §4.10: N = 2048, 403 MB f32).
//
// Unsorted, every query's 2x2 footprint lands in a different part of the table, so each query
// pulls two or three 32 B sectors from DRAM (random sector rate, not streaming bandwidth, sets
// the pace).  Here the batch is first partitioned by the table region its footprint reads: bin =
// (face, band of cell rows), a band holding a few MB of records.  The query kernel then walks the
// partitioned batch in order, so the few bands in flight at any moment stay resident in L2 and
// the table is read from DRAM about once per pass; everything else is coalesced streaming.
//
//   1. k_bin_count    per query its bin (one byte), per tile of TILE queries the
//                     histogram of bins                                             (12 B/q in, 1 B/q out)
//   2. k_bin_scan     per bin: exclusive scan of the tile counts                    (tiny)
//   3. k_bin_scatter  stable partition of the directions into bin order            (13 B/q in, 12 B/q out)
//   4. k_bin_query    the query's chart, cell, footprint and Hermite steps on the
//                     partitioned directions, writing R, R_u, R_v only              (12 B/q in, 12 B/q out)
//   5. k_bin_finish   per original tile: the same positions as step 3 locate each
//                     query's (R, R_u, R_v); the S^2 gradient and normal (§3.4) are
//                     recomputed from the original direction and written in query
//                     order                                                         (25 B/q in, 28 B/q out)
//
// Steps 3 and 5 derive every query's partitioned position by the same deterministic procedure
// (stable within a tile: rounds of RQ queries, warps in order, lanes in order) from the bin
// bytes of step 1, so no permutation array is stored and no bin is ever computed twice.  Per
// query the arithmetic is that of shm_query: the chart, cell, footprint and Hermite sums run in
// step 4, the S^2 gradient and normal in step 5 on the same float32 values, so the outputs equal
// shm_query's.
#include "shm_stage.cuh"

namespace shm {

namespace {

constexpr int BB = 256;            // threads per CTA of the partition kernels
constexpr int NW = BB / 32;        // warps
constexpr int SUBR = 8;            // 32-query sub-rounds per warp and round
constexpr int RQ = BB * SUBR;      // queries per round (a warp takes SUBR * 32 consecutive ones)
constexpr int ROUNDS = 8;          // rounds per tile
constexpr int64_t TILE = (int64_t)RQ * ROUNDS;
constexpr int MAXB = 256;          // bins at most (bin ids are stored as bytes)
constexpr int SCAN_T = 1024;       // threads of the scan kernel
constexpr int SCAN_PER = 8;        // counts per scan thread and chunk

struct BinParams {
    int N;          // interior resolution of glyph 0
    int band_rows;  // cell rows per band
    int nb;         // bands per face
    int B;          // bins = 6 nb
    int64_t nT;     // tiles
    int64_t Q;
    int bulk;       // directions in device memory, 16-byte aligned: rounds arrive by bulk copies
    int nbits;      // bits of the largest bin id
};

// Bin of a direction: face and band of the chart coordinate v (§3.2).  Only the partition uses it
// and every later step reads the stored byte, so it may be approximate: one fast reciprocal, no
// exact cell arithmetic; a query near a band edge may land in the neighbouring band, which costs
// nothing but locality.  Zero / non-finite directions go to bin 0; the query kernel flags them.
__device__ __forceinline__ int bin_of(const BinParams& p, float d0, float d1, float d2)
{
    const float a0 = fabsf(d0), a1 = fabsf(d1), a2 = fabsf(d2);
    int k = 0;
    float m = a0;
    if (a1 > m) { k = 1; m = a1; }
    if (a2 > m) { k = 2; m = a2; }
    if (!(m > 0.0f) || !(m <= 3.402823466e38f)) return 0;
    const float dk = pick3(k, d0, d1, d2);
    const float dv = pick3(k == 0 ? 2 : k - 1, d0, d1, d2);  // the chart's second axis c_f
    const int f = 2 * k + (dk < 0.0f ? 1 : 0);
    const float x = fmaf(__fdividef(dv, m), 0.5f * (float)p.N, 0.5f * (float)(p.N + 1));  // v N + 1/2
    int j = (int)x;  // x >= 0 up to rounding; the clamp covers the rest
    j = min(max(j, 0), p.N);
    if (!(x == x)) j = 0;
    return f * p.nb + j / p.band_rows;
}

__device__ __forceinline__ void load_dir(const float* dirs, int64_t q, float& d0, float& d1, float& d2)
{
    d0 = __ldcs(dirs + 3 * q);
    d1 = __ldcs(dirs + 3 * q + 1);
    d2 = __ldcs(dirs + 3 * q + 2);
}

// ---------------------------------------------------------------------------------- 1. count
// Warp w of the CTA takes queries [t TILE + w TILE/NW, +TILE/NW) in passes of 8 x 32; each lane
// issues all 24 direction loads of a pass before computing any bin, so the SM keeps enough
// bytes in flight for this pure stream.
__global__ void __launch_bounds__(BB) k_bin_count(BinParams p, const float* __restrict__ dirs,
                                                  unsigned char* __restrict__ binb, int32_t* __restrict__ cnt)
{
    __shared__ int hist[NW][MAXB];  // per warp, so that conflicting increments stay within a warp
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < NW * MAXB; i += BB) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t t = blockIdx.x;
    const int64_t wq0 = t * TILE + (int64_t)w * (TILE / NW);
    const int64_t wq1 = min(wq0 + TILE / NW, p.Q);
    for (int64_t qb = wq0; qb < wq1; qb += 8 * 32) {
        float d[8][3];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t q = qb + k * 32 + lane;
            d[k][0] = d[k][1] = d[k][2] = 0.0f;
            if (q < wq1) load_dir(dirs, q, d[k][0], d[k][1], d[k][2]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t q = qb + k * 32 + lane;
            if (q < wq1) {
                const int b = bin_of(p, d[k][0], d[k][1], d[k][2]);
                __stcs(binb + q, (unsigned char)b);
                atomicAdd(&hist[w][b], 1);
            }
        }
    }
    __syncthreads();
    for (int b = tid; b < p.B; b += BB) {
        int c = 0;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) c += hist[ww][b];
        cnt[(int64_t)b * p.nT + t] = c;
    }
}

// ---------------------------------------------------------------------------------- 2. scan
// Exclusive scan of a block's values (one per thread) in thread order; returns the block total.
template <int T>
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long& total, long long* wtot)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = (lane < T / 32) ? wtot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < T / 32) wtot[lane] = s;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const long long before = (w > 0 ? wtot[w - 1] : 0) + x - v;
    total = wtot[T / 32 - 1];
    __syncthreads();  // wtot is reused by the next call
    return before;
}

// One CTA per bin: off[b][t] = sum of cnt[b][t'] over t' < t; tot[b] = the bin's total.
__global__ void __launch_bounds__(SCAN_T) k_bin_scan(BinParams p, const int32_t* __restrict__ cnt,
                                                     long long* __restrict__ off, long long* __restrict__ tot)
{
    __shared__ long long wtot[SCAN_T / 32];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int32_t* c = cnt + (int64_t)b * p.nT;
    long long* o = off + (int64_t)b * p.nT;
    long long carry = 0;
    for (int64_t c0 = 0; c0 < p.nT; c0 += (int64_t)SCAN_T * SCAN_PER) {
        const int64_t i0 = c0 + (int64_t)tid * SCAN_PER;
        int v[SCAN_PER];
        long long s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_PER; ++k) {
            v[k] = (i0 + k < p.nT) ? c[i0 + k] : 0;
            s += v[k];
        }
        long long total;
        long long run = carry + block_exclusive_scan<SCAN_T>(s, total, wtot);
#pragma unroll
        for (int k = 0; k < SCAN_PER; ++k) {
            if (i0 + k < p.nT) o[i0 + k] = run;
            run += v[k];
        }
        carry += total;
    }
    if (tid == 0) tot[b] = carry;
}

// ---------------------------------------------------------------------------------- 3./5. positions
// A round's inputs in original order (directions and bin bytes), brought into shared memory by
// bulk copies (cp.async.bulk on an mbarrier, double-buffered: the next round's copy runs while
// this round is ranked and written), or by plain loads for a short last round.  The finish kernel
// stages the bin bytes only.
template <bool DIRS>
struct RoundIn;
template <>
struct RoundIn<true> {
    float dirs[RQ * 3];
    unsigned char bins[RQ];
};
template <>
struct RoundIn<false> {
    unsigned char bins[RQ];
};
constexpr uint32_t ROUND_DIR_BYTES = RQ * 12, ROUND_BIN_BYTES = RQ;

struct RoundSmem {
    unsigned long long bar[2];   // one mbarrier per input buffer
    int wcnt[NW][MAXB];          // per warp: running count per bin, then the warp's prefix within the round
    int rstart[MAXB];            // first slot of each bin in the round's partitioned order
    long long gdst[MAXB];        // global position of round slot e of bin b = gdst[b] + e
    long long run[MAXB];         // next global position of each bin for this tile
    long long wtot[BB / 32];
    unsigned short slot_src[RQ]; // round slot -> the query's index within the round
    unsigned short src_slot[RQ]; // the query's index within the round -> round slot
    int last_issue[2];           // last round bulk-copied into each buffer (-1: none)
    int abort_flag;
};

constexpr int SCATTER_DYN_SMEM = 2 * (int)sizeof(RoundIn<true>);
constexpr int FINISH_DYN_SMEM = 2 * (int)sizeof(RoundIn<false>);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// A full round comes by bulk copy; the directions only when bulk copies can read them (p.bulk).
template <bool DIRS>
__device__ __forceinline__ bool round_is_bulk(const BinParams& p, int64_t q0)
{
    return (!DIRS || p.bulk) && q0 + RQ <= p.Q;
}

// Lanes of the warp holding the same bin as this lane (b in [0, 256), or -1 for no query):
// peers by one ballot per bin bit, a cost independent of how many distinct bins the warp holds.
__device__ __forceinline__ unsigned bin_peers(int b, int nbits)
{
    unsigned peers = __ballot_sync(0xffffffffu, b >= 0);
    if (b < 0) peers = ~peers;
    for (int k = 0; k < nbits; ++k) {
        const bool bit = (b >> k) & 1;
        const unsigned m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// Thread 0: bulk copies of a full round's inputs into buffer `in`, completing on `bar`.
template <bool DIRS>
__device__ __forceinline__ void round_issue(const float* dirs, const unsigned char* binb, int64_t q0,
                                            RoundIn<DIRS>& in, uint32_t bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((DIRS ? ROUND_DIR_BYTES : 0u) + ROUND_BIN_BYTES)
                 : "memory");
    if constexpr (DIRS)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(in.dirs)), "l"(dirs + 3 * q0), "r"(ROUND_DIR_BYTES), "r"(bar)
                     : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(in.bins)), "l"(binb + q0), "r"(ROUND_BIN_BYTES), "r"(bar)
                 : "memory");
}

// Tile set-up: run[b] = (queries of bins < b) + (queries of bin b in tiles < t); wcnt cleared;
// barriers initialised.
__device__ __forceinline__ void tile_setup(const BinParams& p, int64_t t, const long long* __restrict__ off,
                                           const long long* __restrict__ tot, RoundSmem& sm)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        stage::init(smem_u32(&sm.bar[0]));
        stage::init(smem_u32(&sm.bar[1]));
        sm.last_issue[0] = sm.last_issue[1] = -1;
        sm.abort_flag = 0;
    }
    const long long v = (tid < p.B) ? tot[tid] : 0;
    long long total;
    const long long base = block_exclusive_scan<BB>(v, total, sm.wtot);
    if (tid < p.B) sm.run[tid] = base + off[(int64_t)tid * p.nT + t];
    for (int i = tid; i < NW * MAXB; i += BB) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
}

// Thread 0 after an abort: wait (bounded) for the bulk copies still in flight before the CTA exits.
__device__ __forceinline__ void round_drain(RoundSmem& sm, int32_t* dev_status)
{
    if (threadIdx.x != 0) return;
    if (dev_status) atomicOr(dev_status, SHM_DEV_TIMEOUT);
    for (int b = 0; b < 2; ++b)
        if (sm.last_issue[b] >= 0)
            (void)stage::bar_wait(smem_u32(&sm.bar[b]), (uint32_t)((sm.last_issue[b] >> 1) & 1), stage::DRAIN_NS);
}

// Rounds of tile t that hold queries, and the size of round r.
__device__ __forceinline__ int tile_rounds(const BinParams& p, int64_t t)
{
    const int64_t n = min(TILE, p.Q - t * TILE);
    return (int)((n + RQ - 1) / RQ);
}

__device__ __forceinline__ int round_size(const BinParams& p, int64_t q0) { return (int)min((int64_t)RQ, p.Q - q0); }

// Thread 0: start the bulk copy of round r (if it is a bulk round) into buffer r & 1.
template <bool DIRS>
__device__ __forceinline__ void round_prefetch(const BinParams& p, const float* dirs, const unsigned char* binb,
                                               int64_t t, int r, int nr, RoundIn<DIRS>* in, RoundSmem& sm)
{
    const int64_t q0 = t * TILE + (int64_t)r * RQ;
    if (threadIdx.x != 0 || r >= nr || !round_is_bulk<DIRS>(p, q0)) return;
    round_issue<DIRS>(dirs, binb, q0, in[r & 1], smem_u32(&sm.bar[r & 1]));
    sm.last_issue[r & 1] = r;
}

// Makes round r's inputs available in `in`: waits for its bulk copy or loads it with plain loads
// (short last round, or directions that bulk copies cannot read).  Returns false if the copy did
// not land within the limit.
template <bool DIRS>
__device__ __forceinline__ bool round_acquire(const BinParams& p, const float* __restrict__ dirs,
                                              const unsigned char* __restrict__ binb, int64_t q0, int n_el,
                                              RoundIn<DIRS>& in, RoundSmem& sm, int r)
{
    if (round_is_bulk<DIRS>(p, q0)) {
        if (!stage::bar_wait(smem_u32(&sm.bar[r & 1]), (uint32_t)((r >> 1) & 1), stage::WAIT_NS)) sm.abort_flag = 1;
    } else {
        if constexpr (DIRS)
            for (int i = threadIdx.x; i < 3 * n_el; i += BB) in.dirs[i] = __ldcs(dirs + 3 * q0 + i);
        for (int i = threadIdx.x; i < n_el; i += BB) in.bins[i] = __ldcs(binb + q0 + i);
    }
    __syncthreads();
    return sm.abort_flag == 0;
}

// Ranks of round r: query i of the round (original order) gets its slot in the round's
// partitioned order, stable by i.  Warp w ranks queries w SUBR 32 + k 32 + lane, k < SUBR;
// then per bin the warps' counts are prefixed and the bins' starts and global targets formed.
// Leaves slot_src / src_slot filled and the warp prefixes in wcnt.
template <bool DIRS>
__device__ __forceinline__ void round_rank(const BinParams& p, const RoundIn<DIRS>& in, int n_el, RoundSmem& sm)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int bk[SUBR], rk[SUBR];
#pragma unroll
    for (int k = 0; k < SUBR; ++k) {
        const int i = w * (SUBR * 32) + k * 32 + lane;
        const int b = (i < n_el) ? (int)in.bins[i] : -1;
        const unsigned peers = bin_peers(b, p.nbits);
        int r = 0;
        if (b >= 0) r = sm.wcnt[w][b] + __popc(peers & lt);
        __syncwarp();
        if (b >= 0 && (peers & lt) == 0) sm.wcnt[w][b] += __popc(peers);
        __syncwarp();
        bk[k] = b;
        rk[k] = r;
    }
    __syncthreads();
    long long c = 0;
    if (tid < p.B) {
        int acc = 0;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) {
            const int x = sm.wcnt[ww][tid];
            sm.wcnt[ww][tid] = acc;
            acc += x;
        }
        c = acc;
    }
    long long total;
    const long long start = block_exclusive_scan<BB>(c, total, sm.wtot);
    if (tid < p.B) {
        sm.rstart[tid] = (int)start;
        sm.gdst[tid] = sm.run[tid] - start;
        sm.run[tid] += c;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SUBR; ++k) {
        if (bk[k] < 0) continue;
        const int i = w * (SUBR * 32) + k * 32 + lane;
        const int e = sm.rstart[bk[k]] + sm.wcnt[w][bk[k]] + rk[k];
        sm.slot_src[e] = (unsigned short)i;
        sm.src_slot[i] = (unsigned short)e;
    }
    __syncthreads();
    for (int i = tid; i < NW * MAXB; i += BB) (&sm.wcnt[0][0])[i] = 0;
}

// ---------------------------------------------------------------------------------- 3. scatter
__global__ void __launch_bounds__(BB) k_bin_scatter(BinParams p, const float* __restrict__ dirs,
                                                    const unsigned char* __restrict__ binb,
                                                    const long long* __restrict__ off,
                                                    const long long* __restrict__ tot, float* __restrict__ sorted,
                                                    int32_t* __restrict__ dev_status)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    RoundIn<true>* in = reinterpret_cast<RoundIn<true>*>(dsm);
    __shared__ RoundSmem sm;
    const int64_t t = blockIdx.x;
    tile_setup(p, t, off, tot, sm);
    const int nr = tile_rounds(p, t);
    round_prefetch<true>(p, dirs, binb, t, 0, nr, in, sm);
    for (int r = 0; r < nr; ++r) {
        const int64_t q0 = t * TILE + (int64_t)r * RQ;
        const int n_el = round_size(p, q0);
        round_prefetch<true>(p, dirs, binb, t, r + 1, nr, in, sm);
        RoundIn<true>& cur = in[r & 1];
        if (!round_acquire<true>(p, dirs, binb, q0, n_el, cur, sm, r)) break;
        round_rank<true>(p, cur, n_el, sm);
        // copy-out by slot: consecutive slots of a bin's run go to consecutive addresses
#pragma unroll 4
        for (int e = threadIdx.x; e < n_el; e += BB) {
            const int i = sm.slot_src[e];
            const long long dst = sm.gdst[cur.bins[i]] + e;
            if (dst < p.Q) {
                __stcs(sorted + 3 * dst, cur.dirs[3 * i]);
                __stcs(sorted + 3 * dst + 1, cur.dirs[3 * i + 1]);
                __stcs(sorted + 3 * dst + 2, cur.dirs[3 * i + 2]);
            }
        }
        __syncthreads();
    }
    if (sm.abort_flag) round_drain(sm, dev_status);  // a bulk copy never landed
}

// ---------------------------------------------------------------------------------- 5. finish
// Per round: the bins arrive by bulk copy and are ranked as in step 3; then each thread takes its
// queries in original order, loads the direction (coalesced) and the query's (R, R_u, R_v) from its
// slot of the partitioned order (a bin's slots are contiguous, so a CTA's loads of a round touch
// B short runs that L1 keeps), forms the S^2 gradient and normal and stores them coalesced.
constexpr int FHALF = RQ / BB / 2;  // queries per thread in flight at once

__global__ void __launch_bounds__(BB) k_bin_finish(BinParams p, const float* __restrict__ dirs,
                                                   const unsigned char* __restrict__ binb,
                                                   const long long* __restrict__ off,
                                                   const long long* __restrict__ tot, const float* __restrict__ Rs,
                                                   const float2* __restrict__ cs, float* __restrict__ R,
                                                   float* __restrict__ grad, float* __restrict__ normal,
                                                   float* __restrict__ chart, int32_t* __restrict__ dev_status)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    RoundIn<false>* in = reinterpret_cast<RoundIn<false>*>(dsm);
    __shared__ RoundSmem sm;
    const int64_t t = blockIdx.x;
    const float qnan = __int_as_float(0x7fc00000);
    tile_setup(p, t, off, tot, sm);
    const int nr = tile_rounds(p, t);
    round_prefetch<false>(p, dirs, binb, t, 0, nr, in, sm);
    for (int r = 0; r < nr; ++r) {
        const int64_t q0 = t * TILE + (int64_t)r * RQ;
        const int n_el = round_size(p, q0);
        round_prefetch<false>(p, dirs, binb, t, r + 1, nr, in, sm);
        RoundIn<false>& cur = in[r & 1];
        if (!round_acquire<false>(p, dirs, binb, q0, n_el, cur, sm, r)) break;
        round_rank<false>(p, cur, n_el, sm);
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float d[FHALF][3], v[FHALF][3];
#pragma unroll
            for (int k = 0; k < FHALF; ++k) {
                const int i = threadIdx.x + (h * FHALF + k) * BB;
                d[k][0] = d[k][1] = d[k][2] = 0.0f;
                v[k][0] = v[k][1] = v[k][2] = qnan;
                if (i < n_el) {
                    load_dir(dirs, q0 + i, d[k][0], d[k][1], d[k][2]);
                    const long long src = sm.gdst[cur.bins[i]] + sm.src_slot[i];
                    if (src < p.Q) {
                        const float2 c2 = __ldg(cs + src);
                        v[k][0] = __ldg(Rs + src);
                        v[k][1] = c2.x;
                        v[k][2] = c2.y;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < FHALF; ++k) {
                const int i = threadIdx.x + (h * FHALF + k) * BB;
                if (i >= n_el) continue;
                const int64_t q = q0 + i;
                Chart c;
                Vec3 g{qnan, qnan, qnan}, n{qnan, qnan, qnan};
                if (chart_of(d[k][0], d[k][1], d[k][2], c)) {
                    g = s2_gradient(c, v[k][1], v[k][2]);
                    n = surface_normal(d[k][0], d[k][1], d[k][2], v[k][0], g);
                }
                if (R) __stcs(R + q, v[k][0]);
                if (grad) { __stcs(grad + 3 * q, g.x); __stcs(grad + 3 * q + 1, g.y); __stcs(grad + 3 * q + 2, g.z); }
                if (normal) {
                    __stcs(normal + 3 * q, n.x); __stcs(normal + 3 * q + 1, n.y); __stcs(normal + 3 * q + 2, n.z);
                }
                if (chart) { __stcs(chart + 2 * q, v[k][1]); __stcs(chart + 2 * q + 1, v[k][2]); }
            }
        }
        __syncthreads();
    }
    if (sm.abort_flag) round_drain(sm, dev_status);  // a bulk copy never landed
}

// ---------------------------------------------------------------------------------- 4. query
// The query of §3.2-§3.3 on the partitioned directions, keeping R, R_u, R_v only (the S^2 gradient
// and normal follow in step 5).  Same device functions as shm_query, hence the same values.  CTAs
// take consecutive chunks in order, so the bands in flight at any time are the few the current
// chunks cover; each thread keeps QILP queries in flight.
constexpr int QB = 256, QILP = 2, QCH = QB * QILP * 4;  // threads, queries per thread in flight, chunk

template <int DT, int LAYOUT>
__global__ void __launch_bounds__(QB, 4) k_bin_query(LutView L, int64_t Q, const float* __restrict__ sorted,
                                                               float* __restrict__ Rs, float2* __restrict__ cs,
                                                               int32_t* __restrict__ dev_status)
{
    const GlyphRef G = glyph_ref(L, 0);
    const float qnan = __int_as_float(0x7fc00000);
    uint32_t status = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * QCH; c0 < Q; c0 += (int64_t)gridDim.x * QCH) {
#pragma unroll 1
        for (int r = 0; r < QCH; r += QB * QILP) {
            float d[QILP][3];
#pragma unroll
            for (int u = 0; u < QILP; ++u) {
                const int64_t q = c0 + r + u * QB + threadIdx.x;
                d[u][0] = d[u][1] = d[u][2] = 0.0f;
                if (q < Q) load_dir(sorted, q, d[u][0], d[u][1], d[u][2]);
            }
#pragma unroll
            for (int u = 0; u < QILP; ++u) {
                const int64_t q = c0 + r + u * QB + threadIdx.x;
                if (q >= Q) continue;
                QueryResult o;
                Chart c;
                if (!query_one<DT, LAYOUT>(L, G, d[u][0], d[u][1], d[u][2], o, c)) {
                    o.R = o.Ru = o.Rv = qnan;
                    status |= SHM_DEV_NONFINITE;
                }
                __stcs(Rs + q, o.R);
                __stcs(cs + q, make_float2(o.Ru, o.Rv));
            }
        }
    }
    report_status(dev_status, status);
}

template <int DT, int LAYOUT>
cudaError_t launch_bin_query(const LutView& L, int64_t Q, const float* sorted, float* Rs, float2* cs,
                             int32_t* dev_status, cudaStream_t s)
{
    static int resident = 0;
    if (resident == 0) {
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_bin_query<DT, LAYOUT>, QB, 0) != cudaSuccess || r < 1)
            r = 1;
        resident = r;
    }
    int64_t blocks = (Q + QCH - 1) / QCH;
    const int64_t cap = (int64_t)sm_count() * resident;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_bin_query<DT, LAYOUT><<<(unsigned)blocks, QB, 0, s>>>(L, Q, sorted, Rs, cs, dev_status);
    return cudaGetLastError();
}

cudaError_t launch_bin_query_any(const LutView& L, int64_t Q, const float* sorted, float* Rs, float2* cs,
                                 int32_t* dev_status, cudaStream_t s)
{
    if (L.layout == SHM_LAYOUT_TEXEL) {
        if (L.dtype == SHM_F32) return launch_bin_query<SHM_F32, SHM_LAYOUT_TEXEL>(L, Q, sorted, Rs, cs, dev_status, s);
        if (L.dtype == SHM_F16) return launch_bin_query<SHM_F16, SHM_LAYOUT_TEXEL>(L, Q, sorted, Rs, cs, dev_status, s);
        return launch_bin_query<SHM_BF16, SHM_LAYOUT_TEXEL>(L, Q, sorted, Rs, cs, dev_status, s);
    }
    if (L.dtype == SHM_F32) return launch_bin_query<SHM_F32, SHM_LAYOUT_CELL>(L, Q, sorted, Rs, cs, dev_status, s);
    if (L.dtype == SHM_F16) return launch_bin_query<SHM_F16, SHM_LAYOUT_CELL>(L, Q, sorted, Rs, cs, dev_status, s);
    return launch_bin_query<SHM_BF16, SHM_LAYOUT_CELL>(L, Q, sorted, Rs, cs, dev_status, s);
}

constexpr int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

struct BinLayout {
    BinParams p;
    int64_t o_sorted, o_R, o_chart, o_bin, o_cnt, o_off, o_tot, bytes;
};

// Bands of cell rows holding about band_bytes of records each (at least one row, at most 42 bands
// per face so that the 6 faces' bins fit in a byte).
bool binned_plan(const LutView& L, int64_t Q, int64_t band_bytes, BinLayout* out)
{
    if (L.N_uniform <= 0 || Q < 0) return false;
    const int N = L.N_uniform;
    const int64_t rec = (L.layout == SHM_LAYOUT_CELL ? 4 : 1) * (L.dtype == SHM_F32 ? 16 : 8);
    const int64_t row = (int64_t)(L.layout == SHM_LAYOUT_CELL ? N + 1 : N + 2) * rec;
    if (band_bytes <= 0) band_bytes = BINNED_DEFAULT_BAND_BYTES;
    int64_t rows = band_bytes / row;
    if (rows < 1) rows = 1;
    if (rows > N + 1) rows = N + 1;
    int64_t nb = (N + 1 + rows - 1) / rows;
    if (nb > MAXB / 6) {
        nb = MAXB / 6;
        rows = (N + 1 + nb - 1) / nb;
        nb = (N + 1 + rows - 1) / rows;
    }
    BinLayout z;
    z.p.N = N;
    z.p.band_rows = (int)rows;
    z.p.nb = (int)nb;
    z.p.B = (int)(6 * nb);
    z.p.nT = (Q + TILE - 1) / TILE;
    z.p.Q = Q;
    z.p.bulk = 0;
    z.p.nbits = 1;
    while ((1 << z.p.nbits) < z.p.B) ++z.p.nbits;
    int64_t o = 0;
    z.o_sorted = o; o = align256(o + 12 * Q);
    z.o_R = o;      o = align256(o + 4 * Q);
    z.o_chart = o;  o = align256(o + 8 * Q);
    z.o_bin = o;    o = align256(o + Q);
    z.o_cnt = o;    o = align256(o + 4 * (int64_t)z.p.B * z.p.nT);
    z.o_off = o;    o = align256(o + 8 * (int64_t)z.p.B * z.p.nT);
    z.o_tot = o;    o = align256(o + 8 * (int64_t)z.p.B);
    z.bytes = o;
    *out = z;
    return true;
}

}  // namespace

int64_t binned_workspace_bytes(const LutView& L, int64_t Q, int64_t band_bytes)
{
    BinLayout z;
    if (!binned_plan(L, Q, band_bytes, &z)) return -1;
    return z.bytes;
}

int binned_bins(const LutView& L, int64_t band_bytes, int* band_rows)
{
    BinLayout z;
    if (!binned_plan(L, 0, band_bytes, &z)) return -1;
    if (band_rows) *band_rows = z.p.band_rows;
    return z.p.B;
}

cudaError_t launch_query_binned(const QueryArgs& a, int64_t band_bytes, void* ws, size_t ws_bytes, cudaStream_t s)
{
    BinLayout z;
    if (!binned_plan(a.L, a.Q, band_bytes, &z) || (int64_t)ws_bytes < z.bytes || !ws) return cudaErrorInvalidValue;
    if (a.Q == 0) return cudaSuccess;
    // bulk copies read device memory at 16-byte aligned addresses; other directions use plain loads
    cudaPointerAttributes at;
    z.p.bulk = 0;
    if (((uintptr_t)a.dirs & 15u) == 0 && cudaPointerGetAttributes(&at, a.dirs) == cudaSuccess &&
        at.type == cudaMemoryTypeDevice)
        z.p.bulk = 1;
    (void)cudaGetLastError();
    if (z.p.nT > 0x7fffffff) return cudaErrorInvalidConfiguration;
    unsigned char* w = static_cast<unsigned char*>(ws);
    float* sorted = reinterpret_cast<float*>(w + z.o_sorted);
    float* Rs = reinterpret_cast<float*>(w + z.o_R);
    float* cs = reinterpret_cast<float*>(w + z.o_chart);
    unsigned char* binb = w + z.o_bin;
    int32_t* cnt = reinterpret_cast<int32_t*>(w + z.o_cnt);
    long long* off = reinterpret_cast<long long*>(w + z.o_off);
    long long* tot = reinterpret_cast<long long*>(w + z.o_tot);
    const unsigned nT = (unsigned)z.p.nT;
    k_bin_count<<<nT, BB, 0, s>>>(z.p, a.dirs, binb, cnt);
    k_bin_scan<<<z.p.B, SCAN_T, 0, s>>>(z.p, cnt, off, tot);
    cudaError_t e = ensure_dynamic_smem((const void*)k_bin_scatter, SCATTER_DYN_SMEM);
    if (e == cudaSuccess) e = ensure_dynamic_smem((const void*)k_bin_finish, FINISH_DYN_SMEM);
    if (e != cudaSuccess) return e;
    k_bin_scatter<<<nT, BB, SCATTER_DYN_SMEM, s>>>(z.p, a.dirs, binb, off, tot, sorted, a.dev_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_bin_query_any(a.L, a.Q, sorted, Rs, reinterpret_cast<float2*>(cs), a.dev_status, s);
    if (e != cudaSuccess) return e;
    k_bin_finish<<<nT, BB, FINISH_DYN_SMEM, s>>>(z.p, a.dirs, binb, off, tot, Rs, reinterpret_cast<const float2*>(cs),
                                              a.R, a.grad, a.normal, a.chart, a.dev_status);
    return cudaGetLastError();
}

}  // namespace shm
