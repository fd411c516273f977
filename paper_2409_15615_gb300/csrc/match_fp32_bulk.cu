// Mutual nearest-neighbour matching of descriptors (reciprocity test,
// Sec. III-C), exact FP32 path of kmx_match: the tiled matcher with its
// operands staged by bulk copies.
//
// Every distance is sum_h (x_h - y_h)^2 over the 33 descriptor values, each
// term added with one fused multiply-add in h order, exactly the arithmetic of
// match_fp32.cu (so both give identical bits):
//
//   pack_tiles        descriptor rows -> 128-row tiles stored transposed
//                     ([33][128]); source values as (x, x) pairs, so a pair
//                     loads straight into a paired FP32 instruction, target
//                     values negated (x + (-y) == x - y exactly).  Rows past
//                     the count are zero and ignored later.
//   match_tiles_fp32_bulk
//                     the (row tile x column tile) grid, flattened row-major,
//                     is split into equal contiguous ranges, one per CTA, with
//                     as many CTAs as fit on the GPU at once (every CTA gets
//                     the same number of tiles, +-1).  The source tile stays
//                     in shared memory; target tiles stream through a 3-stage
//                     ring filled by cp.async.bulk (one contiguous 16.5 KB
//                     copy per tile, mbarrier completion), so no register
//                     holds a prefetched tile.  Each thread keeps an 8 x 8
//                     block of distances (paired instructions on column
//                     pairs).  Per row: (best, its column, second best), ties
//                     to the lower column; per column: the best (distance,
//                     row) packed into 64 bits and folded with atomicMin.
//                     When a CTA leaves a row tile (or its range ends) it
//                     writes the rows' summaries as one "segment".
//   merge_segments    per source row, the segments of its row tile in column
//                     order, then the reciprocity test.
//
// Every mbarrier wait is bounded; on timeout the kernel records
// KMX_DERR_TIMEOUT, waits (bounded) for the copies it issued and returns.
#include "bulk_copy.cuh"
#include "kmx_internal.cuh"
#include "match_common.cuh"

namespace {

using kmx::bulk_g2s;
using kmx::mbar_expect_tx;
using kmx::mbar_fence_init;
using kmx::mbar_init;
using kmx::mbar_wait;

constexpr int kThreads = 256;
constexpr int kTile = 128;
constexpr int kDim = KMX_DESC_DIM;
constexpr int kStride = KMX_DESC_STRIDE;
constexpr int kStages = 3;
constexpr uint32_t kPBytes = kDim * kTile * sizeof(float2);  // 33792
constexpr uint32_t kQBytes = kDim * kTile * sizeof(float);   // 16896
constexpr int kCtasPerSm = 2;

struct __align__(16) BulkShared {
    float2 P[kDim][kTile];                              // source tile, (x, x) pairs
    float Q[kStages][kDim][kTile];                      // negated target tiles
    unsigned long long colred[kThreads / 32][kTile];    // per-warp column bests
    uint64_t bar_p;
    uint64_t bar_q[kStages];
    int failed;
};
static_assert(kPBytes % 16 == 0 && kQBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
static_assert(offsetof(BulkShared, Q) % 16 == 0, "bulk copy destinations are 16-byte aligned");

// One thread per row of the padded matrix (rows up to the count rounded up to
// a whole tile).
template <bool kPairs>
__global__ void __launch_bounds__(256) pack_tiles(const float* __restrict__ desc, int64_t n_cap,
                                                  const int64_t* d_n, void* __restrict__ out)
{
    const int64_t n = kmx_count(d_n, n_cap);
    const int64_t n_pad = (n + kTile - 1) / kTile * kTile;
    const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (r >= n_pad) return;
    float v[kStride];
    if (r < n) {
        const float4* row = reinterpret_cast<const float4*>(desc + r * kStride);
#pragma unroll
        for (int c = 0; c < kStride / 4; ++c) {
            const float4 x = __ldg(row + c);
            v[4 * c] = x.x;
            v[4 * c + 1] = x.y;
            v[4 * c + 2] = x.z;
            v[4 * c + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kStride; ++k) v[k] = 0.f;
    }
    const int64_t base = (r / kTile) * kDim * kTile + (r % kTile);
    if (kPairs) {
        float2* o = static_cast<float2*>(out) + base;
#pragma unroll
        for (int k = 0; k < kDim; ++k) o[k * kTile] = make_float2(v[k], v[k]);
    } else {
        float* o = static_cast<float*>(out) + base;
#pragma unroll
        for (int k = 0; k < kDim; ++k) o[k * kTile] = -v[k];
    }
}

__device__ __forceinline__ void row_step(float& b1, int& j1, float& b2, float d, int j)
{
    // columns arrive in ascending order, so an equal distance keeps the
    // earlier (lower) column; NaN compares false and is ignored
    const bool lt1 = d < b1, lt2 = d < b2;
    b2 = lt1 ? b1 : (lt2 ? d : b2);
    j1 = lt1 ? j : j1;
    b1 = lt1 ? d : b1;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    match_tiles_fp32_bulk(const float2* __restrict__ pp, int64_t np_cap, const int64_t* d_np,
                          const float* __restrict__ qn, int64_t nq_cap, const int64_t* d_nq, int ctas,
                          kmx::RowBest* __restrict__ seg, unsigned long long* __restrict__ colbest,
                          unsigned int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BulkShared& S = *reinterpret_cast<BulkShared*>(smem_raw);
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    const int64_t npt = (np + kTile - 1) / kTile;
    const int64_t nqt = (nq + kTile - 1) / kTile;
    const int64_t W = npt * nqt;
    const int64_t G = min((int64_t)ctas, W);
    const int64_t b = blockIdx.x;
    if (b >= G) return;
    const int64_t w0 = b * W / G;
    const int T = (int)((b + 1) * W / G - w0);  // >= 1 because G <= W
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid & 15;                     // column group: columns 4tx..4tx+3 and 64+4tx..64+4tx+3
    const int ty = warp * 2 + ((tid >> 4) & 1);  // row group: rows 8ty..8ty+7

    if (tid == 0) {
        mbar_init(&S.bar_p, 1);
        for (int s = 0; s < kStages; ++s) mbar_init(&S.bar_q[s], 1);
        mbar_fence_init();
        S.failed = 0;
    }
    __syncthreads();
    int64_t rt = w0 / nqt;
    if (tid == 0) {
        mbar_expect_tx(&S.bar_p, kPBytes);
        bulk_g2s(S.P, pp + rt * kDim * kTile, kPBytes, &S.bar_p);
        for (int s = 0; s < kStages && s < T; ++s) {
            mbar_expect_tx(&S.bar_q[s], kQBytes);
            bulk_g2s(S.Q[s], qn + ((w0 + s) % nqt) * kDim * kTile, kQBytes, &S.bar_q[s]);
        }
    }
    int issued = min(T, kStages);  // column tiles whose copy has been issued
    uint32_t p_phase = 0;
    bool p_ready = false;

    float b1[8], b2[8];
    int j1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        b1[i] = INFINITY;
        b2[i] = INFINITY;
        j1[i] = 0x7fffffff;
    }
    bool failed = false;
    int t = 0;
    for (; t < T; ++t) {
        const int64_t w = w0 + t;
        const int64_t col0 = (w % nqt) * kTile;
        const int s = t % kStages;
        if (!p_ready) {
            if (!mbar_wait(&S.bar_p, p_phase)) S.failed = 1;
            p_ready = true;
        }
        if (!mbar_wait(&S.bar_q[s], (uint32_t)(t / kStages) & 1u)) S.failed = 1;

        float2 acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int jp = 0; jp < 4; ++jp) acc[i][jp] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int k = 0; k < kDim; ++k) {
            const float4 c0 = *reinterpret_cast<const float4*>(&S.Q[s][k][tx * 4]);
            const float4 c1 = *reinterpret_cast<const float4*>(&S.Q[s][k][64 + tx * 4]);
            const float2 nc[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                                  make_float2(c1.z, c1.w)};
#pragma unroll
            for (int ih = 0; ih < 4; ++ih) {
                const float4 a2 = *reinterpret_cast<const float4*>(&S.P[k][ty * 8 + 2 * ih]);
                const float2 ai[2] = {make_float2(a2.x, a2.y), make_float2(a2.z, a2.w)};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int jp = 0; jp < 4; ++jp) {
                        const float2 d = __fadd2_rn(ai[h], nc[jp]);
                        acc[2 * ih + h][jp] = __ffma2_rn(d, d, acc[2 * ih + h][jp]);
                    }
                }
            }
        }
        // row bests, this thread's columns in ascending order
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = (jp < 2 ? 0 : 64) + tx * 4 + 2 * (jp & 1) + h;
                const int64_t col = col0 + c;
                if (col < nq) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) row_step(b1[i], j1[i], b2[i], h ? acc[i][jp].y : acc[i][jp].x, (int)col);
                }
            }
        }
        // column bests: this thread's 8 rows (ascending, ties to the lower
        // row), the partner half-warp, then the 8 warps through shared memory
        const int64_t rowbase = rt * kTile + ty * 8;
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float m = INFINITY;
                int mi = -1;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float dij = h ? acc[i][jp].y : acc[i][jp].x;
                    const bool take = rowbase + i < np && (mi < 0 || dij < m);
                    m = take ? dij : m;
                    mi = take ? i : mi;
                }
                unsigned long long best = mi < 0 ? ~0ull : kmx::pack_dist_index(m, (uint32_t)(rowbase + mi));
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, 16);
                best = other < best ? other : best;
                const int c = (jp < 2 ? 0 : 64) + tx * 4 + 2 * (jp & 1) + h;
                if (lane < 16) S.colred[warp][c] = best;
            }
        }
        __syncthreads();  // (1) all waits of this tile are behind every thread
        failed = S.failed != 0;  // uniform: S.failed is written only before (1)
        if (!failed && tid < kTile) {
            unsigned long long best = S.colred[0][tid];
#pragma unroll
            for (int v = 1; v < kThreads / 32; ++v) {
                const unsigned long long o = S.colred[v][tid];
                best = o < best ? o : best;
            }
            const int64_t col = col0 + tid;
            if (col < nq && best != ~0ull) atomicMin(&colbest[col], best);
        }
        const bool seg_end = (t + 1 == T) || ((w + 1) % nqt == 0);
        if (seg_end && !failed) {
            // merge the 16 column groups of each row (one half-warp), write
            // the segment, restart the row bests
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float d1 = b1[i], d2 = b2[i];
                int jj = j1[i];
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    const float od1 = __shfl_xor_sync(0xffffffffu, d1, o);
                    const float od2 = __shfl_xor_sync(0xffffffffu, d2, o);
                    const int oj = __shfl_xor_sync(0xffffffffu, jj, o);
                    kmx::row_merge(d1, jj, d2, od1, oj, od2);
                }
                if (tx == 0 && rowbase + i < np)
                    seg[(b + rt) * kTile + ty * 8 + i] = kmx::RowBest{d1, jj, d2};
                b1[i] = INFINITY;
                b2[i] = INFINITY;
                j1[i] = 0x7fffffff;
            }
        }
        __syncthreads();  // (2) stage s, the source tile and colred are free
        if (failed) break;
        if (tid == 0 && t + kStages < T) {
            mbar_expect_tx(&S.bar_q[s], kQBytes);
            bulk_g2s(S.Q[s], qn + ((w0 + t + kStages) % nqt) * kDim * kTile, kQBytes, &S.bar_q[s]);
        }
        issued = min(T, t + 1 + kStages);
        if (seg_end && t + 1 < T) {
            ++rt;
            if (tid == 0) {
                mbar_expect_tx(&S.bar_p, kPBytes);
                bulk_g2s(S.P, pp + rt * kDim * kTile, kPBytes, &S.bar_p);
            }
            p_phase ^= 1u;
            p_ready = false;
        }
    }
    if (failed && tid == 0) {
        // every barrier has at most one phase outstanding: wait for the
        // source tile's and for each issued column tile not yet consumed
        kmx_raise(err, KMX_DERR_TIMEOUT);
        mbar_wait(&S.bar_p, p_phase);
        for (int u = t; u < issued; ++u) mbar_wait(&S.bar_q[u % kStages], (uint32_t)(u / kStages) & 1u);
    }
}

// One thread per source row: the segments of its row tile, in column order,
// then the reciprocity test against the packed column bests.
__global__ void __launch_bounds__(256) merge_segments(const kmx::RowBest* __restrict__ seg, int ctas,
                                                      int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                                                      const int64_t* d_nq,
                                                      const unsigned long long* __restrict__ colbest,
                                                      kmx::RowBest* __restrict__ merged, int32_t* __restrict__ mflag)
{
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    if (i >= np) return;
    const int64_t npt = (np + kTile - 1) / kTile;
    const int64_t nqt = (nq + kTile - 1) / kTile;
    const int64_t W = npt * nqt;
    kmx::RowBest r{INFINITY, 0x7fffffff, INFINITY};
    if (W > 0) {
        const int64_t G = min((int64_t)ctas, W);
        const int64_t rt = i / kTile;
        // the CTA whose range holds flattened tile x is floor(((x + 1) G - 1) / W)
        const int64_t x0 = rt * nqt, x1 = x0 + nqt - 1;
        const int64_t bf = ((x0 + 1) * G - 1) / W, bl = ((x1 + 1) * G - 1) / W;
        r = seg[(bf + rt) * kTile + (i % kTile)];
        for (int64_t bb = bf + 1; bb <= bl; ++bb) {
            const kmx::RowBest o = seg[(bb + rt) * kTile + (i % kTile)];
            kmx::row_merge(r.d1, r.j1, r.d2, o.d1, o.j1, o.d2);
        }
    }
    merged[i] = r;
    bool mutual = false;
    if (r.j1 >= 0 && r.j1 != 0x7fffffff) mutual = (uint32_t)(colbest[r.j1] & 0xffffffffull) == (uint32_t)i;
    mflag[i] = mutual ? 1 : 0;
}

int64_t tiles_of(int64_t n) { return (n + kTile - 1) / kTile; }

struct BulkScratch {
    float2* pp;
    float* qn;
    kmx::RowBest* seg;
};

BulkScratch carve(void* base, int64_t np_cap, int64_t nq_cap, int max_ctas, size_t* total)
{
    kmx_arena a{static_cast<char*>(base), 0};
    BulkScratch s;
    s.pp = static_cast<float2*>(a.take((size_t)tiles_of(np_cap) * kPBytes));
    s.qn = static_cast<float*>(a.take((size_t)tiles_of(nq_cap) * kQBytes));
    s.seg = static_cast<kmx::RowBest*>(a.take(sizeof(kmx::RowBest) * kTile * (size_t)(max_ctas + tiles_of(np_cap))));
    *total = kmx_align_up(a.used, 256);
    return s;
}

int max_ctas(int sm_count) { return kCtasPerSm * sm_count; }

cudaError_t set_smem_attr()
{
    return kmx_once_per_device(kmx_attr_fp32_bulk, [] {
        return cudaFuncSetAttribute(match_tiles_fp32_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(BulkShared));
    });
}

}  // namespace

size_t kmx_match_fp32_bulk_extra_bytes(int64_t np_cap, int64_t nq_cap, int sm_count)
{
    size_t total = 0;
    carve(nullptr, np_cap, nq_cap, max_ctas(sm_count), &total);
    return total;
}

cudaError_t kmx_match_fp32_bulk_launch(kmx_ctx* ctx, const float* dp, const int32_t* vp, int64_t np_cap,
                                       const int64_t* d_np, const float* dq, const int32_t* vq, int64_t nq_cap,
                                       const int64_t* d_nq, kmx::MatchScratch& s, kmx_corr* out, int64_t cap,
                                       int64_t* n_out)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    const BulkScratch b = carve(s.extra, np_cap, nq_cap, max_ctas(ctx->sm_count), &total);
    cudaError_t e = set_smem_attr();
    if (e) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, match_tiles_fp32_bulk, kThreads,
                                                           sizeof(BulkShared))))
        return e;
    const int ctas = max(1, min(per_sm, kCtasPerSm)) * ctx->sm_count;
    KMX_COUNT_LAUNCH();
    pack_tiles<true><<<kmx_blocks(tiles_of(np_cap) * kTile, 256), 256, 0, st>>>(dp, np_cap, d_np, b.pp);
    KMX_COUNT_LAUNCH();
    pack_tiles<false><<<kmx_blocks(tiles_of(nq_cap) * kTile, 256), 256, 0, st>>>(dq, nq_cap, d_nq, b.qn);
    if ((e = cudaMemsetAsync(s.colbest, 0xFF, sizeof(unsigned long long) * nq_cap, st))) return e;
    KMX_COUNT_LAUNCH();
    match_tiles_fp32_bulk<<<ctas, kThreads, sizeof(BulkShared), st>>>(b.pp, np_cap, d_np, b.qn, nq_cap, d_nq, ctas,
                                                                      b.seg, s.colbest, ctx->d_err);
    if ((e = cudaMemsetAsync(s.mflag, 0, sizeof(int32_t) * (np_cap + 1), st))) return e;
    KMX_COUNT_LAUNCH();
    merge_segments<<<kmx_blocks(np_cap, 256), 256, 0, st>>>(b.seg, ctas, np_cap, d_np, nq_cap, d_nq, s.colbest,
                                                            s.merged, s.mflag);
    if ((e = cudaGetLastError())) return e;
    return kmx::match_emit(ctx, s, np_cap, d_np, vp, vq, out, cap, n_out);
}
