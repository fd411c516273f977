// Mutual nearest-neighbour matching of descriptors (reciprocity test,
// Sec. III-C), exact FP32 path on CUDA cores.
//
// Distances are sum_h (x_h - y_h)^2 over the 33 descriptor values, each term
// added with one fused multiply-add in h order.  A CTA owns a 128-row tile of
// the source descriptors and streams a chunk of 128-column target tiles
// through shared memory (double-buffered: the next tile is prefetched into
// registers while the current one is used); each thread keeps an 8x8 block of
// distances.  The arithmetic uses Blackwell's paired FP32 instructions on
// column pairs: d = x + (-y) (the target tile is stored negated, and
// x + (-y) == x - y exactly) and acc = fma(d, d, acc), two lanes per
// instruction, so every distance is bit-identical to the scalar chain.
// Per row the kernel keeps (best, its column, second best) with ties to the
// lower column; per column the best (distance, row) is folded into a packed
// 64-bit key with atomicMin, which orders by distance then by row.  Row
// partials of the column chunks are merged afterwards, then a pair (i, j) is
// kept iff j = NN_Q(i) and NN_P(j) = i, emitted in ascending i.
#include "kmx_internal.cuh"
#include "match_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 128;
constexpr int kDim = KMX_DESC_DIM;
constexpr int kStride = KMX_DESC_STRIDE;
constexpr int kVec = kStride / 4;                                // float4 per descriptor row
constexpr int kLoads = (kTile * kVec + kThreads - 1) / kThreads;  // float4 loads per thread per tile

struct FpShared {
    float P[kDim][kTile];          // source tile, transposed
    float Qn[2][kDim][kTile];      // negated target tiles, transposed, double-buffered
    unsigned long long colred[kThreads / 32][kTile];
};

// This thread's share of a 128-row tile (rows >= n read as zero).  With a
// row list, tile row r is descriptor row list[row0 + r].
__device__ __forceinline__ void fetch_tile(float4 (&reg)[kLoads], const float* __restrict__ desc,
                                           const int32_t* __restrict__ list, int64_t row0, int64_t n)
{
#pragma unroll
    for (int it = 0; it < kLoads; ++it) {
        const int idx = threadIdx.x + it * kThreads;
        reg[it] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < kTile * kVec) {
            const int r = idx / kVec, c4 = idx % kVec;
            if (row0 + r < n) {
                const int64_t src = list ? (int64_t)list[row0 + r] : row0 + r;
                reg[it] = __ldg(reinterpret_cast<const float4*>(desc + src * kStride) + c4);
            }
        }
    }
}

// Scatter the fetched share into smem[k][r] (k < 33), optionally negated.
__device__ __forceinline__ void store_tile(float (*sm)[kTile], const float4 (&reg)[kLoads], float sign)
{
#pragma unroll
    for (int it = 0; it < kLoads; ++it) {
        const int idx = threadIdx.x + it * kThreads;
        if (idx < kTile * kVec) {
            const int r = idx / kVec, k = (idx % kVec) * 4;
            sm[k][r] = sign * reg[it].x;
            if (k + 1 < kDim) sm[k + 1][r] = sign * reg[it].y;
            if (k + 2 < kDim) sm[k + 2][r] = sign * reg[it].z;
            if (k + 3 < kDim) sm[k + 3][r] = sign * reg[it].w;
        }
    }
}

// Column chunks per row tile of a whole-cloud call; the count used is decided
// on the device (kmx::work_chunks) and published in MatchScratch::chunks.
constexpr int kMaxChunksFp32 = 8;
// Column chunks per row tile of a row-list call (a few fallback rows spread
// over the whole GPU), bounded on the device by the room of the partial
// buffer: kMaxChunksFp32 * (list_cap + 1) entries.
constexpr int kMaxChunksRows = 512;

// The split of the actual work into (row tile, column chunk) blocks is
// computed here from the device-side counts, so a call sized for 121k rows
// that finds 12k descriptors still spreads them over the whole GPU; each CTA
// loops over blocks, so the grid may be smaller than the work (the row-list
// launch takes one CTA per SM).  With a row list the rows are list positions (np = list
// length), colbest may be null (no column bests), and the partials of chunk c
// are part[c * np ...] (packed by the actual list length, so that a short
// list can use many chunks).
__global__ void __launch_bounds__(kThreads) match_tiles_fp32(const float* __restrict__ dp,
                                                             const int32_t* __restrict__ rows_list, int64_t np_cap,
                                                             const int64_t* d_np, const float* __restrict__ dq,
                                                             int64_t nq_cap, const int64_t* d_nq, int target_ctas,
                                                             int max_chunks, kmx::RowBest* __restrict__ part,
                                                             unsigned long long* __restrict__ colbest,
                                                             int* __restrict__ chunks_out, int64_t rows_min)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FpShared& S = *reinterpret_cast<FpShared*>(smem_raw);
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    if (rows_list && np <= rows_min) return;  // a short list: rows_stream takes it
    const int64_t npt = (np + kTile - 1) / kTile;
    const int64_t nqt = (nq + kTile - 1) / kTile;
    const int64_t stride = rows_list ? np : np_cap;  // partials of one chunk
    int maxc = max_chunks;
    if (rows_list) {
        const int64_t room = (int64_t)kMaxChunksFp32 * (np_cap + 1) / (np > 0 ? np : 1);
        if (room < maxc) maxc = (int)room;
    }
    const int chunks = kmx::work_chunks(npt, nqt, target_ctas, maxc);
    if (blockIdx.x == 0 && threadIdx.x == 0) *chunks_out = chunks;
    // (row tile, chunk) blocks, blk = row tile * chunks + chunk; a CTA takes
    // blocks blockIdx.x, blockIdx.x + gridDim.x, ...
    for (int64_t blk = blockIdx.x; blk < npt * chunks; blk += gridDim.x) {
        const int chunk = (int)(blk % chunks);
        const int64_t row0 = (blk / chunks) * kTile;
        const int64_t tiles_per_chunk = (nqt + chunks - 1) / chunks;
        const int64_t qt0 = chunk * tiles_per_chunk;
        const int T = (int)max((int64_t)0, min(nqt, qt0 + tiles_per_chunk) - qt0);
        const int tx = threadIdx.x & 15;                                   // column group
        const int ty = (threadIdx.x >> 5) * 2 + ((threadIdx.x >> 4) & 1);  // row group
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

        float4 reg[kLoads];
        fetch_tile(reg, dp, rows_list, row0, np);
        store_tile(S.P, reg, 1.0f);
        if (T > 0) {
            fetch_tile(reg, dq, nullptr, qt0 * kTile, nq);
            store_tile(S.Qn[0], reg, -1.0f);
        }
        __syncthreads();

        float b1[8], b2[8];
        int j1[8];
    #pragma unroll
        for (int i = 0; i < 8; ++i) {
            b1[i] = INFINITY;
            b2[i] = INFINITY;
            j1[i] = 0x7fffffff;
        }
        for (int t = 0; t < T; ++t) {
            const int buf = t & 1;
            const int64_t col0 = (qt0 + t) * kTile;
            if (t + 1 < T) fetch_tile(reg, dq, nullptr, col0 + kTile, nq);  // in flight during the math
            float2 acc[8][4];
    #pragma unroll
            for (int i = 0; i < 8; ++i)
    #pragma unroll
                for (int jp = 0; jp < 4; ++jp) acc[i][jp] = make_float2(0.f, 0.f);
    #pragma unroll 3
            for (int k = 0; k < kDim; ++k) {
                const float4 a0 = *reinterpret_cast<const float4*>(&S.P[k][ty * 8]);
                const float4 a1 = *reinterpret_cast<const float4*>(&S.P[k][ty * 8 + 4]);
                const float4 c0 = *reinterpret_cast<const float4*>(&S.Qn[buf][k][tx * 8]);
                const float4 c1 = *reinterpret_cast<const float4*>(&S.Qn[buf][k][tx * 8 + 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float2 nc[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                                      make_float2(c1.z, c1.w)};
    #pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 ai = make_float2(a[i], a[i]);
    #pragma unroll
                    for (int jp = 0; jp < 4; ++jp) {
                        const float2 d = __fadd2_rn(ai, nc[jp]);
                        acc[i][jp] = __ffma2_rn(d, d, acc[i][jp]);
                    }
                }
            }
            // row bests (this thread's columns visited in ascending order)
    #pragma unroll
            for (int jp = 0; jp < 4; ++jp) {
    #pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t col = col0 + tx * 8 + 2 * jp + h;
                    if (col < nq) {
    #pragma unroll
                        for (int i = 0; i < 8; ++i)
                            kmx::row_update(b1[i], j1[i], b2[i], h ? acc[i][jp].y : acc[i][jp].x, (int)col);
                    }
                }
            }
            // column bests: this thread's 8 rows, then the partner half-warp, then
            // the 8 warps through shared memory, then one atomicMin per column
            if (colbest) {
    #pragma unroll
                for (int j = 0; j < 8; ++j) {
                    unsigned long long best = ~0ull;
    #pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int64_t row = row0 + ty * 8 + i;
                        if (row < np) {
                            const float dij = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
                            const unsigned long long key = kmx::pack_dist_index(dij, (uint32_t)row);
                            best = key < best ? key : best;
                        }
                    }
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, 16);
                    best = other < best ? other : best;
                    if (lane < 16) S.colred[warp][tx * 8 + j] = best;
                }
                __syncthreads();
                if (threadIdx.x < kTile) {
                    unsigned long long best = S.colred[0][threadIdx.x];
    #pragma unroll
                    for (int w = 1; w < kThreads / 32; ++w) {
                        const unsigned long long o = S.colred[w][threadIdx.x];
                        best = o < best ? o : best;
                    }
                    const int64_t col = col0 + threadIdx.x;
                    if (col < nq && best != ~0ull) atomicMin(&colbest[col], best);
                }
            }
            if (t + 1 < T) store_tile(S.Qn[buf ^ 1], reg, -1.0f);
            __syncthreads();
        }
        // merge the 16 column groups of each row (lanes sharing ty sit in one
        // half-warp: xor offsets 1..8)
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
            const int64_t row = row0 + ty * 8 + i;
            if (tx == 0 && row < np) part[(int64_t)chunk * stride + row] = kmx::RowBest{d1, jj, d2};
        }
        __syncthreads();  // shared tiles are rewritten by the next block
    }
}


// A short row list (at most kStreamRows rows; the tensor-core matcher's
// fallback usually lists a handful): one item per (list row, column chunk),
// each a CTA pass over the chunk's columns.  The arithmetic is the tiled
// kernel's (x - y, then one fused multiply-add per dimension in dimension
// order), so the summaries are the same bits; the partials go to
// part[c * n + r] as the tiled kernel leaves them.  The tiled kernel spends a
// whole 128-row tile on each of these rows.
constexpr int kStreamRows = 64;
constexpr int kStreamChunks = 128;
constexpr int kStreamThreads = 256;
static_assert(kDim == 33 && kStride == 36, "rows_stream unrolls 8 float4 and one scalar per row");

__global__ void __launch_bounds__(kStreamThreads) rows_stream(const float* __restrict__ dp,
                                                              const int32_t* __restrict__ rows, int64_t list_cap,
                                                              const int64_t* d_nlist, const float* __restrict__ dq,
                                                              int64_t nq_cap, const int64_t* d_nq, int64_t part_cap,
                                                              kmx::RowBest* __restrict__ part,
                                                              int* __restrict__ chunks_out)
{
    __shared__ kmx::RowBest red[kStreamThreads / 32];
    const int64_t n = kmx_count(d_nlist, list_cap);
    if (n > kStreamRows) return;  // the tiled kernel takes it
    const int64_t nq = kmx_count(d_nq, nq_cap);
    const int64_t room = part_cap / (n > 0 ? n : 1);
    const int chunks = (int)(room < kStreamChunks ? (room > 1 ? room : 1) : kStreamChunks);
    if (blockIdx.x == 0 && threadIdx.x == 0) *chunks_out = chunks;
    const int64_t per = (nq + chunks - 1) / chunks;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // uniform over the block: every thread reaches the barriers
    for (int64_t item = blockIdx.x; item < n * chunks; item += gridDim.x) {
        const int64_t r = item / chunks;
        const int c = (int)(item % chunks);
        const float* x = dp + (int64_t)rows[r] * kStride;
        float xr[kDim];
#pragma unroll
        for (int k = 0; k < kDim; ++k) xr[k] = __ldg(x + k);
        float b1 = INFINITY, b2 = INFINITY;
        int j1 = 0x7fffffff;
        const int64_t c0 = (int64_t)c * per;
        const int64_t c1 = c0 + per < nq ? c0 + per : nq;
        for (int64_t j = c0 + threadIdx.x; j < c1; j += kStreamThreads) {
            const float* y = dq + j * kStride;
            const float4* y4 = reinterpret_cast<const float4*>(y);
            float acc = 0.f;
#pragma unroll
            for (int q4 = 0; q4 < 8; ++q4) {
                const float4 v = __ldg(y4 + q4);
                float e = __fsub_rn(xr[4 * q4], v.x);
                acc = __fmaf_rn(e, e, acc);
                e = __fsub_rn(xr[4 * q4 + 1], v.y);
                acc = __fmaf_rn(e, e, acc);
                e = __fsub_rn(xr[4 * q4 + 2], v.z);
                acc = __fmaf_rn(e, e, acc);
                e = __fsub_rn(xr[4 * q4 + 3], v.w);
                acc = __fmaf_rn(e, e, acc);
            }
            const float e = __fsub_rn(xr[32], __ldg(y + 32));
            acc = __fmaf_rn(e, e, acc);
            kmx::row_update(b1, j1, b2, acc, (int)j);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float od1 = __shfl_xor_sync(0xffffffffu, b1, o);
            const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
            const float od2 = __shfl_xor_sync(0xffffffffu, b2, o);
            kmx::row_merge(b1, j1, b2, od1, oj, od2);
        }
        if (lane == 0) red[warp] = kmx::RowBest{b1, j1, b2};
        __syncthreads();
        if (threadIdx.x == 0) {
            kmx::RowBest b = red[0];
            for (int w = 1; w < kStreamThreads / 32; ++w)
                kmx::row_merge(b.d1, b.j1, b.d2, red[w].d1, red[w].j1, red[w].d2);
            part[(int64_t)c * n + r] = b;
        }
        __syncthreads();  // red is rewritten by the next item
    }
}

// Opt in to >48 KB of dynamic shared memory once per device (the first call
// happens before any capture of a pair into a CUDA graph).
cudaError_t set_smem_attr()
{
    return kmx_once_per_device(kmx_attr_fp32_tiles, [] {
        return cudaFuncSetAttribute(match_tiles_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(FpShared));
    });
}

}  // namespace

size_t kmx_match_fp32_scratch_bytes(int64_t np_cap, int64_t nq_cap, int* chunks)
{
    *chunks = kMaxChunksFp32;
    return kmx::match_common_bytes(np_cap, nq_cap, kMaxChunksFp32);
}

cudaError_t kmx_match_fp32_launch(kmx_ctx* ctx, const float* dp, int64_t np_cap, const int64_t* d_np,
                                  const float* dq, int64_t nq_cap, const int64_t* d_nq, kmx::MatchScratch& s,
                                  int max_chunks)
{
    cudaError_t e = set_smem_attr();
    if (e) return e;
    const int64_t npt = (np_cap + kTile - 1) / kTile;
    const int64_t blocks = (npt > 0 ? npt : 1) * max_chunks;
    KMX_COUNT_LAUNCH();
    match_tiles_fp32<<<(unsigned)blocks, kThreads, sizeof(FpShared), ctx->stream>>>(
        dp, nullptr, np_cap, d_np, dq, nq_cap, d_nq, 4 * ctx->sm_count, max_chunks, s.part, s.colbest, s.chunks, 0);
    return cudaGetLastError();
}

cudaError_t kmx_match_fp32_rows_launch(kmx_ctx* ctx, const float* dp, const int32_t* rows, int64_t list_cap,
                                       const int64_t* d_nlist, const float* dq, int64_t nq_cap, const int64_t* d_nq,
                                       kmx::RowBest* part, int* chunks_out)
{
    cudaError_t e = set_smem_attr();
    if (e) return e;
    // both kernels read the list length on the device; exactly one of them
    // works (and publishes the chunk count): rows_stream up to kStreamRows
    // rows, the tiled kernel above
    KMX_COUNT_LAUNCH();
    rows_stream<<<(unsigned)(2 * (ctx->sm_count > 0 ? ctx->sm_count : 1)), kStreamThreads, 0, ctx->stream>>>(
        dp, rows, list_cap, d_nlist, dq, nq_cap, d_nq, (int64_t)kMaxChunksFp32 * (list_cap + 1), part, chunks_out);
    // one CTA per SM (the kernel's registers allow one), looping over the
    // (row tile, chunk) blocks: the list is usually short, and then every
    // CTA of a grid sized for list_cap would only check the count and exit
    const int target = 4 * ctx->sm_count;
    const int64_t blocks = ctx->sm_count > 0 ? ctx->sm_count : 1;
    KMX_COUNT_LAUNCH();
    match_tiles_fp32<<<(unsigned)blocks, kThreads, sizeof(FpShared), ctx->stream>>>(
        dp, rows, list_cap, d_nlist, dq, nq_cap, d_nq, target, kMaxChunksRows, part, nullptr, chunks_out,
        kStreamRows);
    return cudaGetLastError();
}

int kmx_match_fp32_max_chunks() { return kMaxChunksFp32; }
