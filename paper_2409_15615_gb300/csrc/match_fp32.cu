// Mutual nearest-neighbour matching of descriptors (reciprocity test,
// Sec. III-C), exact FP32 path on CUDA cores, plus the parts shared with the
// tensor-core path (partial merge, mutual test, ordered emission).
//
// Distances are sum_h (x_h - y_h)^2 over the 33 descriptor values.  A CTA
// owns a 128-row tile of the source descriptors and streams a chunk of
// 128-column target tiles through shared memory; each thread keeps an 8x8
// block of distances.  Per row it keeps (best, its column, second best) with
// ties to the lower column; per column the best (distance, row) is folded
// into a packed 64-bit key with atomicMin, which orders by distance then by
// row.  Row partials of the column chunks are merged afterwards, then a pair
// (i, j) is kept iff j = NN_Q(i) and NN_P(j) = i, emitted in ascending i.
#include "kmx_internal.cuh"
#include "match_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 128;
constexpr int kDim = KMX_DESC_DIM;
constexpr int kStride = KMX_DESC_STRIDE;

// Load a 128-row tile transposed into smem[k][r] (k < 33); rows >= n are 0.
// With a row list, tile row r is descriptor row list[row0 + r].
__device__ __forceinline__ void load_tile_t(float (*sm)[kTile], const float* __restrict__ desc,
                                            const int32_t* __restrict__ list, int64_t row0, int64_t n)
{
    for (int idx = threadIdx.x; idx < kTile * (kStride / 4); idx += kThreads) {
        const int r = idx / (kStride / 4);
        const int c4 = idx % (kStride / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row0 + r < n) {
            const int64_t src = list ? (int64_t)list[row0 + r] : row0 + r;
            v = __ldg(reinterpret_cast<const float4*>(desc + src * kStride) + c4);
        }
        const int k = c4 * 4;
        sm[k][r] = v.x;
        if (k + 1 < kDim) sm[k + 1][r] = v.y;
        if (k + 2 < kDim) sm[k + 2][r] = v.z;
        if (k + 3 < kDim) sm[k + 3][r] = v.w;
    }
}

// The grid is sized from the capacities; the split of the actual work (row
// tiles x column chunks) is computed here from the device-side counts, so a
// call sized for 121k rows that finds 12k descriptors still spreads them over
// the whole GPU.  With a row list the rows are list positions (np = list
// length) and colbest may be null (no column bests).
__global__ void __launch_bounds__(kThreads) match_tiles_fp32(const float* __restrict__ dp,
                                                             const int32_t* __restrict__ rows_list, int64_t np_cap,
                                                             const int64_t* d_np, const float* __restrict__ dq,
                                                             int64_t nq_cap, const int64_t* d_nq, int target_ctas,
                                                             int max_chunks, kmx::RowBest* __restrict__ part,
                                                             unsigned long long* __restrict__ colbest,
                                                             int* __restrict__ chunks_out)
{
    __shared__ __align__(16) float Ps[kDim][kTile];
    __shared__ __align__(16) float Qs[kDim][kTile];
    __shared__ unsigned long long colred[kThreads / 32][kTile];
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    const int64_t npt = (np + kTile - 1) / kTile;
    const int64_t nqt = (nq + kTile - 1) / kTile;
    const int chunks = kmx::work_chunks(npt, nqt, target_ctas, max_chunks);
    if (blockIdx.x == 0 && threadIdx.x == 0) *chunks_out = chunks;
    if ((int64_t)blockIdx.x >= npt * chunks) return;
    const int chunk = (int)(blockIdx.x % chunks);
    const int64_t row0 = (int64_t)(blockIdx.x / chunks) * kTile;
    const int64_t tiles_per_chunk = (nqt + chunks - 1) / chunks;
    const int64_t qt0 = chunk * tiles_per_chunk;
    const int tx = threadIdx.x & 15;                              // column group
    const int ty = (threadIdx.x >> 5) * 2 + ((threadIdx.x >> 4) & 1);  // row group
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    load_tile_t(Ps, dp, rows_list, row0, np);
    float b1[8], b2[8];
    int j1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        b1[i] = INFINITY;
        b2[i] = INFINITY;
        j1[i] = 0x7fffffff;
    }
    for (int64_t qt = qt0; qt < qt0 + tiles_per_chunk && qt < nqt; ++qt) {
        const int64_t col0 = qt * kTile;
        __syncthreads();
        load_tile_t(Qs, dq, nullptr, col0, nq);
        __syncthreads();
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 3
        for (int k = 0; k < kDim; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Ps[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Ps[k][ty * 8 + 4]);
            const float4 c0 = *reinterpret_cast<const float4*>(&Qs[k][tx * 8]);
            const float4 c1 = *reinterpret_cast<const float4*>(&Qs[k][tx * 8 + 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float d = a[i] - c[j];
                    acc[i][j] = fmaf(d, d, acc[i][j]);
                }
        }
        // row bests (columns visited in ascending order)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t col = col0 + tx * 8 + j;
            if (col < nq) {
#pragma unroll
                for (int i = 0; i < 8; ++i) kmx::row_update(b1[i], j1[i], b2[i], acc[i][j], (int)col);
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
                        const unsigned long long key = kmx::pack_dist_index(acc[i][j], (uint32_t)row);
                        best = key < best ? key : best;
                    }
                }
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, 16);
                best = other < best ? other : best;
                if (lane < 16) colred[warp][tx * 8 + j] = best;
            }
            __syncthreads();
            if (threadIdx.x < kTile) {
                unsigned long long best = colred[0][threadIdx.x];
#pragma unroll
                for (int w = 1; w < kThreads / 32; ++w) {
                    const unsigned long long o = colred[w][threadIdx.x];
                    best = o < best ? o : best;
                }
                const int64_t col = col0 + threadIdx.x;
                if (col < nq && best != ~0ull) atomicMin(&colbest[col], best);
            }
        }
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
        if (tx == 0 && row < np) part[(int64_t)chunk * np_cap + row] = kmx::RowBest{d1, jj, d2};
    }
}

}  // namespace

// Up to this many column chunks per row tile; the count used is decided on
// the device (kmx::work_chunks) and published in MatchScratch::chunks.
constexpr int kMaxChunksFp32 = 8;

size_t kmx_match_fp32_scratch_bytes(int64_t np_cap, int64_t nq_cap, int* chunks)
{
    *chunks = kMaxChunksFp32;
    return kmx::match_common_bytes(np_cap, nq_cap, kMaxChunksFp32);
}

cudaError_t kmx_match_fp32_launch(kmx_ctx* ctx, const float* dp, int64_t np_cap, const int64_t* d_np,
                                  const float* dq, int64_t nq_cap, const int64_t* d_nq, kmx::MatchScratch& s,
                                  int max_chunks)
{
    const int64_t npt = (np_cap + kTile - 1) / kTile;
    const int64_t blocks = (npt > 0 ? npt : 1) * max_chunks;
    KMX_COUNT_LAUNCH();
    match_tiles_fp32<<<(unsigned)blocks, kThreads, 0, ctx->stream>>>(
        dp, nullptr, np_cap, d_np, dq, nq_cap, d_nq, 4 * ctx->sm_count, max_chunks, s.part, s.colbest, s.chunks);
    return cudaGetLastError();
}

cudaError_t kmx_match_fp32_rows_launch(kmx_ctx* ctx, const float* dp, const int32_t* rows, int64_t list_cap,
                                       const int64_t* d_nlist, const float* dq, int64_t nq_cap, const int64_t* d_nq,
                                       kmx::RowBest* part, int* chunks_out)
{
    const int64_t npt = (list_cap + kTile - 1) / kTile;
    const int64_t blocks = (npt > 0 ? npt : 1) * kMaxChunksFp32;
    KMX_COUNT_LAUNCH();
    match_tiles_fp32<<<(unsigned)blocks, kThreads, 0, ctx->stream>>>(dp, rows, list_cap, d_nlist, dq, nq_cap, d_nq,
                                                                     4 * ctx->sm_count, kMaxChunksFp32, part,
                                                                     nullptr, chunks_out);
    return cudaGetLastError();
}

int kmx_match_fp32_max_chunks() { return kMaxChunksFp32; }
