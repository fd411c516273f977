// Mutual nearest-neighbour matching (Sec. III-C) with BF16 tensor-core
// distances and exact FP32 re-ranking.
//
//   pack      FP32 descriptor rows -> two BF16 K-major tiles of 128 rows x 48
//             (33 values, zero padded): x = hi + lo, hi = bf16(x),
//             lo = bf16(x - hi).  Both are laid out exactly as the UMMA
//             shared-memory operand (8x16-byte core matrices, no swizzle), so
//             one tile is one contiguous 24 KB bulk copy; plus ||y||^2.  A
//             single BF16 product (2^-9 relative) cannot rank near-duplicate
//             descriptors (plane points), hi.hi + lo.hi + hi.lo (2^-16) can.
//   tc_topk   one CTA per (128-row tile, chunk of 128-column tiles): the row
//             tile stays in shared memory, column tiles stream through a
//             3-stage ring filled by cp.async.bulk (TMA engine, mbarrier
//             completion); a single thread issues tcgen05.mma (kind::f16,
//             M=128 N=128 K=16; three K steps x three products) into one of
//             two TMEM accumulators while the 4 warps read the other one with
//             tcgen05.ld and keep, per row, the 8 smallest ranking keys
//             ||y||^2 - 2 x.y (the row's ||x||^2 does not change the order).
//   rerank    one warp per row: exact FP32 sum_h (x_h - y_h)^2 over the
//             candidates of every chunk, lowest index on ties; rows of the
//             source side give (d1, NN, d2), rows of the target side give the
//             packed (distance, row) best that the reciprocity test reads.
// The column direction is the same kernel with the roles of the two clouds
// swapped.  Every wait on an mbarrier is bounded; on timeout the kernel
// records KMX_DERR_TIMEOUT, drains what it issued and frees its TMEM.
#include "kmx_internal.cuh"
#include "bulk_copy.cuh"
#include "match_common.cuh"

#include <cuda_bf16.h>

namespace {

using kmx::bulk_g2s;
using kmx::mbar_expect_tx;
using kmx::mbar_fence_init;
using kmx::mbar_init;
using kmx::mbar_wait;
using kmx::smem_u32;

constexpr int kTM = 128;                       // rows per tile (UMMA M)
constexpr int kTN = 128;                       // columns per tile (UMMA N)
constexpr int kK = 48;                         // 33 descriptor values padded to 3 x 16
constexpr int kHalfBytes = kTM * kK * 2;       // one BF16 operand tile: 12288
constexpr int kOperandBytes = 2 * kHalfBytes;  // high part, then low part
constexpr int kTileBytes = kOperandBytes + kTM * 4;  // operands + 128 squared norms
constexpr int kCoreStride = 128;               // LBO: next 8-element K chunk
constexpr int kGroupStride = 6 * 128;          // SBO: next 8-row group
constexpr int kStages = 3;                     // column-tile ring
constexpr int kTopK = 8;
constexpr int kMaxChunks = 4;                  // 4 x 8 candidates = one warp in rerank
constexpr int kThreads = 128;
constexpr int kTmemCols = 256;                 // two 128-column FP32 accumulators

struct __align__(8) Cand {
    float v;
    int idx;
};

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05; mbarrier and bulk copy in bulk_copy.cuh)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle, LBO/SBO in bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor for kind::f16: BF16 x BF16 -> FP32, K-major A and B.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// pack
// ---------------------------------------------------------------------------

// One thread per row of the padded matrix.  Rows are centred on the common
// mean of both clouds first (distances do not change; products get smaller).
// The largest squared norm of the side is folded into *maxnorm (float bits of
// a non-negative value order like the value).
__global__ void __launch_bounds__(256) pack_bf16(const float* __restrict__ desc, int64_t n_cap, const int64_t* d_n,
                                                 int64_t rows_pad, const float* __restrict__ mean,
                                                 uint8_t* __restrict__ out, unsigned int* __restrict__ maxnorm)
{
    const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (r >= rows_pad) return;
    const int64_t n = kmx_count(d_n, n_cap);
    float x[kK];
#pragma unroll
    for (int h = 0; h < kK; ++h) x[h] = 0.f;
    if (r < n) {
        const float4* row = reinterpret_cast<const float4*>(desc + r * KMX_DESC_STRIDE);
#pragma unroll
        for (int c = 0; c < KMX_DESC_STRIDE / 4; ++c) {
            const float4 v = __ldg(row + c);
            x[4 * c + 0] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
        }
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) x[h] -= __ldg(mean + h);
    }
    uint8_t* tile = out + (r / kTM) * (int64_t)kTileBytes;
    const int rin = (int)(r % kTM);
    float nrm = 0.f;
#pragma unroll
    for (int c = 0; c < kK / 8; ++c) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint32_t wh = 0, wl = 0;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int h = 8 * c + 2 * e + u;
                const float f = h < KMX_DESC_DIM ? x[h] : 0.f;
                // x = hi + lo with both in BF16: the three products
                // hi.hi + lo.hi + hi.lo recover x.y to ~2^-16 relative
                const __nv_bfloat16 bh = __float2bfloat16_rn(f);
                const __nv_bfloat16 bl = __float2bfloat16_rn(f - __bfloat162float(bh));
                nrm = fmaf(f, f, nrm);
                wh |= (uint32_t)__bfloat16_as_ushort(bh) << (16 * u);
                wl |= (uint32_t)__bfloat16_as_ushort(bl) << (16 * u);
            }
            hi[e] = wh;
            lo[e] = wl;
        }
        const int off = (rin / 8) * kGroupStride + c * kCoreStride + (rin % 8) * 16;
        *reinterpret_cast<uint4*>(tile + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(tile + kHalfBytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    reinterpret_cast<float*>(tile + kOperandBytes)[rin] = r < n ? nrm : INFINITY;
    if (r < n) atomicMax(maxnorm, __float_as_uint(nrm));
}

// ---------------------------------------------------------------------------
// tensor-core top-k
// ---------------------------------------------------------------------------

struct TcShared {
    uint8_t a[kOperandBytes];
    uint8_t b[kStages][kOperandBytes];
    float nrm[2][kTN];
    uint64_t bar_a, bar_b[kStages], bar_mma[2];
    uint32_t tmem;
    int failed;
};

__device__ __forceinline__ void topk_insert(float* tv, int* ti, float v, int j)
{
    tv[kTopK - 1] = v;
    ti[kTopK - 1] = j;
#pragma unroll
    for (int p = kTopK - 1; p > 0; --p) {
        if (tv[p] < tv[p - 1]) {
            const float fv = tv[p];
            tv[p] = tv[p - 1];
            tv[p - 1] = fv;
            const int fi = ti[p];
            ti[p] = ti[p - 1];
            ti[p - 1] = fi;
        }
    }
}

// The grid is sized from the capacities; the (row tile, column chunk) split
// of the actual counts is decided here (kmx::work_chunks) and published in
// *chunks_out for the re-ranking kernel.
__global__ void __launch_bounds__(kThreads, 1) tc_topk(const uint8_t* __restrict__ packA, int64_t rows_cap,
                                                      const int64_t* d_rows, const uint8_t* __restrict__ packB,
                                                      int64_t cols_cap, const int64_t* d_cols, int target_ctas,
                                                      Cand* __restrict__ part, int* __restrict__ chunks_out,
                                                      unsigned int* err)
{
    extern __shared__ uint8_t smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t rows = kmx_count(d_rows, rows_cap), cols = kmx_count(d_cols, cols_cap);
    const int64_t n_rt = (rows + kTM - 1) / kTM;
    const int64_t n_ct = (cols + kTN - 1) / kTN;
    const int chunks = kmx::work_chunks(n_rt, n_ct, target_ctas, kMaxChunks);
    if (blockIdx.x == 0 && tid == 0) *chunks_out = chunks;
    if ((int64_t)blockIdx.x >= n_rt * chunks) return;
    const int chunk = (int)(blockIdx.x % chunks);
    const int64_t row0 = (int64_t)(blockIdx.x / chunks) * kTM;
    const int64_t tiles_per_chunk = (n_ct + chunks - 1) / chunks;
    const int64_t t0 = chunk * tiles_per_chunk;
    const int T = (int)max((int64_t)0, min(n_ct, t0 + tiles_per_chunk) - t0);
    const uint32_t idesc = idesc_bf16(kTM, kTN);

    if (tid == 0) {
        mbar_init(&S.bar_a, 1);
        for (int s = 0; s < kStages; ++s) mbar_init(&S.bar_b[s], 1);
        mbar_init(&S.bar_mma[0], 1);
        mbar_init(&S.bar_mma[1], 1);
        mbar_fence_init();
        S.failed = 0;
    }
    if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;

    float tv[kTopK];
    int ti[kTopK];
#pragma unroll
    for (int k = 0; k < kTopK; ++k) {
        tv[k] = INFINITY;
        ti[k] = -1;
    }
    int issued_b = 0;  // column tiles whose copy thread 0 has issued
    if (tid == 0 && T > 0) {
        mbar_expect_tx(&S.bar_a, kOperandBytes);
        bulk_g2s(S.a, packA + (row0 / kTM) * (int64_t)kTileBytes, kOperandBytes, &S.bar_a);
        for (; issued_b < T && issued_b < kStages; ++issued_b) {
            mbar_expect_tx(&S.bar_b[issued_b], kOperandBytes);
            bulk_g2s(S.b[issued_b], packB + (t0 + issued_b) * (int64_t)kTileBytes, kOperandBytes,
                     &S.bar_b[issued_b]);
        }
    }
    const uint32_t a_base = smem_u32(S.a);
    // thread 0: tile t into accumulator t & 1 -- per K step of 16, the three
    // products hi.hi + lo.hi + hi.lo of the split operands
    auto issue = [&](int t) {
        const uint32_t b_base = smem_u32(S.b[t % kStages]);
        const uint32_t d = tmem + (uint32_t)((t & 1) * kTN);
#pragma unroll
        for (int k = 0; k < kK / 16; ++k) {
            const uint32_t ko = k * 2 * kCoreStride;
            const uint64_t ah = smem_desc(a_base + ko, kCoreStride, kGroupStride);
            const uint64_t al = smem_desc(a_base + kHalfBytes + ko, kCoreStride, kGroupStride);
            const uint64_t bh = smem_desc(b_base + ko, kCoreStride, kGroupStride);
            const uint64_t bl = smem_desc(b_base + kHalfBytes + ko, kCoreStride, kGroupStride);
            umma_bf16(d, ah, bh, idesc, k > 0);
            umma_bf16(d, al, bh, idesc, 1);
            umma_bf16(d, ah, bl, idesc, 1);
        }
        umma_commit(&S.bar_mma[t & 1]);
    };
    if (tid == 0 && T > 0) {
        bool ok = mbar_wait(&S.bar_a, 0) && mbar_wait(&S.bar_b[0], 0);
        if (ok) {
            tc_fence_after();
            issue(0);
        } else {
            S.failed = 1;
        }
    }
    __syncthreads();
    int issued_mma = (T > 0 && !S.failed) ? 1 : 0;
    for (int t = 0; t < T && !S.failed; ++t) {
        const int s = t & 1;
        // column norms of tile t (plain loads; visible after the barrier below)
        S.nrm[s][tid] = reinterpret_cast<const float*>(packB + (t0 + t) * (int64_t)kTileBytes + kOperandBytes)[tid];
        if (tid == 0 && t + 1 < T) {
            if (mbar_wait(&S.bar_b[(t + 1) % kStages], ((t + 1) / kStages) & 1)) {
                tc_fence_after();
                issue(t + 1);
                ++issued_mma;
            } else {
                S.failed = 1;
            }
        }
        if (!mbar_wait(&S.bar_mma[s], (t >> 1) & 1)) S.failed = 1;
        tc_fence_after();
        if (tid == 0 && t + kStages < T) {  // MMA t is done with its stage
            const int st = t % kStages;
            mbar_expect_tx(&S.bar_b[st], kOperandBytes);
            bulk_g2s(S.b[st], packB + (t0 + t + kStages) * (int64_t)kTileBytes, kOperandBytes, &S.bar_b[st]);
            ++issued_b;
        }
        __syncthreads();
        if (S.failed) break;
        const int64_t col0 = (t0 + t) * kTN;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * kTN);
        // Fast path: 32 keys and their minimum without a branch; only when
        // the minimum beats the current 8th key are the keys inserted one by
        // one (rare once the list has filled).
#pragma unroll 1
        for (int c0 = 0; c0 < kTN; c0 += 32) {
            float v[32];
            tmem_ld32(lane_addr + c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = fmaf(-2.0f, v[j], S.nrm[s][c0 + j]);
            float m[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) m[j] = fminf(v[j], v[j + 16]);
#pragma unroll
            for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
                for (int j = 0; j < w; ++j) m[j] = fminf(m[j], m[j + w]);
            if (m[0] < tv[kTopK - 1]) {
#pragma unroll 1
                for (int j = 0; j < 32; ++j) {
                    float vj = v[0];
#pragma unroll
                    for (int k = 1; k < 32; ++k) vj = (j == k) ? v[k] : vj;  // register select, no local memory
                    if (vj < tv[kTopK - 1]) topk_insert(tv, ti, vj, (int)(col0 + c0 + j));
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (S.failed) {
        // drain: every issued copy and MMA must land before the memory goes
        // away.  Each barrier has at most one phase outstanding (a stage is
        // re-armed only after its previous copy was consumed), so waiting for
        // the last phase issued on each barrier suffices.
        if (tid == 0) {
            kmx_raise(err, KMX_DERR_TIMEOUT);
            mbar_wait(&S.bar_a, 0);
            for (int st = 0; st < kStages; ++st) {
                const int last = issued_b - 1 - ((issued_b - 1 - st) % kStages + kStages) % kStages;
                if (last >= 0 && last % kStages == st) mbar_wait(&S.bar_b[st], (last / kStages) & 1);
            }
            for (int k = 0; k < 2; ++k) {
                const int last = issued_mma - 1 - ((issued_mma - 1 - k) % 2 + 2) % 2;
                if (last >= 0 && (last & 1) == k) mbar_wait(&S.bar_mma[k], (last >> 1) & 1);
            }
        }
        __syncthreads();
    } else {
        const int64_t row = row0 + tid;
        if (row < rows) {
            Cand* out = part + ((int64_t)chunk * rows_cap + row) * kTopK;
#pragma unroll
            for (int k = 0; k < kTopK; ++k) out[k] = Cand{tv[k], ti[k]};
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// common mean of both descriptor sets (deterministic: fixed partition, fixed
// summation order)
// ---------------------------------------------------------------------------

constexpr int kSumBlocks = 64;

// Block b sums, per descriptor value, rows [b*R, (b+1)*R) of P followed by Q.
__global__ void __launch_bounds__(64) col_partial(const float* __restrict__ P, int64_t np_cap, const int64_t* d_np,
                                                  const float* __restrict__ Q, int64_t nq_cap, const int64_t* d_nq,
                                                  double* __restrict__ partial)
{
    const int h = threadIdx.x;
    if (h >= KMX_DESC_DIM) return;
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap), n = np + nq;
    const int64_t R = (n + kSumBlocks - 1) / kSumBlocks;
    const int64_t lo = (int64_t)blockIdx.x * R, hi = min(n, lo + R);
    double s = 0.0;
    for (int64_t r = lo; r < hi; ++r) {
        const float v = r < np ? __ldg(P + r * KMX_DESC_STRIDE + h) : __ldg(Q + (r - np) * KMX_DESC_STRIDE + h);
        s += (double)v;
    }
    partial[blockIdx.x * KMX_DESC_DIM + h] = s;
}

__global__ void col_mean(const double* __restrict__ partial, int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                         const int64_t* d_nq, float* __restrict__ mean, unsigned int* __restrict__ maxnorm)
{
    const int h = threadIdx.x;
    const int64_t n = kmx_count(d_np, np_cap) + kmx_count(d_nq, nq_cap);
    if (h < KMX_DESC_DIM) {
        double s = 0.0;
        for (int b = 0; b < kSumBlocks; ++b) s += partial[b * KMX_DESC_DIM + h];
        mean[h] = n > 0 ? (float)(s / (double)n) : 0.f;
    } else if (h < KMX_DESC_STRIDE) {
        mean[h] = 0.f;
    }
    if (h < 2) maxnorm[h] = 0u;
}

// ---------------------------------------------------------------------------
// certified exact FP32 re-ranking
// ---------------------------------------------------------------------------

// Bound on |approximate key - exact key| for one row (keys ||y||^2 - 2 x.y of
// the centred descriptors): the split operands represent x, y to 2^-18
// relative per element and the FP32 accumulation of 144 products adds at
// most ~2^-16 of sum |x_h y_h|, so 2 * 2^-14 * |x| * max|y| covers the
// product term with margin; 2^-18 * max|y|^2 covers the FP32 norms and the
// final fused multiply-add.
__device__ __forceinline__ float key_error_bound(float x_norm2, float ymax_norm2)
{
    return 2.0f * (1.0f / 16384.0f) * sqrtf(x_norm2) * sqrtf(ymax_norm2) + (1.0f / 262144.0f) * ymax_norm2;
}

// One warp per row of X.  Lane c holds candidate c of the chunk lists
// (chunks x 8 <= 32).  With a(k) the k-th smallest approximate key over the
// candidates, a(8) - a(2) > 2E proves that the exact nearest and second-
// nearest columns are among the candidates (each key is within E of its
// exact value); the row is then re-ranked exactly: sum_h (x_h - y_h)^2 in
// FP32 with fmaf in h order, the arithmetic of the exact path, lowest index
// on ties.  Otherwise the row is flagged for the exact fallback.
__global__ void __launch_bounds__(256) rerank(const float* __restrict__ X, int64_t rows_cap, const int64_t* d_rows,
                                              const float* __restrict__ Y, const Cand* __restrict__ part,
                                              const int* __restrict__ d_chunks, const float* __restrict__ mean,
                                              const unsigned int* __restrict__ ymax_bits,
                                              kmx::RowBest* __restrict__ rows_out,
                                              unsigned long long* __restrict__ cols_best,
                                              int32_t* __restrict__ fallback, int* __restrict__ final_chunks)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (final_chunks && i == 0 && lane == 0) *final_chunks = 1;  // rows_out holds whole-row summaries
    if (i >= kmx_count(d_rows, rows_cap)) return;
    const int chunks = *d_chunks;
    int j = -1;
    float a = INFINITY;
    if (lane < chunks * kTopK) {
        const Cand c = part[((int64_t)(lane / kTopK) * rows_cap + i) * kTopK + lane % kTopK];
        j = c.idx;
        if (j >= 0) a = c.v;
    }
    // ranks of the approximate keys (ties by lane), a(2) and a(8)
    int rank = 0, valid = 0;
#pragma unroll
    for (int o = 0; o < 32; ++o) {
        const float ao = __shfl_sync(0xffffffffu, a, o);
        const int jo = __shfl_sync(0xffffffffu, j, o);
        valid += jo >= 0;
        rank += (jo >= 0) && (ao < a || (ao == a && o < lane));
    }
    const float a2 = __shfl_sync(0xffffffffu, a, __ffs(__ballot_sync(0xffffffffu, j >= 0 && rank == 1)) - 1 & 31);
    const float a8 = __shfl_sync(0xffffffffu, a, __ffs(__ballot_sync(0xffffffffu, j >= 0 && rank == 7)) - 1 & 31);
    const float* x = X + i * KMX_DESC_STRIDE;
    float xn2 = 0.f;
#pragma unroll
    for (int h = 0; h < KMX_DESC_DIM; ++h) {
        const float e = __ldg(x + h) - __ldg(mean + h);
        xn2 = fmaf(e, e, xn2);
    }
    const float E = key_error_bound(xn2, __uint_as_float(*ymax_bits));
    const bool certified = valid < kTopK || (a8 - a2 > 2.0f * E);
    if (!certified) {
        if (lane == 0) fallback[i] = 1;
        return;
    }
    float d = INFINITY;
    if (j >= 0) {
        const float* y = Y + (int64_t)j * KMX_DESC_STRIDE;
        float acc = 0.f;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) {
            const float e = __ldg(x + h) - __ldg(y + h);
            acc = fmaf(e, e, acc);
        }
        d = acc;
    }
    float b1 = d;
    int j1 = j >= 0 ? j : 0x7fffffff;
    float b2 = INFINITY;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const float od1 = __shfl_xor_sync(0xffffffffu, b1, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
        const float od2 = __shfl_xor_sync(0xffffffffu, b2, o);
        kmx::row_merge(b1, j1, b2, od1, oj, od2);
    }
    if (lane != 0) return;
    if (rows_out) rows_out[i] = kmx::RowBest{b1, j1, b2};
    if (cols_best && j1 != 0x7fffffff) cols_best[i] = kmx::pack_dist_index(b1, (uint32_t)j1);
}

// Compact the flagged rows into a list (ascending) and publish its length.
__global__ void __launch_bounds__(256) compact_flags(int64_t n_cap, const int64_t* d_n,
                                                     const int32_t* __restrict__ flags,
                                                     const int64_t* __restrict__ pos, int32_t* __restrict__ list,
                                                     int64_t* __restrict__ n_list)
{
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i == 0) *n_list = pos[n_cap];
    if (i >= kmx_count(d_n, n_cap)) return;
    if (flags[i]) list[pos[i]] = (int32_t)i;
}

// Merge the exact fallback partials of each listed row and store them where
// the certified rows went.
__global__ void __launch_bounds__(256) fallback_merge(const kmx::RowBest* __restrict__ part,
                                                      const int* __restrict__ d_chunks, int64_t list_cap,
                                                      const int32_t* __restrict__ list,
                                                      const int64_t* __restrict__ n_list,
                                                      kmx::RowBest* __restrict__ rows_out,
                                                      unsigned long long* __restrict__ cols_best)
{
    const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (r >= min(*n_list, list_cap)) return;
    kmx::RowBest b = part[r];
    const int chunks = *d_chunks;
    for (int c = 1; c < chunks; ++c) {
        const kmx::RowBest o = part[(int64_t)c * list_cap + r];
        kmx::row_merge(b.d1, b.j1, b.d2, o.d1, o.j1, o.d2);
    }
    const int i = list[r];
    if (rows_out) rows_out[i] = b;
    if (cols_best && b.j1 != 0x7fffffff) cols_best[i] = kmx::pack_dist_index(b.d1, (uint32_t)b.j1);
}

size_t tc_smem_bytes()
{
    // ~100 KB: two CTAs per SM, i.e. two 256-column TMEM allocations
    size_t need = sizeof(TcShared) + 1024;
    return need < 96 * 1024 ? 96 * 1024 : need;
}

struct TcBuffers {
    uint8_t *packP, *packQ;
    Cand *candP, *candQ;
    double* partial;
    float* mean;
    unsigned int* maxnorm;  // [0] = P side, [1] = Q side
    int* chunks;            // [0] candP, [1] candQ, [2] fallback P, [3] fallback Q
    int32_t *flagP, *flagQ, *listP, *listQ;
    int64_t *posP, *posQ, *nlist;  // nlist[0] P, [1] Q
    kmx::RowBest *fbP, *fbQ;
};

TcBuffers tc_carve(void* base, int64_t np_cap, int64_t nq_cap, size_t* total)
{
    TcBuffers b{};
    kmx_arena a{static_cast<char*>(base), 0};
    const int64_t tp = (np_cap + kTM - 1) / kTM, tq = (nq_cap + kTM - 1) / kTM;
    const int fc = kmx_match_fp32_max_chunks();
    b.packP = (uint8_t*)a.take((size_t)tp * kTileBytes);
    b.packQ = (uint8_t*)a.take((size_t)tq * kTileBytes);
    b.candP = (Cand*)a.take(sizeof(Cand) * kTopK * (size_t)kMaxChunks * (np_cap + 1));
    b.candQ = (Cand*)a.take(sizeof(Cand) * kTopK * (size_t)kMaxChunks * (nq_cap + 1));
    b.partial = (double*)a.take(sizeof(double) * kSumBlocks * KMX_DESC_DIM);
    b.mean = (float*)a.take(sizeof(float) * KMX_DESC_STRIDE);
    b.maxnorm = (unsigned int*)a.take(sizeof(unsigned int) * 2);
    b.chunks = (int*)a.take(sizeof(int) * 4);
    b.flagP = (int32_t*)a.take(sizeof(int32_t) * (np_cap + 1));
    b.flagQ = (int32_t*)a.take(sizeof(int32_t) * (nq_cap + 1));
    b.listP = (int32_t*)a.take(sizeof(int32_t) * (np_cap + 1));
    b.listQ = (int32_t*)a.take(sizeof(int32_t) * (nq_cap + 1));
    b.posP = (int64_t*)a.take(sizeof(int64_t) * (np_cap + 1));
    b.posQ = (int64_t*)a.take(sizeof(int64_t) * (nq_cap + 1));
    b.nlist = (int64_t*)a.take(sizeof(int64_t) * 2);
    b.fbP = (kmx::RowBest*)a.take(sizeof(kmx::RowBest) * (size_t)fc * (np_cap + 1));
    b.fbQ = (kmx::RowBest*)a.take(sizeof(kmx::RowBest) * (size_t)fc * (nq_cap + 1));
    *total = kmx_align_up(a.used, 256);
    return b;
}

}  // namespace

size_t kmx_match_tc_extra_bytes(int64_t np_cap, int64_t nq_cap, int)
{
    size_t total = 0;
    tc_carve(nullptr, np_cap, nq_cap, &total);
    return total;
}

cudaError_t kmx_match_tc_launch(kmx_ctx* ctx, const float* dp, int64_t np_cap, const int64_t* d_np, const float* dq,
                                int64_t nq_cap, const int64_t* d_nq, kmx::MatchScratch& s)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    TcBuffers b = tc_carve(s.extra, np_cap, nq_cap, &total);
    const int64_t tp = (np_cap + kTM - 1) / kTM, tq = (nq_cap + kTM - 1) / kTM;
    const size_t smem = tc_smem_bytes();
    cudaError_t e = kmx_once_per_device(kmx_attr_tc_topk, [smem] {
        return cudaFuncSetAttribute(tc_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e) return e;
    if ((e = cudaMemsetAsync(b.flagP, 0, sizeof(int32_t) * (np_cap + 1), st))) return e;
    if ((e = cudaMemsetAsync(b.flagQ, 0, sizeof(int32_t) * (nq_cap + 1), st))) return e;
    const int target = 2 * ctx->sm_count;
    // common mean, then split-BF16 packs of the centred rows
    KMX_COUNT_LAUNCH();
    col_partial<<<kSumBlocks, 64, 0, st>>>(dp, np_cap, d_np, dq, nq_cap, d_nq, b.partial);
    KMX_COUNT_LAUNCH();
    col_mean<<<1, 64, 0, st>>>(b.partial, np_cap, d_np, nq_cap, d_nq, b.mean, b.maxnorm);
    KMX_COUNT_LAUNCH();
    pack_bf16<<<kmx_blocks(tp * kTM, 256), 256, 0, st>>>(dp, np_cap, d_np, tp * kTM, b.mean, b.packP, b.maxnorm);
    KMX_COUNT_LAUNCH();
    pack_bf16<<<kmx_blocks(tq * kTM, 256), 256, 0, st>>>(dq, nq_cap, d_nq, tq * kTM, b.mean, b.packQ,
                                                        b.maxnorm + 1);
    // candidates both ways
    KMX_COUNT_LAUNCH();
    tc_topk<<<(unsigned)(tp * kMaxChunks), kThreads, smem, st>>>(b.packP, np_cap, d_np, b.packQ, nq_cap, d_nq, target,
                                                                 b.candP, b.chunks + 0, ctx->d_err);
    KMX_COUNT_LAUNCH();
    tc_topk<<<(unsigned)(tq * kMaxChunks), kThreads, smem, st>>>(b.packQ, nq_cap, d_nq, b.packP, np_cap, d_np, target,
                                                                 b.candQ, b.chunks + 1, ctx->d_err);
    // certified exact re-ranking; uncertified rows are flagged
    KMX_COUNT_LAUNCH();
    rerank<<<kmx_blocks(np_cap, 8), 256, 0, st>>>(dp, np_cap, d_np, dq, b.candP, b.chunks + 0, b.mean, b.maxnorm + 1,
                                                  s.part, nullptr, b.flagP, s.chunks);
    KMX_COUNT_LAUNCH();
    rerank<<<kmx_blocks(nq_cap, 8), 256, 0, st>>>(dq, nq_cap, d_nq, dp, b.candQ, b.chunks + 1, b.mean, b.maxnorm,
                                                  nullptr, s.colbest, b.flagQ, nullptr);
    // exact fallback for the flagged rows of each side
    if ((e = kmx_scan_i32(ctx, b.flagP, np_cap, d_np, b.posP))) return e;
    KMX_COUNT_LAUNCH();
    compact_flags<<<kmx_blocks(np_cap, 256), 256, 0, st>>>(np_cap, d_np, b.flagP, b.posP, b.listP, b.nlist + 0);
    if ((e = kmx_scan_i32(ctx, b.flagQ, nq_cap, d_nq, b.posQ))) return e;
    KMX_COUNT_LAUNCH();
    compact_flags<<<kmx_blocks(nq_cap, 256), 256, 0, st>>>(nq_cap, d_nq, b.flagQ, b.posQ, b.listQ, b.nlist + 1);
    if ((e = kmx_match_fp32_rows_launch(ctx, dp, b.listP, np_cap, b.nlist + 0, dq, nq_cap, d_nq, b.fbP,
                                        b.chunks + 2)))
        return e;
    if ((e = kmx_match_fp32_rows_launch(ctx, dq, b.listQ, nq_cap, b.nlist + 1, dp, np_cap, d_np, b.fbQ,
                                        b.chunks + 3)))
        return e;
    KMX_COUNT_LAUNCH();
    fallback_merge<<<kmx_blocks(np_cap, 256), 256, 0, st>>>(b.fbP, b.chunks + 2, np_cap, b.listP, b.nlist + 0, s.part,
                                                            nullptr);
    KMX_COUNT_LAUNCH();
    fallback_merge<<<kmx_blocks(nq_cap, 256), 256, 0, st>>>(b.fbQ, b.chunks + 3, nq_cap, b.listQ, b.nlist + 1,
                                                            nullptr, s.colbest);
    return cudaGetLastError();
}

// Rows that needed the exact fallback in the last BF16 match on this scratch
// (diagnostics): copies nlist[0..1] to the caller's device buffer.
cudaError_t kmx_match_tc_fallback_counts(kmx_ctx* ctx, const kmx::MatchScratch& s, int64_t np_cap, int64_t nq_cap,
                                         int64_t* dst)
{
    size_t total = 0;
    TcBuffers b = tc_carve(s.extra, np_cap, nq_cap, &total);
    return cudaMemcpyAsync(dst, b.nlist, 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx->stream);
}
