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
#include "match_common.cuh"

#include <cuda_bf16.h>

namespace {

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
constexpr uint32_t kWaitLimit = 1u << 22;

struct __align__(8) Cand {
    float v;
    int idx;
};

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05, mbarrier, bulk copy)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

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

// One thread per row of the padded matrix.
__global__ void __launch_bounds__(256) pack_bf16(const float* __restrict__ desc, int64_t n_cap, const int64_t* d_n,
                                                 int64_t rows_pad, uint8_t* __restrict__ out)
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

__global__ void __launch_bounds__(kThreads, 1) tc_topk(const uint8_t* __restrict__ packA, int64_t rows_cap,
                                                      const int64_t* d_rows, const uint8_t* __restrict__ packB,
                                                      int64_t cols_cap, const int64_t* d_cols, int tiles_per_chunk,
                                                      Cand* __restrict__ part, unsigned int* err)
{
    extern __shared__ uint8_t smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t rows = kmx_count(d_rows, rows_cap), cols = kmx_count(d_cols, cols_cap);
    const int64_t row0 = (int64_t)blockIdx.x * kTM;
    if (row0 >= rows) return;
    const int64_t n_ct = (cols + kTN - 1) / kTN;
    const int64_t t0 = (int64_t)blockIdx.y * tiles_per_chunk;
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
#pragma unroll 1
        for (int c0 = 0; c0 < kTN; c0 += 32) {
            float acc[32];
            tmem_ld32(lane_addr + c0, acc);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float v = fmaf(-2.0f, acc[j], S.nrm[s][c0 + j]);
                if (v < tv[kTopK - 1]) topk_insert(tv, ti, v, (int)(col0 + c0 + j));
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
            Cand* out = part + ((int64_t)blockIdx.y * rows_cap + row) * kTopK;
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
// exact FP32 re-ranking
// ---------------------------------------------------------------------------

// One warp per row of X: lane c holds candidate c of the chunk lists, its
// exact FP32 distance is sum_h (x_h - y_h)^2 accumulated with fmaf in h order
// (the same arithmetic as the exact path).  Writes either the row summary
// (d1, NN, d2) or the packed (distance, row) best of the column side.
__global__ void __launch_bounds__(256) rerank(const float* __restrict__ X, int64_t rows_cap, const int64_t* d_rows,
                                              const float* __restrict__ Y, const Cand* __restrict__ part,
                                              int chunks, kmx::RowBest* __restrict__ rows_out,
                                              unsigned long long* __restrict__ cols_best)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= kmx_count(d_rows, rows_cap)) return;
    int j = -1;
    if (lane < chunks * kTopK) j = part[((int64_t)(lane / kTopK) * rows_cap + i) * kTopK + lane % kTopK].idx;
    float d = INFINITY;
    if (j >= 0) {
        const float* x = X + i * KMX_DESC_STRIDE;
        const float* y = Y + (int64_t)j * KMX_DESC_STRIDE;
        float acc = 0.f;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) {
            const float e = __ldg(x + h) - __ldg(y + h);
            acc = fmaf(e, e, acc);
        }
        d = acc;
    }
    // lexicographic (d, j) minimum over the warp, and the second-smallest d
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

int chunks_for(int64_t row_tiles, int64_t col_tiles, int sm_count)
{
    int64_t c = (2 * (int64_t)sm_count + row_tiles - 1) / (row_tiles > 0 ? row_tiles : 1);
    if (c < 1) c = 1;
    if (c > kMaxChunks) c = kMaxChunks;
    if (c > col_tiles) c = col_tiles > 0 ? col_tiles : 1;
    return (int)c;
}

size_t tc_smem_bytes()
{
    // ~100 KB: two CTAs per SM, i.e. two 256-column TMEM allocations
    size_t need = sizeof(TcShared) + 1024;
    return need < 96 * 1024 ? 96 * 1024 : need;
}

}  // namespace

struct TcPlan {
    int64_t tp, tq;  // row tiles of P and Q
    int cp, cq;      // chunks of the two passes
};

static TcPlan tc_plan(int64_t np_cap, int64_t nq_cap, int sm_count)
{
    TcPlan p;
    p.tp = (np_cap + kTM - 1) / kTM;
    p.tq = (nq_cap + kTM - 1) / kTM;
    p.cp = chunks_for(p.tp, p.tq, sm_count);
    p.cq = chunks_for(p.tq, p.tp, sm_count);
    return p;
}

size_t kmx_match_tc_extra_bytes(int64_t np_cap, int64_t nq_cap, int sm_count)
{
    TcPlan p = tc_plan(np_cap, nq_cap, sm_count);
    kmx_arena a{nullptr, 0};
    a.take((size_t)p.tp * kTileBytes);
    a.take((size_t)p.tq * kTileBytes);
    a.take(sizeof(Cand) * kTopK * (size_t)p.cp * (np_cap + 1));
    a.take(sizeof(Cand) * kTopK * (size_t)p.cq * (nq_cap + 1));
    return kmx_align_up(a.used, 256);
}

cudaError_t kmx_match_tc_launch(kmx_ctx* ctx, const float* dp, int64_t np_cap, const int64_t* d_np, const float* dq,
                                int64_t nq_cap, const int64_t* d_nq, kmx::MatchScratch& s)
{
    cudaStream_t st = ctx->stream;
    TcPlan p = tc_plan(np_cap, nq_cap, ctx->sm_count);
    kmx_arena a{static_cast<char*>(s.extra), 0};
    uint8_t* packP = (uint8_t*)a.take((size_t)p.tp * kTileBytes);
    uint8_t* packQ = (uint8_t*)a.take((size_t)p.tq * kTileBytes);
    Cand* partP = (Cand*)a.take(sizeof(Cand) * kTopK * (size_t)p.cp * (np_cap + 1));
    Cand* partQ = (Cand*)a.take(sizeof(Cand) * kTopK * (size_t)p.cq * (nq_cap + 1));
    const size_t smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(tc_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    KMX_COUNT_LAUNCH();
    pack_bf16<<<kmx_blocks(p.tp * kTM, 256), 256, 0, st>>>(dp, np_cap, d_np, p.tp * kTM, packP);
    KMX_COUNT_LAUNCH();
    pack_bf16<<<kmx_blocks(p.tq * kTM, 256), 256, 0, st>>>(dq, nq_cap, d_nq, p.tq * kTM, packQ);
    KMX_COUNT_LAUNCH();
    tc_topk<<<dim3((unsigned)p.tp, (unsigned)p.cp), kThreads, smem, st>>>(
        packP, np_cap, d_np, packQ, nq_cap, d_nq, (int)((p.tq + p.cp - 1) / p.cp), partP, ctx->d_err);
    KMX_COUNT_LAUNCH();
    tc_topk<<<dim3((unsigned)p.tq, (unsigned)p.cq), kThreads, smem, st>>>(
        packQ, nq_cap, d_nq, packP, np_cap, d_np, (int)((p.tp + p.cq - 1) / p.cq), partQ, ctx->d_err);
    KMX_COUNT_LAUNCH();
    rerank<<<kmx_blocks(np_cap, 8), 256, 0, st>>>(dp, np_cap, d_np, dq, partP, p.cp, s.part, nullptr);
    KMX_COUNT_LAUNCH();
    rerank<<<kmx_blocks(nq_cap, 8), 256, 0, st>>>(dq, nq_cap, d_nq, dp, partQ, p.cq, nullptr, s.colbest);
    return cudaGetLastError();
}
