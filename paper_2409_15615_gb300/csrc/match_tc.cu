// Mutual nearest-neighbour matching (Sec. III-C) with BF16 tensor-core
// distances and exact FP32 re-ranking.  The result equals the exact FP32
// path's (kmx_match, KMX_MATCH_FP32_EXACT) bit for bit.
//
// Why the operands are centred per tile.  A distance taken as
// |x|^2 + |y|^2 - 2 x.y loses the bits that d^2 needs when |x| |y| >> d^2;
// the descriptors of plane points are near-duplicates (d^2 ~ 0.3 against
// |x - mean|^2 ~ 10^3), so one global centre is not enough.  Rows that are
// close in descriptor space are therefore put next to each other (a Morton
// key over four statistics of the histograms, radix-sorted), every 128-row
// tile gets its own centre c, and each tile pair is computed as
//     d^2(x, y) = |x - c_C|^2 + |y - c_C|^2 - 2 (x - c_C).(y - c_C)
// with c_C the centre of the column tile: both factors of the product are
// small exactly for the pairs whose ranking matters.
//
// Stages (both clouds in one launch each where possible):
//   coords/keys/sort  per row four statistics (mean bin of each third of the
//             histogram, log2 of the first third's mass), normalised by their
//             range over both clouds, 7 bits each -> a 28-bit Morton key;
//             one stable radix sort over both clouds (a side bit on top).
//   pack      one CTA per 128-row tile: the tile centre, then per row
//             b = y - c in BF16 in the UMMA operand layout (K-major, 8x16-byte
//             core matrices, no swizzle) with three extra K slots
//             [sqrt(c') |b|, hi(|b|^2), lo(|b|^2)], and a header with |b|, the
//             centre and max |b|^2.  A packed tile is one contiguous bulk copy.
//   nearest   for each row tile, the column tile whose centre is nearest.
//   collect   one CTA per (128-row tile, chunk of column tiles): per column
//             tile the CTA writes its row tile re-centred on the column
//             tile's centre as the A operand [x - c_C, sqrt(c') |x - c_C|,
//             -1/2, -1/2] while the previous tile pair's MMA runs, one thread
//             issues tcgen05.mma (kind::f16, BF16, M = N = 128, three K steps
//             of 16) into one of two TMEM accumulators, and the 4 warps read
//             the other accumulator with tcgen05.ld.  The accumulator holds
//             M = a.b + c' |a| |b| - |b|^2 / 2 (approximately), so
//             L = |a|^2 - 2 M - e is a certified lower bound of the exact
//             d^2, and L + 4.1 c' |a| |b| + 2 e an upper bound.  Per row the
//             thread keeps the two smallest upper bounds U1 <= U2 it has seen
//             and collects every column with L <= U2 (its column index goes
//             to the row's candidate list).  Every column whose exact
//             distance is at most the row's second-smallest exact distance
//             is collected (L <= d <= d(2) <= U2).  A 32-column slice whose
//             largest M cannot give L <= U2 costs one three-input max per two
//             values.  The CTA starts with the nearest column tile, so U2 is
//             tight from the first tile on (outside its chunk that tile only
//             tightens the bounds).
//   rerank    one warp per row: the exact FP32 distance of every collected
//             column (sum_h (x_h - y_h)^2, one fused multiply-add per term in
//             h order: the arithmetic of the exact path), lowest index on
//             ties.  Rows of the source side give (d1, NN, d2); rows of the
//             target side give the packed (distance, row) best that the
//             reciprocity test reads.  A row whose list overflowed goes
//             through the exact FP32 tiles instead.
// Every wait on an mbarrier is bounded; on timeout the kernel records
// KMX_DERR_TIMEOUT, drains what it issued and frees its TMEM.
//
// The certified bounds.  With a, b the FP32 centred rows and their BF16
// roundings a', b' (8 significant bits: relative error <= 2^-8 each),
// |a'.b' - a.b| <= 2^-7 (1 + 2^-9) |a| |b|.  The tensor core's FP32
// accumulation of the 48 products is taken to lose at most 48 * 2^-22 of
// the sum of their magnitudes (a reading: the ISA promises FP32
// accumulation without stating its rounding).  The slot product
// bf16(sqrt(c')|a|) bf16(sqrt(c')|b|) >= (1 - 2^-8)^2 c' |a| |b| with
// c' = 0.008 exceeds both terms together; FP32 rounding of |a|^2, |b|^2,
// the hi/lo split of |b|^2 (2^-16), the accumulation error on the |b|^2
// slots and the rounding of the final exact distance are covered by
// e = 6e-5 (|a|^2 + max |b|^2 of the tile).
#include "kmx_internal.cuh"
#include "bulk_copy.cuh"
#include "match_common.cuh"

#include <cuda_bf16.h>
#include <float.h>

namespace {

using kmx::bulk_g2s;
using kmx::mbar_expect_tx;
using kmx::mbar_fence_init;
using kmx::mbar_init;
using kmx::mbar_wait;
using kmx::smem_u32;

constexpr int kTM = 128;                      // rows per tile (UMMA M)
constexpr int kTN = 128;                      // columns per column tile (UMMA N)
constexpr int kK = 48;                        // 33 values + 3 slots, padded to 3 x 16
constexpr int kOpBytesA = kTM * kK * 2;       // one BF16 row tile: 12288
constexpr int kOpBytesB = kTN * kK * 2;       // one BF16 column tile: 12288
constexpr int kCoreStride = 128;              // LBO: next 8-element K chunk
constexpr int kGroupStride = 6 * 128;         // SBO: next 8-row group
constexpr int kCenterStride = 36;             // floats per stored centre
// packed column tile: operand, then |b| per row, the centre, max |b|^2, and
// the largest |b| of every group of 8 rows
constexpr int kHdrBeta = kOpBytesB;
constexpr int kHdrCenter = kHdrBeta + kTN * 4;
constexpr int kHdrBmax = kHdrCenter + kCenterStride * 4;
constexpr int kHdrGBeta = kHdrBmax + 16;
constexpr int kColBytes = kHdrGBeta + (kTN / 8) * 4;  // 13024, a multiple of 16
constexpr int kStages = 4;                    // column-tile ring
constexpr int kThreads = 256;                 // 8 warps: two per TMEM lane quarter
constexpr int kTmemCols = 256;                // two 128-column FP32 accumulators
constexpr int kMaxChunks = 8;
constexpr int kCandCap = 512;                 // candidate list per row
constexpr float kC = 0.008f;                  // c' of the bounds
constexpr float kSqrtC = 0.08944271909999159f;
constexpr float kUpper = 4.1f * kC;
constexpr float kEfp = 6e-5f;
constexpr int kMortonBits = 7;                // per statistic; 4 x 7 = 28 bits

static_assert(kColBytes % 16 == 0, "bulk copies move multiples of 16 bytes");

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05; mbarrier and bulk copy in bulk_copy.cuh)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory stores -> visible to the tensor core's reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

// 64 consecutive FP32 columns of this thread's TMEM lane: two loads in
// flight, one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v)
{
    uint32_t r[64];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t* q = r + 32 * h;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
              "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15]),
              "=r"(q[16]), "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]), "=r"(q[23]),
              "=r"(q[24]), "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
            : "r"(taddr + 32 * h));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Write 8 operand values (one 16-byte core-matrix row) at chunk c of row r.
__device__ __forceinline__ void store_operand_chunk(uint8_t* tile, int r, int c, const float* v)
{
    uint4 w;
    w.x = pack_bf16x2(v[0], v[1]);
    w.y = pack_bf16x2(v[2], v[3]);
    w.z = pack_bf16x2(v[4], v[5]);
    w.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + (r / 8) * kGroupStride + (r % 8) * 16 + c * kCoreStride) = w;
}

// Write one 48-value operand row (values v[0..47]) at row r of a tile in the
// core-matrix layout.
__device__ __forceinline__ void store_operand_row(uint8_t* tile, int r, const float (&v)[kK])
{
    const int base = (r / 8) * kGroupStride + (r % 8) * 16;
#pragma unroll
    for (int c = 0; c < kK / 8; ++c) {
        uint4 w;
        w.x = pack_bf16x2(v[8 * c + 0], v[8 * c + 1]);
        w.y = pack_bf16x2(v[8 * c + 2], v[8 * c + 3]);
        w.z = pack_bf16x2(v[8 * c + 4], v[8 * c + 5]);
        w.w = pack_bf16x2(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4*>(tile + base + c * kCoreStride) = w;
    }
}

// ---------------------------------------------------------------------------
// locality order
// ---------------------------------------------------------------------------

// The four statistics of a descriptor row: the mean bin of each third of the
// histogram (0 for an empty third) and log2 of the first third's mass
// (at least 0).  All are >= 0, so their float bits order like the values.
__device__ __forceinline__ void row_stats(const float* __restrict__ row, float (&s)[4])
{
    float m0 = 0.f;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        float w = 0.f, m = 0.f;
#pragma unroll
        for (int b = 0; b < 11; ++b) {
            const float h = __ldg(row + 11 * t + b);
            w += h;
            m = fmaf((float)b, h, m);
        }
        s[t] = w > 0.f ? fmaxf(m / w, 0.f) : 0.f;
        if (t == 0) m0 = w;
    }
    s[3] = log2f(fmaxf(m0, 1.f));
}

// Per row of both clouds: the statistics, their range (atomic min / max of
// the float bits) and a non-finite check.  Rows e < np_cap are the source
// cloud, the others the target cloud.
__global__ void __launch_bounds__(256) tc_coords(const float* __restrict__ P, int64_t np_cap,
                                                 const int64_t* d_np, const float* __restrict__ Q, int64_t nq_cap,
                                                 const int64_t* d_nq, float4* __restrict__ coords,
                                                 unsigned int* __restrict__ range, unsigned int* err)
{
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    float lo[4] = {FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX}, hi[4] = {0.f, 0.f, 0.f, 0.f};
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < np_cap + nq_cap;
         e += (int64_t)gridDim.x * 256) {
        const bool side = e >= np_cap;
        const int64_t r = side ? e - np_cap : e;
        if (r >= (side ? nq : np)) continue;
        const float* row = (side ? Q : P) + r * KMX_DESC_STRIDE;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) bad |= !isfinite(__ldg(row + h));
        float s[4];
        row_stats(row, s);
        coords[e] = make_float4(s[0], s[1], s[2], s[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            lo[k] = fminf(lo[k], s[k]);
            hi[k] = fmaxf(hi[k], s[k]);
        }
    }
    if (bad) kmx_raise(err, KMX_DERR_RANGE);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned l = __reduce_min_sync(0xffffffffu, __float_as_uint(lo[k]));
        const unsigned h = __reduce_max_sync(0xffffffffu, __float_as_uint(hi[k]));
        if ((threadIdx.x & 31) == 0) {
            atomicMin(range + k, l);
            atomicMax(range + 4 + k, h);
        }
    }
}

__device__ __forceinline__ uint32_t spread4(uint32_t v)  // 7 bits -> every 4th bit
{
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < kMortonBits; ++b) r |= ((v >> b) & 1u) << (4 * b);
    return r;
}

// Sort keys: side bit 29, "past the count" bit 28, 28-bit Morton code.
__global__ void __launch_bounds__(256) tc_keys(int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                                               const int64_t* d_nq, const float4* __restrict__ coords,
                                               const unsigned int* __restrict__ range, uint32_t* __restrict__ keys,
                                               int32_t* __restrict__ vals)
{
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    const float scale = (float)((1 << kMortonBits) - 1);
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < np_cap + nq_cap;
         e += (int64_t)gridDim.x * 256) {
        const bool side = e >= np_cap;
        const int64_t r = side ? e - np_cap : e;
        uint32_t key = (uint32_t)side << 29;
        if (r < (side ? nq : np)) {
            const float4 c = coords[e];
            const float cs[4] = {c.x, c.y, c.z, c.w};
            uint32_t m = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float lo = __uint_as_float(range[k]), hi = __uint_as_float(range[4 + k]);
                const float t = hi > lo ? (cs[k] - lo) / (hi - lo) : 0.f;
                const uint32_t q = (uint32_t)fminf(fmaxf(t * scale + 0.5f, 0.f), scale);
                m |= spread4(q) << (3 - k);
            }
            key |= m;
        } else {
            key |= 1u << 28;
        }
        keys[e] = key;
        vals[e] = (int32_t)r;
    }
}

// ---------------------------------------------------------------------------
// pack: one CTA of 128 threads per column tile of one cloud
// ---------------------------------------------------------------------------

// Rows of the tile are sorted positions [128 t, 128 t + 128) of the cloud;
// perm maps a sorted position to the descriptor row.  Writes the packed
// column tile and the centre (also to centers[t]).
__global__ void __launch_bounds__(kTN) tc_pack(const float* __restrict__ desc, const int32_t* __restrict__ perm,
                                               int64_t n_cap, const int64_t* d_n, uint8_t* __restrict__ out,
                                               float* __restrict__ centers)
{
    __shared__ float rows_s[kTN][KMX_DESC_DIM + 1];
    __shared__ float cen[kCenterStride];
    __shared__ unsigned int bmax2;
    const int64_t n = kmx_count(d_n, n_cap);
    const int64_t t = blockIdx.x;
    if (t * kTN >= n && !(t == 0)) return;  // tiles past the count are never read
    const int tid = threadIdx.x;
    const int64_t r = t * kTN + tid;
    const bool valid = r < n;
    float y[KMX_DESC_DIM];
    if (valid) {
        const float* row = desc + (int64_t)perm[r] * KMX_DESC_STRIDE;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) y[h] = __ldg(row + h);
    } else {
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) y[h] = 0.f;
    }
#pragma unroll
    for (int h = 0; h < KMX_DESC_DIM; ++h) rows_s[tid][h] = y[h];
    if (tid == 0) bmax2 = 0u;
    __syncthreads();
    const int cnt = (int)max((int64_t)0, min((int64_t)kTN, n - t * kTN));
    if (tid < kCenterStride) {
        float sum = 0.f;
        if (tid < KMX_DESC_DIM)
            for (int i = 0; i < cnt; ++i) sum += rows_s[i][tid];
        cen[tid] = (tid < KMX_DESC_DIM && cnt > 0) ? sum / (float)cnt : 0.f;
    }
    __syncthreads();
    float v[kK];
    float nb = 0.f;
#pragma unroll
    for (int h = 0; h < KMX_DESC_DIM; ++h) {
        const float bv = y[h] - cen[h];
        v[h] = bv;
        nb = fmaf(bv, bv, nb);
    }
    const float beta = sqrtf(nb);
#pragma unroll
    for (int h = KMX_DESC_DIM; h < kK; ++h) v[h] = 0.f;
    if (valid) {
        const float hi = __bfloat162float(__float2bfloat16_rn(nb));
        v[KMX_DESC_DIM] = kSqrtC * beta;
        v[KMX_DESC_DIM + 1] = hi;
        v[KMX_DESC_DIM + 2] = nb - hi;
    } else {
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) v[h] = 0.f;
        v[KMX_DESC_DIM + 1] = INFINITY;  // -1/2 x inf: the padding column never qualifies
    }
    uint8_t* tile = out + t * (int64_t)kColBytes;
    store_operand_row(tile, tid, v);
    reinterpret_cast<float*>(tile + kHdrBeta)[tid] = valid ? beta : 0.f;
    if (valid) atomicMax(&bmax2, __float_as_uint(nb));
    if (tid < kCenterStride) {
        reinterpret_cast<float*>(tile + kHdrCenter)[tid] = cen[tid];
        centers[t * kCenterStride + tid] = cen[tid];
    }
    __syncthreads();
    if (tid < 4) reinterpret_cast<float*>(tile + kHdrBmax)[tid] = tid == 0 ? __uint_as_float(bmax2) : 0.f;
    // the largest |b| of each group of 8 rows (lanes 8k .. 8k + 7 of a warp)
    float gb = valid ? beta : 0.f;
#pragma unroll
    for (int o = 4; o >= 1; o >>= 1) gb = fmaxf(gb, __shfl_xor_sync(0xffffffffu, gb, o));
    if ((tid & 7) == 0) reinterpret_cast<float*>(tile + kHdrGBeta)[tid >> 3] = gb;
}

// For each tile of X (its row tiles are its column tiles): the column tile
// of Y with the nearest centre (ties to the lower tile).  One warp per tile.
__global__ void __launch_bounds__(256) tc_nearest(const float* __restrict__ cx, int64_t nx_cap, const int64_t* d_nx,
                                                  const float* __restrict__ cy, int64_t ny_cap, const int64_t* d_ny,
                                                  int32_t* __restrict__ nearest)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int64_t ntx = (kmx_count(d_nx, nx_cap) + kTN - 1) / kTN;
    const int64_t nty = (kmx_count(d_ny, ny_cap) + kTN - 1) / kTN;
    if (t >= ntx) return;
    float c[KMX_DESC_DIM];
#pragma unroll
    for (int h = 0; h < KMX_DESC_DIM; ++h) c[h] = cx[t * kCenterStride + h];
    float best = INFINITY;
    int bi = 0x7fffffff;
    for (int64_t u = lane; u < nty; u += 32) {
        float d = 0.f;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) {
            const float e = c[h] - cy[u * kCenterStride + h];
            d = fmaf(e, e, d);
        }
        if (d < best) {
            best = d;
            bi = (int)u;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if (lane == 0) nearest[t] = bi == 0x7fffffff ? 0 : bi;
}

// ---------------------------------------------------------------------------
// tensor-core candidate collection
// ---------------------------------------------------------------------------

struct TcShared {
    uint8_t a[2][kOpBytesA];
    uint8_t b[kStages][kColBytes];
    // per row and step (modulo 3: written one step ahead of its reads, while
    // the slowest thread may still read the previous step's): |a|^2 - e,
    // the factor c' |a| of the upper bounds, 2 e, and the second-smallest
    // upper bound over the row's two column slices as of three steps earlier
    float4 rowc[3][kTM];
    float2 ul[3][kTM][2];  // (U1, U2) of the two column slices of every row, by step modulo 3
    uint64_t bar_b[kStages], bar_mma[2];
    uint32_t tmem;
};

// Threads (8 warps) have two roles per step (one 128-column tile):
//   re-centring  thread t writes values 16 (t & 1) .. of row t >> 1 of the A
//                operand (the t & 1 == 1 thread values 16 .. 32 and the three
//                slots); the two threads of a row are neighbouring lanes and
//                add their partial |x - c|^2 with one shuffle;
//   epilogue     warp w reads TMEM lanes (rows) 32 (w & 3) .. + 31 and
//                accumulator columns 64 (w >> 2) .. + 63.  The two threads of
//                a row keep their own bounds and candidate decisions over
//                their own columns (disjoint sets, one list per row).
// Two CTAs per SM (each holds half of the TMEM), so that one CTA's
// re-centring and barrier overlap the other's epilogue.  One barrier per
// step: it publishes the A operand to the MMA and orders the previous
// step's accumulator reads before the next MMA into that accumulator.
//
// The grid is sized from the capacities; the (row tile, column chunk) split
// of the actual counts is decided here (kmx::work_chunks).
__global__ void __launch_bounds__(kThreads, 2) tc_collect(const float* __restrict__ X,
                                                         const int32_t* __restrict__ permX, int64_t nx_cap,
                                                         const int64_t* d_nx, const uint8_t* __restrict__ packY,
                                                         int64_t ny_cap, const int64_t* d_ny,
                                                         const int32_t* __restrict__ nearest, int target_ctas,
                                                         int32_t* __restrict__ cand, int32_t* __restrict__ cnt,
                                                         unsigned int* err)
{
    extern __shared__ uint8_t smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t rows = kmx_count(d_nx, nx_cap), cols = kmx_count(d_ny, ny_cap);
    const int64_t n_rt = (rows + kTM - 1) / kTM;
    const int64_t n_ct = (cols + kTN - 1) / kTN;
    const int chunks = kmx::work_chunks(n_rt, n_ct, target_ctas, kMaxChunks);
    if ((int64_t)blockIdx.x >= n_rt * chunks) return;
    const int chunk = (int)(blockIdx.x % chunks);
    const int64_t rt = blockIdx.x / chunks;
    const int64_t tiles_per_chunk = (n_ct + chunks - 1) / chunks;
    const int64_t t0 = chunk * tiles_per_chunk;
    const int T = (int)max((int64_t)0, min(n_ct, t0 + tiles_per_chunk) - t0);
    if (T == 0) return;
    // the sequence of column tiles: the nearest tile first, then the chunk
    // (without the nearest tile when it lies inside the chunk)
    const int64_t cs = nearest[rt];
    const bool cs_in = cs >= t0 && cs < t0 + T;
    const int nseq = T + (cs_in ? 0 : 1);
    auto tile_of = [&](int s) -> int64_t {
        if (s == 0) return cs;
        const int64_t rr = t0 + s - 1;
        return (cs_in && rr >= cs) ? rr + 1 : rr;
    };
    const uint32_t idesc = idesc_bf16(kTM, kTN);

    // re-centring role
    const int rrow = tid >> 1, part = tid & 1;
    const int64_t xrow = rt * kTM + rrow;
    const bool xvalid = xrow < rows;
    // epilogue role
    const int quarter = warp & 3, slice = warp >> 2;
    const int r = quarter * 32 + lane;
    const int64_t row = rt * kTM + r;
    const bool row_valid = row < rows;

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&S.bar_b[st], 1);
        mbar_init(&S.bar_mma[0], 1);
        mbar_init(&S.bar_mma[1], 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
    if (part == 1) {  // the last K chunk (values 40..47) is zero in every A operand
        const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        store_operand_chunk(S.a[0], rrow, 5, z);
        store_operand_chunk(S.a[1], rrow, 5, z);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;

    float x[17];  // values 16 part .. 16 part + 15 (and 32 for part 1) of this thread's re-centring row
    {
        const float* xr = xvalid ? X + (int64_t)permX[xrow] * KMX_DESC_STRIDE + 16 * part : nullptr;
#pragma unroll
        for (int h = 0; h < 17; ++h) x[h] = (xvalid && (h < 16 || part == 1)) ? __ldg(xr + h) : 0.f;
    }

    int issued_b = 0, issued_mma = 0;
    if (tid == 0) {
        for (; issued_b < nseq && issued_b < kStages; ++issued_b) {
            mbar_expect_tx(&S.bar_b[issued_b], kColBytes);
            bulk_g2s(S.b[issued_b], packY + tile_of(issued_b) * (int64_t)kColBytes, kColBytes, &S.bar_b[issued_b]);
        }
    }
    bool fail = false, failed = false;
    // upper bounds of the columns this thread has seen (own slice only), and
    // the second-smallest upper bound over all four slices of the row as of
    // the last barrier
    float U1 = FLT_MAX, U2 = FLT_MAX, Ush = FLT_MAX;

    for (int s = 0; s <= nseq; ++s) {
        if (s < nseq) {
            // ---- A operand of step s: rows re-centred on the column tile's centre
            if (!mbar_wait(&S.bar_b[s % kStages], (s / kStages) & 1)) fail = true;
            const uint8_t* bt = S.b[s % kStages];
            const float4* cen4 = reinterpret_cast<const float4*>(bt + kHdrCenter) + 4 * part;
            float av[16];
            float p2 = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 cv = cen4[c];
                av[4 * c + 0] = x[4 * c + 0] - cv.x;
                av[4 * c + 1] = x[4 * c + 1] - cv.y;
                av[4 * c + 2] = x[4 * c + 2] - cv.z;
                av[4 * c + 3] = x[4 * c + 3] - cv.w;
            }
#pragma unroll
            for (int h = 0; h < 16; ++h) p2 = fmaf(av[h], av[h], p2);
            float a32 = 0.f;
            if (part == 1) {
                a32 = x[16] - reinterpret_cast<const float*>(bt + kHdrCenter)[32];
                p2 = fmaf(a32, a32, p2);
            }
            uint8_t* at = S.a[s & 1];
            store_operand_chunk(at, rrow, 2 * part, av);
            store_operand_chunk(at, rrow, 2 * part + 1, av + 8);
            // the two partial sums of the row (neighbouring lanes); both lanes
            // form the same total
            p2 += __shfl_xor_sync(0xffffffffu, p2, 1);
            if (part == 1) {
                const float v4[8] = {a32, kSqrtC * sqrtf(p2), -0.5f, -0.5f, 0.f, 0.f, 0.f, 0.f};
                store_operand_chunk(at, rrow, 4, v4);
            }
            if (part == 0) {
                const float bmax2 = reinterpret_cast<const float*>(bt + kHdrBmax)[0];
                const float ef = kEfp * (p2 + bmax2);
                float ush = FLT_MAX;
                if (s >= 3) {
                    // the row's two slices as of step s - 3 (written in the
                    // epilogue of iteration s - 2, published by the barrier of
                    // step s - 1): their upper bounds come from disjoint
                    // columns, so the second smallest of the eight is the
                    // second smallest over all columns they saw
                    const float2 a0 = S.ul[s % 3][rrow][0], a1 = S.ul[s % 3][rrow][1];
                    ush = fminf(fmaxf(a0.x, a1.x), a0.x <= a1.x ? a0.y : a1.y);
                }
                S.rowc[s % 3][rrow] = make_float4(p2 - ef, kUpper * sqrtf(p2), 2.f * ef, ush);
            }
            fence_proxy_async();
        }
        // publishes the A operand and r2 of step s; every thread has finished
        // the epilogue of step s - 2 (accumulator (s & 1) is free) and its
        // reads of the column tile of step s - 2
        tc_fence_before();
        failed = __syncthreads_or(fail) != 0;
        tc_fence_after();
        if (failed) break;
        if (tid == 0) {
            if (s < nseq) {
                const uint32_t a_base = smem_u32(S.a[s & 1]);
                const uint32_t b_base = smem_u32(S.b[s % kStages]);
                const uint32_t d = tmem + (uint32_t)((s & 1) * kTN);
#pragma unroll
                for (int k = 0; k < kK / 16; ++k) {
                    const uint32_t ko = k * 2 * kCoreStride;
                    umma_bf16(d, smem_desc(a_base + ko, kCoreStride, kGroupStride),
                              smem_desc(b_base + ko, kCoreStride, kGroupStride), idesc, k > 0);
                }
                umma_commit(&S.bar_mma[s & 1]);
                ++issued_mma;
            }
            // the stage of step s - 2 is free: its MMA and its epilogue are done
            if (s >= 2 && s - 2 + kStages < nseq) {
                const int st = (s - 2) % kStages;
                mbar_expect_tx(&S.bar_b[st], kColBytes);
                bulk_g2s(S.b[st], packY + tile_of(s - 2 + kStages) * (int64_t)kColBytes, kColBytes, &S.bar_b[st]);
                ++issued_b;
            }
        }
        if (s >= 1) {
            // ---- epilogue of step p = s - 1: this thread's 64 columns
            const int p = s - 1;
            if (!mbar_wait(&S.bar_mma[p & 1], (p >> 1) & 1)) fail = true;
            tc_fence_after();
            const uint8_t* bt = S.b[p % kStages];
            const float4 rc = S.rowc[p % 3][r];
            const float rb = rc.x, ua = rc.y, ue = rc.z;
            Ush = fminf(Ush, rc.w);
            const float* gbeta = reinterpret_cast<const float*>(bt + kHdrGBeta) + slice * 8;
            const bool collect = p > 0 || cs_in;
            const int64_t col0 = tile_of(p) * kTN + slice * 64;
            const uint32_t lane_addr =
                tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((p & 1) * kTN + slice * 64);
            float v[64];
            tmem_ld64(lane_addr, v);
            // the eight groups' smallest lower bounds, independent of each
            // other; one branch for all of them in the common case
            float Lm[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const float* vg = v + 8 * g;
                const float m = fmax3(fmax3(vg[0], vg[1], vg[2]), fmax3(vg[3], vg[4], vg[5]), fmaxf(vg[6], vg[7]));
                // L = |a|^2 - e - 2 M is monotone in M: the group's largest M
                // gives its smallest L
                Lm[g] = fmaf(-2.f, m, rb);
            }
            const float lmin = fmin3(fmin3(Lm[0], Lm[1], Lm[2]), fmin3(Lm[3], Lm[4], Lm[5]), fminf(Lm[6], Lm[7]));
            if (row_valid && lmin <= fminf(U2, Ush)) {
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const float* vg = v + 8 * g;
                    const float Lmin = Lm[g];
                    if (Lmin <= fminf(U2, Ush)) {
                        // the group's two best columns (largest M first): upper
                        // bounds for them
                        float h0 = fmaxf(vg[0], vg[1]), l0 = fminf(vg[0], vg[1]);
                        float h1 = fmaxf(vg[2], vg[3]), l1 = fminf(vg[2], vg[3]);
                        float h2 = fmaxf(vg[4], vg[5]), l2 = fminf(vg[4], vg[5]);
                        float h3 = fmaxf(vg[6], vg[7]), l3 = fminf(vg[6], vg[7]);
                        l0 = fmaxf(fminf(h0, h1), fmaxf(l0, l1));
                        h0 = fmaxf(h0, h1);
                        l2 = fmaxf(fminf(h2, h3), fmaxf(l2, l3));
                        h2 = fmaxf(h2, h3);
                        const float m2 = fmaxf(fminf(h0, h2), fmaxf(l0, l2));
                        const float uadd = fmaf(ua, gbeta[g], ue);
                        const float Ua = Lmin + uadd, Ub = fmaf(-2.f, m2, rb) + uadd;
                        if (Ua < U1) {
                            U2 = fminf(U1, Ub);
                            U1 = Ua;
                        } else if (Ua < U2) {
                            U2 = Ua;
                        }
                        if (collect) {
                            const float thr = fminf(U2, Ush);
                            unsigned msk = 0;
#pragma unroll
                            for (int j = 0; j < 8; ++j) msk |= (fmaf(-2.f, vg[j], rb) <= thr ? 1u : 0u) << j;
                            const int k = __popc(msk);
                            if (k) {
                                int pos = atomicAdd(cnt + row, k);
                                while (msk) {
                                    const int j = __ffs(msk) - 1;
                                    msk &= msk - 1;
                                    if (pos < kCandCap) cand[row * kCandCap + pos] = (int32_t)(col0 + 8 * g + j);
                                    ++pos;
                                }
                            }
                        }
                    }
                }
            }
            S.ul[p % 3][r][slice] = make_float2(U1, U2);
            tc_fence_before();
        }
    }
    if (failed) {
        // drain: every issued copy and MMA must land before the memory goes
        // away.  Each barrier has at most one phase outstanding, so waiting
        // for the last phase issued on each barrier suffices.
        if (tid == 0) {
            kmx_raise(err, KMX_DERR_TIMEOUT);
            for (int st = 0; st < kStages; ++st) {
                const int last = issued_b - 1 - ((issued_b - 1 - st) % kStages + kStages) % kStages;
                if (last >= 0 && last % kStages == st) mbar_wait(&S.bar_b[st], (last / kStages) & 1);
            }
            for (int k = 0; k < 2; ++k) {
                const int last = issued_mma - 1 - ((issued_mma - 1 - k) % 2 + 2) % 2;
                if (last >= 0 && (last & 1) == k) mbar_wait(&S.bar_mma[k], (last >> 1) & 1);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// exact FP32 re-ranking of the collected columns
// ---------------------------------------------------------------------------

// One warp per sorted row position.  Rows whose list overflowed are flagged
// for the exact fallback.  rows_out (source side) gets (d1, NN, d2) at the
// original row; cols_best (target side) the packed (d1, NN).
__global__ void __launch_bounds__(256) tc_rerank(const float* __restrict__ X, const int32_t* __restrict__ permX,
                                                 int64_t nx_cap, const int64_t* d_nx, const float* __restrict__ Y,
                                                 const int32_t* __restrict__ permY, int64_t ny_cap,
                                                 const int64_t* d_ny, const int32_t* __restrict__ cand,
                                                 const int32_t* __restrict__ cnt,
                                                 kmx::RowBest* __restrict__ rows_out,
                                                 unsigned long long* __restrict__ cols_best,
                                                 int32_t* __restrict__ fallback, int* __restrict__ final_chunks)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (final_chunks && i == 0 && lane == 0) *final_chunks = 1;  // rows_out holds whole-row summaries
    if (i >= kmx_count(d_nx, nx_cap)) return;
    const int orig = permX[i];
    const int c = cnt[i];
    if (c > kCandCap) {
        if (lane == 0) fallback[orig] = 1;
        return;
    }
    const float* x = X + (int64_t)orig * KMX_DESC_STRIDE;
    const int64_t ny = kmx_count(d_ny, ny_cap);
    float b1 = INFINITY, b2 = INFINITY;
    int j1 = 0x7fffffff;
    for (int q = lane; q < c; q += 32) {
        const int pos = cand[i * kCandCap + q];
        if (pos < 0 || pos >= ny) continue;  // padding columns are never collected
        const int j = permY[pos];
        const float* y = Y + (int64_t)j * KMX_DESC_STRIDE;
        float acc = 0.f;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) {
            const float e = __ldg(x + h) - __ldg(y + h);
            acc = fmaf(e, e, acc);
        }
        kmx::row_update(b1, j1, b2, acc, j);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const float od1 = __shfl_xor_sync(0xffffffffu, b1, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
        const float od2 = __shfl_xor_sync(0xffffffffu, b2, o);
        kmx::row_merge(b1, j1, b2, od1, oj, od2);
    }
    if (lane != 0) return;
    if (rows_out) rows_out[orig] = kmx::RowBest{b1, j1, b2};
    if (cols_best && j1 != 0x7fffffff) cols_best[orig] = kmx::pack_dist_index(b1, (uint32_t)j1);
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
// the re-ranked rows went.
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
    // at least 96 KB: at most two CTAs per SM, i.e. two 256-column TMEM
    // allocations (a third CTA would wait in tcgen05.alloc)
    const size_t need = sizeof(TcShared) + 1024;
    return need < 96 * 1024 ? 96 * 1024 : need;
}

struct TcBuffers {
    float4* coords;         // [np_cap + nq_cap]
    unsigned int* range;    // [8]: min bits of the 4 statistics, then max bits
    uint32_t *keys, *keys_tmp;
    int32_t *vals, *vals_tmp;  // sorted: [0, np) source rows, [np_cap, np_cap + nq) target rows
    void* sort_scratch;
    uint8_t *packP, *packQ;
    float *cenP, *cenQ;
    int32_t *nearP, *nearQ;
    int32_t *candP, *candQ, *cntP, *cntQ;
    int* chunks;            // [2] fallback P, [3] fallback Q
    int32_t *flagP, *flagQ, *listP, *listQ;
    int64_t *posP, *posQ, *nlist;  // nlist[0] P, [1] Q
    kmx::RowBest *fbP, *fbQ;
};

TcBuffers tc_carve(void* base, int64_t np_cap, int64_t nq_cap, size_t* total)
{
    TcBuffers b{};
    kmx_arena a{static_cast<char*>(base), 0};
    const int64_t n2 = np_cap + nq_cap;
    const int64_t tp = (np_cap + kTN - 1) / kTN, tq = (nq_cap + kTN - 1) / kTN;  // column tiles
    const int fc = kmx_match_fp32_max_chunks();
    b.coords = (float4*)a.take(sizeof(float4) * (size_t)n2);
    b.range = (unsigned int*)a.take(sizeof(unsigned int) * 8);
    b.keys = (uint32_t*)a.take(sizeof(uint32_t) * (size_t)n2);
    b.keys_tmp = (uint32_t*)a.take(sizeof(uint32_t) * (size_t)n2);
    b.vals = (int32_t*)a.take(sizeof(int32_t) * (size_t)n2);
    b.vals_tmp = (int32_t*)a.take(sizeof(int32_t) * (size_t)n2);
    b.sort_scratch = a.take(kmx_sort_scratch_bytes(n2));
    b.packP = (uint8_t*)a.take((size_t)tp * kColBytes);
    b.packQ = (uint8_t*)a.take((size_t)tq * kColBytes);
    b.cenP = (float*)a.take(sizeof(float) * kCenterStride * (size_t)tp);
    b.cenQ = (float*)a.take(sizeof(float) * kCenterStride * (size_t)tq);
    b.nearP = (int32_t*)a.take(sizeof(int32_t) * (size_t)tp);
    b.nearQ = (int32_t*)a.take(sizeof(int32_t) * (size_t)tq);
    b.candP = (int32_t*)a.take(sizeof(int32_t) * kCandCap * (size_t)np_cap);
    b.candQ = (int32_t*)a.take(sizeof(int32_t) * kCandCap * (size_t)nq_cap);
    b.cntP = (int32_t*)a.take(sizeof(int32_t) * (size_t)(np_cap + nq_cap));
    b.cntQ = b.cntP + np_cap;
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
    const int64_t n2 = np_cap + nq_cap;
    const int64_t tp = (np_cap + kTM - 1) / kTM, tq = (nq_cap + kTM - 1) / kTM;    // row tiles
    const int64_t ctp = (np_cap + kTN - 1) / kTN, ctq = (nq_cap + kTN - 1) / kTN;  // column tiles (the same)
    const size_t smem = tc_smem_bytes();
    cudaError_t e = kmx_once_per_device(kmx_attr_tc_topk, [smem] {
        return cudaFuncSetAttribute(tc_collect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e) return e;
    if ((e = cudaMemsetAsync(b.flagP, 0, sizeof(int32_t) * (np_cap + 1), st))) return e;
    if ((e = cudaMemsetAsync(b.flagQ, 0, sizeof(int32_t) * (nq_cap + 1), st))) return e;
    if ((e = cudaMemsetAsync(b.cntP, 0, sizeof(int32_t) * (size_t)n2, st))) return e;
    if ((e = cudaMemsetAsync(b.range, 0xFF, sizeof(unsigned int) * 4, st))) return e;
    if ((e = cudaMemsetAsync(b.range + 4, 0, sizeof(unsigned int) * 4, st))) return e;
    // locality order of both clouds
    const unsigned gb = kmx_stride_blocks(n2, 256, ctx->sm_count);
    KMX_COUNT_LAUNCH();
    tc_coords<<<gb, 256, 0, st>>>(dp, np_cap, d_np, dq, nq_cap, d_nq, b.coords, b.range, ctx->d_err);
    KMX_COUNT_LAUNCH();
    tc_keys<<<gb, 256, 0, st>>>(np_cap, d_np, nq_cap, d_nq, b.coords, b.range, b.keys, b.vals);
    if ((e = cudaGetLastError())) return e;
    if ((e = kmx_sort_u32(ctx, b.keys, b.vals, b.keys_tmp, b.vals_tmp, n2, 32, b.sort_scratch))) return e;
    const int32_t* permP = b.vals;
    const int32_t* permQ = b.vals + np_cap;
    // packed tiles and centres
    KMX_COUNT_LAUNCH();
    tc_pack<<<(unsigned)ctp, kTN, 0, st>>>(dp, permP, np_cap, d_np, b.packP, b.cenP);
    KMX_COUNT_LAUNCH();
    tc_pack<<<(unsigned)ctq, kTN, 0, st>>>(dq, permQ, nq_cap, d_nq, b.packQ, b.cenQ);
    KMX_COUNT_LAUNCH();
    tc_nearest<<<kmx_blocks(ctp, 8), 256, 0, st>>>(b.cenP, np_cap, d_np, b.cenQ, nq_cap, d_nq, b.nearP);
    KMX_COUNT_LAUNCH();
    tc_nearest<<<kmx_blocks(ctq, 8), 256, 0, st>>>(b.cenQ, nq_cap, d_nq, b.cenP, np_cap, d_np, b.nearQ);
    // candidates both ways
    const int target = 2 * ctx->sm_count;
    KMX_COUNT_LAUNCH();
    tc_collect<<<(unsigned)(tp * kMaxChunks), kThreads, smem, st>>>(dp, permP, np_cap, d_np, b.packQ, nq_cap, d_nq,
                                                                    b.nearP, target, b.candP, b.cntP, ctx->d_err);
    KMX_COUNT_LAUNCH();
    tc_collect<<<(unsigned)(tq * kMaxChunks), kThreads, smem, st>>>(dq, permQ, nq_cap, d_nq, b.packP, np_cap, d_np,
                                                                    b.nearQ, target, b.candQ, b.cntQ, ctx->d_err);
    // exact re-ranking; overflowed rows are flagged
    KMX_COUNT_LAUNCH();
    tc_rerank<<<kmx_blocks(np_cap, 8), 256, 0, st>>>(dp, permP, np_cap, d_np, dq, permQ, nq_cap, d_nq, b.candP,
                                                     b.cntP, s.part, nullptr, b.flagP, s.chunks);
    KMX_COUNT_LAUNCH();
    tc_rerank<<<kmx_blocks(nq_cap, 8), 256, 0, st>>>(dq, permQ, nq_cap, d_nq, dp, permP, np_cap, d_np, b.candQ,
                                                     b.cntQ, nullptr, s.colbest, b.flagQ, nullptr);
    if ((e = cudaGetLastError())) return e;
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

// Diagnostics of the last tensor-core match on this scratch: rows that went
// through the exact fallback (source, target) and candidates collected
// (source, target), as four int64 values in the caller's device buffer.
__global__ void tc_stats(const int64_t* __restrict__ nlist, const int32_t* __restrict__ cntP, int64_t np_cap,
                         const int64_t* d_np, const int32_t* __restrict__ cntQ, int64_t nq_cap, const int64_t* d_nq,
                         int64_t* __restrict__ out)
{
    __shared__ unsigned long long sp, sq;
    if (threadIdx.x == 0) {
        sp = 0;
        sq = 0;
    }
    __syncthreads();
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    unsigned long long a = 0, b = 0;
    for (int64_t i = threadIdx.x; i < np; i += blockDim.x) a += (unsigned long long)min(cntP[i], kCandCap);
    for (int64_t i = threadIdx.x; i < nq; i += blockDim.x) b += (unsigned long long)min(cntQ[i], kCandCap);
    atomicAdd(&sp, a);
    atomicAdd(&sq, b);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = nlist[0];
        out[1] = nlist[1];
        out[2] = (int64_t)sp;
        out[3] = (int64_t)sq;
    }
}

cudaError_t kmx_match_tc_stats(kmx_ctx* ctx, void* extra, int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                               const int64_t* d_nq, int64_t* dst)
{
    size_t total = 0;
    TcBuffers b = tc_carve(extra, np_cap, nq_cap, &total);
    KMX_COUNT_LAUNCH();
    tc_stats<<<1, 256, 0, ctx->stream>>>(b.nlist, b.cntP, np_cap, d_np, b.cntQ, nq_cap, d_nq, dst);
    return cudaGetLastError();
}
