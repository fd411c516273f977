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
//   order     a principal-direction tree over the rows of each cloud: a
//             node's rows are split at a whole number of 128-row tiles
//             (left: ceil(len / 256) * 128 rows) by their projection on the
//             node's principal direction (power iteration on up to 256
//             sampled rows).  The upper levels run level by level with one
//             stable radix sort per level keyed by (side, node, quantised
//             projection); below nodes of 16 tiles one CTA per node finishes
//             its subtree in shared memory (bitonic sorts).  The leaves are
//             the 128-row tiles, and they are tight: the rows of a tile are
//             similar descriptors.
//   pack      one CTA per 128-row tile: the tile centre, then per row
//             b = y - c in BF16 in the UMMA operand layout (K-major, 8x16-byte
//             core matrices, no swizzle) with three extra K slots
//             [sqrt(c') |b|, hi(|b|^2), lo(|b|^2)], and a header with |b|, the
//             centre and max |b|^2.  A packed tile is one contiguous bulk copy.
//   plan      one CTA per row tile: the column tile with the nearest centre
//             is compared exactly (FP32, the exact path's arithmetic); its
//             columns up to each row's second-smallest distance d2 are the
//             row's first candidates and d2 its first upper bound U.  A
//             column tile with centre c and radius r = max |y - c| can only
//             hold a column within U of row x if |x - c| - r <= sqrt(U)
//             (triangle inequality; tested first for the whole row tile with
//             its own centre and radius, then row by row, with margins for
//             FP32 rounding).  The tiles that pass form the row tile's list,
//             cut into work items of 32 tiles.
//   collect   persistent CTAs, each taking every gridDim-th work item: per
//             column tile of the item the CTA writes its row tile re-centred
//             on the column tile's centre as the A operand
//             [x - c_C, sqrt(c') |x - c_C|, -1/2, -1/2] while earlier tiles'
//             products run, one thread issues tcgen05.mma (kind::f16, BF16,
//             M = N = 128, three K steps of 16) into one of four TMEM
//             accumulators, and two warpgroups of four warps read them
//             with tcgen05.ld (alternate tiles, two tiles in flight).  The
//             accumulator holds M = a.b + c' |a| |b| - |b|^2 / 2
//             (approximately), so L = |a|^2 - 2 M - e is a certified lower
//             bound of the exact d^2, and L + 4.1 c' |a| |b| + 2 e an upper
//             bound.  Per row the thread keeps the two smallest upper bounds
//             U1 <= U2 (starting from the row's bound U) and collects every
//             column with L <= U2 (its column index goes to the row's
//             candidate list).  Every column whose exact distance is at most
//             the row's second-smallest exact distance is collected
//             (L <= d <= d(2) <= U2).  A group of 8 columns whose largest
//             M cannot give L <= U2 costs three max operations and an FMA.
//             At the end of an item the row's U is lowered to what the item
//             found (atomic minimum), for the items that start later.
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
constexpr int kStages = 6;                    // column-tile ring
constexpr int kThreads = 512;                 // 16 warps (roles in tc_collect)
constexpr int kTmemCols = 512;                // four 128-column FP32 accumulators
constexpr int kCandCap = 512;                 // candidate list per row
constexpr int kItemTiles = 32;                // column tiles per work item
constexpr int kPlanRec = 32;                  // columns of the nearest tile recorded per row in the plan
constexpr int kCandBuf = 16;                  // candidates buffered per row and epilogue warpgroup in the collect kernel
constexpr float kC = 0.008f;                  // c' of the bounds
constexpr float kSqrtC = 0.08944271909999159f;
constexpr float kUpper = 4.1f * kC;
constexpr float kEfp = 6e-5f;
// margins of the tile test: computed distances and radii are within 3e-5
// relative of the exact ones (33 FP32 terms), squares within 1e-4
constexpr float kTolR = 3e-5f;
constexpr float kTolD = 1e-4f;
// bound on the rounding error of |x|^2 + |c|^2 - 2 x.c in FP32, relative to
// (|x| + |c|)^2: 40 u with u = 2^-24, rounded up
constexpr float kDotErr = 3e-6f;

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
// locality order: a principal-direction tree
// ---------------------------------------------------------------------------

constexpr int kTreeSample = 256;  // rows sampled per node for its direction
constexpr int kTreeIters = 2;     // power iterations
constexpr int kTreeThreads = 256;
constexpr int kDirStride = 68;    // floats per node: centre (33), direction (33), projection range (2)
constexpr size_t kTreeSmem = sizeof(float) * kTreeSample * KMX_DESC_DIM;
// Rows of a node tree_local splits in one CTA.  Its gathers of the node's
// descriptor rows run on one SM, so a larger node is faster on the global
// kernels, which spread a level over the whole GPU (on the 2M-point indoor
// pair, 16384 beat 8192, 4096 and 65536).
constexpr int kLocalRows = 16384;
constexpr int kFinishLevels = 4;                         // levels below a node of 16 tiles
constexpr int kFinishRows = kTM << kFinishLevels;        // 2048
constexpr int kFinishSample = 256;                       // rows sampled per node below level0 (at most 2048 rows)
// sampled rows, entries, partition buffer, 16-bit keys
constexpr size_t kFinishSmem = sizeof(float) * kFinishSample * KMX_DESC_DIM + sizeof(int32_t) * 2 * kFinishRows +
                               sizeof(uint16_t) * kFinishRows;

// Rows of the left child of a node of `len` rows: a whole number of tiles,
// ceil(len / 256) * 128; a node of at most 128 rows is a leaf (its left
// child is itself, its right child empty).
__host__ __device__ __forceinline__ int64_t tree_left(int64_t len)
{
    return len > kTM ? (len + 2 * kTM - 1) / (2 * kTM) * kTM : len;
}

// Levels until every node is a leaf.
int tree_levels(int64_t n)
{
    const int64_t tiles = (n + kTM - 1) / kTM;
    int l = 0;
    while ((int64_t{1} << l) < tiles) ++l;
    return l;
}

// (start, len) of node k of level l over a side of n rows.
__device__ __forceinline__ void tree_node(int64_t n, int l, int64_t k, int64_t& start, int64_t& len)
{
    start = 0;
    len = n;
    for (int b = l - 1; b >= 0; --b) {
        const int64_t h = tree_left(len);
        if ((k >> b) & 1) {
            start += h;
            len -= h;
        } else {
            len = h;
        }
    }
}

// The level-l node holding sorted position pos (< n), with its (start, len).
__device__ __forceinline__ int64_t tree_node_of(int64_t n, int l, int64_t pos, int64_t& start, int64_t& len)
{
    start = 0;
    len = n;
    int64_t k = 0;
    for (int b = 0; b < l; ++b) {
        const int64_t h = tree_left(len);
        if (pos - start >= h) {
            k = 2 * k + 1;
            start += h;
            len -= h;
        } else {
            k = 2 * k;
            len = h;
        }
    }
    return k;
}

// Largest node of level l over a side of n rows (the leftmost: a left
// child is never smaller than its sibling).
__host__ __device__ __forceinline__ int64_t level_max(int64_t n, int l)
{
    for (int b = 0; b < l; ++b) n = tree_left(n);
    return n;
}

// The tree works on both clouds' rows packed together: entry e < np is
// source row e, entry np + i target row i (np, nq the device counts).  They
// start as the identity, and *n2 = np + nq.
__global__ void __launch_bounds__(256) tree_init(int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                                                 const int64_t* d_nq, int32_t* __restrict__ vals,
                                                 int64_t* __restrict__ n2)
{
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *n2 = np + nq;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < np + nq; e += (int64_t)gridDim.x * 256)
        vals[e] = (int32_t)(e < np ? e : e - np);
}

// The sorted rows into the layout the later stages read: source rows at
// [0, np), target rows at [np_cap, np_cap + nq).
__global__ void __launch_bounds__(256) tree_out(int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                                                const int64_t* d_nq, const int32_t* __restrict__ vals,
                                                int32_t* __restrict__ perm)
{
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < np + nq; e += (int64_t)gridDim.x * 256)
        perm[e < np ? e : np_cap + (e - np)] = vals[e];
}

// (x - c) . v over the 33 values of descriptor row x (16-byte aligned, read
// as eight float4 and one float).
__device__ __forceinline__ float project(const float* __restrict__ x, const float* c, const float* v)
{
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4 r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = __ldg(x4 + q);
    float p = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        p = fmaf(r[q].x - c[4 * q], v[4 * q], p);
        p = fmaf(r[q].y - c[4 * q + 1], v[4 * q + 1], p);
        p = fmaf(r[q].z - c[4 * q + 2], v[4 * q + 2], p);
        p = fmaf(r[q].w - c[4 * q + 3], v[4 * q + 3], p);
    }
    return fmaf(__ldg(x + 32) - c[32], v[32], p);
}

// Partial sums per column in the sample reductions of a CTA of NT threads
// (7 x 33 <= 256, 31 x 33 <= 1024).
template <int NT>
__host__ __device__ constexpr int col_split()
{
    return NT / KMX_DESC_DIM;
}

// Shared memory of one node's direction (besides the sampled rows), for a
// CTA of NT threads sampling up to S rows.
template <int NT, int S = kTreeSample>
struct DirSmem {
    float part[col_split<NT>()][KMX_DESC_DIM];
    float cvec[KMX_DESC_DIM], vvec[KMX_DESC_DIM], uvec[KMX_DESC_DIM];
    float w[S];
    float redf[2][NT / 32];
    int redi[NT / 32];
    float scale;
    int far;
};

// Centre (D.cvec) and principal direction (D.vvec) of a node of `len` rows
// whose rows are X[perm[0 .. len)], from up to S of them (evenly spaced in
// the current order) held centred in xs; lo / hi (thread 0) get the range of
// the sample's projections.  Every thread of the CTA (NT threads) calls it.
template <int NT, int S>
__device__ void node_direction(const float* __restrict__ X, const int32_t* perm, int64_t len,
                               float (*xs)[KMX_DESC_DIM], DirSmem<NT, S>& D, float& lo, float& hi)
{
    constexpr int kColSplit = col_split<NT>();
    const int m = (int)min(len, (int64_t)S);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cpart = tid / KMX_DESC_DIM, ch = tid - cpart * KMX_DESC_DIM;
    __syncthreads();  // the caller's earlier use of xs and D is over
    // one sampled row per thread: its index, then the row as nine
    // independent loads (all in flight at once)
    for (int i = tid; i < m; i += NT) {
        const float* x = X + (int64_t)perm[(int64_t)i * len / m] * KMX_DESC_STRIDE;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldg(x4 + q);
        const float last = __ldg(x + 32);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xs[i][4 * q] = v[q].x;
            xs[i][4 * q + 1] = v[q].y;
            xs[i][4 * q + 2] = v[q].z;
            xs[i][4 * q + 3] = v[q].w;
        }
        xs[i][32] = last;
    }
    __syncthreads();
    // centre
    if (cpart < kColSplit) {
        float acc = 0.f;
        for (int i = cpart; i < m; i += kColSplit) acc += xs[i][ch];
        D.part[cpart][ch] = acc;
    }
    __syncthreads();
    if (tid < KMX_DESC_DIM) {
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < kColSplit; ++c) acc += D.part[c][tid];
        D.cvec[tid] = acc / (float)m;
    }
    __syncthreads();
    for (int idx = tid; idx < m * KMX_DESC_DIM; idx += NT) {
        const int i = idx / KMX_DESC_DIM, h = idx - i * KMX_DESC_DIM;
        xs[i][h] -= D.cvec[h];
    }
    __syncthreads();
    // start from the sampled row farthest from the centre (lowest index on ties)
    {
        float best = -1.f;
        int bi = 0;
        for (int i = tid; i < m; i += NT) {
            float acc = 0.f;
#pragma unroll
            for (int h = 0; h < KMX_DESC_DIM; ++h) acc = fmaf(xs[i][h], xs[i][h], acc);
            if (acc > best) {
                best = acc;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            D.redf[0][warp] = best;
            D.redi[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            float b = D.redf[0][0];
            int i0 = D.redi[0];
            for (int q = 1; q < NT / 32; ++q)
                if (D.redf[0][q] > b || (D.redf[0][q] == b && D.redi[q] < i0)) {
                    b = D.redf[0][q];
                    i0 = D.redi[q];
                }
            D.far = i0;
        }
        __syncthreads();
        if (tid < KMX_DESC_DIM) D.uvec[tid] = xs[D.far][tid];
    }
    // power iterations v <- S^T S v / |S^T S v| on the centred sample S
    for (int it = 0; it <= kTreeIters; ++it) {
        __syncthreads();
        if (warp == 0) {  // |u|^2 across the warp (lane 0 adds the 33rd value)
            const float a = D.uvec[lane];
            float nn = a * a;
            if (lane == 0) nn = fmaf(D.uvec[32], D.uvec[32], nn);
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
            if (lane == 0) D.scale = nn > 0.f ? rsqrtf(nn) : 0.f;
        }
        __syncthreads();
        if (tid < KMX_DESC_DIM) D.vvec[tid] = D.scale > 0.f ? D.uvec[tid] * D.scale : (tid == 0 ? 1.f : 0.f);
        __syncthreads();
        if (it == kTreeIters) break;
        for (int i = tid; i < m; i += NT) {
            float acc = 0.f;
#pragma unroll
            for (int h = 0; h < KMX_DESC_DIM; ++h) acc = fmaf(xs[i][h], D.vvec[h], acc);
            D.w[i] = acc;
        }
        __syncthreads();
        if (cpart < kColSplit) {
            float acc = 0.f;
            for (int i = cpart; i < m; i += kColSplit) acc = fmaf(D.w[i], xs[i][ch], acc);
            D.part[cpart][ch] = acc;
        }
        __syncthreads();
        if (tid < KMX_DESC_DIM) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < kColSplit; ++c) acc += D.part[c][tid];
            D.uvec[tid] = acc;
        }
    }
    // range of the sample's projections
    lo = INFINITY;
    hi = -INFINITY;
    for (int i = tid; i < m; i += NT) {
        float acc = 0.f;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) acc = fmaf(xs[i][h], D.vvec[h], acc);
        lo = fminf(lo, acc);
        hi = fmaxf(hi, acc);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        D.redf[0][warp] = lo;
        D.redf[1][warp] = hi;
    }
    __syncthreads();
    if (tid == 0)
        for (int q = 1; q < NT / 32; ++q) {
            lo = fminf(lo, D.redf[0][q]);
            hi = fmaxf(hi, D.redf[1][q]);
        }
}

// One CTA per (node of this level, side): the node's centre and principal
// direction and the range of its sample's projections.  Leaves do nothing.
__global__ void __launch_bounds__(kTreeThreads) tree_dir(const float* __restrict__ P, int64_t np_cap,
                                                         const int64_t* d_np, const float* __restrict__ Q,
                                                         int64_t nq_cap, const int64_t* d_nq,
                                                         const int32_t* __restrict__ vals, int level,
                                                         float* __restrict__ dirs)
{
    extern __shared__ float tree_smem[];
    float(*xs)[KMX_DESC_DIM] = reinterpret_cast<float(*)[KMX_DESC_DIM]>(tree_smem);
    __shared__ DirSmem<kTreeThreads> D;
    const int side = blockIdx.y;
    const int64_t k = blockIdx.x;
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    if (level_max(np > nq ? np : nq, level) <= kLocalRows) return;  // tree_local takes this level
    const int64_t n = side ? nq : np;
    int64_t start, len;
    tree_node(n, level, k, start, len);
    if (len <= kTM) return;
    float lo, hi;
    node_direction(side ? Q : P, vals + (side ? kmx_count(d_np, np_cap) : 0) + start, len, xs, D, lo, hi);
    float* d = dirs + (((int64_t)side << level) + k) * kDirStride;
    const int tid = threadIdx.x;
    if (tid < KMX_DESC_DIM) {
        d[tid] = D.cvec[tid];
        d[KMX_DESC_DIM + tid] = D.vvec[tid];
    }
    if (tid == 0) {
        d[2 * KMX_DESC_DIM] = lo;
        d[2 * KMX_DESC_DIM + 1] = hi;
    }
}

// One tree level for nodes that fit in shared memory (at most kLocalRows
// rows), one CTA of NT threads per (node, side), in one launch instead of
// the direction, key and radix-sort launches of a global level.  The split
// is the global levels' split: the first tree_left(len) rows in the order of
// (16-bit key, position), the key being the projection on the node's
// direction quantised over the sample's range.  That set is found without a
// sort: two 256-bin histograms give the key T of the split row and how many
// rows with key T go left; then a stable partition writes the left rows,
// then the right rows, each in their current order, from src to dst.  Leaves
// are copied.  A level that the global kernels ordered (some node of the
// level larger than kLocalRows on the device) is left alone: their radix
// sort wrote dst.
constexpr size_t kLocalSmemBase = kTreeSmem;  // the sampled rows; the 16-bit keys follow
constexpr int kLocalWideCtas = 304;           // from this many CTAs per level, CTAs of 256 threads (4 per SM)

size_t local_smem_bytes(int64_t max_rows)
{
    return kLocalSmemBase + sizeof(uint16_t) * (size_t)((max_rows + 7) / 8 * 8);
}

// Smallest bin b with before + (hist[0] + ... + hist[b]) >= target, and the
// count before it (bins in order), by warp 0 of the CTA; the result in
// *bin / *below.
__device__ __forceinline__ void select_bin(const int* hist, int before, int target, int* bin, int* below)
{
    const int lane = threadIdx.x & 31;
    int c[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        c[q] = hist[lane * 8 + q];
        sum += c[q];
    }
    int incl = sum;  // inclusive prefix over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int run = before + incl - sum;
    int found = -1, fb = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (found < 0 && run + c[q] >= target) {
            found = lane * 8 + q;
            fb = run;
        }
        run += c[q];
    }
    const unsigned hit = __ballot_sync(0xffffffffu, found >= 0);
    const int src = hit ? __ffs(hit) - 1 : 31;
    found = __shfl_sync(0xffffffffu, found, src);
    fb = __shfl_sync(0xffffffffu, fb, src);
    if (lane == 0) {
        *bin = found < 0 ? 255 : found;
        *below = fb;
    }
}

// Rows [0, len) of a node with 16-bit keys key[0 .. len) (written before
// the call): the first h rows in the order of (key, position) go left.  Two
// 256-bin histograms give the key T of the split row and how many rows with
// key T go left; then a stable partition calls put(pos, get(i)) for every
// row i, left rows at positions 0 .. h - 1 and right rows at h .. len - 1,
// each in their current order (get(i) is issued before the round's barrier,
// so that a global load overlaps it).  All NT (>= 256) threads call it;
// hist[256], sel[4] and wsum[NT / 32] are shared scratch.  Ends after a
// barrier.
template <int NT, typename Get, typename Put>
__device__ void split_at(const uint16_t* key, int len, int h, int* hist, int* sel, int* wsum, unsigned int* err,
                         Get get, Put put)
{
    static_assert(NT >= 256, "one thread per bin clears the histograms");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();  // the keys are written
    if (tid < 256) hist[tid] = 0;
    __syncthreads();
    // one shared atomic per distinct bin and warp: keys cluster, and equal
    // bins within a warp would otherwise serialise
    for (int base = 0; base < len; base += NT) {
        const int i = base + tid;
        const int bin = i < len ? (int)(key[i] >> 8) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
    }
    __syncthreads();
    if (warp == 0) select_bin(hist, 0, h, &sel[0], &sel[1]);
    __syncthreads();
    const int b1 = sel[0], below1 = sel[1];
    if (tid < 256) hist[tid] = 0;
    __syncthreads();
    for (int base = 0; base < len; base += NT) {
        const int i = base + tid;
        int bin = -1;
        if (i < len) {
            const int k = key[i];
            if ((k >> 8) == b1) bin = k & 0xff;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
    }
    __syncthreads();
    if (warp == 0) {
        int b2, below2;
        select_bin(hist, below1, h, &b2, &below2);
        if (lane == 0) {
            sel[2] = (b1 << 8) | b2;
            sel[3] = h - below2;
        }
    }
    __syncthreads();
    const int T = sel[2], need = sel[3];
    // stable partition in rounds of NT rows: per round, the counts of
    // key < T (low half of a word) and key == T (high half) before each row
    int run_l = 0, run_e = 0;  // over earlier rounds (uniform)
    for (int base = 0; base < len; base += NT) {
        const int i = base + tid;
        const bool valid = i < len;
        const int32_t v = valid ? get(i) : 0;
        const int k = valid ? (int)key[i] : 0x10000;
        const bool isl = valid && k < T, ise = valid && k == T;
        const unsigned bl = __ballot_sync(0xffffffffu, isl), be = __ballot_sync(0xffffffffu, ise);
        const unsigned lt = (1u << lane) - 1u;
        if (lane == 0) wsum[warp] = __popc(bl) | (__popc(be) << 16);
        __syncthreads();
        int pre = 0, tot = 0;
#pragma unroll 8
        for (int w = 0; w < NT / 32; ++w) {
            const int v = wsum[w];
            pre += w < warp ? v : 0;
            tot += v;
        }
        const int nl = run_l + (pre & 0xffff) + __popc(bl & lt);  // key < T before row i
        const int ne = run_e + (pre >> 16) + __popc(be & lt);     // key == T before row i
        if (valid) {
            const int left_before = nl + min(ne, need);
            const bool left = isl || (ise && ne < need);
            const int pos = left ? left_before : h + (i - left_before);
            if (pos < len) {  // always (the counts add up to h left rows); checked, not assumed
                put(pos, v);
            } else {
                kmx_raise(err, KMX_DERR_CAPACITY);
            }
        }
        run_l += tot & 0xffff;
        run_e += tot >> 16;
        __syncthreads();  // wsum is rewritten by the next round
    }
}

template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) tree_local(const float* __restrict__ P, int64_t np_cap,
                                                           const int64_t* d_np, const float* __restrict__ Q,
                                                           int64_t nq_cap, const int64_t* d_nq,
                                                           const int32_t* __restrict__ src,
                                                           int32_t* __restrict__ dst, int level, unsigned int* err)
{
    constexpr int kWarpsL = NT / 32;
    extern __shared__ float tree_smem[];
    float(*xs)[KMX_DESC_DIM] = reinterpret_cast<float(*)[KMX_DESC_DIM]>(tree_smem);
    uint16_t* key = reinterpret_cast<uint16_t*>(tree_smem + kTreeSample * KMX_DESC_DIM);
    __shared__ DirSmem<NT> D;
    __shared__ int hist[256];
    __shared__ int wsum[kWarpsL];
    __shared__ int sel[4];   // B1, below B1, T, rows of key T that go left
    __shared__ float range[2];
    const int side = blockIdx.y;
    const int tid = threadIdx.x;
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    const int64_t n = side ? nq : np;
    int64_t start, len64;
    tree_node(n, level, blockIdx.x, start, len64);
    const int32_t* gs = src + (side ? np : 0) + start;
    int32_t* gd = dst + (side ? np : 0) + start;
    // a level the global kernels ordered (their sort wrote dst) needs nothing
    if (level_max(np > nq ? np : nq, level) > kLocalRows) return;
    if (len64 <= kTM || len64 > kLocalRows) {  // a leaf (a larger node cannot occur): only the copy
        if (len64 > kLocalRows && tid == 0) kmx_raise(err, KMX_DERR_CAPACITY);
        for (int64_t i = tid; i < len64; i += NT) gd[i] = gs[i];
        return;
    }
    const int len = (int)len64;
    const int h = (int)tree_left(len64);  // 0 < h < len
    const float* X = side ? Q : P;
    float lo, hi;
    node_direction(X, gs, len64, xs, D, lo, hi);
    if (tid == 0) {
        range[0] = lo;
        range[1] = hi;
    }
    __syncthreads();
    lo = range[0];
    hi = range[1];
    const float qs = hi > lo ? 65535.f / (hi - lo) : 0.f;
    int32_t g = tid < len ? gs[tid] : 0;
    for (int i = tid; i < len; i += NT) {
        const int32_t gn = i + NT < len ? gs[i + NT] : 0;  // the next row's index, loaded during this row
        const float p = project(X + (int64_t)g * KMX_DESC_STRIDE, D.cvec, D.vvec);
        key[i] = (uint16_t)fminf(fmaxf((p - lo) * qs, 0.f), 65535.f);  // NaN -> 0
        g = gn;
    }
    split_at<NT>(key, len, h, hist, sel, wsum, err, [&](int i) { return gs[i]; },
                 [&](int pos, int32_t v) { gd[pos] = v; });
}

// The last levels of the tree, below `level0` (whose nodes hold at most
// kFinishRows rows): one CTA per (level-0 node, side) splits its subtree
// level by level in shared memory.  Per node: its direction (from up to
// kFinishSample rows), 16-bit keys of all its rows and split_at, as
// tree_local does; the next level splits each half again.  The entries are
// read from src and written to vals (src may be vals).
__global__ void __launch_bounds__(kTreeThreads) tree_finish(const float* __restrict__ P, int64_t np_cap,
                                                            const int64_t* d_np, const float* __restrict__ Q,
                                                            int64_t nq_cap, const int64_t* d_nq,
                                                            const int32_t* src, int32_t* vals, int level0,
                                                            int levels, unsigned int* err)
{
    extern __shared__ float tree_smem[];
    float(*xs)[KMX_DESC_DIM] = reinterpret_cast<float(*)[KMX_DESC_DIM]>(tree_smem);
    int32_t* perm = reinterpret_cast<int32_t*>(tree_smem + kFinishSample * KMX_DESC_DIM);  // [kFinishRows]
    int32_t* tmp = perm + kFinishRows;                                                    // [kFinishRows]
    uint16_t* key = reinterpret_cast<uint16_t*>(tmp + kFinishRows);                       // [kFinishRows]
    __shared__ DirSmem<kTreeThreads, kFinishSample> D;
    __shared__ int hist[256];
    __shared__ int wsum[kTreeThreads / 32];
    __shared__ int sel[4];
    __shared__ float range[2];
    const int side = blockIdx.y;
    const int tid = threadIdx.x;
    const int64_t np = kmx_count(d_np, np_cap);
    const int64_t n = side ? kmx_count(d_nq, nq_cap) : np;
    int64_t start, len;
    tree_node(n, level0, blockIdx.x, start, len);
    const float* X = side ? Q : P;
    const int32_t* gs = src + (side ? np : 0) + start;
    int32_t* gv = vals + (side ? np : 0) + start;
    if (len <= kTM || len > kFinishRows) {  // a leaf (a larger node cannot occur): only the copy
        if (len > kFinishRows && tid == 0) kmx_raise(err, KMX_DERR_CAPACITY);
        if (gs != gv)
            for (int64_t i = tid; i < len; i += kTreeThreads) gv[i] = gs[i];
        return;
    }
    for (int i = tid; i < len; i += kTreeThreads) perm[i] = gs[i];
    for (int l = level0; l < levels; ++l) {
        const int sub = l - level0;
        for (int c = 0; c < (1 << sub); ++c) {
            // the sub-node's range within the CTA's rows
            int64_t cs = 0, cl = len;
            for (int b = sub - 1; b >= 0; --b) {
                const int64_t h = tree_left(cl);
                if ((c >> b) & 1) {
                    cs += h;
                    cl -= h;
                } else {
                    cl = h;
                }
            }
            if (cl <= kTM) continue;
            float lo, hi;
            node_direction(X, perm + cs, cl, xs, D, lo, hi);
            if (tid == 0) {
                range[0] = lo;
                range[1] = hi;
            }
            __syncthreads();
            lo = range[0];
            hi = range[1];
            const float qs = hi > lo ? 65535.f / (hi - lo) : 0.f;
            for (int i = tid; i < cl; i += kTreeThreads) {
                const float p = project(X + (int64_t)perm[cs + i] * KMX_DESC_STRIDE, D.cvec, D.vvec);
                key[i] = (uint16_t)fminf(fmaxf((p - lo) * qs, 0.f), 65535.f);  // NaN -> 0
            }
            split_at<kTreeThreads>(key, (int)cl, (int)tree_left(cl), hist, sel, wsum, err,
                                   [&](int i) { return perm[cs + i]; }, [&](int pos, int32_t v) { tmp[pos] = v; });
            for (int i = tid; i < cl; i += kTreeThreads) perm[cs + i] = tmp[i];
            // (the next node_direction starts with a barrier)
        }
    }
    __syncthreads();
    for (int i = tid; i < len; i += kTreeThreads) gv[i] = perm[i];
}

// Sort key of every packed entry for this level: side (top bit), node index
// (level bits), then the row's projection on its node's direction,
// quantised over the sample's range (0 in a leaf).  *n_sort gets the count
// the radix sort takes (0 when tree_local takes the level).
__global__ void __launch_bounds__(256) tree_key(const float* __restrict__ P, int64_t np_cap, const int64_t* d_np,
                                                const float* __restrict__ Q, int64_t nq_cap, const int64_t* d_nq,
                                                const int32_t* __restrict__ vals, int level, int key_bits,
                                                const float* __restrict__ dirs, uint32_t* __restrict__ keys,
                                                int64_t* __restrict__ n_sort)
{
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    // the entries this level's radix sort orders: all of them, or none when
    // every node fits tree_local
    const bool global = level_max(np > nq ? np : nq, level) > kLocalRows;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_sort = global ? np + nq : 0;
    if (!global) return;
    const int pbits = key_bits - 1 - level;
    const int qbits = pbits < 22 ? pbits : 22;
    const float qmax = (float)((1u << qbits) - 1u);
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < np + nq; e += (int64_t)gridDim.x * 256) {
        const int side = e >= np;
        const int64_t pos = side ? e - np : e;
        int64_t start, len;
        const int64_t k = tree_node_of(side ? nq : np, level, pos, start, len);
        uint32_t q = 0;
        if (len > kTM) {
            const float* d = dirs + (((int64_t)side << level) + k) * kDirStride;
            const float* x = (side ? Q : P) + (int64_t)vals[e] * KMX_DESC_STRIDE;
            const float p = project(x, d, d + KMX_DESC_DIM);
            const float lo = d[2 * KMX_DESC_DIM], hi = d[2 * KMX_DESC_DIM + 1];
            const float t = hi > lo ? (p - lo) / (hi - lo) * qmax : 0.f;
            q = (uint32_t)fminf(fmaxf(t, 0.f), qmax) << (pbits - qbits);
        }
        keys[e] = ((uint32_t)side << (key_bits - 1)) | ((uint32_t)k << pbits) | q;
    }
}

// ---------------------------------------------------------------------------
// pack: one CTA of 128 threads per column tile of one cloud
// ---------------------------------------------------------------------------

// Rows of the tile are sorted positions [128 t, 128 t + 128) of the cloud;
// perm maps a sorted position to the descriptor row.  Writes the packed
// column tile, and to centers[t] the centre (33 values) and the largest
// |y - c|^2 of the tile (at 33).  A non-finite descriptor value raises
// KMX_DERR_RANGE.
__global__ void __launch_bounds__(kTN) tc_pack(const float* __restrict__ desc, const int32_t* __restrict__ perm,
                                               int64_t n_cap, const int64_t* d_n, uint8_t* __restrict__ out,
                                               float* __restrict__ centers, unsigned int* err)
{
    __shared__ float rows_s[kTN][KMX_DESC_DIM + 1];
    __shared__ float cen[kCenterStride];
    __shared__ unsigned int bmax2;
    const int64_t n = kmx_count(d_n, n_cap);
    const int tid = threadIdx.x;
    // the tiles below the count (tile 0 always), blockIdx.x, blockIdx.x +
    // gridDim.x, ...; tiles past the count are never read
    const int64_t tiles = n > 0 ? (n + kTN - 1) / kTN : 1;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t r = t * kTN + tid;
        const bool valid = r < n;
        float y[KMX_DESC_DIM];
        if (valid) {
            const float* row = desc + (int64_t)perm[r] * KMX_DESC_STRIDE;
    #pragma unroll
            for (int h = 0; h < KMX_DESC_DIM; ++h) y[h] = __ldg(row + h);
            bool bad = false;
    #pragma unroll
            for (int h = 0; h < KMX_DESC_DIM; ++h) bad |= !isfinite(y[h]);
            if (bad) kmx_raise(err, KMX_DERR_RANGE);
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
        if (tid == 0) centers[t * kCenterStride + KMX_DESC_DIM] = __uint_as_float(bmax2);
        // the largest |b| of each group of 8 rows (lanes 8k .. 8k + 7 of a warp)
        float gb = valid ? beta : 0.f;
    #pragma unroll
        for (int o = 4; o >= 1; o >>= 1) gb = fmaxf(gb, __shfl_xor_sync(0xffffffffu, gb, o));
        if ((tid & 7) == 0) reinterpret_cast<float*>(tile + kHdrGBeta)[tid >> 3] = gb;
        __syncthreads();  // the shared rows, centre and maximum are rewritten by the next tile
    }
}

// ---------------------------------------------------------------------------
// plan: first candidates, first bounds and the column tiles each row tile needs
// ---------------------------------------------------------------------------

// Squared distance between a row tile's centre cR (shared, 16-byte aligned,
// 33 values) and the centre of tile u (a 36-float row of centres, 16-byte
// aligned): two interleaved chains of paired FP32 terms, then their sum.  It
// only decides which tiles are tested, within the tile test's margins.
__device__ __forceinline__ float centre_dist2(const float* __restrict__ cR, const float* __restrict__ c)
{
    const float4* c4 = reinterpret_cast<const float4*>(c);
    const float4* r4 = reinterpret_cast<const float4*>(cR);
    float2 d = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 v = __ldg(c4 + q), r = r4[q];
        float2 e = __fadd2_rn(make_float2(r.x, r.y), make_float2(-v.x, -v.y));
        d = __ffma2_rn(e, e, d);
        e = __fadd2_rn(make_float2(r.z, r.w), make_float2(-v.z, -v.w));
        d = __ffma2_rn(e, e, d);
    }
    const float e = cR[32] - __ldg(c + 32);
    return fmaf(e, e, d.x + d.y);
}

// False only when no column of a tile with centre distance `dist` and radius
// `rad` can lie within squared distance u2: for every column y,
// |x - y| >= |x - c| - |y - c| >= dist - rad (margins for FP32 rounding).
__device__ __forceinline__ bool tile_may_hold(float dist, float rad, float u2)
{
    const float g = dist * (1.f - kTolR) - rad * (1.f + kTolR);
    return !(g > 0.f && g * g * (1.f - kTolD) > u2);
}

// One CTA of 128 threads (thread = row) per row tile rt of X, with cenX and
// cenY the centres and squared radii of both clouds' tiles (tc_pack).
//   1. the column tile cs with the centre nearest to the row tile's centre
//      (lowest index on ties);
//   2. each row's exact FP32 distances to the columns of cs (the exact
//      path's arithmetic): its second-smallest d2 over distinct columns is
//      an upper bound of the row's d(2); the columns with distance <= d2
//      are its first candidates (cnt[row] = their number), and ub[row] = d2;
//   3. every other column tile that tile_may_hold for some row of the tile
//      (first for the whole tile: centre distance minus both radii against
//      the largest d2, then row by row), in increasing order, into
//      need[rt * need_stride ...]; nneed[rt] = their number, and the list is
//      cut into items (rt, first) of kItemTiles tiles appended to `items`.
__device__ __forceinline__ void plan_tile(const float* __restrict__ X, const int32_t* __restrict__ permX,
                                          int64_t nx_cap, const int64_t* d_nx, const float* __restrict__ cenX,
                                          const float* __restrict__ Y, const int32_t* __restrict__ permY,
                                          int64_t ny_cap, const int64_t* d_ny, const float* __restrict__ cenY,
                                          int32_t* __restrict__ cand, int32_t* __restrict__ cnt,
                                          float* __restrict__ ub, int32_t* __restrict__ need, int64_t need_stride,
                                          int32_t* __restrict__ nneed, int2* __restrict__ items,
                                          int* __restrict__ n_items, const int64_t rt)
{
    // the nearest tile's rows (negated, zero-padded to 36) in the exact pass,
    // then the surviving tiles (centre, radius at [33]) in the tile lists
    __shared__ __align__(16) float ysc[kTN][kCenterStride];
    float(*ys)[kCenterStride] = ysc;
    float(*sc)[kCenterStride] = ysc;
    __shared__ int32_t sid[kTN];
    __shared__ uint8_t rec[kPlanRec][kTM];  // per row: columns recorded in the first pass
    __shared__ __align__(16) float cR[kCenterStride];
    __shared__ unsigned needbits[kTN / 32];
    __shared__ int wcnt[kTN / 32];
    __shared__ float redf[kTN / 32];
    __shared__ int redi[kTN / 32];
    __shared__ int s_cs, s_total;
    __shared__ float s_maxu;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t rows = kmx_count(d_nx, nx_cap), cols = kmx_count(d_ny, ny_cap);
    if (rt * kTM >= rows || cols <= 0) return;
    const int64_t n_ct = (cols + kTN - 1) / kTN;
    const int64_t xrow = rt * kTM + tid;
    const bool valid = xrow < rows;
    float x[KMX_DESC_DIM];
    {
        const float* xr = valid ? X + (int64_t)permX[xrow] * KMX_DESC_STRIDE : nullptr;
#pragma unroll
        for (int h = 0; h < KMX_DESC_DIM; ++h) x[h] = valid ? __ldg(xr + h) : 0.f;
    }
    if (tid < KMX_DESC_DIM) cR[tid] = cenX[rt * kCenterStride + tid];
    const float rR = sqrtf(cenX[rt * kCenterStride + KMX_DESC_DIM]);
    __syncthreads();
    // 1. nearest column tile
    {
        float best = INFINITY;
        int bi = 0x7fffffff;
        for (int64_t u = tid; u < n_ct; u += kTM) {
            const float d = centre_dist2(cR, cenY + u * kCenterStride);
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
        if (lane == 0) {
            redf[warp] = best;
            redi[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            float b = redf[0];
            int i0 = redi[0];
            for (int q = 1; q < kTN / 32; ++q)
                if (redf[q] < b || (redf[q] == b && redi[q] < i0)) {
                    b = redf[q];
                    i0 = redi[q];
                }
            s_cs = i0 == 0x7fffffff ? 0 : i0;
            s_total = 0;
        }
        __syncthreads();
    }
    const int64_t cs = s_cs;
    {
        const int64_t yp = cs * kTN + tid;
        const bool yv = yp < cols;
        const float* yr = yv ? Y + (int64_t)permY[yp] * KMX_DESC_STRIDE : nullptr;
#pragma unroll
        for (int h = 0; h < kCenterStride; ++h) ys[tid][h] = (yv && h < KMX_DESC_DIM) ? -__ldg(yr + h) : 0.f;
    }
    __syncthreads();
    // 2. exact distances to the nearest tile.  One pass finds d1 <= d2 and
    // records the columns whose distance was at most the running second-
    // smallest (a superset of those with distance <= d2: the running value
    // never falls below the final one); only the recorded columns are
    // compared again (with the same arithmetic, so the same values) and those
    // within d2 become candidates.  More than kPlanRec records: a second
    // pass over the whole tile.
    const int ncol = (int)min((int64_t)kTN, cols - cs * kTN);
    float d2 = INFINITY;
    if (valid) {
        // the exact path's arithmetic: x + (-y) per dimension, one fused
        // multiply-add per term in dimension order
        auto dist = [&](int j) -> float {
            const float4* y4 = reinterpret_cast<const float4*>(ys[j]);
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 yv4 = y4[c];
                float e = __fadd_rn(x[4 * c], yv4.x);
                acc = fmaf(e, e, acc);
                e = __fadd_rn(x[4 * c + 1], yv4.y);
                acc = fmaf(e, e, acc);
                e = __fadd_rn(x[4 * c + 2], yv4.z);
                acc = fmaf(e, e, acc);
                e = __fadd_rn(x[4 * c + 3], yv4.w);
                acc = fmaf(e, e, acc);
            }
            const float e = __fadd_rn(x[32], ys[j][32]);
            return fmaf(e, e, acc);
        };
        // the same for columns j and j + 1 at once, one in each half of the
        // paired FP32 instructions (each half the arithmetic above)
        auto dist_pair = [&](int j) -> float2 {
            const float4* ya = reinterpret_cast<const float4*>(ys[j]);
            const float4* yb = reinterpret_cast<const float4*>(ys[j + 1]);
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 va = ya[c], vb = yb[c];
                float2 e = __fadd2_rn(make_float2(x[4 * c], x[4 * c]), make_float2(va.x, vb.x));
                acc = __ffma2_rn(e, e, acc);
                e = __fadd2_rn(make_float2(x[4 * c + 1], x[4 * c + 1]), make_float2(va.y, vb.y));
                acc = __ffma2_rn(e, e, acc);
                e = __fadd2_rn(make_float2(x[4 * c + 2], x[4 * c + 2]), make_float2(va.z, vb.z));
                acc = __ffma2_rn(e, e, acc);
                e = __fadd2_rn(make_float2(x[4 * c + 3], x[4 * c + 3]), make_float2(va.w, vb.w));
                acc = __ffma2_rn(e, e, acc);
            }
            const float2 e = __fadd2_rn(make_float2(x[32], x[32]), make_float2(ys[j][32], ys[j + 1][32]));
            return __ffma2_rn(e, e, acc);
        };
        float d1 = INFINITY;
        int nrec = 0;
        auto take = [&](float acc, int j) {
            if (acc < d1) {
                d2 = d1;
                d1 = acc;
            } else if (acc < d2) {
                d2 = acc;
            }
            if (acc <= d2) {
                if (nrec < kPlanRec) rec[nrec][tid] = (uint8_t)j;
                ++nrec;
            }
        };
        int j = 0;
        for (; j + 1 < ncol; j += 2) {
            const float2 acc = dist_pair(j);
            take(acc.x, j);
            take(acc.y, j + 1);
        }
        if (j < ncol) take(dist(j), j);
        int k = 0;
        if (nrec <= kPlanRec) {
            for (int i = 0; i < nrec; ++i) {
                const int j = rec[i][tid];
                if (dist(j) <= d2) cand[xrow * kCandCap + k++] = (int32_t)(cs * kTN + j);
            }
        } else {
            for (int j = 0; j < ncol; ++j)
                if (dist(j) <= d2) cand[xrow * kCandCap + k++] = (int32_t)(cs * kTN + j);
        }
        cnt[xrow] = k;
        ub[xrow] = d2;
    }
    {
        float mu = valid ? d2 : 0.f;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        if (lane == 0) redf[warp] = mu;
        __syncthreads();
        if (tid == 0) s_maxu = fmaxf(fmaxf(redf[0], redf[1]), fmaxf(redf[2], redf[3]));
        __syncthreads();
    }
    const float maxu = s_maxu;
    float xx = 0.f;
#pragma unroll
    for (int h = 0; h < KMX_DESC_DIM; ++h) xx = fmaf(x[h], x[h], xx);
    const float xn = sqrtf(xx);
    // 3. the other column tiles, 128 at a time
    for (int64_t base = 0; base < n_ct; base += kTN) {
        const int64_t u = base + tid;
        bool surv = false;
        float ru = 0.f;
        if (u < n_ct && u != cs) {
            const float* c = cenY + u * kCenterStride;
            const float d = centre_dist2(cR, c);
            ru = sqrtf(__ldg(c + KMX_DESC_DIM));
            surv = tile_may_hold(sqrtf(d), rR + ru, maxu);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, surv);
        if (lane == 0) wcnt[warp] = __popc(bal);
        if (tid < kTN / 32) needbits[tid] = 0u;
        __syncthreads();
        int off = 0;
        for (int q = 0; q < warp; ++q) off += wcnt[q];
        const int nsurv = wcnt[0] + wcnt[1] + wcnt[2] + wcnt[3];
        if (surv) {
            const int idx = off + __popc(bal & ((1u << lane) - 1u));
            sid[idx] = (int32_t)u;
            const float4* c4 = reinterpret_cast<const float4*>(cenY + u * kCenterStride);
            float4* s4 = reinterpret_cast<float4*>(sc[idx]);
            float cc = 0.f;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float4 v = __ldg(c4 + q);
                s4[q] = v;
                if (q < 8) {
                    cc = fmaf(v.x, v.x, cc);
                    cc = fmaf(v.y, v.y, cc);
                    cc = fmaf(v.z, v.z, cc);
                    cc = fmaf(v.w, v.w, cc);
                } else {
                    cc = fmaf(v.x, v.x, cc);
                }
            }
            sc[idx][KMX_DESC_DIM] = ru;            // radius
            sc[idx][KMX_DESC_DIM + 1] = cc;        // |c|^2
            sc[idx][KMX_DESC_DIM + 2] = sqrtf(cc); // |c|
        }
        __syncthreads();
        // two surviving tiles per step (independent chains)
        for (int q = 0; q < nsurv; q += 2) {
            const int q1 = min(q + 1, nsurv - 1);
            bool nd0 = false, nd1 = false;
            if (valid) {
                // |x - c|^2 = |x|^2 + |c|^2 - 2 x.c with paired FMAs; its
                // error is below 40 u (|x| + |c|)^2 (u = 2^-24), taken off
                // before the test
                const float4* ca = reinterpret_cast<const float4*>(sc[q]);
                const float4* cb = reinterpret_cast<const float4*>(sc[q1]);
                float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 va = ca[c], vb = cb[c];
                    const float2 x0 = make_float2(x[4 * c], x[4 * c + 1]);
                    const float2 x1 = make_float2(x[4 * c + 2], x[4 * c + 3]);
                    da = __ffma2_rn(x0, make_float2(va.x, va.y), da);
                    db = __ffma2_rn(x0, make_float2(vb.x, vb.y), db);
                    da = __ffma2_rn(x1, make_float2(va.z, va.w), da);
                    db = __ffma2_rn(x1, make_float2(vb.z, vb.w), db);
                }
                const float4 ta = ca[8], tb = cb[8];  // [32], radius, |c|^2, |c|
                const float xca = fmaf(x[32], ta.x, da.x + da.y);
                const float xcb = fmaf(x[32], tb.x, db.x + db.y);
                const float sa_ = xn + ta.w, sb_ = xn + tb.w;
                const float dda = fmaf(-2.f, xca, xx + ta.z) - kDotErr * sa_ * sa_;
                const float ddb = fmaf(-2.f, xcb, xx + tb.z) - kDotErr * sb_ * sb_;
                nd0 = tile_may_hold(sqrtf(fmaxf(dda, 0.f)), ta.y, d2);
                nd1 = q + 1 < nsurv && tile_may_hold(sqrtf(fmaxf(ddb, 0.f)), tb.y, d2);
            }
            const unsigned b0 = __ballot_sync(0xffffffffu, nd0);
            const unsigned b1 = __ballot_sync(0xffffffffu, nd1);
            if (lane == 0) {
                if (b0) atomicOr(&needbits[q >> 5], 1u << (q & 31));
                if (b1) atomicOr(&needbits[(q + 1) >> 5], 1u << ((q + 1) & 31));
            }
        }
        __syncthreads();
        if (tid < nsurv) {
            const unsigned word = needbits[tid >> 5];
            if ((word >> (tid & 31)) & 1u) {
                int rank = __popc(word & ((1u << (tid & 31)) - 1u));
                for (int q = 0; q < (tid >> 5); ++q) rank += __popc(needbits[q]);
                need[rt * need_stride + s_total + rank] = sid[tid];
            }
        }
        __syncthreads();
        if (tid == 0)
            s_total += __popc(needbits[0]) + __popc(needbits[1]) + __popc(needbits[2]) + __popc(needbits[3]);
        __syncthreads();
    }
    if (tid == 0) {
        const int total = s_total;
        nneed[rt] = total;
        const int nit = (total + kItemTiles - 1) / kItemTiles;
        if (nit > 0) {
            const int b = atomicAdd(n_items, nit);
            for (int i = 0; i < nit; ++i) items[b + i] = make_int2((int)rt, i * kItemTiles);
        }
    }
}

// One direction of the plan (rows X against column tiles of Y).
struct PlanDir {
    const float* X;
    const int32_t* permX;
    int64_t nx_cap;
    const int64_t* d_nx;
    const float* cenX;
    const float* Y;
    const int32_t* permY;
    int64_t ny_cap;
    const int64_t* d_ny;
    const float* cenY;
    int32_t* cand;
    int32_t* cnt;
    float* ub;
    int32_t* need;
    int64_t need_stride;
    int32_t* nneed;
    int2* items;
    int* n_items;
};

// Both directions in one launch (one tail instead of two): CTAs take row
// tiles from a counter (*next, zeroed before the launch), first those of
// direction a, then those of b, up to the device counts.
__global__ void __launch_bounds__(kTM) tc_plan(PlanDir a, PlanDir b, int* __restrict__ next)
{
    __shared__ int s_k;
    const int64_t ta = (kmx_count(a.d_nx, a.nx_cap) + kTM - 1) / kTM;
    const int64_t tb = (kmx_count(b.d_nx, b.nx_cap) + kTM - 1) / kTM;
    for (;;) {
        if (threadIdx.x == 0) s_k = atomicAdd(next, 1);
        __syncthreads();
        const int64_t k = s_k;
        __syncthreads();  // s_k is read before thread 0 takes the next tile
        if (k >= ta + tb) break;
        const bool second = k >= ta;
        const PlanDir d = second ? b : a;
        plan_tile(d.X, d.permX, d.nx_cap, d.d_nx, d.cenX, d.Y, d.permY, d.ny_cap, d.d_ny, d.cenY, d.cand, d.cnt, d.ub,
                  d.need, d.need_stride, d.nneed, d.items, d.n_items, second ? k - ta : k);
        __syncthreads();  // the next tile rewrites the shared arrays
    }
}

// ---------------------------------------------------------------------------
// tensor-core candidate collection
// ---------------------------------------------------------------------------

constexpr int kAStages = 6;   // re-centred row tiles in flight
constexpr int kAccBufs = 4;   // TMEM accumulators (4 x 128 columns: the whole TMEM)
// Tile t goes to epilogue warpgroup t % 2; with even ring sizes every phase
// of a barrier of the A ring or of the accumulators gets its arrivals from
// the same warpgroup.
static_assert(kAStages % 2 == 0 && kAccBufs % 2 == 0, "rings alternate between the two epilogue warpgroups");

struct TcShared {
    uint8_t a[kAStages][kOpBytesA];
    uint8_t b[kStages][kColBytes];
    // per row and A stage: |a|^2 - e, the factor c' |a| of the upper bounds, 2 e
    float4 rowc[kAStages][kTM];
    float gb[kAStages][kTN / 8];  // the column tile's largest |b| per group of 8
    float2 ul[kTM][2];            // latest (U1, U2) of every row from each epilogue warpgroup
    // candidates of the current item per (warpgroup, row), appended to the row's
    // global list when full and at the item's end (stride 17: no bank conflicts)
    int32_t cbuf[2][kTM][kCandBuf + 1];
    uint64_t full_b[kStages], empty_b[kStages];
    uint64_t full_a[kAStages], empty_a[kAStages];
    uint64_t acc_full[kAccBufs], acc_empty[kAccBufs];
    uint32_t tmem;
    int failed;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Epilogue warps only (warps 8..15).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Persistent CTAs; CTA b takes the work items b, b + gridDim.x, ... (an item
// is up to kItemTiles column tiles of one row tile's list).  Warp roles (16
// warps), each running its own loop over the CTA's sequence of column tiles
// and handing tiles on through mbarriers, so that copying, re-centring,
// tensor-core products and the epilogue of different tiles overlap:
//   warp 1 (lane 0)   producer: bulk-copies column tiles into a 4-stage ring;
//   warps 4..7        re-centring: thread = row; the row re-centred on the
//                     column tile's centre as the A operand (3-stage ring),
//                     and the row's constants of the bounds;
//   warp 0 (lane 0)   issues tcgen05.mma (M = N = 128, three K steps) into one
//                     of four TMEM accumulators and commits to the barriers
//                     that free the accumulator's reader, the A stage and the
//                     B stage;
//   warps 8..15       epilogue, two warpgroups: warps 8..11 take the tiles
//                     t with t % 2 == 0, warps 12..15 the others; warp w reads
//                     TMEM lanes 32 (w & 3) .. + 31, all 128 columns of the
//                     tile's accumulator in two halves of 64.
// The two epilogue threads of a row (one per warpgroup) keep their own upper
// bounds over their own tiles' columns and publish them after every tile;
// each combines its own with the other's latest published pair (their column
// sets are disjoint, so any snapshot is a valid bound).  Both start an item from the row's bound U
// counted as two columns at U (the two best columns of the plan's tile,
// which no item holds); at an item boundary the epilogue warps meet on a
// named barrier, so that no thread reads a bound of the previous item's row.
__global__ void __launch_bounds__(kThreads, 1) tc_collect(const float* __restrict__ X,
                                                         const int32_t* __restrict__ permX, int64_t nx_cap,
                                                         const int64_t* d_nx, const uint8_t* __restrict__ packY,
                                                         const int32_t* __restrict__ need, int64_t need_stride,
                                                         const int32_t* __restrict__ nneed,
                                                         const int2* __restrict__ items, const int* __restrict__ n_items,
                                                         float* __restrict__ ub, int32_t* __restrict__ cand,
                                                         int32_t* __restrict__ cnt, unsigned int* err)
{
    extern __shared__ uint8_t smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t rows = kmx_count(d_nx, nx_cap);
    const int nit = *n_items;
    if ((int)blockIdx.x >= nit) return;
    const int stride = (int)gridDim.x;
    auto item_tiles = [&](int it, const int32_t*& tl, int64_t& rt) -> int {
        const int2 item = items[it];
        rt = item.x;
        tl = need + (int64_t)item.x * need_stride + item.y;
        return min(kItemTiles, nneed[item.x] - item.y);
    };

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(&S.full_b[st], 1);
            mbar_init(&S.empty_b[st], 1 + 4);      // MMA commit + the 4 re-centring warps
        }
        for (int st = 0; st < kAStages; ++st) {
            mbar_init(&S.full_a[st], 4);           // re-centring warps
            mbar_init(&S.empty_a[st], 1 + 4);      // MMA commit + the 4 warps of the tile's epilogue warpgroup
        }
        for (int k = 0; k < kAccBufs; ++k) {
            mbar_init(&S.acc_full[k], 1);          // MMA commit
            mbar_init(&S.acc_empty[k], 4);         // the 4 warps of the tile's epilogue warpgroup
        }
        mbar_fence_init();
        S.failed = 0;
    }
    if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    volatile int* failed = &S.failed;
    int issued_b = 0, issued_mma = 0;

    if (warp == 1) {
        // ---- producer
        if (lane == 0) {
            int t = 0;
            for (int it = blockIdx.x; it < nit && !*failed; it += stride) {
                const int32_t* tl;
                int64_t rt;
                const int nt = item_tiles(it, tl, rt);
                for (int k = 0; k < nt; ++k, ++t) {
                    const int st = t % kStages;
                    if (t >= kStages && !mbar_wait(&S.empty_b[st], ((t / kStages) - 1) & 1)) {
                        *failed = 1;
                        break;
                    }
                    mbar_expect_tx(&S.full_b[st], kColBytes);
                    bulk_g2s(S.b[st], packY + (int64_t)tl[k] * kColBytes, kColBytes, &S.full_b[st]);
                    issued_b = t + 1;
                }
            }
        }
    } else if (warp == 0) {
        // ---- tensor-core products
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTM, kTN);
            int t = 0;
            for (int it = blockIdx.x; it < nit && !*failed; it += stride) {
                const int32_t* tl;
                int64_t rt;
                const int nt = item_tiles(it, tl, rt);
                for (int k = 0; k < nt; ++k, ++t) {
                    const int st = t % kStages, sa = t % kAStages, ab = t % kAccBufs;
                    bool ok = mbar_wait(&S.full_b[st], (t / kStages) & 1) &&
                              mbar_wait(&S.full_a[sa], (t / kAStages) & 1);
                    if (ok && t >= kAccBufs) ok = mbar_wait(&S.acc_empty[ab], ((t / kAccBufs) - 1) & 1);
                    if (!ok) {
                        *failed = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(S.a[sa]);
                    const uint32_t b_base = smem_u32(S.b[st]);
                    const uint32_t d = tmem + (uint32_t)(ab * kTN);
#pragma unroll
                    for (int kk = 0; kk < kK / 16; ++kk) {
                        const uint32_t ko = kk * 2 * kCoreStride;
                        umma_bf16(d, smem_desc(a_base + ko, kCoreStride, kGroupStride),
                                  smem_desc(b_base + ko, kCoreStride, kGroupStride), idesc, kk > 0);
                    }
                    umma_commit(&S.acc_full[ab]);
                    umma_commit(&S.empty_a[sa]);
                    umma_commit(&S.empty_b[st]);
                    issued_mma = t + 1;
                }
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ---- re-centring: thread = row
        const int rrow = tid - 128;
        int64_t cur = -1;
        float x[KMX_DESC_DIM];
        int t = 0;
        bool dead = false;
        for (int it = blockIdx.x; it < nit && !dead; it += stride) {
            const int32_t* tl;
            int64_t rt;
            const int nt = item_tiles(it, tl, rt);
            if (rt != cur) {
                cur = rt;
                const int64_t xrow = rt * kTM + rrow;
                const bool xvalid = xrow < rows;
                const float* xr = xvalid ? X + (int64_t)permX[xrow] * KMX_DESC_STRIDE : nullptr;
#pragma unroll
                for (int h = 0; h < KMX_DESC_DIM; ++h) x[h] = xvalid ? __ldg(xr + h) : 0.f;
            }
            for (int k = 0; k < nt; ++k, ++t) {
                const int st = t % kStages, sa = t % kAStages;
                bool ok = !*failed;
                if (ok && t >= kAStages) ok = mbar_wait(&S.empty_a[sa], ((t / kAStages) - 1) & 1);
                if (ok) ok = mbar_wait(&S.full_b[st], (t / kStages) & 1);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) *failed = 1;
                    dead = true;
                    break;
                }
                const uint8_t* bt = S.b[st];
                const float4* cen4 = reinterpret_cast<const float4*>(bt + kHdrCenter);
                float v[kK];
                // paired FP32 operations (the same per-lane rounding); |a|^2
                // as two interleaved partial sums
                float2 q2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 cv = cen4[c];
                    // x + (-c) is exactly x - c
                    const float2 d0 = __fadd2_rn(make_float2(x[4 * c + 0], x[4 * c + 1]), make_float2(-cv.x, -cv.y));
                    const float2 d1 = __fadd2_rn(make_float2(x[4 * c + 2], x[4 * c + 3]), make_float2(-cv.z, -cv.w));
                    v[4 * c + 0] = d0.x;
                    v[4 * c + 1] = d0.y;
                    v[4 * c + 2] = d1.x;
                    v[4 * c + 3] = d1.y;
                    q2 = __ffma2_rn(d0, d0, q2);
                    q2 = __ffma2_rn(d1, d1, q2);
                }
                v[32] = x[32] - reinterpret_cast<const float*>(bt + kHdrCenter)[32];
                const float p2 = fmaf(v[32], v[32], q2.x + q2.y);
                const float al = sqrtf(p2);
                v[KMX_DESC_DIM] = kSqrtC * al;
                v[KMX_DESC_DIM + 1] = -0.5f;
                v[KMX_DESC_DIM + 2] = -0.5f;
#pragma unroll
                for (int h = KMX_DESC_DIM + 3; h < kK; ++h) v[h] = 0.f;
                store_operand_row(S.a[sa], rrow, v);
                const float bmax2 = reinterpret_cast<const float*>(bt + kHdrBmax)[0];
                const float ef = kEfp * (p2 + bmax2);
                S.rowc[sa][rrow] = make_float4(p2 - ef, kUpper * al, 2.f * ef, 0.f);
                if (rrow < kTN / 8) S.gb[sa][rrow] = reinterpret_cast<const float*>(bt + kHdrGBeta)[rrow];
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&S.empty_b[st]);  // done with the column tile's header
                    mbar_arrive(&S.full_a[sa]);
                }
            }
        }
    } else if (warp >= 8) {
        // ---- epilogue
        const int quarter = warp & 3, wg = (warp - 8) >> 2;  // warpgroup wg takes the tiles t with t % 2 == wg
        const int r = quarter * 32 + lane;
        int32_t* cbuf = S.cbuf[wg][r];
        int nbuf = 0;
        // one atomic per flush reserves the places in the row's global list
        auto flush_cands = [&](int64_t row, int nb) {
            const int pos = atomicAdd(cnt + row, nb);
            for (int i = 0; i < nb; ++i)
                if (pos + i < kCandCap) cand[row * kCandCap + pos + i] = cbuf[i];
        };
        int t = 0;
        bool dead = false;
        // every epilogue warp runs every item (after a failure without
        // waiting or working), so that all meet on each named barrier
        for (int it = blockIdx.x; it < nit; it += stride) {
            const int32_t* tl;
            int64_t rt;
            const int nt = item_tiles(it, tl, rt);
            const int64_t row = rt * kTM + r;
            const bool row_valid = row < rows;
            float U1 = row_valid ? __ldcg(ub + row) : FLT_MAX, U2 = U1;
            epi_sync();  // the previous item's bounds are no longer read
            *reinterpret_cast<volatile unsigned long long*>(&S.ul[r][wg]) =
                (unsigned long long)__float_as_uint(U1) | ((unsigned long long)__float_as_uint(U2) << 32);
            epi_sync();
            for (int k = 0; k < nt; ++k, ++t) {
                if ((t & 1) != wg) continue;  // the other warpgroup's tile
                const int sa = t % kAStages, ab = t % kAccBufs;
                if (dead) continue;
                bool ok = !*failed;
                if (ok) ok = mbar_wait(&S.acc_full[ab], (t / kAccBufs) & 1);
                // the A stage (row constants) cannot be refilled before this
                // warpgroup's arrival on empty_a, so its phase t / kAStages is
                // the current one: the wait only acquires the re-centring writes
                if (ok) ok = mbar_wait(&S.full_a[sa], (t / kAStages) & 1);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) *failed = 1;
                    dead = true;
                    continue;
                }
                tc_fence_after();
                const float4 rc = S.rowc[sa][r];
                const float rb = rc.x, ua = rc.y, ue = rc.z;
                // one 64-bit load: the pair is never seen half written
                const unsigned long long ou = *reinterpret_cast<volatile unsigned long long*>(&S.ul[r][wg ^ 1]);
                const float2 other =
                    make_float2(__uint_as_float((uint32_t)ou), __uint_as_float((uint32_t)(ou >> 32)));
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * kTN);
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {  // the two 64-column halves of the tile
                    float v[64];
                    tmem_ld64(tbase + (uint32_t)(h * 64), v);
                    if (h == 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&S.acc_empty[ab]);  // the accumulator is read
                    }
                    const float* gbeta = S.gb[sa] + h * 8;
                    const int64_t col0 = (int64_t)tl[k] * kTN + h * 64;
                    // the second-smallest upper bound over both warpgroups' columns
                    const float Ush = fminf(fmaxf(U1, other.x), U1 <= other.x ? U2 : other.y);
                    float Lm[8];
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const float* vg = v + 8 * g;
                        const float m =
                            fmax3(fmax3(vg[0], vg[1], vg[2]), fmax3(vg[3], vg[4], vg[5]), fmaxf(vg[6], vg[7]));
                        // L = |a|^2 - e - 2 M is monotone in M: the group's
                        // largest M gives its smallest L
                        Lm[g] = fmaf(-2.f, m, rb);
                    }
                    const float lmin =
                        fmin3(fmin3(Lm[0], Lm[1], Lm[2]), fmin3(Lm[3], Lm[4], Lm[5]), fminf(Lm[6], Lm[7]));
                    if (row_valid && lmin <= fminf(U2, Ush)) {
#pragma unroll
                        for (int g = 0; g < 8; ++g) {
                            const float* vg = v + 8 * g;
                            const float Lmin = Lm[g];
                            if (Lmin <= fminf(U2, Ush)) {
                                // the group's two best columns (largest M
                                // first): upper bounds for them
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
                                const float thr = fminf(U2, Ush);
                                unsigned msk = 0;
#pragma unroll
                                for (int j = 0; j < 8; ++j) msk |= (fmaf(-2.f, vg[j], rb) <= thr ? 1u : 0u) << j;
                                while (msk) {
                                    const int j = __ffs(msk) - 1;
                                    msk &= msk - 1;
                                    if (nbuf == kCandBuf) {
                                        flush_cands(row, nbuf);
                                        nbuf = 0;
                                    }
                                    cbuf[nbuf++] = (int32_t)(col0 + 8 * g + j);
                                }
                            }
                        }
                    }
                }
                *reinterpret_cast<volatile unsigned long long*>(&S.ul[r][wg]) =
                    (unsigned long long)__float_as_uint(U1) | ((unsigned long long)__float_as_uint(U2) << 32);
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.empty_a[sa]);  // the row constants are read
            }
            if (!dead && nbuf > 0) flush_cands(row, nbuf);
            nbuf = 0;
            if (!dead && row_valid) {
                // lower the row's bound for the items that start later (bounds
                // are >= 0, so their bits order like integers)
                const unsigned long long ou = *reinterpret_cast<volatile unsigned long long*>(&S.ul[r][wg ^ 1]);
                const float ox = __uint_as_float((uint32_t)ou), oy = __uint_as_float((uint32_t)(ou >> 32));
                const float Uf = fminf(U2, fminf(fmaxf(U1, ox), U1 <= ox ? U2 : oy));
                if (Uf >= 0.f) atomicMin(reinterpret_cast<int*>(ub + row), __float_as_int(Uf));
            }
        }
    }
    __syncthreads();
    if (*failed) {
        // drain: every issued copy and MMA must land before the memory goes
        // away (each waits for the last phase its barrier has outstanding)
        if (tid == 32) {
            for (int st = 0; st < kStages; ++st) {
                const int last = issued_b - 1 - ((issued_b - 1 - st) % kStages + kStages) % kStages;
                if (last >= 0 && last % kStages == st) mbar_wait(&S.full_b[st], (last / kStages) & 1);
            }
        }
        if (tid == 0) {
            kmx_raise(err, KMX_DERR_TIMEOUT);
            for (int k = 0; k < kAccBufs; ++k) {
                const int last = issued_mma - 1 - ((issued_mma - 1 - k) % kAccBufs + kAccBufs) % kAccBufs;
                if (last >= 0 && last % kAccBufs == k) mbar_wait(&S.acc_full[k], (last / kAccBufs) & 1);
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

// Four sorted row positions per warp, eight lanes each (lane s takes
// candidates s, s + 8, ...).  Rows whose list overflowed are appended to the
// exact fallback's list (in any order: each row's summary is its own).
// rows_out (source side) gets (d1, NN, d2) at the original row; cols_best
// (target side) the packed (d1, NN).
__global__ void __launch_bounds__(256) tc_rerank(const float* __restrict__ X, const int32_t* __restrict__ permX,
                                                 int64_t nx_cap, const int64_t* d_nx, const float* __restrict__ Y,
                                                 const int32_t* __restrict__ permY, int64_t ny_cap,
                                                 const int64_t* d_ny, const int32_t* __restrict__ cand,
                                                 const int32_t* __restrict__ cnt,
                                                 kmx::RowBest* __restrict__ rows_out,
                                                 unsigned long long* __restrict__ cols_best,
                                                 int32_t* __restrict__ fb_list, int64_t* __restrict__ fb_n,
                                                 int* __restrict__ final_chunks)
{
    const int lane = threadIdx.x & 31, s = lane & 7;
    if (final_chunks && blockIdx.x == 0 && threadIdx.x == 0) *final_chunks = 1;  // rows_out holds whole-row summaries
    const int64_t nx = kmx_count(d_nx, nx_cap), ny = kmx_count(d_ny, ny_cap);
    // groups of four rows per warp, strided over the grid (the loop is
    // uniform over the warp: its shuffles need every lane)
    for (int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 4; base < nx;
         base += (int64_t)gridDim.x * 32) {
        const int64_t i = base + (lane >> 3);
        const bool active = i < nx;
        const int orig = active ? permX[i] : 0;
        const int c = active ? cnt[i] : 0;
        float b1 = INFINITY, b2 = INFINITY;
        int j1 = 0x7fffffff;
        if (c <= kCandCap && c > s) {
            // the row once, then every candidate with the exact path's arithmetic
            // (one fused multiply-add per term in h order)
            float x[KMX_DESC_DIM];
            const float4* x4 = reinterpret_cast<const float4*>(X + (int64_t)orig * KMX_DESC_STRIDE);
    #pragma unroll
            for (int q4 = 0; q4 < 8; ++q4) {
                const float4 v = __ldg(x4 + q4);
                x[4 * q4] = v.x;
                x[4 * q4 + 1] = v.y;
                x[4 * q4 + 2] = v.z;
                x[4 * q4 + 3] = v.w;
            }
            x[32] = __ldg(X + (int64_t)orig * KMX_DESC_STRIDE + 32);
            for (int q = s; q < c; q += 8) {
                const int pos = cand[i * kCandCap + q];
                if (pos < 0 || pos >= ny) continue;  // padding columns are never collected
                const int j = permY[pos];
                const float* y = Y + (int64_t)j * KMX_DESC_STRIDE;
                const float4* y4 = reinterpret_cast<const float4*>(y);
                float acc = 0.f;
    #pragma unroll
                for (int q4 = 0; q4 < 8; ++q4) {
                    const float4 v = __ldg(y4 + q4);
                    float e = x[4 * q4] - v.x;
                    acc = fmaf(e, e, acc);
                    e = x[4 * q4 + 1] - v.y;
                    acc = fmaf(e, e, acc);
                    e = x[4 * q4 + 2] - v.z;
                    acc = fmaf(e, e, acc);
                    e = x[4 * q4 + 3] - v.w;
                    acc = fmaf(e, e, acc);
                }
                const float e = x[32] - __ldg(y + 32);
                acc = fmaf(e, e, acc);
                kmx::row_update(b1, j1, b2, acc, j);
            }
        }
    #pragma unroll
        for (int o = 4; o >= 1; o >>= 1) {  // within the row's eight lanes
            const float od1 = __shfl_xor_sync(0xffffffffu, b1, o);
            const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
            const float od2 = __shfl_xor_sync(0xffffffffu, b2, o);
            kmx::row_merge(b1, j1, b2, od1, oj, od2);
        }
        if (s != 0 || !active) continue;
        if (c > kCandCap) {
            fb_list[atomicAdd(reinterpret_cast<unsigned long long*>(fb_n), 1ull)] = orig;  // at most nx entries
            continue;
        }
        if (rows_out) rows_out[orig] = kmx::RowBest{b1, j1, b2};
        if (cols_best && j1 != 0x7fffffff) cols_best[orig] = kmx::pack_dist_index(b1, (uint32_t)j1);
    }
}

// Merge the exact fallback partials of each listed row (chunk c's partials
// at part[c * list length ...]) and store them where the re-ranked rows went.
// One warp per row: lane l merges chunks l, l + 32, ..., then the lanes
// merge (the summary of a union does not depend on the merge order).
__global__ void __launch_bounds__(256) fallback_merge(const kmx::RowBest* __restrict__ part,
                                                      const int* __restrict__ d_chunks, int64_t list_cap,
                                                      const int32_t* __restrict__ list,
                                                      const int64_t* __restrict__ n_list,
                                                      kmx::RowBest* __restrict__ rows_out,
                                                      unsigned long long* __restrict__ cols_best)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = min(*n_list, list_cap);
    const int chunks = *d_chunks;
    const int64_t warps = (int64_t)gridDim.x * 8;
    for (int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); r < n; r += warps) {
        float d1 = INFINITY, d2 = INFINITY;
        int j1 = 0x7fffffff;
        for (int c = lane; c < chunks; c += 32) {
            const kmx::RowBest o = part[(int64_t)c * n + r];
            kmx::row_merge(d1, j1, d2, o.d1, o.j1, o.d2);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float od1 = __shfl_xor_sync(0xffffffffu, d1, o);
            const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
            const float od2 = __shfl_xor_sync(0xffffffffu, d2, o);
            kmx::row_merge(d1, j1, d2, od1, oj, od2);
        }
        if (lane != 0) continue;
        const int i = list[r];
        if (rows_out) rows_out[i] = kmx::RowBest{d1, j1, d2};
        if (cols_best && j1 != 0x7fffffff) cols_best[i] = kmx::pack_dist_index(d1, (uint32_t)j1);
    }
}

size_t tc_smem_bytes()
{
    // at least 120 KB: one CTA per SM, whose TMEM allocation is all 512
    // columns (a second CTA would wait in tcgen05.alloc)
    const size_t need = sizeof(TcShared) + 1024;
    return need < 120 * 1024 ? 120 * 1024 : need;
}

struct TcBuffers {
    uint32_t *keys, *keys_tmp;
    int32_t *vals, *vals_tmp;  // the tree's packed entries (source rows, then target rows), level to level
    int32_t* vals_sort;        // the radix sort's temporary values
    int32_t* perm;             // sorted: [0, np) source rows, [np_cap, np_cap + nq) target rows
    int64_t* n2;               // np + nq on the device
    int64_t* nsort;            // the entries a global level's radix sort takes (np + nq or 0)
    void* sort_scratch;
    float* dirs;               // [2 << (levels - 1)][kDirStride]
    uint8_t *packP, *packQ;
    float *cenP, *cenQ;
    float *ubP, *ubQ;
    int32_t *needP, *needQ, *nneedP, *nneedQ;
    int2 *itemsP, *itemsQ;
    int* nitems;               // [0] source rows, [1] target rows, [2] the plan's tile counter
    int32_t *candP, *candQ, *cntP, *cntQ;
    int* chunks;               // [2] fallback P, [3] fallback Q
    int32_t *listP, *listQ;    // fallback rows (original indices)
    int64_t* nlist;            // their counts: [0] P, [1] Q
    kmx::RowBest *fbP, *fbQ;
};

int tc_levels(int64_t np_cap, int64_t nq_cap)
{
    const int lp = tree_levels(np_cap), lq = tree_levels(nq_cap);
    return lp > lq ? lp : lq;
}

TcBuffers tc_carve(void* base, int64_t np_cap, int64_t nq_cap, size_t* total)
{
    TcBuffers b{};
    kmx_arena a{static_cast<char*>(base), 0};
    const int64_t n2 = np_cap + nq_cap;
    const int64_t tp = (np_cap + kTN - 1) / kTN, tq = (nq_cap + kTN - 1) / kTN;  // tiles of either cloud
    const int levels = tc_levels(np_cap, nq_cap);
    const int fc = kmx_match_fp32_max_chunks();
    b.keys = (uint32_t*)a.take(sizeof(uint32_t) * (size_t)n2);
    b.keys_tmp = (uint32_t*)a.take(sizeof(uint32_t) * (size_t)n2);
    b.vals = (int32_t*)a.take(sizeof(int32_t) * (size_t)n2);
    b.vals_tmp = (int32_t*)a.take(sizeof(int32_t) * (size_t)n2);
    b.vals_sort = (int32_t*)a.take(sizeof(int32_t) * (size_t)n2);
    b.perm = (int32_t*)a.take(sizeof(int32_t) * (size_t)n2);
    b.n2 = (int64_t*)a.take(sizeof(int64_t));
    b.nsort = (int64_t*)a.take(sizeof(int64_t));
    b.sort_scratch = a.take(kmx_sort_scratch_bytes(n2));
    b.dirs = (float*)a.take(sizeof(float) * kDirStride * ((size_t)2 << (levels > 0 ? levels - 1 : 0)));
    b.packP = (uint8_t*)a.take((size_t)tp * kColBytes);
    b.packQ = (uint8_t*)a.take((size_t)tq * kColBytes);
    b.cenP = (float*)a.take(sizeof(float) * kCenterStride * (size_t)tp);
    b.cenQ = (float*)a.take(sizeof(float) * kCenterStride * (size_t)tq);
    b.ubP = (float*)a.take(sizeof(float) * (size_t)np_cap);
    b.ubQ = (float*)a.take(sizeof(float) * (size_t)nq_cap);
    b.needP = (int32_t*)a.take(sizeof(int32_t) * (size_t)tp * (size_t)tq);
    b.needQ = (int32_t*)a.take(sizeof(int32_t) * (size_t)tq * (size_t)tp);
    b.nneedP = (int32_t*)a.take(sizeof(int32_t) * (size_t)tp);
    b.nneedQ = (int32_t*)a.take(sizeof(int32_t) * (size_t)tq);
    b.itemsP = (int2*)a.take(sizeof(int2) * (size_t)tp * (size_t)((tq + kItemTiles - 1) / kItemTiles));
    b.itemsQ = (int2*)a.take(sizeof(int2) * (size_t)tq * (size_t)((tp + kItemTiles - 1) / kItemTiles));
    b.nitems = (int*)a.take(sizeof(int) * 4);
    b.candP = (int32_t*)a.take(sizeof(int32_t) * kCandCap * (size_t)np_cap);
    b.candQ = (int32_t*)a.take(sizeof(int32_t) * kCandCap * (size_t)nq_cap);
    b.cntP = (int32_t*)a.take(sizeof(int32_t) * (size_t)(np_cap + nq_cap));
    b.cntQ = b.cntP + np_cap;
    b.chunks = (int*)a.take(sizeof(int) * 4);
    b.listP = (int32_t*)a.take(sizeof(int32_t) * (np_cap + 1));
    b.listQ = (int32_t*)a.take(sizeof(int32_t) * (nq_cap + 1));
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
    const int64_t tp = (np_cap + kTN - 1) / kTN, tq = (nq_cap + kTN - 1) / kTN;
    const int levels = tc_levels(np_cap, nq_cap);
    const int key_bits = levels <= 14 ? 24 : 32;
    if (levels > 30) return cudaErrorInvalidValue;
    const size_t smem = tc_smem_bytes();
    cudaError_t e = kmx_once_per_device(kmx_attr_tc_topk, [smem] {
        cudaError_t r = cudaFuncSetAttribute(tc_collect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r) return r;
        r = cudaFuncSetAttribute(tree_dir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTreeSmem);
        if (r) return r;
        r = cudaFuncSetAttribute(tree_local<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)local_smem_bytes(kLocalRows));
        if (r) return r;
        r = cudaFuncSetAttribute(tree_local<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)local_smem_bytes(kLocalRows));
        if (r) return r;
        return cudaFuncSetAttribute(tree_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFinishSmem);
    });
    if (e) return e;
    if ((e = cudaMemsetAsync(b.nlist, 0, sizeof(int64_t) * 2, st))) return e;
    if ((e = cudaMemsetAsync(b.cntP, 0, sizeof(int32_t) * (size_t)n2, st))) return e;
    if ((e = cudaMemsetAsync(b.nitems, 0, sizeof(int) * 3, st))) return e;
    // locality order of both clouds: one tree level per sort
    const unsigned gb = kmx_stride_blocks(n2, 256, ctx->sm_count);
    KMX_COUNT_LAUNCH();
    tree_init<<<gb, 256, 0, st>>>(np_cap, d_np, nq_cap, d_nq, b.vals, b.n2);
    const int level0 = levels > kFinishLevels ? levels - kFinishLevels : 0;
    // Levels whose nodes can exceed kLocalRows at the capacities run the
    // global kernels (direction, keys, radix sort), which do nothing on the
    // device once every node fits; tree_local then splits the level (or,
    // after the global kernels, does nothing).  The entries alternate
    // between vals and vals_tmp: the sort and tree_local read one and write
    // the other.
    int64_t node_max = np_cap > nq_cap ? np_cap : nq_cap;  // largest node of level l at any device count
    int32_t* cur = b.vals;                                  // the entries as the last level left them
    for (int l = 0; l < level0; ++l, node_max = tree_left(node_max)) {
        int32_t* next = cur == b.vals ? b.vals_tmp : b.vals;
        if (node_max > kLocalRows) {
            KMX_COUNT_LAUNCH();
            tree_dir<<<dim3(1u << l, 2), kTreeThreads, kTreeSmem, st>>>(dp, np_cap, d_np, dq, nq_cap, d_nq, cur, l,
                                                                         b.dirs);
            KMX_COUNT_LAUNCH();
            // 16-bit keys (two radix passes) while they leave at least 9 bits
            // of projection (levels 0..6), wider keys below
            const int kb = l <= 6 ? 16 : key_bits;
            tree_key<<<gb, 256, 0, st>>>(dp, np_cap, d_np, dq, nq_cap, d_nq, cur, l, kb, b.dirs, b.keys, b.nsort);
            if ((e = cudaGetLastError())) return e;
            if ((e = kmx_sort_u32(ctx, b.keys, cur, b.keys_tmp, b.vals_sort, n2, b.nsort, kb, b.sort_scratch,
                                  next)))
                return e;
        }
        const int64_t rows = node_max < kLocalRows ? node_max : kLocalRows;
        KMX_COUNT_LAUNCH();
        if ((int64_t{2} << l) >= kLocalWideCtas) {
            tree_local<256><<<dim3(1u << l, 2), 256, local_smem_bytes(rows), st>>>(dp, np_cap, d_np, dq, nq_cap,
                                                                                  d_nq, cur, next, l, ctx->d_err);
        } else {
            tree_local<1024><<<dim3(1u << l, 2), 1024, local_smem_bytes(rows), st>>>(dp, np_cap, d_np, dq, nq_cap,
                                                                                    d_nq, cur, next, l, ctx->d_err);
        }
        if ((e = cudaGetLastError())) return e;
        cur = next;
    }
    if (levels > 0) {  // the subtrees of at most 16 tiles, one CTA each
        KMX_COUNT_LAUNCH();
        tree_finish<<<dim3(1u << level0, 2), kTreeThreads, kFinishSmem, st>>>(dp, np_cap, d_np, dq, nq_cap, d_nq,
                                                                             cur, b.vals, level0, levels,
                                                                             ctx->d_err);
        if ((e = cudaGetLastError())) return e;
    }
    KMX_COUNT_LAUNCH();
    tree_out<<<gb, 256, 0, st>>>(np_cap, d_np, nq_cap, d_nq, b.vals, b.perm);
    const int32_t* permP = b.perm;
    const int32_t* permQ = b.perm + np_cap;
    // packed tiles, centres and radii
    KMX_COUNT_LAUNCH();
    tc_pack<<<kmx_stride_blocks(tp, 1, ctx->sm_count, 16), kTN, 0, st>>>(dp, permP, np_cap, d_np, b.packP, b.cenP,
                                                                        ctx->d_err);
    KMX_COUNT_LAUNCH();
    tc_pack<<<kmx_stride_blocks(tq, 1, ctx->sm_count, 16), kTN, 0, st>>>(dq, permQ, nq_cap, d_nq, b.packQ, b.cenQ,
                                                                        ctx->d_err);
    // first candidates, bounds and tile lists both ways
    const PlanDir planP{dp, permP, np_cap, d_np, b.cenP, dq, permQ, nq_cap, d_nq, b.cenQ, b.candP,
                        b.cntP, b.ubP, b.needP, tq, b.nneedP, b.itemsP, b.nitems + 0};
    const PlanDir planQ{dq, permQ, nq_cap, d_nq, b.cenQ, dp, permP, np_cap, d_np, b.cenP, b.candQ,
                        b.cntQ, b.ubQ, b.needQ, tp, b.nneedQ, b.itemsQ, b.nitems + 1};
    KMX_COUNT_LAUNCH();
    // about five CTAs per SM fit (registers); more would only wait for the counter
    tc_plan<<<kmx_stride_blocks(tp + tq, 1, ctx->sm_count, 5), kTM, 0, st>>>(planP, planQ, b.nitems + 2);
    // tensor-core candidates both ways: one persistent CTA per SM
    const unsigned grid = (unsigned)(ctx->sm_count > 0 ? ctx->sm_count : 1);
    KMX_COUNT_LAUNCH();
    tc_collect<<<grid, kThreads, smem, st>>>(dp, permP, np_cap, d_np, b.packQ, b.needP, tq, b.nneedP, b.itemsP,
                                             b.nitems + 0, b.ubP, b.candP, b.cntP, ctx->d_err);
    KMX_COUNT_LAUNCH();
    tc_collect<<<grid, kThreads, smem, st>>>(dq, permQ, nq_cap, d_nq, b.packP, b.needQ, tp, b.nneedQ, b.itemsQ,
                                             b.nitems + 1, b.ubQ, b.candQ, b.cntQ, ctx->d_err);
    // exact re-ranking; overflowed rows are flagged
    KMX_COUNT_LAUNCH();
    tc_rerank<<<kmx_stride_blocks(np_cap, 32, ctx->sm_count), 256, 0, st>>>(
        dp, permP, np_cap, d_np, dq, permQ, nq_cap, d_nq, b.candP, b.cntP, s.part, nullptr, b.listP, b.nlist + 0,
        s.chunks);
    KMX_COUNT_LAUNCH();
    tc_rerank<<<kmx_stride_blocks(nq_cap, 32, ctx->sm_count), 256, 0, st>>>(
        dq, permQ, nq_cap, d_nq, dp, permP, np_cap, d_np, b.candQ, b.cntQ, nullptr, s.colbest, b.listQ, b.nlist + 1,
        nullptr);
    if ((e = cudaGetLastError())) return e;
    // exact fallback for the flagged rows of each side
    if ((e = kmx_match_fp32_rows_launch(ctx, dp, b.listP, np_cap, b.nlist + 0, dq, nq_cap, d_nq, b.fbP,
                                        b.chunks + 2)))
        return e;
    if ((e = kmx_match_fp32_rows_launch(ctx, dq, b.listQ, nq_cap, b.nlist + 1, dp, np_cap, d_np, b.fbQ,
                                        b.chunks + 3)))
        return e;
    KMX_COUNT_LAUNCH();
    fallback_merge<<<kmx_stride_blocks(np_cap, 8, ctx->sm_count), 256, 0, st>>>(b.fbP, b.chunks + 2, np_cap,
                                                                                b.listP, b.nlist + 0, s.part, nullptr);
    KMX_COUNT_LAUNCH();
    fallback_merge<<<kmx_stride_blocks(nq_cap, 8, ctx->sm_count), 256, 0, st>>>(b.fbQ, b.chunks + 3, nq_cap,
                                                                                b.listQ, b.nlist + 1, nullptr,
                                                                                s.colbest);
    return cudaGetLastError();
}

// Diagnostics of the last tensor-core match on this scratch: rows that went
// through the exact fallback (source, target), candidates collected
// (source, target) and tile pairs computed on the tensor cores (source row
// tiles, target row tiles), as six int64 values in the caller's device
// buffer.
__global__ void tc_stats(const int64_t* __restrict__ nlist, const int32_t* __restrict__ cntP, int64_t np_cap,
                         const int64_t* d_np, const int32_t* __restrict__ cntQ, int64_t nq_cap, const int64_t* d_nq,
                         const int32_t* __restrict__ nneedP, const int32_t* __restrict__ nneedQ,
                         int64_t* __restrict__ out)
{
    __shared__ unsigned long long sp, sq, tp, tq;
    if (threadIdx.x == 0) {
        sp = 0;
        sq = 0;
        tp = 0;
        tq = 0;
    }
    __syncthreads();
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    unsigned long long a = 0, b = 0, c = 0, d = 0;
    for (int64_t i = threadIdx.x; i < np; i += blockDim.x) a += (unsigned long long)min(cntP[i], kCandCap);
    for (int64_t i = threadIdx.x; i < nq; i += blockDim.x) b += (unsigned long long)min(cntQ[i], kCandCap);
    if (nq > 0)
        for (int64_t i = threadIdx.x; i < (np + kTM - 1) / kTM; i += blockDim.x) c += (unsigned long long)nneedP[i];
    if (np > 0)
        for (int64_t i = threadIdx.x; i < (nq + kTM - 1) / kTM; i += blockDim.x) d += (unsigned long long)nneedQ[i];
    atomicAdd(&sp, a);
    atomicAdd(&sq, b);
    atomicAdd(&tp, c);
    atomicAdd(&tq, d);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = nlist[0];
        out[1] = nlist[1];
        out[2] = (int64_t)sp;
        out[3] = (int64_t)sq;
        out[4] = (int64_t)tp;
        out[5] = (int64_t)tq;
    }
}

cudaError_t kmx_match_tc_stats(kmx_ctx* ctx, void* extra, int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                               const int64_t* d_nq, int64_t* dst)
{
    size_t total = 0;
    TcBuffers b = tc_carve(extra, np_cap, nq_cap, &total);
    KMX_COUNT_LAUNCH();
    tc_stats<<<1, 256, 0, ctx->stream>>>(b.nlist, b.cntP, np_cap, d_np, b.cntQ, nq_cap, d_nq, b.nneedP, b.nneedQ,
                                         dst);
    return cudaGetLastError();
}
