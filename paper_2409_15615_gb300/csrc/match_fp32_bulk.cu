// Mutual nearest-neighbour matching of descriptors (reciprocity test,
// Sec. III-C), exact FP32 path of kmx_match: the tiled matcher with its
// operands staged by bulk copies and the all-zero dimensions of a tile pair
// skipped.
//
// Every distance is sum_h (x_h - y_h)^2 over the 33 descriptor values, each
// term added with one fused multiply-add in h order, exactly the arithmetic of
// match_fp32.cu.  A term whose x_h and y_h are both zero is fma(+-0, +-0,
// acc) = acc, so leaving it out gives the same bits; FPFH histograms are
// mostly zeros (about 70 % of the entries on LiDAR scans), and rows with
// similar zero patterns are grouped into the same tiles so that whole
// dimensions of a 128 x 128 tile pair are zero on both sides:
//
//   mask_insert    per row: the nonzero mask of its 33 values, counted in a
//                  hash table of (side, mask); the first row of a mask lists it.
//   mask_rank      per distinct mask: the rows with a smaller mask on its side
//                  (masks compared with dimension 0 as the most significant
//                  bit), i.e. where its group starts.  A few hundred to a
//                  thousand distinct masks occur per cloud, so this is cheap.
//   place_pack     each row at the next free position of its group (rows with
//                  one mask are interchangeable: their order inside a group
//                  changes neither a tile's mask nor any result), written into
//                  the packed tiles: transposed [33][128]; source values as
//                  (x, x) pairs (one load per paired FP32 instruction), target
//                  values negated (x + (-y) == x - y exactly); the original
//                  row index beside each tile; the tile's nonzero mask (OR of
//                  its rows).
//   match_tiles_fp32_bulk
//                  the (row tile x column tile) grid, flattened row-major, is
//                  cut into chunks of consecutive tile pairs (about 8 per
//                  resident CTA, smaller ones for the end of the sequence)
//                  that the CTAs, 1 or 2 per SM (the context's residency),
//                  take from a counter.  The source tile stays
//                  in shared memory; target tiles stream through a 3-stage
//                  ring filled by cp.async.bulk (mbarrier completion).  For a
//                  tile pair only the dimensions set in either tile's mask are
//                  visited, in ascending order.  Each thread keeps an 8 x 8
//                  block of distances.  Per row: (best, its column, second
//                  best), ties to the lower original column; per column: the
//                  best (distance, original row) packed into 64 bits and folded
//                  with atomicMin.  When a CTA leaves a row tile (or its chunk
//                  ends) it writes the rows' summaries as one "segment".
//   merge_segments per source row, the segments of its row tile, then the
//                  reciprocity test; results land at the original row.
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
constexpr uint32_t kPermBytes = kTile * sizeof(int32_t);     // 512
constexpr int kCtasPerSm = 2;
constexpr int kChunksPerCta = 8;      // default chunks of the tile sequence per resident CTA (load balance)
constexpr int kMaxChunksPerCta = 32;  // the largest setting (kmx_set_match_chunks)
constexpr int kTailChunksPerCta = 4;  // smaller chunks per CTA for the end of the sequence
constexpr int kMinChunk = 4;       // tile pairs per chunk at least (more than kStages - 1)

// Thread 0's position in its own stream of tile pairs (kept in shared memory:
// only thread 0 uses it): the chunk being produced, the offset in it, the tile
// index and column tile of the next item, its ring stage.
struct Producer {
    int64_t x;
    int c;
    int o;
    int ct;
    int par;
    int st;
    int len;  // length of chunk c
};

// The flattened tile sequence (row-major over packed row tiles x column
// tiles) is cut into chunks that CTAs take from a counter, so a CTA whose
// tile pairs need many dimensions simply takes fewer chunks: NA chunks of
// LA pairs, then the last W - WA pairs (about one large chunk per CTA) in
// chunks of LB <= LA pairs, so that the CTAs finish within a small chunk of
// each other.  Chunks are contiguous and only the last one may be short, so
// the segment of chunk c in row tile rt can live in slot c + rt (unique,
// below NC + npt).
struct ChunkGeo {
    int LA, NA, LB, NC;
    int64_t WA;
};

struct __align__(16) BulkShared {
    float2 P[kDim][kTile];                              // source tile, (x, x) pairs
    float Q[kStages][kDim][kTile];                      // negated target tiles
    unsigned long long colred[kThreads / 32][kTile];    // per-warp column bests
    int32_t pperm[kTile];                               // original row of each tile row
    int32_t qperm[kStages][kTile];                      // original column of each tile column
    unsigned long long pm[2];                           // nonzero masks of row tiles rt & ~1, rt | 1
    unsigned long long qm[kStages][2];                  // the same for each stage's column tile
    uint64_t bar_p;
    uint64_t bar_q[kStages];
    Producer prod;
    ChunkGeo cg;                                        // the chunk geometry (thread 0 writes it once)
    int chunk[2];                                       // chunk ids of the current and next local chunk
    int end_item;                                       // first local item past the stream (INT_MAX = unknown)
    int failed;
};
static_assert(kPBytes % 16 == 0 && kQBytes % 16 == 0 && kPermBytes % 16 == 0, "bulk copies move 16-byte units");
static_assert(offsetof(BulkShared, Q) % 16 == 0 && offsetof(BulkShared, pperm) % 16 == 0 &&
                  offsetof(BulkShared, qperm) % 16 == 0 && offsetof(BulkShared, pm) % 16 == 0 &&
                  offsetof(BulkShared, qm) % 16 == 0,
              "bulk copy destinations are 16-byte aligned");

__host__ __device__ __forceinline__ int64_t tiles_of(int64_t n) { return (n + kTile - 1) / kTile; }

// Both sides of one matching call (side 0 = source rows, side 1 = target).
struct SortSides {
    const float* desc[2];
    int64_t cap[2];
    const int64_t* d_n[2];
    int32_t* rowslot[2];           // [cap] hash slot of each row's mask
    unsigned long long* keys;      // [T] (side << 33) | mask, ~0 = empty
    int32_t* count;                // [T] rows per mask
    int32_t* cursor;               // [T] placement cursor per mask
    int64_t* gstart;               // [T] first position of each mask's group
    int32_t* distinct;             // [T] slots in use
    int32_t* n_distinct;           // [1]
    uint32_t T;                    // power of two >= 2 (cap0 + cap1)
    void* packed[2];               // side 0: float2 pairs, side 1: negated floats
    int32_t* perm[2];              // [tiles * 128] original row per packed position, -1 = padding
    unsigned long long* mask[2];   // [tiles] nonzero dimensions of each packed tile
    unsigned long long* colbest;   // [cap1] reset here
};

__device__ __forceinline__ unsigned long long row_mask(const float* __restrict__ row, float (&v)[kStride])
{
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int c = 0; c < kStride / 4; ++c) {
        const float4 x = __ldg(r4 + c);
        v[4 * c] = x.x;
        v[4 * c + 1] = x.y;
        v[4 * c + 2] = x.z;
        v[4 * c + 3] = x.w;
    }
    unsigned long long m = 0;
#pragma unroll
    for (int k = 0; k < kDim; ++k) m |= (unsigned long long)(v[k] != 0.f) << k;
    return m;  // bit k = dimension k
}

__device__ __forceinline__ bool row_finite(const float (&v)[kStride])
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < kDim; ++k) ok &= fabsf(v[k]) <= 3.402823466e38f;  // false for NaN and +-inf
    return ok;
}

// Order of masks: dimension 0 is the most significant bit.
__device__ __forceinline__ unsigned long long mask_order(unsigned long long m) { return __brevll(m) >> (64 - kDim); }

__global__ void __launch_bounds__(256) mask_insert(SortSides S, unsigned int* err)
{
    const int64_t n0 = kmx_count(S.d_n[0], S.cap[0]), n1 = kmx_count(S.d_n[1], S.cap[1]);
    const int64_t t0 = tiles_of(n0), t1 = tiles_of(n1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n0 + n1; t += stride) {
        const int s = t < n0 ? 0 : 1;
        const int64_t i = s ? t - n0 : t;
        float v[kStride];
        const unsigned long long key = ((unsigned long long)s << kDim) | row_mask(S.desc[s] + i * kStride, v);
        if (!row_finite(v)) kmx_raise(err, KMX_DERR_RANGE);
        if (s == 1) S.colbest[i] = ~0ull;
        // lanes with the same key share one insert (a few masks hold most rows)
        const unsigned same_key = __match_any_sync(__activemask(), key);
        const int key_leader = __ffs(same_key) - 1;
        int slot = 0;
        if ((int)(threadIdx.x & 31) == key_leader) slot = kmx_hash_insert(S.keys, S.T, key);
        slot = __shfl_sync(same_key, slot, key_leader);
        S.rowslot[s][i] = slot;
        if (slot < 0) {  // cannot happen at load <= 1/2; reported, never written past
            kmx_raise(err, KMX_DERR_HASHFULL);
            continue;
        }
        // one atomic per distinct slot in the warp (a few masks hold most rows)
        const unsigned same = __match_any_sync(__activemask(), slot);
        if ((threadIdx.x & 31) == __ffs(same) - 1 &&
            atomicAdd(&S.count[slot], __popc(same)) == 0)
            S.distinct[atomicAdd(S.n_distinct, 1)] = slot;
    }
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < t0 + t1; t += stride) {
        if (t < t0)
            S.mask[0][t] = 0;
        else
            S.mask[1][t - t0] = 0;
    }
}

// Sort key of distinct mask e: (side << 40) | mask order.
__device__ __forceinline__ unsigned long long distinct_order(const SortSides& S, int64_t e)
{
    const unsigned long long key = S.keys[S.distinct[e]];
    return ((key >> kDim) << 40) | mask_order(key);
}

constexpr int kRankChunk = 2048;

// One warp per distinct mask: the rows of the smaller masks on its side give
// where its group starts.  The compact list is staged through shared memory
// in chunks; the lanes of a warp stride over a chunk.
__global__ void __launch_bounds__(256) mask_rank(SortSides S)
{
    __shared__ unsigned long long so[kRankChunk];
    __shared__ int32_t sc[kRankChunk];
    const int nd = *S.n_distinct;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    // uniform over the block so that every thread reaches the barriers
    for (int64_t e0 = (int64_t)blockIdx.x * (blockDim.x >> 5); e0 < nd; e0 += wstride) {
        const int64_t e = e0 + warp;
        const unsigned long long me = e < nd ? distinct_order(S, e) : 0ull;
        const unsigned long long lo = me & ~((1ull << 40) - 1);  // same side, any mask
        int64_t start = 0;
        for (int f0 = 0; f0 < nd; f0 += kRankChunk) {
            const int len = min(kRankChunk, nd - f0);
            __syncthreads();
            for (int f = threadIdx.x; f < len; f += blockDim.x) {
                so[f] = distinct_order(S, f0 + f);
                sc[f] = S.count[S.distinct[f0 + f]];
            }
            __syncthreads();
            for (int f = lane; f < len; f += 32) {
                const unsigned long long o = so[f];
                if (o >= lo && o < me) start += sc[f];
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) start += __shfl_xor_sync(0xffffffffu, start, o);
        if (lane == 0 && e < nd) S.gstart[S.distinct[e]] = start;
    }
}

// Slots cover each side's padded rows: slot < n is row `slot`, placed and
// packed; n <= slot < tiles * 128 is a padding position, zeroed.
__global__ void __launch_bounds__(256) place_pack(SortSides S)
{
    const int64_t n0 = kmx_count(S.d_n[0], S.cap[0]), n1 = kmx_count(S.d_n[1], S.cap[1]);
    const int64_t pad0 = tiles_of(n0) * kTile, pad1 = tiles_of(n1) * kTile;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < pad0 + pad1; t += stride) {
        const int s = t < pad0 ? 0 : 1;
        const int64_t slot = s ? t - pad0 : t;
        float v[kStride];
        int64_t pos;
        int32_t orig;
        if (slot < (s ? n1 : n0)) {
            const int hs = S.rowslot[s][slot];
            if (hs < 0) continue;  // table overflow, already reported
            const unsigned long long m = row_mask(S.desc[s] + slot * kStride, v);
            // one atomic per distinct slot in the warp; lanes take consecutive places
            const unsigned same = __match_any_sync(__activemask(), hs);
            const int lane = threadIdx.x & 31, leader = __ffs(same) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&S.cursor[hs], __popc(same));
            base = __shfl_sync(same, base, leader);
            pos = S.gstart[hs] + base + __popc(same & ((1u << lane) - 1u));
            orig = (int32_t)slot;
            if (m) atomicOr(&S.mask[s][pos / kTile], m);
        } else {
            // source padding rows hold +inf, so their distances are +inf (or 0
            // in a tile pair with no dimension to visit, where the index
            // 0xffffffff still loses every tie); target padding columns are
            // skipped by index
#pragma unroll
            for (int k = 0; k < kStride; ++k) v[k] = s == 0 ? INFINITY : 0.f;
            pos = slot;
            orig = -1;
        }
        S.perm[s][pos] = orig;
        const int64_t base = (pos / kTile) * kDim * kTile + (pos % kTile);
        if (s == 0) {
            float2* o = static_cast<float2*>(S.packed[0]) + base;
#pragma unroll
            for (int k = 0; k < kDim; ++k) o[k * kTile] = make_float2(v[k], v[k]);
        } else {
            float* o = static_cast<float*>(S.packed[1]) + base;
#pragma unroll
            for (int k = 0; k < kDim; ++k) o[k * kTile] = -v[k];
        }
    }
}

// Row best as one key: distance bits (non-negative floats order like their
// bits) above the original column, so the minimum key is the best distance
// with ties to the lower column, in any visiting order; the second best is the
// second smallest of {b1, b2, d} = min(b2, max(b1, d)).  Needs finite
// distances (descriptors are checked when they are packed).
__device__ __forceinline__ void row_step(unsigned long long& k1, float& b2, float d, uint32_t j)
{
    const float b1 = __uint_as_float((uint32_t)(k1 >> 32));
    b2 = fminf(b2, fmaxf(b1, d));
    const unsigned long long kd = ((unsigned long long)__float_as_uint(d) << 32) | j;
    k1 = kd < k1 ? kd : k1;
}

constexpr unsigned long long kNoBest = (0x7f800000ull << 32) | 0x7fffffffull;  // (+inf, no column)

__device__ __forceinline__ ChunkGeo chunk_geo(int64_t W, int ctas, int chunks_per_cta)
{
    const int64_t per = (int64_t)chunks_per_cta * ctas;
    int64_t LA = (W + per - 1) / per;
    if (LA < kMinChunk) LA = kMinChunk;
    const int64_t tail = W < ctas * LA ? W : ctas * LA;
    const int64_t NA = (W - tail) / LA;
    const int64_t WA = NA * LA;
    const int64_t tper = (int64_t)kTailChunksPerCta * ctas;
    int64_t LB = (W - WA + tper - 1) / tper;
    if (LB < kMinChunk) LB = kMinChunk;
    const int64_t NB = (W - WA + LB - 1) / LB;
    return ChunkGeo{(int)LA, (int)NA, (int)LB, (int)(NA + NB), WA};
}

__device__ __forceinline__ int64_t chunk_start(const ChunkGeo& g, int c)
{
    return c < g.NA ? (int64_t)c * g.LA : g.WA + (int64_t)(c - g.NA) * g.LB;
}

__device__ __forceinline__ int chunk_len(const ChunkGeo& g, int c) { return c < g.NA ? g.LA : g.LB; }

__device__ __forceinline__ int64_t chunk_of(const ChunkGeo& g, int64_t x)
{
    return x < g.WA ? x / g.LA : g.NA + (x - g.WA) / g.LB;
}

__device__ __forceinline__ int read_end(const BulkShared& S) { return *reinterpret_cast<const volatile int*>(&S.end_item); }

// Thread 0 only, for consecutive local items u: take a new chunk when the
// current one is used up, stop (recording the end of the stream) when the
// counter has run out or the tile sequence has ended, else issue the copies
// of the item's column tile into its ring stage.
__device__ __forceinline__ bool produce(BulkShared& S, int u, const ChunkGeo& cg, int64_t W, int nqt,
                                        int32_t* counter, const float* __restrict__ qn,
                                        const int32_t* __restrict__ qperm,
                                        const unsigned long long* __restrict__ qmask, int& issued)
{
    Producer& P = S.prod;
    if (P.o == P.len) {
        P.par ^= 1;
        P.o = 0;
        P.c = atomicAdd(counter, 1);
        S.chunk[P.par] = P.c;
        P.x = chunk_start(cg, P.c);
        P.len = chunk_len(cg, P.c);
        P.ct = (int)(P.x % nqt);
    }
    if (P.c >= cg.NC || P.x >= W) {
        S.end_item = u;
        return false;
    }
    // the tile's nonzero mask travels with it, in the 16-byte pair holding it
    // (the mask arrays have tiles + 1 entries and start 16-byte aligned)
    mbar_expect_tx(&S.bar_q[P.st], kQBytes + kPermBytes + 16);
    bulk_g2s(S.Q[P.st], qn + (int64_t)P.ct * kDim * kTile, kQBytes, &S.bar_q[P.st]);
    bulk_g2s(S.qperm[P.st], qperm + (int64_t)P.ct * kTile, kPermBytes, &S.bar_q[P.st]);
    bulk_g2s(S.qm[P.st], qmask + (P.ct & ~1), 16, &S.bar_q[P.st]);
    issued = u + 1;
    ++P.o;
    ++P.x;
    if (++P.ct == nqt) P.ct = 0;
    if (++P.st == kStages) P.st = 0;
    return true;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    match_tiles_fp32_bulk(const float2* __restrict__ pp, const int32_t* __restrict__ pperm,
                          const unsigned long long* __restrict__ pmask, int64_t np_cap, const int64_t* d_np,
                          const float* __restrict__ qn, const int32_t* __restrict__ qperm,
                          const unsigned long long* __restrict__ qmask, int64_t nq_cap, const int64_t* d_nq,
                          int ctas, int chunks_per_cta, int32_t* __restrict__ counter,
                          kmx::RowBest* __restrict__ seg,
                          unsigned long long* __restrict__ colbest, unsigned int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BulkShared& S = *reinterpret_cast<BulkShared*>(smem_raw);
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    const int npt = (int)tiles_of(np);
    const int nqt = (int)tiles_of(nq);
    const int64_t W = (int64_t)npt * nqt;
    if (W == 0) return;
    const ChunkGeo& cg = S.cg;  // read from shared memory where needed (registers are full)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid & 15;                     // column group: columns 4tx..4tx+3 and 64+4tx..64+4tx+3
    const int ty = warp * 2 + ((tid >> 4) & 1);  // row group: rows 8ty..8ty+7

    if (tid == 0) {
        mbar_init(&S.bar_p, 1);
        for (int s = 0; s < kStages; ++s) mbar_init(&S.bar_q[s], 1);
        mbar_fence_init();
        S.failed = 0;
        S.end_item = INT_MAX;
        S.cg = chunk_geo(W, ctas, chunks_per_cta);
    }
    __syncthreads();
    int issued = 0;  // meaningful in thread 0: local items whose copies were issued
    if (tid == 0) {
        const int c0 = atomicAdd(counter, 1);
        S.chunk[0] = c0;
        if (c0 >= cg.NC) {
            S.end_item = 0;
        } else {
            const int64_t x0 = chunk_start(cg, c0);
            S.prod = Producer{x0, c0, 0, (int)(x0 % nqt), 0, 0, chunk_len(cg, c0)};
            const int64_t rt0 = x0 / nqt;
            mbar_expect_tx(&S.bar_p, kPBytes + kPermBytes + 16);
            bulk_g2s(S.P, pp + rt0 * kDim * kTile, kPBytes, &S.bar_p);
            bulk_g2s(S.pperm, pperm + rt0 * kTile, kPermBytes, &S.bar_p);
            bulk_g2s(S.pm, pmask + (rt0 & ~1), 16, &S.bar_p);
            for (int u = 0; u < kStages; ++u)
                if (!produce(S, u, cg, W, nqt, counter, qn, qperm, qmask, issued)) break;
        }
    }
    __syncthreads();
    if (read_end(S) == 0) return;
    // this thread's view of the current item: chunk id and parity, items
    // left in the chunk after it, row and column tile, ring stage and phase
    int cid = S.chunk[0];
    int kpar = 0;
    int left = chunk_len(cg, cid) - 1;
    int rt = (int)(chunk_start(cg, cid) / nqt);
    int ct = (int)(chunk_start(cg, cid) - (int64_t)rt * nqt);
    int s = 0;
    uint32_t qphase = 0;
    uint32_t p_phase = 0;
    bool p_ready = false;
    unsigned long long mrow = 0;

    unsigned long long k1[8];
    float b2[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        k1[i] = kNoBest;
        b2[i] = INFINITY;
    }
    bool failed = false;
    int t = 0;
    for (; t < read_end(S); ++t) {
        const int64_t col0 = (int64_t)ct * kTile;
        if (!p_ready) {
            if (!mbar_wait(&S.bar_p, p_phase)) S.failed = 1;
            p_ready = true;
            mrow = S.pm[rt & 1];
        }
        if (!mbar_wait(&S.bar_q[s], qphase)) S.failed = 1;

        float2 acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int jp = 0; jp < 4; ++jp) acc[i][jp] = make_float2(0.f, 0.f);
        // dimensions that are zero in every row of both tiles add exactly
        // nothing; the others are visited in ascending order
        for (unsigned long long m = mrow | S.qm[s][ct & 1]; m; m &= m - 1) {
            const int kk = __ffsll((long long)m) - 1;
            const float4 c0 = *reinterpret_cast<const float4*>(&S.Q[s][kk][tx * 4]);
            const float4 c1 = *reinterpret_cast<const float4*>(&S.Q[s][kk][64 + tx * 4]);
            const float2 nc[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                                  make_float2(c1.z, c1.w)};
#pragma unroll
            for (int ih = 0; ih < 4; ++ih) {
                const float4 a2 = *reinterpret_cast<const float4*>(&S.P[kk][ty * 8 + 2 * ih]);
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
        // row bests over this thread's columns (padding columns skipped)
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = (jp < 2 ? 0 : 64) + tx * 4 + 2 * (jp & 1) + h;
                if (col0 + c < nq) {
                    const uint32_t jo = (uint32_t)S.qperm[s][c];
#pragma unroll
                    for (int i = 0; i < 8; ++i) row_step(k1[i], b2[i], h ? acc[i][jp].y : acc[i][jp].x, jo);
                }
            }
        }
        // column bests: over this thread's 8 rows the smallest distance and
        // the lowest original row reaching it (padding rows count as +inf),
        // then the partner half-warp, then the 8 warps through shared memory
        const int64_t rowbase = (int64_t)rt * kTile + ty * 8;
        uint32_t ro[8];  // padding rows: 0xffffffff (perm -1), distance +inf
#pragma unroll
        for (int i = 0; i < 8; ++i) ro[i] = (uint32_t)S.pperm[ty * 8 + i];
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float m = h ? acc[0][jp].y : acc[0][jp].x;
#pragma unroll
                for (int i = 1; i < 8; ++i) m = fminf(m, h ? acc[i][jp].y : acc[i][jp].x);
                uint32_t r = 0xffffffffu;
#pragma unroll
                for (int i = 0; i < 8; ++i) r = (h ? acc[i][jp].y : acc[i][jp].x) == m ? min(r, ro[i]) : r;
                unsigned long long best = r == 0xffffffffu ? ~0ull : kmx::pack_dist_index(m, r);
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, 16);
                best = other < best ? other : best;
                // stored at (2 jp + h) * 16 + tx: lanes write consecutive words
                if (lane < 16) S.colred[warp][(2 * jp + h) * 16 + tx] = best;
            }
        }
        __syncthreads();  // (1) all waits of this tile are behind every thread
        failed = S.failed != 0;  // uniform: S.failed is written only before (1)
        if (!failed && tid < kTile) {
            // column tid of the tile was stored at (2 jp + h) * 16 + tx
            const int q = tid & 63;
            const int jp = (tid >> 6) * 2 + ((q & 3) >> 1), h = q & 1, ctx = q >> 2;
            const int p = (2 * jp + h) * 16 + ctx;
            unsigned long long best = S.colred[0][p];
#pragma unroll
            for (int v = 1; v < kThreads / 32; ++v) {
                const unsigned long long ov = S.colred[v][p];
                best = ov < best ? ov : best;
            }
            if (col0 + tid < nq && best != ~0ull) atomicMin(&colbest[S.qperm[s][tid]], best);
        }
        const bool seg_end = (left == 0) || (ct + 1 == nqt);  // row tile, chunk or sequence ends
        if (seg_end && !failed) {
            // merge the 16 column groups of each row (one half-warp), write
            // the segment of (chunk, row tile), restart the row bests
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float d1 = __uint_as_float((uint32_t)(k1[i] >> 32)), d2 = b2[i];
                int jj = (int)(uint32_t)k1[i];
#pragma unroll
                for (int sh = 1; sh < 16; sh <<= 1) {
                    const float od1 = __shfl_xor_sync(0xffffffffu, d1, sh);
                    const float od2 = __shfl_xor_sync(0xffffffffu, d2, sh);
                    const int oj = __shfl_xor_sync(0xffffffffu, jj, sh);
                    kmx::row_merge(d1, jj, d2, od1, oj, od2);
                }
                if (tx == 0 && rowbase + i < np)
                    seg[((int64_t)cid + rt) * kTile + ty * 8 + i] = kmx::RowBest{d1, jj, d2};
                k1[i] = kNoBest;
                b2[i] = INFINITY;
            }
        }
        __syncthreads();  // (2) stage s, the source tile and colred are free
        if (failed) break;
        if (tid == 0 && read_end(S) == INT_MAX) produce(S, t + kStages, cg, W, nqt, counter, qn, qperm, qmask, issued);
        // advance to the next item (its chunk id is known: it was produced
        // kStages items ago); a new row tile reloads the source tile
        if (t + 1 < read_end(S)) {
            int rt1;
            if (left > 0) {
                --left;
                rt1 = rt;
                if (++ct == nqt) {
                    ct = 0;
                    rt1 = rt + 1;
                }
            } else {
                kpar ^= 1;
                cid = S.chunk[kpar];
                left = chunk_len(cg, cid) - 1;
                const int64_t x1 = chunk_start(cg, cid);
                rt1 = (int)(x1 / nqt);
                ct = (int)(x1 - (int64_t)rt1 * nqt);
            }
            if (rt1 != rt) {
                if (tid == 0) {
                    mbar_expect_tx(&S.bar_p, kPBytes + kPermBytes + 16);
                    bulk_g2s(S.P, pp + (int64_t)rt1 * kDim * kTile, kPBytes, &S.bar_p);
                    bulk_g2s(S.pperm, pperm + (int64_t)rt1 * kTile, kPermBytes, &S.bar_p);
                    bulk_g2s(S.pm, pmask + (rt1 & ~1), 16, &S.bar_p);
                }
                rt = rt1;
                p_phase ^= 1u;
                p_ready = false;
            }
        }
        if (++s == kStages) {
            s = 0;
            qphase ^= 1u;
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

// One thread per packed source position: the segments of its row tile (one
// per chunk that touched it, in ascending column order; row_merge resolves
// ties by original column), then the reciprocity test; results go to the
// original row.
__global__ void __launch_bounds__(256) merge_segments(const kmx::RowBest* __restrict__ seg,
                                                      const int32_t* __restrict__ pperm, int ctas,
                                                      int chunks_per_cta, int64_t np_cap,
                                                      const int64_t* d_np, int64_t nq_cap, const int64_t* d_nq,
                                                      const unsigned long long* __restrict__ colbest,
                                                      kmx::RowBest* __restrict__ merged, int32_t* __restrict__ mflag)
{
    const int64_t np = kmx_count(d_np, np_cap), nq = kmx_count(d_nq, nq_cap);
    const int64_t npt = tiles_of(np);
    const int64_t nqt = tiles_of(nq);
    const int64_t W = npt * nqt;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < np; i += (int64_t)gridDim.x * 256) {
        kmx::RowBest r{INFINITY, 0x7fffffff, INFINITY};
        if (W > 0) {
            const ChunkGeo cg = chunk_geo(W, ctas, chunks_per_cta);
            const int64_t rt = i / kTile;
            const int64_t cf = chunk_of(cg, rt * nqt), cl = chunk_of(cg, rt * nqt + nqt - 1);
            r = seg[(cf + rt) * kTile + (i % kTile)];
            for (int64_t c = cf + 1; c <= cl; ++c) {
                const kmx::RowBest o = seg[(c + rt) * kTile + (i % kTile)];
                kmx::row_merge(r.d1, r.j1, r.d2, o.d1, o.j1, o.d2);
            }
        }
        const int32_t orig = pperm[i];
        merged[orig] = r;
        bool mutual = false;
        if (r.j1 >= 0 && r.j1 != 0x7fffffff) mutual = (uint32_t)(colbest[r.j1] & 0xffffffffull) == (uint32_t)orig;
        mflag[orig] = mutual ? 1 : 0;
    }
}

struct BulkScratch {
    SortSides sort;
    kmx::RowBest* seg;
    int32_t* chunk_counter;
};

uint32_t mask_table_size(int64_t np_cap, int64_t nq_cap)
{
    uint64_t t = 1024;
    while (t < (uint64_t)(2 * (np_cap + nq_cap + 1))) t <<= 1;
    return (uint32_t)t;
}

BulkScratch carve(void* base, int64_t np_cap, int64_t nq_cap, int max_ctas, size_t* total)
{
    kmx_arena a{static_cast<char*>(base), 0};
    BulkScratch s{};
    const int64_t cap[2] = {np_cap, nq_cap};
    for (int side = 0; side < 2; ++side) {
        const int64_t tiles = tiles_of(cap[side]);
        s.sort.packed[side] = a.take((size_t)tiles * (side ? kQBytes : kPBytes));
        s.sort.perm[side] = static_cast<int32_t*>(a.take((size_t)tiles * kPermBytes));
        s.sort.mask[side] = static_cast<unsigned long long*>(a.take(sizeof(unsigned long long) * (tiles + 1)));
        s.sort.rowslot[side] = static_cast<int32_t*>(a.take(sizeof(int32_t) * (cap[side] + 1)));
    }
    const uint32_t T = mask_table_size(np_cap, nq_cap);
    s.sort.T = T;
    s.sort.keys = static_cast<unsigned long long*>(a.take(sizeof(unsigned long long) * T));
    // count, cursor, the distinct counter and the chunk counter are adjacent:
    // one memset clears them
    s.sort.count = static_cast<int32_t*>(a.take(sizeof(int32_t) * (2 * (size_t)T + 2)));
    s.sort.cursor = s.sort.count + T;
    s.sort.n_distinct = s.sort.count + 2 * (size_t)T;
    s.chunk_counter = s.sort.count + 2 * (size_t)T + 1;
    s.sort.gstart = static_cast<int64_t*>(a.take(sizeof(int64_t) * T));
    s.sort.distinct = static_cast<int32_t*>(a.take(sizeof(int32_t) * T));
    s.seg = static_cast<kmx::RowBest*>(
        a.take(sizeof(kmx::RowBest) * kTile *
               (size_t)((kMaxChunksPerCta + kTailChunksPerCta) * max_ctas + 1 + tiles_of(np_cap))));
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
    BulkScratch b = carve(s.extra, np_cap, nq_cap, max_ctas(ctx->sm_count), &total);
    b.sort.desc[0] = dp;
    b.sort.desc[1] = dq;
    b.sort.cap[0] = np_cap;
    b.sort.cap[1] = nq_cap;
    b.sort.d_n[0] = d_np;
    b.sort.d_n[1] = d_nq;
    b.sort.colbest = s.colbest;
    cudaError_t e = set_smem_attr();
    if (e) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, match_tiles_fp32_bulk, kThreads,
                                                           sizeof(BulkShared))))
        return e;
    const int want = ctx->match_ctas_per_sm > 0 ? ctx->match_ctas_per_sm : kCtasPerSm;
    const int ctas = max(1, min(per_sm, min(want, kCtasPerSm))) * ctx->sm_count;
    const int cpc = ctx->match_chunks_per_cta > 0 ? min(ctx->match_chunks_per_cta, kMaxChunksPerCta) : kChunksPerCta;
    const unsigned small_grid = 4u * (unsigned)ctx->sm_count;  // grid-stride over the actual rows
    if ((e = cudaMemsetAsync(b.sort.keys, 0xFF, sizeof(unsigned long long) * b.sort.T, st))) return e;
    if ((e = cudaMemsetAsync(b.sort.count, 0, sizeof(int32_t) * (2 * (size_t)b.sort.T + 2), st))) return e;
    KMX_COUNT_LAUNCH();
    mask_insert<<<small_grid, 256, 0, st>>>(b.sort, ctx->d_err);
    KMX_COUNT_LAUNCH();
    mask_rank<<<small_grid, 256, 0, st>>>(b.sort);
    KMX_COUNT_LAUNCH();
    place_pack<<<small_grid, 256, 0, st>>>(b.sort);
    KMX_COUNT_LAUNCH();
    match_tiles_fp32_bulk<<<ctas, kThreads, sizeof(BulkShared), st>>>(
        static_cast<const float2*>(b.sort.packed[0]), b.sort.perm[0], b.sort.mask[0], np_cap, d_np,
        static_cast<const float*>(b.sort.packed[1]), b.sort.perm[1], b.sort.mask[1], nq_cap, d_nq, ctas, cpc,
        b.chunk_counter, b.seg, s.colbest, ctx->d_err);
    KMX_COUNT_LAUNCH();
    merge_segments<<<kmx_stride_blocks(np_cap, 256, ctx->sm_count), 256, 0, st>>>(
        b.seg, b.sort.perm[0], ctas, cpc, np_cap, d_np, nq_cap, d_nq, s.colbest, s.merged, s.mflag);
    if ((e = cudaGetLastError())) return e;
    return kmx::match_emit(ctx, s, np_cap, d_np, vp, vq, out, cap, n_out);
}
