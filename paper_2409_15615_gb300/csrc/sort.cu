// Stable least-significant-digit radix sort of (uint32 key, int32 value)
// pairs, 8 bits per pass.  The tensor-core matcher uses it to put descriptor
// rows in the order of a locality key, so that 128-row tiles hold similar
// descriptors.
//
// One pass over digit position p:
//   count    block b counts the digits of its 2048 elements; counts are laid
//            out digit-major (counts[d * blocks + b], blocks = the blocks
//            below the element count, which may be a device value) so that
//            their exclusive scan is, for every (digit, block), the first
//            output position of that block's elements with that digit;
//   scan     kmx_scan_i32 over the 256 * blocks counts;
//   scatter  block b writes element e with digit d to
//            scan[d * blocks + b] + (elements of the block before e with
//            digit d).  Elements are taken in index order (item k of thread
//            t is element 256 k + t), warps resolve equal digits with
//            __match_any_sync, and the per-digit prefixes over warps and
//            items are kept in shared memory, so the pass is stable.
#include "kmx_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kPerBlock = kThreads * kItems;
constexpr int kDigits = 256;
constexpr int kWarps = kThreads / 32;

// Blocks that hold elements below the count: the digit-major counts use
// this stride, so that their scan covers no empty block.
__device__ __forceinline__ int live_blocks(int64_t n)
{
    const int64_t b = (n + kPerBlock - 1) / kPerBlock;
    return (int)(b > 0 ? b : 1);
}

__global__ void __launch_bounds__(kThreads) radix_count(const uint32_t* __restrict__ keys, int64_t n_cap,
                                                        const int64_t* d_n, int shift, int32_t* __restrict__ counts,
                                                        int64_t* __restrict__ n_counts)
{
    __shared__ int hist[kDigits];
    const int64_t n = kmx_count(d_n, n_cap);
    const int blocks = live_blocks(n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_counts = (int64_t)kDigits * blocks;
    if ((int)blockIdx.x >= blocks) return;  // block-uniform
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kPerBlock;
    // one shared atomic per distinct digit and warp: the digits of a block
    // often coincide (sorted prefixes), and equal addresses serialise
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int64_t e = base + k * kThreads + threadIdx.x;
        const int d = e < n ? (int)((keys[e] >> shift) & 0xFFu) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[d], __popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * blocks + blockIdx.x] = hist[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) radix_scatter(const uint32_t* __restrict__ keys,
                                                          const int32_t* __restrict__ vals, int64_t n_cap,
                                                          const int64_t* d_n, int shift,
                                                          const int64_t* __restrict__ offs,
                                                          uint32_t* __restrict__ keys_out,
                                                          int32_t* __restrict__ vals_out)
{
    const int64_t n = kmx_count(d_n, n_cap);
    if ((int64_t)blockIdx.x * kPerBlock >= n) return;  // no element here (block-uniform)
    const int blocks = live_blocks(n);
    __shared__ int wcount[kWarps][kDigits];  // this item's count per warp and digit, then its warp prefix
    __shared__ int running[kDigits];         // elements of earlier items, per digit
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    running[tid] = 0;
    const int64_t base = (int64_t)blockIdx.x * kPerBlock;
    const int64_t first = offs[(int64_t)tid * blocks + blockIdx.x];  // thread tid holds digit tid's start
    __shared__ int64_t start[kDigits];
    start[tid] = first;
    for (int k = 0; k < kItems; ++k) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcount[w][tid] = 0;
        __syncthreads();
        const int64_t e = base + k * kThreads + tid;
        const bool valid = e < n;
        const uint32_t key = valid ? keys[e] : 0u;
        const int d = (int)((key >> shift) & 0xFFu);
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        int rank = 0;
        if (valid) {
            const unsigned peers = __match_any_sync(vmask, d);
            rank = __popc(peers & lt);
            if (rank == 0) wcount[warp][d] = __popc(peers);
        }
        __syncthreads();
        {  // thread tid: exclusive prefix over warps of digit tid
            int acc = running[tid];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const int c = wcount[w][tid];
                wcount[w][tid] = acc;
                acc += c;
            }
            running[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = start[d] + wcount[warp][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = vals[e];
        }
        __syncthreads();
    }
}

// The result back into the callers' arrays after an odd number of passes.
__global__ void __launch_bounds__(256) radix_copy(const uint32_t* __restrict__ ks, const int32_t* __restrict__ vs,
                                                  int64_t n_cap, const int64_t* d_n, uint32_t* __restrict__ kd,
                                                  int32_t* __restrict__ vd)
{
    const int64_t n = kmx_count(d_n, n_cap);
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256) {
        kd[e] = ks[e];
        vd[e] = vs[e];
    }
}

}  // namespace

int kmx_sort_blocks(int64_t n) { return (int)((n + kPerBlock - 1) / kPerBlock); }

size_t kmx_sort_scratch_bytes(int64_t n)
{
    const int64_t b = kmx_sort_blocks(n) > 0 ? kmx_sort_blocks(n) : 1;
    kmx_arena a{nullptr, 0};
    a.take(sizeof(int32_t) * (size_t)(kDigits * b + 1));
    a.take(sizeof(int64_t) * (size_t)(kDigits * b + 1));
    a.take(sizeof(int64_t));
    return kmx_align_up(a.used, 256);
}

cudaError_t kmx_sort_u32(kmx_ctx* ctx, uint32_t* keys, int32_t* vals, uint32_t* keys_tmp, int32_t* vals_tmp,
                         int64_t n, const int64_t* d_n, int bits, void* scratch, int32_t* vals_out)
{
    if (n <= 0) return cudaSuccess;
    const int blocks = kmx_sort_blocks(n);
    kmx_arena a{static_cast<char*>(scratch), 0};
    int32_t* counts = (int32_t*)a.take(sizeof(int32_t) * (size_t)(kDigits * blocks + 1));
    int64_t* offs = (int64_t*)a.take(sizeof(int64_t) * (size_t)(kDigits * blocks + 1));
    int64_t* n_counts = (int64_t*)a.take(sizeof(int64_t));  // counts actually laid out (256 x live blocks)
    const int64_t m = (int64_t)kDigits * blocks;
    const int passes = (bits + 7) / 8;
    uint32_t *ki = keys, *ko = keys_tmp;
    int32_t* vi = vals;
    cudaError_t e;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        // values: with vals_out the passes alternate so that the last one
        // writes vals_out; otherwise between vals and vals_tmp
        int32_t* vo = vals_out ? (((passes - 1 - p) & 1) ? vals_tmp : vals_out) : (vi == vals ? vals_tmp : vals);
        KMX_COUNT_LAUNCH();
        radix_count<<<blocks, kThreads, 0, ctx->stream>>>(ki, n, d_n, shift, counts, n_counts);
        if ((e = cudaGetLastError())) return e;
        if ((e = kmx_scan_i32_live(ctx, counts, m, n_counts, offs))) return e;
        KMX_COUNT_LAUNCH();
        radix_scatter<<<blocks, kThreads, 0, ctx->stream>>>(ki, vi, n, d_n, shift, offs, ko, vo);
        if ((e = cudaGetLastError())) return e;
        uint32_t* tk = ki;
        ki = ko;
        ko = tk;
        vi = vo;
    }
    if (!vals_out && vi != vals) {  // an odd number of passes: the result is in the temporaries
        KMX_COUNT_LAUNCH();
        radix_copy<<<kmx_stride_blocks(n, 256, ctx->sm_count), 256, 0, ctx->stream>>>(ki, vi, n, d_n, keys, vals);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}
