// Device-wide exclusive prefix sum in one pass (decoupled look-back, after
// Merrill and Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016).  Used to turn per-point counts into CSR offsets and to
// compact flagged points in order.
//
// Each CTA claims the next tile id from a counter (so a tile only ever waits
// for tiles claimed before it, by CTAs already running), scans its tile,
// publishes the tile total as an "aggregate", then looks back over the
// predecessors' status words, summing aggregates until it meets an
// "inclusive prefix", and publishes its own inclusive prefix.  A status word
// holds the flag in its top two bits and the value below, so one 64-bit load
// sees both.  Every spin is bounded: when it runs out the CTA records
// KMX_DERR_TIMEOUT and finishes with a wrong prefix instead of waiting on.
//
// The status words live in one zeroed area per context.  Each CTA counts
// itself finished after its last status access, and the last one zeroes the
// words the scan used, so the next scan on the context starts from zeros
// without a memset (one graph node less per scan).  kmx_sync zeroes the area
// again whenever a device error was recorded.
#include "kmx_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int64_t kTile = kThreads * kItems;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagIncl = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;
constexpr uint32_t kPollLimit = 1u << 22;

__device__ __forceinline__ unsigned long long load_status(const unsigned long long* p)
{
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ void store_status(unsigned long long* p, unsigned long long v)
{
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// status[0] is the tile counter, status[1] the count of finished CTAs,
// status[2 + t] the status word of tile t; all zero before the launch and
// zeroed again by the last CTA.  Entries at i >= count read as 0; out[i] is
// written for i < len, or with live_only for i <= count only (the tiles that
// start past the count just count themselves finished).
template <typename T>
__global__ void __launch_bounds__(kThreads) scan_onepass(const T* __restrict__ in, int64_t len, int64_t count_cap,
                                                         const int64_t* __restrict__ d_count,
                                                         int64_t* __restrict__ out,
                                                         unsigned long long* __restrict__ status, int64_t tiles,
                                                         unsigned int* __restrict__ err, bool live_only)
{
    __shared__ int64_t wsum[kThreads / 32];
    __shared__ int64_t tile_prefix;
    __shared__ int last;
    __shared__ int64_t tile_id;
    if (threadIdx.x == 0) tile_id = (int64_t)atomicAdd(status, 1ull);
    __syncthreads();
    const int64_t tile = tile_id;
    if (tile >= tiles) {  // the area was not zero at launch: an earlier scan did not finish
        if (threadIdx.x == 0) kmx_raise(err, KMX_DERR_TIMEOUT);
        return;
    }
    const int64_t count = d_count ? min(*d_count, count_cap) : count_cap;
    if (live_only && tile * kTile > count) {  // block-uniform: no output of this tile is wanted
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(status + 1, 1ull) == (unsigned long long)(tiles - 1);
            __threadfence();
        }
        __syncthreads();
        if (last)
            for (int64_t i = threadIdx.x; i < tiles + 2; i += kThreads) store_status(&status[i], 0ull);
        return;
    }
    const int64_t base = tile * kTile + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = base + i;
        v[i] = idx < count ? (int64_t)in[idx] : 0;
        s += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kThreads / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < kThreads / 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kThreads / 32) wsum[lane] = w;
        const int64_t total = __shfl_sync(0xffffffffu, w, kThreads / 32 - 1);
        unsigned long long* st = status + 2;
        int64_t excl = 0;
        if (tile == 0) {
            if (lane == 0) store_status(&st[0], kFlagIncl | ((unsigned long long)total & kValueMask));
        } else {
            if (lane == 0) store_status(&st[tile], kFlagAgg | ((unsigned long long)total & kValueMask));
            int64_t pred = tile - 1;
            uint32_t polls = 0;
            bool timed_out = false;
            while (true) {
                const int64_t t = pred - lane;
                // before tile 0 there is nothing: an inclusive prefix of 0
                unsigned long long w_st = t >= 0 ? load_status(&st[t]) : kFlagIncl;
                while (__any_sync(0xffffffffu, (w_st >> 62) == 0)) {
                    if (++polls > kPollLimit) {
                        timed_out = true;
                        break;
                    }
                    if ((w_st >> 62) == 0) w_st = load_status(&st[t]);
                }
                if (timed_out) break;
                const unsigned incl = __ballot_sync(0xffffffffu, (w_st >> 62) == 2);
                const int stop = incl ? __ffs(incl) - 1 : 32;  // nearest inclusive predecessor
                int64_t c = lane <= stop ? (int64_t)(w_st & kValueMask) : 0;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                excl += c;
                if (incl) break;
                pred -= 32;
            }
            if (lane == 0) {
                if (timed_out) kmx_raise(err, KMX_DERR_TIMEOUT);
                store_status(&st[tile], kFlagIncl | ((unsigned long long)(excl + total) & kValueMask));
            }
        }
        if (lane == 0) {
            tile_prefix = excl;
            // this CTA's status accesses are done (the look-back's loads were
            // consumed by the warp before lane 0 got here)
            __threadfence();
            last = atomicAdd(status + 1, 1ull) == (unsigned long long)(tiles - 1);
            // acquire side: the zero stores below come after every other
            // CTA's status stores, which preceded their own fenced increments
            __threadfence();
        }
    }
    __syncthreads();
    if (last) {
        // every CTA has finished with the status words: leave them zero
        for (int64_t i = threadIdx.x; i < tiles + 2; i += kThreads) store_status(&status[i], 0ull);
    }
    int64_t e = tile_prefix + x - s + (warp ? wsum[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = base + i;
        if (idx < len) out[idx] = e;
        e += v[i];
    }
}

int64_t tiles_for(int64_t len) { return len > 0 ? (len + kTile - 1) / kTile : 1; }

}  // namespace

int64_t kmx_scan_words(int64_t n) { return tiles_for(n + 1) + 2; }

cudaError_t kmx_scan_reserve(kmx_ctx* ctx, int64_t words)
{
    if (ctx->scan_status && words <= ctx->scan_words) return cudaSuccess;
    int64_t want = ctx->scan_words + ctx->scan_words / 2;
    if (want < words) want = words;
    if (want < 4096) want = 4096;
    if (ctx->scan_status) cudaFreeAsync(ctx->scan_status, ctx->stream);
    ctx->scan_status = nullptr;
    ctx->scan_words = 0;
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, (size_t)want * 8, ctx->stream);
    if (e) return e;
    if ((e = cudaMemsetAsync(p, 0, (size_t)want * 8, ctx->stream))) {
        cudaFreeAsync(p, ctx->stream);
        return e;
    }
    ctx->scan_status = static_cast<unsigned long long*>(p);
    ctx->scan_words = want;
    return cudaSuccess;
}

static cudaError_t scan_launch(kmx_ctx* ctx, const int32_t* in, int64_t n, const int64_t* d_n, int64_t* out,
                               bool live_only)
{
    const int64_t len = n + 1;
    const int64_t tiles = tiles_for(len);
    cudaError_t e = kmx_scan_reserve(ctx, kmx_scan_words(n));
    if (e) return e;
    KMX_COUNT_LAUNCH();
    scan_onepass<int32_t><<<(unsigned)tiles, kThreads, 0, ctx->stream>>>(in, len, n, d_n, out, ctx->scan_status,
                                                                          tiles, ctx->d_err, live_only);
    return cudaGetLastError();
}

cudaError_t kmx_scan_i32(kmx_ctx* ctx, const int32_t* in, int64_t n, const int64_t* d_n, int64_t* out)
{
    return scan_launch(ctx, in, n, d_n, out, false);
}

cudaError_t kmx_scan_i32_live(kmx_ctx* ctx, const int32_t* in, int64_t n, const int64_t* d_n, int64_t* out)
{
    return scan_launch(ctx, in, n, d_n, out, true);
}
