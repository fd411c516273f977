// Device-wide exclusive prefix sum (three-phase: tile scans, a recursive scan
// of the tile totals, then a uniform add).  Used to turn per-point counts into
// CSR offsets and to compact flagged points in order.
#include "kmx_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int64_t kTile = kThreads * kItems;

// Scan one tile of `len` entries; entries at i >= count read as 0.  Writes the
// tile-local exclusive prefix for i < len and the tile total.
template <typename T>
__global__ void __launch_bounds__(kThreads) scan_tiles(const T* __restrict__ in, int64_t len, int64_t count_cap,
                                                       const int64_t* __restrict__ d_count,
                                                       int64_t* __restrict__ out, int64_t* __restrict__ tile_sums)
{
    int64_t count = d_count ? min(*d_count, count_cap) : count_cap;
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < count ? (int64_t)in[idx] : 0;
        s += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __shared__ int64_t wsum[kThreads / 32];
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kThreads / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < kThreads / 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kThreads / 32) wsum[lane] = w;
    }
    __syncthreads();
    int64_t excl = x - s + (warp ? wsum[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = base + i;
        if (idx < len) out[idx] = excl;
        excl += v[i];
    }
    if (threadIdx.x == kThreads - 1) tile_sums[blockIdx.x] = excl;
}

__global__ void __launch_bounds__(kThreads) add_tile_offsets(int64_t* __restrict__ out, int64_t len,
                                                             const int64_t* __restrict__ tile_offs)
{
    int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t add = tile_offs[blockIdx.x];
    if (add == 0) return;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t idx = base + i;
        if (idx < len) out[idx] += add;
    }
}

size_t level_bytes(int64_t len)
{
    int64_t nb = (len + kTile - 1) / kTile;
    if (nb <= 1) return 256;
    // tile sums (nb) + their exclusive scan (nb + 1), then the next level
    return kmx_align_up((size_t)(2 * nb + 1) * sizeof(int64_t), 256) + level_bytes(nb + 1);
}

template <typename T>
cudaError_t scan_level(const T* in, int64_t len, int64_t count_cap, const int64_t* d_count, int64_t* out,
                       char* scratch, cudaStream_t s)
{
    int64_t nb = (len + kTile - 1) / kTile;
    if (nb < 1) nb = 1;
    int64_t* sums = reinterpret_cast<int64_t*>(scratch);
    int64_t* offs = sums + nb;
    KMX_COUNT_LAUNCH();
    scan_tiles<T><<<(unsigned)nb, kThreads, 0, s>>>(in, len, count_cap, d_count, out, sums);
    if (nb == 1) return cudaGetLastError();
    char* next = scratch + kmx_align_up((size_t)(2 * nb + 1) * sizeof(int64_t), 256);
    cudaError_t e = scan_level<int64_t>(sums, nb + 1, nb, nullptr, offs, next, s);
    if (e != cudaSuccess) return e;
    KMX_COUNT_LAUNCH();
    add_tile_offsets<<<(unsigned)nb, kThreads, 0, s>>>(out, len, offs);
    return cudaGetLastError();
}

}  // namespace

size_t kmx_scan_scratch_bytes(int64_t n) { return level_bytes(n + 1); }

cudaError_t kmx_scan_i32(const int32_t* in, int64_t n, const int64_t* d_n, int64_t* out, void* scratch,
                         cudaStream_t s)
{
    return scan_level<int32_t>(in, n + 1, n, d_n, out, static_cast<char*>(scratch), s);
}
