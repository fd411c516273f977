// Internal declarations shared by the kmx CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

#include "kmx.h"

// Process-wide count of kernels launched by the library (kmx_launch_count).
extern std::atomic<long long> kmx_g_launches;
#define KMX_COUNT_LAUNCH() kmx_g_launches.fetch_add(1, std::memory_order_relaxed)

// Device-side error bits, accumulated with atomicOr into kmx_ctx::d_err.
enum : unsigned int {
    KMX_DERR_RANGE = 1u,
    KMX_DERR_CAPACITY = 2u,
    KMX_DERR_HASHFULL = 4u,
    KMX_DERR_TIMEOUT = 8u,
};

struct kmx_ctx {
    int device;
    cudaStream_t stream;
    void* ws;              // scratch, stream-ordered allocation
    size_t ws_size;
    unsigned int* d_err;   // device error bits
    unsigned int* h_err;   // pinned host mirror for kmx_sync
    int sm_count;
    int match_ctas_per_sm;  // exact matcher residency, 0 = default
    int match_chunks_per_cta;  // exact matcher work items per resident CTA, 0 = default
    unsigned long long* scan_status;  // zeroed look-back area of the scans (scan.cu)
    int64_t scan_words;
    char msg[256];
};

struct kmx_grid {
    kmx_ctx* ctx;           // compared, never dereferenced after kmx_destroy
    int device;             // device and stream the grid memory belongs to
    cudaStream_t stream;
    int64_t n_cap;
    const int64_t* d_n;     // actual count (caller's cell or grid-owned copy)
    float cell;
    double inv_cell;        // 1 / (cell * (1 + KMX_CELL_MARGIN))
    int64_t* d_n_sorted;    // points actually bucketed (device)
    uint32_t table_size;    // power of two
    unsigned long long* keys;  // [table_size] packed cell keys, ~0 = empty
    int2* cells;            // [table_size] (start, count) in sorted order
    float4* sorted;         // [n_cap] points in cell order, w = original index (int bits)
    int32_t* sslot;         // [n_cap] hash slot of each sorted point's cell
    const float4* pts;      // caller's points in original order
    int64_t* d_n_own;       // grid-owned count when the caller passed none
    void* mem;
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

#define KMX_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull
#define KMX_KEY_BIAS 1048576  // 2^20: 21-bit fields hold indices in (-2^20, 2^20)

// MurmurHash3 64-bit finaliser (public domain), used to spread packed keys.
__device__ __forceinline__ uint32_t kmx_hash64(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

__device__ __forceinline__ unsigned long long kmx_pack_key(int kx, int ky, int kz)
{
    return ((unsigned long long)(uint32_t)(kx + KMX_KEY_BIAS) << 42) |
           ((unsigned long long)(uint32_t)(ky + KMX_KEY_BIAS) << 21) |
           (unsigned long long)(uint32_t)(kz + KMX_KEY_BIAS);
}

// Open-addressing insert with linear probing; returns the slot or -1 when the
// table is full (at most table_size probes, so the loop always ends).
__device__ __forceinline__ int kmx_hash_insert(unsigned long long* keys, uint32_t size, unsigned long long key)
{
    uint32_t mask = size - 1u;
    uint32_t h = kmx_hash64(key) & mask;
    for (uint32_t probe = 0; probe < size; ++probe) {
        unsigned long long prev = atomicCAS(&keys[h], KMX_EMPTY_KEY, key);
        if (prev == KMX_EMPTY_KEY || prev == key) return (int)h;
        h = (h + 1u) & mask;
    }
    return -1;
}

// Lookup; returns the slot or -1 if the key is absent.
__device__ __forceinline__ int kmx_hash_find(const unsigned long long* __restrict__ keys, uint32_t size,
                                             unsigned long long key)
{
    uint32_t mask = size - 1u;
    uint32_t h = kmx_hash64(key) & mask;
    for (uint32_t probe = 0; probe < size; ++probe) {
        unsigned long long k = __ldg(&keys[h]);
        if (k == key) return (int)h;
        if (k == KMX_EMPTY_KEY) return -1;
        h = (h + 1u) & mask;
    }
    return -1;
}

__device__ __forceinline__ int64_t kmx_count(const int64_t* d_n, int64_t cap)
{
    if (!d_n) return cap;
    int64_t n = *d_n;
    return n < cap ? n : cap;
}

__device__ __forceinline__ void kmx_raise(unsigned int* err, unsigned int bit)
{
    atomicOr(err, bit);
}

// ---------------------------------------------------------------------------
// host-side launch helpers (defined in the .cu files)
// ---------------------------------------------------------------------------

static inline unsigned int kmx_blocks(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (unsigned int)b;
}

static inline size_t kmx_align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Blocks for a grid-stride kernel over at most `cap_items` items of which only
// a device-side count are real: enough for the capacity, but never more than
// `per_sm` resident blocks per SM (the rest would only be scheduled to exit).
static inline unsigned int kmx_stride_blocks(int64_t cap_items, int items_per_block, int sm_count, int per_sm = 8)
{
    const unsigned int b = kmx_blocks(cap_items, items_per_block);
    const unsigned int lim = (unsigned int)(per_sm * (sm_count > 0 ? sm_count : 1));
    return b < lim ? b : lim;
}

// Blocks for a grid-stride kernel, capped at one wave: the blocks of `kernel`
// (at `threads` threads, `smem` dynamic shared bytes) that fit on every SM at
// once, as its registers and shared memory allow.  Every block then starts at
// launch and takes an equal share of the items; a grid above one wave would
// leave its last blocks to run alone on a partly empty GPU.
template <typename Kernel>
static inline cudaError_t kmx_wave_blocks(Kernel kernel, int threads, size_t smem, int64_t cap_items,
                                          int items_per_block, int sm_count, unsigned int* blocks)
{
    int per_sm = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e) return e;
    *blocks = kmx_stride_blocks(cap_items, items_per_block, sm_count, per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

// Bump allocator over the context scratch.  With base == nullptr it only
// measures (every pointer it returns is null and `used` is the total).
struct kmx_arena {
    char* base;
    size_t used;
    void* take(size_t bytes)
    {
        used = kmx_align_up(used, 256);
        size_t off = used;
        used += bytes;
        return base ? static_cast<void*>(base + off) : nullptr;
    }
};

// One-time, per-device set-up actions (function attributes): bit `bit` of a
// per-device mask records that fn() succeeded on the current device.
enum { kmx_attr_fp32_tiles = 0, kmx_attr_tc_topk = 1, kmx_attr_fp32_bulk = 2, kmx_attr_gnc = 3, kmx_attr_ground = 4 };
template <typename F>
inline cudaError_t kmx_once_per_device(int bit, F fn)
{
    static std::atomic<unsigned long long> done[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return fn();
    const unsigned long long m = 1ull << bit;
    if (done[dev].load(std::memory_order_acquire) & m) return cudaSuccess;
    e = fn();
    if (e == cudaSuccess) done[dev].fetch_or(m, std::memory_order_release);
    return e;
}

// scan.cu: exclusive prefix sum of n int32 values (values at i >= *d_n count
// as 0) into out[0..n] (int64, out[n] = total), on the context stream.  One
// launch; its look-back status words come from the context's zeroed area,
// grown here when needed (so a first call of a size must not be inside a
// graph capture).  A look-back wait that runs out raises KMX_DERR_TIMEOUT.
cudaError_t kmx_scan_i32(kmx_ctx* ctx, const int32_t* in, int64_t n, const int64_t* d_n, int64_t* out);
// The same, but only out[0 .. min(*d_n, n)] are written (the tiles past the
// count do no work).
cudaError_t kmx_scan_i32_live(kmx_ctx* ctx, const int32_t* in, int64_t n, const int64_t* d_n, int64_t* out);
// Status words a scan of n values uses.
int64_t kmx_scan_words(int64_t n);
// Make the context's zeroed status area hold at least `words` words.
cudaError_t kmx_scan_reserve(kmx_ctx* ctx, int64_t words);

// sort.cu: stable LSD radix sort of the first min(*d_n, n) (key, value)
// pairs (all n when d_n is null) by the low `bits` bits of the key (8 per
// pass, rounded up), on the context stream; the result is in (keys, vals),
// or, with vals_out, the values are in vals_out (distinct from vals and
// vals_tmp; vals is then left unchanged and the keys end in either keys
// array).  Entries past the count are left alone.  scratch:
// kmx_sort_scratch_bytes(n).  Its scans use the context's look-back area
// (grown on first use of a size).
size_t kmx_sort_scratch_bytes(int64_t n);
cudaError_t kmx_sort_u32(kmx_ctx* ctx, uint32_t* keys, int32_t* vals, uint32_t* keys_tmp, int32_t* vals_tmp,
                         int64_t n, const int64_t* d_n, int bits, void* scratch, int32_t* vals_out = nullptr);

// voxel.cu
size_t kmx_voxelize_scratch_bytes(int64_t n_raw);
// d_n: nullable device count of the points actually present (<= n_raw)
cudaError_t kmx_voxelize_launch(kmx_ctx* ctx, const float* xyz, int64_t n_raw, const int64_t* d_n, int stride, float v,
                                float* out4, int64_t cap, int64_t* n_out, int32_t* assign, void* scratch);

// grid.cu
size_t kmx_grid_bytes(int64_t n_cap, uint32_t* table_size);
size_t kmx_grid_scratch_bytes(int64_t n_cap, uint32_t table_size);
cudaError_t kmx_grid_build_launch(kmx_ctx* ctx, kmx_grid* g, void* scratch);

// normals.cu
size_t kmx_normals_scratch_bytes(int64_t n_cap);
cudaError_t kmx_normals_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* p, float* normal4,
                               uint8_t* flags, int64_t* offs, int32_t* nbr, int64_t nbr_cap, int64_t* needed,
                               void* scratch);

// fpfh.cu
size_t kmx_fasterpfh_scratch_bytes(int64_t n_cap, bool need_spfh, int64_t nbr_cap);
cudaError_t kmx_fasterpfh_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* p, const float* normal4,
                                 uint8_t* flags, const int64_t* offs, const int32_t* nbr, int64_t nbr_cap,
                                 float* desc, int32_t* valid, int64_t* n_valid, float* spfh, void* scratch);

// ground.cu: geometric suppression; kmx_ground_bins_of is -1 for invalid
// parameters
int kmx_ground_bins_of(const kmx_ground_params* p);
size_t kmx_ground_scratch_bytes(int64_t n, int nb);
cudaError_t kmx_ground_launch(kmx_ctx* ctx, const float* xyz, int64_t n, int stride, const kmx_ground_params* prm,
                              float* out, int64_t* n_out, uint8_t* ground, double* planes, void* scratch);

// fpfh_search.cu: the classic FPFH baseline (classic = true) or the
// list-free Faster-PFH (classic = false)
size_t kmx_fpfh_search_scratch_bytes(int64_t n_cap, bool need_spfh);
cudaError_t kmx_fpfh_search_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* p, bool classic,
                                   float* normal4, uint8_t* flags, float* desc, int32_t* valid, int64_t* n_valid,
                                   float* spfh, void* scratch);

// prune.cu
size_t kmx_prune_scratch_bytes(int64_t corr_cap, int32_t n_tau);
cudaError_t kmx_prune_launch(kmx_ctx* ctx, const kmx_corr* corr, int64_t cap, const int64_t* d_n,
                             const float4* src4, const float4* tgt4, int32_t n_tau, double beta, int32_t* sel,
                             int64_t* n_sel, int32_t* core_out, int32_t* kmax, int32_t* inlier, int64_t* n_inlier,
                             void* scratch);

// gnc.cu
int64_t kmx_gnc_max_points();
cudaError_t kmx_gnc_launch(kmx_ctx* ctx, const kmx_corr* corr, const int32_t* sel, const int32_t* inlier,
                           const int64_t* d_n, int64_t cap, const float4* src4, const float4* tgt4, double noise_bound,
                           int max_iters, double mu_factor, double tol, double* R, double* t, float* w,
                           int32_t* stats);

// match_fp32.cu / match_tc.cu
size_t kmx_match_scratch_bytes(int64_t np_cap, int64_t nq_cap, int mode);
cudaError_t kmx_match_launch(kmx_ctx* ctx, const float* dp, const int32_t* vp, int64_t np_cap,
                             const int64_t* d_np, const float* dq, const int32_t* vq, int64_t nq_cap,
                             const int64_t* d_nq, int mode, kmx_corr* out, int64_t cap, int64_t* n_out,
                             void* scratch);
