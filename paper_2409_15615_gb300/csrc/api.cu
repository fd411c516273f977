// C ABI entry points of kmx.h: argument checks, scratch management and the
// launch sequences of each stage.  No entry point synchronises except
// kmx_sync / kmx_destroy, and none falls back to the CPU.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <new>

#include "kmx_internal.cuh"
#include "match_common.cuh"

namespace {

kmx_status fail(kmx_ctx* c, kmx_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
        va_end(ap);
    }
    return s;
}

kmx_status cuda_fail(kmx_ctx* c, cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation) return fail(c, KMX_ENOMEM, "%s: out of device memory", where);
    return fail(c, KMX_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Makes the context's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

kmx_status ensure_ws(kmx_ctx* c, size_t bytes)
{
    if (bytes <= c->ws_size && c->ws) return KMX_OK;
    size_t want = bytes > c->ws_size + c->ws_size / 2 ? bytes : c->ws_size + c->ws_size / 2;
    if (want < (1u << 20)) want = 1u << 20;
    if (c->ws) cudaFreeAsync(c->ws, c->stream);
    c->ws = nullptr;
    c->ws_size = 0;
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, want, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "scratch allocation");
    c->ws = p;
    c->ws_size = want;
    return KMX_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

kmx_status launched(kmx_ctx* c, cudaError_t e, const char* where)
{
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return KMX_OK;
}

// Polls a flag that nothing sets, a bounded number of times, then records a
// timeout: the bounded-wait pattern, exercised without any fault.
__global__ void bounded_wait(const volatile unsigned int* flag, long long polls, unsigned int* err)
{
    if (threadIdx.x != 0) return;
    for (long long i = 0; i < polls; ++i)
        if (*flag) return;
    atomicOr(err, KMX_DERR_TIMEOUT);
}

}  // namespace

std::atomic<long long> kmx_g_launches{0};

extern "C" {

int64_t kmx_launch_count(void) { return (int64_t)kmx_g_launches.load(std::memory_order_relaxed); }

kmx_status kmx_params_default(float v, kmx_params* out)
{
    if (!out || !(v > 0.0f) || !isfinite(v)) return KMX_EINVAL;
    out->voxel = v;
    out->r_normal = 3.5f * v;
    out->r_fpfh = 5.0f * v;
    out->tau_num = 3;
    out->tau_lin = 0.99f;
    out->hist_bins = 11;
    out->viewpoint[0] = out->viewpoint[1] = out->viewpoint[2] = 0.0f;
    return KMX_OK;
}

kmx_status kmx_create(kmx_ctx** out, int device, void* cuda_stream)
{
    if (!out) return KMX_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return KMX_EINVAL;
    DeviceGuard g(device);
    if (!g.ok) return KMX_ECUDA;
    kmx_ctx* c = new (std::nothrow) kmx_ctx();
    if (!c) return KMX_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    // the error word is cleared on the context's stream, and waited for, so
    // that no kernel of the context can run before it is zero
    if (cudaMalloc(&c->d_err, sizeof(unsigned int)) != cudaSuccess ||
        cudaMallocHost(&c->h_err, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        if (c->d_err) cudaFree(c->d_err);
        if (c->h_err) cudaFreeHost(c->h_err);
        delete c;
        return KMX_ENOMEM;
    }
    *c->h_err = 0;
    c->msg[0] = 0;
    *out = c;
    return KMX_OK;
}

void kmx_destroy(kmx_ctx* c)
{
    if (!c) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->ws) cudaFree(c->ws);
    if (c->scan_status) cudaFree(c->scan_status);
    cudaFree(c->d_err);
    cudaFreeHost(c->h_err);
    delete c;
}

kmx_status kmx_set_stream(kmx_ctx* c, void* cuda_stream)
{
    if (!c) return KMX_EINVAL;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    return KMX_OK;
}

kmx_status kmx_set_match_residency(kmx_ctx* c, int ctas_per_sm)
{
    if (!c || ctas_per_sm < 0 || ctas_per_sm > 2) return KMX_EINVAL;
    c->match_ctas_per_sm = ctas_per_sm;
    return KMX_OK;
}

kmx_status kmx_set_match_chunks(kmx_ctx* c, int chunks_per_cta)
{
    if (!c || chunks_per_cta < 0 || chunks_per_cta > 32) return KMX_EINVAL;
    c->match_chunks_per_cta = chunks_per_cta;
    return KMX_OK;
}

kmx_status kmx_reserve(kmx_ctx* c, int64_t bytes)
{
    if (!c || bytes < 0) return KMX_EINVAL;
    DeviceGuard g(c->device);
    return ensure_ws(c, (size_t)bytes);
}

kmx_status kmx_sync(kmx_ctx* c)
{
    if (!c) return KMX_EINVAL;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "kmx_sync");
    e = cudaMemcpy(c->h_err, c->d_err, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "kmx_sync");
    const unsigned int bits = *c->h_err;
    if (!bits) return KMX_OK;
    // clear on the context's own stream (a non-blocking stream is not ordered
    // against the legacy default stream) and wait, so that the next call's
    // kernels start from zeros; a scan that gave up may have left its status
    // words set
    e = cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess && c->scan_status)
        e = cudaMemsetAsync(c->scan_status, 0, sizeof(unsigned long long) * (size_t)c->scan_words, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "kmx_sync");
    if (bits & KMX_DERR_RANGE) return fail(c, KMX_ERANGE, "a voxel or cell index does not fit in 21 bits");
    if (bits & KMX_DERR_CAPACITY) return fail(c, KMX_ECAPACITY, "an output buffer is too small");
    if (bits & KMX_DERR_HASHFULL) return fail(c, KMX_ENOMEM, "hash table full");
    if (bits & KMX_DERR_TIMEOUT) return fail(c, KMX_ETIMEOUT, "device wait timed out");
    return fail(c, KMX_ECUDA, "unknown device error bits 0x%x", bits);
}

const char* kmx_last_error(const kmx_ctx* c) { return c ? c->msg : "null context"; }

kmx_status kmx_check_timeout(kmx_ctx* c, int64_t polls)
{
    if (!c) return KMX_EINVAL;
    if (polls < 1 || polls > (1ll << 24)) return fail(c, KMX_EINVAL, "kmx_check_timeout: polls out of range");
    DeviceGuard g(c->device);
    kmx_status s = ensure_ws(c, 256);
    if (s) return s;
    unsigned int* flag = static_cast<unsigned int*>(c->ws);
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), c->stream);
    if (e) return cuda_fail(c, e, "kmx_check_timeout");
    KMX_COUNT_LAUNCH();
    bounded_wait<<<1, 32, 0, c->stream>>>(flag, (long long)polls, c->d_err);
    return launched(c, cudaGetLastError(), "kmx_check_timeout");
}

kmx_status kmx_voxelize(kmx_ctx* c, const float* d_xyz, int64_t n_raw, int32_t stride, float voxel, float* d_out4,
                        int64_t cap, int64_t* d_n_out, int32_t* d_assign)
{
    if (!c) return KMX_EINVAL;
    if (n_raw < 0 || n_raw > INT32_MAX - 1 || (stride != 3 && stride != 4) || !(voxel > 0.0f) || !isfinite(voxel) ||
        cap < 0 || !d_n_out || (n_raw > 0 && (!d_xyz || !d_out4)) || (d_out4 && !aligned16(d_out4)))
        return fail(c, KMX_EINVAL, "kmx_voxelize: bad argument");
    DeviceGuard g(c->device);
    kmx_status s = ensure_ws(c, kmx_voxelize_scratch_bytes(n_raw));
    if (s) return s;
    return launched(c,
                    kmx_voxelize_launch(c, d_xyz, n_raw, nullptr, stride, voxel, d_out4, cap, d_n_out, d_assign,
                                        c->ws),
                    "kmx_voxelize");
}

kmx_status kmx_voxelize_count(kmx_ctx* c, const float* d_xyz, int64_t n_cap, const int64_t* d_n_raw, int32_t stride,
                              float voxel, float* d_out4, int64_t cap, int64_t* d_n_out, int32_t* d_assign)
{
    if (!c) return KMX_EINVAL;
    if (n_cap < 0 || n_cap > INT32_MAX - 1 || !d_n_raw || (stride != 3 && stride != 4) || !(voxel > 0.0f) ||
        !isfinite(voxel) || cap < 0 || !d_n_out || (n_cap > 0 && (!d_xyz || !d_out4)) || (d_out4 && !aligned16(d_out4)))
        return fail(c, KMX_EINVAL, "kmx_voxelize_count: bad argument");
    DeviceGuard g(c->device);
    kmx_status s = ensure_ws(c, kmx_voxelize_scratch_bytes(n_cap));
    if (s) return s;
    return launched(c,
                    kmx_voxelize_launch(c, d_xyz, n_cap, d_n_raw, stride, voxel, d_out4, cap, d_n_out, d_assign,
                                        c->ws),
                    "kmx_voxelize_count");
}

kmx_status kmx_ground_params_default(kmx_ground_params* out)
{
    if (!out) return KMX_EINVAL;
    const float zr[5] = {2.7f, 12.3f, 22.1f, 41.1f, 80.0f};
    const int32_t rings[4] = {2, 4, 4, 4}, sectors[4] = {16, 32, 54, 32};
    for (int k = 0; k < 5; ++k) out->zone_r[k] = zr[k];
    for (int k = 0; k < 4; ++k) {
        out->zone_rings[k] = rings[k];
        out->zone_sectors[k] = sectors[k];
    }
    out->quant_log2 = 8;
    out->z_limit = 80.0f;
    out->n_lpr = 20;
    out->th_seeds = 0.125f;
    out->th_dist = 0.125f;
    out->n_iter = 3;
    out->max_slope = 1.0f;
    out->max_ground_z = -0.8f;
    out->min_points = 10;
    out->max_bin_points = 65536;
    return KMX_OK;
}

int32_t kmx_ground_bins(const kmx_ground_params* p) { return kmx_ground_bins_of(p); }

kmx_status kmx_suppress_ground(kmx_ctx* c, const float* d_xyz, int64_t n, int32_t stride, const kmx_ground_params* p,
                               float* d_out, int64_t* d_n_out, uint8_t* d_ground, double* d_planes)
{
    if (!c) return KMX_EINVAL;
    const int nb = kmx_ground_bins_of(p);
    if (nb < 0) return fail(c, KMX_EINVAL, "kmx_suppress_ground: bad parameters");
    if (n < 0 || n > INT32_MAX - 1 || (stride != 3 && stride != 4) || !d_n_out || (n > 0 && (!d_xyz || !d_out)) ||
        (n > 0 && d_out == d_xyz))
        return fail(c, KMX_EINVAL, "kmx_suppress_ground: bad argument");
    DeviceGuard g(c->device);
    kmx_status s = ensure_ws(c, kmx_ground_scratch_bytes(n, nb));
    if (s) return s;
    return launched(c, kmx_ground_launch(c, d_xyz, n, stride, p, d_out, d_n_out, d_ground, d_planes, c->ws),
                    "kmx_suppress_ground");
}

kmx_status kmx_build_grid(kmx_ctx* c, const float* d_xyz4, int64_t n_cap, const int64_t* d_n, float cell,
                          kmx_grid** out)
{
    if (!c) return KMX_EINVAL;
    if (!out || n_cap < 0 || n_cap > INT32_MAX - 1 || !(cell > 0.0f) || !isfinite(cell) ||
        (n_cap > 0 && !d_xyz4) || (d_xyz4 && !aligned16(d_xyz4)))
        return fail(c, KMX_EINVAL, "kmx_build_grid: bad argument");
    DeviceGuard dg(c->device);
    if (*out) {  // rebuild in place: same context, enough capacity, no allocation
        kmx_grid* g = *out;
        if (g->ctx != c || g->n_cap < n_cap) return fail(c, KMX_EINVAL, "kmx_build_grid: grid cannot be reused");
        g->d_n = d_n;
        g->cell = cell;
        g->pts = reinterpret_cast<const float4*>(d_xyz4);
        g->stream = c->stream;
        kmx_status s = ensure_ws(c, kmx_grid_scratch_bytes(g->n_cap, g->table_size));
        if (s != KMX_OK) return s;
        return launched(c, kmx_grid_build_launch(c, g, c->ws), "kmx_build_grid");
    }
    kmx_grid* g = new (std::nothrow) kmx_grid();
    if (!g) return KMX_ENOMEM;
    g->ctx = c;
    g->device = c->device;
    g->stream = c->stream;
    g->n_cap = n_cap;
    g->d_n = d_n;
    g->cell = cell;
    g->pts = reinterpret_cast<const float4*>(d_xyz4);
    uint32_t T = 0;
    const size_t bytes = kmx_grid_bytes(n_cap, &T);
    g->table_size = T;
    cudaError_t e = cudaMallocAsync(&g->mem, bytes, c->stream);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(c, e, "kmx_build_grid");
    }
    kmx_arena a{static_cast<char*>(g->mem), 0};
    g->keys = (unsigned long long*)a.take(sizeof(unsigned long long) * T);
    g->cells = (int2*)a.take(sizeof(int2) * T);
    g->sorted = (float4*)a.take(sizeof(float4) * (n_cap + 1));
    g->sslot = (int32_t*)a.take(sizeof(int32_t) * (n_cap + 1));
    g->d_n_own = (int64_t*)a.take(sizeof(int64_t));
    g->d_n_sorted = (int64_t*)a.take(sizeof(int64_t));
    kmx_status s = ensure_ws(c, kmx_grid_scratch_bytes(n_cap, T));
    if (s == KMX_OK) s = launched(c, kmx_grid_build_launch(c, g, c->ws), "kmx_build_grid");
    if (s != KMX_OK) {
        cudaFreeAsync(g->mem, c->stream);
        delete g;
        return s;
    }
    *out = g;
    return KMX_OK;
}

void kmx_grid_free(kmx_grid* g)
{
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaFreeAsync(g->mem, g->stream);
    delete g;
}

static kmx_status check_params(kmx_ctx* c, const kmx_grid* g, const kmx_params* p, const char* who)
{
    if (!g || !p) return fail(c, KMX_EINVAL, "%s: null grid or params", who);
    if (!(p->r_fpfh > 0.0f) || !(p->r_normal > 0.0f) || p->r_normal > p->r_fpfh || !isfinite(p->r_fpfh))
        return fail(c, KMX_EINVAL, "%s: need 0 < r_normal <= r_fpfh", who);
    if (g->cell < p->r_fpfh) return fail(c, KMX_EINVAL, "%s: grid cell %g < r_fpfh %g", who, g->cell, p->r_fpfh);
    if (p->hist_bins != 11) return fail(c, KMX_EINVAL, "%s: only 11 bins per feature are supported", who);
    if (p->tau_num < 0 || !(p->tau_lin >= 0.0f)) return fail(c, KMX_EINVAL, "%s: bad thresholds", who);
    if (g->ctx != c) return fail(c, KMX_EINVAL, "%s: grid belongs to another context", who);
    return KMX_OK;
}

kmx_status kmx_normals(kmx_ctx* c, const kmx_grid* g, const kmx_params* p, float* d_normal4, uint8_t* d_flags,
                       int64_t* d_nbr_offs, int32_t* d_nbr, int64_t nbr_cap, int64_t* d_needed)
{
    if (!c) return KMX_EINVAL;
    kmx_status s = check_params(c, g, p, "kmx_normals");
    if (s) return s;
    if (!d_normal4 || !aligned16(d_normal4) || !d_flags || !d_nbr_offs || !d_needed || nbr_cap < 0)
        return fail(c, KMX_EINVAL, "kmx_normals: bad argument");
    DeviceGuard dg(c->device);
    s = ensure_ws(c, kmx_normals_scratch_bytes(g->n_cap));
    if (s) return s;
    return launched(c,
                    kmx_normals_launch(c, g, p, d_normal4, d_flags, d_nbr_offs, d_nbr, nbr_cap, d_needed, c->ws),
                    "kmx_normals");
}

kmx_status kmx_fasterpfh(kmx_ctx* c, const kmx_grid* g, const kmx_params* p, const float* d_normal4,
                         uint8_t* d_flags, const int64_t* d_nbr_offs, const int32_t* d_nbr, int64_t nbr_cap,
                         float* d_desc, int32_t* d_valid, int64_t* d_n_valid, float* d_spfh)
{
    if (!c) return KMX_EINVAL;
    kmx_status s = check_params(c, g, p, "kmx_fasterpfh");
    if (s) return s;
    if (!d_normal4 || !aligned16(d_normal4) || !d_flags || !d_nbr_offs || !d_nbr || nbr_cap < 0 || !d_desc ||
        !aligned16(d_desc) || !d_valid || !d_n_valid || (d_spfh && !aligned16(d_spfh)))
        return fail(c, KMX_EINVAL, "kmx_fasterpfh: bad argument");
    DeviceGuard dg(c->device);
    s = ensure_ws(c, kmx_fasterpfh_scratch_bytes(g->n_cap, d_spfh == nullptr, nbr_cap));
    if (s) return s;
    return launched(c,
                    kmx_fasterpfh_launch(c, g, p, d_normal4, d_flags, d_nbr_offs, d_nbr, nbr_cap, d_desc, d_valid,
                                         d_n_valid, d_spfh, c->ws),
                    "kmx_fasterpfh");
}

static kmx_status fpfh_search(kmx_ctx* c, const kmx_grid* g, const kmx_params* p, bool classic, float* d_normal4,
                              uint8_t* d_flags, float* d_desc, int32_t* d_valid, int64_t* d_n_valid, float* d_spfh,
                              const char* who)
{
    if (!c) return KMX_EINVAL;
    kmx_status s = check_params(c, g, p, who);
    if (s) return s;
    if (!d_normal4 || !aligned16(d_normal4) || !d_flags || !d_desc || !aligned16(d_desc) || !d_valid || !d_n_valid ||
        (d_spfh && !aligned16(d_spfh)))
        return fail(c, KMX_EINVAL, "%s: bad argument", who);
    DeviceGuard dg(c->device);
    s = ensure_ws(c, kmx_fpfh_search_scratch_bytes(g->n_cap, d_spfh == nullptr));
    if (s) return s;
    return launched(c,
                    kmx_fpfh_search_launch(c, g, p, classic, d_normal4, d_flags, d_desc, d_valid, d_n_valid, d_spfh,
                                           c->ws),
                    who);
}

kmx_status kmx_features(kmx_ctx* c, const kmx_grid* g, const kmx_params* p, float* d_normal4, uint8_t* d_flags,
                        float* d_desc, int32_t* d_valid, int64_t* d_n_valid, float* d_spfh)
{
    return fpfh_search(c, g, p, false, d_normal4, d_flags, d_desc, d_valid, d_n_valid, d_spfh, "kmx_features");
}

kmx_status kmx_fpfh_classic(kmx_ctx* c, const kmx_grid* g, const kmx_params* p, float* d_normal4, uint8_t* d_flags,
                            float* d_desc, int32_t* d_valid, int64_t* d_n_valid, float* d_spfh)
{
    return fpfh_search(c, g, p, true, d_normal4, d_flags, d_desc, d_valid, d_n_valid, d_spfh, "kmx_fpfh_classic");
}

kmx_status kmx_prune(kmx_ctx* c, const kmx_corr* d_corr, int64_t corr_cap, const int64_t* d_n_corr,
                     const float* d_src4, const float* d_tgt4, int32_t n_tau, double beta, int32_t* d_sel,
                     int64_t* d_n_sel, int32_t* d_core, int32_t* d_kmax, int32_t* d_inlier, int64_t* d_n_inlier)
{
    if (!c) return KMX_EINVAL;
    if (corr_cap < 0 || corr_cap > INT32_MAX - 1 || (corr_cap > 0 && !d_corr) || !d_src4 || !aligned16(d_src4) ||
        !d_tgt4 || !aligned16(d_tgt4) || n_tau < 1 || n_tau > 16384 || !(beta > 0.0) || !std::isfinite(beta) ||
        !d_sel || !d_n_sel || !d_core || !d_kmax || !d_inlier || !d_n_inlier)
        return fail(c, KMX_EINVAL, "kmx_prune: bad argument");
    DeviceGuard dg(c->device);
    kmx_status s = ensure_ws(c, kmx_prune_scratch_bytes(corr_cap, n_tau));
    if (s) return s;
    return launched(c,
                    kmx_prune_launch(c, d_corr, corr_cap, d_n_corr, reinterpret_cast<const float4*>(d_src4),
                                     reinterpret_cast<const float4*>(d_tgt4), n_tau, beta, d_sel, d_n_sel, d_core,
                                     d_kmax, d_inlier, d_n_inlier, c->ws),
                    "kmx_prune");
}

kmx_status kmx_gnc(kmx_ctx* c, const kmx_corr* d_corr, const int32_t* d_sel, const int32_t* d_inlier,
                   const int64_t* d_n_inlier, int64_t inlier_cap, const float* d_src4, const float* d_tgt4,
                   double noise_bound, int32_t max_iters, double mu_factor, double tol, double* d_R, double* d_t,
                   float* d_w, int32_t* d_stats)
{
    if (!c) return KMX_EINVAL;
    if (!d_corr || !d_sel || !d_inlier || inlier_cap < 0 || inlier_cap > kmx_gnc_max_points() || !d_src4 ||
        !aligned16(d_src4) || !d_tgt4 || !aligned16(d_tgt4) || !(noise_bound > 0.0) || !std::isfinite(noise_bound) ||
        max_iters < 0 || !(mu_factor > 1.0) || !std::isfinite(mu_factor) || !(tol >= 0.0) || !d_R || !d_t ||
        (inlier_cap > 0 && !d_w) || !d_stats)
        return fail(c, KMX_EINVAL, "kmx_gnc: bad argument");
    DeviceGuard dg(c->device);
    return launched(c,
                    kmx_gnc_launch(c, d_corr, d_sel, d_inlier, d_n_inlier, inlier_cap,
                                   reinterpret_cast<const float4*>(d_src4), reinterpret_cast<const float4*>(d_tgt4),
                                   noise_bound, max_iters, mu_factor, tol, d_R, d_t, d_w, d_stats),
                    "kmx_gnc");
}

kmx_status kmx_match(kmx_ctx* c, const float* d_desc_p, const int32_t* d_valid_p, int64_t np_cap,
                     const int64_t* d_np, const float* d_desc_q, const int32_t* d_valid_q, int64_t nq_cap,
                     const int64_t* d_nq, int32_t mode, kmx_corr* d_out, int64_t cap, int64_t* d_n_out)
{
    if (!c) return KMX_EINVAL;
    if (np_cap < 0 || nq_cap < 0 || np_cap > INT32_MAX - 1 || nq_cap > INT32_MAX - 1 || cap < 0 || !d_n_out ||
        (np_cap > 0 && (!d_desc_p || !aligned16(d_desc_p))) || (nq_cap > 0 && (!d_desc_q || !aligned16(d_desc_q))) ||
        (cap > 0 && !d_out))
        return fail(c, KMX_EINVAL, "kmx_match: bad argument");
    if (mode != KMX_MATCH_FP32_EXACT && mode != KMX_MATCH_BF16_RERANK)
        return fail(c, KMX_EINVAL, "kmx_match: unknown mode %d", mode);
    DeviceGuard dg(c->device);
    return launched(c,
                    kmx_match_launch(c, d_desc_p, d_valid_p, np_cap, d_np, d_desc_q, d_valid_q, nq_cap, d_nq, mode,
                                     d_out, cap, d_n_out, nullptr),
                    "kmx_match");
}

kmx_status kmx_match_diag(kmx_ctx* c, int64_t np_cap, const int64_t* d_np, int64_t nq_cap, const int64_t* d_nq,
                          int64_t* d_out)
{
    if (!c) return KMX_EINVAL;
    if (np_cap <= 0 || nq_cap <= 0 || np_cap > INT32_MAX - 1 || nq_cap > INT32_MAX - 1 || !d_out)
        return fail(c, KMX_EINVAL, "kmx_match_diag: bad argument");
    const size_t extra = kmx_match_tc_extra_bytes(np_cap, nq_cap, c->sm_count);
    if (kmx::match_common_bytes(np_cap, nq_cap, 1, extra) > c->ws_size)
        return fail(c, KMX_EINVAL, "kmx_match_diag: no tensor-core match of these capacities on this context");
    DeviceGuard dg(c->device);
    kmx::MatchScratch s = kmx::match_common_carve(c->ws, np_cap, nq_cap, 1, extra);
    return launched(c, kmx_match_tc_stats(c, s.extra, np_cap, d_np, nq_cap, d_nq, d_out), "kmx_match_diag");
}

}  // extern "C"

// Matching dispatch (scratch is taken from the context here because the size
// depends on the mode).
cudaError_t kmx_match_launch(kmx_ctx* c, const float* dp, const int32_t* vp, int64_t np_cap, const int64_t* d_np,
                             const float* dq, const int32_t* vq, int64_t nq_cap, const int64_t* d_nq, int mode,
                             kmx_corr* out, int64_t cap, int64_t* n_out, void*)
{
    cudaStream_t st = c->stream;
    if (np_cap == 0 || nq_cap == 0) {
        return cudaMemsetAsync(n_out, 0, sizeof(int64_t), st);
    }
    if (mode == KMX_MATCH_FP32_EXACT) {
        const size_t extra = kmx_match_fp32_bulk_extra_bytes(np_cap, nq_cap, c->sm_count);
        const size_t bytes = kmx::match_common_bytes(np_cap, nq_cap, 1, extra);
        if (ensure_ws(c, bytes) != KMX_OK) return cudaErrorMemoryAllocation;
        kmx::MatchScratch s = kmx::match_common_carve(c->ws, np_cap, nq_cap, 1, extra);
        return kmx_match_fp32_bulk_launch(c, dp, vp, np_cap, d_np, dq, vq, nq_cap, d_nq, s, out, cap, n_out);
    }
    if (mode == KMX_MATCH_BF16_RERANK) {
        const size_t extra = kmx_match_tc_extra_bytes(np_cap, nq_cap, c->sm_count);
        const size_t bytes = kmx::match_common_bytes(np_cap, nq_cap, 1, extra);
        if (ensure_ws(c, bytes) != KMX_OK) return cudaErrorMemoryAllocation;
        kmx::MatchScratch s = kmx::match_common_carve(c->ws, np_cap, nq_cap, 1, extra);
        cudaError_t e = cudaMemsetAsync(s.colbest, 0xFF, sizeof(unsigned long long) * nq_cap, st);
        if (e) return e;
        if ((e = kmx_match_tc_launch(c, dp, np_cap, d_np, dq, nq_cap, d_nq, s))) return e;
        return kmx::match_finalize(c, s, np_cap, d_np, vp, vq, out, cap, n_out);
    }
    return cudaErrorNotSupported;
}
