// Algorithm 1, step 1 (Sec. III-C, App. A): one radius search per point with
// r_FPFH (Eq. A1), the r_normal subsample P_normal, PCA normal and linearity,
// and the reliability flag B.
//
// Queries are taken in cell order so that neighbouring threads or warps walk
// the same cells (their candidate loads coincide or share cache lines).  The
// kernels pick one of two layouts from the device point count, the same way in
// every launch (kThreadQueryMin, search_common.cuh):
//  - large clouds: one thread per query.  The thread walks its 27-cell stencil
//    in the order of the stored lists and sums in that order.
//  - small clouds (too few queries to fill the GPU one per thread): one warp
//    per query.  The 27 stencil cells are looked up by 27 lanes at once, their
//    candidate ranges are flattened into one index space, and all 32 lanes
//    test candidates.
// Two passes: the first counts |I| and accumulates the P_normal mean; after a
// prefix sum of the counts the second writes the CSR lists and accumulates
// the covariance centred on that mean.
//
// The 3x3 eigen-problem starts from the closed form (Smith 1961:
// trigonometric eigenvalues) in FP32, refines the well-separated extreme
// eigenvalue by FP64 Newton steps on the characteristic polynomial and takes
// the other two from a quadratic in FP64; the normal is the best-conditioned
// cross product of two rows of A - l3 I in FP64 (search_common.cuh).  GB300 issues FP64
// at a small fraction of the FP32 rate and a warp instruction costs the same
// with 1 or 32 active lanes, so the search stores each query's moments and a
// separate pass solves them one query per thread.
#include "search_common.cuh"

using namespace kmxs;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kQPerWarp = 4;                    // queries per warp in the warp-per-query fill pass
constexpr int kQPerBlock = kWarps * kQPerWarp;  // = 32, queries per block per step in that mode

struct NormScratch {
    int32_t* cnt;    // [n+1] |I(q)|
    float4* mean;    // [n] P_normal mean minus the query point; w = |P_normal| (int bits)
    float4* mom;     // [n][3] centred moments s1x s1y s1z sxx | sxy sxz syy syz | szz - - -
};

NormScratch carve(void* base, int64_t n, size_t* total)
{
    NormScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.cnt = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.mean = (float4*)a.take(sizeof(float4) * (n + 1));
    s.mom = (float4*)a.take(sizeof(float4) * 3 * (n + 1));
    *total = kmx_align_up(a.used, 256);
    return s;
}

// Pass 1: |I(q)|, |P_normal| and the P_normal mean (relative to q), per
// sorted position.
__global__ void __launch_bounds__(kThreads) search_count(GridView g, Radii R, NormScratch s)
{
    const int lane = threadIdx.x & 31;
    const int64_t n_sorted = *g.n_sorted;
    if (n_sorted < kThreadQueryMin) {  // one warp per query
        const int64_t warps = (int64_t)gridDim.x * kWarps;
        for (int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); w * kQPerWarp < n_sorted; w += warps) {
            StencilCache sc;
            for (int k = 0; k < kQPerWarp && w * kQPerWarp + k < n_sorted; ++k) {
                const float4 q = g.sorted[w * kQPerWarp + k];
                const int qi = __float_as_int(q.w);
                const int total = sc.get(g, w * kQPerWarp + k, lane);
                const int start = sc.start, excl = sc.excl;
                int nf = 0, nn = 0;
                float sx = 0.f, sy = 0.f, sz = 0.f;
                for (int base = 0; base < total; base += 32) {
                    const int t = base + lane;
                    const int pos = candidate(t, start, excl);
                    bool inF = false, inN = false;
                    float dx = 0.f, dy = 0.f, dz = 0.f;
                    if (t < total) {
                        const float4 a = g.sorted[pos];
                        dx = a.x - q.x;
                        dy = a.y - q.y;
                        dz = a.z - q.z;
                        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        inF = within(a, q, d2, R.rf2, R.rf2d);
                        inN = inF && within(a, q, d2, R.rn2, R.rn2d);
                    }
                    nf += __popc(__ballot_sync(kFull, inF));
                    nn += __popc(__ballot_sync(kFull, inN));
                    if (inN) {
                        sx += dx;
                        sy += dy;
                        sz += dz;
                    }
                }
                sx = warp_sum(sx);
                sy = warp_sum(sy);
                sz = warp_sum(sz);
                if (lane == 0) {
                    s.cnt[qi] = nf;
                    const float inv = nn > 0 ? 1.0f / (float)nn : 0.0f;
                    s.mean[qi] = make_float4(sx * inv, sy * inv, sz * inv, __int_as_float(nn));
                }
            }
        }
        return;
    }
    // one thread per query
    for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < n_sorted; p += (int64_t)gridDim.x * kThreads) {
        const float4 q = g.sorted[p];
        const int qi = __float_as_int(q.w);
        const Sweep1 r = sweep1(g, R, p, q);
        s.cnt[qi] = r.nf;
        const float inv = r.nn > 0 ? 1.0f / (float)r.nn : 0.0f;
        s.mean[qi] = make_float4(r.sx * inv, r.sy * inv, r.sz * inv, __int_as_float(r.nn));
    }
}

struct NormOut {
    float4* normal4;
    uint8_t* flags;
    const int64_t* offs;
    int32_t* nbr;
    int64_t nbr_cap;
    int64_t n_cap;
    int64_t* needed;
    int tau_num;
    float tau_lin;
    float vp[3];
};

// Pass 2: CSR lists and centred second moments over P_normal per sorted
// position; the moments go to scratch for solve_normals.  Five blocks per SM
// (a few registers spilled): no faster alone, but faster beside the other
// cloud's kernels on a second stream.
__global__ void __launch_bounds__(kThreads, 5) search_fill(GridView g, Radii R, NormScratch s, NormOut o,
                                                           unsigned int* err)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t total_list = o.offs[o.n_cap];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *o.needed = total_list;
        if (o.nbr && total_list > o.nbr_cap) kmx_raise(err, KMX_DERR_CAPACITY);
    }
    const bool write = o.nbr && total_list <= o.nbr_cap;
    const int64_t n_sorted = *g.n_sorted;
    if (n_sorted < kThreadQueryMin) {  // one warp per query
        for (int64_t chunk = blockIdx.x; chunk * kQPerBlock < n_sorted; chunk += gridDim.x) {
            StencilCache sc;  // the warp's queries are consecutive in cell order
            for (int k = 0; k < kQPerWarp; ++k) {
                const int slot = warp * kQPerWarp + k;
                const int64_t p = chunk * kQPerBlock + slot;
                if (p >= n_sorted) break;
                const float4 q = g.sorted[p];
                const int qi = __float_as_int(q.w);
                const float4 mq = s.mean[qi];
                const int total = sc.get(g, p, lane);
                const int start = sc.start, excl = sc.excl;
                int64_t out = o.offs[qi];
                float s1x = 0.f, s1y = 0.f, s1z = 0.f;
                float sxx = 0.f, sxy = 0.f, sxz = 0.f, syy = 0.f, syz = 0.f, szz = 0.f;
                for (int base = 0; base < total; base += 32) {
                    const int t = base + lane;
                    const int pos = candidate(t, start, excl);
                    bool inF = false, inN = false;
                    float dx = 0.f, dy = 0.f, dz = 0.f;
                    int idx = 0;
                    if (t < total) {
                        const float4 a = g.sorted[pos];
                        idx = __float_as_int(a.w);
                        dx = a.x - q.x;
                        dy = a.y - q.y;
                        dz = a.z - q.z;
                        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        inF = within(a, q, d2, R.rf2, R.rf2d);
                        inN = inF && within(a, q, d2, R.rn2, R.rn2d);
                    }
                    const unsigned bal = __ballot_sync(kFull, inF);
                    if (inF && write) o.nbr[out + __popc(bal & ((1u << lane) - 1u))] = idx;
                    out += __popc(bal);
                    if (inN) {
                        const float ex = dx - mq.x, ey = dy - mq.y, ez = dz - mq.z;
                        s1x += ex;
                        s1y += ey;
                        s1z += ez;
                        sxx = fmaf(ex, ex, sxx);
                        sxy = fmaf(ex, ey, sxy);
                        sxz = fmaf(ex, ez, sxz);
                        syy = fmaf(ey, ey, syy);
                        syz = fmaf(ey, ez, syz);
                        szz = fmaf(ez, ez, szz);
                    }
                }
                s1x = warp_sum(s1x);
                s1y = warp_sum(s1y);
                s1z = warp_sum(s1z);
                sxx = warp_sum(sxx);
                sxy = warp_sum(sxy);
                sxz = warp_sum(sxz);
                syy = warp_sum(syy);
                syz = warp_sum(syz);
                szz = warp_sum(szz);
                if (lane == 0) {
                    float4* m = s.mom + 3 * (int64_t)qi;
                    m[0] = make_float4(s1x, s1y, s1z, sxx);
                    m[1] = make_float4(sxy, sxz, syy, syz);
                    m[2] = make_float4(szz, 0.f, 0.f, 0.f);
                }
            }
        }
        return;
    }
    // one thread per query
    for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < n_sorted; p += (int64_t)gridDim.x * kThreads) {
        const float4 q = g.sorted[p];
        const int qi = __float_as_int(q.w);
        const float4 mq = s.mean[qi];
        float mom[9];
        sweep2(g, R, p, q, mq.x, mq.y, mq.z, mom, write ? o.nbr + o.offs[qi] : nullptr);
        float4* m = s.mom + 3 * (int64_t)qi;
        m[0] = make_float4(mom[0], mom[1], mom[2], mom[3]);
        m[1] = make_float4(mom[4], mom[5], mom[6], mom[7]);
        m[2] = make_float4(mom[8], 0.f, 0.f, 0.f);
    }
}

// Pass 3: per bucketed point (one per thread), the FP64 eigen-solve of its
// moments, orientation toward the viewpoint and the linearity test.
__global__ void __launch_bounds__(kThreads) solve_normals(GridView g, NormScratch s, NormOut o)
{
    const int64_t n_sorted = *g.n_sorted;
    for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < n_sorted; p += (int64_t)gridDim.x * kThreads) {
        const float4 q = g.sorted[p];
        const int qi = __float_as_int(q.w);
        const int nN = __float_as_int(s.mean[qi].w);
        const int mF = (int)(o.offs[qi + 1] - o.offs[qi]);
        uint8_t flag = 0;
        float4 nout = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mF >= o.tau_num && nN >= o.tau_num) {
            const float4* m = s.mom + 3 * (int64_t)qi;
            const float4 m0 = m[0], m1 = m[1], m2 = m[2];
            float mom[9] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x};
            double plin;
            flag |= 4;
            if (normal_from_moments(mom, nN, q.x, q.y, q.z, o.vp, &nout, &plin) && plin < (double)o.tau_lin)
                flag |= 1;
        }
        o.normal4[qi] = nout;
        o.flags[qi] = flag;
    }
}

// Zero the counts |I(q)| of the actual points, and the normals and flags of
// the whole capacity: points that a range error kept out of the grid keep
// zeros, the others are written by search_fill.
__global__ void clear_counts(int32_t* cnt, float4* normal4, uint8_t* flags, const int64_t* d_n, int64_t n_cap)
{
    const int64_t n = kmx_count(d_n, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_cap; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) cnt[i] = 0;
        normal4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        flags[i] = 0;
    }
}

// When the lists did not fit (search_fill wrote none of them), every offset
// becomes 0: a later stage then reads empty lists instead of entries past
// the end of the list buffer.  `needed` (the full length) is left for the
// caller to size the buffer.
__global__ void empty_lists_on_overflow(int64_t* offs, int64_t n_cap, const int64_t* needed, int64_t nbr_cap)
{
    if (*needed <= nbr_cap) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_cap; i += (int64_t)gridDim.x * blockDim.x)
        offs[i] = 0;
}

}  // namespace

size_t kmx_normals_scratch_bytes(int64_t n_cap)
{
    size_t total = 0;
    carve(nullptr, n_cap, &total);
    return total;
}

cudaError_t kmx_normals_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* prm, float* normal4,
                               uint8_t* flags, int64_t* offs, int32_t* nbr, int64_t nbr_cap, int64_t* needed,
                               void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    NormScratch s = carve(scratch, g->n_cap, &total);
    GridView gv{g->sorted, g->cells, g->keys, g->table_size, g->inv_cell, g->d_n_sorted, g->sslot};
    Radii R;
    R.rf2 = prm->r_fpfh * prm->r_fpfh;
    R.rn2 = prm->r_normal * prm->r_normal;
    R.rf2d = (double)prm->r_fpfh * (double)prm->r_fpfh;
    R.rn2d = (double)prm->r_normal * (double)prm->r_normal;
    const int64_t n = g->n_cap;
    cudaError_t e;
    KMX_COUNT_LAUNCH();
    clear_counts<<<kmx_stride_blocks(n, 256, ctx->sm_count), 256, 0, st>>>(
        s.cnt, reinterpret_cast<float4*>(normal4), flags, g->d_n, n);
    KMX_COUNT_LAUNCH();
    search_count<<<kmx_stride_blocks(n, kQPerBlock, ctx->sm_count), kThreads, 0, st>>>(gv, R, s);
    if ((e = kmx_scan_i32(ctx, s.cnt, n, g->d_n, offs))) return e;
    NormOut o{reinterpret_cast<float4*>(normal4), flags, offs, nbr, nbr_cap, n, needed, prm->tau_num,
              prm->tau_lin, {prm->viewpoint[0], prm->viewpoint[1], prm->viewpoint[2]}};
    KMX_COUNT_LAUNCH();
    search_fill<<<kmx_stride_blocks(n, kQPerBlock, ctx->sm_count), kThreads, 0, st>>>(gv, R, s, o, ctx->d_err);
    KMX_COUNT_LAUNCH();
    solve_normals<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(gv, s, o);
    if (nbr) {
        KMX_COUNT_LAUNCH();
        empty_lists_on_overflow<<<kmx_stride_blocks(n + 1, 256, ctx->sm_count), 256, 0, st>>>(offs, n, needed,
                                                                                             nbr_cap);
    }
    return cudaGetLastError();
}
