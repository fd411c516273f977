// Algorithm 1, step 1 (Sec. III-C, App. A): one radius search per point with
// r_FPFH (Eq. A1), the r_normal subsample P_normal, PCA normal and linearity,
// and the reliability flag B.
//
// One thread per query, queries taken in cell order so that neighbouring
// threads walk the same cells (their candidate loads coincide or share cache
// lines).  A thread walks its 27-cell stencil in the order of the stored
// lists and sums in that order (no shuffles, no cross-lane reductions).  Two
// passes: the first counts |I| and accumulates the P_normal mean; after a
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

// Pass 1: |I(q)|, |P_normal| and the P_normal mean (relative to q); one
// thread per query (sorted position), its stencil walked in list order.
__global__ void __launch_bounds__(kThreads) search_count(GridView g, Radii R, NormScratch s)
{
    const int64_t n_sorted = *g.n_sorted;
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

// Pass 2: CSR lists and centred second moments over P_normal, one thread
// per query; the moments go to scratch for solve_normals.
__global__ void __launch_bounds__(kThreads) search_fill(GridView g, Radii R, NormScratch s, NormOut o,
                                                        unsigned int* err)
{
    const int64_t total_list = o.offs[o.n_cap];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *o.needed = total_list;
        if (o.nbr && total_list > o.nbr_cap) kmx_raise(err, KMX_DERR_CAPACITY);
    }
    const bool write = o.nbr && total_list <= o.nbr_cap;
    const int64_t n_sorted = *g.n_sorted;
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
    search_count<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(gv, R, s);
    if ((e = kmx_scan_i32(ctx, s.cnt, n, g->d_n, offs))) return e;
    NormOut o{reinterpret_cast<float4*>(normal4), flags, offs, nbr, nbr_cap, n, needed, prm->tau_num,
              prm->tau_lin, {prm->viewpoint[0], prm->viewpoint[1], prm->viewpoint[2]}};
    KMX_COUNT_LAUNCH();
    search_fill<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(gv, R, s, o, ctx->d_err);
    KMX_COUNT_LAUNCH();
    solve_normals<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(gv, s, o);
    if (nbr) {
        KMX_COUNT_LAUNCH();
        empty_lists_on_overflow<<<kmx_stride_blocks(n + 1, 256, ctx->sm_count), 256, 0, st>>>(offs, n, needed,
                                                                                             nbr_cap);
    }
    return cudaGetLastError();
}
