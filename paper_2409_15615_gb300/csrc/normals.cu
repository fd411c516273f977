// Algorithm 1, step 1 (Sec. III-C, App. A): one radius search per point with
// r_FPFH (Eq. A1), the r_normal subsample P_normal, PCA normal and linearity,
// and the reliability flag B.
//
// One warp per query, queries taken in cell order so that neighbouring warps
// walk the same cells (L1/L2 reuse).  The 27 stencil cells are looked up by
// 27 lanes at once and their candidate ranges are flattened into one index
// space, so all 32 lanes test candidates regardless of how the points are
// spread over the cells.  Two passes: the first counts |I| and accumulates the
// P_normal mean; after a prefix sum of the counts the second writes the CSR
// lists and accumulates the covariance centred on that mean.
//
// The 3x3 eigen-problem is solved in FP64 (closed form, Smith 1961:
// trigonometric eigenvalues, eigenvector of the smallest one from the
// best-conditioned cross product of two rows of A - l3 I).  GB300 issues FP64
// at a small fraction of the FP32 rate and a warp instruction costs the same
// with 1 or 32 active lanes, so each block first gathers the covariances of
// its 32 queries in shared memory and then solves them one per lane.
#include "kmx_internal.cuh"
#include "grid_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kQPerWarp = 4;                    // queries per warp in the fill pass
constexpr int kQPerBlock = kWarps * kQPerWarp;  // = 32, one per lane of the solving warp
constexpr unsigned kFull = 0xffffffffu;

struct NormScratch {
    int32_t* cnt;    // [n+1] |I(q)|
    float4* mean;    // [n] P_normal mean minus the query point; w = |P_normal| (int bits)
    void* scan;
};

NormScratch carve(void* base, int64_t n, size_t* total)
{
    NormScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.cnt = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.mean = (float4*)a.take(sizeof(float4) * (n + 1));
    s.scan = a.take(kmx_scan_scratch_bytes(n));
    *total = kmx_align_up(a.used, 256);
    return s;
}

struct GridView {
    const float4* __restrict__ sorted;
    const int2* __restrict__ cells;
    const unsigned long long* __restrict__ keys;
    uint32_t T;
    double inv_cell;
    const int64_t* n_sorted;
};

struct Radii {
    float rf2, rn2;     // FP32 squared radii
    double rf2d, rn2d;  // FP64 squared radii, (double)r * (double)r
};

// Is a within radius of q?  FP32 unless the FP32 distance lies within 1e-5
// (relative) of r^2, where the FP64 expression ((dx*dx + dy*dy) + dz*dz) <
// r*r decides; FP32 error is far below that band, so the set is exact.
__device__ __forceinline__ bool within(float4 a, float4 q, float d2, float r2, double r2d)
{
    if (fabsf(d2 - r2) > 1e-5f * r2) return d2 < r2;
    double dx = __dsub_rn((double)a.x, (double)q.x);
    double dy = __dsub_rn((double)a.y, (double)q.y);
    double dz = __dsub_rn((double)a.z, (double)q.z);
    double e = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return e < r2d;
}

// Lane l < 27 gets (start, count) of stencil cell l; returns the candidate
// total and leaves each lane's exclusive prefix in *excl.
__device__ __forceinline__ int stencil(const GridView& g, float4 q, int lane, int* start, int* excl)
{
    int cx, cy, cz;
    kmx_cell_index(q.x, g.inv_cell, &cx);
    kmx_cell_index(q.y, g.inv_cell, &cy);
    kmx_cell_index(q.z, g.inv_cell, &cz);
    int st = 0, ct = 0;
    if (lane < 27) {
        int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
        int slot = kmx_hash_find(g.keys, g.T, kmx_pack_key(cx + dx, cy + dy, cz + dz));
        if (slot >= 0) {
            int2 c = g.cells[slot];
            st = c.x;
            ct = c.y;
        }
    }
    int incl = ct;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    *start = st;
    *excl = incl - ct;
    return __shfl_sync(kFull, incl, 31);
}

// Candidate number t -> position in the sorted point array.
__device__ __forceinline__ int candidate(int t, int start, int excl)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        int e = __shfl_sync(kFull, excl, lo + step);
        if (e <= t) lo += step;
    }
    int cs = __shfl_sync(kFull, start, lo);
    int ce = __shfl_sync(kFull, excl, lo);
    return cs + (t - ce);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Pass 1: |I(q)|, |P_normal| and the P_normal mean (relative to q).
__global__ void __launch_bounds__(kThreads) search_count(GridView g, Radii R, NormScratch s)
{
    const int lane = threadIdx.x & 31;
    const int64_t n_sorted = *g.n_sorted;
    for (int64_t p = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); p < n_sorted; p += (int64_t)gridDim.x * kWarps) {
        const float4 q = g.sorted[p];
        const int qi = __float_as_int(q.w);
        int start, excl;
        const int total = stencil(g, q, lane, &start, &excl);
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

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Eigenvalues l1 >= l2 >= l3 of a symmetric 3x3 matrix and a unit eigenvector
// of l3.  Returns false if the matrix is a multiple of the identity.
__device__ __forceinline__ bool eig_sym3(double a00, double a01, double a02, double a11, double a12, double a22,
                                         double* l, double* nv)
{
    const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    const double q = (a00 + a11 + a22) / 3.0;
    const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
    if (!(p2 > 0.0)) {
        l[0] = l[1] = l[2] = q;
        nv[0] = 0.0;
        nv[1] = 0.0;
        nv[2] = 1.0;
        return false;
    }
    const double p = sqrt(p2 / 6.0);
    const double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) + a02 * (a01 * a12 - b11 * a02);
    double r = det / (2.0 * p * p * p);
    r = fmin(1.0, fmax(-1.0, r));
    const double phi = acos(r) / 3.0;
    l[0] = q + 2.0 * p * cos(phi);
    l[2] = q + 2.0 * p * cos(phi + 2.0943951023931957);  // + 2 pi / 3
    l[1] = 3.0 * q - l[0] - l[2];
    const double r0[3] = {a00 - l[2], a01, a02};
    const double r1[3] = {a01, a11 - l[2], a12};
    const double r2[3] = {a02, a12, a22 - l[2]};
    double c0[3], c1[3], c2[3];
    cross3(r0, r1, c0);
    cross3(r0, r2, c1);
    cross3(r1, r2, c2);
    const double n0 = c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2];
    const double n1 = c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2];
    const double n2 = c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2];
    double cx = c0[0], cy = c0[1], cz = c0[2], nb = n0;
    if (n1 > nb) {
        cx = c1[0];
        cy = c1[1];
        cz = c1[2];
        nb = n1;
    }
    if (n2 > nb) {
        cx = c2[0];
        cy = c2[1];
        cz = c2[2];
        nb = n2;
    }
    if (!(nb > 0.0)) {
        nv[0] = 0.0;
        nv[1] = 0.0;
        nv[2] = 1.0;
        return true;
    }
    const double inv = 1.0 / sqrt(nb);
    nv[0] = cx * inv;
    nv[1] = cy * inv;
    nv[2] = cz * inv;
    return true;
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

// Pass 2: CSR lists and centred second moments over P_normal (a warp per
// query, kQPerWarp queries per warp), then the FP64 eigen-solve, orientation
// and linearity test with one query per lane of warp 0.
__global__ void __launch_bounds__(kThreads) search_fill(GridView g, Radii R, NormScratch s, NormOut o,
                                                        unsigned int* err)
{
    __shared__ float sm_mom[9][kQPerBlock];  // s1x s1y s1z sxx sxy sxz syy syz szz
    __shared__ float sm_q[3][kQPerBlock];
    __shared__ int sm_qi[kQPerBlock], sm_nN[kQPerBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t total_list = o.offs[o.n_cap];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *o.needed = total_list;
        if (o.nbr && total_list > o.nbr_cap) kmx_raise(err, KMX_DERR_CAPACITY);
    }
    const bool write = o.nbr && total_list <= o.nbr_cap;
    const int64_t n_sorted = *g.n_sorted;
    // uniform over the block: every thread reaches the barriers
    for (int64_t chunk = blockIdx.x; chunk * kQPerBlock < n_sorted; chunk += gridDim.x) {
        for (int k = 0; k < kQPerWarp; ++k) {
            const int slot = warp * kQPerWarp + k;
            const int64_t p = chunk * kQPerBlock + slot;
            if (p >= n_sorted) {
                if (lane == 0) sm_qi[slot] = -1;
                continue;
            }
            const float4 q = g.sorted[p];
            const int qi = __float_as_int(q.w);
            const float4 mq = s.mean[qi];
            int start, excl;
            const int total = stencil(g, q, lane, &start, &excl);
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
                sm_mom[0][slot] = s1x;
                sm_mom[1][slot] = s1y;
                sm_mom[2][slot] = s1z;
                sm_mom[3][slot] = sxx;
                sm_mom[4][slot] = sxy;
                sm_mom[5][slot] = sxz;
                sm_mom[6][slot] = syy;
                sm_mom[7][slot] = syz;
                sm_mom[8][slot] = szz;
                sm_q[0][slot] = q.x;
                sm_q[1][slot] = q.y;
                sm_q[2][slot] = q.z;
                sm_qi[slot] = qi;
                sm_nN[slot] = __float_as_int(mq.w);
            }
        }
        __syncthreads();
        if (warp == 0 && sm_qi[lane] >= 0) {
            const int qi = sm_qi[lane];
            const int nN = sm_nN[lane];
            const int mF = (int)(o.offs[qi + 1] - o.offs[qi]);
            uint8_t flag = 0;
            float4 nout = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mF >= o.tau_num && nN >= o.tau_num) {
                const double inv = 1.0 / (double)nN;
                const double m0 = (double)sm_mom[0][lane] * inv, m1 = (double)sm_mom[1][lane] * inv;
                const double m2 = (double)sm_mom[2][lane] * inv;
                const double c00 = (double)sm_mom[3][lane] * inv - m0 * m0, c01 = (double)sm_mom[4][lane] * inv - m0 * m1;
                const double c02 = (double)sm_mom[5][lane] * inv - m0 * m2, c11 = (double)sm_mom[6][lane] * inv - m1 * m1;
                const double c12 = (double)sm_mom[7][lane] * inv - m1 * m2, c22 = (double)sm_mom[8][lane] * inv - m2 * m2;
                double l[3], nv[3];
                eig_sym3(c00, c01, c02, c11, c12, c22, l, nv);
                flag |= 4;
                if (l[0] > 0.0) {
                    const double view = nv[0] * ((double)o.vp[0] - (double)sm_q[0][lane]) +
                                        nv[1] * ((double)o.vp[1] - (double)sm_q[1][lane]) +
                                        nv[2] * ((double)o.vp[2] - (double)sm_q[2][lane]);
                    bool flip = view < 0.0;
                    if (view == 0.0) flip = nv[0] != 0.0 ? nv[0] < 0.0 : (nv[1] != 0.0 ? nv[1] < 0.0 : nv[2] < 0.0);
                    const double sgn = flip ? -1.0 : 1.0;
                    const double plin = (l[0] - l[1]) / l[0];
                    nout = make_float4((float)(sgn * nv[0]), (float)(sgn * nv[1]), (float)(sgn * nv[2]), (float)plin);
                    if (plin < (double)o.tau_lin) flag |= 1;
                }
            }
            o.normal4[qi] = nout;
            o.flags[qi] = flag;
        }
        __syncthreads();  // the shared moments are rewritten by the next chunk
    }
}

// |I(q)| of points that a range error kept out of the grid stays 0.
__global__ void clear_counts(int32_t* cnt, const int64_t* d_n, int64_t n_cap)
{
    const int64_t n = kmx_count(d_n, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] = 0;
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
    GridView gv{g->sorted, g->cells, g->keys, g->table_size, g->inv_cell, g->d_n_sorted};
    Radii R;
    R.rf2 = prm->r_fpfh * prm->r_fpfh;
    R.rn2 = prm->r_normal * prm->r_normal;
    R.rf2d = (double)prm->r_fpfh * (double)prm->r_fpfh;
    R.rn2d = (double)prm->r_normal * (double)prm->r_normal;
    const int64_t n = g->n_cap;
    cudaError_t e;
    // points outside the bucketed set (only after a range error) keep zeros
    if ((e = cudaMemsetAsync(normal4, 0, sizeof(float4) * n, st))) return e;
    if ((e = cudaMemsetAsync(flags, 0, n, st))) return e;
    KMX_COUNT_LAUNCH();
    clear_counts<<<kmx_stride_blocks(n, 256, ctx->sm_count), 256, 0, st>>>(s.cnt, g->d_n, n);
    KMX_COUNT_LAUNCH();
    search_count<<<kmx_stride_blocks(n, kWarps, ctx->sm_count), kThreads, 0, st>>>(gv, R, s);
    if ((e = kmx_scan_i32(s.cnt, n, g->d_n, offs, s.scan, st, ctx->d_err))) return e;
    NormOut o{reinterpret_cast<float4*>(normal4), flags, offs, nbr, nbr_cap, n, needed, prm->tau_num,
              prm->tau_lin, {prm->viewpoint[0], prm->viewpoint[1], prm->viewpoint[2]}};
    KMX_COUNT_LAUNCH();
    search_fill<<<kmx_stride_blocks(n, kQPerBlock, ctx->sm_count), kThreads, 0, st>>>(gv, R, s, o, ctx->d_err);
    return cudaGetLastError();
}
