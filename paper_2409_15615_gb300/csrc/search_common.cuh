// Device helpers of the radius searches: the grid view, the exact radius
// test of Eq. A1, the 27-cell stencil walked by a warp, and the FP64
// eigen-solve and orientation that turn second moments into a normal
// (Sec. III-C).  Shared by the Faster-PFH search (one search, r_FPFH) and the
// classic FPFH baseline (separate searches).
#pragma once

#include "kmx_internal.cuh"
#include "grid_common.cuh"

#include <climits>

namespace kmxs {

constexpr unsigned kFull = 0xffffffffu;

struct GridView {
    const float4* __restrict__ sorted;
    const int2* __restrict__ cells;
    const unsigned long long* __restrict__ keys;
    uint32_t T;
    double inv_cell;
    const int64_t* n_sorted;
    const int32_t* __restrict__ sslot;  // hash slot of each sorted point's cell
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

// The packed cell key of the point at sorted position p: the grid build
// computed it (FP64 floor of x / cell) and kept its hash slot.
__device__ __forceinline__ unsigned long long cell_key_at(const GridView& g, int64_t p)
{
    return __ldg(g.keys + __ldg(g.sslot + p));
}

__device__ __forceinline__ void unpack_cell(unsigned long long key, int* cx, int* cy, int* cz)
{
    *cx = (int)((key >> 42) & 0x1FFFFFull) - KMX_KEY_BIAS;
    *cy = (int)((key >> 21) & 0x1FFFFFull) - KMX_KEY_BIAS;
    *cz = (int)(key & 0x1FFFFFull) - KMX_KEY_BIAS;
}

// Lane l < 27 gets (start, count) of cell l of the stencil around cell
// (cx, cy, cz); returns the candidate total and leaves each lane's exclusive
// prefix in *excl.  Every query of one cell has the same stencil.
__device__ __forceinline__ int stencil_at(const GridView& g, int cx, int cy, int cz, int lane, int* start, int* excl)
{
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

// The stencil of the query at sorted position p.
__device__ __forceinline__ int stencil(const GridView& g, int64_t p, int lane, int* start, int* excl)
{
    int cx, cy, cz;
    unpack_cell(cell_key_at(g, p), &cx, &cy, &cz);
    return stencil_at(g, cx, cy, cz, lane, start, excl);
}

// The stencil of the last query a warp searched, reused while the next
// queries (consecutive in cell order) sit in the same cell.
struct StencilCache {
    unsigned long long key = KMX_EMPTY_KEY;
    int start = 0, excl = 0, total = 0;

    __device__ __forceinline__ int get(const GridView& g, int64_t p, int lane)
    {
        const unsigned long long k = cell_key_at(g, p);
        if (k != key) {
            int x, y, z;
            unpack_cell(k, &x, &y, &z);
            total = stencil_at(g, x, y, z, lane, &start, &excl);
            key = k;
        }
        return total;
    }
};

// Device point count from which the radius searches (normals, the list-free
// FPFH path) give each query one thread; below it one warp takes a query, so
// that a small cloud still fills the GPU.  Every search kernel applies the
// same rule, which keeps the list and list-free paths bit-identical.
constexpr int64_t kThreadQueryMin = 65536;

// One thread per query: calls f(a) for every bucketed point a of the 27-cell
// stencil around sorted position p, in the order of the stored neighbour
// lists (cells dx fastest, then dy, then dz; points of a cell in sorted
// order).
template <typename F>
__device__ __forceinline__ void for_each_candidate(const GridView& g, int64_t p, F&& f)
{
    int cx, cy, cz;
    unpack_cell(cell_key_at(g, p), &cx, &cy, &cz);
    for (int c = 0; c < 27; ++c) {
        const int dx = c % 3 - 1, dy = (c / 3) % 3 - 1, dz = c / 9 - 1;
        const int slot = kmx_hash_find(g.keys, g.T, kmx_pack_key(cx + dx, cy + dy, cz + dz));
        if (slot < 0) continue;
        const int2 cell = __ldg(g.cells + slot);
        for (int i = 0; i < cell.y; ++i) f(__ldg(g.sorted + cell.x + i));
    }
}

// Sweep 1 of a query at q, one thread: |I| (r_FPFH), |P_normal| (r_normal)
// and the sum of the P_normal offsets from q, in list order.
struct Sweep1 {
    int nf = 0, nn = 0;
    float sx = 0.f, sy = 0.f, sz = 0.f;
};

__device__ __forceinline__ Sweep1 sweep1(const GridView& g, const Radii& R, int64_t p, float4 q)
{
    Sweep1 r;
    for_each_candidate(g, p, [&](float4 a) {
        const float dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (within(a, q, d2, R.rf2, R.rf2d)) {
            ++r.nf;
            if (within(a, q, d2, R.rn2, R.rn2d)) {
                ++r.nn;
                r.sx += dx;
                r.sy += dy;
                r.sz += dz;
            }
        }
    });
    return r;
}

// Moments of the P_normal offsets centred on their mean (mx, my, mz), one
// thread, in list order: s1 (3), then xx xy xz yy yz zz.  With nbr, the
// r_FPFH neighbours' indices are written from nbr[0] on.
__device__ __forceinline__ void sweep2(const GridView& g, const Radii& R, int64_t p, float4 q, float mx, float my,
                                       float mz, float (&mom)[9], int32_t* nbr)
{
#pragma unroll
    for (int i = 0; i < 9; ++i) mom[i] = 0.f;
    int64_t out = 0;
    for_each_candidate(g, p, [&](float4 a) {
        const float dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (!within(a, q, d2, R.rf2, R.rf2d)) return;
        if (nbr) nbr[out++] = __float_as_int(a.w);
        if (within(a, q, d2, R.rn2, R.rn2d)) {
            const float ex = dx - mx, ey = dy - my, ez = dz - mz;
            mom[0] += ex;
            mom[1] += ey;
            mom[2] += ez;
            mom[3] = fmaf(ex, ex, mom[3]);
            mom[4] = fmaf(ex, ey, mom[4]);
            mom[5] = fmaf(ex, ez, mom[5]);
            mom[6] = fmaf(ey, ey, mom[6]);
            mom[7] = fmaf(ey, ez, mom[7]);
            mom[8] = fmaf(ez, ez, mom[8]);
        }
    });
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

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Eigenvalues l1 >= l2 >= l3 of a symmetric 3x3 matrix and a unit eigenvector
// of l3.  Returns false if the matrix is a multiple of the identity.
//
// GB300 issues FP64 at a small fraction of the FP32 rate, and an FP64 divide
// or square root is a long instruction sequence, so the reciprocals and
// reciprocal square roots below start from the FP32 intrinsic and take one
// FP64 Newton-Raphson step (r <- r (2 - x r) for 1/x, r <- r (3 - x r^2) / 2
// for 1/sqrt(x)), which squares the FP32 start's relative error (about 1e-7)
// to about 1e-14: far below the 1e-8 the eigenvalues are accurate to.
// Arguments outside [2^-100, 2^100] take the FP64 operation itself.
__device__ __forceinline__ bool fp32_range(double x) { return x > 0x1p-100 && x < 0x1p100; }

__device__ __forceinline__ double recip64(double x)
{
    if (!fp32_range(x)) return 1.0 / x;
    const double r = (double)__frcp_rn((float)x);
    return r * fma(-x, r, 2.0);
}

__device__ __forceinline__ double rsqrt64(double x)
{
    if (!fp32_range(x)) return 1.0 / sqrt(x);
    const double r = (double)rsqrtf((float)x);
    return r * fma(-0.5 * x, r * r, 1.5);
}

// sqrt(x) = x / sqrt(x) for x > 0, 0 for x <= 0
__device__ __forceinline__ double sqrt64(double x)
{
    if (!(x > 0.0)) return 0.0;
    return fp32_range(x) ? x * rsqrt64(x) : sqrt(x);
}

__device__ __forceinline__ bool eig_sym3(double a00, double a01, double a02, double a11, double a12, double a22,
                                         double* l, double* nv)
{
    const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    const double q = (a00 + a11 + a22) * (1.0 / 3.0);
    const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
    if (!(p2 > 0.0)) {
        l[0] = l[1] = l[2] = q;
        nv[0] = 0.0;
        nv[1] = 0.0;
        nv[2] = 1.0;
        return false;
    }
    // Eigenvalues of the traceless B = A - qI are the roots of
    // g(mu) = mu^3 - (p2 / 2) mu - det(B), i.e. 2p cos(phi + 2 pi k / 3) with
    // p = sqrt(p2 / 6), phi = acos(r) / 3, r = det(B) / (2 p^3).  GB300 issues
    // FP64 slowly and acos / cos in FP64 dominated this solve, so: the
    // trigonometric form in FP32 for a start, two FP64 Newton steps on the
    // extreme root that is well separated (the largest when r >= 0, i.e. when
    // the two smaller roots are the closer pair; else the smallest), and the
    // other two in FP64 from the quadratic mu^2 + m mu + (m^2 - p2 / 2) = 0
    // (sum of the roots 0, sum of their pairwise products -p2 / 2), whose
    // square root resolves a close pair to ~1e-8 p.  Beyond p (below -p) g is
    // increasing and convex (concave), so Newton started there (the start is
    // clamped; pf is within 2^-23 of p) moves monotonically to that extreme
    // root.  Eigenvalues come out to ~1e-8 relative or better, the smallest
    // one to FP64 accuracy where the normal is well posed.
    const double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) + a02 * (a01 * a12 - b11 * a02);
    const float pf = sqrtf((float)p2 / 6.0f);
    const float rf = fminf(1.0f, fmaxf(-1.0f, (float)det / (2.0f * pf * pf * pf)));
    const float phi = acosf(rf) / 3.0f;
    const double edge = (double)pf * (1.0 + 0x1p-20);
    const bool top = rf >= 0.0f;
    double mu = top ? fmax((double)(2.0f * pf * cosf(phi)), edge)
                    : fmin((double)(2.0f * pf * cosf(phi + 2.0943951f)), -edge);
    const double h = 0.5 * p2;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double g = mu * (mu * mu - h) - det;
        const double dg = 3.0 * mu * mu - h;
        if (dg > 0.0) mu -= g * recip64(dg);  // dg > 0 beyond +-p
    }
    const double sd = sqrt64(2.0 * p2 - 3.0 * mu * mu);
    if (top) {
        l[0] = q + mu;
        l[1] = q + 0.5 * (-mu + sd);
        l[2] = q + 0.5 * (-mu - sd);
    } else {
        l[0] = q + 0.5 * (-mu + sd);
        l[1] = q + 0.5 * (-mu - sd);
        l[2] = q + mu;
    }
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
    const double inv = rsqrt64(nb);
    nv[0] = cx * inv;
    nv[1] = cy * inv;
    nv[2] = cz * inv;
    return true;
}

// Normal of a query from the moments of its P_normal offsets e = (a - q) - m0
// (m0 the FP32 mean used for centring): mom = (sum e, then the six products
// xx xy xz yy yz zz).  The covariance (1/n normaliser) is formed and solved
// in FP64, the normal oriented toward vp (first non-zero component positive
// when n . (vp - q) = 0) and p_lin = (l1 - l2) / l1 stored in w.  Returns
// false (and a zero normal) when l1 = 0.
__device__ __forceinline__ bool normal_from_moments(const float* mom, int nN, float qx, float qy, float qz,
                                                    const float* vp, float4* nout, double* plin_out)
{
    const double inv = recip64((double)nN);
    const double m0 = (double)mom[0] * inv, m1 = (double)mom[1] * inv, m2 = (double)mom[2] * inv;
    const double c00 = (double)mom[3] * inv - m0 * m0, c01 = (double)mom[4] * inv - m0 * m1;
    const double c02 = (double)mom[5] * inv - m0 * m2, c11 = (double)mom[6] * inv - m1 * m1;
    const double c12 = (double)mom[7] * inv - m1 * m2, c22 = (double)mom[8] * inv - m2 * m2;
    double l[3], nv[3];
    eig_sym3(c00, c01, c02, c11, c12, c22, l, nv);
    *nout = make_float4(0.f, 0.f, 0.f, 0.f);
    *plin_out = 0.0;
    if (!(l[0] > 0.0)) return false;
    const double view = nv[0] * ((double)vp[0] - (double)qx) + nv[1] * ((double)vp[1] - (double)qy) +
                        nv[2] * ((double)vp[2] - (double)qz);
    bool flip = view < 0.0;
    if (view == 0.0) flip = nv[0] != 0.0 ? nv[0] < 0.0 : (nv[1] != 0.0 ? nv[1] < 0.0 : nv[2] < 0.0);
    const double sgn = flip ? -1.0 : 1.0;
    const double plin = (l[0] - l[1]) / l[0];
    *nout = make_float4((float)(sgn * nv[0]), (float)(sgn * nv[1]), (float)(sgn * nv[2]), (float)plin);
    *plin_out = plin;
    return true;
}

}  // namespace kmxs
