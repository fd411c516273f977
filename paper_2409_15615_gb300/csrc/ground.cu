// Geometric suppression (Sec. III-B): ground removal before the descriptors.
//
// The paper uses Patchwork (Lim et al., RA-L 2021) and does not restate it;
// this is the stand-in: Patchwork's concentric zone model with region-wise
// ground plane fitting.  Every decision is made on exact integers or on one
// fixed sequence of IEEE FP64 operations (no contraction, no transcendental),
// so the result does not depend on the order in which threads meet points.
//
//   gs_bin      per point: zone (r^2 against the zone edges), ring, sector of
//               the pseudo-angle, quantised coordinates; member count per bin
//   scan        bin starts
//   gs_scatter  members grouped per bin (any order inside a bin)
//   gs_fit      a block per bin: the sum of the n_lpr lowest quantised
//               heights (repeated block minimum of (height, index) keys),
//               seeds, least-squares height field z = a x + b y + c from
//               exact int64 moments (centred exactly, FP64 Cramer), n_iter
//               refits on the members within th_dist, uprightness and
//               elevation tests; ground members are marked
//   scan        positions of the kept points
//   gs_compact  kept points in input order
#include <cmath>

#include "kmx_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

struct GP {
    double r[5], r2[5];
    int rings[4], sect[4], off[4];
    double Q, zlim, thd, slope2;
    long long ths, mz;
    int n_lpr, n_iter, min_pts, max_pts, nb;
};

struct GroundScratch {
    int32_t* bin;      // [n] bin of each point, -1 = none
    int4* q;           // [n] quantised coordinates of binned points
    int32_t* keep;     // [n+1] 1 = kept
    int64_t* pos;      // [n+1] exclusive scan of keep
    int32_t* members;  // [n] points grouped per bin
    int32_t* cnt;      // [nb+1] members per bin
    int64_t* bstart;   // [nb+1] first member of each bin
    int32_t* cursor;   // [nb+1] fill cursor per bin
    void* scan;
};

GroundScratch carve(void* base, int64_t n, int nb, size_t* total)
{
    GroundScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.bin = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.q = (int4*)a.take(sizeof(int4) * (n + 1));
    s.keep = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.pos = (int64_t*)a.take(sizeof(int64_t) * (n + 1));
    s.members = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.cnt = (int32_t*)a.take(sizeof(int32_t) * (nb + 1));
    s.bstart = (int64_t*)a.take(sizeof(int64_t) * (nb + 1));
    s.cursor = (int32_t*)a.take(sizeof(int32_t) * (nb + 1));
    s.scan = a.take(kmx_scan_scratch_bytes(n > nb ? n : nb));
    *total = kmx_align_up(a.used, 256);
    return s;
}

// Monotone stand-in for the polar angle on [0, 4): quadrant + |y| / (|x| + |y|).
__device__ __forceinline__ double pseudo_angle(double x, double y)
{
    if (y >= 0.0) {
        if (x >= 0.0) return __ddiv_rn(y, __dadd_rn(x, y));
        return __dsub_rn(1.0, __ddiv_rn(x, __dsub_rn(y, x)));
    }
    if (x < 0.0) return __dsub_rn(2.0, __ddiv_rn(y, __dsub_rn(-x, y)));
    return __dadd_rn(3.0, __ddiv_rn(x, __dsub_rn(x, y)));
}

__device__ __forceinline__ int quant(float v, double Q) { return (int)rint(__dmul_rn((double)v, Q)); }

__global__ void __launch_bounds__(kThreads) gs_bin(const float* __restrict__ xyz, int64_t n, int stride, GP P,
                                                   GroundScratch s)
{
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const float* p = xyz + i * stride;
        const double x = (double)p[0], y = (double)p[1], z = (double)p[2];
        int b = -1;
        if (fabs(z) < P.zlim) {
            const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
            for (int k = 0; k < 4; ++k) {
                if (r2 >= P.r2[k] && r2 < P.r2[k + 1]) {
                    const double r = __dsqrt_rn(r2);
                    double ring = floor(__ddiv_rn(__dmul_rn(__dsub_rn(r, P.r[k]), (double)P.rings[k]),
                                                  __dsub_rn(P.r[k + 1], P.r[k])));
                    ring = fmin(ring, (double)(P.rings[k] - 1));
                    double sec = floor(__ddiv_rn(__dmul_rn(pseudo_angle(x, y), (double)P.sect[k]), 4.0));
                    sec = fmin(sec, (double)(P.sect[k] - 1));
                    b = P.off[k] + (int)ring * P.sect[k] + (int)sec;
                    s.q[i] = make_int4(quant(p[0], P.Q), quant(p[1], P.Q), quant(p[2], P.Q), 0);
                    break;
                }
            }
        }
        s.bin[i] = b;
        s.keep[i] = 1;
        if (b >= 0) atomicAdd(&s.cnt[b], 1);
    }
}

__global__ void __launch_bounds__(kThreads) gs_scatter(int64_t n, GroundScratch s)
{
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const int b = s.bin[i];
        if (b < 0) continue;
        const int at = atomicAdd(&s.cursor[b], 1);
        s.members[s.bstart[b] + at] = (int32_t)i;
    }
}

struct Moments {
    long long v[9];  // n, Sx, Sy, Sz, Sxx, Sxy, Syy, Sxz, Syz
};

__device__ __forceinline__ void add_moments(Moments& m, const int4 q)
{
    const long long xq = q.x, yq = q.y, zq = q.z;
    m.v[0] += 1;
    m.v[1] += xq;
    m.v[2] += yq;
    m.v[3] += zq;
    m.v[4] += xq * xq;
    m.v[5] += xq * yq;
    m.v[6] += yq * yq;
    m.v[7] += xq * zq;
    m.v[8] += yq * zq;
}

// Block-wide exact sums of the nine moments (thread 0 gets the result).  The
// caller separates consecutive calls by a barrier after thread 0's use.
__device__ __forceinline__ void block_moments(Moments& m, long long (*red)[9])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        long long v = m.v[j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(kFull, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            long long t = 0;
            for (int w = 0; w < kWarps; ++w) t += red[w][j];
            m.v[j] = t;
        }
    }
}

// a * b - c * d, exact whenever the result fits in 64 bits (modular
// arithmetic; by Cauchy-Schwarz every centred moment here does).
__device__ __forceinline__ long long cross_diff(long long a, long long b, long long c, long long d)
{
    return (long long)((unsigned long long)a * (unsigned long long)b - (unsigned long long)c * (unsigned long long)d);
}

// Least-squares height field from exact moments: false when fewer than 3
// points or the system is singular.
__device__ __forceinline__ bool solve_plane(const Moments& m, double* pl)
{
    const long long n = m.v[0], Sx = m.v[1], Sy = m.v[2], Sz = m.v[3];
    if (n < 3) return false;
    const double cxx = __ll2double_rn(cross_diff(n, m.v[4], Sx, Sx));
    const double cxy = __ll2double_rn(cross_diff(n, m.v[5], Sx, Sy));
    const double cyy = __ll2double_rn(cross_diff(n, m.v[6], Sy, Sy));
    const double cxz = __ll2double_rn(cross_diff(n, m.v[7], Sx, Sz));
    const double cyz = __ll2double_rn(cross_diff(n, m.v[8], Sy, Sz));
    const double det = __dsub_rn(__dmul_rn(cxx, cyy), __dmul_rn(cxy, cxy));
    if (!(det > 0.0)) return false;
    const double a = __ddiv_rn(__dsub_rn(__dmul_rn(cxz, cyy), __dmul_rn(cyz, cxy)), det);
    const double b = __ddiv_rn(__dsub_rn(__dmul_rn(cyz, cxx), __dmul_rn(cxz, cxy)), det);
    const double c = __ddiv_rn(__dsub_rn(__dsub_rn(__ll2double_rn(Sz), __dmul_rn(a, __ll2double_rn(Sx))),
                                         __dmul_rn(b, __ll2double_rn(Sy))),
                               __ll2double_rn(n));
    pl[0] = a;
    pl[1] = b;
    pl[2] = c;
    return true;
}

// th^2 (1 + a^2 + b^2): the squared vertical residual below which a point is
// within th of the plane orthogonally (quantised units).
__device__ __forceinline__ double plane_threshold(const double* pl, double thd)
{
    return __dmul_rn(__dmul_rn(thd, thd), __dadd_rn(__dadd_rn(1.0, __dmul_rn(pl[0], pl[0])), __dmul_rn(pl[1], pl[1])));
}

__device__ __forceinline__ bool near_plane(const double* pl, double thr, const int4 q)
{
    const double e = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(pl[0], (double)q.x), __dmul_rn(pl[1], (double)q.y)), pl[2]),
                               (double)q.z);
    return __dmul_rn(e, e) < thr;
}

__global__ void __launch_bounds__(kThreads) gs_fit(GP P, GroundScratch s, double* __restrict__ planes)
{
    __shared__ long long red[kWarps][9];
    __shared__ unsigned long long kred[kWarps];
    __shared__ double sp[3];
    __shared__ long long s_lpr;
    __shared__ int sok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int bin = blockIdx.x; bin < P.nb; bin += gridDim.x) {
        const int m = s.cnt[bin];
        const int32_t* mem = s.members + s.bstart[bin];
        double* out = planes ? planes + (int64_t)bin * 4 : nullptr;
        if (m < P.min_pts || m > P.max_pts) {  // uniform over the block
            if (out && threadIdx.x < 4) out[threadIdx.x] = 0.0;
            continue;
        }
        // sum of the k lowest quantised heights: k rounds of a block minimum
        // over (height, index) keys above the previous one
        const int k = m < P.n_lpr ? m : P.n_lpr;
        long long lpr = 0;  // meaningful in thread 0
        unsigned long long last = 0;
        for (int round = 0; round < k; ++round) {
            unsigned long long best = ~0ull;
            for (int t = threadIdx.x; t < m; t += kThreads) {
                const int i = mem[t];
                const unsigned long long key =
                    ((unsigned long long)(uint32_t)(s.q[i].z + 0x40000000) << 32) | (uint32_t)i;
                if ((round == 0 || key > last) && key < best) best = key;
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const unsigned long long v = __shfl_down_sync(kFull, best, o);
                best = v < best ? v : best;
            }
            if (lane == 0) kred[warp] = best;
            __syncthreads();
            unsigned long long mn = kred[0];
            for (int w = 1; w < kWarps; ++w) mn = kred[w] < mn ? kred[w] : mn;
            __syncthreads();  // kred is rewritten by the next round
            last = mn;
            if (threadIdx.x == 0) lpr += (long long)(uint32_t)(mn >> 32) - 0x40000000ll;
        }
        // seeds: zq * k < lpr + ths * k, then the fit
        if (threadIdx.x == 0) s_lpr = lpr;
        __syncthreads();
        const long long lim = s_lpr + P.ths * (long long)k;
        Moments mo{};
        for (int t = threadIdx.x; t < m; t += kThreads) {
            const int4 q = s.q[mem[t]];
            if ((long long)q.z * (long long)k < lim) add_moments(mo, q);
        }
        block_moments(mo, red);
        if (threadIdx.x == 0) {
            double pl[3];
            sok = solve_plane(mo, pl) ? 1 : 0;
            if (sok) {
                sp[0] = pl[0];
                sp[1] = pl[1];
                sp[2] = pl[2];
            }
        }
        __syncthreads();
        if (!sok) {
            if (out && threadIdx.x == 0) {
                out[0] = out[1] = out[2] = 0.0;
                out[3] = 1.0;
            }
            __syncthreads();
            continue;
        }
        // refits on the members within th_dist of the current plane
        for (int it = 0; it < P.n_iter; ++it) {
            const double pl[3] = {sp[0], sp[1], sp[2]};
            const double thr = plane_threshold(pl, P.thd);
            Moments mi{};
            for (int t = threadIdx.x; t < m; t += kThreads) {
                const int4 q = s.q[mem[t]];
                if (near_plane(pl, thr, q)) add_moments(mi, q);
            }
            __syncthreads();  // every thread has read sp
            block_moments(mi, red);
            if (threadIdx.x == 0) {
                double np_[3];
                sok = solve_plane(mi, np_) ? 1 : 0;
                if (sok) {
                    sp[0] = np_[0];
                    sp[1] = np_[1];
                    sp[2] = np_[2];
                }
            }
            __syncthreads();
            if (!sok) break;
        }
        // final classification, uprightness and elevation
        const double pl[3] = {sp[0], sp[1], sp[2]};
        const double thr = plane_threshold(pl, P.thd);
        Moments mf{};
        for (int t = threadIdx.x; t < m; t += kThreads) {
            const int4 q = s.q[mem[t]];
            if (near_plane(pl, thr, q)) {
                mf.v[0] += 1;
                mf.v[3] += q.z;
            }
        }
        __syncthreads();  // every thread has read sp and sok
        block_moments(mf, red);
        if (threadIdx.x == 0) {
            int status = 4;
            if (!(__dadd_rn(__dmul_rn(pl[0], pl[0]), __dmul_rn(pl[1], pl[1])) <= P.slope2)) status = 2;
            else if (mf.v[0] == 0 || !(mf.v[3] < P.mz * mf.v[0])) status = 3;
            sok = status;
            if (out) {
                out[0] = pl[0];
                out[1] = pl[1];
                out[2] = pl[2];
                out[3] = (double)status;
            }
        }
        __syncthreads();
        if (sok == 4) {
            for (int t = threadIdx.x; t < m; t += kThreads) {
                const int i = mem[t];
                if (near_plane(pl, thr, s.q[i])) s.keep[i] = 0;
            }
        }
        __syncthreads();  // shared state is reused by the next bin
    }
}

__global__ void __launch_bounds__(kThreads) gs_compact(const float* __restrict__ xyz, int64_t n, int stride,
                                                       GroundScratch s, float* __restrict__ out, int64_t* n_out,
                                                       uint8_t* __restrict__ ground)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = s.pos[n];
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const int kp = s.keep[i];
        if (ground) ground[i] = kp ? 0 : 1;
        if (kp) {
            const float* p = xyz + i * stride;
            float* o = out + s.pos[i] * stride;
            for (int a = 0; a < stride; ++a) o[a] = p[a];
        }
    }
}

bool make_gp(const kmx_ground_params* p, GP* g)
{
    double prev = 0.0;
    for (int k = 0; k < 5; ++k) {
        const double r = (double)p->zone_r[k];
        if (!(r > prev) || !std::isfinite(r)) return false;
        g->r[k] = r;
        g->r2[k] = r * r;
        prev = r;
    }
    int off = 0;
    for (int k = 0; k < 4; ++k) {
        if (p->zone_rings[k] < 1 || p->zone_sectors[k] < 1 || p->zone_rings[k] > 1024 || p->zone_sectors[k] > 1024)
            return false;
        g->rings[k] = p->zone_rings[k];
        g->sect[k] = p->zone_sectors[k];
        g->off[k] = off;
        off += p->zone_rings[k] * p->zone_sectors[k];
    }
    if (off > 65536) return false;
    g->nb = off;
    if (p->quant_log2 < 0 || p->quant_log2 > 12) return false;
    g->Q = std::ldexp(1.0, p->quant_log2);
    const double zl = (double)p->z_limit;
    // quantised coordinates stay within +-2^15, so with at most 2^16 members
    // per bin every moment product fits in 63 bits
    if (!(zl > 0.0) || !(g->r[4] * g->Q <= 32768.0) || !(zl * g->Q <= 32768.0)) return false;
    g->zlim = zl;
    if (!(p->th_seeds > 0.0f) || !(p->th_dist > 0.0f) || !(p->max_slope > 0.0f) || !std::isfinite(p->th_seeds) ||
        !std::isfinite(p->th_dist) || !std::isfinite(p->max_slope) || !std::isfinite(p->max_ground_z) ||
        !(std::fabs((double)p->max_ground_z) < 32768.0))
        return false;
    if (p->n_lpr < 1 || p->n_lpr > 1024 || p->n_iter < 0 || p->n_iter > 64 || p->min_points < 3 ||
        p->max_bin_points < p->min_points || p->max_bin_points > 65536)
        return false;
    g->ths = (long long)std::nearbyint((double)p->th_seeds * g->Q);
    g->thd = (double)p->th_dist * g->Q;
    g->mz = (long long)std::nearbyint((double)p->max_ground_z * g->Q);
    g->slope2 = (double)p->max_slope * (double)p->max_slope;
    g->n_lpr = p->n_lpr;
    g->n_iter = p->n_iter;
    g->min_pts = p->min_points;
    g->max_pts = p->max_bin_points;
    return true;
}

}  // namespace

int kmx_ground_bins_of(const kmx_ground_params* p)
{
    GP g;
    return (p && make_gp(p, &g)) ? g.nb : -1;
}

size_t kmx_ground_scratch_bytes(int64_t n, int nb)
{
    size_t total = 0;
    carve(nullptr, n, nb, &total);
    return total;
}

cudaError_t kmx_ground_launch(kmx_ctx* ctx, const float* xyz, int64_t n, int stride, const kmx_ground_params* prm,
                              float* out, int64_t* n_out, uint8_t* ground, double* planes, void* scratch)
{
    GP P;
    make_gp(prm, &P);  // validated by the caller
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    GroundScratch s = carve(scratch, n, P.nb, &total);
    cudaError_t e;
    if ((e = cudaMemsetAsync(s.cnt, 0, sizeof(int32_t) * (P.nb + 1), st))) return e;
    if ((e = cudaMemsetAsync(s.cursor, 0, sizeof(int32_t) * (P.nb + 1), st))) return e;
    if (n == 0) {
        if (planes && (e = cudaMemsetAsync(planes, 0, sizeof(double) * 4 * P.nb, st))) return e;
        return cudaMemsetAsync(n_out, 0, sizeof(int64_t), st);
    }
    const unsigned nbp = kmx_stride_blocks(n, kThreads, ctx->sm_count);
    KMX_COUNT_LAUNCH();
    gs_bin<<<nbp, kThreads, 0, st>>>(xyz, n, stride, P, s);
    if ((e = kmx_scan_i32(s.cnt, P.nb, nullptr, s.bstart, s.scan, st, ctx->d_err))) return e;
    KMX_COUNT_LAUNCH();
    gs_scatter<<<nbp, kThreads, 0, st>>>(n, s);
    KMX_COUNT_LAUNCH();
    gs_fit<<<(unsigned)P.nb, kThreads, 0, st>>>(P, s, planes);
    if ((e = kmx_scan_i32(s.keep, n, nullptr, s.pos, s.scan, st, ctx->d_err))) return e;
    KMX_COUNT_LAUNCH();
    gs_compact<<<nbp, kThreads, 0, st>>>(xyz, n, stride, s, out, n_out, ground);
    return cudaGetLastError();
}
