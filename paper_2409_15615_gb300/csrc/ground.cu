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
//               heights (a shared histogram above the lowest height),
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
constexpr int kHist = 2048;   // height window of the lowest-point histogram (quanta)
constexpr int kStage = 8192;  // bins up to this size are staged in shared memory (16-bit coordinates, 64 KB)

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

// Ring and sector indices are floor(u) of an FP64 expression u.  Its FP32
// estimate (inputs exact in FP32, a few roundings of 2^-24 relative) is off
// by less than 2^-24 times (4 |u| + 2 g), g the factor by which the
// expression magnifies an absolute error of its first operand: r rings /
// (R1 - R0) for the ring, the sector count for the sector.  The margin
// (1 + |u| + g) 2^-20 is more than twice that; when no integer lies within
// it of the estimate, the estimate's floor is the FP64 one, else the FP64
// expression decides.  So the indices are exactly the FP64 definition's.
struct Estimate {
    float u, gain;
};

__device__ __forceinline__ Estimate ring_f32(double r2, const GP& P, int k)
{
    const float r = __fsqrt_rn(__double2float_rn(r2));
    const float r0 = (float)P.r[k], r1 = (float)P.r[k + 1];
    const float w = __fsub_rn(r1, r0);
    return {__fdiv_rn(__fmul_rn(__fsub_rn(r, r0), (float)P.rings[k]), w),
            __fdiv_rn(__fmul_rn(r, (float)P.rings[k]), w)};
}

__device__ __forceinline__ Estimate sector_f32(float x, float y, int sect)
{
    float p;
    if (y >= 0.f) p = x >= 0.f ? __fdiv_rn(y, __fadd_rn(x, y)) : __fsub_rn(1.f, __fdiv_rn(x, __fsub_rn(y, x)));
    else p = x < 0.f ? __fsub_rn(2.f, __fdiv_rn(y, __fsub_rn(-x, y))) : __fadd_rn(3.f, __fdiv_rn(x, __fsub_rn(x, y)));
    return {__fmul_rn(__fmul_rn(p, (float)sect), 0.25f), 4.f * (float)sect};
}

template <typename F>
__device__ __forceinline__ int floor_exactish(Estimate e, F exact)
{
    const float m = __fmul_rn(__fadd_rn(__fadd_rn(1.f, fabsf(e.u)), e.gain), 0x1p-20f);
    const float lo = floorf(__fsub_rn(e.u, m)), hi = floorf(__fadd_rn(e.u, m));
    if (lo == hi && lo >= 0.f && lo < 1048576.f) return (int)lo;
    return (int)floor(exact());
}

// One atomic per distinct bin in a warp: consecutive scan points mostly fall
// into the same few bins near the sensor, and per-point atomics on one
// address would serialise.  Every lane of the warp calls it (from one call
// site); returns this lane's offset within its group's share.
__device__ __forceinline__ int warp_aggregated_add(int32_t* counters, int key, bool active)
{
    const unsigned act = __ballot_sync(kFull, active);
    if (!active) return 0;
    const unsigned grp = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    const int rank = __popc(grp & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&counters[key], __popc(grp));
    base = __shfl_sync(grp, base, leader);
    return base + rank;
}

__global__ void __launch_bounds__(kThreads) gs_bin(const float* __restrict__ xyz, int64_t n, int stride, GP P,
                                                   GroundScratch s)
{
    // n rounded up to a warp: the trip count is uniform over a warp, so the
    // aggregated atomic sees every lane
    const int64_t n_up = (n + 31) & ~31ll;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n_up; i += (int64_t)gridDim.x * kThreads) {
        int b = -1;
        const float* p = xyz + (i < n ? i : 0) * stride;
        const double x = (double)p[0], y = (double)p[1], z = (double)p[2];
        if (i < n && fabs(z) < P.zlim) {
            const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
            for (int k = 0; k < 4; ++k) {
                if (r2 >= P.r2[k] && r2 < P.r2[k + 1]) {
                    const int ring = min(floor_exactish(ring_f32(r2, P, k), [&] {
                        const double r = __dsqrt_rn(r2);
                        return __ddiv_rn(__dmul_rn(__dsub_rn(r, P.r[k]), (double)P.rings[k]),
                                         __dsub_rn(P.r[k + 1], P.r[k]));
                    }), P.rings[k] - 1);
                    const int sec = min(floor_exactish(sector_f32(p[0], p[1], P.sect[k]), [&] {
                        return __ddiv_rn(__dmul_rn(pseudo_angle(x, y), (double)P.sect[k]), 4.0);
                    }), P.sect[k] - 1);
                    b = P.off[k] + ring * P.sect[k] + sec;
                    s.q[i] = make_int4(quant(p[0], P.Q), quant(p[1], P.Q), quant(p[2], P.Q), 0);
                    break;
                }
            }
        }
        if (i < n) {
            s.bin[i] = b;
            s.keep[i] = 1;
        }
        warp_aggregated_add(s.cnt, b < 0 ? 0 : b, b >= 0);
    }
}

__global__ void __launch_bounds__(kThreads) gs_scatter(int64_t n, GroundScratch s)
{
    const int64_t n_up = (n + 31) & ~31ll;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n_up; i += (int64_t)gridDim.x * kThreads) {
        const int b = i < n ? s.bin[i] : -1;
        const int at = warp_aggregated_add(s.cursor, b < 0 ? 0 : b, b >= 0);
        if (b >= 0) s.members[s.bstart[b] + at] = (int32_t)i;
    }
}

struct Moments {
    long long v[9];  // n, Sx, Sy, Sz, Sxx, Sxy, Syy, Sxz, Syz
};

// |coordinate| <= 32767, so every product fits in 32 bits
__device__ __forceinline__ void add_moments(Moments& m, const int4 q)
{
    m.v[0] += 1;
    m.v[1] += q.x;
    m.v[2] += q.y;
    m.v[3] += q.z;
    m.v[4] += q.x * q.x;
    m.v[5] += q.x * q.y;
    m.v[6] += q.y * q.y;
    m.v[7] += q.x * q.z;
    m.v[8] += q.y * q.z;
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

// The same decision at FP32 cost for most points: the FP32 estimate of the
// residual differs from the FP64 one by less than M = S * 2^-20 (S the sum of
// the magnitudes of its terms; about eight roundings of 2^-24 each, twice
// over), and a residual below sqrt(thr) (1 - 2^-20) or above sqrt(thr)
// (1 + 2^-20) gets that answer from the FP64 test too.  Only points in
// between run the FP64 expression, so the outcome is identical.
struct PlaneTest {
    double pl[3];
    double thr;
    float af, bf, cf, lo, hi;
};

__device__ __forceinline__ PlaneTest plane_test(const double* pl, double thd)
{
    PlaneTest t;
    t.pl[0] = pl[0];
    t.pl[1] = pl[1];
    t.pl[2] = pl[2];
    t.thr = plane_threshold(pl, thd);
    const double T = __dsqrt_rn(t.thr);
    t.af = __double2float_rn(pl[0]);
    t.bf = __double2float_rn(pl[1]);
    t.cf = __double2float_rn(pl[2]);
    t.lo = __double2float_rd(__dmul_rn(T, 1.0 - 0x1p-20));
    t.hi = __double2float_ru(__dmul_rn(T, 1.0 + 0x1p-20));
    return t;
}

__device__ __forceinline__ bool near_plane(const PlaneTest& t, const int4 q)
{
    const float x = (float)q.x, y = (float)q.y, z = (float)q.z;
    const float ax = __fmul_rn(t.af, x), by = __fmul_rn(t.bf, y);
    const float e = __fsub_rn(__fadd_rn(__fadd_rn(ax, by), t.cf), z);
    const float m = __fmul_rn(__fadd_rn(__fadd_rn(fabsf(ax), fabsf(by)), __fadd_rn(fabsf(t.cf), fabsf(z))), 0x1p-20f);
    const float ae = fabsf(e);
    if (__fadd_rn(ae, m) < t.lo) return true;
    if (__fsub_rn(ae, m) > t.hi) return false;
    return near_plane(t.pl, t.thr, q);
}

__global__ void __launch_bounds__(kThreads) gs_fit(GP P, GroundScratch s, double* __restrict__ planes)
{
    __shared__ long long red[kWarps][9];
    __shared__ unsigned long long kred[kWarps];
    __shared__ double sp[3];
    __shared__ PlaneTest spt;  // the current plane's test constants (thread 0 computes them)
    __shared__ long long s_lpr;
    __shared__ int sok, s_fallback;
    __shared__ int ired[kWarps];
    __shared__ int hist[kHist];
    extern __shared__ short4 sq[];  // [kStage] (|coordinate| <= 32767)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int bin = blockIdx.x; bin < P.nb; bin += gridDim.x) {
        const int m = s.cnt[bin];
        const int32_t* mem = s.members + s.bstart[bin];
        double* out = planes ? planes + (int64_t)bin * 4 : nullptr;
        if (m < P.min_pts || m > P.max_pts) {  // uniform over the block
            if (out && threadIdx.x < 4) out[threadIdx.x] = 0.0;
            continue;
        }
        // the members' quantised coordinates, read by every pass below
        const bool staged = m <= kStage;
        if (staged)
            for (int t = threadIdx.x; t < m; t += kThreads) {
                const int4 q = s.q[mem[t]];
                sq[t] = make_short4((short)q.x, (short)q.y, (short)q.z, 0);
            }
        __syncthreads();
        auto member = [&](int t) {
            if (!staged) return s.q[mem[t]];
            const short4 v = sq[t];
            return make_int4(v.x, v.y, v.z, 0);
        };
        // sum of the k lowest quantised heights (ties do not change it): the
        // lowest height, then a shared histogram of the heights within kHist
        // quanta of it, walked by warp 0; when the k lowest are not all in
        // that window, k rounds of a block minimum over (height, index) keys
        const int k = m < P.n_lpr ? m : P.n_lpr;
        int zmin = INT_MAX;
        for (int t = threadIdx.x; t < m; t += kThreads) zmin = min(zmin, member(t).z);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) zmin = min(zmin, __shfl_down_sync(kFull, zmin, o));
        if (lane == 0) ired[warp] = zmin;
        for (int j = threadIdx.x; j < kHist; j += kThreads) hist[j] = 0;
        __syncthreads();
        zmin = ired[0];
        for (int w = 1; w < kWarps; ++w) zmin = min(zmin, ired[w]);
        for (int t = threadIdx.x; t < m; t += kThreads) {
            const int d = member(t).z - zmin;
            if (d < kHist) atomicAdd(&hist[d], 1);
        }
        __syncthreads();
        if (warp == 0) {
            long long sum = 0;
            int need = k;
            for (int base = 0; base < kHist && need > 0; base += 32) {
                const int c = hist[base + lane];
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const int take = max(0, min(c, need - (incl - c)));
                long long part = (long long)take * (long long)(zmin + base + lane);
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
                sum += part;
                need -= min(need, __shfl_sync(kFull, incl, 31));
            }
            if (lane == 0) {
                s_lpr = sum;
                s_fallback = need > 0 ? 1 : 0;
            }
        }
        __syncthreads();
        if (s_fallback) {
            long long lpr = 0;  // meaningful in thread 0
            unsigned long long last = 0;
            for (int round = 0; round < k; ++round) {
                unsigned long long best = ~0ull;
                for (int t = threadIdx.x; t < m; t += kThreads) {
                    const unsigned long long key =
                        ((unsigned long long)(uint32_t)(member(t).z + 0x40000000) << 32) | (uint32_t)mem[t];
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
            if (threadIdx.x == 0) s_lpr = lpr;
        }
        // seeds: zq * k < lpr + ths * k, then the fit
        __syncthreads();
        const long long lim = s_lpr + P.ths * (long long)k;
        Moments mo{};
        for (int t = threadIdx.x; t < m; t += kThreads) {
            const int4 q = member(t);
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
                spt = plane_test(pl, P.thd);
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
            const PlaneTest pt = spt;
            Moments mi{};
            for (int t = threadIdx.x; t < m; t += kThreads) {
                const int4 q = member(t);
                if (near_plane(pt, q)) add_moments(mi, q);
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
                    spt = plane_test(np_, P.thd);
                }
            }
            __syncthreads();
            if (!sok) break;
        }
        // final classification, uprightness and elevation
        const double pl[3] = {sp[0], sp[1], sp[2]};
        const PlaneTest pt = spt;
        Moments mf{};
        for (int t = threadIdx.x; t < m; t += kThreads) {
            const int4 q = member(t);
            if (near_plane(pt, q)) {
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
            for (int t = threadIdx.x; t < m; t += kThreads)
                if (near_plane(pt, member(t))) s.keep[mem[t]] = 0;
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
    // quantised coordinates stay within +-32767 (16 bits), so with at most
    // 2^16 members per bin every moment product fits in 63 bits
    if (!(zl > 0.0) || !(g->r[4] * g->Q <= 32767.0) || !(zl * g->Q <= 32767.0)) return false;
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
    if ((e = kmx_scan_i32(ctx, s.cnt, P.nb, nullptr, s.bstart))) return e;
    KMX_COUNT_LAUNCH();
    gs_scatter<<<nbp, kThreads, 0, st>>>(n, s);
    if ((e = kmx_once_per_device(kmx_attr_ground, [] {
             return cudaFuncSetAttribute(gs_fit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kStage * sizeof(short4)));
         })))
        return e;
    KMX_COUNT_LAUNCH();
    gs_fit<<<(unsigned)P.nb, kThreads, kStage * sizeof(short4), st>>>(P, s, planes);
    if ((e = kmx_scan_i32(ctx, s.keep, n, nullptr, s.pos))) return e;
    KMX_COUNT_LAUNCH();
    gs_compact<<<nbp, kThreads, 0, st>>>(xyz, n, stride, s, out, n_out, ground);
    return cudaGetLastError();
}
