// Voxel downsampling (the voxelised clouds of Sec. III-A).
//
// Sort-free design: a device hash table maps packed voxel keys to slots; the
// lowest input index of each voxel (atomicMin) fixes the output order ("order
// of first member"), a prefix sum over first-member flags numbers the voxels,
// a counting scatter groups members per voxel, and the centroid is the FP64
// input-order sum (computed exactly in integers when an exponent test shows
// that sum is exact, else in input order), so the result does not depend on
// atomic ordering.
#include "kmx_internal.cuh"

namespace {

constexpr int kThreads = 256;

struct VoxScratch {
    unsigned long long* keys;  // [T]   \ one allocation, cleared by one
    uint32_t* vmin;            // [T]    > all-ones memset: empty key, no
    uint32_t* vcnt;            // [T]   /  member yet, member count - 1
    int32_t* vout;             // [T] output voxel index
    int32_t* pslot;            // [n] slot of each point
    int32_t* flag;             // [n] first-member flag, later member count per output voxel
    int64_t* oidx;             // [n+1] exclusive scan of flags
    int64_t* vstart;           // [n+1] member offsets per output voxel
    int32_t* cursor;           // [n] fill cursor per output voxel
    int32_t* members;          // [n] grouped members (arbitrary order inside a voxel)
    float4* run;               // [n] member coordinates per voxel, in input order
    uint32_t T;
};

uint32_t table_size_for(int64_t n)
{
    uint64_t t = 1024;
    while (t < (uint64_t)(2 * n)) t <<= 1;
    return (uint32_t)t;
}

// keys, lowest member and member count of every table slot
size_t table_bytes(uint32_t T) { return (sizeof(unsigned long long) + 2 * sizeof(uint32_t)) * (size_t)T; }

VoxScratch carve(void* base, int64_t n, size_t* total)
{
    VoxScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.T = table_size_for(n);
    auto take = [&](size_t b) { return a.take(b); };
    s.keys = (unsigned long long*)take(table_bytes(s.T));
    s.vmin = reinterpret_cast<uint32_t*>(s.keys + s.T);
    s.vcnt = s.vmin + s.T;
    s.vout = (int32_t*)take(sizeof(int32_t) * s.T);
    s.pslot = (int32_t*)take(sizeof(int32_t) * (n + 1));
    s.flag = (int32_t*)take(sizeof(int32_t) * (n + 1));
    s.oidx = (int64_t*)take(sizeof(int64_t) * (n + 1));
    s.vstart = (int64_t*)take(sizeof(int64_t) * (n + 1));
    s.cursor = (int32_t*)take(sizeof(int32_t) * (n + 1));
    s.members = (int32_t*)take(sizeof(int32_t) * (n + 1));
    s.run = (float4*)take(sizeof(float4) * (n + 1));
    *total = kmx_align_up(a.used, 256);
    return s;
}

// floor(x / v) with the quotient rounded once in FP64 (IEEE division).  The
// FP32 quotient is within one FP32 ulp of the FP64 one; when no integer lies
// within four ulps of it (plus a tiny absolute term for quotients near 0),
// its floor is the FP64 floor, else the FP64 division decides.  GB300 issues
// FP64 slowly; the result is exactly the FP64 definition's.
__device__ __forceinline__ bool voxel_index(float x, float vf, double v, int* k)
{
    const float qf = __fdiv_rn(x, vf);
    const float m = fmaf(fabsf(qf), 0x1p-22f, 0x1p-100f);
    const float lo = floorf(__fsub_rn(qf, m)), hi = floorf(__fadd_rn(qf, m));
    const double q = lo == hi ? (double)lo : floor(__ddiv_rn((double)x, v));
    if (!(fabs(q) < 1048576.0)) return false;
    *k = (int)q;
    return true;
}

// Consecutive scan points often fall into one voxel, so the lanes of a warp
// with the same key share one insert and one update of the voxel's count and
// lowest member (the group's lowest lane holds its lowest index).
__global__ void __launch_bounds__(kThreads) vox_insert(const float* __restrict__ xyz, int64_t n_cap,
                                                       const int64_t* d_n, int stride, float vf, double v,
                                                       VoxScratch s, unsigned int* err)
{
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool ok = false;
    unsigned long long key = 0;
    if (r < kmx_count(d_n, n_cap)) {
        const float* p = xyz + r * stride;
        int kx, ky, kz;
        ok = voxel_index(p[0], vf, v, &kx) & voxel_index(p[1], vf, v, &ky) & voxel_index(p[2], vf, v, &kz);
        if (ok) {
            key = kmx_pack_key(kx, ky, kz);
        } else {
            kmx_raise(err, KMX_DERR_RANGE);
            s.pslot[r] = -1;
        }
    }
    const unsigned act = __ballot_sync(0xffffffffu, ok);  // every lane of the (full) warp gets here
    if (!ok) return;
    const unsigned grp = __match_any_sync(act, key);
    const int leader = __ffs(grp) - 1;
    int slot = 0;
    if (lane == leader) {
        slot = kmx_hash_insert(s.keys, s.T, key);
        if (slot >= 0) {
            atomicMin(&s.vmin[slot], (uint32_t)r);
            atomicAdd(&s.vcnt[slot], (uint32_t)__popc(grp));  // from all-ones: count - 1
        } else {
            kmx_raise(err, KMX_DERR_HASHFULL);
        }
    }
    slot = __shfl_sync(grp, slot, leader);
    s.pslot[r] = slot;
}

__global__ void __launch_bounds__(kThreads) vox_first_flag(int64_t n_cap, const int64_t* d_n, VoxScratch s)
{
    int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= kmx_count(d_n, n_cap)) return;
    int slot = s.pslot[r];
    s.flag[r] = (slot >= 0 && s.vmin[slot] == (uint32_t)r) ? 1 : 0;
}

// For each first member: number its voxel, record the member count per output
// voxel (in `flag`, whose first-member flags the scan has consumed), zero the
// voxel's fill cursor for vox_scatter, publish the voxel count.  Every output
// voxel o < count is written here, and the scan of the counts reads no entry
// past the count, so neither array needs clearing beforehand.
__global__ void __launch_bounds__(kThreads) vox_number(int64_t n, const int64_t* d_n, VoxScratch s, int64_t cap,
                                                       int64_t* n_out, unsigned int* err)
{
    int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r == 0) {
        int64_t tot = s.oidx[n];
        *n_out = tot;
        if (tot > cap) kmx_raise(err, KMX_DERR_CAPACITY);
    }
    if (r >= kmx_count(d_n, n)) return;
    if (s.oidx[r + 1] == s.oidx[r]) return;  // not a first member
    int slot = s.pslot[r];
    int64_t o = s.oidx[r];
    s.vout[slot] = (int32_t)o;
    s.flag[o] = (int32_t)(s.vcnt[slot] + 1u);
    s.cursor[o] = 0;
}

__global__ void __launch_bounds__(kThreads) vox_scatter(int64_t n, const int64_t* d_n, VoxScratch s,
                                                        int32_t* __restrict__ assign)
{
    int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= kmx_count(d_n, n)) return;
    int slot = s.pslot[r];
    if (slot < 0) return;
    int32_t o = s.vout[slot];
    if (assign) assign[r] = o;
    int pos = atomicAdd(&s.cursor[o], 1);
    s.members[s.vstart[o] + pos] = (int32_t)r;
}

// Exponent bookkeeping for the exactness test of an FP64 sum of FP32 values:
// if every nonzero |x| is a normal FP32 number with binary exponent in
// [emin, emax], all values are multiples of 2^(emin-23) and every partial sum
// of L of them is below L * 2^(emax+1); when that quotient fits in 53 bits,
// i.e. emax - emin <= 29 - ceil(log2 L), every partial sum is exact and the
// FP64 result is the same in any summation order.
__device__ __forceinline__ void exp_range(float x, int& emin, int& emax, bool& odd)
{
    const uint32_t bits = __float_as_uint(x) & 0x7fffffffu;
    if (bits == 0) return;
    const int e = (int)(bits >> 23);
    if (e == 0 || e == 255) {  // subnormal, inf or nan: no shortcut
        odd = true;
        return;
    }
    emin = min(emin, e);
    emax = max(emax, e);
}

// The FP64 sum of a voxel's members in input order: each member's rank (the
// number of smaller member indices) places its coordinates in a per-voxel run.
__device__ void ordered_sum(const float* __restrict__ xyz, int stride, const int32_t* m, int L, float4* run,
                            double& sx, double& sy, double& sz)
{
    for (int e = 0; e < L; ++e) {
        const int32_t me = m[e];
        int rank = 0;
        for (int f = 0; f < L; ++f) rank += (m[f] < me);
        const float* p = xyz + (int64_t)me * stride;
        run[rank] = make_float4(p[0], p[1], p[2], 0.f);
    }
    sx = sy = sz = 0.0;
    for (int e = 0; e < L; ++e) {
        const float4 p = run[e];
        sx = __dadd_rn(sx, (double)p.x);
        sy = __dadd_rn(sy, (double)p.y);
        sz = __dadd_rn(sz, (double)p.z);
    }
}

// When the exponent test passes, the exact sum is computed in integers: every
// value is m * 2^(e - 150) with a 24-bit integer m (normal number, biased
// exponent e), so it is the integer m << (e - emin) times 2^(emin - 150); the
// shift is at most 29 - ceil(log2 L) and the sum of L such integers stays
// below 2^53, so it converts to FP64 exactly.
__device__ __forceinline__ long long scaled_int(float x, int emin)
{
    const uint32_t bits = __float_as_uint(x);
    const uint32_t mag = bits & 0x7fffffffu;
    if (mag == 0) return 0;
    const long long m = (long long)((mag & 0x7fffffu) | 0x800000u) << ((int)(mag >> 23) - emin);
    return (bits >> 31) ? -m : m;
}

// isum * 2^(emin - 150) in FP64 (exact: |isum| < 2^53 and the power of two is
// a normal FP64 number for every emin in [1, 255]).
__device__ __forceinline__ double scaled_sum(long long isum, int emin)
{
    const double p2 = __longlong_as_double((long long)(emin - 150 + 1023) << 52);
    return __dmul_rn(__ll2double_rn(isum), p2);
}

constexpr int kCentroidThreads = 128;  // small blocks spread a few thousand voxels over every SM
constexpr int kBigVoxel = 32;          // members above which a whole warp sums the voxel (vox_centroid_big)

// One thread per output voxel of at most kBigVoxel members.  A first pass
// over the members finds each axis's exponent range; if the exponent test
// passes, the FP64 input-order sum equals the exact sum, which a second pass
// accumulates in 64-bit integers (integer pipe; GB300's FP64 rate made the
// FP64 adds the bottleneck).  Otherwise (a voxel whose coordinates span a huge
// range, e.g. values near zero next to larger ones) the members are summed in
// FP64 in input order.
__global__ void __launch_bounds__(kCentroidThreads) vox_centroid(const float* __restrict__ xyz, int stride,
                                                                 int64_t n, VoxScratch s,
                                                                 float4* __restrict__ out, int64_t cap)
{
    const int64_t o = (int64_t)blockIdx.x * kCentroidThreads + threadIdx.x;
    const int64_t nv = s.oidx[n];
    if (o >= nv || o >= cap) return;
    const int64_t b = s.vstart[o];
    const int L = (int)(s.vstart[o + 1] - b);
    if (L > kBigVoxel) return;  // vox_centroid_big
    const int32_t* m = s.members + b;
    int emin[3] = {255, 255, 255}, emax[3] = {0, 0, 0};
    bool odd = false;
    // unrolled so that the loads of several members are in flight together
    // (the index load and the coordinate load of one member are dependent)
#pragma unroll 8
    for (int e = 0; e < L; ++e) {
        const float* p = xyz + (int64_t)__ldg(m + e) * stride;
        exp_range(p[0], emin[0], emax[0], odd);
        exp_range(p[1], emin[1], emax[1], odd);
        exp_range(p[2], emin[2], emax[2], odd);
    }
    const int lg = 32 - __clz(L > 1 ? L - 1 : 1);  // ceil(log2 L) for L >= 2
    bool exact = !odd;
    for (int a = 0; a < 3; ++a)
        if (emax[a] >= emin[a] && emax[a] - emin[a] > 29 - lg) exact = false;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    if (exact) {
        long long ix = 0, iy = 0, iz = 0;
#pragma unroll 8
        for (int e = 0; e < L; ++e) {
            const float* p = xyz + (int64_t)__ldg(m + e) * stride;
            ix += scaled_int(p[0], emin[0]);
            iy += scaled_int(p[1], emin[1]);
            iz += scaled_int(p[2], emin[2]);
        }
        sx = scaled_sum(ix, emin[0]);
        sy = scaled_sum(iy, emin[1]);
        sz = scaled_sum(iz, emin[2]);
    } else {
        ordered_sum(xyz, stride, m, L, s.run + b, sx, sy, sz);
    }
    const double c = (double)L;
    out[o] = make_float4(__double2float_rn(__ddiv_rn(sx, c)), __double2float_rn(__ddiv_rn(sy, c)),
                         __double2float_rn(__ddiv_rn(sz, c)), 0.0f);
}

// One warp per voxel with more than kBigVoxel members (dense cells near a
// scanner): the lanes split the members, the exponent ranges and the integer
// sums are combined with shuffles (integer addition is exact in any order);
// a voxel that fails the exponent test is summed in input order by lane 0.
__global__ void __launch_bounds__(kThreads) vox_centroid_big(const float* __restrict__ xyz, int stride, int64_t n,
                                                            VoxScratch s, float4* __restrict__ out, int64_t cap)
{
    const int lane = threadIdx.x & 31;
    const int64_t nv = min(s.oidx[n], cap);
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t o = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; o < nv; o += warps) {
        const int64_t b = s.vstart[o];
        const int L = (int)(s.vstart[o + 1] - b);
        if (L <= kBigVoxel) continue;
        const int32_t* m = s.members + b;
        int emin[3] = {255, 255, 255}, emax[3] = {0, 0, 0};
        bool odd = false;
        for (int e = lane; e < L; e += 32) {
            const float* p = xyz + (int64_t)__ldg(m + e) * stride;
            exp_range(p[0], emin[0], emax[0], odd);
            exp_range(p[1], emin[1], emax[1], odd);
            exp_range(p[2], emin[2], emax[2], odd);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int sh = 16; sh >= 1; sh >>= 1) {
                emin[a] = min(emin[a], __shfl_xor_sync(0xffffffffu, emin[a], sh));
                emax[a] = max(emax[a], __shfl_xor_sync(0xffffffffu, emax[a], sh));
            }
        }
        odd = __any_sync(0xffffffffu, odd);
        const int lg = 32 - __clz(L - 1);  // ceil(log2 L), L > 32
        bool exact = !odd;
        for (int a = 0; a < 3; ++a)
            if (emax[a] >= emin[a] && emax[a] - emin[a] > 29 - lg) exact = false;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        if (exact) {
            long long ix = 0, iy = 0, iz = 0;
            for (int e = lane; e < L; e += 32) {
                const float* p = xyz + (int64_t)__ldg(m + e) * stride;
                ix += scaled_int(p[0], emin[0]);
                iy += scaled_int(p[1], emin[1]);
                iz += scaled_int(p[2], emin[2]);
            }
#pragma unroll
            for (int sh = 16; sh >= 1; sh >>= 1) {
                ix += __shfl_xor_sync(0xffffffffu, ix, sh);
                iy += __shfl_xor_sync(0xffffffffu, iy, sh);
                iz += __shfl_xor_sync(0xffffffffu, iz, sh);
            }
            sx = scaled_sum(ix, emin[0]);
            sy = scaled_sum(iy, emin[1]);
            sz = scaled_sum(iz, emin[2]);
        } else if (lane == 0) {
            ordered_sum(xyz, stride, m, L, s.run + b, sx, sy, sz);
        }
        if (lane == 0) {
            const double c = (double)L;
            out[o] = make_float4(__double2float_rn(__ddiv_rn(sx, c)), __double2float_rn(__ddiv_rn(sy, c)),
                                 __double2float_rn(__ddiv_rn(sz, c)), 0.0f);
        }
        __syncwarp();
    }
}

}  // namespace

size_t kmx_voxelize_scratch_bytes(int64_t n_raw)
{
    size_t total = 0;
    carve(nullptr, n_raw, &total);
    return total;
}

cudaError_t kmx_voxelize_launch(kmx_ctx* ctx, const float* xyz, int64_t n, const int64_t* d_n, int stride, float v,
                                float* out4, int64_t cap, int64_t* n_out, int32_t* assign, void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    VoxScratch s = carve(scratch, n, &total);
    cudaError_t e;
    if ((e = cudaMemsetAsync(s.keys, 0xFF, table_bytes(s.T), st))) return e;
    if (n == 0) {
        return cudaMemsetAsync(n_out, 0, sizeof(int64_t), st);
    }
    unsigned nb = kmx_blocks(n, kThreads);
    KMX_COUNT_LAUNCH();
    vox_insert<<<nb, kThreads, 0, st>>>(xyz, n, d_n, stride, v, (double)v, s, ctx->d_err);
    KMX_COUNT_LAUNCH();
    vox_first_flag<<<nb, kThreads, 0, st>>>(n, d_n, s);
    if ((e = kmx_scan_i32(ctx, s.flag, n, d_n, s.oidx))) return e;
    KMX_COUNT_LAUNCH();
    vox_number<<<nb, kThreads, 0, st>>>(n, d_n, s, cap, n_out, ctx->d_err);
    // member offsets per output voxel: scan of the counts vox_number left in `flag`
    if ((e = kmx_scan_i32(ctx, s.flag, n, n_out, s.vstart))) return e;
    KMX_COUNT_LAUNCH();
    vox_scatter<<<nb, kThreads, 0, st>>>(n, d_n, s, assign);
    KMX_COUNT_LAUNCH();
    vox_centroid<<<kmx_blocks(n, kCentroidThreads), kCentroidThreads, 0, st>>>(xyz, stride, n, s,
                                                                                    reinterpret_cast<float4*>(out4), cap);
    KMX_COUNT_LAUNCH();
    vox_centroid_big<<<4u * (unsigned)ctx->sm_count, kThreads, 0, st>>>(xyz, stride, n, s,
                                                                         reinterpret_cast<float4*>(out4), cap);
    return cudaGetLastError();
}
