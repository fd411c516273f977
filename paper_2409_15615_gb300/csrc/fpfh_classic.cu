// Classic FPFH (Rusu et al. 2009), the baseline Faster-PFH is compared with
// in Sec. III-C (Fig. 2(a)): three radius searches and no reliability test.
//
//   classic_normals  search 1, r_normal: PCA normal of every point with
//                    |P_normal| >= 3 (a warp per query; one sweep of the
//                    stencil for the mean, a second for the centred moments;
//                    FP64 solve and orientation as in Faster-PFH)
//   scan/scatter     J = the points with a normal, ascending
//   classic_spfh     search 2, r_FPFH: SPFH (Eqs. A2-A4) of every point with
//                    a normal, over its neighbours with a normal
//   classic_fpfh     search 3, r_FPFH: FPFH (Eq. A5) over the same
//                    neighbours, row jpos[q] of the output
//
// Only normals and SPFH rows pass between the searches, as in the classic
// pipeline; no neighbour list is stored.  Queries are taken in the grid's
// cell order so that neighbouring warps walk the same cells.
#include "pfh_common.cuh"
#include "search_common.cuh"

using namespace kmxs;
using namespace kmxp;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kQPerWarp = 4;
constexpr int kQPerBlock = kWarps * kQPerWarp;  // = 32, one per lane of the solving warp
constexpr int kMinNormal = 3;                   // PCA of fewer points fixes no plane

struct ClassicScratch {
    int32_t* jflag;  // [n+1] 1 if the point has a normal
    int64_t* jpos;   // [n+1] exclusive prefix of jflag
    float* spfh;     // [n][36] when the caller passes none
    void* scan;
};

ClassicScratch carve(void* base, int64_t n, bool need_spfh, size_t* total)
{
    ClassicScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.jflag = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.jpos = (int64_t*)a.take(sizeof(int64_t) * (n + 1));
    s.spfh = need_spfh ? (float*)a.take(sizeof(float) * kStride * (n + 1)) : nullptr;
    s.scan = a.take(kmx_scan_scratch_bytes(n));
    *total = kmx_align_up(a.used, 256);
    return s;
}

// Search 1: P_normal(q) = { s : |a_s - a_q| < r_normal } and its normal.
// flags: bit0 = has a normal (= in J), bit1 = in J, bit2 = PCA evaluated.
__global__ void __launch_bounds__(kThreads) classic_normals(GridView g, Radii R, float vp0, float vp1, float vp2,
                                                            float4* __restrict__ normal4,
                                                            uint8_t* __restrict__ flags, int32_t* __restrict__ jflag)
{
    __shared__ float sm_mom[9][kQPerBlock];
    __shared__ float sm_q[3][kQPerBlock];
    __shared__ int sm_qi[kQPerBlock], sm_nN[kQPerBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_sorted = *g.n_sorted;
    const float vp[3] = {vp0, vp1, vp2};
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
            int start, excl;
            const int total = stencil(g, q, lane, &start, &excl);
            // sweep 1: |P_normal| and the mean offset from q
            int nn = 0;
            float sx = 0.f, sy = 0.f, sz = 0.f;
            for (int base = 0; base < total; base += 32) {
                const int t = base + lane;
                const int pos = candidate(t, start, excl);
                bool inN = false;
                float dx = 0.f, dy = 0.f, dz = 0.f;
                if (t < total) {
                    const float4 a = g.sorted[pos];
                    dx = a.x - q.x;
                    dy = a.y - q.y;
                    dz = a.z - q.z;
                    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    inN = within(a, q, d2, R.rn2, R.rn2d);
                }
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
            const float inv = nn > 0 ? 1.0f / (float)nn : 0.0f;
            const float mx = sx * inv, my = sy * inv, mz = sz * inv;
            // sweep 2: moments of the offsets centred on that mean
            float s1x = 0.f, s1y = 0.f, s1z = 0.f;
            float sxx = 0.f, sxy = 0.f, sxz = 0.f, syy = 0.f, syz = 0.f, szz = 0.f;
            if (nn >= kMinNormal) {
                for (int base = 0; base < total; base += 32) {
                    const int t = base + lane;
                    const int pos = candidate(t, start, excl);
                    if (t < total) {
                        const float4 a = g.sorted[pos];
                        const float dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
                        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        if (within(a, q, d2, R.rn2, R.rn2d)) {
                            const float ex = dx - mx, ey = dy - my, ez = dz - mz;
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
                sm_qi[slot] = __float_as_int(q.w);
                sm_nN[slot] = nn;
            }
        }
        __syncthreads();
        if (warp == 0 && sm_qi[lane] >= 0) {
            const int qi = sm_qi[lane];
            const int nN = sm_nN[lane];
            uint8_t flag = 0;
            float4 nout = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nN >= kMinNormal) {
                float mom[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) mom[i] = sm_mom[i][lane];
                double plin;
                flag |= 4;
                if (normal_from_moments(mom, nN, sm_q[0][lane], sm_q[1][lane], sm_q[2][lane], vp, &nout, &plin))
                    flag |= 3;
            }
            normal4[qi] = nout;
            flags[qi] = flag;
            jflag[qi] = flag & 1;
        }
        __syncthreads();  // the shared moments are rewritten by the next chunk
    }
}

__global__ void __launch_bounds__(kThreads) scatter_classic(int64_t n_cap, const int64_t* d_n,
                                                            const int32_t* __restrict__ jflag,
                                                            const int64_t* __restrict__ jpos,
                                                            int32_t* __restrict__ valid, int64_t* n_valid)
{
    const int64_t n = kmx_count(d_n, n_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_valid = jpos[n_cap];
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < n; q += (int64_t)gridDim.x * kThreads)
        if (jflag[q]) valid[jpos[q]] = (int32_t)q;
}

// Search 2: SPFH(q) over k != q within r_FPFH that have a normal.
__global__ void __launch_bounds__(kThreads) classic_spfh(GridView g, Radii R, const float4* __restrict__ normal4,
                                                         const uint8_t* __restrict__ flags,
                                                         float* __restrict__ spfh)
{
    __shared__ int hist[kWarps][kStride];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_sorted = *g.n_sorted;
    const float PI = 3.14159265358979f;
    for (int64_t p = (int64_t)blockIdx.x * kWarps + warp; p < n_sorted; p += (int64_t)gridDim.x * kWarps) {
        const float4 q = g.sorted[p];
        const int qi = __float_as_int(q.w);
        float* row = spfh + (int64_t)qi * kStride;
        if (!(flags[qi] & 1)) {
            row[lane] = 0.f;
            if (lane < kStride - 32) row[32 + lane] = 0.f;
            continue;
        }
        hist[warp][lane] = 0;
        if (lane < kStride - 32) hist[warp][32 + lane] = 0;
        __syncwarp();
        const float4 nq = normal4[qi];
        int start, excl;
        const int total = stencil(g, q, lane, &start, &excl);
        int pairs = 0;
        for (int base = 0; base < total; base += 32) {
            const int t = base + lane;
            const int pos = candidate(t, start, excl);
            bool ok = false;
            if (t < total) {
                const float4 a = g.sorted[pos];
                const int k = __float_as_int(a.w);
                const float dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (k != qi && within(a, q, d2, R.rf2, R.rf2d) && (__ldg(&flags[k]) & 1)) {
                    float f[3];
                    ok = pair_features(q, nq, a, __ldg(&normal4[k]), f);
                    if (ok) {
                        atomicAdd(&hist[warp][feature_bin(f[0], -PI, PI)], 1);
                        atomicAdd(&hist[warp][kH + feature_bin(f[1], -1.f, 1.f)], 1);
                        atomicAdd(&hist[warp][2 * kH + feature_bin(f[2], -1.f, 1.f)], 1);
                    }
                }
            }
            pairs += __popc(__ballot_sync(kFull, ok));
        }
        __syncwarp();
        const float scale = pairs > 0 ? 100.0f / (float)pairs : 0.f;
        row[lane] = (float)hist[warp][lane] * scale;
        if (lane < kStride - 32) row[32 + lane] = lane == 0 ? (float)hist[warp][32] * scale : 0.f;
        __syncwarp();  // the histogram is cleared for the next query
    }
}

// Search 3: FPFH(q) = SPFH(q) + (1/m) sum_k SPFH(k) / w_k over the same
// neighbours; lane l owns bin l, the rows are added in the order the stencil
// yields them with compensated summation.
__global__ void __launch_bounds__(kThreads) classic_fpfh(GridView g, Radii R, const uint8_t* __restrict__ flags,
                                                         const int64_t* __restrict__ jpos,
                                                         const float* __restrict__ spfh, float* __restrict__ desc)
{
    __shared__ int32_t sk[kWarps][32];
    __shared__ float sw[kWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_sorted = *g.n_sorted;
    for (int64_t p = (int64_t)blockIdx.x * kWarps + warp; p < n_sorted; p += (int64_t)gridDim.x * kWarps) {
        const float4 q = g.sorted[p];
        const int qi = __float_as_int(q.w);
        if (!(flags[qi] & 1)) continue;
        int start, excl;
        const int total = stencil(g, q, lane, &start, &excl);
        float acc = 0.f, comp = 0.f, acc32 = 0.f, comp32 = 0.f;
        int m = 0;
        for (int base = 0; base < total; base += 32) {
            const int t = base + lane;
            const int pos = candidate(t, start, excl);
            int k = -1;
            float w = 0.f;
            if (t < total) {
                const float4 a = g.sorted[pos];
                const int kk = __float_as_int(a.w);
                const float dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (kk != qi && d2 > 0.f && within(a, q, d2, R.rf2, R.rf2d) && (__ldg(&flags[kk]) & 1)) {
                    k = kk;
                    w = 1.0f / sqrtf(d2);
                }
            }
            const unsigned bal = __ballot_sync(kFull, k >= 0);
            const int cnt = __popc(bal);
            if (k >= 0) {
                const int slot = __popc(bal & ((1u << lane) - 1u));
                sk[warp][slot] = k;
                sw[warp][slot] = w;
            }
            __syncwarp();
            m += cnt;
#pragma unroll 4
            for (int i = 0; i < cnt; ++i) {
                const float* r = spfh + (int64_t)sk[warp][i] * kStride;
                const float we = sw[warp][i];
                kahan_add(acc, comp, __ldg(&r[lane]) * we);
                if (lane == 0) kahan_add(acc32, comp32, __ldg(&r[32]) * we);
            }
            __syncwarp();
        }
        const float* rq = spfh + (int64_t)qi * kStride;
        const float invm = m > 0 ? 1.0f / (float)m : 0.f;
        float* out = desc + jpos[qi] * kStride;
        out[lane] = rq[lane] + acc * invm;
        if (lane < kStride - 32) out[32 + lane] = lane == 0 ? rq[32] + acc32 * invm : 0.f;
    }
}

}  // namespace

size_t kmx_fpfh_classic_scratch_bytes(int64_t n_cap, bool need_spfh)
{
    size_t total = 0;
    carve(nullptr, n_cap, need_spfh, &total);
    return total;
}

cudaError_t kmx_fpfh_classic_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* prm, float* normal4,
                                    uint8_t* flags, float* desc, int32_t* valid, int64_t* n_valid, float* spfh,
                                    void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    ClassicScratch s = carve(scratch, g->n_cap, spfh == nullptr, &total);
    float* sp = spfh ? spfh : s.spfh;
    GridView gv{g->sorted, g->cells, g->keys, g->table_size, g->inv_cell, g->d_n_sorted};
    Radii R;
    R.rf2 = prm->r_fpfh * prm->r_fpfh;
    R.rn2 = prm->r_normal * prm->r_normal;
    R.rf2d = (double)prm->r_fpfh * (double)prm->r_fpfh;
    R.rn2d = (double)prm->r_normal * (double)prm->r_normal;
    const int64_t n = g->n_cap;
    cudaError_t e;
    // points outside the bucketed set (only after a range error) keep zeros
    // and stay out of J
    if ((e = cudaMemsetAsync(normal4, 0, sizeof(float4) * n, st))) return e;
    if ((e = cudaMemsetAsync(flags, 0, n, st))) return e;
    if ((e = cudaMemsetAsync(s.jflag, 0, sizeof(int32_t) * (n + 1), st))) return e;
    KMX_COUNT_LAUNCH();
    classic_normals<<<kmx_stride_blocks(n, kQPerBlock, ctx->sm_count), kThreads, 0, st>>>(
        gv, R, prm->viewpoint[0], prm->viewpoint[1], prm->viewpoint[2], reinterpret_cast<float4*>(normal4), flags,
        s.jflag);
    if ((e = kmx_scan_i32(s.jflag, n, g->d_n, s.jpos, s.scan, st, ctx->d_err))) return e;
    KMX_COUNT_LAUNCH();
    scatter_classic<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(n, g->d_n, s.jflag, s.jpos,
                                                                                         valid, n_valid);
    const unsigned nbw = kmx_stride_blocks(n, kWarps, ctx->sm_count);
    KMX_COUNT_LAUNCH();
    classic_spfh<<<nbw, kThreads, 0, st>>>(gv, R, reinterpret_cast<const float4*>(normal4), flags, sp);
    KMX_COUNT_LAUNCH();
    classic_fpfh<<<nbw, kThreads, 0, st>>>(gv, R, flags, s.jpos, sp, desc);
    return cudaGetLastError();
}
