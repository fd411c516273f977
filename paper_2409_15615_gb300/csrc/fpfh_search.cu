// Descriptors computed by walking the grid again for every stage instead of
// storing neighbour lists: the classic FPFH baseline and a list-free
// Faster-PFH.  On this GPU a 27-cell stencil walk of an L2-resident grid costs
// less than writing the CSR lists once and gathering them three times.
//
// Classic FPFH (Rusu et al. 2009), the baseline of Sec. III-C (Fig. 2(a)):
//   walk_normals<classic>  search 1, r_normal: PCA normal of every point with
//                          |P_normal| >= 3; J = the points with a normal
//   spfh_walk              search 2, r_FPFH: SPFH (Eqs. A2-A4) over the
//                          neighbours with a normal
//   fpfh_walk              search 3, r_FPFH: FPFH (Eq. A5), row jpos[q]
// Faster-PFH (Algorithm 1 and Eqs. A2-A5), the same sets as kmx_normals +
// kmx_fasterpfh:
//   walk_normals<faster>   |I| (r_FPFH), P_normal and its normal; B from
//                          tau_num and tau_lin (step 1)
//   valid_walk             |I_valid(q)| over the neighbours with B; J (step 2)
//   spfh_walk, fpfh_walk   over B neighbours, for B points / for J
// The normals take one thread per query on a large cloud and one warp per
// query on a small one, by the same rule as kmx_normals (kThreadQueryMin);
// the other stages take one warp per query.  Queries run in the grid's cell
// order so that neighbouring threads and warps walk the same cells.  The neighbours a stage visits come
// in the same order as in the stored lists of kmx_normals, so every sum is
// formed in the same order and the list-free Faster-PFH reproduces the
// list-based one bit for bit.
#include "pfh_common.cuh"
#include "search_common.cuh"

using namespace kmxs;
using namespace kmxp;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kQPerWarp = 4;
constexpr int kQPerBlock = kWarps * kQPerWarp;  // = 32, one per lane of the solving warp
constexpr int kMinNormal = 3;                   // classic: PCA of fewer points fixes no plane

struct ClassicScratch {
    int32_t* jflag;  // [n+1] 1 if the point is in J
    int64_t* jpos;   // [n+1] exclusive prefix of jflag
    float* spfh;     // [n][36] when the caller passes none
};

ClassicScratch carve(void* base, int64_t n, bool need_spfh, size_t* total)
{
    ClassicScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.jflag = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.jpos = (int64_t*)a.take(sizeof(int64_t) * (n + 1));
    s.spfh = need_spfh ? (float*)a.take(sizeof(float) * kStride * (n + 1)) : nullptr;
    *total = kmx_align_up(a.used, 256);
    return s;
}

// Normals.  Classic: P_normal(q) = { s : |a_s - a_q| < r_normal }, PCA when
// |P_normal| >= 3; flags bit0 = bit1 = has a normal (J), jflag written.
// Faster-PFH (step 1): also |I(q)| over r_FPFH; PCA when |I| >= tau_num and
// |P_normal| >= tau_num; bit0 = B (normal and p_lin < tau_lin).  bit2 = PCA.
template <bool kClassic>
__global__ void __launch_bounds__(kThreads) walk_normals(GridView g, Radii R, float vp0, float vp1, float vp2,
                                                         int tau_num, float tau_lin, float4* __restrict__ normal4,
                                                         uint8_t* __restrict__ flags, int32_t* __restrict__ jflag)
{
    __shared__ float sm_mom[9][kQPerBlock];
    __shared__ float sm_q[3][kQPerBlock];
    __shared__ int sm_qi[kQPerBlock], sm_nN[kQPerBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_sorted = *g.n_sorted;
    const float vp[3] = {vp0, vp1, vp2};
    if (n_sorted >= kThreadQueryMin) {
        // one thread per query: the two sweeps of kmx_normals (the same
        // order, so the same bits), then the FP64 solve of its moments
        for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < n_sorted; p += (int64_t)gridDim.x * kThreads) {
            const float4 q = g.sorted[p];
            const int qi = __float_as_int(q.w);
            const Sweep1 r = sweep1(g, R, p, q);
            const bool pca = kClassic ? r.nn >= kMinNormal : (r.nf >= tau_num && r.nn >= tau_num);
            uint8_t flag = 0;
            float4 nout = make_float4(0.f, 0.f, 0.f, 0.f);
            if (pca) {
                const float inv = r.nn > 0 ? 1.0f / (float)r.nn : 0.0f;
                float mom[9];
                sweep2(g, R, p, q, r.sx * inv, r.sy * inv, r.sz * inv, mom, nullptr);
                double plin;
                flag |= 4;
                const bool has = normal_from_moments(mom, r.nn, q.x, q.y, q.z, vp, &nout, &plin);
                if (kClassic && has) flag |= 3;
                if (!kClassic && has && plin < (double)tau_lin) flag |= 1;
            }
            normal4[qi] = nout;
            flags[qi] = flag;
            if (kClassic) jflag[qi] = flag & 1;
        }
        return;
    }
    // one warp per query (the same layout as kmx_normals on a small cloud);
    // the block's 32 queries are solved by warp 0, one per lane
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
            const int total = stencil(g, p, lane, &start, &excl);
            // sweep 1: |I|, |P_normal| and the mean offset from q
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
            const float inv = nn > 0 ? 1.0f / (float)nn : 0.0f;
            const float mx = sx * inv, my = sy * inv, mz = sz * inv;
            // sweep 2: moments of the offsets centred on that mean
            float s1x = 0.f, s1y = 0.f, s1z = 0.f;
            float sxx = 0.f, sxy = 0.f, sxz = 0.f, syy = 0.f, syz = 0.f, szz = 0.f;
            const bool pca = kClassic ? nn >= kMinNormal : (nf >= tau_num && nn >= tau_num);
            if (pca) {
                for (int base = 0; base < total; base += 32) {
                    const int t = base + lane;
                    const int pos = candidate(t, start, excl);
                    if (t < total) {
                        const float4 a = g.sorted[pos];
                        const float dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
                        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        if (within(a, q, d2, R.rf2, R.rf2d) && within(a, q, d2, R.rn2, R.rn2d)) {
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
                sm_nN[slot] = pca ? nn : -1;
            }
        }
        __syncthreads();
        if (warp == 0 && sm_qi[lane] >= 0) {
            const int qi = sm_qi[lane];
            const int nN = sm_nN[lane];
            uint8_t flag = 0;
            float4 nout = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nN >= 0) {
                float mom[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) mom[i] = sm_mom[i][lane];
                double plin;
                flag |= 4;
                const bool has = normal_from_moments(mom, nN, sm_q[0][lane], sm_q[1][lane], sm_q[2][lane], vp, &nout,
                                                     &plin);
                if (kClassic && has) flag |= 3;
                if (!kClassic && has && plin < (double)tau_lin) flag |= 1;
            }
            normal4[qi] = nout;
            flags[qi] = flag;
            if (kClassic) jflag[qi] = flag & 1;
        }
        __syncthreads();  // the shared moments are rewritten by the next chunk
    }
}

// Step 2: q enters J iff B[q] and |I_valid(q)| = |{ k in I(q) : B[k] }| >=
// tau_num (q itself counted); sets flags bit1 and jflag.
__global__ void __launch_bounds__(kThreads) valid_walk(GridView g, Radii R, int tau_num, uint8_t* flags,
                                                       int32_t* __restrict__ jflag)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_sorted = *g.n_sorted;
    for (int64_t p = (int64_t)blockIdx.x * kWarps + warp; p < n_sorted; p += (int64_t)gridDim.x * kWarps) {
        const float4 q = g.sorted[p];
        const int qi = __float_as_int(q.w);
        const uint8_t fq = flags[qi];
        if (!(fq & 1)) continue;
        int start, excl;
        const int total = stencil(g, p, lane, &start, &excl);
        int mv = 0;
        for (int base = 0; base < total; base += 32) {
            const int t = base + lane;
            const int pos = candidate(t, start, excl);
            bool ok = false;
            if (t < total) {
                const float4 a = g.sorted[pos];
                const float dx = a.x - q.x, dy = a.y - q.y, dz = a.z - q.z;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                // bit0 is never written here, so reading a byte that another
                // warp is updating sees the same B
                ok = within(a, q, d2, R.rf2, R.rf2d) && (flags[__float_as_int(a.w)] & 1);
            }
            mv += __popc(__ballot_sync(kFull, ok));
        }
        if (lane == 0 && mv >= tau_num) {
            jflag[qi] = 1;
            flags[qi] = (uint8_t)(fq | 2u);
        }
    }
}

__global__ void __launch_bounds__(kThreads) scatter_j(int64_t n_cap, const int64_t* d_n,
                                                            const int32_t* __restrict__ jflag,
                                                            const int64_t* __restrict__ jpos,
                                                            int32_t* __restrict__ valid, int64_t* n_valid)
{
    const int64_t n = kmx_count(d_n, n_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_valid = jpos[n_cap];
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < n; q += (int64_t)gridDim.x * kThreads)
        if (jflag[q]) valid[jpos[q]] = (int32_t)q;
}

// SPFH(q) (Eqs. A2-A4) for q with bit0, over k != q within r_FPFH with bit0.
__global__ void __launch_bounds__(kThreads) spfh_walk(GridView g, Radii R, const float4* __restrict__ normal4,
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
        const int total = stencil(g, p, lane, &start, &excl);
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

// FPFH(q) = SPFH(q) + (1/m) sum_k SPFH(k) / w_k (Eq. A5) for q in J (bit1),
// over the neighbours the SPFH stage used; lane l owns bin l, the rows are
// added in the order the stencil yields them with compensated summation.
__global__ void __launch_bounds__(kThreads) fpfh_walk(GridView g, Radii R, const uint8_t* __restrict__ flags,
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
        if (!(flags[qi] & 2)) continue;
        int start, excl;
        const int total = stencil(g, p, lane, &start, &excl);
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
                kahan_add_prod(acc, comp, __ldg(&r[lane]), we);
                if (lane == 0) kahan_add_prod(acc32, comp32, __ldg(&r[32]), we);
            }
            __syncwarp();
        }
        const float* rq = spfh + (int64_t)qi * kStride;
        const float invm = m > 0 ? 1.0f / (float)m : 0.f;
        float* out = desc + jpos[qi] * kStride;
        out[lane] = fmaf(acc, invm, rq[lane]);
        if (lane < kStride - 32) out[32 + lane] = lane == 0 ? fmaf(acc32, invm, rq[32]) : 0.f;
    }
}

}  // namespace

size_t kmx_fpfh_search_scratch_bytes(int64_t n_cap, bool need_spfh)
{
    size_t total = 0;
    carve(nullptr, n_cap, need_spfh, &total);
    return total;
}

cudaError_t kmx_fpfh_search_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* prm, bool classic,
                                   float* normal4, uint8_t* flags, float* desc, int32_t* valid, int64_t* n_valid,
                                   float* spfh, void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    ClassicScratch s = carve(scratch, g->n_cap, spfh == nullptr, &total);
    float* sp = spfh ? spfh : s.spfh;
    GridView gv{g->sorted, g->cells, g->keys, g->table_size, g->inv_cell, g->d_n_sorted, g->sslot};
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
    const unsigned nbn = kmx_stride_blocks(n, kQPerBlock, ctx->sm_count);
    const unsigned nbw = kmx_stride_blocks(n, kWarps, ctx->sm_count);
    const float4* n4 = reinterpret_cast<const float4*>(normal4);
    KMX_COUNT_LAUNCH();
    if (classic) {
        walk_normals<true><<<nbn, kThreads, 0, st>>>(gv, R, prm->viewpoint[0], prm->viewpoint[1], prm->viewpoint[2],
                                                     prm->tau_num, prm->tau_lin, reinterpret_cast<float4*>(normal4),
                                                     flags, s.jflag);
    } else {
        walk_normals<false><<<nbn, kThreads, 0, st>>>(gv, R, prm->viewpoint[0], prm->viewpoint[1],
                                                      prm->viewpoint[2], prm->tau_num, prm->tau_lin,
                                                      reinterpret_cast<float4*>(normal4), flags, s.jflag);
        KMX_COUNT_LAUNCH();
        valid_walk<<<nbw, kThreads, 0, st>>>(gv, R, prm->tau_num, flags, s.jflag);
    }
    if ((e = kmx_scan_i32(ctx, s.jflag, n, g->d_n, s.jpos))) return e;
    KMX_COUNT_LAUNCH();
    scatter_j<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(n, g->d_n, s.jflag, s.jpos, valid,
                                                                                   n_valid);
    KMX_COUNT_LAUNCH();
    spfh_walk<<<nbw, kThreads, 0, st>>>(gv, R, n4, flags, sp);
    KMX_COUNT_LAUNCH();
    fpfh_walk<<<nbw, kThreads, 0, st>>>(gv, R, flags, s.jpos, sp, desc);
    return cudaGetLastError();
}
