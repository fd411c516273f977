// Algorithm 1, step 2 and the Faster-PFH descriptors (App. A, Eqs. A2-A5).
//
//   spfh_kernel  for q with B: Darboux-frame features (Eq. A2) of every pair
//                (q, k), k in I_valid(q) \ {q}, binned (Eq. A3) into a
//                per-warp shared-memory histogram and scaled by 100 / pairs
//                (Eq. A4); in the same pass |I_valid(q)| = |{ i in M[q] : B[i] }|
//                and so q in J iff B[q] and |I_valid(q)| >= tau_num
//   scan/scatter J in ascending point order
//   fpfh_kernel  FPFH(q) = SPFH(q) + (1/m) sum_k SPFH(k) / w_k (Eq. A5), four
//                rows per warp, a lane owning four bins, compensated summation
//
// I_valid is never materialised: the SPFH and FPFH kernels walk M[q] and
// skip entries without B (one byte gathered per neighbour).
#include "pfh_common.cuh"

using namespace kmxp;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

struct PfhScratch {
    int32_t* jflag;  // [n+1]
    int64_t* jpos;   // [n+1]
    float* spfh;     // [n][36] when the caller passes none
};

PfhScratch carve(void* base, int64_t n, bool need_spfh, size_t* total)
{
    PfhScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.jflag = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.jpos = (int64_t*)a.take(sizeof(int64_t) * (n + 1));
    s.spfh = need_spfh ? (float*)a.take(sizeof(float) * kStride * (n + 1)) : nullptr;
    *total = kmx_align_up(a.used, 256);
    return s;
}

__global__ void __launch_bounds__(kThreads) scatter_valid(int64_t n_cap, const int64_t* d_n,
                                                          const int32_t* __restrict__ jflag,
                                                          const int64_t* __restrict__ jpos,
                                                          int32_t* __restrict__ valid, int64_t* n_valid)
{
    const int64_t n = kmx_count(d_n, n_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_valid = jpos[n_cap];
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < n; q += (int64_t)gridDim.x * kThreads)
        if (jflag[q]) valid[jpos[q]] = (int32_t)q;
}

__global__ void __launch_bounds__(kThreads, 4) spfh_kernel(int64_t n_cap, const int64_t* d_n,
                                                        const float4* __restrict__ pts,
                                                        const float4* __restrict__ normal4, uint8_t* flags,
                                                        const int64_t* __restrict__ offs,
                                                        const int32_t* __restrict__ nbr, int tau_num,
                                                        float* __restrict__ spfh, int32_t* __restrict__ jflag)
{
    __shared__ int hist[kWarps][kStride];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = kmx_count(d_n, n_cap);
    for (int64_t q = (int64_t)blockIdx.x * kWarps + warp; q < n; q += (int64_t)gridDim.x * kWarps) {
        float* row = spfh + q * kStride;
        const uint8_t fq = flags[q];
        if (!(fq & 1)) {
            row[lane] = 0.f;
            if (lane < kStride - 32) row[32 + lane] = 0.f;
            if (lane == 0) {
                jflag[q] = 0;
                if (fq & 2) flags[q] = (uint8_t)(fq & ~2u);
            }
            continue;
        }
        hist[warp][lane] = 0;
        if (lane < kStride - 32) hist[warp][32 + lane] = 0;
        __syncwarp();
        const float4 pq = pts[q];
        const float4 nq = normal4[q];
        const float PI = 3.14159265358979f;
        const int64_t b = offs[q], e = offs[q + 1];
        int pairs = 0, mv = 0;
        // two list entries per lane and step: both indices, then both
        // neighbours' point, normal and flag, are requested before any use
        for (int64_t t0 = b; t0 < e; t0 += 64) {
            const int64_t ta = t0 + lane, tb = ta + 32;
            const bool ha = ta < e, hb = tb < e;
            const int ka = ha ? nbr[ta] : 0;
            const int kb = hb ? nbr[tb] : 0;
            float4 pa = pq, na = nq, pb = pq, nb = nq;
            bool va = false, vb = false;
            if (ha) {
                pa = __ldg(&pts[ka]);
                na = __ldg(&normal4[ka]);
                va = (flags[ka] & 1) != 0;
            }
            if (hb) {
                pb = __ldg(&pts[kb]);
                nb = __ldg(&normal4[kb]);
                vb = (flags[kb] & 1) != 0;
            }
            bool oka = false, okb = false;
            float f[3];
            if (ha && ka != q && va) {
                oka = pair_features(pq, nq, pa, na, f);
                if (oka) {
                    atomicAdd(&hist[warp][feature_bin(f[0], -PI, PI)], 1);
                    atomicAdd(&hist[warp][kH + feature_bin(f[1], -1.f, 1.f)], 1);
                    atomicAdd(&hist[warp][2 * kH + feature_bin(f[2], -1.f, 1.f)], 1);
                }
            }
            if (hb && kb != q && vb) {
                okb = pair_features(pq, nq, pb, nb, f);
                if (okb) {
                    atomicAdd(&hist[warp][feature_bin(f[0], -PI, PI)], 1);
                    atomicAdd(&hist[warp][kH + feature_bin(f[1], -1.f, 1.f)], 1);
                    atomicAdd(&hist[warp][2 * kH + feature_bin(f[2], -1.f, 1.f)], 1);
                }
            }
            pairs += __popc(__ballot_sync(kFull, oka)) + __popc(__ballot_sync(kFull, okb));
            mv += __popc(__ballot_sync(kFull, va)) + __popc(__ballot_sync(kFull, vb));
        }
        if (lane == 0) {
            const bool inJ = mv >= tau_num;  // q itself is in M[q] with B
            jflag[q] = inJ ? 1 : 0;
            flags[q] = (uint8_t)((fq & ~2u) | (inJ ? 2u : 0u));
        }
        __syncwarp();
        const float scale = pairs > 0 ? 100.0f / (float)pairs : 0.f;
        row[lane] = (float)hist[warp][lane] * scale;
        if (lane < kStride - 32) row[32 + lane] = lane == 0 ? (float)hist[warp][32] * scale : 0.f;
        __syncwarp();  // the histogram is cleared for the next query
    }
}

// Four rows per warp: the 8 lanes of group g = lane / 8 take row j of J; lane
// s = lane % 8 owns bins 4 s .. 4 s + 3 (s = 0 also bin 32) and loads them as
// one float4 of each neighbour's SPFH row, so the four groups keep four rows
// in flight per step.  Every bin adds its neighbours' values in list order
// with the compensated product-sum the list-free path uses (the same bits).
__global__ void __launch_bounds__(kThreads) fpfh_kernel(int64_t n_cap, const int32_t* __restrict__ valid,
                                                        const int64_t* __restrict__ n_valid,
                                                        const float4* __restrict__ pts,
                                                        const uint8_t* __restrict__ flags,
                                                        const int64_t* __restrict__ offs,
                                                        const int32_t* __restrict__ nbr,
                                                        const float* __restrict__ spfh, float* __restrict__ desc)
{
    // per group, the valid neighbours of one 8-entry chunk of its row's list,
    // in list order: their index and weight 1 / w_k
    __shared__ int32_t sk[kWarps][4][8];
    __shared__ float sw[kWarps][4][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 3, s = lane & 7;
    const int64_t nv = min(*n_valid, n_cap);
    const int64_t warps = (int64_t)gridDim.x * kWarps;
    for (int64_t w4 = (int64_t)blockIdx.x * kWarps + warp; w4 * 4 < nv; w4 += warps) {
        const int64_t j = w4 * 4 + g;
        const bool active = j < nv;
        int q = -1;
        float4 pq = make_float4(0.f, 0.f, 0.f, 0.f);
        int64_t b = 0, e = 0;
        if (active) {
            q = valid[j];
            pq = pts[q];
            b = offs[q];
            e = offs[q + 1];
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
        float acc32 = 0.f, comp32 = 0.f;
        int m = 0;
        for (int64_t c = 0; __any_sync(kFull, b + c < e); c += 8) {
            const int64_t t = b + c + s;
            int k = -1;
            float wt = 0.f;
            if (t < e) {
                const int kk = nbr[t];
                if (kk != q && (__ldg(&flags[kk]) & 1)) {
                    const float4 pk = __ldg(&pts[kk]);
                    const float dx = pk.x - pq.x, dy = pk.y - pq.y, dz = pk.z - pq.z;
                    const float d2 = dot3(dx, dy, dz, dx, dy, dz);
                    if (d2 > 0.f) {
                        k = kk;
                        wt = 1.0f / sqrtf(d2);
                    }
                }
            }
            const unsigned gb = (__ballot_sync(kFull, k >= 0) >> (8 * g)) & 0xFFu;
            const int cnt = __popc(gb);
            if (k >= 0) {
                const int slot = __popc(gb & ((1u << s) - 1u));
                sk[warp][g][slot] = k;
                sw[warp][g][slot] = wt;
            }
            __syncwarp();
            m += cnt;
            const int steps = __reduce_max_sync(kFull, (unsigned)cnt);
#pragma unroll 4
            for (int i = 0; i < steps; ++i) {
                if (i < cnt) {
                    const float* r = spfh + (int64_t)sk[warp][g][i] * kStride;
                    const float we = sw[warp][g][i];
                    const float4 v = __ldg(reinterpret_cast<const float4*>(r) + s);
                    kahan_add_prod(acc[0], comp[0], v.x, we);
                    kahan_add_prod(acc[1], comp[1], v.y, we);
                    kahan_add_prod(acc[2], comp[2], v.z, we);
                    kahan_add_prod(acc[3], comp[3], v.w, we);
                    if (s == 0) kahan_add_prod(acc32, comp32, __ldg(&r[32]), we);
                }
            }
            __syncwarp();
        }
        if (active) {
            const float* rq = spfh + (int64_t)q * kStride;
            const float invm = m > 0 ? 1.0f / (float)m : 0.f;
            float* out = desc + j * kStride;
            const float4 rv = reinterpret_cast<const float4*>(rq)[s];
            reinterpret_cast<float4*>(out)[s] = make_float4(fmaf(acc[0], invm, rv.x), fmaf(acc[1], invm, rv.y),
                                                            fmaf(acc[2], invm, rv.z), fmaf(acc[3], invm, rv.w));
            if (s == 0)
                reinterpret_cast<float4*>(out)[8] = make_float4(fmaf(acc32, invm, rq[32]), 0.f, 0.f, 0.f);
        }
    }
}

}  // namespace

size_t kmx_fasterpfh_scratch_bytes(int64_t n_cap, bool need_spfh)
{
    size_t total = 0;
    carve(nullptr, n_cap, need_spfh, &total);
    return total;
}

cudaError_t kmx_fasterpfh_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* prm, const float* normal4,
                                 uint8_t* flags, const int64_t* offs, const int32_t* nbr, float* desc,
                                 int32_t* valid, int64_t* n_valid, float* spfh, void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    PfhScratch s = carve(scratch, g->n_cap, spfh == nullptr, &total);
    float* sp = spfh ? spfh : s.spfh;
    const int64_t n = g->n_cap;
    cudaError_t e = cudaSuccess;
    // one wave each: both kernels are latency-bound gathers whose queries cost
    // about the same, so every resident block takes an equal share
    unsigned nbs = 0, nbf = 0;
    if ((e = kmx_wave_blocks(spfh_kernel, kThreads, 0, n, kWarps, ctx->sm_count, &nbs))) return e;
    if ((e = kmx_wave_blocks(fpfh_kernel, kThreads, 0, n, 4 * kWarps, ctx->sm_count, &nbf))) return e;
    // spfh_kernel writes the J flag of every point below the count; the scan
    // reads no other entry
    KMX_COUNT_LAUNCH();
    spfh_kernel<<<nbs, kThreads, 0, st>>>(n, g->d_n, g->pts, reinterpret_cast<const float4*>(normal4), flags,
                                          offs, nbr, prm->tau_num, sp, s.jflag);
    if ((e = kmx_scan_i32(ctx, s.jflag, n, g->d_n, s.jpos))) return e;
    KMX_COUNT_LAUNCH();
    scatter_valid<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(n, g->d_n, s.jflag, s.jpos,
                                                                                       valid, n_valid);
    KMX_COUNT_LAUNCH();
    fpfh_kernel<<<nbf, kThreads, 0, st>>>(n, valid, n_valid, g->pts, flags, offs, nbr, sp, desc);
    return cudaGetLastError();
}
