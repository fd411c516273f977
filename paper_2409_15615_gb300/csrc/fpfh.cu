// Algorithm 1, step 2 and the Faster-PFH descriptors (App. A, Eqs. A2-A5).
//
//   spfh_kernel  for q with B: Darboux-frame features (Eq. A2) of every pair
//                (q, k), k in I_valid(q) \ {q}, binned (Eq. A3) into a
//                per-warp shared-memory histogram and scaled by 100 / pairs
//                (Eq. A4); in the same pass |I_valid(q)| = |{ i in M[q] : B[i] }|
//                and so q in J iff B[q] and |I_valid(q)| >= tau_num, and the
//                m neighbours k != q of I_valid(q) with w_k > 0 are stored in
//                list order with their weight 1 / w_k (scratch, in the list's
//                own slots from offs[q] on)
//   scan/scatter J in ascending point order
//   fpfh_kernel  FPFH(q) = SPFH(q) + (1/m) sum_k SPFH(k) / w_k (Eq. A5) over
//                that stored list, four rows per warp, a lane owning four
//                bins, compensated summation
//
// M[q] is walked once, by the SPFH pass, which gathers every neighbour's
// point, normal and B anyway; the FPFH pass reads its neighbours and weights
// contiguously instead of gathering them again.
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
    int2* wlist;     // [nbr_cap] (k, bits of 1 / w_k) of q's FPFH neighbours from offs[q] on
    int32_t* wcnt;   // [n+1] their number m
};

PfhScratch carve(void* base, int64_t n, bool need_spfh, int64_t nbr_cap, size_t* total)
{
    PfhScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.jflag = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.jpos = (int64_t*)a.take(sizeof(int64_t) * (n + 1));
    s.spfh = need_spfh ? (float*)a.take(sizeof(float) * kStride * (n + 1)) : nullptr;
    s.wlist = (int2*)a.take(sizeof(int2) * (size_t)(nbr_cap > 0 ? nbr_cap : 1));
    s.wcnt = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
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
                                                        const int32_t* __restrict__ nbr, int64_t nbr_cap,
                                                        int tau_num, float* __restrict__ spfh,
                                                        int32_t* __restrict__ jflag, int2* __restrict__ wlist,
                                                        int32_t* __restrict__ wcnt)
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
                wcnt[q] = 0;
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
        // entries at or past nbr_cap are not read (inconsistent offsets)
        const int64_t b = offs[q], e = min(offs[q + 1], nbr_cap);
        int pairs = 0, mv = 0, m = 0;
        const unsigned below = (1u << lane) - 1u;
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
            // FPFH's neighbours in list order: k != q with B at a distance
            // w_k > 0, stored with 1 / w_k (the expressions fpfh_kernel used
            // to evaluate, so the same bits) from offs[q] on; there are at
            // most as many as list entries
            const bool fa = ha && ka != q && va, fb = hb && kb != q && vb;
            float wa = 0.f, wb = 0.f;
            bool ua = false, ub = false;
            if (fa) {
                const float dx = pa.x - pq.x, dy = pa.y - pq.y, dz = pa.z - pq.z;
                const float d2 = dot3(dx, dy, dz, dx, dy, dz);
                ua = d2 > 0.f;
                if (ua) wa = 1.0f / sqrtf(d2);
            }
            if (fb) {
                const float dx = pb.x - pq.x, dy = pb.y - pq.y, dz = pb.z - pq.z;
                const float d2 = dot3(dx, dy, dz, dx, dy, dz);
                ub = d2 > 0.f;
                if (ub) wb = 1.0f / sqrtf(d2);
            }
            const unsigned ba = __ballot_sync(kFull, ua), bb = __ballot_sync(kFull, ub);
            if (ua) wlist[b + m + __popc(ba & below)] = make_int2(ka, __float_as_int(wa));
            if (ub) wlist[b + m + __popc(ba) + __popc(bb & below)] = make_int2(kb, __float_as_int(wb));
            m += __popc(ba) + __popc(bb);
        }
        if (lane == 0) {
            const bool inJ = mv >= tau_num;  // q itself is in M[q] with B
            jflag[q] = inJ ? 1 : 0;
            wcnt[q] = m;
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
// in flight per step.  The neighbours and weights come from the list
// spfh_kernel stored (coalesced, eight entries per group and step, passed
// between the group's lanes by shuffles).  Every bin adds its neighbours'
// values in list order with the compensated product-sum the list-free path
// uses (the same bits; the four bins of a lane go through it in pairs,
// kahan_add_prod2).
__global__ void __launch_bounds__(kThreads, 6) fpfh_kernel(int64_t n_cap, const int32_t* __restrict__ valid,
                                                           const int64_t* __restrict__ n_valid,
                                                           const int64_t* __restrict__ offs,
                                                           const int2* __restrict__ wlist,
                                                           const int32_t* __restrict__ wcnt,
                                                           const float* __restrict__ spfh, float* __restrict__ desc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 3, s = lane & 7;
    const int lead = lane & ~7;  // lane 0 of the group
    const int64_t nv = min(*n_valid, n_cap);
    const int64_t warps = (int64_t)gridDim.x * kWarps;
    for (int64_t w4 = (int64_t)blockIdx.x * kWarps + warp; w4 * 4 < nv; w4 += warps) {
        const int64_t j = w4 * 4 + g;
        const bool active = j < nv;
        int q = 0, m = 0;
        int64_t b = 0;
        if (active) {
            q = valid[j];
            b = offs[q];
            m = wcnt[q];
        }
        // bins 4 s .. 4 s + 3 as two pairs of sums (negated compensations)
        float2 acc01 = make_float2(0.f, 0.f), acc23 = make_float2(0.f, 0.f);
        float2 nc01 = make_float2(0.f, 0.f), nc23 = make_float2(0.f, 0.f);
        float acc32 = 0.f, comp32 = 0.f;
        for (int c = 0; __any_sync(kFull, c < m); c += 8) {
            const int cnt = min(max(m - c, 0), 8);  // this group's entries in the chunk
            const int2 ent = s < cnt ? __ldg(&wlist[b + c + s]) : make_int2(0, 0);
            const int steps = __reduce_max_sync(kFull, (unsigned)cnt);
#pragma unroll 4
            for (int i = 0; i < steps; ++i) {
                const int k = __shfl_sync(kFull, ent.x, lead + i);
                const float we = __int_as_float(__shfl_sync(kFull, ent.y, lead + i));
                if (i < cnt) {
                    const float* r = spfh + (int64_t)k * kStride;
                    const float4 v = __ldg(reinterpret_cast<const float4*>(r) + s);
                    const float2 we2 = make_float2(we, we);
                    kahan_add_prod2(acc01, nc01, make_float2(v.x, v.y), we2);
                    kahan_add_prod2(acc23, nc23, make_float2(v.z, v.w), we2);
                    if (s == 0) kahan_add_prod(acc32, comp32, __ldg(&r[32]), we);
                }
            }
        }
        if (active) {
            const float* rq = spfh + (int64_t)q * kStride;
            const float invm = m > 0 ? 1.0f / (float)m : 0.f;
            float* out = desc + j * kStride;
            const float4 rv = reinterpret_cast<const float4*>(rq)[s];
            reinterpret_cast<float4*>(out)[s] = make_float4(fmaf(acc01.x, invm, rv.x), fmaf(acc01.y, invm, rv.y),
                                                            fmaf(acc23.x, invm, rv.z), fmaf(acc23.y, invm, rv.w));
            if (s == 0)
                reinterpret_cast<float4*>(out)[8] = make_float4(fmaf(acc32, invm, rq[32]), 0.f, 0.f, 0.f);
        }
    }
}

}  // namespace

size_t kmx_fasterpfh_scratch_bytes(int64_t n_cap, bool need_spfh, int64_t nbr_cap)
{
    size_t total = 0;
    carve(nullptr, n_cap, need_spfh, nbr_cap, &total);
    return total;
}

cudaError_t kmx_fasterpfh_launch(kmx_ctx* ctx, const kmx_grid* g, const kmx_params* prm, const float* normal4,
                                 uint8_t* flags, const int64_t* offs, const int32_t* nbr, int64_t nbr_cap,
                                 float* desc, int32_t* valid, int64_t* n_valid, float* spfh, void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    PfhScratch s = carve(scratch, g->n_cap, spfh == nullptr, nbr_cap, &total);
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
                                          offs, nbr, nbr_cap, prm->tau_num, sp, s.jflag, s.wlist, s.wcnt);
    if ((e = kmx_scan_i32(ctx, s.jflag, n, g->d_n, s.jpos))) return e;
    KMX_COUNT_LAUNCH();
    scatter_valid<<<kmx_stride_blocks(n, kThreads, ctx->sm_count), kThreads, 0, st>>>(n, g->d_n, s.jflag, s.jpos,
                                                                                       valid, n_valid);
    KMX_COUNT_LAUNCH();
    fpfh_kernel<<<nbf, kThreads, 0, st>>>(n, valid, n_valid, offs, s.wlist, s.wcnt, sp, desc);
    return cudaGetLastError();
}
