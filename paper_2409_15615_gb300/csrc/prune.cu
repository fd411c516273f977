// Correspondence pruning of Sec. III-D on the device: the ratio filter (the
// N_tau correspondences with the lowest d1 / d2), the pairwise-invariant
// compatibility graph of Eq. 3, and the maximum k-core.
//
//   ratio_keys        ratio = d1 / d2 in FP64 (1 when d2 = 0), a 4096-bucket
//                     histogram of it.
//   ratio_threshold   one block: the first bucket B at which the cumulative
//                     count reaches N_tau.
//   ratio_candidates  the correspondences in buckets <= B (every one of the
//                     N_tau lowest is among them; all others rank higher).
//   ratio_rank        each candidate's exact rank among the candidates by
//                     (ratio, i); ranks < N_tau give the selection in
//                     ascending order, with both end points gathered.
//   graph_build       one 32-bit word of the adjacency bit matrix per thread:
//                     k ~ k' iff | |b_k - b_k'| - |a_k - a_k'| | <= 2 beta.  The
//                     test runs in FP32; within a band around the threshold it
//                     is decided again in FP64 as ((dx dx + dy dy) + dz dz),
//                     sqrt, |db - da| <= 2 beta, so every edge is the FP64
//                     decision.
//   kcore             one cooperative launch: the core numbers as the fixed
//                     point of c(v) <- H({c(u) : u ~ v}) started from the
//                     degrees (H = h-index: the largest h with at least h
//                     values >= h; the values only decrease and stay above the
//                     core numbers, so in-place updates converge to them),
//                     sweeps separated by a bounded grid barrier, until a
//                     sweep changes nothing; then the largest core number
//                     and the positions of the maximum k-core in ascending
//                     order.
#include "kmx_internal.cuh"

#include <cooperative_groups.h>

namespace {

constexpr int kBuckets = 4096;
constexpr int kThreads = 256;
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr int kMaxSweeps = 1 << 16;
constexpr int kHistCap = 2048;  // per-warp histogram of capped neighbour values (values below it)

struct PruneScratch {
    double* ratio;            // [n_cap]
    int32_t* bucket;          // [n_cap]
    int32_t* hist;            // [kBuckets]
    int32_t* cand;            // [n_cap]
    unsigned long long* ckey; // [n_cap] candidate ratio bits
    int32_t* ci;              // [n_cap] candidate source index i
    int32_t* n_cand;          // [1]
    int32_t* thr;             // [1] threshold bucket
    float4* pa;               // [n_tau] source end point of each selected correspondence
    float4* pb;               // [n_tau] target end point
    uint32_t* adj;            // [n_tau][words]
    int32_t* core;            // [n_tau] working values (copied to the caller)
    uint32_t* sync;           // [8] barrier count, barrier generation, change counters x3, work counters x3
};

__device__ __forceinline__ int64_t corr_count(const int64_t* d_n, int64_t cap)
{
    if (!d_n) return cap;
    const int64_t n = *d_n;
    return n < 0 ? 0 : (n > cap ? cap : n);
}

__global__ void __launch_bounds__(kThreads) ratio_keys(const kmx_corr* __restrict__ corr, int64_t cap,
                                                      const int64_t* d_n, PruneScratch s)
{
    const int64_t n = corr_count(d_n, cap);
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads) {
        const double d1 = (double)corr[k].d1, d2 = (double)corr[k].d2;
        const double r = d2 > 0.0 ? __ddiv_rn(d1, d2) : 1.0;
        s.ratio[k] = r;
        int b = (int)(r * (double)kBuckets);  // r in [0, 1]; exact scaling by a power of two
        b = b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
        s.bucket[k] = b;
        atomicAdd(&s.hist[b], 1);
    }
}

__global__ void __launch_bounds__(1024) ratio_threshold(int32_t n_tau, PruneScratch s)
{
    __shared__ int32_t part[1024];
    constexpr int kPer = kBuckets / 1024;
    int32_t loc = 0;
    for (int e = 0; e < kPer; ++e) loc += s.hist[threadIdx.x * kPer + e];
    part[threadIdx.x] = loc;
    __syncthreads();
    // inclusive prefix over the 1024 partial sums (Hillis-Steele)
    for (int o = 1; o < 1024; o <<= 1) {
        const int32_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int32_t before = threadIdx.x ? part[threadIdx.x - 1] : 0;
    if (threadIdx.x == 1023 && part[1023] < n_tau) *s.thr = kBuckets - 1;  // fewer than N_tau in all
    if (before < n_tau && part[threadIdx.x] >= n_tau) {
        int32_t c = before;
        for (int e = 0; e < kPer; ++e) {
            c += s.hist[threadIdx.x * kPer + e];
            if (c >= n_tau) {
                *s.thr = threadIdx.x * kPer + e;
                break;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) ratio_candidates(const kmx_corr* __restrict__ corr, int64_t cap,
                                                            const int64_t* d_n, PruneScratch s)
{
    const int64_t n = corr_count(d_n, cap);
    const int32_t thr = *s.thr;
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < n; k += (int64_t)gridDim.x * kThreads)
        if (s.bucket[k] <= thr) {
            const int c = atomicAdd(s.n_cand, 1);
            s.cand[c] = (int32_t)k;
            s.ckey[c] = (unsigned long long)__double_as_longlong(s.ratio[k]);
            s.ci[c] = corr[k].i;
        }
}

// (ratio, i) lexicographic: a non-negative double orders like its bits.
__device__ __forceinline__ bool key_less(unsigned long long ra, int32_t ia, unsigned long long rb, int32_t ib)
{
    return ra < rb || (ra == rb && ia < ib);
}

// One warp per candidate: its rank among the candidates (the lanes stride
// over the compact keys).
__global__ void __launch_bounds__(kThreads) ratio_rank(const kmx_corr* __restrict__ corr, int32_t n_tau,
                                                      const float4* __restrict__ src4,
                                                      const float4* __restrict__ tgt4, PruneScratch s,
                                                      int32_t* __restrict__ sel)
{
    const int m = *s.n_cand;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (kThreads / 32);
    for (int c = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); c < m; c += warps) {
        const unsigned long long rk = s.ckey[c];
        const int32_t ik = s.ci[c];
        int rank = 0;
        for (int f = lane; f < m; f += 32) rank += key_less(s.ckey[f], s.ci[f], rk, ik);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
        if (lane == 0 && rank < n_tau) {
            const int32_t k = s.cand[c];
            sel[rank] = k;
            const kmx_corr e = corr[k];
            s.pa[rank] = src4[e.i];
            s.pb[rank] = tgt4[e.j];
        }
    }
}

__device__ __forceinline__ bool edge_fp64(float4 a, float4 a2, float4 b, float4 b2, double two_beta)
{
    const double ax = (double)a.x - (double)a2.x, ay = (double)a.y - (double)a2.y, az = (double)a.z - (double)a2.z;
    const double bx = (double)b.x - (double)b2.x, by = (double)b.y - (double)b2.y, bz = (double)b.z - (double)b2.z;
    const double da = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az)));
    const double db = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz)));
    return fabs(__dadd_rn(db, -da)) <= two_beta;
}

// Thread (v, w): bits u = 32 w .. 32 w + 31 of row v.  The degree of v is the
// popcount of its row.
__global__ void __launch_bounds__(kThreads) graph_build(int32_t n_tau, const int64_t* d_n_sel, double two_beta,
                                                       PruneScratch s, int32_t words)
{
    const int64_t nsel = *d_n_sel;
    const int64_t total = nsel * words;
    const float tb = (float)two_beta;
    // consecutive threads share w (the 32 end-point pairs they read are the same)
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < total; t += (int64_t)gridDim.x * kThreads) {
        const int w = (int)(t / nsel), v = (int)(t - (int64_t)w * nsel);
        const float4 a = s.pa[v], b = s.pb[v];
        uint32_t bits = 0;
        for (int e = 0; e < 32; ++e) {
            const int u = w * 32 + e;
            if (u >= nsel || u == v) continue;
            const float4 a2 = s.pa[u], b2 = s.pb[u];
            const float ax = a.x - a2.x, ay = a.y - a2.y, az = a.z - a2.z;
            const float bx = b.x - b2.x, by = b.y - b2.y, bz = b.z - b2.z;
            const float da = sqrtf(fmaf(az, az, fmaf(ay, ay, ax * ax)));
            const float db = sqrtf(fmaf(bz, bz, fmaf(by, by, bx * bx)));
            const float gap = fabsf(db - da) - tb;
            // FP32 carries a few ulp of the distances; decide again in FP64 near the threshold
            const float band = 1e-5f * (1.0f + da + db);
            bool on;
            if (gap > band)
                on = false;
            else if (gap < -band)
                on = true;
            else
                on = edge_fp64(a, a2, b, b2, two_beta);
            bits |= (uint32_t)on << e;
        }
        s.adj[(int64_t)v * words + w] = bits;
        if (bits) atomicAdd(&s.core[v], __popc(bits));
    }
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }

// Bounded grid barrier (sense by generation); false when a spin ran out.
__device__ bool grid_barrier(uint32_t* count, uint32_t* gen, uint32_t nblocks)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const uint32_t g = ld_volatile(gen);
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            uint32_t it = 0;
            while (ld_volatile(gen) == g) {
                if (++it > kSpinLimit) {
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// count of neighbours u of v with c(u) >= h over the block's snapshot of c
// (warp-wide, every lane gets it)
__device__ __forceinline__ int count_ge(const uint32_t* __restrict__ row, int words, const int32_t* snap, int h)
{
    int cnt = 0;
    for (int w = threadIdx.x & 31; w < words; w += 32) {
        uint32_t bits = row[w];
        while (bits) {
            const int e = __ffs(bits) - 1;
            bits &= bits - 1;
            cnt += snap[w * 32 + e] >= h;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    return cnt;
}

__global__ void __launch_bounds__(kThreads) kcore(const int64_t* d_n_sel, int32_t words, PruneScratch s,
                                                 int32_t* __restrict__ core_out, int32_t* __restrict__ kmax_out,
                                                 int32_t* __restrict__ inlier, int64_t* __restrict__ n_inlier,
                                                 unsigned int* __restrict__ err)
{
    const int nsel = (int)*d_n_sel;
    const uint32_t nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    int32_t* c = s.core;
    uint32_t* bar_count = s.sync;
    uint32_t* bar_gen = s.sync + 1;
    uint32_t* changed = s.sync + 2;  // three rotating counters
    // dynamic shared memory: per-warp histograms of kHistCap ints, then the
    // snapshot of c taken at the start of each sweep
    extern __shared__ int32_t dyn[];
    int32_t* hist = dyn + (threadIdx.x >> 5) * kHistCap;
    int32_t* snap = dyn + (kThreads / 32) * kHistCap;
    uint32_t* work = s.sync + 5;  // three rotating per-sweep vertex counters
    __shared__ uint32_t block_changed;
    bool ok = true;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        if (threadIdx.x == 0) block_changed = 0;
        for (int v = threadIdx.x; v < nsel; v += kThreads) snap[v] = *reinterpret_cast<const volatile int32_t*>(&c[v]);
        __syncthreads();
        while (true) {
            int v = 0;
            if (lane == 0) v = (int)atomicAdd(&work[sweep % 3], 1u);
            v = __shfl_sync(0xffffffffu, v, 0);
            if (v >= nsel) break;
            const int cv = snap[v];
            if (cv == 0) continue;
            const uint32_t* row = s.adj + (int64_t)v * words;
            int h = cv;
            if (count_ge(row, words, snap, cv) < cv) {
                if (cv < kHistCap) {
                    // histogram of min(c(u), cv), then the largest h with at
                    // least h values >= h, scanning 32 h's at a time from cv down
                    for (int e = lane; e <= cv; e += 32) hist[e] = 0;
                    __syncwarp();
                    for (int w = lane; w < words; w += 32) {
                        uint32_t bits = row[w];
                        while (bits) {
                            const int b = __ffs(bits) - 1;
                            bits &= bits - 1;
                            atomicAdd(&hist[min(snap[w * 32 + b], cv)], 1);
                        }
                    }
                    __syncwarp();
                    int suffix = 0;
                    for (int top = cv;; top -= 32) {
                        const int hh = top - lane;
                        int x = hh >= 0 ? hist[hh] : 0;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int y = __shfl_up_sync(0xffffffffu, x, o);
                            if (lane >= o) x += y;
                        }
                        const unsigned hit = __ballot_sync(0xffffffffu, hh >= 0 && suffix + x >= hh);
                        if (hit) {
                            h = top - (__ffs(hit) - 1);
                            break;
                        }
                        suffix += __shfl_sync(0xffffffffu, x, 31);
                    }
                    __syncwarp();
                } else {
                    // the largest h < cv with count_ge(h) >= h (count_ge falls as h grows)
                    int lo = 0, hi = cv - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (count_ge(row, words, snap, mid) >= mid)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    h = lo;
                }
            }
            if (h != cv) {
                if (lane == 0) {
                    *reinterpret_cast<volatile int32_t*>(&c[v]) = h;
                    atomicAdd(&block_changed, 1u);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (block_changed) atomicAdd(&changed[sweep % 3], block_changed);
            if (blockIdx.x == 0) {
                changed[(sweep + 1) % 3] = 0;
                work[(sweep + 1) % 3] = 0;
            }
        }
        if (!grid_barrier(bar_count, bar_gen, nblocks)) {
            ok = false;
            break;
        }
        if (ld_volatile(&changed[sweep % 3]) == 0) break;
    }
    if (!ok) {
        if (threadIdx.x == 0) kmx_raise(err, KMX_DERR_TIMEOUT);
        return;
    }
    if (blockIdx.x != 0) return;
    // block 0: largest core number, then the maximum k-core in ascending order
    __shared__ int32_t red[kThreads];
    __shared__ int32_t base;
    int32_t mx = 0;
    for (int v = threadIdx.x; v < nsel; v += kThreads) {
        const int32_t cv = *reinterpret_cast<const volatile int32_t*>(&c[v]);
        core_out[v] = cv;
        mx = max(mx, cv);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    const int32_t kmax = red[0];
    if (threadIdx.x == 0) {
        *kmax_out = kmax;
        base = 0;
    }
    __syncthreads();
    for (int v0 = 0; v0 < nsel; v0 += kThreads) {
        const int v = v0 + threadIdx.x;
        const bool in = v < nsel && nsel > 0 && *reinterpret_cast<const volatile int32_t*>(&c[v]) == kmax;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        __shared__ int32_t wcount[kThreads / 32];
        if (lane == 0) wcount[threadIdx.x >> 5] = __popc(bal);
        __syncthreads();
        int off = base;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) off += wcount[w];
        if (in) inlier[off + __popc(bal & ((1u << lane) - 1u))] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) tot += wcount[w];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_inlier = base;
}

__global__ void set_n_sel(const int64_t* d_n, int64_t cap, int32_t n_tau, int64_t* n_sel)
{
    const int64_t n = corr_count(d_n, cap);
    *n_sel = n < n_tau ? n : n_tau;
}

int32_t words_for(int32_t n_tau) { return (n_tau + 31) / 32; }

PruneScratch carve(void* base, int64_t cap, int32_t n_tau, size_t* total)
{
    kmx_arena a{static_cast<char*>(base), 0};
    PruneScratch s{};
    s.ratio = static_cast<double*>(a.take(sizeof(double) * (cap + 1)));
    s.bucket = static_cast<int32_t*>(a.take(sizeof(int32_t) * (cap + 1)));
    s.cand = static_cast<int32_t*>(a.take(sizeof(int32_t) * (cap + 1)));
    s.ckey = static_cast<unsigned long long*>(a.take(sizeof(unsigned long long) * (cap + 1)));
    s.ci = static_cast<int32_t*>(a.take(sizeof(int32_t) * (cap + 1)));
    s.pa = static_cast<float4*>(a.take(sizeof(float4) * (n_tau + 1)));
    s.pb = static_cast<float4*>(a.take(sizeof(float4) * (n_tau + 1)));
    s.adj = static_cast<uint32_t*>(a.take(sizeof(uint32_t) * ((size_t)n_tau * words_for(n_tau) + 1)));
    // zeroed together: histogram, candidate count, threshold, core (degree) counters, sync words
    const size_t zero_words = kBuckets + 2 + (size_t)n_tau + 8;
    int32_t* z = static_cast<int32_t*>(a.take(sizeof(int32_t) * zero_words));
    s.hist = z;
    s.n_cand = z + kBuckets;
    s.thr = z + kBuckets + 1;
    s.core = z + kBuckets + 2;
    s.sync = reinterpret_cast<uint32_t*>(z + kBuckets + 2 + n_tau);
    *total = kmx_align_up(a.used, 256);
    return s;
}

size_t zero_bytes(int32_t n_tau) { return sizeof(int32_t) * (kBuckets + 2 + (size_t)n_tau + 8); }

}  // namespace

size_t kmx_prune_scratch_bytes(int64_t corr_cap, int32_t n_tau)
{
    size_t total = 0;
    carve(nullptr, corr_cap, n_tau, &total);
    return total;
}

cudaError_t kmx_prune_launch(kmx_ctx* ctx, const kmx_corr* corr, int64_t cap, const int64_t* d_n,
                             const float4* src4, const float4* tgt4, int32_t n_tau, double beta, int32_t* sel,
                             int64_t* n_sel, int32_t* core_out, int32_t* kmax, int32_t* inlier, int64_t* n_inlier,
                             void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    PruneScratch s = carve(scratch, cap, n_tau, &total);
    cudaError_t e;
    if ((e = cudaMemsetAsync(s.hist, 0, zero_bytes(n_tau), st))) return e;
    const unsigned grid = 4u * (unsigned)ctx->sm_count;
    KMX_COUNT_LAUNCH();
    set_n_sel<<<1, 1, 0, st>>>(d_n, cap, n_tau, n_sel);
    KMX_COUNT_LAUNCH();
    ratio_keys<<<grid, kThreads, 0, st>>>(corr, cap, d_n, s);
    KMX_COUNT_LAUNCH();
    ratio_threshold<<<1, 1024, 0, st>>>(n_tau, s);
    KMX_COUNT_LAUNCH();
    ratio_candidates<<<grid, kThreads, 0, st>>>(corr, cap, d_n, s);
    KMX_COUNT_LAUNCH();
    ratio_rank<<<grid, kThreads, 0, st>>>(corr, n_tau, src4, tgt4, s, sel);
    const int32_t words = words_for(n_tau);
    KMX_COUNT_LAUNCH();
    graph_build<<<grid, kThreads, 0, st>>>(n_tau, n_sel, 2.0 * beta, s, words);
    // one CTA per SM (co-resident under a cooperative launch: the sweeps wait
    // on one another through the grid barrier)
    const size_t snap_bytes = sizeof(int32_t) * ((size_t)n_tau + (size_t)(kThreads / 32) * kHistCap);
    // this call is never captured (cooperative launch), so the opt-in is set
    // to the exact size on every call
    if (snap_bytes > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kcore, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)snap_bytes)))
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kcore, kThreads, snap_bytes))) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const unsigned kgrid = (unsigned)ctx->sm_count;
    const int64_t* n_sel_c = n_sel;
    int32_t words_c = words;
    unsigned int* err = ctx->d_err;
    void* args[] = {(void*)&n_sel_c, (void*)&words_c, (void*)&s, (void*)&core_out, (void*)&kmax, (void*)&inlier,
                    (void*)&n_inlier, (void*)&err};
    KMX_COUNT_LAUNCH();
    return cudaLaunchCooperativeKernel((const void*)kcore, dim3(kgrid), dim3(kThreads), args, snap_bytes, st);
}
