// Shared end of both matching paths: merge row partials, reciprocity test
// (Sec. III-C), ordered emission of the correspondence set A.
#include "match_common.cuh"

namespace kmx {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) merge_mutual(const RowBest* __restrict__ part,
                                                         const int* __restrict__ d_chunks, int64_t np_cap,
                                                         const int64_t* d_np,
                                                         const unsigned long long* __restrict__ colbest,
                                                         RowBest* __restrict__ merged, int32_t* __restrict__ mflag)
{
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= kmx_count(d_np, np_cap)) return;
    RowBest r = part[i];
    const int chunks = *d_chunks;
    for (int c = 1; c < chunks; ++c) {
        const RowBest o = part[(int64_t)c * np_cap + i];
        row_merge(r.d1, r.j1, r.d2, o.d1, o.j1, o.d2);
    }
    merged[i] = r;
    bool mutual = false;
    if (r.j1 >= 0 && r.j1 != 0x7fffffff) mutual = (uint32_t)(colbest[r.j1] & 0xffffffffull) == (uint32_t)i;
    mflag[i] = mutual ? 1 : 0;
}

__global__ void __launch_bounds__(kThreads) emit(int64_t np_cap, const int64_t* d_np,
                                                 const RowBest* __restrict__ merged,
                                                 const int32_t* __restrict__ mflag, const int64_t* __restrict__ mpos,
                                                 const int32_t* __restrict__ vp, const int32_t* __restrict__ vq,
                                                 kmx_corr* __restrict__ out, int64_t cap, int64_t* n_out,
                                                 unsigned int* err)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t tot = mpos[np_cap];
        *n_out = tot;
        if (tot > cap) kmx_raise(err, KMX_DERR_CAPACITY);
    }
    const int64_t n = kmx_count(d_np, np_cap);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        if (!mflag[i]) continue;
        const int64_t p = mpos[i];
        if (p >= cap) continue;
        const RowBest r = merged[i];
        kmx_corr c;
        c.i = vp ? vp[i] : (int32_t)i;
        c.j = vq ? vq[r.j1] : r.j1;
        c.d1 = sqrtf(r.d1);
        c.d2 = sqrtf(r.d2);
        out[p] = c;
    }
}

}  // namespace

size_t match_common_bytes(int64_t np_cap, int64_t nq_cap, int chunks, size_t extra)
{
    kmx_arena a{nullptr, 0};
    a.take(sizeof(RowBest) * (size_t)chunks * (np_cap + 1));
    a.take(sizeof(unsigned long long) * (nq_cap + 1));
    a.take(sizeof(int32_t) * (np_cap + 1));
    a.take(sizeof(int64_t) * (np_cap + 1));
    a.take(sizeof(RowBest) * (np_cap + 1));
    a.take(sizeof(int) * 4);
    a.take(extra);
    return kmx_align_up(a.used, 256);
}

MatchScratch match_common_carve(void* base, int64_t np_cap, int64_t nq_cap, int chunks, size_t extra)
{
    MatchScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.part = (RowBest*)a.take(sizeof(RowBest) * (size_t)chunks * (np_cap + 1));
    s.colbest = (unsigned long long*)a.take(sizeof(unsigned long long) * (nq_cap + 1));
    s.mflag = (int32_t*)a.take(sizeof(int32_t) * (np_cap + 1));
    s.mpos = (int64_t*)a.take(sizeof(int64_t) * (np_cap + 1));
    s.merged = (RowBest*)a.take(sizeof(RowBest) * (np_cap + 1));
    s.chunks = (int*)a.take(sizeof(int) * 4);
    s.extra = a.take(extra);
    return s;
}

cudaError_t match_finalize(kmx_ctx* ctx, const MatchScratch& s, int64_t np_cap, const int64_t* d_np,
                           const int32_t* vp, const int32_t* vq, kmx_corr* out, int64_t cap, int64_t* n_out)
{
    cudaStream_t st = ctx->stream;
    RowBest* merged = s.merged;
    cudaError_t e;
    if ((e = cudaMemsetAsync(s.mflag, 0, sizeof(int32_t) * (np_cap + 1), st))) return e;
    const unsigned nb = kmx_blocks(np_cap, kThreads);
    KMX_COUNT_LAUNCH();
    merge_mutual<<<nb, kThreads, 0, st>>>(s.part, s.chunks, np_cap, d_np, s.colbest, merged, s.mflag);
    if ((e = cudaGetLastError())) return e;
    return match_emit(ctx, s, np_cap, d_np, vp, vq, out, cap, n_out);
}

cudaError_t match_emit(kmx_ctx* ctx, const MatchScratch& s, int64_t np_cap, const int64_t* d_np,
                       const int32_t* vp, const int32_t* vq, kmx_corr* out, int64_t cap, int64_t* n_out)
{
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    if ((e = kmx_scan_i32(ctx, s.mflag, np_cap, d_np, s.mpos))) return e;
    KMX_COUNT_LAUNCH();
    emit<<<kmx_stride_blocks(np_cap, kThreads, ctx->sm_count), kThreads, 0, st>>>(np_cap, d_np, s.merged, s.mflag,
                                                                                   s.mpos, vp, vq, out, cap, n_out,
                                                                                   ctx->d_err);
    return cudaGetLastError();
}

}  // namespace kmx
