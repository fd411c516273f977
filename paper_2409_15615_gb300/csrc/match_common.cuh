// Pieces shared by the FP32 and the tensor-core matching paths.
#pragma once

#include "kmx_internal.cuh"

namespace kmx {

// Best and second-best squared distance of one row, with the column of the
// best (ties to the lower column).
struct RowBest {
    float d1;
    int j1;
    float d2;
};

__device__ __forceinline__ void row_update(float& b1, int& j1, float& b2, float d, int j)
{
    if (d < b1 || (d == b1 && j < j1)) {
        b2 = b1;
        b1 = d;
        j1 = j;
    } else if (d < b2) {
        b2 = d;
    }
}

// Merge another (disjoint-column) summary into (d1, j1, d2).
__device__ __forceinline__ void row_merge(float& d1, int& j1, float& d2, float od1, int oj, float od2)
{
    if (od1 < d1 || (od1 == d1 && oj < j1)) {
        d2 = fminf(d1, od2);
        d1 = od1;
        j1 = oj;
    } else {
        d2 = fminf(d2, od1);
    }
}

// Column chunks per row tile so that row_tiles x chunks reaches about
// `target` CTAs (clamped to [1, max_chunks] and to the column tiles).
__host__ __device__ __forceinline__ int work_chunks(int64_t row_tiles, int64_t col_tiles, int64_t target,
                                                    int max_chunks)
{
    int64_t c = row_tiles > 0 ? (target + row_tiles - 1) / row_tiles : 1;
    if (c < 1) c = 1;
    if (c > max_chunks) c = max_chunks;
    if (c > col_tiles) c = col_tiles > 0 ? col_tiles : 1;
    return (int)c;
}

// Non-negative float distance in the high word, index in the low word: the
// unsigned order is (distance, index) lexicographic.
__device__ __forceinline__ unsigned long long pack_dist_index(float d, uint32_t idx)
{
    return ((unsigned long long)__float_as_uint(d) << 32) | idx;
}

struct MatchScratch {
    RowBest* part;                // [chunks][np_cap]
    unsigned long long* colbest;  // [nq_cap] packed (distance, row)
    int32_t* mflag;               // [np_cap + 1]
    int64_t* mpos;                // [np_cap + 1]
    RowBest* merged;              // [np_cap] merged row summaries
    int* chunks;                  // chunk count chosen on the device (row partials in `part`)
    void* extra;                  // path-specific scratch
};

size_t match_common_bytes(int64_t np_cap, int64_t nq_cap, int chunks, size_t extra = 0);
MatchScratch match_common_carve(void* base, int64_t np_cap, int64_t nq_cap, int chunks, size_t extra = 0);

// Merge the row partials (as many chunks as *s.chunks says), apply the
// reciprocity test and emit A in ascending source row.
cudaError_t match_finalize(kmx_ctx* ctx, const MatchScratch& s, int64_t np_cap, const int64_t* d_np,
                           const int32_t* vp, const int32_t* vq, kmx_corr* out, int64_t cap, int64_t* n_out);

// The tail of match_finalize for paths that merge their own partials: given
// s.merged and s.mflag (1 = mutual, every row < n_p written), number the
// mutual rows and emit A in ascending source row.
cudaError_t match_emit(kmx_ctx* ctx, const MatchScratch& s, int64_t np_cap, const int64_t* d_np,
                       const int32_t* vp, const int32_t* vq, kmx_corr* out, int64_t cap, int64_t* n_out);

}  // namespace kmx

// match_tc.cu
size_t kmx_match_tc_extra_bytes(int64_t np_cap, int64_t nq_cap, int sm_count);
cudaError_t kmx_match_tc_launch(kmx_ctx* ctx, const float* dp, int64_t np_cap, const int64_t* d_np, const float* dq,
                                int64_t nq_cap, const int64_t* d_nq, kmx::MatchScratch& s);
// diagnostics of the last tensor-core match on the scratch `extra` (see kmx_match_diag)
cudaError_t kmx_match_tc_stats(kmx_ctx* ctx, void* extra, int64_t np_cap, const int64_t* d_np, int64_t nq_cap,
                               const int64_t* d_nq, int64_t* dst);

// match_fp32_bulk.cu: the exact FP32 path of kmx_match (packs both sides,
// matches, merges and emits A)
size_t kmx_match_fp32_bulk_extra_bytes(int64_t np_cap, int64_t nq_cap, int sm_count);
cudaError_t kmx_match_fp32_bulk_launch(kmx_ctx* ctx, const float* dp, const int32_t* vp, int64_t np_cap,
                                       const int64_t* d_np, const float* dq, const int32_t* vq, int64_t nq_cap,
                                       const int64_t* d_nq, kmx::MatchScratch& s, kmx_corr* out, int64_t cap,
                                       int64_t* n_out);

// match_fp32.cu
int kmx_match_fp32_max_chunks();
// exact FP32 row summaries for the descriptor rows listed in rows[0..*d_nlist)
// (chunk c of list position r at part[c * list length + r]; part holds
// kmx_match_fp32_max_chunks() * (list_cap + 1) entries and the chunk count,
// at most 512, is published in *chunks_out); no column bests
cudaError_t kmx_match_fp32_rows_launch(kmx_ctx* ctx, const float* dp, const int32_t* rows, int64_t list_cap,
                                       const int64_t* d_nlist, const float* dq, int64_t nq_cap, const int64_t* d_nq,
                                       kmx::RowBest* part, int* chunks_out);
size_t kmx_match_fp32_scratch_bytes(int64_t np_cap, int64_t nq_cap, int* chunks);
cudaError_t kmx_match_fp32_launch(kmx_ctx* ctx, const float* dp, int64_t np_cap, const int64_t* d_np,
                                  const float* dq, int64_t nq_cap, const int64_t* d_nq, kmx::MatchScratch& s,
                                  int chunks);
