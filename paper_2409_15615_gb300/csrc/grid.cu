// Hashed uniform grid: the radius-search structure used in place of the K-d
// tree of Algorithm 1.  Points are bucketed by cell with a counting sort
// (hash insert + prefix sum + scatter); inside a cell they are put back in
// ascending point order so that every later traversal is deterministic.
#include "kmx_internal.cuh"
#include "grid_common.cuh"

namespace {

constexpr int kThreads = 256;

struct GridScratch {
    int32_t* pslot;   // [n] cell slot of each point
    int32_t* cnt;     // [T] points per slot
    int64_t* start;   // [T+1] exclusive scan of cnt
    int32_t* cursor;  // [T] fill cursor
    int32_t* tmp;     // [n] point indices grouped by cell
};

GridScratch carve(void* base, int64_t n, uint32_t T, size_t* total)
{
    GridScratch s{};
    kmx_arena a{static_cast<char*>(base), 0};
    s.pslot = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    s.cnt = (int32_t*)a.take(2 * sizeof(int32_t) * T);  // cnt and cursor, cleared together
    s.cursor = s.cnt ? s.cnt + T : nullptr;
    s.start = (int64_t*)a.take(sizeof(int64_t) * (T + 1));
    s.tmp = (int32_t*)a.take(sizeof(int32_t) * (n + 1));
    *total = kmx_align_up(a.used, 256);
    return s;
}

__global__ void __launch_bounds__(kThreads) grid_insert(const float4* __restrict__ pts, int64_t n_cap,
                                                        const int64_t* d_n, double inv_cell,
                                                        unsigned long long* keys, uint32_t T, GridScratch s,
                                                        unsigned int* err)
{
    const int64_t n = kmx_count(d_n, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        float4 p = pts[i];
        int cx, cy, cz;
        bool ok = kmx_cell_index(p.x, inv_cell, &cx) & kmx_cell_index(p.y, inv_cell, &cy) &
                  kmx_cell_index(p.z, inv_cell, &cz);
        if (!ok) {
            kmx_raise(err, KMX_DERR_RANGE);
            s.pslot[i] = -1;
            continue;
        }
        int slot = kmx_hash_insert(keys, T, kmx_pack_key(cx, cy, cz));
        s.pslot[i] = slot;
        if (slot < 0) {
            kmx_raise(err, KMX_DERR_HASHFULL);
            continue;
        }
        atomicAdd(&s.cnt[slot], 1);
    }
}

__global__ void __launch_bounds__(kThreads) grid_cells(uint32_t T, GridScratch s, int2* __restrict__ cells,
                                                       int64_t* __restrict__ n_sorted)
{
    int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t == 0) *n_sorted = s.start[T];
    if (t >= T) return;
    cells[t] = make_int2((int)s.start[t], s.cnt[t]);
}

__global__ void __launch_bounds__(kThreads) grid_scatter(int64_t n_cap, const int64_t* d_n, GridScratch s)
{
    const int64_t n = kmx_count(d_n, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const int slot = s.pslot[i];
        if (slot < 0) continue;
        const int pos = atomicAdd(&s.cursor[slot], 1);
        s.tmp[s.start[slot] + pos] = (int32_t)i;
    }
}

// One thread per point: its rank in the cell (the number of smaller point
// indices there) places it, so each cell holds its points in ascending index
// order, with the index in w.
__global__ void __launch_bounds__(kThreads) grid_fill(const float4* __restrict__ pts, int64_t n_cap,
                                                      const int64_t* d_n, GridScratch s, float4* __restrict__ sorted,
                                                      int32_t* __restrict__ sslot)
{
    const int64_t n = kmx_count(d_n, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const int slot = s.pslot[i];
        if (slot < 0) continue;
        const int L = s.cnt[slot];
        const int64_t b = s.start[slot];
        const int32_t* seg = s.tmp + b;
        int rank = 0;
        for (int f = 0; f < L; ++f) rank += (seg[f] < (int32_t)i);
        const float4 p = pts[i];
        sorted[b + rank] = make_float4(p.x, p.y, p.z, __int_as_float((int32_t)i));
        sslot[b + rank] = slot;
    }
}

}  // namespace

size_t kmx_grid_bytes(int64_t n_cap, uint32_t* table_size)
{
    uint64_t T = 1024;
    while (T < (uint64_t)(2 * n_cap)) T <<= 1;
    *table_size = (uint32_t)T;
    kmx_arena a{nullptr, 0};
    a.take(sizeof(unsigned long long) * T);
    a.take(sizeof(int2) * T);
    a.take(sizeof(float4) * (n_cap + 1));
    a.take(sizeof(int32_t) * (n_cap + 1));  // cell slot per sorted point
    a.take(sizeof(int64_t));  // grid-owned count
    a.take(sizeof(int64_t));  // bucketed count
    return kmx_align_up(a.used, 256);
}

size_t kmx_grid_scratch_bytes(int64_t n_cap, uint32_t T)
{
    size_t total = 0;
    carve(nullptr, n_cap, T, &total);
    return total;
}

cudaError_t kmx_grid_build_launch(kmx_ctx* ctx, kmx_grid* g, void* scratch)
{
    cudaStream_t st = ctx->stream;
    size_t total = 0;
    uint32_t T = g->table_size;
    GridScratch s = carve(scratch, g->n_cap, T, &total);
    cudaError_t e;
    if ((e = cudaMemsetAsync(g->keys, 0xFF, sizeof(unsigned long long) * T, st))) return e;
    if ((e = cudaMemsetAsync(s.cnt, 0, 2 * sizeof(int32_t) * T, st))) return e;  // cnt and cursor
    g->inv_cell = 1.0 / ((double)g->cell * (1.0 + KMX_CELL_MARGIN));
    const unsigned nb = kmx_stride_blocks(g->n_cap, kThreads, ctx->sm_count);
    KMX_COUNT_LAUNCH();
    grid_insert<<<nb, kThreads, 0, st>>>(g->pts, g->n_cap, g->d_n, g->inv_cell, g->keys, T, s, ctx->d_err);
    if ((e = kmx_scan_i32(ctx, s.cnt, T, nullptr, s.start))) return e;
    KMX_COUNT_LAUNCH();
    grid_cells<<<kmx_blocks(T, kThreads), kThreads, 0, st>>>(T, s, g->cells, g->d_n_sorted);
    KMX_COUNT_LAUNCH();
    grid_scatter<<<nb, kThreads, 0, st>>>(g->n_cap, g->d_n, s);
    KMX_COUNT_LAUNCH();
    grid_fill<<<nb, kThreads, 0, st>>>(g->pts, g->n_cap, g->d_n, s, g->sorted, g->sslot);
    return cudaGetLastError();
}
