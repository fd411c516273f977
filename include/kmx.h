/*
 * kmx.h - C ABI of the GB300 (sm_103a) implementation of the KISS-Matcher
 * front end (arXiv 2409.15615): voxel downsampling, radius neighbourhoods,
 * reliable normals, Faster-PFH descriptors and mutual nearest-neighbour
 * descriptor matching.  The output is the correspondence set A that the
 * k-core pruning of Sec. III-D consumes.
 *
 * General conventions (apply to every entry point below)
 *  - Pointers named d_* are DEVICE memory owned by the caller.  The library
 *    never frees them and never keeps them past the call, except where a
 *    function says so (kmx_build_grid keeps d_xyz4).
 *  - Every call is asynchronous on the context's stream (kmx_set_stream).
 *    Scalar results (counts) are written to caller-provided device int64
 *    cells, so a pipeline of calls needs no host synchronisation.  Host
 *    return values report only argument and launch errors.
 *  - Errors detected on the device (index range, capacity, hash overflow)
 *    are recorded in the context and reported by the next kmx_sync(), which
 *    synchronises the stream, returns the first such error and clears it.
 *    Outputs of a call whose device error is reported are unspecified.
 *  - Sizes named *_cap are host-side capacities (upper bounds); the matching
 *    d_n* argument, when non-NULL, holds the actual count on the device (as
 *    written by an earlier call) and must be <= the capacity.  When it is
 *    NULL the capacity is the exact count.
 *  - Scratch memory is owned by the context; a call may grow it with
 *    stream-ordered allocation (cudaMallocAsync).  kmx_reserve() sizes it in
 *    advance.
 *  - Point clouds are float32.  "xyz4" layout is [n][4] (x, y, z, pad),
 *    16-byte aligned rows.
 *  - No function aborts the process, traps the device or falls back to the
 *    CPU.
 */
#ifndef KMX_H
#define KMX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KMX_OK = 0,
    KMX_EINVAL = 1,    /* bad argument: NULL pointer, negative size, bad stride, misaligned row */
    KMX_ENOMEM = 2,    /* device allocation failed */
    KMX_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    KMX_ERANGE = 4,    /* a voxel or grid-cell index does not fit in 21 bits */
    KMX_ECAPACITY = 5, /* an output buffer was too small; the needed size is in the *needed cell */
    KMX_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
    KMX_EBUSY = 7      /* the context is in use by a stream capture */
} kmx_status;

/* Faster-PFH parameters (Sec. III-C and Sec. IV-B).  All radii are in the
 * units of the cloud.  kmx_params_default(v) sets the paper's values:
 * r_normal = 3.5 v, r_fpfh = 5.0 v, tau_num = 3, tau_lin = 0.99, 11 bins per
 * angular feature (33-D descriptor), viewpoint at the origin. */
typedef struct {
    float voxel;        /* voxel size v */
    float r_normal;     /* normal radius, <= r_fpfh (Sec. III-C) */
    float r_fpfh;       /* FPFH radius (Eq. A1) */
    int32_t tau_num;    /* cardinality threshold (Algorithm 1) */
    float tau_lin;      /* linearity threshold (Algorithm 1) */
    int32_t hist_bins;  /* H of Eq. A3; only 11 is supported */
    float viewpoint[3]; /* normals are oriented toward this point */
} kmx_params;

/* Geometric suppression (Sec. III-B): ground removal before the descriptors.
 * The paper uses Patchwork (Lim et al., RA-L 2021) without restating it;
 * kmx_suppress_ground implements a stand-in with Patchwork's concentric zone
 * model and region-wise ground plane fitting.  Sensor frame, z up; lengths in
 * the cloud's units.  kmx_ground_params_default() sets: zone edges 2.7, 12.3,
 * 22.1, 41.1, 80 m; rings 2, 4, 4, 4 and sectors 16, 32, 54, 32 per zone;
 * quant_log2 8; z_limit 80; n_lpr 20; th_seeds = th_dist = 0.125; n_iter 3;
 * max_slope 1 (45 degrees); max_ground_z -0.8 (a sensor ~1.7 m above the
 * road); min_points 10; max_bin_points 65536. */
typedef struct {
    float zone_r[5];          /* zone edges, increasing, > 0 */
    int32_t zone_rings[4];    /* equal-width rings per zone, 1..1024 */
    int32_t zone_sectors[4];  /* sectors per zone (equal steps of the pseudo-angle), 1..1024 */
    int32_t quant_log2;       /* the fit works on coordinates rounded to 2^-quant_log2, 0..12;
                                 zone_r[4] and z_limit times 2^quant_log2 must not exceed 32767 */
    float z_limit;            /* points with |z| >= z_limit are never ground */
    int32_t n_lpr;            /* lowest points averaged into the seed height, 1..1024 */
    float th_seeds;           /* seeds lie below that height + th_seeds */
    float th_dist;            /* ground points lie within th_dist of the plane (orthogonally) */
    int32_t n_iter;           /* refits, 0..64 */
    float max_slope;          /* accept a plane with a^2 + b^2 <= max_slope^2 */
    float max_ground_z;       /* accept a plane whose ground points' mean height is below this */
    int32_t min_points;       /* bins with fewer members are not fitted (>= 3) */
    int32_t max_bin_points;   /* bins with more members are not fitted (<= 65536) */
} kmx_ground_params;

/* Descriptor rows: 33 used floats padded to 36 (144 bytes). */
#define KMX_DESC_DIM 33
#define KMX_DESC_STRIDE 36

/* One correspondence of A (Sec. III-C): i indexes the source (voxelised)
 * cloud, j the target cloud; d1 and d2 are the descriptor distances from
 * FPFH(i) to its nearest and second-nearest target descriptors (d2 feeds the
 * ratio test of Sec. III-D). */
typedef struct {
    int32_t i, j;
    float d1, d2;
} kmx_corr;

typedef enum {
    KMX_MATCH_FP32_EXACT = 0, /* exact FP32 distances on CUDA cores */
    /* BF16 tensor-core distances (FP32 accumulation) on descriptors sorted
     * into similar 128-row tiles (the leaves of a principal-direction tree)
     * and centred per tile pair give, per row, a candidate list that provably
     * holds every column whose exact distance is at most the row's
     * second-smallest one (certified lower and upper bounds); tile pairs
     * that the triangle inequality rules out (centre distance minus tile
     * radius beyond a row's bound) are not computed; the candidates are
     * re-ranked exactly in FP32, and a row whose
     * list overflows (512) goes through the exact FP32 tiles.  The result
     * equals KMX_MATCH_FP32_EXACT's, including KMX_ERANGE for NaN or
     * infinite values. */
    KMX_MATCH_BF16_RERANK = 1
} kmx_match_mode;

typedef struct kmx_ctx kmx_ctx;   /* opaque, owned by the library */
typedef struct kmx_grid kmx_grid; /* opaque, owned by the library */

/* Fill *out with the paper's parameters for voxel size v (Sec. IV-B).
 * Returns KMX_EINVAL if out is NULL or v is not positive and finite. */
kmx_status kmx_params_default(float v, kmx_params* out);

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out is owned by the
 * caller and released with kmx_destroy.
 * A context owns a scratch area and a small zeroed area for the look-back
 * words of its prefix scans; a call grows either one (stream-ordered) when
 * it needs more.  To capture a call sequence into a CUDA graph, run it once
 * with the same sizes first, so that the captured calls allocate nothing.
 * Calls on one context must be ordered (one stream, or events between
 * streams): they share these areas. */
kmx_status kmx_create(kmx_ctx** out, int device, void* cuda_stream);

/* Release the context and its scratch memory (synchronises its stream). */
void kmx_destroy(kmx_ctx* ctx);

/* Issue subsequent work on another stream of the same device. */
kmx_status kmx_set_stream(kmx_ctx* ctx, void* cuda_stream);

/* Residency of the exact FP32 matcher (kmx_match, KMX_MATCH_FP32_EXACT):
 * its tile kernel runs as ctas_per_sm resident CTAs on every SM (1 or 2;
 * 0 restores the default, 2).  Each CTA holds about 95 KB of shared memory and
 * half of an SM's registers, so with 2 the matcher fills the GPU (fastest
 * for one matching at a time) and with 1 half of every SM stays free for
 * kernels on other streams, e.g. the feature chains of other pairs in
 * flight.  The results do not depend on it.  Not from the paper: a
 * scheduling choice.  Returns KMX_EINVAL for other values. */
kmx_status kmx_set_match_residency(kmx_ctx* ctx, int ctas_per_sm);

/* Work-item size of the exact FP32 matcher (KMX_MATCH_FP32_EXACT): its tile
 * kernel cuts the (row tile x column tile) sequence into about
 * chunks_per_cta chunks per resident CTA, which the CTAs take from a device
 * counter (smaller ones at the end of the sequence); 1..32, 0 restores the
 * default 8.  Larger values balance uneven tile pairs better, smaller ones
 * keep a source tile longer in shared memory.  The results do not depend on
 * it.  Not from the paper: a scheduling parameter (the batch autotuner
 * searches it).  Returns KMX_EINVAL for other values. */
kmx_status kmx_set_match_chunks(kmx_ctx* ctx, int chunks_per_cta);

/* Make sure the context scratch holds at least `bytes` bytes. */
kmx_status kmx_reserve(kmx_ctx* ctx, int64_t bytes);

/* Wait for the context's stream; return (and clear) the first device-side
 * error recorded since the last kmx_sync, else KMX_OK. */
kmx_status kmx_sync(kmx_ctx* ctx);

/* Human-readable description of the last error reported on this context. */
const char* kmx_last_error(const kmx_ctx* ctx);

/* Number of CUDA kernels the library has launched in this process, over all
 * contexts (diagnostics; a relaxed atomic counter, never reset).  Not from
 * the paper: it lets a caller count the device work of a call sequence. */
int64_t kmx_launch_count(void);

/* Failure-path check (not from the paper): launch one block that polls a
 * device flag nothing sets, at most `polls` times, the
 * same bounded-wait pattern the tensor-core matcher uses on its mbarriers
 * (polls <= 2^24, a few seconds at most).
 * When the polls run out the kernel records KMX_ETIMEOUT and returns, so the
 * next kmx_sync reports KMX_ETIMEOUT and the context stays usable. */
kmx_status kmx_check_timeout(kmx_ctx* ctx, int64_t polls);

/*
 * Voxel downsampling: the voxelised input clouds of Sec. III-A ("unordered
 * voxelized point clouds with a voxel size v").
 *   d_xyz     [n_raw][stride] float32 points, stride 3 or 4.
 *   voxel     v > 0.  A point belongs to voxel floor(x / v) per axis, with
 *             the quotient computed in FP64 (half-open cells).
 *   d_out4    [cap][4] float32: the centroid of each occupied voxel (its
 *             members summed in FP64 in input order, divided by the count in
 *             FP64, rounded to FP32), w = 0.  Voxels appear in the order of
 *             their first member in the input.
 *   d_n_out   device int64: number of voxels written.
 *   d_assign  nullable [n_raw] int32: voxel index of every input point.
 * Device errors: KMX_ERANGE if some |floor(x / v)| >= 2^20; KMX_ECAPACITY if
 * the voxel count exceeds cap.
 */
kmx_status kmx_voxelize(kmx_ctx* ctx, const float* d_xyz, int64_t n_raw, int32_t stride, float voxel,
                        float* d_out4, int64_t cap, int64_t* d_n_out, int32_t* d_assign);

/* kmx_voxelize with the number of input points in device memory, for a
 * chain without host synchronisation (e.g. after kmx_suppress_ground):
 * d_xyz holds n_cap rows of which the first *d_n_raw (clamped to n_cap) are
 * voxelised; otherwise identical to kmx_voxelize (same output, order and
 * errors).  d_n_raw is required. */
kmx_status kmx_voxelize_count(kmx_ctx* ctx, const float* d_xyz, int64_t n_cap, const int64_t* d_n_raw,
                              int32_t stride, float voxel, float* d_out4, int64_t cap, int64_t* d_n_out,
                              int32_t* d_assign);

/* Fill *out with the default suppression parameters (see kmx_ground_params).
 * KMX_EINVAL if out is NULL. */
kmx_status kmx_ground_params_default(kmx_ground_params* out);

/* Number of bins of the zone model, or -1 if the parameters are invalid. */
int32_t kmx_ground_bins(const kmx_ground_params* params);

/*
 * Geometric suppression (Sec. III-B): removes ground points before the
 * descriptors, so that the many mutually consistent but wrong matches on the
 * ground plane do not dominate pruning, and fewer points reach the later
 * steps.  The stand-in for the paper's Patchwork, per point and per bin of
 * the zone model:
 *   bin       zone by x^2 + y^2 against the zone edges, ring by the radius,
 *             sector by the pseudo-angle (quadrant + |y| / (|x| + |y|)).
 *   seeds     members below (sum of the n_lpr lowest quantised heights) / k
 *             + th_seeds, decided in integers.
 *   plane     least-squares height field z = a x + b y + c over the seeds
 *             (exact integer moments, FP64 Cramer's rule), refitted n_iter
 *             times over the members within th_dist of the plane.
 *   accept    a^2 + b^2 <= max_slope^2 and the ground members' mean height
 *             below max_ground_z; those members are removed.
 * Every decision is exact or a fixed sequence of IEEE FP64 operations, so the
 * result is independent of thread order (and equals the CPU oracle's).
 *   d_xyz     [n][stride] float32 points (stride 3 or 4), sensor frame.
 *   d_out     [n][stride] float32 out, distinct from d_xyz: the kept points
 *             in input order, d_n_out of them.
 *   d_n_out   device int64 out: number of kept points.
 *   d_ground  nullable [n] uint8 out: 1 for removed (ground) points.
 *   d_planes  nullable [kmx_ground_bins()][4] double out per bin: a, b, c
 *             (quantised units) and a status: 0 too few or too many members,
 *             1 no fit, 2 too steep, 3 too high, 4 ground.
 * Host errors: KMX_EINVAL for invalid parameters or arguments.
 */
kmx_status kmx_suppress_ground(kmx_ctx* ctx, const float* d_xyz, int64_t n, int32_t stride,
                               const kmx_ground_params* params, float* d_out, int64_t* d_n_out, uint8_t* d_ground,
                               double* d_planes);

/*
 * Hashed uniform grid over a cloud, the search structure that stands in for
 * the K-d tree of Algorithm 1 (radius search of Eq. A1).
 *   d_xyz4    [n_cap][4] float32 points; KEPT by the grid: it must stay valid
 *             and unchanged until kmx_grid_free.
 *   n_cap     number of rows (exact if d_n is NULL).
 *   d_n       nullable device int64 actual count (e.g. kmx_voxelize's d_n_out).
 *   cell      cell edge > 0.  Searches visit the 27 cells around a point, so
 *             kmx_normals requires cell >= r_fpfh (else KMX_EINVAL).
 *   out       *out == NULL: a new grid is allocated (stream-ordered) and
 *             returned.  *out != NULL: that grid (built on this context with a
 *             capacity >= n_cap) is rebuilt in place over the new points
 *             without allocating, which keeps a whole pair free of
 *             allocations (e.g. for CUDA-graph capture).
 * Device errors: KMX_ERANGE if a cell index does not fit in 21 bits.
 */
kmx_status kmx_build_grid(kmx_ctx* ctx, const float* d_xyz4, int64_t n_cap, const int64_t* d_n, float cell,
                          kmx_grid** out);

/* Release a grid: stream-ordered free on the device and stream its context
 * had when the grid was built.  It may be called after kmx_destroy of that
 * context, as long as the stream still exists. */
void kmx_grid_free(kmx_grid* grid);

/*
 * Algorithm 1, step 1: one radius search with r_fpfh per point (Eq. A1,
 * including the point itself), the r_normal subsample P_normal, PCA normal
 * and linearity p_lin = (l1 - l2) / l1 (Sec. III-C), and the reliability flag
 * B (|I| >= tau_num, |P_normal| >= tau_num, p_lin < tau_lin).
 *   d_normal4  [n_cap][4] float32: unit normal oriented toward the viewpoint
 *              (n . (vp - a_q) >= 0) and p_lin in w, for every point that
 *              reached PCA; zeros otherwise.
 *   d_flags    [n_cap] uint8: bit0 = B[q]; bit2 = PCA evaluated; bit1 = 0.
 *   d_nbr_offs [n_cap + 1] int64 CSR offsets of the neighbour lists.
 *   d_nbr      [nbr_cap] int32: I(q) for every q (in the order the grid
 *              visits them); Algorithm 1's M[q] is this list where B[q].
 *              May be NULL to count only.
 *   d_needed   device int64: total list length (d_nbr_offs[n]).
 * The neighbour sets are exact: a distance within FP32 rounding of a radius
 * is decided again in FP64 as ((dx*dx + dy*dy) + dz*dz) < r*r.
 * Device errors: KMX_ECAPACITY if the lists need more than nbr_cap entries
 * (normals and flags are still written; the lists are not, and every offset
 * is set to 0 so that a following kmx_fasterpfh reads empty lists; d_needed
 * holds the length to allocate).
 */
kmx_status kmx_normals(kmx_ctx* ctx, const kmx_grid* grid, const kmx_params* params, float* d_normal4,
                       uint8_t* d_flags, int64_t* d_nbr_offs, int32_t* d_nbr, int64_t nbr_cap,
                       int64_t* d_needed);

/*
 * Algorithm 1, step 2 and the descriptors of Eqs. A2-A5.
 *   I_valid(q) = { i in M[q] : B[i] }; q enters J iff B[q] and
 *   |I_valid(q)| >= tau_num.  SPFH(q) (Eq. A4) is built for every q with B
 *   over k in I_valid(q) without q, each third scaled by 100 / (number of
 *   contributing pairs); FPFH(q) = SPFH(q) + (1/m) sum_k SPFH(k) / w_k (Eq. A5)
 *   with w_k = |a_k - a_q| over the m neighbours k != q.
 *   d_normal4, d_nbr_offs, d_nbr  as written by kmx_normals (or any input of
 *              the same layout).
 *   nbr_cap    entries of d_nbr (as passed to kmx_normals; KMX_EINVAL if
 *              negative); list entries at or past it are not read.  The context scratch holds one
 *              8-byte entry per list entry (each point's FPFH neighbours
 *              and weights, written by the SPFH pass for the FPFH pass).
 *   d_flags    [n] uint8 in/out: bit0 (B) is read; bit1 is set for q in J.
 *   d_desc     [n_cap][36] float32: row j holds FPFH(J[j]) for j < |J|
 *              (33 values + 3 zeros); other rows are not written.
 *   d_valid    [n_cap] int32: J in ascending point order.
 *   d_n_valid  device int64: |J|.
 *   d_spfh     nullable [n_cap][36] float32: SPFH of every point (zero rows
 *              for points without B); NULL keeps it in scratch.
 */
kmx_status kmx_fasterpfh(kmx_ctx* ctx, const kmx_grid* grid, const kmx_params* params, const float* d_normal4,
                         uint8_t* d_flags, const int64_t* d_nbr_offs, const int32_t* d_nbr, int64_t nbr_cap,
                         float* d_desc, int32_t* d_valid, int64_t* d_n_valid, float* d_spfh);

/*
 * Algorithm 1 (steps 1 and 2) and the descriptors of Eqs. A2-A5 in one call,
 * without neighbour lists: every stage walks the grid's 27-cell stencil
 * again instead of reading stored lists.  Same definitions, sets and
 * summation order as kmx_normals followed by kmx_fasterpfh, so the outputs
 * equal theirs bit for bit:
 *   d_normal4  [n_cap][4] float32 out: as kmx_normals.
 *   d_flags    [n_cap] uint8 out: bit0 = B, bit1 = in J, bit2 = PCA evaluated.
 *   d_desc     [n_cap][36] float32 out: row j holds FPFH(J[j]) for j < |J|.
 *   d_valid    [n_cap] int32 out: J in ascending point order.
 *   d_n_valid  device int64 out: |J|.
 *   d_spfh     nullable [n_cap][36] float32 out: SPFH of every point the grid
 *              holds (zero rows for points without B).
 * Host errors: KMX_EINVAL as kmx_normals.  No capacity error can occur.
 */
kmx_status kmx_features(kmx_ctx* ctx, const kmx_grid* grid, const kmx_params* params, float* d_normal4,
                        uint8_t* d_flags, float* d_desc, int32_t* d_valid, int64_t* d_n_valid, float* d_spfh);

/*
 * Classic FPFH (Rusu et al. 2009), the baseline Faster-PFH is compared with
 * in Sec. III-C (Fig. 2(a)): three radius searches on the grid and no
 * reliability test (tau_num and tau_lin are not read).
 *   (i)   r_normal search; a point has a normal when |P_normal| >= 3 and
 *         l1 > 0 (PCA, FP64 solve, oriented toward params->viewpoint);
 *   (ii)  r_fpfh search; SPFH (Eqs. A2-A4) of every point with a normal over
 *         its neighbours with a normal (itself excluded);
 *   (iii) r_fpfh search; FPFH (Eq. A5) over the same neighbours.
 * J is the set of points with a normal.  Radius tests are exact as in
 * kmx_normals.  No neighbour lists are written.
 *   d_normal4  [n_cap][4] float32 out: normal and p_lin for points with a
 *              normal, zeros otherwise.
 *   d_flags    [n_cap] uint8 out: bit0 = has a normal, bit1 = in J (the
 *              same), bit2 = PCA evaluated.
 *   d_desc     [n_cap][36] float32 out: row j holds FPFH(J[j]) for j < |J|.
 *   d_valid    [n_cap] int32 out: J in ascending point order.
 *   d_n_valid  device int64 out: |J|.
 *   d_spfh     nullable [n_cap][36] float32 out: SPFH of every point the
 *              grid holds (zero rows for points without a normal).
 * Host errors: KMX_EINVAL as kmx_normals (grid cell below r_fpfh, radii,
 * misaligned buffers).  All outputs are device memory owned by the caller.
 */
kmx_status kmx_fpfh_classic(kmx_ctx* ctx, const kmx_grid* grid, const kmx_params* params, float* d_normal4,
                            uint8_t* d_flags, float* d_desc, int32_t* d_valid, int64_t* d_n_valid, float* d_spfh);

/*
 * Mutual nearest-neighbour matching of descriptors (reciprocity test,
 * Sec. III-C) under Euclidean distance; ties go to the lower row.
 *   d_desc_p   [np_cap][36] float32 source descriptors (rows as written by
 *              kmx_fasterpfh); d_valid_p maps row -> source point index.
 *   d_desc_q   [nq_cap][36] float32 target descriptors; d_valid_q likewise.
 *   d_np/d_nq  nullable device row counts.
 *   mode       kmx_match_mode.
 *   d_out      [cap] kmx_corr sorted by source row; (i, j) are point
 *              indices taken through d_valid_p / d_valid_q.
 *   d_n_out    device int64: |A|.
 * Device errors: KMX_ECAPACITY if |A| > cap (the first cap pairs are kept);
 * in KMX_MATCH_FP32_EXACT mode KMX_ERANGE if a descriptor value among the
 * first n_p / n_q rows is NaN or infinite (A is then unspecified).
 */
kmx_status kmx_match(kmx_ctx* ctx, const float* d_desc_p, const int32_t* d_valid_p, int64_t np_cap,
                     const int64_t* d_np, const float* d_desc_q, const int32_t* d_valid_q, int64_t nq_cap,
                     const int64_t* d_nq, int32_t mode, kmx_corr* d_out, int64_t cap, int64_t* d_n_out);

/* Diagnostics of the last kmx_match(..., KMX_MATCH_BF16_RERANK, ...) on this
 * context (not from the paper): six device int64 values in d_out: the rows
 * of the source and of the target cloud whose candidate list overflowed and
 * went through the exact FP32 tiles, the candidates collected for the source
 * rows and for the target rows in total, and the 128 x 128 tile pairs whose
 * distances went through the tensor cores with source rows and with target
 * rows (the tiles that the triangle-inequality test could not rule out).  np_cap, d_np, nq_cap, d_nq
 * are those of that call, and no other call may have used the context's
 * scratch since.  KMX_EINVAL if the context's scratch cannot hold a match of
 * these capacities. */
kmx_status kmx_match_diag(kmx_ctx* ctx, int64_t np_cap, const int64_t* d_np, int64_t nq_cap, const int64_t* d_nq,
                          int64_t* d_out);

/*
 * Correspondence pruning of Sec. III-D, the step after matching: the ratio
 * filter keeps the n_tau correspondences with the lowest d1 / d2 (Lowe's
 * ratio; FP64 division, 1 when d2 = 0; ties to the lower i), the pairwise
 * invariant of Eq. 3 joins selected correspondences k and k' when
 * | |b_k - b_k'| - |a_k - a_k'| | <= 2 beta (norms in FP64 of the FP32 end
 * points, as ((dx dx + dy dy) + dz dz)), and the maximum k-core of that graph
 * holds the candidate inliers passed on to the solver (Sec. III-E).
 *   d_corr     [corr_cap] kmx_corr as written by kmx_match; d_n_corr nullable
 *              device count.  (i, j) index d_src4 / d_tgt4.
 *   d_src4, d_tgt4  voxelised end points [.][4] float32 (a = source, b = target).
 *   n_tau      1 .. 16384 (the paper uses 3000); beta > 0 (the paper: 1.5 v).
 *   d_sel      [n_tau] int32: indices into d_corr, ascending (ratio, i).
 *   d_n_sel    device int64: min(n_corr, n_tau).
 *   d_core     [n_tau] int32: core number of each selected correspondence
 *              (position p of d_sel) in the compatibility graph.
 *   d_kmax     device int32: the largest core number (0 without edges).
 *   d_inlier   [n_tau] int32: positions p with core number kmax, ascending.
 *   d_n_inlier device int64: their count.
 * The core numbers come from a cooperative launch (its blocks wait on one
 * another through a bounded grid barrier): do not capture this call into a
 * CUDA graph.  Device errors: KMX_ETIMEOUT if a barrier wait ran out.
 */
kmx_status kmx_prune(kmx_ctx* ctx, const kmx_corr* d_corr, int64_t corr_cap, const int64_t* d_n_corr,
                     const float* d_src4, const float* d_tgt4, int32_t n_tau, double beta, int32_t* d_sel,
                     int64_t* d_n_sel, int32_t* d_core, int32_t* d_kmax, int32_t* d_inlier, int64_t* d_n_inlier);

/*
 * Robust pose (Sec. III-E): GNC with the truncated-least-squares loss (the
 * paper's solver, Yang et al. 2020) on the correspondences of the maximum
 * k-core, around a weighted rigid alignment (Horn's unit-quaternion closed
 * form).  Point k < *d_n_inlier is a_k = d_src4[c.i], b_k = d_tgt4[c.j] with
 * c = d_corr[d_sel[d_inlier[k]]] (the outputs of kmx_prune).
 *   noise_bound  c of the TLS loss (the paper: beta); max_iters (100),
 *              mu_factor (1.4) and tol (1e-12, on the weighted cost) set the
 *              GNC schedule.
 *   d_R        [9] float64, row-major, and d_t [3] float64: b ~ R a + t.
 *   d_w        [inlier_cap] float32: the final weight of each point.
 *   d_stats    [4] int32: iterations, points with weight > 0.5, points,
 *              status (0, or 1 with fewer than 3 points: R = I, t = 0).
 * inlier_cap <= 4096 (one block holds the points); more points on the device
 * raise KMX_ECAPACITY.  Residuals and moments are FP32 on coordinates centred
 * on their FP64 centroids, so the pose agrees with an FP64 solver to about
 * 1e-5 relative.
 */
kmx_status kmx_gnc(kmx_ctx* ctx, const kmx_corr* d_corr, const int32_t* d_sel, const int32_t* d_inlier,
                   const int64_t* d_n_inlier, int64_t inlier_cap, const float* d_src4, const float* d_tgt4,
                   double noise_bound, int32_t max_iters, double mu_factor, double tol, double* d_R, double* d_t,
                   float* d_w, int32_t* d_stats);

/*
 * Exact FP32 mutual matching without any allocation (the paper has no
 * counterpart: this is a service for callers of this library).  Callers that
 * cannot allocate device memory while they match (a process whose memory
 * pool already owns the device, a real-time loop that must not block on the
 * driver's allocator, a host framework that forbids allocation calls from
 * plug-in code) get the result of kmx_match(..., KMX_MATCH_FP32_EXACT, ...)
 * without a context and without cudaMalloc, cudaFree or any allocating
 * library routine.  It runs the dense exact tile kernel (every descriptor
 * dimension visited; the same distances, ties and emission as kmx_match),
 * not kmx_match's zero-skipping one, and it does not check the descriptors
 * for NaN or infinite values (kmx_match reports those as KMX_ERANGE; here the
 * result is then unspecified).
 *   Arguments are those of kmx_match (same layouts and meaning) plus the
 *   cudaStream_t to run on; work goes to the device current at the call.
 *   Scratch is a fixed device array of about 6 MB inside the library,
 *   reserved on every device that loads the library until the process exits.
 *   np_cap and nq_cap may not exceed KMX_NOALLOC_MAX_ROWS: larger requests
 *   return KMX_EINVAL and launch nothing.
 *   The first call on a device (and the first after the device's CUDA context
 *   changed) looks the array's address up with that device current; make
 *   that first call before any stream capture.
 *   All calls share the one array: calls whose work overlaps on the GPU (on
 *   different streams, or from several threads) race and corrupt each
 *   other's results; serialise them.
 *   Device-side results: *d_n_out = |A| (the first cap pairs are written, so
 *   *d_n_out > cap signals overflow of `cap`), or *d_n_out = -1 when a
 *   bounded wait of the prefix scan gave up (KMX_ETIMEOUT of the other entry
 *   points; d_out is then unspecified).
 * Returns KMX_OK, KMX_EINVAL (bad argument or size beyond the maximum) or
 * KMX_ECUDA (the context or symbol lookup, or a launch, failed).
 */
#define KMX_NOALLOC_MAX_ROWS 32768
kmx_status kmx_match_noalloc(const float* d_desc_p, const int32_t* d_valid_p, int64_t np_cap, const int64_t* d_np,
                             const float* d_desc_q, const int32_t* d_valid_q, int64_t nq_cap, const int64_t* d_nq,
                             kmx_corr* d_out, int64_t cap, int64_t* d_n_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KMX_H */
