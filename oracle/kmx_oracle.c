/*
 * kmx_oracle.c - plain, slow FP64 CPU oracle of the KISS-Matcher front end
 * (arXiv 2409.15615): voxelisation, radius search, Faster-PFH (Algorithm 1,
 * Eqs. A1-A5) and mutual nearest-neighbour matching (Sec. III-C).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Conventions
 *  - Inputs are FP32 (as the GPU receives them); every derived quantity is
 *    computed in FP64.  Compile with -ffp-contract=off so that each written
 *    expression is evaluated operation by operation, exactly as written.
 *  - Squared distance between points s and q is
 *        d2 = (dx*dx + dy*dy) + dz*dz,  dx = (double)x_s - (double)x_q, ...
 *    and "inside radius r" means d2 < (double)r * (double)r  (Eq. A1 with the
 *    strict inequality of the paper, compared in squared form).
 *  - OpenMP parallelises independent per-point loops only; every result is
 *    deterministic and independent of the thread count.
 *
 * Readings of passages the paper leaves open (each one is a choice, not a
 * statement of the paper):
 *  R1 voxel filter: half-open cells floor(x / v) in FP64; the representative
 *     of a voxel is the centroid of its members, summed in FP64 in input
 *     order and rounded to FP32; voxels are emitted in order of their first
 *     member in the input.
 *  R2 the query point belongs to its own neighbourhood I(q) (distance 0 < r)
 *     and counts toward tau_num, but it is left out of the SPFH and FPFH sums
 *     (its direction vector is 0/0 and its weight 1/0).
 *  R3 "I_valid < tau_num" in Algorithm 1 is read as |I_valid| < tau_num.
 *  R4 step 2 of Algorithm 1 runs once on the step-1 flags (no cascade).
 *  R5 normals point toward the viewpoint: n . (vp - a_q) >= 0; if that dot
 *     product is exactly 0 the first non-zero component is made positive.
 *  R6 the source point of a pair is the one whose normal makes the smaller
 *     angle with the line through both points: |n_q . d| >= |n_k . d| keeps q
 *     as source (ties keep q).
 *  R7 v = d x u and w = u x v are unit vectors; a pair with |d x u| < 1e-6
 *     (d and u within 1e-6 rad of parallel, where the Darboux frame is not
 *     defined to FP32 accuracy) is skipped and does not count in the SPFH
 *     normaliser.
 *  R8 atan2 is the four-quadrant arctangent.
 *  R9 H = 11 bins per feature; feature ranges are [-pi, pi], [-1, 1],
 *     [-1, 1]; bins are 0-based, bin = floor(H (f - lo) / (hi - lo)) clamped
 *     to [0, H-1] (the clamp plays the role of the epsilon in Eq. A3).
 * R10 FPFH keeps the unnormalised scale of Eq. A5.
 * R11 descriptors are compared by Euclidean distance; ties in the nearest
 *     neighbour go to the lower index.
 * R12 covariance uses the 1/n normaliser.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ERANGE 4
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* helpers                                                                   */
/* ------------------------------------------------------------------------ */

static double sqdist(const float* a, const float* b)
{
    double dx = (double)a[0] - (double)b[0];
    double dy = (double)a[1] - (double)b[1];
    double dz = (double)a[2] - (double)b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

typedef struct {
    int64_t key;
    int64_t idx;
} keyidx;

static int cmp_keyidx(const void* pa, const void* pb)
{
    const keyidx* a = (const keyidx*)pa;
    const keyidx* b = (const keyidx*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

static int cmp_i32(const void* pa, const void* pb)
{
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------ */
/* voxelisation (input to the method, Sec. III-A; reading R1)                */
/* ------------------------------------------------------------------------ */

/* Packed key of one voxel index triple; returns 0 if any |k| >= 2^20. */
static int voxel_key(const float* p, double v, int64_t* key)
{
    int64_t k[3];
    for (int a = 0; a < 3; ++a) {
        double kd = floor((double)p[a] / v);
        if (!(fabs(kd) < 1048576.0)) return 0;
        k[a] = (int64_t)kd + 1048576;
    }
    *key = (k[0] << 42) | (k[1] << 21) | k[2];
    return 1;
}

/*
 * Voxelise n points (row stride `stride` floats, 3 or 4).  Writes the FP32
 * centroids as [n_out][4] (w = 0) into out4 (capacity n rows), the voxel index
 * of every input point into assign[n] (nullable) and the voxel count into
 * *n_out.  Returns ORC_ERANGE if a voxel index does not fit in 21 bits.
 */
int orc_voxelize(const float* xyz, int64_t n, int stride, float v, float* out4,
                 int32_t* assign, int64_t* n_out)
{
    if (n < 0 || (stride != 3 && stride != 4) || !(v > 0.0f)) return ORC_EINVAL;
    *n_out = 0;
    if (n == 0) return ORC_OK;
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * (size_t)n);
    if (!ki) return ORC_ENOMEM;
    for (int64_t r = 0; r < n; ++r) {
        if (!voxel_key(xyz + r * stride, (double)v, &ki[r].key)) {
            free(ki);
            return ORC_ERANGE;
        }
        ki[r].idx = r;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    /* groups of equal key; within a group members ascend in input order */
    int64_t ng = 0;
    int64_t* gstart = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t s = 0; s < n; ++s)
        if (s == 0 || ki[s].key != ki[s - 1].key) gstart[ng++] = s;
    gstart[ng] = n;
    /* order groups by their first (lowest-index) member */
    keyidx* order = (keyidx*)malloc(sizeof(keyidx) * (size_t)ng);
    for (int64_t g = 0; g < ng; ++g) {
        order[g].key = ki[gstart[g]].idx;
        order[g].idx = g;
    }
    qsort(order, (size_t)ng, sizeof(keyidx), cmp_keyidx);
    for (int64_t o = 0; o < ng; ++o) {
        int64_t g = order[o].idx;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        int64_t cnt = gstart[g + 1] - gstart[g];
        for (int64_t s = gstart[g]; s < gstart[g + 1]; ++s) {
            const float* p = xyz + ki[s].idx * stride;
            sx = sx + (double)p[0];
            sy = sy + (double)p[1];
            sz = sz + (double)p[2];
            if (assign) assign[ki[s].idx] = (int32_t)o;
        }
        out4[o * 4 + 0] = (float)(sx / (double)cnt);
        out4[o * 4 + 1] = (float)(sy / (double)cnt);
        out4[o * 4 + 2] = (float)(sz / (double)cnt);
        out4[o * 4 + 3] = 0.0f;
    }
    *n_out = ng;
    free(order);
    free(gstart);
    free(ki);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* radius search S_rFPFH (Eq. A1)                                            */
/* ------------------------------------------------------------------------ */

/*
 * Brute force: I(q) = { s : |a_s - a_q| < r }, every s tested.  Lists are in
 * ascending s and include q.  offs has n+1 entries; nbr may be NULL to count.
 */
int orc_radius_bruteforce(const float* p4, int64_t n, float r, int64_t* offs, int32_t* nbr)
{
    double r2 = (double)r * (double)r;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        int64_t c = 0;
        for (int64_t s = 0; s < n; ++s)
            if (sqdist(p4 + 4 * s, p4 + 4 * q) < r2) ++c;
        cnt[q] = c;
    }
    offs[0] = 0;
    for (int64_t q = 0; q < n; ++q) offs[q + 1] = offs[q] + cnt[q];
    free(cnt);
    if (!nbr) return ORC_OK;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        int64_t o = offs[q];
        for (int64_t s = 0; s < n; ++s)
            if (sqdist(p4 + 4 * s, p4 + 4 * q) < r2) nbr[o++] = (int32_t)s;
    }
    return ORC_OK;
}

/*
 * Same sets as orc_radius_bruteforce, found through a uniform grid of cell
 * size slightly above r (points sorted by cell, 27 neighbouring cells looked
 * up by binary search).  Each list is sorted ascending before it is written,
 * so the output is identical to the brute-force output.
 */
int orc_radius_grid(const float* p4, int64_t n, float r, int64_t* offs, int32_t* nbr)
{
    double r2 = (double)r * (double)r;
    double cell = (double)r * (1.0 + 1e-6);
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * (size_t)(n > 0 ? n : 1));
    int64_t* cc = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t s = 0; s < n; ++s) {
        for (int a = 0; a < 3; ++a) {
            double kd = floor((double)p4[4 * s + a] / cell);
            if (!(fabs(kd) < 1048000.0)) {
                free(ki);
                free(cc);
                return ORC_ERANGE;
            }
            cc[3 * s + a] = (int64_t)kd + 1048576;
        }
        ki[s].key = (cc[3 * s] << 42) | (cc[3 * s + 1] << 21) | cc[3 * s + 2];
        ki[s].idx = s;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            offs[0] = 0;
            for (int64_t q = 0; q < n; ++q) offs[q + 1] = offs[q] + cnt[q];
            if (!nbr) break;
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t q = 0; q < n; ++q) {
            int64_t c = 0;
            int64_t o = pass ? offs[q] : 0;
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        int64_t key = ((cc[3 * q] + dx) << 42) | ((cc[3 * q + 1] + dy) << 21) |
                                      (cc[3 * q + 2] + dz);
                        /* lower bound of key in the sorted array */
                        int64_t lo = 0, hi = n;
                        while (lo < hi) {
                            int64_t mid = (lo + hi) / 2;
                            if (ki[mid].key < key) lo = mid + 1;
                            else hi = mid;
                        }
                        for (int64_t t = lo; t < n && ki[t].key == key; ++t) {
                            int64_t s = ki[t].idx;
                            if (sqdist(p4 + 4 * s, p4 + 4 * q) < r2) {
                                if (pass) nbr[o] = (int32_t)s;
                                ++o;
                                ++c;
                            }
                        }
                    }
            if (pass)
                qsort(nbr + offs[q], (size_t)c, sizeof(int32_t), cmp_i32);
            else
                cnt[q] = c;
        }
    }
    free(cnt);
    free(cc);
    free(ki);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* symmetric 3x3 eigen-decomposition: cyclic Jacobi (Golub & Van Loan,       */
/* Matrix Computations, Sec. 8.5, "cyclic Jacobi")                           */
/* ------------------------------------------------------------------------ */

/*
 * A (row-major 3x3, symmetric) -> eigenvalues w[3] in descending order and
 * the matching unit eigenvectors as the columns of V (row-major).  Sweeps
 * until the off-diagonal mass is below 1e-30 of the total (or 100 sweeps).
 */
void orc_eig3_jacobi(const double* Ain, double* w, double* Vout)
{
    double A[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = Ain[3 * i + j];
            V[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double tot = off * 2.0 + A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-30 * tot) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation that zeroes A[p][q] */
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                for (int k = 0; k < 3; ++k) { /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) { /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) { /* V <- V J */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    /* sort eigenpairs by descending eigenvalue */
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (A[ord[j]][ord[j]] > A[ord[i]][ord[i]]) {
                int t = ord[i];
                ord[i] = ord[j];
                ord[j] = t;
            }
    for (int i = 0; i < 3; ++i) {
        w[i] = A[ord[i]][ord[i]];
        for (int k = 0; k < 3; ++k) Vout[3 * k + i] = V[k][ord[i]];
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, step 1: reliable normals                                     */
/* ------------------------------------------------------------------------ */

/*
 * For every q with its r_FPFH neighbourhood I(q) given as CSR (offs, nbr):
 *   |I| < tau_num                  -> skipped             (Alg. 1, step 1)
 *   P_normal = { s in I : |a_s - a_q| < r_normal }       (subsampling)
 *   |P_normal| < tau_num           -> skipped
 *   PCA of P_normal: n = eigenvector of the smallest eigenvalue,
 *   p_lin = (l1 - l2) / l1                               (Sec. III-C)
 *   p_lin < tau_lin                -> B[q] = 1
 * normal4[q] = (nx, ny, nz, p_lin) oriented by reading R5 for every q that
 * reached PCA (else zeros); evals[q] = (l1, l2, l3) (nullable); flags[q] bit0
 * = B[q], bit2 = "PCA evaluated".  n_normal[q] = |P_normal| (nullable).
 */
int orc_normals(const float* p4, int64_t n, const int64_t* offs, const int32_t* nbr, float r_normal,
                int tau_num, double tau_lin, const double* vp, double* normal4, double* evals,
                uint8_t* flags, int32_t* n_normal)
{
    double rn2 = (double)r_normal * (double)r_normal;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        flags[q] = 0;
        for (int a = 0; a < 4; ++a) normal4[4 * q + a] = 0.0;
        if (evals)
            for (int a = 0; a < 3; ++a) evals[3 * q + a] = 0.0;
        int64_t m = offs[q + 1] - offs[q];
        if (n_normal) n_normal[q] = 0;
        if (m < tau_num) continue;
        /* P_normal: subsample of I(q) with the normal radius */
        int64_t cnt = 0;
        double mu[3] = {0.0, 0.0, 0.0};
        for (int64_t t = offs[q]; t < offs[q + 1]; ++t) {
            int64_t s = nbr[t];
            if (sqdist(p4 + 4 * s, p4 + 4 * q) < rn2) {
                for (int a = 0; a < 3; ++a) mu[a] = mu[a] + (double)p4[4 * s + a];
                ++cnt;
            }
        }
        if (n_normal) n_normal[q] = (int32_t)cnt;
        if (cnt < tau_num) continue;
        for (int a = 0; a < 3; ++a) mu[a] = mu[a] / (double)cnt;
        double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t t = offs[q]; t < offs[q + 1]; ++t) {
            int64_t s = nbr[t];
            if (sqdist(p4 + 4 * s, p4 + 4 * q) < rn2) {
                double d[3];
                for (int a = 0; a < 3; ++a) d[a] = (double)p4[4 * s + a] - mu[a];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) C[3 * a + b] = C[3 * a + b] + d[a] * d[b];
            }
        }
        for (int a = 0; a < 9; ++a) C[a] = C[a] / (double)cnt;
        double w[3], V[9];
        orc_eig3_jacobi(C, w, V);
        flags[q] |= 4;
        if (evals)
            for (int a = 0; a < 3; ++a) evals[3 * q + a] = w[a];
        if (!(w[0] > 0.0)) continue; /* all members coincide: no normal */
        double nv[3] = {V[2], V[5], V[8]}; /* column of the smallest eigenvalue */
        double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        for (int a = 0; a < 3; ++a) nv[a] = nv[a] / nn;
        double view = 0.0;
        for (int a = 0; a < 3; ++a) view = view + nv[a] * (vp[a] - (double)p4[4 * q + a]);
        int flip = 0;
        if (view < 0.0) flip = 1;
        else if (view == 0.0) {
            for (int a = 0; a < 3; ++a)
                if (nv[a] != 0.0) {
                    flip = nv[a] < 0.0;
                    break;
                }
        }
        if (flip)
            for (int a = 0; a < 3; ++a) nv[a] = -nv[a];
        double plin = (w[0] - w[1]) / w[0];
        for (int a = 0; a < 3; ++a) normal4[4 * q + a] = nv[a];
        normal4[4 * q + 3] = plin;
        if (plin < tau_lin) flags[q] |= 1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, step 2: valid neighbours and the final query set J           */
/* ------------------------------------------------------------------------ */

/*
 * For q with B[q] (flags bit0): I_valid(q) = { i in M[q] : B[i] } keeping the
 * order of M[q]; M[q] is the r_FPFH list of q.  q enters J iff
 * |I_valid(q)| >= tau_num (readings R3, R4).  Writes the I_valid CSR (empty
 * for q without B), sets flags bit1 for q in J, writes J ascending and |J|.
 */
int orc_valid_filter(int64_t n, const int64_t* offs, const int32_t* nbr, uint8_t* flags, int tau_num,
                     int64_t* voffs, int32_t* vnbr, int32_t* J, int64_t* nJ)
{
    voffs[0] = 0;
    int64_t nj = 0;
    for (int64_t q = 0; q < n; ++q) {
        int64_t o = voffs[q];
        if (flags[q] & 1) {
            for (int64_t t = offs[q]; t < offs[q + 1]; ++t)
                if (flags[nbr[t]] & 1) vnbr[o++] = nbr[t];
        }
        voffs[q + 1] = o;
    }
    for (int64_t q = 0; q < n; ++q) {
        flags[q] &= (uint8_t)~2u;
        if ((flags[q] & 1) && voffs[q + 1] - voffs[q] >= tau_num) {
            flags[q] |= 2;
            J[nj++] = (int32_t)q;
        }
    }
    *nJ = nj;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Darboux-frame angular features (Eq. A2) and bins (Eq. A3)                 */
/* ------------------------------------------------------------------------ */

static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double* a, const double* b)
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/*
 * Angular features of the pair (q, k) with normals nq, nk (Eq. A2 with
 * readings R6-R8).  Returns 1 and writes f[3] = (f1, f2, f3), or returns 0
 * if the pair is degenerate (coincident points or |d x u| < 1e-6).
 */
int orc_pair_features(const float* pq, const double* nq, const float* pk, const double* nk, double* f)
{
    double dv[3];
    for (int a = 0; a < 3; ++a) dv[a] = (double)pk[a] - (double)pq[a];
    double dist = sqrt(dot3(dv, dv));
    if (!(dist > 0.0)) return 0;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = dv[a] / dist;
    const double *u, *nb;
    if (fabs(dot3(nq, d)) >= fabs(dot3(nk, d))) {
        u = nq;
        nb = nk;
    } else {
        u = nk;
        nb = nq;
        for (int a = 0; a < 3; ++a) d[a] = -d[a];
    }
    double x[3];
    cross3(d, u, x);
    double s = sqrt(dot3(x, x));
    if (s < 1e-6) return 0;
    double v[3], w[3];
    for (int a = 0; a < 3; ++a) v[a] = x[a] / s;
    cross3(u, v, w);
    f[0] = atan2(dot3(w, nb), dot3(u, nb));
    f[1] = dot3(v, nb);
    f[2] = dot3(u, d);
    return 1;
}

/* Bin of feature value f on [lo, hi] with H bins (Eq. A3, reading R9). */
int orc_bin(double f, double lo, double hi, int H)
{
    double t = floor((double)H * (f - lo) / (hi - lo));
    if (t < 0.0) t = 0.0;
    if (t > (double)(H - 1)) t = (double)(H - 1);
    return (int)t;
}

/* ------------------------------------------------------------------------ */
/* SPFH (Eq. A4) and FPFH (Eq. A5)                                           */
/* ------------------------------------------------------------------------ */

/*
 * How close the pair (q, k) is to a decision that FP32 rounding could flip:
 * the smallest of |(|n_q.d| - |n_k.d|)| (source choice), | |d x u| - 1e-6 |
 * (degenerate-pair test), the distance of f1 to an interior bin edge or to
 * +-pi (the atan2 branch cut), and the distance of f2, f3 to an interior bin
 * edge.  Used by the tests only, to list the points whose exact histogram is
 * ill-posed at FP32 precision.
 */
static double pair_margin(const float* pq, const double* nq, const float* pk, const double* nk, int H)
{
    const double PI = 3.14159265358979323846;
    double dv[3];
    for (int a = 0; a < 3; ++a) dv[a] = (double)pk[a] - (double)pq[a];
    double dist = sqrt(dot3(dv, dv));
    if (!(dist > 0.0)) return INFINITY;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = dv[a] / dist;
    double m = fabs(fabs(dot3(nq, d)) - fabs(dot3(nk, d)));
    const double* u = fabs(dot3(nq, d)) >= fabs(dot3(nk, d)) ? nq : nk;
    if (u == nk)
        for (int a = 0; a < 3; ++a) d[a] = -d[a];
    double x[3];
    cross3(d, u, x);
    double s = sqrt(dot3(x, x));
    m = fmin(m, fabs(s - 1e-6));
    double f[3];
    if (!orc_pair_features(pq, nq, pk, nk, f)) return m;
    const double lo[3] = {-PI, -1.0, -1.0}, hi[3] = {PI, 1.0, 1.0};
    for (int l = 0; l < 3; ++l) {
        double w = (hi[l] - lo[l]) / (double)H;
        double t = (f[l] - lo[l]) / w;
        double e = fabs(t - floor(t + 0.5)) * w;
        if (l > 0 && (f[l] - lo[l] < 0.5 * w || hi[l] - f[l] < 0.5 * w)) {
            /* outer ends of [-1, 1] are not edges (values cannot wrap) */
            double tt = floor(t + 0.5);
            if (tt <= 0.0 || tt >= (double)H) e = INFINITY;
        }
        m = fmin(m, e);
    }
    return m;
}

/*
 * SPFH of every q with B[q] over k in I_valid(q), k != q (reading R2):
 * sub-histogram l counts the bins of f_l and is scaled by 100 / c, c the
 * number of contributing pairs (reading R7).  spfh is [n][3H] (rows of q
 * without B are zero); npairs[q] = c (nullable); margin[q] (nullable) is the
 * smallest pair_margin over the pairs of q (+inf without pairs); n_marg[q]
 * (nullable) counts the pairs of q whose pair_margin is below `band`.
 */
int orc_spfh(const float* p4, const double* normal4, int64_t n, const uint8_t* flags, const int64_t* voffs,
             const int32_t* vnbr, int H, double* spfh, int32_t* npairs, double* margin, double band,
             int32_t* n_marg)
{
    const double PI = 3.14159265358979323846;
    const double lo[3] = {-PI, -1.0, -1.0}, hi[3] = {PI, 1.0, 1.0};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        double* row = spfh + (size_t)q * 3 * H;
        for (int h = 0; h < 3 * H; ++h) row[h] = 0.0;
        if (npairs) npairs[q] = 0;
        if (margin) margin[q] = INFINITY;
        if (n_marg) n_marg[q] = 0;
        if (!(flags[q] & 1)) continue;
        int64_t c = 0;
        for (int64_t t = voffs[q]; t < voffs[q + 1]; ++t) {
            int64_t k = vnbr[t];
            if (k == q) continue;
            if (margin || n_marg) {
                double pm = pair_margin(p4 + 4 * q, normal4 + 4 * q, p4 + 4 * k, normal4 + 4 * k, H);
                if (margin) margin[q] = fmin(margin[q], pm);
                if (n_marg && pm < band) n_marg[q] += 1;
            }
            double f[3];
            if (!orc_pair_features(p4 + 4 * q, normal4 + 4 * q, p4 + 4 * k, normal4 + 4 * k, f)) continue;
            for (int l = 0; l < 3; ++l) row[l * H + orc_bin(f[l], lo[l], hi[l], H)] += 1.0;
            ++c;
        }
        if (c > 0)
            for (int h = 0; h < 3 * H; ++h) row[h] = row[h] * (100.0 / (double)c);
        if (npairs) npairs[q] = (int32_t)c;
    }
    return ORC_OK;
}

/*
 * FPFH of every q in J (row j of fpfh for q = J[j]):
 *   FPFH(q) = SPFH(q) + (1/m) sum_k SPFH(k) / w_k,
 * k over I_valid(q) without q, w_k = |a_k - a_q|, m the number of such k.
 */
int orc_fpfh(const float* p4, int64_t nJ, const int32_t* J, const int64_t* voffs, const int32_t* vnbr,
             const double* spfh, int D, double* fpfh)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < nJ; ++j) {
        int64_t q = J[j];
        double* out = fpfh + (size_t)j * D;
        double acc[256];
        for (int h = 0; h < D; ++h) acc[h] = 0.0;
        int64_t m = 0;
        for (int64_t t = voffs[q]; t < voffs[q + 1]; ++t) {
            int64_t k = vnbr[t];
            if (k == q) continue;
            double w = sqrt(sqdist(p4 + 4 * k, p4 + 4 * q));
            if (!(w > 0.0)) continue;
            for (int h = 0; h < D; ++h) acc[h] = acc[h] + spfh[(size_t)k * D + h] / w;
            ++m;
        }
        for (int h = 0; h < D; ++h)
            out[h] = spfh[(size_t)q * D + h] + (m > 0 ? acc[h] / (double)m : 0.0);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* nearest descriptors for mutual matching (Sec. III-C, reciprocity test)    */
/* ------------------------------------------------------------------------ */

/*
 * For every row i of X [nx][D]: the nearest row of Y [ny][D] by Euclidean
 * distance (ties to the lower index), its distance d1 and the second-smallest
 * distance d2 over all rows (d2 = +inf when ny < 2).  Outputs may be NULL.
 */
int orc_nearest(const double* X, int64_t nx, const double* Y, int64_t ny, int D, int32_t* nn, double* d1,
                double* d2)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nx; ++i) {
        double b1 = INFINITY, b2 = INFINITY;
        int64_t j1 = -1;
        const double* x = X + (size_t)i * D;
        for (int64_t j = 0; j < ny; ++j) {
            const double* y = Y + (size_t)j * D;
            double s = 0.0;
            for (int h = 0; h < D; ++h) {
                double e = x[h] - y[h];
                s = s + e * e;
            }
            if (s < b1) {
                b2 = b1;
                b1 = s;
                j1 = j;
            } else if (s < b2) {
                b2 = s;
            }
        }
        if (nn) nn[i] = (int32_t)j1;
        if (d1) d1[i] = sqrt(b1);
        if (d2) d2[i] = sqrt(b2);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* k-core of an undirected graph (Sec. III-D; Batagelj & Zaversnik 2003)     */
/* ------------------------------------------------------------------------ */

/*
 * Core number of every vertex of the graph given as symmetric CSR (offs,
 * adj) by repeated removal of a vertex of minimum remaining degree.
 * O(V^2 + E) with a linear scan for the minimum: plain, not fast.
 */
int orc_core_numbers(int64_t nv, const int64_t* offs, const int32_t* adj, int32_t* core)
{
    int64_t* deg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    uint8_t* gone = (uint8_t*)calloc((size_t)(nv > 0 ? nv : 1), 1);
    for (int64_t v = 0; v < nv; ++v) deg[v] = offs[v + 1] - offs[v];
    int64_t k = 0;
    for (int64_t step = 0; step < nv; ++step) {
        int64_t best = -1;
        for (int64_t v = 0; v < nv; ++v)
            if (!gone[v] && (best < 0 || deg[v] < deg[best])) best = v;
        if (deg[best] > k) k = deg[best];
        core[best] = (int32_t)k;
        gone[best] = 1;
        for (int64_t t = offs[best]; t < offs[best + 1]; ++t)
            if (!gone[adj[t]]) deg[adj[t]] -= 1;
    }
    free(gone);
    free(deg);
    return ORC_OK;
}
