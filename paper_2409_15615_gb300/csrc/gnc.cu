// Robust pose from the pruned correspondences (Sec. III-E): graduated
// non-convexity with the truncated-least-squares loss (GNC-TLS, Yang et al.,
// RA-L 2020) around a weighted closed-form rigid alignment (Horn 1987, unit
// quaternions).
//
// One CTA per problem (the maximum k-core holds a few thousand
// correspondences).  The points sit in shared memory, centred on their
// unweighted centroids (taken in FP64), so the FP32 residuals and moments
// carry only the spread of the cloud; the block reductions end in FP64 in one
// warp; the 4 x 4 symmetric eigenproblem of Horn's method is solved by cyclic
// Jacobi in thread 0.  The GNC schedule is the one of the paper's solver:
// weights w = 1 first; mu = c^2 / (2 r_max^2 - c^2); each iteration sets
// w = 1 for r^2 <= mu/(mu+1) c^2, 0 for r^2 >= (mu+1)/mu c^2 and
// c sqrt(mu (mu+1)) / r - mu between, refits, and multiplies mu by the
// factor; it stops when fewer than 3 weights are positive (keeping the
// previous fit) or when the weighted cost repeats within tol.
#include "kmx_internal.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kMaxPoints = 4096;
constexpr int kWarpsG = kThreads / 32;

struct GncOut {
    double* R;       // [9] row-major
    double* t;       // [3]
    float* w;        // [cap] final weights
    int32_t* stats;  // [4]: iterations, weights > 0.5, points, status (0 ok, 1 fewer than 3 points, 2 too many)
};

// Sum of up to 16 per-thread FP32 values over the block (warp sums in FP32,
// the kWarpsG warp sums added in FP64 by warp 0); every thread gets the
// totals in tot[].
template <int N>
__device__ __forceinline__ void block_sum(const float (&v)[N], double* red, double (&tot)[N])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        x[i] = v[i];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x[i] += __shfl_xor_sync(0xffffffffu, x[i], o);
    }
    __syncthreads();  // red is reused
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[i * kWarpsG + warp] = (double)x[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double y = lane < kWarpsG ? red[i * kWarpsG + lane] : 0.0;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane == 0) red[i * kWarpsG] = y;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) tot[i] = red[i * kWarpsG];
}

// Eigenvector of the largest eigenvalue of a symmetric 4 x 4 matrix (cyclic
// Jacobi rotations).
__device__ void jacobi4_max(float (&A)[4][4], float (&q)[4])
{
    float V[4][4] = {{1.f, 0.f, 0.f, 0.f}, {0.f, 1.f, 0.f, 0.f}, {0.f, 0.f, 1.f, 0.f}, {0.f, 0.f, 0.f, 1.f}};
    // every index below is a compile-time constant after unrolling, so the
    // two matrices stay in registers
    for (int sweep = 0; sweep < 12; ++sweep) {
        float off = 0.f, diag = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            diag += A[i][i] * A[i][i];
#pragma unroll
            for (int j = i + 1; j < 4; ++j) off += A[i][j] * A[i][j];
        }
        if (off <= 1e-14f * diag) break;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int r = p + 1; r < 4; ++r) {
                const float apr = A[p][r];
                if (apr == 0.f) continue;
                const float theta = (A[r][r] - A[p][p]) / (2.f * apr);
                const float tt = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
                const float c = 1.f / sqrtf(tt * tt + 1.f), s = tt * c;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float akp = A[k][p], akr = A[k][r];
                    A[k][p] = c * akp - s * akr;
                    A[k][r] = s * akp + c * akr;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float apk = A[p][k], ark = A[r][k];
                    A[p][k] = c * apk - s * ark;
                    A[r][k] = s * apk + c * ark;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float vkp = V[k][p], vkr = V[k][r];
                    V[k][p] = c * vkp - s * vkr;
                    V[k][r] = s * vkp + c * vkr;
                }
            }
        }
    }
    float bestv = A[0][0];
    float qv[4] = {V[0][0], V[1][0], V[2][0], V[3][0]};
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        if (A[i][i] > bestv) {
            bestv = A[i][i];
#pragma unroll
            for (int k = 0; k < 4; ++k) qv[k] = V[k][i];
        }
    }
    float nrm = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) nrm += qv[k] * qv[k];
    nrm = 1.f / sqrtf(nrm);
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = qv[k] * nrm;
}

struct Shared {
    double red[16 * kWarpsG];
    float R[9];      // current rotation (FP32, for the residuals)
    float tc[3];     // translation in the centred frame: b' = R a' + tc
    double Rd[9];    // current rotation, FP64 copy for the output
    double c0[6];    // unweighted centroids of a and b (FP64)
};

// Per-point state in dynamic shared memory (struct of arrays).
struct Pts {
    float* ax;
    float* ay;
    float* az;
    float* bx;
    float* by;
    float* bz;
    float* w;
    float* r2;
};

// Weighted fit in the centred frame: moments of the weighted points, then
// Horn's quaternion (thread 0).  Returns the total weight.
__device__ double fit(const Pts& P, int n, Shared& S)
{
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = 0.f;
    for (int k = threadIdx.x; k < n; k += kThreads) {
        const float wk = P.w[k];
        const float ax = P.ax[k], ay = P.ay[k], az = P.az[k], bx = P.bx[k], by = P.by[k], bz = P.bz[k];
        v[0] += wk;
        v[1] += wk * ax;
        v[2] += wk * ay;
        v[3] += wk * az;
        v[4] += wk * bx;
        v[5] += wk * by;
        v[6] += wk * bz;
        v[7] += wk * ax * bx;
        v[8] += wk * ax * by;
        v[9] += wk * ax * bz;
        v[10] += wk * ay * bx;
        v[11] += wk * ay * by;
        v[12] += wk * ay * bz;
        v[13] += wk * az * bx;
        v[14] += wk * az * by;
        v[15] += wk * az * bz;
    }
    double tot[16];
    block_sum<16>(v, S.red, tot);
    if (threadIdx.x == 0) {
        const double sw = tot[0] > 0.0 ? tot[0] : 1.0;
        const double ca[3] = {tot[1] / sw, tot[2] / sw, tot[3] / sw};
        const double cb[3] = {tot[4] / sw, tot[5] / sw, tot[6] / sw};
        // centred cross-covariance S_ij = sum w (a_i - ca_i)(b_j - cb_j)
        double H[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) H[i][j] = tot[7 + 3 * i + j] - sw * ca[i] * cb[j];
        const float Sxx = (float)H[0][0], Sxy = (float)H[0][1], Sxz = (float)H[0][2];
        const float Syx = (float)H[1][0], Syy = (float)H[1][1], Syz = (float)H[1][2];
        const float Szx = (float)H[2][0], Szy = (float)H[2][1], Szz = (float)H[2][2];
        float N[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                         {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                         {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                         {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
        float q[4];
        jacobi4_max(N, q);
        const double q0 = q[0], qx = q[1], qy = q[2], qz = q[3];
        const double Rm[9] = {q0 * q0 + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - q0 * qz), 2 * (qx * qz + q0 * qy),
                              2 * (qx * qy + q0 * qz), q0 * q0 - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - q0 * qx),
                              2 * (qx * qz - q0 * qy), 2 * (qy * qz + q0 * qx), q0 * q0 - qx * qx - qy * qy + qz * qz};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            S.Rd[i] = Rm[i];
            S.R[i] = (float)Rm[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
            S.tc[i] = (float)(cb[i] - (Rm[3 * i] * ca[0] + Rm[3 * i + 1] * ca[1] + Rm[3 * i + 2] * ca[2]));
    }
    __syncthreads();
    return tot[0];
}

__device__ __forceinline__ float resid2(const Shared& S, float ax, float ay, float az, float bx, float by, float bz)
{
    const float rx = bx - (S.R[0] * ax + S.R[1] * ay + S.R[2] * az) - S.tc[0];
    const float ry = by - (S.R[3] * ax + S.R[4] * ay + S.R[5] * az) - S.tc[1];
    const float rz = bz - (S.R[6] * ax + S.R[7] * ay + S.R[8] * az) - S.tc[2];
    return rx * rx + ry * ry + rz * rz;
}

__global__ void __launch_bounds__(kThreads, 1)
    gnc_tls(const kmx_corr* __restrict__ corr, const int32_t* __restrict__ sel, const int32_t* __restrict__ inlier,
            const int64_t* __restrict__ d_n, int64_t cap, const float4* __restrict__ src4,
            const float4* __restrict__ tgt4, double c2, int max_iters, double mu_factor, double tol, GncOut o,
            unsigned int* err)
{
    __shared__ Shared S;
    const int64_t n64 = d_n ? min(*d_n, cap) : cap;
    const int tid = threadIdx.x;
    if (n64 > (int64_t)kMaxPoints) {  // more points than shared memory holds
        if (tid == 0) {
            kmx_raise(err, KMX_DERR_CAPACITY);
            o.stats[3] = 2;
        }
        return;
    }
    const int n = (int)n64;
    if (n < 3) {
        if (tid == 0) {
            for (int i = 0; i < 9; ++i) o.R[i] = (i % 4 == 0) ? 1.0 : 0.0;
            o.t[0] = o.t[1] = o.t[2] = 0.0;
            o.stats[0] = 0;
            o.stats[1] = 0;
            o.stats[2] = n;
            o.stats[3] = 1;
        }
        for (int k = tid; k < n; k += kThreads) o.w[k] = 0.f;
        return;
    }
    extern __shared__ float dyn[];
    const Pts P{dyn, dyn + kMaxPoints, dyn + 2 * kMaxPoints, dyn + 3 * kMaxPoints, dyn + 4 * kMaxPoints,
                dyn + 5 * kMaxPoints, dyn + 6 * kMaxPoints, dyn + 7 * kMaxPoints};
    // unweighted centroids in FP64, the reference frame of the FP32 work:
    // offsets from the first point are summed, then it is added back
    const kmx_corr c0 = corr[sel[inlier[0]]];
    const float4 a0 = src4[c0.i], b0 = tgt4[c0.j];
    {
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = tid; k < n; k += kThreads) {
            const kmx_corr c = corr[sel[inlier[k]]];
            const float4 a = src4[c.i], b = tgt4[c.j];
            P.ax[k] = a.x;  // raw for now, centred below
            P.ay[k] = a.y;
            P.az[k] = a.z;
            P.bx[k] = b.x;
            P.by[k] = b.y;
            P.bz[k] = b.z;
            v[0] += a.x - a0.x;
            v[1] += a.y - a0.y;
            v[2] += a.z - a0.z;
            v[3] += b.x - b0.x;
            v[4] += b.y - b0.y;
            v[5] += b.z - b0.z;
        }
        double tot[6];
        block_sum<6>(v, S.red, tot);
        if (tid == 0) {
            S.c0[0] = (double)a0.x + tot[0] / n;
            S.c0[1] = (double)a0.y + tot[1] / n;
            S.c0[2] = (double)a0.z + tot[2] / n;
            S.c0[3] = (double)b0.x + tot[3] / n;
            S.c0[4] = (double)b0.y + tot[4] / n;
            S.c0[5] = (double)b0.z + tot[5] / n;
        }
        __syncthreads();
    }
    const double ca0[3] = {S.c0[0], S.c0[1], S.c0[2]};
    const double cb0[3] = {S.c0[3], S.c0[4], S.c0[5]};
    for (int k = tid; k < n; k += kThreads) {
        P.ax[k] = (float)((double)P.ax[k] - ca0[0]);
        P.ay[k] = (float)((double)P.ay[k] - ca0[1]);
        P.az[k] = (float)((double)P.az[k] - ca0[2]);
        P.bx[k] = (float)((double)P.bx[k] - cb0[0]);
        P.by[k] = (float)((double)P.by[k] - cb0[1]);
        P.bz[k] = (float)((double)P.bz[k] - cb0[2]);
        P.w[k] = 1.f;
    }
    __syncthreads();
    fit(P, n, S);
    float rmax = 0.f;
    for (int k = tid; k < n; k += kThreads) {
        const float r = resid2(S, P.ax[k], P.ay[k], P.az[k], P.bx[k], P.by[k], P.bz[k]);
        P.r2[k] = r;
        rmax = fmaxf(rmax, r);
    }
    {
#pragma unroll
        for (int sh = 16; sh >= 1; sh >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, sh));
        __syncthreads();
        if ((tid & 31) == 0) S.red[tid >> 5] = rmax;
        __syncthreads();
        double m = 0.0;
        for (int i = 0; i < kWarpsG; ++i) m = fmax(m, S.red[i]);
        rmax = (float)m;
        __syncthreads();
    }
    int iters = 0;
    if ((double)rmax > c2) {
        double mu = c2 / fmax(2.0 * (double)rmax - c2, 1e-30);
        double prev_cost = INFINITY;
        for (int it = 0; it < max_iters; ++it) {
            const float lo = (float)(mu / (mu + 1.0) * c2), hi = (float)((mu + 1.0) / mu * c2);
            const float cw = (float)(sqrt(c2) * sqrt(mu * (mu + 1.0))), muf = (float)mu;
            float npos[1] = {0.f};
            for (int k = tid; k < n; k += kThreads) {
                const float r = P.r2[k];
                const float wk = r <= lo ? 1.f : (r >= hi ? 0.f : cw / sqrtf(fmaxf(r, 1e-30f)) - muf);
                P.w[k] = wk;
                npos[0] += wk > 0.f ? 1.f : 0.f;
            }
            double ctot[1];
            block_sum<1>(npos, S.red, ctot);
            if (ctot[0] < 3.0) break;  // the current fit stays; w are the weights that stopped it
            fit(P, n, S);
            ++iters;
            float cv[1] = {0.f};
            for (int k = tid; k < n; k += kThreads) {
                const float r = resid2(S, P.ax[k], P.ay[k], P.az[k], P.bx[k], P.by[k], P.bz[k]);
                P.r2[k] = r;
                cv[0] += P.w[k] * r;
            }
            double cost[1];
            block_sum<1>(cv, S.red, cost);
            if (fabs(cost[0] - prev_cost) < tol) break;
            prev_cost = cost[0];
            mu *= mu_factor;
        }
    }
    // outputs: R, t in the original frame (b = R a + t with t = cb0 + tc - R ca0)
    float good[1] = {0.f};
    for (int k = tid; k < n; k += kThreads) {
        o.w[k] = P.w[k];
        good[0] += P.w[k] > 0.5f ? 1.f : 0.f;
    }
    double gt[1];
    block_sum<1>(good, S.red, gt);
    if (tid == 0) {
        for (int i = 0; i < 9; ++i) o.R[i] = S.Rd[i];
        for (int i = 0; i < 3; ++i)
            o.t[i] = cb0[i] + (double)S.tc[i] -
                     (S.Rd[3 * i] * ca0[0] + S.Rd[3 * i + 1] * ca0[1] + S.Rd[3 * i + 2] * ca0[2]);
        o.stats[0] = iters;
        o.stats[1] = (int32_t)gt[0];
        o.stats[2] = n;
        o.stats[3] = 0;
    }
}

size_t smem_bytes() { return sizeof(float) * 8 * (size_t)kMaxPoints; }

}  // namespace

int64_t kmx_gnc_max_points() { return kMaxPoints; }

cudaError_t kmx_gnc_launch(kmx_ctx* ctx, const kmx_corr* corr, const int32_t* sel, const int32_t* inlier,
                           const int64_t* d_n, int64_t cap, const float4* src4, const float4* tgt4, double noise_bound,
                           int max_iters, double mu_factor, double tol, double* R, double* t, float* w,
                           int32_t* stats)
{
    cudaError_t e = kmx_once_per_device(kmx_attr_gnc, [] {
        return cudaFuncSetAttribute(gnc_tls, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
    });
    if (e) return e;
    KMX_COUNT_LAUNCH();
    gnc_tls<<<1, kThreads, smem_bytes(), ctx->stream>>>(corr, sel, inlier, d_n, cap, src4, tgt4, noise_bound * noise_bound,
                                             max_iters, mu_factor, tol, GncOut{R, t, w, stats}, ctx->d_err);
    return cudaGetLastError();
}
