// Device helpers of the descriptors (App. A): the Darboux-frame pair
// features of Eq. A2, the binning of Eq. A3 and the compensated sum used for
// Eq. A5.  Shared by Faster-PFH and the classic FPFH baseline, which differ
// only in which pairs they visit.
#pragma once

#include "kmx_internal.cuh"

namespace kmxp {

constexpr int kH = 11;
constexpr int kD = 3 * kH;  // 33
constexpr int kStride = KMX_DESC_STRIDE;
static_assert(kD == KMX_DESC_DIM, "three sub-histograms of H bins");

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz)
{
    return fmaf(az, bz, fmaf(ay, by, ax * bx));
}

// Angular features of the pair (q, k) (Eq. A2): the point whose normal is
// closer to parallel with the connecting line is the source; v and w are unit
// vectors.  Returns false for coincident points or |d x u| < 1e-6.
__device__ __forceinline__ bool pair_features(float4 pq, float4 nq, float4 pk, float4 nk, float* f)
{
    float dx = pk.x - pq.x, dy = pk.y - pq.y, dz = pk.z - pq.z;
    const float dd = dot3(dx, dy, dz, dx, dy, dz);
    if (!(dd > 0.f)) return false;
    const float inv = 1.0f / sqrtf(dd);
    dx *= inv;
    dy *= inv;
    dz *= inv;
    const float cq = fabsf(dot3(nq.x, nq.y, nq.z, dx, dy, dz));
    const float ck = fabsf(dot3(nk.x, nk.y, nk.z, dx, dy, dz));
    float4 u = nq, nb = nk;
    if (!(cq >= ck)) {
        u = nk;
        nb = nq;
        dx = -dx;
        dy = -dy;
        dz = -dz;
    }
    // v = d x u / |d x u|
    float vx = dy * u.z - dz * u.y;
    float vy = dz * u.x - dx * u.z;
    float vz = dx * u.y - dy * u.x;
    const float s = sqrtf(dot3(vx, vy, vz, vx, vy, vz));
    if (s < 1e-6f) return false;
    const float is = 1.0f / s;
    vx *= is;
    vy *= is;
    vz *= is;
    // w = u x v
    const float wx = u.y * vz - u.z * vy;
    const float wy = u.z * vx - u.x * vz;
    const float wz = u.x * vy - u.y * vx;
    f[0] = atan2f(dot3(wx, wy, wz, nb.x, nb.y, nb.z), dot3(u.x, u.y, u.z, nb.x, nb.y, nb.z));
    f[1] = dot3(vx, vy, vz, nb.x, nb.y, nb.z);
    f[2] = dot3(u.x, u.y, u.z, dx, dy, dz);
    return true;
}

// 0-based bin (Eq. A3) with the upper end clamped to H-1.
__device__ __forceinline__ int feature_bin(float f, float lo, float hi)
{
    float t = floorf((float)kH * (f - lo) / (hi - lo));
    t = fminf(fmaxf(t, 0.f), (float)(kH - 1));
    return (int)t;
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float term)
{
    const float y = term - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Compensated sum of the term a * b, its product fused with the subtraction
// of the compensation (one rounding), so that every kernel that adds the
// same terms in the same order gets the same bits.
__device__ __forceinline__ void kahan_add_prod(float& sum, float& comp, float a, float b)
{
    const float y = fmaf(a, b, -comp);
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// kahan_add_prod on two independent sums at once, in paired FP32
// instructions; ncomp holds the negated compensation.  Each component takes
// exactly kahan_add_prod's roundings: fma(a, b, -c), then s + y, then
// -((t - s) - y) computed as y + (s - t) (round-to-nearest is symmetric under
// negation, and s - t is the fma of t, -1 and s).  The paired form issues half
// the instructions for the same bits.
__device__ __forceinline__ void kahan_add_prod2(float2& sum, float2& ncomp, float2 a, float2 b)
{
    const float2 y = __ffma2_rn(a, b, ncomp);
    const float2 t = __fadd2_rn(sum, y);
    const float2 e = __ffma2_rn(t, make_float2(-1.f, -1.f), sum);
    ncomp = __fadd2_rn(y, e);
    sum = t;
}

}  // namespace kmxp
