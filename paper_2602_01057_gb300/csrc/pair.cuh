// Per-pair arithmetic of the general path (world coordinates), shared by the
// detector-tile kernels and the explicit-ray kernels: the closed form of
// Eqs. 7-11 for one ray and one Gaussian with the ray re-based at the foot of
// the perpendicular from mu, the erf factor of a finite segment, the pair's
// gradient, and a transposed warp reduction of per-lane gradient vectors.
#pragma once
#include "rgrt_internal.h"

namespace rgrt {
namespace {

constexpr float SQRT2PI = 2.50662827463100050f;
constexpr float INV_SQRT2PI = 0.398942280401432678f;
constexpr float INV_SQRTPI = 0.564189583547756287f;
constexpr float SQRT_HALF = 0.707106781186547524f;
constexpr float W_SAT = 4.0f;     // |w| >= 4: erf(w) == +-1 in binary32

struct Ray {
    float ox, oy, oz, dx, dy, dz, ta, tb;
};

struct PairGeo {
    float px, py, pz;      // recentred delta (perpendicular to d)
    float ta, tb;          // segment relative to the foot of the perpendicular
    float Pdx, Pdy, Pdz;   // P d
    float Ppx, Ppy, Ppz;   // P delta
    float A, B, C, rA, iA, m;
};

// general path: A, B, C, m of Eq. 7/9 with delta re-based at the foot of the
// perpendicular from mu (B small, no cancellation in C - B^2/A)
template <class Rec>
__device__ __forceinline__ void pair_geo(const Ray &r, const Rec &s, PairGeo &q)
{
    float ex = r.ox - s.g0.x, ey = r.oy - s.g0.y, ez = r.oz - s.g0.z;
    float tau = r.dx * ex + r.dy * ey + r.dz * ez;
    q.px = ex - tau * r.dx; q.py = ey - tau * r.dy; q.pz = ez - tau * r.dz;
    q.ta = r.ta + tau; q.tb = r.tb + tau;
    const float P00 = s.g1.x, P01 = s.g1.y, P02 = s.g1.z, P11 = s.g1.w, P12 = s.g2.x, P22 = s.g2.y;
    q.Pdx = P00 * r.dx + P01 * r.dy + P02 * r.dz;
    q.Pdy = P01 * r.dx + P11 * r.dy + P12 * r.dz;
    q.Pdz = P02 * r.dx + P12 * r.dy + P22 * r.dz;
    q.Ppx = P00 * q.px + P01 * q.py + P02 * q.pz;
    q.Ppy = P01 * q.px + P11 * q.py + P12 * q.pz;
    q.Ppz = P02 * q.px + P12 * q.py + P22 * q.pz;
    q.A = r.dx * q.Pdx + r.dy * q.Pdy + r.dz * q.Pdz;
    q.B = q.px * q.Pdx + q.py * q.Pdy + q.pz * q.Pdz;
    q.C = q.px * q.Ppx + q.py * q.Ppy + q.pz * q.Ppz;
    q.rA = rsqrtf(q.A);
    q.iA = q.rA * q.rA;
    q.m = q.C - q.B * q.B * q.iA;
}

// transposed warp reduction of N values: after it, lane l holds the warp sum
// of value owner_index(l) in v[0] (when that index is < N and l is even).
template <int N, int OFF>
__device__ __forceinline__ void tr_stage(float *v, int lane)
{
    if (N == 1) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], OFF);
    } else {
        constexpr int H = (N + 1) / 2;
        const bool hi = (lane & OFF) != 0;
#pragma unroll
        for (int i = 0; i < H; i++) {
            float a = v[i];
            float b = (i + H < N) ? v[i + H] : 0.0f;
            float send = hi ? a : b;
            float keep = hi ? b : a;
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
        }
    }
}

template <int N>
__device__ __forceinline__ int tr_reduce(float *v, int lane)
{
    constexpr int N1 = N, H1 = (N1 + 1) / 2;
    constexpr int N2 = N1 == 1 ? 1 : H1, H2 = (N2 + 1) / 2;
    constexpr int N3 = N2 == 1 ? 1 : H2, H3 = (N3 + 1) / 2;
    constexpr int N4 = N3 == 1 ? 1 : H3, H4 = (N4 + 1) / 2;
    constexpr int N5 = N4 == 1 ? 1 : H4;
    tr_stage<N1, 16>(v, lane);
    tr_stage<N2, 8>(v, lane);
    tr_stage<N3, 4>(v, lane);
    tr_stage<N4, 2>(v, lane);
    tr_stage<N5, 1>(v, lane);
    // walk the splits backwards: the lane's element sits at position p of
    // each stage's array; it is a padding zero if p ever falls outside it
    int p = 0;
    bool ok = true;
    if (N4 > 1 && (lane & 2)) { p += H4; ok &= p < N4; }
    if (N3 > 1 && (lane & 4)) { p += H3; ok &= p < N3; }
    if (N2 > 1 && (lane & 8)) { p += H2; ok &= p < N2; }
    if (N1 > 1 && (lane & 16)) { p += H1; ok &= p < N1; }
    // a plain butterfly stage (one value left) leaves both partners with the
    // same sum: only the partner with a clear bit owns it
    if (N1 == 1) ok &= !(lane & 16);
    if (N2 == 1) ok &= !(lane & 8);
    if (N3 == 1) ok &= !(lane & 4);
    if (N4 == 1) ok &= !(lane & 2);
    ok &= !(lane & 1);
    return ok ? p : N;
}

// general-path value: K = rho sqrt(2pi/A) e^{-m/2}; returns K Phi
__device__ __forceinline__ float general_value(const PairGeo &q, float rho)
{
    const float E = __expf(-0.5f * q.m);
    const float K = rho * SQRT2PI * q.rA * E;
    const float sc = q.rA * SQRT_HALF;
    const float wa = (q.A * q.ta + q.B) * sc, wb = (q.A * q.tb + q.B) * sc;
    float phi = 1.0f;
    if (!(wa <= -W_SAT && wb >= W_SAT)) phi = 0.5f * (erff(wb) - erff(wa));
    return K * phi;
}

// general-path gradient of one pair: dmu[3], G_P[6], drho (times dL/dI)
__device__ __forceinline__ void general_grad(const Ray &ray, const PairGeo &q, float rho, float gw,
                                             float *val)
{
    const float E = __expf(-0.5f * q.m);
    const float K = rho * SQRT2PI * q.rA * E;
    const float sc = q.rA * SQRT_HALF;
    const float wa = (q.A * q.ta + q.B) * sc, wb = (q.A * q.tb + q.B) * sc;
    float phi = 1.0f, dPhiB = 0.0f, dPhiA = 0.0f;
    if (!(wa <= -W_SAT && wb >= W_SAT)) {
        phi = 0.5f * (erff(wb) - erff(wa));
        const float ea = __expf(-wa * wa), eb = __expf(-wb * wb);
        dPhiB = (eb - ea) * q.rA * INV_SQRT2PI;
        const float tA = 2.0f * q.A;
        const float r32 = rsqrtf(tA) / tA;  // (2A)^-3/2
        // an infinite end contributes nothing (its Gaussian factor is 0)
        const float xa = isinf(q.ta) ? 0.0f : ea * (q.A * q.ta - q.B);
        const float xb = isinf(q.tb) ? 0.0f : eb * (q.A * q.tb - q.B);
        dPhiA = (xb - xa) * INV_SQRTPI * r32;
    }
    const float f = K * phi;
    const float fC = -0.5f * f;
    const float fB = f * q.B * q.iA + K * dPhiB;
    const float fA = -0.5f * f * q.iA * (1.0f + q.B * q.B * q.iA) + K * dPhiA;
    // gradient w.r.t. the recentred delta: fB P d + 2 fC P delta
    const float gx = fB * q.Pdx + 2.0f * fC * q.Ppx;
    const float gy = fB * q.Pdy + 2.0f * fC * q.Ppy;
    const float gz = fB * q.Pdz + 2.0f * fC * q.Ppz;
    const float dg = ray.dx * gx + ray.dy * gy + ray.dz * gz;
    const float st = K * q.A * dPhiB;  // d f / d(segment shift)
    // d mu = -(I - d d^T) grad - d * st
    val[0] = gw * (-(gx - ray.dx * dg) - ray.dx * st);
    val[1] = gw * (-(gy - ray.dy * dg) - ray.dy * st);
    val[2] = gw * (-(gz - ray.dz * dg) - ray.dz * st);
    // symmetric gradient w.r.t. P: fA d d^T + fB sym(d p^T) + fC p p^T
    const float hB = 0.5f * fB;
    val[3] = gw * (fA * ray.dx * ray.dx + 2.0f * hB * ray.dx * q.px + fC * q.px * q.px);
    val[4] = gw * (fA * ray.dx * ray.dy + hB * (ray.dx * q.py + q.px * ray.dy) + fC * q.px * q.py);
    val[5] = gw * (fA * ray.dx * ray.dz + hB * (ray.dx * q.pz + q.px * ray.dz) + fC * q.px * q.pz);
    val[6] = gw * (fA * ray.dy * ray.dy + 2.0f * hB * ray.dy * q.py + fC * q.py * q.py);
    val[7] = gw * (fA * ray.dy * ray.dz + hB * (ray.dy * q.pz + q.py * ray.dz) + fC * q.py * q.pz);
    val[8] = gw * (fA * ray.dz * ray.dz + 2.0f * hB * ray.dz * q.pz + fC * q.pz * q.pz);
    val[9] = gw * (SQRT2PI * q.rA * E * phi);
}


}  // namespace
}  // namespace rgrt
