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
    float sh;              // shift of the ray parameter to the recentred origin
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
    q.sh = tau;
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

// Kernel of the primitives: 0 = the Gaussian of Eq. 2; 1 = Epanechnikov,
// rho (1 - m / kappa^2)_+ with kappa^2 = 7 (the support whose normalised
// kernel has covariance Sigma).  Per kernel, in the view-space form:
//   QSCALE  factor of Q/A in the exponent argument (arg = QSCALE Q / A):
//           -log2(e)/2 for the Gaussian (arg feeds ex2), -1/kappa^2 for
//           Epanechnikov (c = 1 + arg is the kernel's profile factor);
//   FAC     alpha = rho FAC: the line integral per unit alpha is
//           A^-1/2 e^{-m/2} (FAC = sqrt(2 pi)) or A^-1/2 c^{3/2}
//           (FAC = 4 kappa / 3);
//   SKIP    K^2 of the per-warp skip boxes (a margin over the support);
//   BALL    radius, in sigma_max, beyond which a segment end has no effect.
template <int KER> struct Kern;
template <> struct Kern<0> {
    static constexpr float QSCALE = -0.721347520444481703f;
    static constexpr float FAC = 2.50662827463100050f;
    static constexpr float SKIP = 9.2f;
    static constexpr float BALL = 8.66f;   // (3 + 4 sqrt 2): erf(w) == +-1 beyond
};
template <> struct Kern<1> {
    static constexpr float KAPPA2 = 7.0f;
    static constexpr float QSCALE = -1.0f / 7.0f;
    static constexpr float FAC = 3.52766841475278f;   // 4 sqrt(7) / 3
    static constexpr float SKIP = 7.2f;
    static constexpr float BALL = 2.66f;              // sqrt(7) (1 + 0.5%)
};

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Epanechnikov on the general path: the integrand along the line is
// rho (c - A s^2 / kappa^2) for |s| <= a = sqrt(kappa^2 c / A), s measured
// from the Mahalanobis-closest point t* = -B/A; over [s0, s1] = the segment
// clipped to [-a, a] the integral is rho [c s - A s^3 / (3 kappa^2)] between
// them.  ea / eb: the lower / upper end is the segment's own (not +-a).
struct EpanSeg {
    float c, s0, s1;
    bool ea, eb, any;
};

__device__ __forceinline__ EpanSeg epan_seg(const PairGeo &q)
{
    constexpr float K2 = Kern<1>::KAPPA2;
    EpanSeg e;
    e.c = 1.0f - q.m * (1.0f / K2);
    e.any = false;
    e.ea = e.eb = false;
    e.s0 = e.s1 = 0.0f;
    if (!(e.c > 0.0f)) return e;
    const float a = sqrtf(K2 * e.c) * q.rA;
    const float sh = q.B * q.iA;
    const float sa = q.ta + sh, sb = q.tb + sh;
    e.ea = sa > -a;
    e.eb = sb < a;
    e.s0 = e.ea ? sa : -a;
    e.s1 = e.eb ? sb : a;
    e.any = e.s1 > e.s0;
    return e;
}

__device__ __forceinline__ float epan_F(const EpanSeg &e, float A, float s)
{
    return s * (e.c - A * s * s * (1.0f / (3.0f * Kern<1>::KAPPA2)));
}

// general-path value of one pair (rho times the kernel's line integral over
// the segment): Gaussian K Phi with K = rho sqrt(2pi/A) e^{-m/2}
// Time of flight (explicit rays, Gaussian kernel): a weight N(t; t_c,
// sigma_T^2) along the ray, tau = 1/sigma_T^2 (0: none), t_c in the ray's
// parameter.  The weighted integrand keeps the form of Eq. 7 with
// A' = A + tau, B' = B - tau t_c, C' = C + tau t_c^2 and the factor
// sqrt(tau / 2 pi); tof_geo returns the primed pair (t_c moved to the
// recentred origin like the segment) and that factor.
__device__ __forceinline__ float tof_geo(const PairGeo &q, float tc_ray, float tau, PairGeo &qp,
                                         float &tc)
{
    qp = q;
    tc = tc_ray + q.sh;
    qp.A = q.A + tau;
    qp.B = q.B - tau * tc;
    qp.C = q.C + tau * tc * tc;
    qp.rA = rsqrtf(qp.A);
    qp.iA = qp.rA * qp.rA;
    qp.m = qp.C - qp.B * qp.B * qp.iA;
    return sqrtf(tau) * INV_SQRT2PI;
}

template <int KER>
__device__ __forceinline__ float general_value(const PairGeo &q0, float rho, float tc_ray = 0.0f,
                                               float tau = 0.0f)
{
    if (KER == 1) {
        const EpanSeg e = epan_seg(q0);
        return e.any ? rho * (epan_F(e, q0.A, e.s1) - epan_F(e, q0.A, e.s0)) : 0.0f;
    }
    PairGeo qt;
    float tc, scale = 1.0f;
    if (tau > 0.0f) scale = tof_geo(q0, tc_ray, tau, qt, tc);
    const PairGeo &q = tau > 0.0f ? qt : q0;
    const float E = __expf(-0.5f * q.m);
    const float K = scale * rho * SQRT2PI * q.rA * E;
    const float sc = q.rA * SQRT_HALF;
    const float wa = (q.A * q.ta + q.B) * sc, wb = (q.A * q.tb + q.B) * sc;
    float phi = 1.0f;
    if (!(wa <= -W_SAT && wb >= W_SAT)) phi = 0.5f * (erff(wb) - erff(wa));
    return K * phi;
}

// general-path gradient of one pair: dmu[3], G_P[6], drho (times dL/dI).
// From the partials fA, fB, fC of the value in A, B, C and st, its
// derivative for a shift of both segment ends:
//   d mu = -(I - d d^T)(fB P d + 2 fC P p) - d st,
//   G_P = fA d d^T + fB sym(d p^T) + fC p p^T.
template <int KER>
__device__ __forceinline__ void general_grad(const Ray &ray, const PairGeo &q0, float rho, float gw,
                                             float *val, float tc_ray = 0.0f, float tau = 0.0f)
{
    float fA, fB, fC, st, frho;
    PairGeo qt;
    float tc = 0.0f, scale = 1.0f;
    if (KER == 0 && tau > 0.0f) scale = tof_geo(q0, tc_ray, tau, qt, tc);
    // the partials below are taken in the primed pair; A', B', C' move with
    // A, B, C one for one, and t_c shifts with the segment
    const PairGeo &q = (KER == 0 && tau > 0.0f) ? qt : q0;
    if (KER == 1) {
        // Leibniz: the clipped ends +-a carry a zero integrand; the segment's
        // own ends move with B and A through s = t + B/A
        constexpr float iK2 = 1.0f / Kern<1>::KAPPA2;
        const EpanSeg e = epan_seg(q);
        if (!e.any) {
#pragma unroll
            for (int k = 0; k < 10; k++) val[k] = 0.0f;
            return;
        }
        const float L = e.s1 - e.s0;
        const float phi1 = e.eb ? rho * (e.c - q.A * e.s1 * e.s1 * iK2) : 0.0f;
        const float phi0 = e.ea ? rho * (e.c - q.A * e.s0 * e.s0 * iK2) : 0.0f;
        const float bA = q.B * q.iA;
        fC = -rho * L * iK2;
        fB = 2.0f * rho * bA * L * iK2 + (phi1 - phi0) * q.iA;
        fA = -rho * (bA * bA * L + (e.s1 * e.s1 * e.s1 - e.s0 * e.s0 * e.s0) * (1.0f / 3.0f)) * iK2
             - (phi1 - phi0) * bA * q.iA;
        st = phi1 - phi0;
        frho = epan_F(e, q.A, e.s1) - epan_F(e, q.A, e.s0);
    } else {
        const float E = __expf(-0.5f * q.m);
        const float K = scale * rho * SQRT2PI * q.rA * E;
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
        fC = -0.5f * f;
        fB = f * q.B * q.iA + K * dPhiB;
        fA = -0.5f * f * q.iA * (1.0f + q.B * q.B * q.iA) + K * dPhiA;
        st = K * q.A * dPhiB;
        if (tau > 0.0f) st += tau * (2.0f * fC * tc - fB);   // d f / d t_c
        frho = scale * SQRT2PI * q.rA * E * phi;
    }
    // gradient w.r.t. the recentred delta: fB P d + 2 fC P delta
    const float gx = fB * q.Pdx + 2.0f * fC * q.Ppx;
    const float gy = fB * q.Pdy + 2.0f * fC * q.Ppy;
    const float gz = fB * q.Pdz + 2.0f * fC * q.Ppz;
    const float dg = ray.dx * gx + ray.dy * gy + ray.dz * gz;
    val[0] = gw * (-(gx - ray.dx * dg) - ray.dx * st);
    val[1] = gw * (-(gy - ray.dy * dg) - ray.dy * st);
    val[2] = gw * (-(gz - ray.dz * dg) - ray.dz * st);
    const float hB = 0.5f * fB;
    val[3] = gw * (fA * ray.dx * ray.dx + 2.0f * hB * ray.dx * q.px + fC * q.px * q.px);
    val[4] = gw * (fA * ray.dx * ray.dy + hB * (ray.dx * q.py + q.px * ray.dy) + fC * q.px * q.py);
    val[5] = gw * (fA * ray.dx * ray.dz + hB * (ray.dx * q.pz + q.px * ray.dz) + fC * q.px * q.pz);
    val[6] = gw * (fA * ray.dy * ray.dy + 2.0f * hB * ray.dy * q.py + fC * q.py * q.py);
    val[7] = gw * (fA * ray.dy * ray.dz + hB * (ray.dy * q.pz + q.py * ray.dz) + fC * q.py * q.pz);
    val[8] = gw * (fA * ray.dz * ray.dz + 2.0f * hB * ray.dz * q.pz + fC * q.pz * q.pz);
    val[9] = gw * frho;
}


}  // namespace
}  // namespace rgrt
