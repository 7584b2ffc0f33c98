// Per-tile ray integration (a3) and its adjoint (a5).
//
// One CTA per detector tile of tile_w x tile_h rays, one ray per thread,
// warps laid out as 8 x 4 ray blocks.  The tile's Gaussian list (ordered by
// footprint position, then id) is walked in chunks: the CTA gathers each
// chunk's records, turning every Gaussian into its view-space form for this
// view (see below) together with its detector bounding box, into one of two
// shared-memory buffers.  A warp skips a Gaussian whose box misses its 8 x 4
// block, or (cone beam) whose footprint ellipse misses it (a warp-uniform
// branch); otherwise every lane evaluates its pair and the pair counts when
// m <= 9 (3-sigma cut).  FP32 throughout, FP32 accumulation per ray.
// 3-D PET LORs (direction e_w + kappa e_v, kappa per detector column) have a
// view-space form of their own (prep_record, pet3d_chain).
//
// The closed form (Eqs. 7-11) for a ray and one Gaussian is
//   rho sqrt(2 pi / A) exp(-m/2),  A = d^T P d,  m = C - B^2/A,
// with unit d.  Two exact rewritings make the per-pair work small:
//  * m does not depend on the length of d, and
//      A C - B^2 = (d x delta)^T cof(P) (d x delta),  cof(P) = Sigma / det Sigma,
//    so m = Q / A with Q = c^T S c, c = d x delta, S = Sigma / det Sigma.
//  * In the frame (e_u, e_v, e_w) of a view every ray is fixed by its
//    detector coordinates (u, v).  For parallel rays (CT parallel beam, PET)
//    d = e_w: A = P'_ww is a per-(Gaussian, view) constant and
//    c = du e_v - dv e_u with (du, dv) = (u - mu_u, v - mu_v), so Q is a 2x2
//    quadratic form.  For cone-beam rays from the source S, d~ = (u, v, dsd)
//    and delta = S - mu is the same for every ray of the view; writing
//    d~ = d~0 + (du, dv, 0) with d~0 the ray through mu, c = du g_u + dv g_v
//    (g_u = e_u x delta, g_v = e_v x delta) and A(du, dv) = d~^T P' d~ are
//    both quadratic in (du, dv), and the integral along the physical ray is
//    |d~| rho sqrt(2 pi / A) exp(-Q/(2A)).
// Both forms avoid the cancellation of C - B^2/A entirely.  Segment ends
// (erf terms) only matter for a Gaussian whose 3-sigma ball lies within
// 5.66 sigma of a segment end (then |w| < 4 is possible); such Gaussians take
// the general path below, in world coordinates, with the ray re-based at the
// foot of the perpendicular from mu.
#include "pair.cuh"

namespace rgrt {
namespace {

constexpr int CH = 256;             // records per chunk (one per thread in the prep)
// chunk buffers of the forward: with two, a chunk's records are prepared into
// one buffer while slower warps still read the other, and a single barrier
// per chunk suffices.  The staged records (52 B each) leave the general-path
// fields in global memory so that two buffers still fit 4 CTAs per SM.
constexpr int NBUF = 2;
constexpr int ADJ_BS = 128;         // threads of an adjoint CTA (one Gaussian each)
constexpr float M_PER_ARG = -1.38629436111989061f;        // m = arg * (-2 ln 2)
constexpr float CUT_ARG = -6.49212768400033233f;          // arg at m = 9
constexpr int NG = 10;            // general path: dmu[3], G_P[6], drho
constexpr int NV_CONE = 12;       // view-space moments, cone beam

// a Gaussian in the view of the current tile (shared memory)
// The Q coefficients carry the factor -log2(e)/2 (and, for parallel rays, 1/A)
// so that arg = Q/A * (-log2(e)/2) feeds ex2 directly; m = -2 ln2 arg.
struct VRec {
    float4 c0;  // u0, v0, k M_uu, 2 k M_uv               (k = -log2(e)/2, x 1/A for parallel rays)
    float4 c1;  // k M_vv, A0 (cone) | 1/A (parallel), 2 a_u (cone) | 1/sqrt(A) (parallel), 2 a_v
    float4 c2;  // P'_uu, 2 P'_uv, P'_vv, alpha = rho sqrt(2 pi) (cone) | alpha/sqrt(A) (parallel)
    float4 bb;  // u_lo, u_hi, v_lo, v_hi of the detector box (skip test)
    float4 g0;  // mu, rho                      (general path)
    float4 g1;  // P00 P01 P02 P11              (general path)
    float4 g2;  // P12 P22, gid bits, 1 = view-space path / 0 = general path
    float4 t4;  // parallel rays: the closest approach along the ray, t* = x + y du + z dv, and 1/A (w)
};

// the forward's copy of a VRec: the view-space coefficients and the gid
// (general-path records read mu, rho and P from the global records by gid)
struct SRec {
    float4 c0, c1, c2;
    uint32_t gid;
};

// a chunk of staged records in shared memory, one array per field: the
// preparing threads write consecutive 16-byte (4-byte) words, free of bank
// conflicts, and a warp reads one record at a time (broadcast)
struct SChunk {
    float4 c0[CH], c1[CH], c2[CH];
    uint32_t gid[CH];
    __device__ __forceinline__ SRec operator[](int j) const
    {
        SRec r;
        r.c0 = c0[j];
        r.c1 = c1[j];
        r.c2 = c2[j];
        r.gid = gid[j];
        return r;
    }
};

// the general-path fields of record gid (mu, rho | P00 P01 P02 P11 | P12 P22)
struct GRec {
    float4 g0, g1, g2;
};
__device__ __forceinline__ GRec load_grec(const float4 *__restrict__ rec, uint32_t gid)
{
    const float4 *r = rec + REC_F4 * (size_t)gid;
    GRec o;
    o.g0 = __ldg(r);
    o.g1 = __ldg(r + 1);
    o.g2 = __ldg(r + 2);
    return o;
}

__device__ __forceinline__ bool cone_interval(float K2, float dsd, float ae, float aw, float see,
                                              float sew, float sww, float &lo, float &hi)
{
    float alpha = aw * aw - K2 * sww;
    if (!(alpha > 0.0f)) return false;
    float beta = dsd * (ae * aw - K2 * sew);
    float disc = aw * aw * see - 2.0f * ae * aw * sew + ae * ae * sww - K2 * (see * sww - sew * sew);
    disc = fmaxf(disc, 0.0f);
    float r = dsd * sqrtf(K2 * disc);
    lo = (beta - r) / alpha;
    hi = (beta + r) / alpha;
    return true;
}

// Every detector geometry's view frame is a rotation about z (geom_tables):
// e_v = (0, 0, 1), e_u = (a, b, 0), e_w = (p, q, 0).  The transforms below
// use that shape: a symmetric X in the frame costs 18 operations instead of
// six general quadratic forms, and a frame matrix back to world as many.
struct AxFrame {
    float a, b, p, q;
};
__device__ __forceinline__ AxFrame ax_frame(const float *F)
{
    AxFrame f;
    f.a = F[0]; f.b = F[1]; f.p = F[6]; f.q = F[7];
    return f;
}

// X (symmetric, packed 00 01 02 11 12 22) in the frame: (uu, uv, uw, vv, vw, ww)
__device__ __forceinline__ void to_frame_ax(const float *X, const AxFrame &f, float *o)
{
    const float xa = X[0] * f.a + X[1] * f.b, xb = X[1] * f.a + X[3] * f.b;   // X e_u (x, y)
    const float xp = X[0] * f.p + X[1] * f.q, xq = X[1] * f.p + X[3] * f.q;   // X e_w (x, y)
    o[0] = f.a * xa + f.b * xb;
    o[1] = X[2] * f.a + X[4] * f.b;
    o[2] = f.a * xp + f.b * xq;
    o[3] = X[5];
    o[4] = X[2] * f.p + X[4] * f.q;
    o[5] = f.p * xp + f.q * xq;
}

// symmetric G' (packed uu uv uw vv vw ww) back to world, G = E G' E^T with
// E = [e_u e_v e_w]: world x = a u + p w, y = b u + q w, z = v
__device__ __forceinline__ void from_frame_ax(const float *Gf, const AxFrame &f, float *G)
{
    const float hu0 = Gf[0] * f.a + Gf[2] * f.p, hw0 = Gf[2] * f.a + Gf[5] * f.p;
    const float hu1 = Gf[0] * f.b + Gf[2] * f.q, hw1 = Gf[2] * f.b + Gf[5] * f.q;
    G[0] = f.a * hu0 + f.p * hw0;
    G[1] = f.a * hu1 + f.p * hw1;
    G[2] = f.a * Gf[1] + f.p * Gf[4];
    G[3] = f.b * hu1 + f.q * hw1;
    G[4] = f.b * Gf[1] + f.q * Gf[4];
    G[5] = Gf[3];
}

// The footprint of a cone-beam record on the detector: rays at offset
// (du, dv) from (u0, v0) with m <= K^2 satisfy Q - K^2 A <= 0, Q and A
// quadratics in (du, dv):
//   G(du, dv) = a du^2 + 2 b du dv + c dv^2 + 2 d du + 2 e dv + f <= 0.
// When the quadratic part is positive definite (an ellipse: the K-sigma
// ellipsoid lies in front of the source) G is convex, and G(x) >= G(x0) +
// grad G(x0).(x - x0) bounds it from below over a rectangle around x0.
struct Conic {
    float a, b, c, d, e, f;
    bool ok;
};

// the footprint conic of a cone-beam view-space record (offsets from u0, v0)
template <int KER>
__device__ __forceinline__ Conic cone_conic(const VRec &r)
{
    const float4 c0 = r.c0, c1 = r.c1, c2 = r.c2;
    const float K2 = Kern<KER>::SKIP, ik = 1.0f / Kern<KER>::QSCALE;
    Conic cn;
    cn.a = c0.z * ik - K2 * c2.x;
    cn.b = 0.5f * (c0.w * ik - K2 * c2.y);
    cn.c = c1.x * ik - K2 * c2.z;
    cn.d = -0.5f * K2 * c1.z;
    cn.e = -0.5f * K2 * c1.w;
    cn.f = -K2 * c1.y;
    cn.ok = cn.a > 0.0f && cn.a * cn.c - cn.b * cn.b > 1e-3f * cn.a * cn.c;
    return cn;
}

// gather one record and turn it into its view-space form for frame F
// (3-D PET: kap0, kap1 are the extreme LOR slopes of the tile's columns)
template <int GM, int KER>
__device__ __forceinline__ void prep_record(const DevGeom &g, const float *F, uint32_t gid,
                                            const float4 *__restrict__ rec,
                                            const float4 *__restrict__ crec, VRec &out,
                                            float kap0 = 0.0f, float kap1 = 0.0f)
{
    constexpr bool CONE = GM == GM_CONE;
    const float4 *r = rec + REC_F4 * (size_t)gid;
    float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3), r4 = __ldg(r + 4);
    out.t4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float4 k1 = __ldg(crec + CREC_F4 * (size_t)gid + 1), k2 = __ldg(crec + CREC_F4 * (size_t)gid + 2);
    const float Sg[6] = { k1.x, k1.y, k1.z, k1.w, k2.x, k2.y };
    const float P[6] = { r1.x, r1.y, r1.z, r1.w, r2.x, r2.y };
    const float Sh[6] = { r2.z, r2.w, r3.x, r3.y, r3.z, r3.w };
    const float m[3] = { r0.x, r0.y, r0.z };
    const float rho = r0.w, smax = r4.x;
    const AxFrame fr = ax_frame(F);
    const float mu_u = m[0] * fr.a + m[1] * fr.b;
    const float mu_v = m[2];
    const float mu_w = m[0] * fr.p + m[1] * fr.q;
    float Pf[6], Sf[6], Gf[6];   // P, Sigma / det Sigma and Sigma in the frame
    to_frame_ax(P, fr, Pf);
    to_frame_ax(Sh, fr, Sf);
    to_frame_ax(Sg, fr, Gf);
    float ulo = -INFINITY, uhi = INFINITY, vlo = -INFINITY, vhi = INFINITY;
    bool sat;
    if (CONE) {
        const float D = mu_w + g.dso;           // depth of mu from the source
        float suu = Gf[0], svv = Gf[3], sww = Gf[5];
        float suw = Gf[2], svw = Gf[4];
        float lo, hi;
        if (cone_interval(Kern<KER>::SKIP, g.dsd, mu_u, D, suu, suw, sww, lo, hi)) { ulo = lo; uhi = hi; }
        if (cone_interval(Kern<KER>::SKIP, g.dsd, mu_v, D, svv, svw, sww, lo, hi)) { vlo = lo; vhi = hi; }
        const float iD = 1.0f / D;
        const float u0 = g.dsd * mu_u * iD, v0 = g.dsd * mu_v * iD;
        // A(du, dv) = d~^T P' d~, d~ = (u0 + du, v0 + dv, dsd)
        const float au = Pf[0] * u0 + Pf[1] * v0 + Pf[2] * g.dsd;
        const float av = Pf[1] * u0 + Pf[3] * v0 + Pf[4] * g.dsd;
        const float aw = Pf[2] * u0 + Pf[4] * v0 + Pf[5] * g.dsd;
        const float A0 = au * u0 + av * v0 + aw * g.dsd;
        // g_u = e_u x delta = (0, D, -mu_v), g_v = e_v x delta = (-D, 0, mu_u)
        const float guv = D, guw = -mu_v, gvu = -D, gvw = mu_u;
        const float cu1 = Sf[3] * guv + Sf[4] * guw, cu2 = Sf[4] * guv + Sf[5] * guw;  // (S' g_u)_{v,w}
        const float cv0 = Sf[0] * gvu + Sf[2] * gvw, cv1 = Sf[1] * gvu + Sf[4] * gvw,
                    cv2 = Sf[2] * gvu + Sf[5] * gvw;                                  // S' g_v
        const float Muu = guv * cu1 + guw * cu2;
        const float Muv = guv * cv1 + guw * cv2;
        const float Mvv = gvu * cv0 + gvw * cv2;
        const float k = Kern<KER>::QSCALE;
        out.c0 = make_float4(u0, v0, k * Muu, 2.0f * k * Muv);
        out.c1 = make_float4(k * Mvv, A0, 2.0f * au, 2.0f * av);
        out.c2 = make_float4(Pf[0], 2.0f * Pf[1], Pf[3], rho * Kern<KER>::FAC);

        // both segment ends (source, detector plane) beyond the 8.66-sigma ball
        sat = D >= Kern<KER>::BALL * smax && (g.dsd - D) >= Kern<KER>::BALL * smax;
    } else if (GM == GM_PET3D) {
        // LOR through (u, z) at w = 0 with direction d~ = e_w + kappa e_v:
        // with du = u - mu_u and v~ = z - mu_v + kappa mu_w (the LOR's height
        // at depth mu_w, relative to mu), c = d~ x delta = (-v~, du, -kappa du),
        //   Q = du^2 (S'_vv - 2 kappa S'_vw + kappa^2 S'_ww)
        //     + 2 du v~ (kappa S'_uw - S'_uv) + v~^2 S'_uu,
        //   A = d~^T P' d~ = P'_ww (1 + kappa (2 P'_vw + kappa P'_vv) / P'_ww),
        // and the integral along the unit ray is |d~| rho sqrt(2 pi / A)
        // exp(-Q / 2A); the coefficients carry the 1/P'_ww.
        float hu = sqrtf(Kern<KER>::SKIP * Gf[0]);
        ulo = mu_u - hu; uhi = mu_u + hu;
        // heights z whose LORs can meet the box ellipsoid (the bounds at the
        // two extreme slopes span those of every slope between them)
        const float svv = Gf[3], svw = Gf[4], sww = Gf[5];
        vlo = INFINITY; vhi = -INFINITY;
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const float kap = e ? kap1 : kap0;
            const float zc = mu_v - kap * mu_w;
            const float half = sqrtf(fmaxf(Kern<KER>::SKIP * (svv - 2.0f * kap * svw + kap * kap * sww), 0.0f));
            vlo = fminf(vlo, zc - half);
            vhi = fmaxf(vhi, zc + half);
        }
        const float iP = 1.0f / Pf[5];
        const float k = Kern<KER>::QSCALE * iP;
        out.c0 = make_float4(mu_u, mu_v, mu_w, k * Sf[0]);
        out.c1 = make_float4(k * Sf[3], -2.0f * k * Sf[4], k * Sf[5], -2.0f * k * Sf[1]);
        out.c2 = make_float4(2.0f * k * Sf[2], 2.0f * Pf[4] * iP, Pf[3] * iP, rho * Kern<KER>::FAC * sqrtf(iP));
        // the LOR ends on the ring: beyond the ball if the ball is inside it
        const float rxy = sqrtf(m[0] * m[0] + m[1] * m[1]);
        sat = rxy + Kern<KER>::BALL * smax <= sqrtf(g.radius2);
    } else {
        float hu = sqrtf(Kern<KER>::SKIP * Gf[0]);
        float hv = sqrtf(Kern<KER>::SKIP * Gf[3]);
        ulo = mu_u - hu; uhi = mu_u + hu; vlo = mu_v - hv; vhi = mu_v + hv;
        const float iA = 1.0f / Pf[5];
        const float rA = sqrtf(iA);
        // c = du e_v - dv e_u: M_uu = S'_vv, M_uv = -S'_uv, M_vv = S'_uu
        const float k = Kern<KER>::QSCALE * iA;
        out.c0 = make_float4(mu_u, mu_v, k * Sf[3], -2.0f * k * Sf[1]);
        out.c1 = make_float4(k * Sf[0], iA, rA, 0.0f);
        out.c2 = make_float4(0.0f, 0.0f, 0.0f, rho * Kern<KER>::FAC * rA);
        // along the ray (direction e_w) the exponent is smallest at
        // t* = mu_w - (P'_uw du + P'_vw dv) / P'_ww
        out.t4 = make_float4(mu_w, -Pf[2] * iA, -Pf[4] * iA, iA);

        if (g.pet) {
            float rxy = sqrtf(m[0] * m[0] + m[1] * m[1]);
            sat = rxy + Kern<KER>::BALL * smax <= sqrtf(g.radius2);
        } else {
            sat = mu_w - Kern<KER>::BALL * smax >= g.t_a && mu_w + Kern<KER>::BALL * smax <= g.t_b;
        }
    }
    out.bb = make_float4(ulo, uhi, vlo, vhi);
    out.g0 = r0;
    out.g1 = r1;
    out.g2 = make_float4(r2.x, r2.y, __uint_as_float(gid), sat ? 1.0f : 0.0f);
}

// ray of detector pixel (u, v) in view frame F (FP32), for the general path
// (3-D PET: v is the LOR's mid-height, kap its slope dz/dw)
template <int GM>
__device__ __forceinline__ Ray make_ray(const DevGeom &g, const float *F, float u, float v, float kap = 0.0f)
{
    float op0, op1, op2, dp0, dp1, dp2, ta, tb;
    if (GM == GM_PET3D) {
        // o' = (u, v, 0), d' = (0, kappa, 1)/L, L = sqrt(1 + kappa^2); the LOR
        // runs over w in [-h, h], h = sqrt(R^2 - u^2), i.e. t = w L
        const float L = sqrtf(1.0f + kap * kap), iL = 1.0f / L;
        const float h = sqrtf(fmaxf(g.radius2 - u * u, 0.0f));
        op0 = u; op1 = v; op2 = 0.0f;
        dp0 = 0.0f; dp1 = kap * iL; dp2 = iL;
        ta = -h * L; tb = h * L;
    } else if (GM == GM_CONE) {
        // d' = (u, v, dsd)/L;  o' = closest point to the origin on the ray,
        // o' = dso/L^2 (dsd u, dsd v, -(u^2+v^2)) (no cancellation);
        // segment from the source (t_a) to the pixel (t_b), measured from o'
        float uv2 = u * u + v * v;
        float L2 = uv2 + g.dsd * g.dsd;
        float iL = rsqrtf(L2);
        float c = g.dso / L2;
        dp0 = u * iL; dp1 = v * iL; dp2 = g.dsd * iL;
        op0 = c * g.dsd * u; op1 = c * g.dsd * v; op2 = -c * uv2;
        ta = -g.dso * g.dsd * iL;
        tb = (uv2 + g.dsd * (g.dsd - g.dso)) * iL;
    } else {
        op0 = u; op1 = v; op2 = 0.0f;
        dp0 = 0.0f; dp1 = 0.0f; dp2 = 1.0f;
        if (g.pet) {
            float h = sqrtf(fmaxf(g.radius2 - u * u, 0.0f));
            ta = -h; tb = h;
        } else {
            ta = g.t_a; tb = g.t_b;
        }
    }
    Ray r;
    r.ox = op0 * F[0] + op1 * F[3] + op2 * F[6];
    r.oy = op0 * F[1] + op1 * F[4] + op2 * F[7];
    r.oz = op0 * F[2] + op1 * F[5] + op2 * F[8];
    r.dx = dp0 * F[0] + dp1 * F[3] + dp2 * F[6];
    r.dy = dp0 * F[1] + dp1 * F[4] + dp2 * F[7];
    r.dz = dp0 * F[2] + dp1 * F[5] + dp2 * F[8];
    r.ta = ta;
    r.tb = tb;
    return r;
}

struct TileCtx {
    int vl, tx, ty, view, col, row;
    bool valid;                        // the thread's pixel is on the detector
    bool live;                         // ... and has a ray (3-D PET: a ring pair)
    float wu_lo, wu_hi, wv_lo, wv_hi;  // detector box of this warp's (half-warp's) rays
    float zoff, dz;                    // 3-D PET: mid-height offset of the rows, axial LOR rise
    float kap0, kap1;                  // 3-D PET: LOR slopes at the tile's extreme columns
    long long out_idx;
};

// 3-D PET: LOR slope dz/dw at radial position u (dz: axial rise over the chord)
__device__ __forceinline__ float pet3d_slope(const DevGeom &g, float dz, float u)
{
    return 0.5f * dz / sqrtf(fmaxf(g.radius2 - u * u, 1e-30f));
}

// 3-D PET view: (offset of the row heights, axial rise, rows with a ring pair)
__device__ __forceinline__ void pet3d_view(const DevGeom &g, int view, float &zoff, float &dz, int &rows)
{
    const int delta = pet3d_delta(g, view), ad = abs(delta);
    zoff = 0.5f * (float)ad * g.ring_pitch;
    dz = (float)delta * g.ring_pitch;
    rows = g.n_rows - ad;
}

// 3-D PET: LOR slopes at the extreme |u| of columns c0..c1
__device__ __forceinline__ void pet3d_slopes(const DevGeom &g, float dz, int c0, int c1, float &k0, float &k1)
{
    const float ua = __ldg(g.utab + c0), ub = __ldg(g.utab + c1);
    const float amin = (ua <= 0.0f && ub >= 0.0f) ? 0.0f : fminf(fabsf(ua), fabsf(ub));
    const float amax = fmaxf(fabsf(ua), fabsf(ub));
    k0 = pet3d_slope(g, dz, amin);
    k1 = pet3d_slope(g, dz, amax);
}

// Half-warp blocks (4 x 4 rays per half-warp) for the parallel-ray and 3-D
// PET geometries, whose footprints span a few bins; cone-beam footprints are
// large enough that whole-warp 8 x 4 blocks waste little and build their
// lists for less.
template <int GM>
struct HalfBlocks {
    static constexpr bool value = GM != GM_CONE;
};

template <int GM>
__device__ __forceinline__ TileCtx tile_ctx(const DevGeom &g, uint32_t tile)
{
    constexpr bool HALF = HalfBlocks<GM>::value;
    TileCtx c;
    int T = g.tiles_x * g.tiles_y;
    c.vl = (int)(tile / (uint32_t)T);
    int tin = (int)tile - c.vl * T;
    c.ty = tin / g.tiles_x;
    c.tx = tin - c.ty * g.tiles_x;
    c.view = g.v0 + c.vl;
    // a warp takes an 8 x 4 block of rays (HALF: each half-warp a 4 x 4 half of it)
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int wpr = g.tile_w >> 3;  // warps per tile row
    int wx = w % wpr, wy = w / wpr;
    int c0 = c.tx * g.tile_w + wx * 8 + (HALF ? 4 * (lane >> 4) : 0), r0 = c.ty * g.tile_h + wy * 4;
    c.col = c0 + (HALF ? (lane & 3) : (lane & 7));
    c.row = r0 + (HALF ? ((lane >> 2) & 3) : (lane >> 3));
    c.valid = c.col < g.n_cols && c.row < g.n_rows;
    int rows = g.n_rows;
    c.zoff = c.dz = c.kap0 = c.kap1 = 0.0f;
    if (GM == GM_PET3D) {
        pet3d_view(g, c.view, c.zoff, c.dz, rows);
        const int tc0 = c.tx * g.tile_w;
        pet3d_slopes(g, c.dz, tc0, min(tc0 + g.tile_w - 1, g.n_cols - 1), c.kap0, c.kap1);
    }
    c.live = c.valid && c.row < rows;
    if (c0 < g.n_cols && r0 < rows) {
        int c1 = min(c0 + (HALF ? 3 : 7), g.n_cols - 1), r1 = min(r0 + 3, rows - 1);
        c.wu_lo = __ldg(g.utab + c0); c.wu_hi = __ldg(g.utab + c1);
        c.wv_lo = __ldg(g.vtab + r0) + c.zoff; c.wv_hi = __ldg(g.vtab + r1) + c.zoff;
    } else {
        c.wu_lo = INFINITY; c.wu_hi = -INFINITY; c.wv_lo = INFINITY; c.wv_hi = -INFINITY;
    }
    c.out_idx = (long long)c.view * g.stride_view + (long long)c.row * g.stride_row + c.col;
    return c;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per chunk: every thread turns one record into its view-space form and tests
// its detector box against the ray block of every warp of the tile (bit w of
// msk), or with half-warp blocks of every half-warp (bit 2w + h, h the half of
// warp w); then each warp compacts, in record order, the records that touch
// its block (each of its halves' blocks) into a list of view-space records and
// a list of general ones.  The two halves of a warp walk their own lists side
// by side: smaller blocks leave fewer lanes evaluating pairs outside the
// footprint.
constexpr uint32_t MSK_VS = 1u << 16;   // msk: the record takes the view-space path
struct ChunkLists {
    uint8_t vs[16][CH];
    uint8_t gen[16][CH];
};

template <int GM, int KER, bool TOF>
__device__ __forceinline__ void prep_chunk(const DevGeom &g, const float *F, const uint32_t *gids,
                                           uint32_t base, uint32_t stride, int cnt,
                                           const float4 *rec, const float4 *crec, SChunk *sv,
                                           const float4 *wbox, int nw, uint32_t *msk,
                                           float kap0, float kap1)
{
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t gid = __ldg(gids + base + (uint32_t)i * stride);
        VRec vr;
        prep_record<GM, KER>(g, F, gid, rec, crec, vr, kap0, kap1);
        if (TOF) {
            // time of flight (parallel rays): the pair's value times the
            // kernel of width s^2 = 1/A + sigma_T^2 at t* - t_k (the
            // convolution of the Gaussian's profile along the ray with the
            // TOF kernel): c1.y = -log2(e) / (2 s^2), c1.z = 1/sqrt(2 pi s^2),
            // c2.xyz = the coefficients of t*
            const float s2 = vr.t4.w + g.tof_s2;
            vr.c1.y = Kern<0>::QSCALE / s2;
            vr.c1.z = rsqrtf(2.0f * 3.14159265358979324f * s2);
            vr.c2.x = vr.t4.x;
            vr.c2.y = vr.t4.y;
            vr.c2.z = vr.t4.z;
        }
        sv->c0[i] = vr.c0;
        sv->c1[i] = vr.c1;
        sv->c2[i] = vr.c2;
        sv->gid[i] = gid;
        const float4 bb = vr.bb;
        // a block inside the footprint's box may still miss the footprint
        // ellipse: skip it when the tangent plane of G at the block centre
        // stays above tol over the block (a pair with m <= 9 + 9e-4 has
        // G <= -0.19 A < 0 at K^2 = 9.2, so none is lost).  Cone beam only:
        // the small footprints of the parallel-ray workloads fill their boxes'
        // blocks, and the test there cost more than it saved.
        Conic cn;
        cn.ok = false;
        float u0 = 0.0f, v0 = 0.0f;
        if (GM == GM_CONE) {
            cn = cone_conic<KER>(vr);
            u0 = vr.c0.x;
            v0 = vr.c0.y;
        }
        const float tol = 1e-3f * fabsf(cn.f);
        uint32_t m = 0;
        for (int w = 0; w < (HalfBlocks<GM>::value ? 2 * nw : nw); w++) {
            const float4 wb = wbox[w];
            bool hit = !(bb.y < wb.x || bb.x > wb.y || bb.w < wb.z || bb.z > wb.w);
            if (GM == GM_CONE && hit && cn.ok) {
                const float cu = 0.5f * (wb.x + wb.y) - u0, cv = 0.5f * (wb.z + wb.w) - v0;
                const float hu = 0.5f * (wb.y - wb.x), hv = 0.5f * (wb.w - wb.z);
                const float gu = cn.a * cu + cn.b * cv + cn.d, gv = cn.b * cu + cn.c * cv + cn.e;
                const float G = cu * (gu + cn.d) + cv * (gv + cn.e) + cn.f;
                hit = G - 2.0f * (fabsf(gu) * hu + fabsf(gv) * hv) <= tol;
            }
            m |= (uint32_t)hit << w;
        }
        if (vr.g2.w != 0.0f) m |= MSK_VS;
        msk[i] = m;
    }
}

// warp-private compaction; returns the list lengths in nvs, ngen
// nvs, ngen: the lengths of this lane's lists
template <bool HALF>
__device__ __forceinline__ void build_lists(int cnt, const uint32_t *msk, ChunkLists &L, int w,
                                            int lane, int &nvs, int &ngen)
{
    const uint32_t lt = (1u << lane) - 1u;
    if (!HALF) {
        nvs = 0;
        ngen = 0;
        for (int b = 0; b < cnt; b += 32) {
            const int i = b + lane;
            const uint32_t m = i < cnt ? msk[i] : 0u;
            const bool in = (m >> w) & 1u;
            const bool vs = (m & MSK_VS) != 0u;
            const uint32_t bv = __ballot_sync(0xffffffffu, in && vs);
            const uint32_t bg = __ballot_sync(0xffffffffu, in && !vs);
            if (in && vs) L.vs[w][nvs + __popc(bv & lt)] = (uint8_t)i;
            if (in && !vs) L.gen[w][ngen + __popc(bg & lt)] = (uint8_t)i;
            nvs += __popc(bv);
            ngen += __popc(bg);
        }
        __syncwarp();
        return;
    }
    int v0 = 0, v1 = 0, g0 = 0, g1 = 0;
    for (int b = 0; b < cnt; b += 32) {
        const int i = b + lane;
        const uint32_t m = i < cnt ? msk[i] : 0u;
        const bool in0 = (m >> (2 * w)) & 1u, in1 = (m >> (2 * w + 1)) & 1u;
        const bool vs = (m & MSK_VS) != 0u;
        const uint32_t bv0 = __ballot_sync(0xffffffffu, in0 && vs);
        const uint32_t bv1 = __ballot_sync(0xffffffffu, in1 && vs);
        const uint32_t bg0 = __ballot_sync(0xffffffffu, in0 && !vs);
        const uint32_t bg1 = __ballot_sync(0xffffffffu, in1 && !vs);
        if (in0 && vs) L.vs[2 * w][v0 + __popc(bv0 & lt)] = (uint8_t)i;
        if (in1 && vs) L.vs[2 * w + 1][v1 + __popc(bv1 & lt)] = (uint8_t)i;
        if (in0 && !vs) L.gen[2 * w][g0 + __popc(bg0 & lt)] = (uint8_t)i;
        if (in1 && !vs) L.gen[2 * w + 1][g1 + __popc(bg1 & lt)] = (uint8_t)i;
        v0 += __popc(bv0);
        v1 += __popc(bv1);
        g0 += __popc(bg0);
        g1 += __popc(bg1);
    }
    __syncwarp();
    const bool h = lane >= 16;
    nvs = h ? v1 : v0;
    ngen = h ? g1 : g0;
}

// the warps' detector boxes, wbox[w] (HALF: the half-warps', wbox[2w + h])
template <bool HALF>
__device__ __forceinline__ void warp_box(const TileCtx &c, float4 *wbox)
{
    if ((threadIdx.x & (HALF ? 15 : 31)) == 0)
        wbox[threadIdx.x >> (HALF ? 4 : 5)] = make_float4(c.wu_lo, c.wu_hi, c.wv_lo, c.wv_hi);
}

// view-space value of one pair (without the |d~| factor of cone beam and
// 3-D PET); returns arg = QSCALE m (Gaussian: -m log2(e)/2; Epanechnikov:
// -m/kappa^2).  kap: the ray's slope (3-D PET).
template <int GM, int KER, class R>
__device__ __forceinline__ float vs_value(const R &r, float u, float v, float kap, float &arg)
{
    const float4 c0 = r.c0, c1 = r.c1, c2 = r.c2;
    float rA = 1.0f;
    if (GM == GM_PET3D) {
        const float du = u - c0.x, vt = fmaf(kap, c0.z, v - c0.y);
        const float muu = fmaf(fmaf(c1.z, kap, c1.y), kap, c1.x);
        const float muv2 = fmaf(c2.x, kap, c1.w);
        const float q = du * (muu * du + muv2 * vt) + c0.w * vt * vt;
        const float An = fmaf(fmaf(c2.z, kap, c2.y), kap, 1.0f);
        rA = rsqrt_approx(An);
        arg = q * (rA * rA);
        if (KER == 1) {
            const float c = 1.0f + arg;
            const float pc = c > 0.0f ? c * sqrt_approx(c) : 0.0f;
            return c2.w * rA * pc;
        }
        return c2.w * rA * ex2_approx(arg);
    }
    const float du = u - c0.x, dv = v - c0.y;
    const float q = du * (c0.z * du + c0.w * dv) + c1.x * dv * dv;
    if (GM == GM_CONE) {
        const float A = c1.y + du * (c1.z + c2.x * du + c2.y * dv) + dv * (c1.w + c2.z * dv);
        rA = rsqrt_approx(A);
        arg = q * (rA * rA);
    } else {
        arg = q;
    }
    if (KER == 1) {
        const float c = 1.0f + arg;                      // 1 - m / kappa^2
        const float pc = c > 0.0f ? c * sqrt_approx(c) : 0.0f;
        return c2.w * rA * pc;
    }
    return c2.w * rA * ex2_approx(arg);
}

// the pair counts (Gaussian: m <= 9; Epanechnikov: inside the support)
template <int KER>
__device__ __forceinline__ bool vs_keep(float arg)
{
    return KER == 1 ? arg > -1.0f : arg >= CUT_ARG;
}

// forward integration of tile `tile` of geometry g (one ray per thread)
template <int GM, bool STATS, int KER, bool TOF = false>
__device__ __forceinline__ void forward_tile(const DevGeom &g, uint32_t tile,
                                             const float4 *__restrict__ rec,
                                             const float4 *__restrict__ crec,
                                             const uint32_t *__restrict__ gids,
                                             const uint2 *__restrict__ ranges,
                                             float *__restrict__ out, Stats *stats)
{
    __shared__ SChunk sv_buf[NBUF];
    __shared__ ChunkLists lists;
    __shared__ uint32_t msk_buf[NBUF][CH];
    __shared__ float4 wbox[16];
    __shared__ float Fs[9];
    constexpr bool CONE = GM == GM_CONE;
    const TileCtx c = tile_ctx<GM>(g, tile);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr bool HALF = HalfBlocks<GM>::value;
    const int hw = HALF ? threadIdx.x >> 4 : w;   // this lane's lists
    if (threadIdx.x < 9) Fs[threadIdx.x] = __ldg(g.frames + 9 * (size_t)c.view + threadIdx.x);
    warp_box<HALF>(c, wbox);
    __syncthreads();
    float F[9];
#pragma unroll
    for (int i = 0; i < 9; i++) F[i] = Fs[i];
    const float u = __ldg(g.utab + min(c.col, g.n_cols - 1));
    const float v = __ldg(g.vtab + min(c.row, g.n_rows - 1)) + c.zoff;
    const float kap = GM == GM_PET3D ? pet3d_slope(g, c.dz, u) : 0.0f;
    const float L = CONE ? sqrtf(u * u + v * v + g.dsd * g.dsd)
                  : GM == GM_PET3D ? sqrtf(1.0f + kap * kap) : 1.0f;
    const uint2 rg = ranges[tile];
    float acc_vs = 0.0f, acc_gen = 0.0f;
    // time of flight (parallel rays, Gaussian kernel): one sum per bin
    float acc_t[TOF ? TOF_MAX : 1];
#pragma unroll
    for (int q = 0; q < (TOF ? TOF_MAX : 1); q++) acc_t[q] = 0.0f;
    unsigned n_eval = 0, n_kept = 0;
    // chunk c takes list entries c, c + nch, c + 2 nch, ...: the lists are
    // ordered by footprint position, and interleaving spreads every chunk
    // over the whole tile, which keeps the warps' shares of it even
    const uint32_t nlist = rg.y - rg.x;
    const uint32_t nch = (nlist + CH - 1) / CH;
    for (uint32_t ch = 0; ch < nch; ch++) {
        const int cnt = (int)((nlist - ch + nch - 1) / nch);
        const SChunk &sv = sv_buf[ch % NBUF];
        uint32_t *msk = msk_buf[ch % NBUF];
        prep_chunk<GM, KER, TOF>(g, F, gids, rg.x + ch, nch, cnt, rec, crec, &sv_buf[ch % NBUF], wbox, nw, msk,
                                 c.kap0, c.kap1);
        // every thread has prepared this chunk and (with two buffers) left the
        // previous one, whose buffer the next chunk's preparation reuses
        __syncthreads();
        int nvs, ngen;
        build_lists<HALF>(cnt, msk, lists, w, lane, nvs, ngen);
        int k = 0;
        if (TOF) {
            for (; k < nvs; k++) {
                const SRec r = sv[lists.vs[hw][k]];
                float a0;
                const float v0 = vs_value<GM, KER>(r, u, v, kap, a0);
                if (STATS) n_kept += vs_keep<KER>(a0);
                if (!vs_keep<KER>(a0)) continue;
                const float ts = r.c2.x + r.c2.y * (u - r.c0.x) + r.c2.z * (v - r.c0.y) - g.tof_t0;
                const float vn = v0 * r.c1.z;
#pragma unroll
                for (int b = 0; b < TOF_MAX; b++) {
                    if (b >= g.n_tof) break;
                    const float x = ts - (float)b * g.tof_h;
                    acc_t[b] = fmaf(vn, ex2_approx(r.c1.y * x * x), acc_t[b]);
                }
            }
        }
        for (; k + 1 < nvs; k += 2) {
            const int j0 = lists.vs[hw][k], j1 = lists.vs[hw][k + 1];
            float a0, a1;
            const float v0 = vs_value<GM, KER>(sv[j0], u, v, kap, a0);
            const float v1 = vs_value<GM, KER>(sv[j1], u, v, kap, a1);
            acc_vs += vs_keep<KER>(a0) ? v0 : 0.0f;
            acc_vs += vs_keep<KER>(a1) ? v1 : 0.0f;
            if (STATS) n_kept += vs_keep<KER>(a0) + vs_keep<KER>(a1);
        }
        if (k < nvs) {
            float a0;
            const float v0 = vs_value<GM, KER>(sv[lists.vs[hw][k]], u, v, kap, a0);
            acc_vs += vs_keep<KER>(a0) ? v0 : 0.0f;
            if (STATS) n_kept += vs_keep<KER>(a0);
        }
        if (ngen > 0) {
            const Ray ray = make_ray<GM>(g, F, u, v, kap);
            for (int k2 = 0; k2 < ngen; k2++) {
                const GRec r = load_grec(rec, sv.gid[lists.gen[hw][k2]]);
                PairGeo q;
                pair_geo(ray, r, q);
                if (STATS) n_kept += q.m <= PAIR_CUT2;
                if (TOF) {
                    if (q.m <= PAIR_CUT2) {
#pragma unroll
                        for (int b = 0; b < TOF_MAX; b++) {
                            if (b >= g.n_tof) break;
                            acc_t[b] += general_value<KER>(q, r.g0.w, g.tof_t0 + (float)b * g.tof_h, g.tof_tau);
                        }
                    }
                    continue;
                }
                const float val = general_value<KER>(q, r.g0.w);
                acc_gen += q.m <= PAIR_CUT2 ? val : 0.0f;
            }
        }
        if (STATS) n_eval += nvs + ngen;
        if (NBUF == 1) __syncthreads();
    }
    if (TOF) {
        if (c.valid) {
#pragma unroll
            for (int b = 0; b < TOF_MAX; b++) {
                if (b >= g.n_tof) break;
                out[c.out_idx + (long long)b * g.stride_tof] = c.live ? acc_t[b] : 0.0f;
            }
        }
    } else if (c.valid) {
        out[c.out_idx] = c.live ? acc_gen + L * acc_vs : 0.0f;
    }
    if (STATS) {
        unsigned long long e = c.live ? n_eval : 0, kk = c.live ? n_kept : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            kk += __shfl_xor_sync(0xffffffffu, kk, o);
        }
        if (lane == 0) {
            atomicAdd(&stats->pairs_eval, e);
            atomicAdd(&stats->pairs_kept, kk);
        }
    }
}

template <int GM, bool STATS, int KER>
__global__ void __launch_bounds__(256, 4) k_forward(DevGeom g, const float4 *__restrict__ rec,
                                                    const float4 *__restrict__ crec,
                                                    const uint32_t *__restrict__ gids,
                                                    const uint2 *__restrict__ ranges,
                                                    float *__restrict__ out, Stats *stats)
{
    forward_tile<GM, STATS, KER>(g, blockIdx.x, rec, crec, gids, ranges, out, stats);
}

// time-of-flight sinograms (PET ring, Gaussian kernel): one sum per bin per ray
template <bool STATS>
__global__ void __launch_bounds__(256, 2) k_forward_tof(DevGeom g, const float4 *__restrict__ rec,
                                                        const float4 *__restrict__ crec,
                                                        const uint32_t *__restrict__ gids,
                                                        const uint2 *__restrict__ ranges,
                                                        float *__restrict__ out, Stats *stats)
{
    forward_tile<GM_PARALLEL, STATS, 0, true>(g, blockIdx.x, rec, crec, gids, ranges, out, stats);
}

__device__ __forceinline__ void cross_acc(const float *a, const float *b, float s, float *o)
{
    o[0] += s * (a[1] * b[2] - a[2] * b[1]);
    o[1] += s * (a[2] * b[0] - a[0] * b[2]);
    o[2] += s * (a[0] * b[1] - a[1] * b[0]);
}

// Gradient w.r.t. (mu, rho, G_P, G_S) of one Gaussian from its view-space
// moments s[] summed over the tile's rays:
//   cone:  s = [SQ_u, SQ_v, SQ_uu, SQ_uv, SQ_vv, SA, SA_u, SA_v, SA_uu, SA_uv, SA_vv, Sw]
//   par.:  s = [SQ_u, SQ_v, SQ_uu, SQ_uv, SQ_vv, SA, Sw]
// where SQ_x = sum (dL/dQ / alpha) x, SA_x = sum (dL/dA / alpha) x (x a
// monomial in du, dv), Sw = sum dL/dI |d~| A^-1/2 e^{-m/2} and
// alpha = rho sqrt(2 pi).  With c = du g_u + dv g_v and d~ = d~0 + (du, dv, 0):
//   dL/dS'  = sum dL/dQ c c^T
//   dL/dP'  = sum dL/dA d~ d~^T
//   dL/dmu' = -2 sum dL/dQ (S' c) x d~      (Q = c^T S' c, c = d~ x (S - mu'))
//   dL/drho = sqrt(2 pi) Sw
// out16 = (dmu[3], drho, G_P[6], G_S[6]) in world coordinates.
// tof4 (nullable; parallel rays with time of flight): the moments of the
// TOF weight's derivatives (see adjoint_tile), added to dL/dmu' and dL/dP'.
template <int GM, int KER>
__device__ __forceinline__ void view_chain(const DevGeom &g, const float *F, const float4 *rec,
                                           uint32_t gid, const float *s, float *out16,
                                           const float *tof4 = nullptr)
{
    constexpr bool CONE = GM == GM_CONE;
    const float4 *r = rec + REC_F4 * (size_t)gid;
    const float4 r0 = __ldg(r), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
    const float Sh[6] = { r2.z, r2.w, r3.x, r3.y, r3.z, r3.w };
    const float m[3] = { r0.x, r0.y, r0.z };
    const float alpha = r0.w * Kern<KER>::FAC;
    const AxFrame fr = ax_frame(F);
    float Sf[6];
    to_frame_ax(Sh, fr, Sf);
    const float mu_u = m[0] * fr.a + m[1] * fr.b;
    const float mu_v = m[2];
    const float mu_w = m[0] * fr.p + m[1] * fr.q;
    const float SQu = alpha * s[0], SQv = alpha * s[1], SQuu = alpha * s[2], SQuv = alpha * s[3],
                SQvv = alpha * s[4];
    float gu[3], gv[3], d0[3], GPf[6], GSf[6];
    float Sw;
    if (CONE) {
        const float D = mu_w + g.dso;
        const float u0 = g.dsd * mu_u / D, v0 = g.dsd * mu_v / D;
        gu[0] = 0.0f; gu[1] = D; gu[2] = -mu_v;
        gv[0] = -D; gv[1] = 0.0f; gv[2] = mu_u;
        d0[0] = u0; d0[1] = v0; d0[2] = g.dsd;
        const float SA = alpha * s[5], SAu = alpha * s[6], SAv = alpha * s[7], SAuu = alpha * s[8],
                    SAuv = alpha * s[9], SAvv = alpha * s[10];
        Sw = s[11];
        // dL/dP' = SA d0 d0^T + (d0 m^T + m d0^T) + N,  m = (SAu, SAv, 0)
        GPf[0] = SA * d0[0] * d0[0] + 2.0f * d0[0] * SAu + SAuu;
        GPf[1] = SA * d0[0] * d0[1] + d0[0] * SAv + SAu * d0[1] + SAuv;
        GPf[2] = SA * d0[0] * d0[2] + SAu * d0[2];
        GPf[3] = SA * d0[1] * d0[1] + 2.0f * d0[1] * SAv + SAvv;
        GPf[4] = SA * d0[1] * d0[2] + SAv * d0[2];
        GPf[5] = SA * d0[2] * d0[2];
    } else {
        // c = du e_v - dv e_u: "g_u" = e_v, "g_v" = -e_u (frame coordinates), d~ = e_w
        gu[0] = 0.0f; gu[1] = 1.0f; gu[2] = 0.0f;
        gv[0] = -1.0f; gv[1] = 0.0f; gv[2] = 0.0f;
        d0[0] = 0.0f; d0[1] = 0.0f; d0[2] = 1.0f;
        Sw = s[6];
        GPf[0] = GPf[1] = GPf[2] = GPf[3] = GPf[4] = 0.0f;
        GPf[5] = alpha * s[5];
    }
    float cu[3], cv[3];   // S' g_u, S' g_v
    cu[0] = Sf[0] * gu[0] + Sf[1] * gu[1] + Sf[2] * gu[2];
    cu[1] = Sf[1] * gu[0] + Sf[3] * gu[1] + Sf[4] * gu[2];
    cu[2] = Sf[2] * gu[0] + Sf[4] * gu[1] + Sf[5] * gu[2];
    cv[0] = Sf[0] * gv[0] + Sf[1] * gv[1] + Sf[2] * gv[2];
    cv[1] = Sf[1] * gv[0] + Sf[3] * gv[1] + Sf[4] * gv[2];
    cv[2] = Sf[2] * gv[0] + Sf[4] * gv[1] + Sf[5] * gv[2];
    {
        const int ia[6] = { 0, 0, 0, 1, 1, 2 }, ib[6] = { 0, 1, 2, 1, 2, 2 };
#pragma unroll
        for (int e = 0; e < 6; e++) {
            const int a = ia[e], b = ib[e];
            GSf[e] = SQuu * gu[a] * gu[b] + SQuv * (gu[a] * gv[b] + gv[a] * gu[b]) + SQvv * gv[a] * gv[b];
        }
    }
    // T = sum dL/dQ (S'c) x d~ = cu x d0 SQu + cv x d0 SQv
    //     + cu x e_u SQuu + (cu x e_v + cv x e_u) SQuv + cv x e_v SQvv
    // (the last three only for the cone: parallel rays keep d~ = e_w)
    float T[3] = { 0.0f, 0.0f, 0.0f };
    cross_acc(cu, d0, SQu, T);
    cross_acc(cv, d0, SQv, T);
    if (CONE) {
        const float eU[3] = { 1.0f, 0.0f, 0.0f }, eV[3] = { 0.0f, 1.0f, 0.0f };
        cross_acc(cu, eU, SQuu, T);
        cross_acc(cu, eV, SQuv, T);
        cross_acc(cv, eU, SQuv, T);
        cross_acc(cv, eV, SQvv, T);
    }
    float dmuf[3] = { -2.0f * T[0], -2.0f * T[1], -2.0f * T[2] };
    if (!CONE && tof4) {
        // the TOF weight W(t*, s^2): t* = mu_w + k_u du + k_v dv with
        // k_u = -P'_uw / P'_ww, k_v = -P'_vw / P'_ww, s^2 = 1/P'_ww + sigma_T^2.
        // tof4 = alpha-free sums of val dW/dt* (1, du, dv) and val dW/ds^2.
        const float4 r1 = __ldg(rec + REC_F4 * (size_t)gid + 1), r2 = __ldg(rec + REC_F4 * (size_t)gid + 2);
        const float P[6] = { r1.x, r1.y, r1.z, r1.w, r2.x, r2.y };
        float Pf[6];
        to_frame_ax(P, fr, Pf);
        const float ipw = 1.0f / Pf[5];
        const float ku = -Pf[2] * ipw, kv = -Pf[4] * ipw;
        const float T0 = alpha * tof4[0], Tu = alpha * tof4[1], Tv = alpha * tof4[2], S0 = alpha * tof4[3];
        dmuf[0] -= ku * T0;        // du = u - mu_u: dt*/dmu_u = -k_u
        dmuf[1] -= kv * T0;
        dmuf[2] += T0;
        // symmetric-entry gradients (the full matrix holds P'_uw twice)
        GPf[2] -= 0.5f * Tu * ipw;
        GPf[4] -= 0.5f * Tv * ipw;
        GPf[5] -= (ku * Tu + kv * Tv) * ipw + S0 * ipw * ipw;
    }
    out16[0] = dmuf[0] * fr.a + dmuf[2] * fr.p;
    out16[1] = dmuf[0] * fr.b + dmuf[2] * fr.q;
    out16[2] = dmuf[1];
    out16[3] = Kern<KER>::FAC * Sw;
    from_frame_ax(GPf, fr, out16 + 4);
    from_frame_ax(GSf, fr, out16 + 10);
}

// Gradient of one Gaussian from its 3-D PET view-space moments, summed over
// the tile's LORs (d~ = e_w + kappa e_v, c = d~ x (o - mu') = (-v~, du,
// -kappa du), see prep_record), in the normalised variables of the record
// (A_n = A / P'_ww, Q_n = Q / P'_ww; h = -dL/dQ_n / alpha', gA = dL/dA_n /
// alpha', w = dL/dI |d~| A_n^-1/2 K(m), alpha' = alpha / sqrt(P'_ww)):
//   s = [h v~^2, h v~ du, h kappa v~ du, h du^2, h kappa du^2, h kappa^2 du^2,
//        h v~, h v~ kappa, h du, h du kappa, h du kappa^2,
//        gA, gA kappa, gA kappa^2, w]
// With dL/dQ = -alpha P'_ww^-3/2 h and dL/dA = alpha P'_ww^-3/2 gA:
//   dL/dS'  = sum dL/dQ c c^T,   dL/dP' = sum dL/dA d~ d~^T,
//   dL/dmu' = -2 sum dL/dQ (S'c) x d~,  dL/drho = FAC P'_ww^-1/2 sum w.
template <int KER>
__device__ __forceinline__ void pet3d_chain(const float *F, const float4 *rec, uint32_t gid,
                                            const float *s, float *out16)
{
    const float4 *r = rec + REC_F4 * (size_t)gid;
    const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
    const float P[6] = { r1.x, r1.y, r1.z, r1.w, r2.x, r2.y };
    const float Sh[6] = { r2.z, r2.w, r3.x, r3.y, r3.z, r3.w };
    const AxFrame fr = ax_frame(F);
    float Sf[6];
    to_frame_ax(Sh, fr, Sf);
    const float Pww = (P[0] * fr.p + P[1] * fr.q) * fr.p + (P[1] * fr.p + P[3] * fr.q) * fr.q;
    const float ipw = 1.0f / Pww;
    const float aw = sqrtf(ipw);
    const float ah = r0.w * Kern<KER>::FAC * aw * ipw;
    float GSf[6], GPf[6];
    GSf[0] = -ah * s[0];   // uu: c_u c_u = v~^2
    GSf[1] = ah * s[1];    // uv: -v~ du
    GSf[2] = -ah * s[2];   // uw: kappa v~ du
    GSf[3] = -ah * s[3];   // vv: du^2
    GSf[4] = ah * s[4];    // vw: -kappa du^2
    GSf[5] = -ah * s[5];   // ww: kappa^2 du^2
    GPf[0] = GPf[1] = GPf[2] = 0.0f;
    GPf[3] = ah * s[13];   // vv: kappa^2
    GPf[4] = ah * s[12];   // vw: kappa
    GPf[5] = ah * s[11];   // ww: 1
    // columns of S' and (S' c) x d~ =
    //   -v~ (S'e_u x e_w) - v~ kappa (S'e_u x e_v) + du (S'e_v x e_w)
    //   + du kappa (S'e_v x e_v - S'e_w x e_w) - du kappa^2 (S'e_w x e_v)
    // with x x e_u = (0, x_w, -x_v), x x e_v = (-x_w, 0, x_u), x x e_w = (x_v, -x_u, 0)
    const float cu[3] = { Sf[0], Sf[1], Sf[2] }, cv[3] = { Sf[1], Sf[3], Sf[4] }, cw[3] = { Sf[2], Sf[4], Sf[5] };
    const float M0 = s[6], M1 = s[7], M2 = s[8], M3 = s[9], M4 = s[10];
    float T[3];
    T[0] = -M0 * cu[1] - M1 * (-cu[2]) + M2 * cv[1] + M3 * (-cv[2] - cw[1]) - M4 * (-cw[2]);
    T[1] = -M0 * (-cu[0]) + M2 * (-cv[0]) + M3 * cw[0];
    T[2] = -M1 * cu[0] + M3 * cv[0] - M4 * cw[0];
    const float dmuf[3] = { 2.0f * ah * T[0], 2.0f * ah * T[1], 2.0f * ah * T[2] };
    out16[0] = dmuf[0] * fr.a + dmuf[2] * fr.p;
    out16[1] = dmuf[0] * fr.b + dmuf[2] * fr.q;
    out16[2] = dmuf[1];
    out16[3] = Kern<KER>::FAC * aw * s[14];
    from_frame_ax(GPf, fr, out16 + 4);
    from_frame_ax(GSf, fr, out16 + 10);
}

// Adjoint, one Gaussian per thread.  A CTA takes a tile: it stages the
// tile's dL/dI (times |d~| for cone beam) and pixel coordinates in shared
// memory, then every thread walks the tile's rays for one Gaussian of the
// list at a time (all lanes of a warp read the same ray: broadcasts), keeping
// that Gaussian's view-space moments in registers -- no cross-thread
// reduction -- and finishes with the parameter chain and one set of vector
// atomics per (Gaussian, tile).  The tile list is ordered by footprint
// position, so the 32 Gaussians of a warp sit close together: rows and
// 8-column groups that none of their boxes touches are skipped.  Within a row
// the Q and A quadratics are evaluated in Horner form in du with the dv terms
// hoisted.  For 3-D PET the LOR slope kappa varies from column to column:
// the moments carry its powers (pet3d_chain).
// Time of flight, general path: the world-space form of every pair of the
// Gaussian's box, once per bin, added to val.  Out of line: it is rarely
// taken, and inlined it crowds the view-space loop out of the instruction
// cache.
template <int KER>
__device__ __noinline__ void tof_general_box(const DevGeom &g, const float *F, const float *su, const float *svr,
                                             const float *sgl, int tw, const VRec &r, int ilo, int ihi, int jlo,
                                             int jhi, float *val)
{
    float Fl[9];
    for (int q = 0; q < 9; q++) Fl[q] = F[q];
    for (int j = jlo; j <= jhi; j++) {
        const float vj = svr[j];
        for (int i = ilo; i <= ihi; i++) {
            const Ray ray = make_ray<GM_PARALLEL>(g, Fl, su[i], vj, 0.0f);
            PairGeo q;
            pair_geo(ray, r, q);
            if (!(q.m <= PAIR_CUT2)) continue;
            for (int b = 0; b < g.n_tof; b++) {
                const float gw = sgl[b * 256 + j * tw + i];
                if (gw == 0.0f) continue;
                float pv[NG];
                general_grad<KER>(ray, q, r.g0.w, gw, pv, g.tof_t0 + (float)b * g.tof_h, g.tof_tau);
                for (int qq = 0; qq < NG; qq++) val[qq] += pv[qq];
            }
        }
    }
}

template <int GM, int TW, int KER, bool TOF = false>
__device__ __forceinline__ void adjoint_tile(const DevGeom &g, uint32_t tile,
                                             const float4 *__restrict__ rec,
                                             const float4 *__restrict__ crec,
                                             const uint32_t *__restrict__ gids,
                                             const uint2 *__restrict__ ranges,
                                             const float *__restrict__ dLdI,
                                             float4 *__restrict__ grad)
{
    constexpr bool CONE = GM == GM_CONE, P3 = GM == GM_PET3D;
    // dL/dI |d~| of the tile's rays, row-major (0 outside the detector); with
    // time of flight one such tile per bin (bin b at b * 256)
    __shared__ float sgl[TOF ? TOF_MAX * 256 : 256];
    __shared__ float su[32], svr[32];
    __shared__ float skap[P3 ? 32 : 1];   // 3-D PET: LOR slope of every column
    __shared__ float Fs[9];
    const int T = g.tiles_x * g.tiles_y;
    const int vl = (int)(tile / (uint32_t)T);
    const int tin = (int)tile - vl * T;
    const int ty = tin / g.tiles_x, tx = tin - ty * g.tiles_x;
    const int view = g.v0 + vl;
    const int TH = g.tile_h;
    const int c0 = tx * TW, r0 = ty * TH;
    float zoff = 0.0f, dz = 0.0f, kap0 = 0.0f, kap1 = 0.0f;
    int rows = g.n_rows;
    if (P3) {
        pet3d_view(g, view, zoff, dz, rows);
        pet3d_slopes(g, dz, c0, min(c0 + TW - 1, g.n_cols - 1), kap0, kap1);
    }
    if (threadIdx.x < 9) Fs[threadIdx.x] = __ldg(g.frames + 9 * (size_t)view + threadIdx.x);
    if (threadIdx.x < TW) {
        su[threadIdx.x] = __ldg(g.utab + min(c0 + (int)threadIdx.x, g.n_cols - 1));
        if (P3) skap[threadIdx.x] = pet3d_slope(g, dz, su[threadIdx.x]);
    }
    if (threadIdx.x < TH) svr[threadIdx.x] = __ldg(g.vtab + min(r0 + (int)threadIdx.x, g.n_rows - 1)) + zoff;
    for (int r = threadIdx.x; r < TW * TH; r += blockDim.x) {
        const int col = c0 + r % TW, row = r0 + r / TW;
        if (TOF) {
            const bool in = col < g.n_cols && row < rows;
            const long long idx = (long long)view * g.stride_view + (long long)row * g.stride_row + col;
            for (int b = 0; b < g.n_tof; b++) sgl[b * 256 + r] = in ? __ldg(dLdI + idx + b * g.stride_tof) : 0.0f;
            continue;
        }
        float gl = 0.0f;
        if (col < g.n_cols && row < rows) {
            const long long idx = (long long)view * g.stride_view + (long long)row * g.stride_row + col;
            gl = __ldg(dLdI + idx);
            if (CONE) {
                const float u = __ldg(g.utab + col), v = __ldg(g.vtab + row);
                gl *= sqrtf(u * u + v * v + g.dsd * g.dsd);
            }
            if (P3) {
                const float kap = pet3d_slope(g, dz, __ldg(g.utab + col));
                gl *= sqrtf(1.0f + kap * kap);
            }
        }
        sgl[r] = gl;
    }
    __syncthreads();
    float F[9];
#pragma unroll
    for (int i = 0; i < 9; i++) F[i] = Fs[i];
    const uint2 rg = ranges[tile];
    // every lane of a warp runs the same number of rounds (inactive lanes idle)
    const uint32_t n = rg.y - rg.x;
    const uint32_t rounds = (n + blockDim.x - 1) / blockDim.x;
    for (uint32_t rd = 0; rd < rounds; rd++) {
        const uint32_t k = rg.x + rd * blockDim.x + threadIdx.x;
        const bool active = k < rg.y;
        VRec r;
        uint32_t gid = 0;
        if (active) {
            gid = __ldg(gids + k);
            prep_record<GM, KER>(g, F, gid, rec, crec, r, kap0, kap1);
        } else {
            r.bb = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
            r.g2 = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
        }
        const float4 bb = r.bb;
        const bool vs = r.g2.w != 0.0f;
        // the Gaussian's box in tile pixels (rows jlo..jhi, columns ilo..ihi)
        int jlo = TH, jhi = -1, ilo = TW, ihi = -1;
        for (int j = 0; j < TH; j++) {
            const bool in = svr[j] >= bb.z && svr[j] <= bb.w;
            jlo = in && j < jlo ? j : jlo;
            jhi = in ? j : jhi;
        }
#pragma unroll
        for (int i = 0; i < TW; i++) {
            const bool in = su[i] >= bb.x && su[i] <= bb.y;
            ilo = in && i < ilo ? i : ilo;
            ihi = in ? i : ihi;
        }
        // 8-column groups of the tile the box touches (3-D PET), and 4-column
        // groups (the other geometries)
        uint32_t groups = 0, groups4 = 0;
#pragma unroll
        for (int c8 = 0; c8 < TW / 8; c8++) groups |= (uint32_t)(ilo <= 8 * c8 + 7 && ihi >= 8 * c8) << c8;
        if (ilo <= ihi) groups4 = (2u << (ihi >> 2)) - (1u << (ilo >> 2));
        float o[16];
        bool any = false;
        if (!P3 && __any_sync(0xffffffffu, active && vs)) {
            // view-space moments (see view_chain for their meaning)
            const float u0 = r.c0.x, v0 = r.c0.y, kMuu = r.c0.z, kMuv2 = r.c0.w, kMvv = r.c1.x;
            float s[NV_CONE];
#pragma unroll
            for (int q = 0; q < NV_CONE; q++) s[q] = 0.0f;
            // time of flight (parallel rays): a pair's value times the bin's
            // weight W_k = N(t* - t_k; 0, s^2), s^2 = 1/A + sigma_T^2.  The
            // value's gradient takes the view-space moments with the pair's
            // weight G = sum_k g_k W_k in place of dL/dI; the weights'
            // gradients take four more sums, of val dW/dt* (1, du, dv) and of
            // val dW/ds^2 (per unit alpha), chained in view_chain.
            float tof4[4] = { 0.0f, 0.0f, 0.0f, 0.0f };
            float ns = 0.0f, is2 = 0.0f;
            if (TOF) {
                const float s2 = r.t4.w + g.tof_s2;
                is2 = 1.0f / s2;
                ns = Kern<0>::QSCALE * is2;
            }
            const float nrm = TOF ? rsqrtf(2.0f * 3.14159265358979324f / is2) : 0.0f;
            for (int j = 0; j < TH; j++) {
                const float vj = svr[j];
                const bool rowin = active && vs && j >= jlo && j <= jhi;
                // rows and 4-column groups that no Gaussian of the warp touches
                // are skipped (the lists are ordered by footprint position, so
                // a warp's Gaussians sit close together in the tile)
                const uint32_t need = __reduce_or_sync(0xffffffffu, rowin ? groups4 : 0u);
                if (need == 0u || !rowin) continue;
                const float dv = vj - v0, dv2 = dv * dv;
                const float a1 = kMuv2 * dv, a0 = kMvv * dv2;
                float b2 = 0.0f, b1 = 0.0f, b0 = 0.0f, iAc = 0.0f, rAc = 0.0f;
                if (CONE) {
                    b2 = r.c2.x;
                    b1 = r.c1.z + r.c2.y * dv;
                    b0 = r.c1.y + r.c1.w * dv + r.c2.z * dv2;
                } else {
                    iAc = r.c1.y;
                    rAc = r.c1.z;
                }
                float H0 = 0.0f, H1 = 0.0f, H2 = 0.0f, G0 = 0.0f, G1 = 0.0f, G2 = 0.0f, Sw = 0.0f;
                float T0r = 0.0f, Tur = 0.0f, S0r = 0.0f;
                const float *gl_row = sgl + j * TW;
                auto pixel = [&](int i) {
                    const float du = su[i] - u0;
                    const float qv = (kMuu * du + a1) * du + a0;
                    float rA, iA, arg;
                    if (CONE) {
                        const float A = (b2 * du + b1) * du + b0;
                        rA = rsqrt_approx(A);
                        iA = rA * rA;
                        arg = qv * iA;
                    } else {
                        rA = rAc;
                        iA = iAc;
                        arg = qv;
                    }
                    float wv, h, gA;
                    if (TOF) {
                        // the bins' weights at this pair's t*, and their sums
                        const float ts = r.t4.x + r.t4.y * du + r.t4.z * dv - g.tof_t0;
                        float Ge = 0.0f, D1 = 0.0f, D2 = 0.0f;
                        for (int b = 0; b < g.n_tof; b++) {
                            const float x = ts - (float)b * g.tof_h, x2 = x * x;
                            const float gw = sgl[b * 256 + j * TW + i] * ex2_approx(ns * x2);
                            Ge += gw;
                            D1 = fmaf(gw, x, D1);
                            D2 = fmaf(gw, x2, D2);
                        }
                        Ge *= nrm;
                        D1 *= -nrm * is2;                                   // sum g_k dW_k/dt*
                        D2 = 0.5f * is2 * (nrm * is2 * D2 - Ge);           // sum g_k dW_k/ds^2
                        const bool keep = arg >= CUT_ARG;
                        const float vu = keep ? rA * ex2_approx(arg) : 0.0f;   // value per unit alpha
                        wv = Ge * vu;
                        h = 0.5f * wv * iA;
                        gA = h * (arg * M_PER_ARG - 1.0f);
                        const float v1 = vu * D1;
                        T0r += v1;
                        Tur = fmaf(v1, du, Tur);
                        S0r = fmaf(vu, D2, S0r);
                    } else if (KER == 1) {
                        // f = alpha A^-1/2 c^3/2, c = 1 - Q/(kappa^2 A): -dL/dQ / alpha =
                        // 1.5 w rA iA sqrt(c) / kappa^2, dL/dA / alpha = w rA iA sqrt(c) (1.5 - 2c)
                        const float c = 1.0f + arg;
                        const float sc = c > 0.0f ? sqrt_approx(c) : 0.0f;
                        const float t = gl_row[i] * rA * sc;
                        wv = t * c;
                        h = (1.5f / Kern<1>::KAPPA2) * t * iA;
                        gA = t * iA * (1.5f - 2.0f * c);
                    } else {
                        wv = arg >= CUT_ARG ? gl_row[i] * rA * ex2_approx(arg) : 0.0f;
                        h = 0.5f * wv * iA;
                        gA = h * (arg * M_PER_ARG - 1.0f);
                    }
                    const float hd = h * du, gd = gA * du;
                    H0 += h; H1 += hd; H2 += hd * du;
                    G0 += gA; G1 += gd; G2 += gd * du;
                    Sw += wv;
                };
                if (!TOF) {
                    // 4-column groups that some Gaussian of the warp needs
#pragma unroll
                    for (int c4 = 0; c4 < TW / 4; c4++) {
                        if (!((need >> c4) & 1u)) continue;
#pragma unroll
                        for (int i = 4 * c4; i < 4 * c4 + 4; i++) pixel(i);
                    }
                } else {
                    // time of flight (parallel rays): a pixel costs a loop over
                    // the bins, so each lane visits only its row's chord of the
                    // footprint, arg(du) = kMuu du^2 + a1 du + a0 >= the cut
                    // (kMuu < 0), widened to whole columns on either side (each
                    // pixel is still tested); uniformly spaced columns only,
                    // else the box.  (Without time of flight the lanes' uneven
                    // chords cost more in divergence than they save.)
                    int ia = ilo, ib = ihi;
                    const float thr = KER == 1 ? -1.0f : CUT_ARG;
                    if (g.uinv != 0.0f && kMuu < 0.0f && ia <= ib) {
                        const float cc = a0 - thr;
                        const float D = a1 * a1 - 4.0f * kMuu * cc;
                        if (D < 0.0f) {
                            ib = ia - 1;
                        } else {
                            const float sq = sqrtf(D), i2a = 0.5f / kMuu;
                            const float d1 = (-a1 + sq) * i2a, d2 = (-a1 - sq) * i2a;   // d1 <= d2
                            const float x1 = (u0 + d1 - su[0]) * g.uinv, x2 = (u0 + d2 - su[0]) * g.uinv;
                            const int ja = (int)floorf(fminf(fmaxf(x1, (float)ia), (float)ib + 1.0f));
                            const int jb = (int)ceilf(fmaxf(fminf(x2, (float)ib), (float)ia - 1.0f));
                            ia = max(ia, ja);
                            ib = min(ib, jb);
                        }
                    }
                    for (int i = ia; i <= ib; i++) pixel(i);
                }
                // dL/dQ = -h:  SQ_x = -sum h x ;  SA_x = sum gA x
                s[0] -= H1;
                s[1] -= H0 * dv;
                s[2] -= H2;
                s[3] -= H1 * dv;
                s[4] -= H0 * dv2;
                s[5] += G0;
                s[6] += G1;
                s[7] += G0 * dv;
                s[8] += G2;
                s[9] += G1 * dv;
                s[10] += G0 * dv2;
                s[11] += Sw;
                if (TOF) {
                    tof4[0] += T0r;
                    tof4[1] += Tur;
                    tof4[2] = fmaf(T0r, dv, tof4[2]);
                    tof4[3] += S0r;
                }
            }
            if (active && vs) {
                if (!CONE) s[6] = s[11];   // parallel layout: [SQ.. (5), SA, Sw]
#pragma unroll
                for (int q = 0; q < NV_CONE; q++) any |= s[q] != 0.0f;
                if (TOF) any |= tof4[0] != 0.0f || tof4[1] != 0.0f || tof4[2] != 0.0f || tof4[3] != 0.0f;
                if (any) view_chain<GM, KER>(g, F, rec, gid, s, o, TOF ? tof4 : nullptr);
            }
        }
        if (P3 && __any_sync(0xffffffffu, active && vs)) {
            // columns outer: the LOR slope kappa is fixed along a column, so
            // the column's kappa terms are taken once and its rows need only
            // five kappa-free sums (h, h v~, h v~^2, gA, w), folded into the 15
            // moments with the column's du and kappa powers afterwards
            const float4 c0 = r.c0, c1 = r.c1, c2 = r.c2;
            float s[15];
#pragma unroll
            for (int q = 0; q < 15; q++) s[q] = 0.0f;
#pragma unroll 1
            for (int i = 0; i < TW; i++) {
                const bool colin = active && vs && i >= ilo && i <= ihi;
                if (!__any_sync(0xffffffffu, colin)) continue;
                // rows that any lane's box holds in this column
                const int rlo = __reduce_min_sync(0xffffffffu, colin ? jlo : TH);
                const int rhi = __reduce_max_sync(0xffffffffu, colin ? jhi : -1);
                if (!colin) continue;
                const float du = su[i] - c0.x, kap = skap[i];
                const float muu = fmaf(fmaf(c1.z, kap, c1.y), kap, c1.x);
                const float muv2 = fmaf(c2.x, kap, c1.w);
                const float rA = rsqrt_approx(fmaf(fmaf(c2.z, kap, c2.y), kap, 1.0f));
                const float iA = rA * rA;
                const float Kq = muu * du * du, Lq = muv2 * du;
                const float vt0 = fmaf(kap, c0.z, -c0.y);     // v~ = v + vt0
                float H0 = 0.0f, Hv = 0.0f, Hvv = 0.0f, G0 = 0.0f, W = 0.0f;
                for (int j = rlo; j <= rhi; j++) {
                    const float vt = svr[j] + vt0;
                    const float qv = fmaf(fmaf(c0.w, vt, Lq), vt, Kq);   // du (muu du + muv2 v~) + S_uu v~^2
                    const float arg = qv * iA;
                    const float gl = sgl[j * TW + i];
                    float wv, h, gA;
                    if (KER == 1) {
                        const float c = 1.0f + arg;
                        const float sc = c > 0.0f ? sqrt_approx(c) : 0.0f;
                        const float t = gl * rA * sc;
                        wv = t * c;
                        h = (1.5f / Kern<1>::KAPPA2) * t * iA;
                        gA = t * iA * (1.5f - 2.0f * c);
                    } else {
                        wv = arg >= CUT_ARG ? gl * rA * ex2_approx(arg) : 0.0f;
                        h = 0.5f * wv * iA;
                        gA = h * (arg * M_PER_ARG - 1.0f);
                    }
                    const float hv = h * vt;
                    H0 += h;
                    Hv += hv;
                    Hvv = fmaf(hv, vt, Hvv);
                    G0 += gA;
                    W += wv;
                }
                const float hd = H0 * du, hvd = Hv * du, kk = kap * kap;
                s[0] += Hvv;
                s[1] += hvd;
                s[2] = fmaf(kap, hvd, s[2]);
                s[3] = fmaf(hd, du, s[3]);
                s[4] = fmaf(kap * hd, du, s[4]);
                s[5] = fmaf(kk * hd, du, s[5]);
                s[6] += Hv;
                s[7] = fmaf(kap, Hv, s[7]);
                s[8] += hd;
                s[9] = fmaf(kap, hd, s[9]);
                s[10] = fmaf(kk, hd, s[10]);
                s[11] += G0;
                s[12] = fmaf(kap, G0, s[12]);
                s[13] = fmaf(kk, G0, s[13]);
                s[14] += W;
            }
            if (active && vs) {
#pragma unroll
                for (int q = 0; q < 15; q++) any |= s[q] != 0.0f;
                if (any) pet3d_chain<KER>(F, rec, gid, s, o);
            }
        }
        if (__any_sync(0xffffffffu, active && !vs)) {
            float val[NG];
#pragma unroll
            for (int q = 0; q < NG; q++) val[q] = 0.0f;
            if (active && !vs) {
                if (TOF) tof_general_box<KER>(g, Fs, su, svr, sgl, TW, r, ilo, ihi, jlo, jhi, val);
                for (int j = jlo; j <= (TOF ? -1 : jhi); j++) {
                    const float vj = svr[j];
                    for (int i = ilo; i <= ihi; i++) {
                        const float gw0 = sgl[j * TW + i];
                        if (gw0 == 0.0f) continue;
                        const float u = su[i];
                        const Ray ray = make_ray<GM>(g, F, u, vj, P3 ? skap[i] : 0.0f);
                        PairGeo q;
                        pair_geo(ray, r, q);
                        if (!(q.m <= PAIR_CUT2)) continue;
                        // sgl holds dL/dI |d~|; the general form wants dL/dI
                        const float gw = CONE ? gw0 * rsqrtf(u * u + vj * vj + g.dsd * g.dsd)
                                       : P3 ? gw0 * rsqrtf(1.0f + skap[i] * skap[i]) : gw0;
                        float pv[NG];
                        general_grad<KER>(ray, q, r.g0.w, gw, pv);
#pragma unroll
                        for (int qq = 0; qq < NG; qq++) val[qq] += pv[qq];
                    }
                }
#pragma unroll
                for (int q = 0; q < NG; q++) any |= val[q] != 0.0f;
                o[0] = val[0]; o[1] = val[1]; o[2] = val[2]; o[3] = val[9];
                o[4] = val[3]; o[5] = val[4]; o[6] = val[5]; o[7] = val[6];
                o[8] = val[7]; o[9] = val[8];
#pragma unroll
                for (int q = 10; q < 16; q++) o[q] = 0.0f;
            }
        }
        if (active && any) {
            float4 *gp = grad + GRAD_F4 * (size_t)gid;
            atomicAdd(gp, make_float4(o[0], o[1], o[2], o[3]));
            atomicAdd(gp + 1, make_float4(o[4], o[5], o[6], o[7]));
            atomicAdd(gp + 2, make_float4(o[8], o[9], o[10], o[11]));
            if (vs) atomicAdd(gp + 3, make_float4(o[12], o[13], o[14], o[15]));
        }
    }
}

template <int GM, int TW, int KER>
__global__ void __launch_bounds__(ADJ_BS) k_adjoint(DevGeom g, const float4 *__restrict__ rec,
                                                 const float4 *__restrict__ crec,
                                                 const uint32_t *__restrict__ gids,
                                                 const uint2 *__restrict__ ranges,
                                                 const float *__restrict__ dLdI,
                                                 float4 *__restrict__ grad)
{
    adjoint_tile<GM, TW, KER>(g, blockIdx.x, rec, crec, gids, ranges, dLdI, grad);
}

// time-of-flight sinograms (PET ring, Gaussian kernel)
template <int TW>
__global__ void __launch_bounds__(ADJ_BS) k_adjoint_tof(DevGeom g, const float4 *__restrict__ rec,
                                                     const float4 *__restrict__ crec,
                                                     const uint32_t *__restrict__ gids,
                                                     const uint2 *__restrict__ ranges,
                                                     const float *__restrict__ dLdI,
                                                     float4 *__restrict__ grad)
{
    adjoint_tile<GM_PARALLEL, TW, 0, true>(g, blockIdx.x, rec, crec, gids, ranges, dLdI, grad);
}

// Persistent forms over a batch of scans: every CTA takes (scan, tile) work
// items from an atomic counter until all are done.  Items are numbered scan
// by scan (ScanDesc::item_begin); the CTA finds its scan by binary search.
__device__ __forceinline__ bool next_item(const ScanDesc *d, int nscan, uint32_t total,
                                          uint32_t *queue, uint32_t &item, int &scan)
{
    __shared__ uint32_t s_item;
    __shared__ int s_scan;
    __syncthreads();   // the previous item is finished by every thread
    if (threadIdx.x == 0) {
        const uint32_t it = atomicAdd(queue, 1u);
        int lo = 0, hi = nscan - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].item_begin <= it) lo = mid; else hi = mid - 1;
        }
        s_item = it;
        s_scan = lo;
    }
    __syncthreads();
    item = s_item;
    scan = s_scan;
    return item < total;
}

template <bool CONE>
__global__ void __launch_bounds__(256, 4) k_forward_persistent(const ScanDesc *__restrict__ d,
                                                               int nscan, uint32_t total,
                                                               uint32_t *queue)
{
    uint32_t item;
    int scan;
    while (next_item(d, nscan, total, queue, item, scan)) {
        const ScanDesc &sd = d[scan];
        forward_tile<CONE ? GM_CONE : GM_PARALLEL, false, 0>(sd.g, item - sd.item_begin, sd.rec, sd.crec, sd.gids, sd.ranges,
                                  sd.out, nullptr);
    }
}

template <bool CONE, int TW>
__global__ void __launch_bounds__(ADJ_BS) k_adjoint_persistent(const ScanDesc *__restrict__ d, int nscan,
                                                              uint32_t total, uint32_t *queue)
{
    uint32_t item;
    int scan;
    while (next_item(d, nscan, total, queue, item, scan)) {
        const ScanDesc &sd = d[scan];
        adjoint_tile<CONE ? GM_CONE : GM_PARALLEL, TW, 0>(sd.g, item - sd.item_begin, sd.rec, sd.crec, sd.gids, sd.ranges,
                               sd.dLdI, sd.grad);
    }
}

}  // namespace

cudaError_t launch_forward_persistent(bool cone, const ScanDesc *d, int nscan, uint32_t total,
                                      uint32_t *queue, int tile_threads, int grid, cudaStream_t s)
{
    if (total == 0) return cudaSuccess;
    if (cone) k_forward_persistent<true><<<grid, tile_threads, 0, s>>>(d, nscan, total, queue);
    else k_forward_persistent<false><<<grid, tile_threads, 0, s>>>(d, nscan, total, queue);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_persistent(bool cone, int tile_w, const ScanDesc *d, int nscan,
                                      uint32_t total, uint32_t *queue, int grid, cudaStream_t s)
{
    if (total == 0) return cudaSuccess;
#define RGRT_ADJP(C, TW) k_adjoint_persistent<C, TW><<<grid, ADJ_BS, 0, s>>>(d, nscan, total, queue)
    if (cone) {
        if (tile_w == 8) RGRT_ADJP(true, 8);
        else if (tile_w == 16) RGRT_ADJP(true, 16);
        else RGRT_ADJP(true, 32);
    } else {
        if (tile_w == 8) RGRT_ADJP(false, 8);
        else if (tile_w == 16) RGRT_ADJP(false, 16);
        else RGRT_ADJP(false, 32);
    }
#undef RGRT_ADJP
    count_launches(1);
    return cudaGetLastError();
}

template <class K>
int grid_for(K kernel, int threads)
{
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    return nsm * (per < 1 ? 1 : per);
}

int persistent_grid(bool forward, bool cone, int tile_w, int tile_threads)
{
    if (forward)
        return cone ? grid_for(k_forward_persistent<true>, tile_threads)
                    : grid_for(k_forward_persistent<false>, tile_threads);
    if (cone)
        return tile_w == 8 ? grid_for(k_adjoint_persistent<true, 8>, ADJ_BS)
             : tile_w == 16 ? grid_for(k_adjoint_persistent<true, 16>, ADJ_BS)
                            : grid_for(k_adjoint_persistent<true, 32>, ADJ_BS);
    return tile_w == 8 ? grid_for(k_adjoint_persistent<false, 8>, ADJ_BS)
         : tile_w == 16 ? grid_for(k_adjoint_persistent<false, 16>, ADJ_BS)
                        : grid_for(k_adjoint_persistent<false, 32>, ADJ_BS);
}

cudaError_t launch_forward(const DevGeom &g, int nv, const float4 *rec, const float4 *crec,
                           const uint32_t *gids, const uint2 *ranges, float *out, Stats *stats,
                           int ker, cudaStream_t s)
{
    unsigned nt = (unsigned)nv * g.tiles_x * g.tiles_y;
    if (nt == 0) return cudaSuccess;
    int bs = g.tile_w * g.tile_h;
#define RGRT_FWD(M, S, K) k_forward<M, S, K><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, out, stats)
#define RGRT_FWD_K(M, K) { if (stats) RGRT_FWD(M, true, K); else RGRT_FWD(M, false, K); }
#define RGRT_FWD_M(K)                                  \
    if (g.kind == GM_CONE) RGRT_FWD_K(GM_CONE, K)      \
    else if (g.kind == GM_PET3D) RGRT_FWD_K(GM_PET3D, K) \
    else RGRT_FWD_K(GM_PARALLEL, K)
    if (g.n_tof > 0) {   // PET ring, Gaussian kernel (checked by the caller)
        if (stats) k_forward_tof<true><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, out, stats);
        else k_forward_tof<false><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, out, stats);
    } else if (ker == 1) { RGRT_FWD_M(1) } else { RGRT_FWD_M(0) }
#undef RGRT_FWD_M
#undef RGRT_FWD_K
#undef RGRT_FWD
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const DevGeom &g, int nv, const float4 *rec, const float4 *crec,
                           const uint32_t *gids, const uint2 *ranges, const float *dLdI,
                           float4 *grad, int ker, cudaStream_t s)
{
    unsigned nt = (unsigned)nv * g.tiles_x * g.tiles_y;
    if (nt == 0) return cudaSuccess;
    const int bs = ADJ_BS;
#define RGRT_ADJ(M, TW, K) k_adjoint<M, TW, K><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, dLdI, grad)
#define RGRT_ADJ_W(M, K)                                      \
    {                                                         \
        if (g.tile_w == 8) RGRT_ADJ(M, 8, K);                 \
        else if (g.tile_w == 16) RGRT_ADJ(M, 16, K);          \
        else RGRT_ADJ(M, 32, K);                              \
    }
#define RGRT_ADJ_K(K)                                         \
    if (g.kind == GM_CONE) RGRT_ADJ_W(GM_CONE, K)             \
    else if (g.kind == GM_PET3D) RGRT_ADJ_W(GM_PET3D, K)      \
    else RGRT_ADJ_W(GM_PARALLEL, K)
    if (g.n_tof > 0) {   // PET ring, Gaussian kernel (checked by the caller)
        if (g.tile_w == 8) k_adjoint_tof<8><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, dLdI, grad);
        else if (g.tile_w == 16) k_adjoint_tof<16><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, dLdI, grad);
        else k_adjoint_tof<32><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, dLdI, grad);
    } else if (ker == 1) { RGRT_ADJ_K(1) } else { RGRT_ADJ_K(0) }
#undef RGRT_ADJ_K
#undef RGRT_ADJ_W
#undef RGRT_ADJ
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rgrt
