// Record build (a0) and per-view culling (a2, first half).
//
// Everything that decides which tiles a Gaussian lands in is evaluated with
// explicit round-to-nearest binary32 intrinsics (__fmul_rn, __fadd_rn, ...),
// so no multiply-add is contracted and the result is fixed by the written
// operation order: that order is the culling specification, and the tile
// lists are reproducible bit for bit by any IEEE binary32 implementation of
// it.
#include "rgrt_internal.h"

namespace rgrt {
namespace {

__device__ __forceinline__ float M(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float A(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float S(float a, float b) { return __fsub_rn(a, b); }

// e^x: Cody-Waite reduction x = n ln2 + r, |r| <= ln2/2, and the degree-7
// Taylor polynomial of e^r in Horner form (truncation below 6e-9 relative).
__device__ __forceinline__ float exp_spec(float x)
{
    const float LOG2E = 0x1.715476p+0f;
    const float LN2_HI = 0x1.62e4p-1f;     // ln 2 truncated to 15 significant bits
    const float LN2_LO = 0x1.7f7d1cp-20f;  // ln 2 - LN2_HI
    float n = rintf(M(x, LOG2E));
    float r = S(S(x, M(n, LN2_HI)), M(n, LN2_LO));
    float p = 0x1.a01a02p-13f;
    p = A(M(p, r), 0x1.6c16c2p-10f);
    p = A(M(p, r), 0x1.111112p-7f);
    p = A(M(p, r), 0x1.555556p-5f);
    p = A(M(p, r), 0x1.555556p-3f);
    p = A(M(p, r), 0.5f);
    p = A(M(p, r), 1.0f);
    p = A(M(p, r), 1.0f);
    return ldexpf(p, (int)n);
}

__global__ void k_records(const float *__restrict__ mu, const float *__restrict__ ls,
                          const float *__restrict__ q, const float *__restrict__ rho, int64_t n,
                          float4 *__restrict__ rec, float4 *__restrict__ crec, uint32_t *bad)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float qw = q[4 * k], qx = q[4 * k + 1], qy = q[4 * k + 2], qz = q[4 * k + 3];
    // a non-finite parameter (a diverged optimisation, corrupted input) is
    // reported to the host, which refuses the projection
    if (bad && !(isfinite(mu[3 * k]) && isfinite(mu[3 * k + 1]) && isfinite(mu[3 * k + 2]) &&
                 isfinite(ls[3 * k]) && isfinite(ls[3 * k + 1]) && isfinite(ls[3 * k + 2]) &&
                 isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) && isfinite(rho[k])))
        atomicOr(bad, 1u);
    float n2 = A(A(A(M(qw, qw), M(qx, qx)), M(qy, qy)), M(qz, qz));
    float w, x, y, z;
    if (!(n2 > 0.0f) || !(n2 < INFINITY)) {
        w = 1.0f; x = y = z = 0.0f;
    } else {
        float nr = __fsqrt_rn(n2);
        w = __fdiv_rn(qw, nr); x = __fdiv_rn(qx, nr); y = __fdiv_rn(qy, nr); z = __fdiv_rn(qz, nr);
    }
    float R[3][3];
    R[0][0] = S(1.0f, M(2.0f, A(M(y, y), M(z, z))));
    R[0][1] = M(2.0f, S(M(x, y), M(w, z)));
    R[0][2] = M(2.0f, A(M(x, z), M(w, y)));
    R[1][0] = M(2.0f, A(M(x, y), M(w, z)));
    R[1][1] = S(1.0f, M(2.0f, A(M(x, x), M(z, z))));
    R[1][2] = M(2.0f, S(M(y, z), M(w, x)));
    R[2][0] = M(2.0f, S(M(x, z), M(w, y)));
    R[2][1] = M(2.0f, A(M(y, z), M(w, x)));
    R[2][2] = S(1.0f, M(2.0f, A(M(x, x), M(y, y))));
    float l0 = ls[3 * k], l1 = ls[3 * k + 1], l2 = ls[3 * k + 2];
    float s2[3] = { exp_spec(M(2.0f, l0)), exp_spec(M(2.0f, l1)), exp_spec(M(2.0f, l2)) };
    const int ia[6] = { 0, 0, 0, 1, 1, 2 }, ib[6] = { 0, 1, 2, 1, 2, 2 };
    float sig[6];
#pragma unroll
    for (int e = 0; e < 6; e++) {
        int a = ia[e], b = ib[e];
        sig[e] = A(A(M(M(R[a][0], R[b][0]), s2[0]), M(M(R[a][1], R[b][1]), s2[1])),
                   M(M(R[a][2], R[b][2]), s2[2]));
    }
    float m0 = mu[3 * k], m1 = mu[3 * k + 1], m2 = mu[3 * k + 2];
    crec[CREC_F4 * k + 0] = make_float4(m0, m1, m2, 0.0f);
    crec[CREC_F4 * k + 1] = make_float4(sig[0], sig[1], sig[2], sig[3]);
    crec[CREC_F4 * k + 2] = make_float4(sig[4], sig[5], 0.0f, 0.0f);

    // integration record: P = R diag(e^-2l) R^T and S = Sigma / det Sigma =
    // R diag(e^-2(l_b + l_c)) R^T ({k, b, c} = {0, 1, 2}); not part of the
    // culling specification, ordinary arithmetic.
    float p2[3] = { expf(-2.0f * l0), expf(-2.0f * l1), expf(-2.0f * l2) };
    float c2[3] = { expf(-2.0f * (l1 + l2)), expf(-2.0f * (l0 + l2)), expf(-2.0f * (l0 + l1)) };
    float P[6], Sh[6];
#pragma unroll
    for (int e = 0; e < 6; e++) {
        int a = ia[e], b = ib[e];
        P[e] = R[a][0] * R[b][0] * p2[0] + R[a][1] * R[b][1] * p2[1] + R[a][2] * R[b][2] * p2[2];
        Sh[e] = R[a][0] * R[b][0] * c2[0] + R[a][1] * R[b][1] * c2[1] + R[a][2] * R[b][2] * c2[2];
    }
    float smax = expf(fmaxf(l0, fmaxf(l1, l2)));
    rec[REC_F4 * k + 0] = make_float4(m0, m1, m2, rho[k]);
    rec[REC_F4 * k + 1] = make_float4(P[0], P[1], P[2], P[3]);
    rec[REC_F4 * k + 2] = make_float4(P[4], P[5], Sh[0], Sh[1]);
    rec[REC_F4 * k + 3] = make_float4(Sh[2], Sh[3], Sh[4], Sh[5]);
    rec[REC_F4 * k + 4] = make_float4(smax, 0.0f, 0.0f, 0.0f);
}

// e_a^T Sigma e_b, Sigma packed (00,01,02,11,12,22)
__device__ __forceinline__ float form_spec(const float *Sg, const float *a, const float *b)
{
    float t0 = A(A(M(Sg[0], b[0]), M(Sg[1], b[1])), M(Sg[2], b[2]));
    float t1 = A(A(M(Sg[1], b[0]), M(Sg[3], b[1])), M(Sg[4], b[2]));
    float t2 = A(A(M(Sg[2], b[0]), M(Sg[4], b[1])), M(Sg[5], b[2]));
    return A(A(M(a[0], t0), M(a[1], t1)), M(a[2], t2));
}

__device__ __forceinline__ float dot_spec(const float *m, const float *e)
{
    return A(A(M(m[0], e[0]), M(m[1], e[1])), M(m[2], e[2]));
}

// detector interval along one axis whose cone-beam rays meet the K-sigma
// ellipsoid: roots of (n.a)^2 = K^2 n^T Sigma n for the planes through the
// source containing the other detector axis; false if unbounded.
__device__ __forceinline__ bool cone_spec(float K2, float dsd, float ae, float aw, float see,
                                          float sew, float sww, float &lo, float &hi)
{
    float alpha = S(M(aw, aw), M(K2, sww));
    if (!(alpha > 0.0f)) return false;
    float beta = M(dsd, S(M(ae, aw), M(K2, sew)));
    float disc = S(A(S(M(M(aw, aw), see), M(M(M(2.0f, ae), aw), sew)), M(M(ae, ae), sww)),
                   M(K2, S(M(see, sww), M(sew, sew))));
    if (!(disc > 0.0f)) disc = 0.0f;
    float r = M(dsd, __fsqrt_rn(M(K2, disc)));
    lo = __fdiv_rn(S(beta, r), alpha);
    hi = __fdiv_rn(A(beta, r), alpha);
    return true;
}

// first index whose table value is >= x (n if none), and the last whose
// value is <= x (-1 if none), by binary search over the increasing table
__device__ __forceinline__ int lower_idx(const float *tab, int n, float x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(tab + mid) >= x) hi = mid; else lo = mid + 1;
    }
    return lo;
}
__device__ __forceinline__ int upper_idx(const float *tab, int n, float x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(tab + mid) > x) hi = mid; else lo = mid + 1;
    }
    return lo - 1;
}

// The same two searches started from a guess: for a uniformly spaced table
// (t0 + i step in binary32, inv = 1/step) the guess is within a step of the
// answer and a short walk in the table makes it exact -- the answer is
// defined by the table comparisons alone, so it equals the binary search's.
// inv == 0 (an irregular table) falls back to the binary search; NaN gives
// what the binary search gives (n, n - 1).
__device__ __forceinline__ int lower_idx_g(const float *tab, int n, float x, float t0, float inv)
{
    if (inv == 0.0f || !(x == x)) return lower_idx(tab, n, x);
    int i = (int)fminf(fmaxf(ceilf((x - t0) * inv), 0.0f), (float)n);
    while (i > 0 && __ldg(tab + i - 1) >= x) i--;
    while (i < n && __ldg(tab + i) < x) i++;
    return i;
}
__device__ __forceinline__ int upper_idx_g(const float *tab, int n, float x, float t0, float inv)
{
    if (inv == 0.0f || !(x == x)) return upper_idx(tab, n, x);
    // first index whose value is > x, minus one
    int i = (int)fminf(fmaxf(floorf((x - t0) * inv) + 1.0f, 0.0f), (float)n);
    while (i > 0 && __ldg(tab + i - 1) > x) i--;
    while (i < n && __ldg(tab + i) <= x) i++;
    return i - 1;
}

// one thread per (view of the chunk, Gaussian), view-major
__global__ void k_cull(DevGeom g, int nv, const float4 *__restrict__ crec, int64_t n,
                       uint32_t *__restrict__ cnt, uint2 *__restrict__ rect)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nv * n) return;
    int vl = (int)(idx / n);
    int64_t k = idx - (int64_t)vl * n;
    const float *F = g.frames + 9 * (size_t)(g.v0 + vl);
    float eu[3] = { __ldg(F + 0), __ldg(F + 1), __ldg(F + 2) };
    float ev[3] = { __ldg(F + 3), __ldg(F + 4), __ldg(F + 5) };
    float ew[3] = { __ldg(F + 6), __ldg(F + 7), __ldg(F + 8) };
    float4 c0 = crec[CREC_F4 * k], c1 = crec[CREC_F4 * k + 1], c2 = crec[CREC_F4 * k + 2];
    float m[3] = { c0.x, c0.y, c0.z };
    float Sg[6] = { c1.x, c1.y, c1.z, c1.w, c2.x, c2.y };
    const float K2 = CULL_K2;
    float mu_u = dot_spec(m, eu), mu_v = dot_spec(m, ev);
    float ulo = -INFINITY, uhi = INFINITY, vlo = -INFINITY, vhi = INFINITY;
    if (g.kind == 1) {
        float aw = A(dot_spec(m, ew), g.dso);
        float suu = form_spec(Sg, eu, eu), svv = form_spec(Sg, ev, ev), sww = form_spec(Sg, ew, ew);
        float suw = form_spec(Sg, eu, ew), svw = form_spec(Sg, ev, ew);
        float lo, hi;
        if (cone_spec(K2, g.dsd, mu_u, aw, suu, suw, sww, lo, hi)) { ulo = lo; uhi = hi; }
        if (cone_spec(K2, g.dsd, mu_v, aw, svv, svw, sww, lo, hi)) { vlo = lo; vhi = hi; }
    } else {
        float hu = __fsqrt_rn(M(K2, form_spec(Sg, eu, eu)));
        float hv = __fsqrt_rn(M(K2, form_spec(Sg, ev, ev)));
        ulo = S(mu_u, hu); uhi = A(mu_u, hu); vlo = S(mu_v, hv); vhi = A(mu_v, hv);
    }
    int i0 = lower_idx_g(g.utab, g.n_cols, ulo, g.u0, g.uinv);
    int i1 = upper_idx_g(g.utab, g.n_cols, uhi, g.u0, g.uinv);
    int j0, j1;
    if (g.kind == GM_PET3D) {
        // 3-D PET: the LOR of radial position s and mid-height z has
        // direction e_w + kappa e_v, kappa = dz / (2 sqrt(R^2 - s^2)), and
        // a . x = z along it for a = e_v - kappa e_w, so it can meet the
        // K-sigma ellipsoid only if z lies in mu.a +- sqrt(K^2 a^T Sigma a).
        // Both bounds are convex / concave in kappa, so over the columns
        // i0..i1 the union of these intervals is spanned by their values at
        // the two extreme slopes.  Rows are ring pairs (mid-heights
        // vtab + zoff); rows past the segment's last pair hold no LOR.
        j0 = 0;
        j1 = -1;
        if (i0 <= i1) {
            const int delta = pet3d_delta(g, g.v0 + vl), ad = abs(delta);
            const float dz = M((float)delta, g.ring_pitch), zoff = M(M(0.5f, (float)ad), g.ring_pitch);
            const float ua = __ldg(g.utab + i0), ub = __ldg(g.utab + i1);
            const float amin = (ua <= 0.0f && ub >= 0.0f) ? 0.0f : fminf(fabsf(ua), fabsf(ub));
            const float amax = fmaxf(fabsf(ua), fabsf(ub));
            const float h2a = S(g.radius2, M(amin, amin)), h2b = S(g.radius2, M(amax, amax));
            const int last = g.n_rows - 1 - ad;
            if (!(h2b > 0.0f)) {
                j1 = last;
            } else {
                const float mu_w = dot_spec(m, ew);
                const float svv = form_spec(Sg, ev, ev), svw = form_spec(Sg, ev, ew), sww = form_spec(Sg, ew, ew);
                float zlo = INFINITY, zhi = -INFINITY;
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const float kap = __fdiv_rn(M(0.5f, dz), __fsqrt_rn(e ? h2b : h2a));
                    const float zc = S(mu_v, M(kap, mu_w));
                    const float t = A(S(svv, M(M(2.0f, kap), svw)), M(M(kap, kap), sww));
                    const float half = __fsqrt_rn(fmaxf(M(K2, t), 0.0f));
                    zlo = fminf(zlo, S(zc, half));
                    zhi = fmaxf(zhi, A(zc, half));
                }
                j0 = lower_idx_g(g.vtab, g.n_rows, S(zlo, zoff), g.v0f, g.vinv);
                j1 = min(upper_idx_g(g.vtab, g.n_rows, S(zhi, zoff), g.v0f, g.vinv), last);
            }
        }
    } else {
        j0 = lower_idx_g(g.vtab, g.n_rows, vlo, g.v0f, g.vinv);
        j1 = upper_idx_g(g.vtab, g.n_rows, vhi, g.v0f, g.vinv);
    }
    if (i0 > i1 || j0 > j1) {
        cnt[idx] = 0;
        rect[idx] = make_uint2(0u, 0u);
    } else {
        unsigned tx0 = i0 / g.tile_w, tx1 = i1 / g.tile_w, ty0 = j0 / g.tile_h, ty1 = j1 / g.tile_h;
        cnt[idx] = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
        // pixel box (the tiles follow from it)
        rect[idx] = make_uint2((unsigned)i0 | ((unsigned)i1 << 16), (unsigned)j0 | ((unsigned)j1 << 16));
    }
}

}  // namespace

cudaError_t launch_records(const float *mu, const float *ls, const float *q, const float *rho,
                           int64_t n, float4 *rec, float4 *crec, uint32_t *bad, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int bs = 256;
    k_records<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(mu, ls, q, rho, n, rec, crec, bad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cull(const DevGeom &g, int nv, const float4 *crec, int64_t n, uint32_t *cnt,
                        uint2 *rect, cudaStream_t s)
{
    int64_t tot = (int64_t)nv * n;
    if (tot <= 0) return cudaSuccess;
    int bs = 256;
    k_cull<<<(unsigned)((tot + bs - 1) / bs), bs, 0, s>>>(g, nv, crec, n, cnt, rect);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rgrt
