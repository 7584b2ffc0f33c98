// Per-tile ray integration (a3) and its adjoint (a5).
//
// One CTA per detector tile of tile_w x tile_h rays, one ray per thread,
// warps laid out as 8 x 4 ray blocks.  The tile's Gaussian list (ascending
// ids) is walked in chunks: the CTA gathers each chunk's records into shared
// memory together with the Gaussian's detector bounding box for this view;
// a warp skips a Gaussian whose box misses its 8 x 4 block (a warp-uniform
// branch), otherwise every lane evaluates its pair:
//   delta = o - mu, recentred on the foot of the perpendicular from mu
//   A = d^T P d, B = d^T P delta, C = delta^T P delta        (Eq. 7)
//   m = C - B^2/A                                             (Eq. 9)
//   f = rho sqrt(2 pi / A) exp(-m/2) Phi                      (Eqs. 10-11)
//   Phi = 1/2 [erf(w_b) - erf(w_a)], w = (A t + B)/sqrt(2A)  (finite segment)
// and the pair counts when m <= 9 (3-sigma cut).  FP32 throughout, FP32
// accumulation per ray.
#include "rgrt_internal.h"

namespace rgrt {
namespace {

constexpr float SQRT2PI = 2.50662827463100050f;
constexpr float INV_SQRT2PI = 0.398942280401432678f;
constexpr float INV_SQRTPI = 0.564189583547756287f;
constexpr float SQRT_HALF = 0.707106781186547524f;
constexpr float SKIP_K2 = 9.2f;   // skip boxes: a little wider than the 3-sigma cut
constexpr float W_SAT = 4.0f;     // |w| >= 4: erf(w) == +-1 in binary32
constexpr int FWD_CH = 128;
constexpr int ADJ_CH = 64;
constexpr int NG = 10;            // adjoint components per pair: dmu[3], G_P[6], drho

struct SRec {
    float4 a;   // mu, rho
    float4 b;   // P00 P01 P02 P11
    float4 c;   // P12 P22, gid (bits), 0
    float4 bb;  // u_lo, u_hi, v_lo, v_hi of the (skip) detector box
};

struct Ray {
    float ox, oy, oz, dx, dy, dz, ta, tb;
};

__device__ __forceinline__ float quad_form(const float *Sg, const float *a, const float *b)
{
    float t0 = Sg[0] * b[0] + Sg[1] * b[1] + Sg[2] * b[2];
    float t1 = Sg[1] * b[0] + Sg[3] * b[1] + Sg[4] * b[2];
    float t2 = Sg[2] * b[0] + Sg[4] * b[1] + Sg[5] * b[2];
    return a[0] * t0 + a[1] * t1 + a[2] * t2;
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

// gather one record and its detector box for view frame F
template <bool CONE>
__device__ __forceinline__ void prep_record(const DevGeom &g, const float *F, uint32_t gid,
                                            const float4 *__restrict__ rec,
                                            const float4 *__restrict__ crec, SRec &out)
{
    float4 r0 = __ldg(rec + REC_F4 * (size_t)gid);
    float4 r1 = __ldg(rec + REC_F4 * (size_t)gid + 1);
    float4 r2 = __ldg(rec + REC_F4 * (size_t)gid + 2);
    float4 c1 = __ldg(crec + CREC_F4 * (size_t)gid + 1);
    float4 c2 = __ldg(crec + CREC_F4 * (size_t)gid + 2);
    float Sg[6] = { c1.x, c1.y, c1.z, c1.w, c2.x, c2.y };
    float m[3] = { r0.x, r0.y, r0.z };
    float eu[3] = { F[0], F[1], F[2] }, ev[3] = { F[3], F[4], F[5] }, ew[3] = { F[6], F[7], F[8] };
    float mu_u = m[0] * eu[0] + m[1] * eu[1] + m[2] * eu[2];
    float mu_v = m[0] * ev[0] + m[1] * ev[1] + m[2] * ev[2];
    float ulo = -INFINITY, uhi = INFINITY, vlo = -INFINITY, vhi = INFINITY;
    if (CONE) {
        float aw = m[0] * ew[0] + m[1] * ew[1] + m[2] * ew[2] + g.dso;
        float suu = quad_form(Sg, eu, eu), svv = quad_form(Sg, ev, ev), sww = quad_form(Sg, ew, ew);
        float suw = quad_form(Sg, eu, ew), svw = quad_form(Sg, ev, ew);
        float lo, hi;
        if (cone_interval(SKIP_K2, g.dsd, mu_u, aw, suu, suw, sww, lo, hi)) { ulo = lo; uhi = hi; }
        if (cone_interval(SKIP_K2, g.dsd, mu_v, aw, svv, svw, sww, lo, hi)) { vlo = lo; vhi = hi; }
    } else {
        float hu = sqrtf(SKIP_K2 * quad_form(Sg, eu, eu));
        float hv = sqrtf(SKIP_K2 * quad_form(Sg, ev, ev));
        ulo = mu_u - hu; uhi = mu_u + hu; vlo = mu_v - hv; vhi = mu_v + hv;
    }
    out.a = r0;
    out.b = r1;
    out.c = make_float4(r2.x, r2.y, __uint_as_float(gid), 0.0f);
    out.bb = make_float4(ulo, uhi, vlo, vhi);
}

// ray of detector pixel (u, v) in view frame F (FP32; see ray set-up notes)
template <bool CONE>
__device__ __forceinline__ Ray make_ray(const DevGeom &g, const float *F, float u, float v)
{
    float op0, op1, op2, dp0, dp1, dp2, ta, tb;
    if (CONE) {
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

struct PairGeo {
    float px, py, pz;      // recentred delta (perpendicular to d)
    float ta, tb;          // segment relative to the foot of the perpendicular
    float Pdx, Pdy, Pdz;   // P d
    float Ppx, Ppy, Ppz;   // P delta
    float A, B, C, rA, iA, m;
};

__device__ __forceinline__ void pair_geo(const Ray &r, const SRec &s, PairGeo &q)
{
    float ex = r.ox - s.a.x, ey = r.oy - s.a.y, ez = r.oz - s.a.z;
    float tau = r.dx * ex + r.dy * ey + r.dz * ez;
    q.px = ex - tau * r.dx; q.py = ey - tau * r.dy; q.pz = ez - tau * r.dz;
    q.ta = r.ta + tau; q.tb = r.tb + tau;
    const float P00 = s.b.x, P01 = s.b.y, P02 = s.b.z, P11 = s.b.w, P12 = s.c.x, P22 = s.c.y;
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

struct TileCtx {
    int vl, tx, ty, view, col, row;
    bool valid;
    float wu_lo, wu_hi, wv_lo, wv_hi;  // detector box of this warp's 8 x 4 rays
    long long out_idx;
};

__device__ __forceinline__ TileCtx tile_ctx(const DevGeom &g)
{
    TileCtx c;
    int T = g.tiles_x * g.tiles_y;
    c.vl = blockIdx.x / T;
    int tin = blockIdx.x - c.vl * T;
    c.ty = tin / g.tiles_x;
    c.tx = tin - c.ty * g.tiles_x;
    c.view = g.v0 + c.vl;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int wpr = g.tile_w >> 3;  // warps per tile row
    int wx = w % wpr, wy = w / wpr;
    int c0 = c.tx * g.tile_w + wx * 8, r0 = c.ty * g.tile_h + wy * 4;
    c.col = c0 + (lane & 7);
    c.row = r0 + (lane >> 3);
    c.valid = c.col < g.n_cols && c.row < g.n_rows;
    if (c0 < g.n_cols && r0 < g.n_rows) {
        int c1 = min(c0 + 7, g.n_cols - 1), r1 = min(r0 + 3, g.n_rows - 1);
        c.wu_lo = __ldg(g.utab + c0); c.wu_hi = __ldg(g.utab + c1);
        c.wv_lo = __ldg(g.vtab + r0); c.wv_hi = __ldg(g.vtab + r1);
    } else {
        c.wu_lo = INFINITY; c.wu_hi = -INFINITY; c.wv_lo = INFINITY; c.wv_hi = -INFINITY;
    }
    c.out_idx = (long long)c.view * g.stride_view + (long long)c.row * g.stride_row + c.col;
    return c;
}

__device__ __forceinline__ bool box_hits(const TileCtx &c, const float4 &bb)
{
    return !(bb.y < c.wu_lo || bb.x > c.wu_hi || bb.w < c.wv_lo || bb.z > c.wv_hi);
}

template <bool CONE>
__global__ void __launch_bounds__(256) k_forward(DevGeom g, const float4 *__restrict__ rec,
                                                 const float4 *__restrict__ crec,
                                                 const uint32_t *__restrict__ gids,
                                                 const uint2 *__restrict__ ranges,
                                                 float *__restrict__ out, Stats *stats)
{
    __shared__ SRec srec[FWD_CH];
    __shared__ float Fs[9];
    TileCtx c = tile_ctx(g);
    if (threadIdx.x < 9) Fs[threadIdx.x] = __ldg(g.frames + 9 * (size_t)c.view + threadIdx.x);
    __syncthreads();
    float F[9];
#pragma unroll
    for (int i = 0; i < 9; i++) F[i] = Fs[i];
    float u = __ldg(g.utab + min(c.col, g.n_cols - 1));
    float v = __ldg(g.vtab + min(c.row, g.n_rows - 1));
    Ray ray = make_ray<CONE>(g, F, u, v);
    uint2 rg = ranges[blockIdx.x];
    float acc = 0.0f;
    unsigned long long n_eval = 0, n_kept = 0;
    const int nthr = blockDim.x;
    for (uint32_t base = rg.x; base < rg.y; base += FWD_CH) {
        int cnt = min((uint32_t)FWD_CH, rg.y - base);
        for (int i = threadIdx.x; i < cnt; i += nthr)
            prep_record<CONE>(g, F, __ldg(gids + base + i), rec, crec, srec[i]);
        __syncthreads();
        for (int j = 0; j < cnt; j++) {
            float4 bb = srec[j].bb;
            if (!box_hits(c, bb)) continue;
            SRec s;
            s.a = srec[j].a; s.b = srec[j].b; s.c = srec[j].c;
            PairGeo q;
            pair_geo(ray, s, q);
            float E = __expf(-0.5f * q.m);
            float K = s.a.w * SQRT2PI * q.rA * E;
            float sc = q.rA * SQRT_HALF;
            float wa = (q.A * q.ta + q.B) * sc, wb = (q.A * q.tb + q.B) * sc;
            float phi = 1.0f;
            if (!(wa <= -W_SAT && wb >= W_SAT)) phi = 0.5f * (erff(wb) - erff(wa));
            bool keep = c.valid && q.m <= PAIR_CUT2;
            acc += keep ? K * phi : 0.0f;
            n_eval += c.valid;
            n_kept += keep;
        }
        __syncthreads();
    }
    if (c.valid) out[c.out_idx] = acc;
    if (stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
            n_kept += __shfl_xor_sync(0xffffffffu, n_kept, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&stats->pairs_eval, n_eval);
            atomicAdd(&stats->pairs_kept, n_kept);
        }
    }
}

template <bool CONE>
__global__ void __launch_bounds__(256) k_adjoint(DevGeom g, const float4 *__restrict__ rec,
                                                 const float4 *__restrict__ crec,
                                                 const uint32_t *__restrict__ gids,
                                                 const uint2 *__restrict__ ranges,
                                                 const float *__restrict__ dLdI,
                                                 float4 *__restrict__ grad)
{
    __shared__ SRec srec[ADJ_CH];
    __shared__ float part[ADJ_CH][8][NG];   // per record, per warp, per component
    __shared__ float Fs[9];
    TileCtx c = tile_ctx(g);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x < 9) Fs[threadIdx.x] = __ldg(g.frames + 9 * (size_t)c.view + threadIdx.x);
    __syncthreads();
    float F[9];
#pragma unroll
    for (int i = 0; i < 9; i++) F[i] = Fs[i];
    float u = __ldg(g.utab + min(c.col, g.n_cols - 1));
    float v = __ldg(g.vtab + min(c.row, g.n_rows - 1));
    Ray ray = make_ray<CONE>(g, F, u, v);
    float gw = c.valid ? __ldg(dLdI + c.out_idx) : 0.0f;
    uint2 rg = ranges[blockIdx.x];
    const int nthr = blockDim.x;
    for (uint32_t base = rg.x; base < rg.y; base += ADJ_CH) {
        int cnt = min((uint32_t)ADJ_CH, rg.y - base);
        for (int i = threadIdx.x; i < cnt; i += nthr)
            prep_record<CONE>(g, F, __ldg(gids + base + i), rec, crec, srec[i]);
        __syncthreads();
        for (int j = 0; j < cnt; j++) {
            float4 bb = srec[j].bb;
            if (!box_hits(c, bb)) {
                if (lane < NG) part[j][w][lane] = 0.0f;
                continue;
            }
            SRec s;
            s.a = srec[j].a; s.b = srec[j].b; s.c = srec[j].c;
            PairGeo q;
            pair_geo(ray, s, q);
            float val[NG];
            bool keep = c.valid && q.m <= PAIR_CUT2 && gw != 0.0f;
            if (keep) {
                float E = __expf(-0.5f * q.m);
                float K = s.a.w * SQRT2PI * q.rA * E;
                float sc = q.rA * SQRT_HALF;
                float wa = (q.A * q.ta + q.B) * sc, wb = (q.A * q.tb + q.B) * sc;
                float phi = 1.0f, dPhiB = 0.0f, dPhiA = 0.0f;
                if (!(wa <= -W_SAT && wb >= W_SAT)) {
                    phi = 0.5f * (erff(wb) - erff(wa));
                    float ea = __expf(-wa * wa), eb = __expf(-wb * wb);
                    dPhiB = (eb - ea) * q.rA * INV_SQRT2PI;
                    float tA = 2.0f * q.A;
                    float r32 = rsqrtf(tA) / tA;  // (2A)^-3/2
                    dPhiA = (eb * (q.A * q.tb - q.B) - ea * (q.A * q.ta - q.B)) * INV_SQRTPI * r32;
                }
                float f = K * phi;
                float fC = -0.5f * f;
                float fB = f * q.B * q.iA + K * dPhiB;
                float fA = -0.5f * f * q.iA * (1.0f + q.B * q.B * q.iA) + K * dPhiA;
                // gradient w.r.t. the recentred delta: fB P d + 2 fC P delta
                float gx = fB * q.Pdx + 2.0f * fC * q.Ppx;
                float gy = fB * q.Pdy + 2.0f * fC * q.Ppy;
                float gz = fB * q.Pdz + 2.0f * fC * q.Ppz;
                float dg = ray.dx * gx + ray.dy * gy + ray.dz * gz;
                float st = K * q.A * dPhiB;  // d f / d(segment shift)
                // d mu = -(I - d d^T) grad - d * st
                val[0] = gw * (-(gx - ray.dx * dg) - ray.dx * st);
                val[1] = gw * (-(gy - ray.dy * dg) - ray.dy * st);
                val[2] = gw * (-(gz - ray.dz * dg) - ray.dz * st);
                // symmetric gradient w.r.t. P: fA d d^T + fB sym(d p^T) + fC p p^T
                float hB = 0.5f * fB;
                val[3] = gw * (fA * ray.dx * ray.dx + 2.0f * hB * ray.dx * q.px + fC * q.px * q.px);
                val[4] = gw * (fA * ray.dx * ray.dy + hB * (ray.dx * q.py + q.px * ray.dy) + fC * q.px * q.py);
                val[5] = gw * (fA * ray.dx * ray.dz + hB * (ray.dx * q.pz + q.px * ray.dz) + fC * q.px * q.pz);
                val[6] = gw * (fA * ray.dy * ray.dy + 2.0f * hB * ray.dy * q.py + fC * q.py * q.py);
                val[7] = gw * (fA * ray.dy * ray.dz + hB * (ray.dy * q.pz + q.py * ray.dz) + fC * q.py * q.pz);
                val[8] = gw * (fA * ray.dz * ray.dz + 2.0f * hB * ray.dz * q.pz + fC * q.pz * q.pz);
                val[9] = gw * (SQRT2PI * q.rA * E * phi);
            } else {
#pragma unroll
                for (int k = 0; k < NG; k++) val[k] = 0.0f;
            }
            int idx = tr_reduce<NG>(val, lane);
            if (idx < NG) part[j][w][idx] = val[0];
        }
        __syncthreads();
        // sum over warps, then one set of vector atomics per Gaussian
        for (int e = threadIdx.x; e < cnt * NG; e += nthr) {
            int j = e / NG, k = e - j * NG;
            float s = 0.0f;
            for (int ww = 0; ww < nw; ww++) s += part[j][ww][k];
            part[j][0][k] = s;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += nthr) {
            const float *p = part[j][0];
            bool any = false;
#pragma unroll
            for (int k = 0; k < NG; k++) any |= p[k] != 0.0f;
            if (!any) continue;
            uint32_t gid = __float_as_uint(srec[j].c.z);
            float4 *gp = grad + GRAD_F4 * (size_t)gid;
            atomicAdd(gp, make_float4(p[0], p[1], p[2], p[9]));
            atomicAdd(gp + 1, make_float4(p[3], p[4], p[5], p[6]));
            atomicAdd(reinterpret_cast<float2 *>(gp + 2), make_float2(p[7], p[8]));
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_forward(const DevGeom &g, int nv, const float4 *rec, const float4 *crec,
                           const uint32_t *gids, const uint2 *ranges, float *out, Stats *stats,
                           cudaStream_t s)
{
    unsigned nt = (unsigned)nv * g.tiles_x * g.tiles_y;
    if (nt == 0) return cudaSuccess;
    int bs = g.tile_w * g.tile_h;
    if (g.kind == 1)
        k_forward<true><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, out, stats);
    else
        k_forward<false><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, out, stats);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const DevGeom &g, int nv, const float4 *rec, const float4 *crec,
                           const uint32_t *gids, const uint2 *ranges, const float *dLdI,
                           float4 *grad, cudaStream_t s)
{
    unsigned nt = (unsigned)nv * g.tiles_x * g.tiles_y;
    if (nt == 0) return cudaSuccess;
    int bs = g.tile_w * g.tile_h;
    if (g.kind == 1)
        k_adjoint<true><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, dLdI, grad);
    else
        k_adjoint<false><<<nt, bs, 0, s>>>(g, rec, crec, gids, ranges, dLdI, grad);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rgrt
