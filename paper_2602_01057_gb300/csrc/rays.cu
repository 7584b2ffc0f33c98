// Explicit rays: any set of lines (o, d, [t_a, t_b]) given by the caller, e.g.
// a helical cone-beam trajectory or a list-mode PET event set, projected with
// the closed form of Eqs. 7-12 (general path, world coordinates).
//
// Rays are grouped in blocks of RB consecutive rays (one CTA, one ray per
// thread); a caller whose neighbouring rays are close gets tight blocks.
// Binning per projection:
//  * every Gaussian gets a bounding ball (mu, K sigma_max), K^2 = 9.0625: its
//    K-sigma ellipsoid -- which holds every point where m <= 9 -- lies inside
//    it; the scene box is the union of the balls;
//  * every block gets a reference line L0 (one of its rays, re-based at the
//    point nearest the scene centre) and dev = the largest distance from L0 of
//    the end points of its rays' lines clipped to the scene box.  A line that
//    meets a Gaussian's ellipsoid does so inside the scene box, at a point no
//    further than dev from L0 (distance to a line is convex along a segment),
//    so the Gaussian can pair with the block only if
//        dist(mu, L0) <= K sigma_max + dev;
//  * the same bound is taken per warp (32 rays); per block, one warp counts
//    and then emits the Gaussians that pass the block's test and then a
//    warp's test into that warp's list, visiting them through clusters of 32
//    Morton-ordered balls (a cluster ball holds its members' balls, so only
//    the members of the clusters the block meets are tested).
// Integration and adjoint: every warp walks its own list, 32 records at a
// time staged in its own slice of shared memory (no barrier across the CTA),
// and skips a record when no lane's line meets its bounding ball.
#include "pair.cuh"

namespace rgrt {
namespace {

constexpr int RB = 128;    // rays per block
constexpr int CULL_BS = 256;
constexpr int NG_RAYS = 10;  // general_grad components: dmu[3], G_P[6], drho
// bounding-ball radius factor: K sigma_max with K^2 the culling constant (a
// margin over the 3-sigma cut), widened by a few ulp for the FP32 tests
#define BALL_K (3.0103986f * (1.0f + 1e-5f))

struct SRec {
    float4 g0, g1, g2;     // (mu, rho), (P00 P01 P02 P11), (P12 P22, id, bounding-ball radius)
};

__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float norm2(float3 a) { return a.x * a.x + a.y * a.y + a.z * a.z; }

// normalise d, re-base o at the point of the line nearest the world origin
// (FP64, once per ray), shift the segment accordingly; flag invalid rays
__global__ void k_rays_prep(const float *__restrict__ o3, const float *__restrict__ d3,
                            const float *__restrict__ t2, const float *__restrict__ tof2, int64_t n,
                            float4 *ro, float4 *rd, float2 *tof, uint32_t *bad)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double ox = o3[3 * r], oy = o3[3 * r + 1], oz = o3[3 * r + 2];
    const double dx = d3[3 * r], dy = d3[3 * r + 1], dz = d3[3 * r + 2];
    const double ta = t2[2 * r], tb = t2[2 * r + 1];
    const double len = sqrt(dx * dx + dy * dy + dz * dz);
    const bool ok = isfinite(ox) && isfinite(oy) && isfinite(oz) && isfinite(len) && len > 0.0 &&
                    !isnan(ta) && !isnan(tb) && ta <= tb;
    double tc = 0.0, sT = 0.0;
    if (tof2) {
        tc = tof2[2 * r];
        sT = tof2[2 * r + 1];
    }
    const bool tof_ok = !tof2 || (!isnan(sT) && (!(sT > 0.0) || isinf(sT) || isfinite(tc)));
    if (!ok || !tof_ok) {
        atomicOr(bad, 1u);
        ro[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        rd[r] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
        if (tof) tof[r] = make_float2(0.0f, 0.0f);
        return;
    }
    const double ux = dx / len, uy = dy / len, uz = dz / len;
    const double s = ox * ux + oy * uy + oz * uz;   // o = o' + s u
    ro[r] = make_float4((float)(ox - s * ux), (float)(oy - s * uy), (float)(oz - s * uz), (float)(ta + s));
    rd[r] = make_float4((float)ux, (float)uy, (float)uz, (float)(tb + s));
    // time of flight: centre in the re-based parameter, tau = 1 / sigma_T^2
    // (a width <= 0 or infinite means none)
    if (tof) tof[r] = sT > 0.0 && !isinf(sT) ? make_float2((float)(tc + s), (float)(1.0 / (sT * sT)))
                                             : make_float2(0.0f, 0.0f);
}

// bounding balls (mu, K sigma_max) and per-CTA partial scene boxes
__global__ void k_balls(const float4 *__restrict__ rec, int64_t n, float4 *ball, float4 *part)
{
    __shared__ float red[6][CULL_BS / 32];
    float lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    const float K = BALL_K;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float4 m = __ldg(rec + REC_F4 * k);
        const float r = K * __ldg(rec + REC_F4 * k + 4).x;
        ball[k] = make_float4(m.x, m.y, m.z, r);
        lo[0] = fminf(lo[0], m.x - r); hi[0] = fmaxf(hi[0], m.x + r);
        lo[1] = fminf(lo[1], m.y - r); hi[1] = fmaxf(hi[1], m.y + r);
        lo[2] = fminf(lo[2], m.z - r); hi[2] = fmaxf(hi[2], m.z + r);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 3; c++) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; c++) { red[c][w] = lo[c]; red[3 + c][w] = hi[c]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < CULL_BS / 32; j++)
            for (int c = 0; c < 3; c++) {
                red[c][0] = fminf(red[c][0], red[c][j]);
                red[3 + c][0] = fmaxf(red[3 + c][0], red[3 + c][j]);
            }
        part[2 * blockIdx.x] = make_float4(red[0][0], red[1][0], red[2][0], 0.0f);
        part[2 * blockIdx.x + 1] = make_float4(red[3][0], red[4][0], red[5][0], 0.0f);
    }
}

// scene box from the partials, widened by a margin; also the margin
// (scene[0].w) used by the block test
__global__ void k_scene(const float4 *part, int nparts, float4 *scene)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int j = 0; j < nparts; j++) {
        const float4 a = part[2 * j], b = part[2 * j + 1];
        lo[0] = fminf(lo[0], a.x); lo[1] = fminf(lo[1], a.y); lo[2] = fminf(lo[2], a.z);
        hi[0] = fmaxf(hi[0], b.x); hi[1] = fmaxf(hi[1], b.y); hi[2] = fmaxf(hi[2], b.z);
    }
    float ext = 0.0f;
    for (int c = 0; c < 3; c++) ext = fmaxf(ext, fmaxf(fabsf(lo[c]), fabsf(hi[c])));
    // FP32 slack of the clipping and distance arithmetic (a few ulp of the
    // largest coordinate), generously
    const float eps = ext * 6.1e-5f + 1e-30f;
    scene[0] = make_float4(lo[0] - eps, lo[1] - eps, lo[2] - eps, eps);
    scene[1] = make_float4(hi[0] + eps, hi[1] + eps, hi[2] + eps, 0.0f);
}

// clip the line (o + t d) to the box; false if it misses
__device__ __forceinline__ bool clip_line(float3 o, float3 d, float4 lo, float4 hi, float &t0, float &t1)
{
    t0 = -INFINITY;
    t1 = INFINITY;
    const float oo[3] = { o.x, o.y, o.z }, dd[3] = { d.x, d.y, d.z };
    const float ll[3] = { lo.x, lo.y, lo.z }, hh[3] = { hi.x, hi.y, hi.z };
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (dd[c] == 0.0f) {
            if (oo[c] < ll[c] || oo[c] > hh[c]) return false;
        } else {
            const float inv = 1.0f / dd[c];
            const float a = (ll[c] - oo[c]) * inv, b = (hh[c] - oo[c]) * inv;
            t0 = fmaxf(t0, fminf(a, b));
            t1 = fminf(t1, fmaxf(a, b));
        }
    }
    return t0 <= t1;
}

// per block: reference line (p0, d0) and deviation dev; blk[2b] = (p0, dev),
// blk[2b+1] = (d0, 1) or (0, 0, 0, 0) for a block none of whose lines meets
// the scene box
__global__ void __launch_bounds__(RB) k_ray_blocks(const float4 *__restrict__ ro,
                                                   const float4 *__restrict__ rd, int64_t n,
                                                   const float4 *__restrict__ scene, float4 *blk,
                                                   float4 *wblk)
{
    __shared__ int s_hit[RB];
    __shared__ float s_dev[RB / 32];
    __shared__ float4 s_ref[2];
    const int64_t r = blockIdx.x * (int64_t)RB + threadIdx.x;
    const float4 lo = scene[0], hi = scene[1];
    float3 o = make_float3(0.0f, 0.0f, 0.0f), d = make_float3(0.0f, 0.0f, 1.0f);
    float t0 = 0.0f, t1 = 0.0f;
    bool hit = false;
    if (r < n) {
        const float4 a = __ldg(ro + r), b = __ldg(rd + r);
        o = make_float3(a.x, a.y, a.z);
        d = make_float3(b.x, b.y, b.z);
        hit = clip_line(o, d, lo, hi, t0, t1);
    }
    s_hit[threadIdx.x] = hit;
    // the same bound per warp (32 rays): used by the integration kernels to
    // skip, warp by warp, the Gaussians of the block's list that miss it
    {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const unsigned hb = __ballot_sync(0xffffffffu, hit);
        float4 wP = make_float4(0.0f, 0.0f, 0.0f, 0.0f), wD = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (hb) {
            const unsigned up = hb & 0xffff0000u;
            const int rl = __ffs(up ? up : hb) - 1;
            const float ax = __shfl_sync(0xffffffffu, o.x, rl), ay = __shfl_sync(0xffffffffu, o.y, rl),
                        az = __shfl_sync(0xffffffffu, o.z, rl);
            const float bxx = __shfl_sync(0xffffffffu, d.x, rl), byy = __shfl_sync(0xffffffffu, d.y, rl),
                        bzz = __shfl_sync(0xffffffffu, d.z, rl);
            const float cx = 0.5f * (lo.x + hi.x), cy = 0.5f * (lo.y + hi.y), cz = 0.5f * (lo.z + hi.z);
            const float s = (cx - ax) * bxx + (cy - ay) * byy + (cz - az) * bzz;
            wP = make_float4(ax + s * bxx, ay + s * byy, az + s * bzz, 0.0f);
            wD = make_float4(bxx, byy, bzz, 1.0f);
            float dv = 0.0f;
            if (hit) {
                const float3 d0 = make_float3(bxx, byy, bzz);
                const float3 ea = make_float3(o.x + t0 * d.x - wP.x, o.y + t0 * d.y - wP.y, o.z + t0 * d.z - wP.z);
                const float3 eb = make_float3(o.x + t1 * d.x - wP.x, o.y + t1 * d.y - wP.y, o.z + t1 * d.z - wP.z);
                dv = sqrtf(fmaxf(norm2(cross3(ea, d0)), norm2(cross3(eb, d0))));
            }
            for (int k = 16; k > 0; k >>= 1) dv = fmaxf(dv, __shfl_xor_sync(0xffffffffu, dv, k));
            wP.w = dv + lo.w;
        }
        if (lane == 0) {
            wblk[2 * ((size_t)blockIdx.x * (RB / 32) + w)] = wP;
            wblk[2 * ((size_t)blockIdx.x * (RB / 32) + w) + 1] = wD;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ref = -1;
        for (int j = 0; j < RB && ref < 0; j++) {
            const int k = (j + RB / 2) % RB;
            if (s_hit[k]) ref = k;
        }
        if (ref < 0) {
            s_ref[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            s_ref[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else {
            const int64_t rr = blockIdx.x * (int64_t)RB + ref;
            const float4 a = __ldg(ro + rr), b = __ldg(rd + rr);
            // point of the reference line nearest the scene centre
            const float cx = 0.5f * (lo.x + hi.x), cy = 0.5f * (lo.y + hi.y), cz = 0.5f * (lo.z + hi.z);
            const float s = (cx - a.x) * b.x + (cy - a.y) * b.y + (cz - a.z) * b.z;
            s_ref[0] = make_float4(a.x + s * b.x, a.y + s * b.y, a.z + s * b.z, 0.0f);
            s_ref[1] = make_float4(b.x, b.y, b.z, 1.0f);
        }
    }
    __syncthreads();
    const float4 P = s_ref[0], D = s_ref[1];
    float dev = 0.0f;
    if (hit && D.w != 0.0f) {
        const float3 d0 = make_float3(D.x, D.y, D.z);
        const float3 ea = make_float3(o.x + t0 * d.x - P.x, o.y + t0 * d.y - P.y, o.z + t0 * d.z - P.z);
        const float3 eb = make_float3(o.x + t1 * d.x - P.x, o.y + t1 * d.y - P.y, o.z + t1 * d.z - P.z);
        dev = sqrtf(fmaxf(norm2(cross3(ea, d0)), norm2(cross3(eb, d0))));
    }
    for (int k = 16; k > 0; k >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, k));
    if ((threadIdx.x & 31) == 0) s_dev[threadIdx.x >> 5] = dev;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < RB / 32; j++) dev = fmaxf(dev, s_dev[j]);
        blk[2 * blockIdx.x] = make_float4(P.x, P.y, P.z, dev + lo.w);
        blk[2 * blockIdx.x + 1] = D;
    }
}

// the block test, written with explicit IEEE operations so that the count
// and emit kernels take the same decision for every (block, Gaussian)
__device__ __forceinline__ bool block_hit(const float4 P, const float4 D, const float4 ball)
{
    const float vx = __fsub_rn(ball.x, P.x), vy = __fsub_rn(ball.y, P.y), vz = __fsub_rn(ball.z, P.z);
    const float cx = __fsub_rn(__fmul_rn(vy, D.z), __fmul_rn(vz, D.y));
    const float cy = __fsub_rn(__fmul_rn(vz, D.x), __fmul_rn(vx, D.z));
    const float cz = __fsub_rn(__fmul_rn(vx, D.y), __fmul_rn(vy, D.x));
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz));
    const float R = __fadd_rn(ball.w, P.w);
    return d2 <= __fmul_rn(R, R);
}

constexpr int WPB = RB / 32;   // warps (and lists) per ray block
static_assert(WPB == RAYS_WPB, "one list per warp of a ray block");

// ---- two-level cull: clusters of 32 bounding balls along a Morton curve ----
//
// The balls are sorted by the Morton code of their centres in the scene box;
// every 32 consecutive sorted balls form a cluster, bounded by a ball holding
// all of them (centre: the middle of their box, radius: the largest distance
// from it to a member's far side, widened by the scene's FP32 slack).  A
// member ball that meets a block's cylinder lies inside its cluster's ball,
// so the cluster meets it too: a ray block tests the clusters and then only
// the members of the clusters it meets.  Lists come out in cluster order and,
// within a cluster, in member order -- the same order in the count and the
// emit pass.
constexpr int CL = 32;         // balls per cluster
constexpr int BIN_BS = 128;    // one warp per ray block in the count and emit kernels

__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(const float4 *__restrict__ ball, int64_t n, const float4 *__restrict__ scene,
                         uint32_t *code, uint32_t *perm)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 lo = scene[0], hi = scene[1], b = ball[k];
    const float ex = hi.x - lo.x, ey = hi.y - lo.y, ez = hi.z - lo.z;
    const float fx = ex > 0.0f ? (b.x - lo.x) / ex : 0.0f;
    const float fy = ey > 0.0f ? (b.y - lo.y) / ey : 0.0f;
    const float fz = ez > 0.0f ? (b.z - lo.z) / ez : 0.0f;
    const uint32_t qx = (uint32_t)fminf(fmaxf(fx * 1023.0f, 0.0f), 1023.0f);
    const uint32_t qy = (uint32_t)fminf(fmaxf(fy * 1023.0f, 0.0f), 1023.0f);
    const uint32_t qz = (uint32_t)fminf(fmaxf(fz * 1023.0f, 0.0f), 1023.0f);
    code[k] = spread10(qx) | (spread10(qy) << 1) | (spread10(qz) << 2);
    perm[k] = (uint32_t)k;
}

// one warp per cluster: the sorted balls and ids, and the cluster ball
__global__ void k_clusters(const float4 *__restrict__ ball, const uint32_t *__restrict__ perm, int64_t n,
                           int64_t nc, const float4 *__restrict__ scene, float4 *sball, uint32_t *sgid,
                           float4 *cball)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= nc) return;
    const int64_t j = c * CL + lane;
    const bool valid = j < n;
    const uint32_t gid = valid ? __ldg(perm + j) : 0u;
    const float4 b = valid ? __ldg(ball + gid) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (valid) {
        sball[j] = b;
        sgid[j] = gid;
    }
    float lo[3] = { valid ? b.x - b.w : INFINITY, valid ? b.y - b.w : INFINITY, valid ? b.z - b.w : INFINITY };
    float hi[3] = { valid ? b.x + b.w : -INFINITY, valid ? b.y + b.w : -INFINITY, valid ? b.z + b.w : -INFINITY };
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    const float cx = 0.5f * (lo[0] + hi[0]), cy = 0.5f * (lo[1] + hi[1]), cz = 0.5f * (lo[2] + hi[2]);
    float r = 0.0f;
    if (valid) {
        const float dx = b.x - cx, dy = b.y - cy, dz = b.z - cz;
        r = sqrtf(dx * dx + dy * dy + dz * dz) + b.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) cball[c] = make_float4(cx, cy, cz, r * (1.0f + 2e-5f) + scene[0].w);
}

// Visit, in order, the members of the clusters that ray block (P, D) meets:
// visit(j, ball, hit) runs on every lane for every member slot j of such a
// cluster (hit: the slot holds a ball that passes the block's bound).
template <class F>
__device__ __forceinline__ void walk_clusters(const float4 P, const float4 D, const float4 *__restrict__ cball,
                                              const float4 *__restrict__ sball, int64_t n, int64_t nc,
                                              int lane, F visit)
{
    for (int64_t cb = 0; cb < nc; cb += 32) {
        const int64_t ci = cb + lane;
        const bool hc = ci < nc && block_hit(P, D, __ldg(cball + ci));
        uint32_t m = __ballot_sync(0xffffffffu, hc);
        while (m) {
            const int64_t c = cb + (__ffs(m) - 1);
            m &= m - 1u;
            const int64_t j = c * CL + lane;
            const bool valid = j < n;
            const float4 bl = valid ? __ldg(sball + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            visit(j, bl, valid && block_hit(P, D, bl));
        }
    }
}

// per block: how many Gaussians pass the block's bound and then each warp's
// bound; cnt[WPB b + w] = the length of warp w's list
__global__ void __launch_bounds__(BIN_BS) k_rays_count(const float4 *__restrict__ blk,
                                                       const float4 *__restrict__ wblk,
                                                       const float4 *__restrict__ cball,
                                                       const float4 *__restrict__ sball, int64_t n,
                                                       int64_t nc, int64_t T, uint32_t *cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * BIN_BS + threadIdx.x) >> 5;
    if (b >= T) return;
    const float4 P = blk[2 * b], D = blk[2 * b + 1];
    float4 wP[WPB], wD[WPB];
#pragma unroll
    for (int w = 0; w < WPB; w++) {
        wP[w] = wblk[2 * ((size_t)b * WPB + w)];
        wD[w] = wblk[2 * ((size_t)b * WPB + w) + 1];
    }
    uint32_t c[WPB] = {};
    if (D.w != 0.0f)
        walk_clusters(P, D, cball, sball, n, nc, lane, [&](int64_t j, float4 bl, bool hit) {
            (void)j;
            if (hit) {
#pragma unroll
                for (int w = 0; w < WPB; w++) c[w] += wD[w].w != 0.0f && block_hit(wP[w], wD[w], bl);
            }
        });
#pragma unroll
    for (int w = 0; w < WPB; w++) {
        uint32_t v = c[w];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == w) cnt[(size_t)b * WPB + w] = v;
    }
}

// blocks b0 .. b0 + nb - 1; off[] (per warp list) relative to the range
__global__ void __launch_bounds__(BIN_BS) k_rays_emit(const float4 *__restrict__ blk,
                                                      const float4 *__restrict__ wblk,
                                                      const float4 *__restrict__ cball,
                                                      const float4 *__restrict__ sball,
                                                      const uint32_t *__restrict__ sgid, int64_t n,
                                                      int64_t nc, int64_t b0, int64_t nb,
                                                      const uint32_t *__restrict__ off,
                                                      const uint32_t *__restrict__ cnt,
                                                      uint32_t *gids, uint2 *ranges)
{
    const int lane = threadIdx.x & 31;
    const int64_t bi = ((int64_t)blockIdx.x * BIN_BS + threadIdx.x) >> 5;   // block within the range
    if (bi >= nb) return;
    const int64_t b = b0 + bi;
    const float4 P = blk[2 * b], D = blk[2 * b + 1];
    float4 wP[WPB], wD[WPB];
    uint32_t beg[WPB], num[WPB], pos[WPB], total_num = 0;
#pragma unroll
    for (int w = 0; w < WPB; w++) {
        wP[w] = wblk[2 * ((size_t)b * WPB + w)];
        wD[w] = wblk[2 * ((size_t)b * WPB + w) + 1];
        beg[w] = off[(size_t)bi * WPB + w];
        num[w] = cnt[(size_t)b * WPB + w];
        pos[w] = beg[w];
        total_num += num[w];
    }
    if (lane < WPB) ranges[(size_t)bi * WPB + lane] = make_uint2(beg[lane], beg[lane] + num[lane]);
    if (D.w == 0.0f || total_num == 0) return;
    const uint32_t lt = (1u << lane) - 1u;
    walk_clusters(P, D, cball, sball, n, nc, lane, [&](int64_t j, float4 bl, bool hit) {
        const uint32_t gid = hit ? __ldg(sgid + j) : 0u;
#pragma unroll
        for (int w = 0; w < WPB; w++) {
            const bool h = hit && wD[w].w != 0.0f && block_hit(wP[w], wD[w], bl);
            const uint32_t bal = __ballot_sync(0xffffffffu, h);
            const uint32_t at = pos[w] + __popc(bal & lt);
            if (h && at < beg[w] + num[w]) gids[at] = gid;
            pos[w] += __popc(bal);
        }
    });
}

// a warp stages up to 32 records of its own list (lane i: entry beg + i):
// mu, rho, P, the id and the radius K sigma_max of the bounding ball
__device__ __forceinline__ void stage_warp(const float4 *__restrict__ rec,
                                           const uint32_t *__restrict__ gids, uint32_t beg, int cnt,
                                           int lane, SRec *sr)
{
    if (lane < cnt) {
        const uint32_t gid = __ldg(gids + beg + lane);
        const float4 *r = rec + REC_F4 * (size_t)gid;
        const float4 r2 = __ldg(r + 2);
        sr[lane].g0 = __ldg(r);
        sr[lane].g1 = __ldg(r + 1);
        sr[lane].g2 = make_float4(r2.x, r2.y, __uint_as_float(gid), BALL_K * __ldg(r + 4).x);
    }
    __syncwarp();
}

// Does the lane's line pass within the bounding ball (mu, rb) of a staged
// record?  A pair with m <= 9 has its line within 3 sigma_max of mu, inside
// the ball (K = 3.0104 sigma_max): a warp skips a record no lane's line meets
// before the closed form is evaluated.
__device__ __forceinline__ bool line_meets_ball(const Ray &ray, const SRec &s)
{
    const float ex = s.g0.x - ray.ox, ey = s.g0.y - ray.oy, ez = s.g0.z - ray.oz;
    const float cx = ey * ray.dz - ez * ray.dy, cy = ez * ray.dx - ex * ray.dz, cz = ex * ray.dy - ey * ray.dx;
    return cx * cx + cy * cy + cz * cz <= s.g2.w * s.g2.w;
}


__device__ __forceinline__ Ray load_ray(const float4 *ro, const float4 *rd, int64_t r)
{
    const float4 a = __ldg(ro + r), b = __ldg(rd + r);
    Ray y;
    y.ox = a.x; y.oy = a.y; y.oz = a.z; y.ta = a.w;
    y.dx = b.x; y.dy = b.y; y.dz = b.z; y.tb = b.w;
    return y;
}

// one ray per thread; blocks b0 .. b0 + gridDim.x - 1; every warp walks its
// own list (no barrier across the CTA)
template <int KER>
__global__ void __launch_bounds__(RB) k_rays_forward(const float4 *__restrict__ ro,
                                                     const float4 *__restrict__ rd,
                                                     const float2 *__restrict__ tof, int64_t n,
                                                     int64_t b0, const float4 *__restrict__ rec,
                                                     const uint32_t *__restrict__ gids,
                                                     const uint2 *__restrict__ ranges, float *out)
{
    __shared__ SRec sr_all[WPB][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SRec *sr = sr_all[w];
    const int64_t r = (b0 + blockIdx.x) * (int64_t)RB + threadIdx.x;
    const bool valid = r < n;
    const Ray ray = load_ray(ro, rd, valid ? r : 0);
    const float2 tf = tof && valid ? __ldg(tof + r) : make_float2(0.0f, 0.0f);
    const uint2 rg = ranges[(size_t)blockIdx.x * WPB + w];
    float acc = 0.0f;
    for (uint32_t c = rg.x; c < rg.y; c += 32) {
        const int cnt = (int)min(32u, rg.y - c);
        __syncwarp();
        stage_warp(rec, gids, c, cnt, lane, sr);
        for (int i = 0; i < cnt; i++) {
            if (!__any_sync(0xffffffffu, valid && line_meets_ball(ray, sr[i]))) continue;
            PairGeo q;
            pair_geo(ray, sr[i], q);
            if (q.m <= PAIR_CUT2) acc += general_value<KER>(q, sr[i].g0.w, tf.x, tf.y);
        }
    }
    if (valid) out[r] = acc;
}

// one ray per thread, warp-private lists; per Gaussian a transposed warp
// reduction of the pair gradients and one atomic per component per warp
template <int KER>
__global__ void __launch_bounds__(RB) k_rays_adjoint(const float4 *__restrict__ ro,
                                                     const float4 *__restrict__ rd,
                                                     const float2 *__restrict__ tof, int64_t n,
                                                     int64_t b0, const float4 *__restrict__ rec,
                                                     const uint32_t *__restrict__ gids,
                                                     const uint2 *__restrict__ ranges,
                                                     const float *__restrict__ dLdI, float *grad)
{
    __shared__ SRec sr_all[WPB][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SRec *sr = sr_all[w];
    const int64_t r = (b0 + blockIdx.x) * (int64_t)RB + threadIdx.x;
    const bool valid = r < n;
    const Ray ray = load_ray(ro, rd, valid ? r : 0);
    const float wgt = valid ? __ldg(dLdI + r) : 0.0f;
    const float2 tf = tof && valid ? __ldg(tof + r) : make_float2(0.0f, 0.0f);
    const uint2 rg = ranges[(size_t)blockIdx.x * WPB + w];
    // accumulator slot of general_grad's components: dmu[3], G_P[6], drho
    const int slot[NG_RAYS] = { 0, 1, 2, 4, 5, 6, 7, 8, 9, 3 };
    if (!__any_sync(0xffffffffu, wgt != 0.0f)) return;
    for (uint32_t c = rg.x; c < rg.y; c += 32) {
        const int cnt = (int)min(32u, rg.y - c);
        __syncwarp();
        stage_warp(rec, gids, c, cnt, lane, sr);
        for (int i = 0; i < cnt; i++) {
            if (!__any_sync(0xffffffffu, valid && wgt != 0.0f && line_meets_ball(ray, sr[i]))) continue;
            PairGeo q;
            pair_geo(ray, sr[i], q);
            const bool act = valid && wgt != 0.0f && q.m <= PAIR_CUT2;
            if (!__any_sync(0xffffffffu, act)) continue;
            float v[NG_RAYS];
            if (act) {
                general_grad<KER>(ray, q, sr[i].g0.w, wgt, v, tf.x, tf.y);
            } else {
#pragma unroll
                for (int k = 0; k < NG_RAYS; k++) v[k] = 0.0f;
            }
            const int own = tr_reduce<NG_RAYS>(v, lane);
            if (own < NG_RAYS) {
                const uint32_t gid = __float_as_uint(sr[i].g2.z);
                atomicAdd(grad + 4 * GRAD_F4 * (size_t)gid + slot[own], v[0]);
            }
        }
    }
}

}  // namespace

cudaError_t launch_rays_prep(const float *o3, const float *d3, const float *t2, const float *tof2, int64_t n,
                             float4 *ro, float4 *rd, float2 *tof, uint32_t *bad, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_rays_prep<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(o3, d3, t2, tof2, n, ro, rd, tof, bad);
    count_launches(1);
    return cudaGetLastError();
}

int rays_blocks(int64_t n) { return (int)((n + RB - 1) / RB); }

int rays_ball_parts(int64_t n)
{
    int64_t b = (n + CULL_BS - 1) / CULL_BS;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

namespace {
struct ClusterBufs {
    uint32_t *code, *perm, *code_alt, *perm_alt, *tmp, *sgid;
    float4 *sball, *cball;
};
ClusterBufs carve_clusters(void *base, int64_t n)
{
    const int64_t nc = (n + CL - 1) / CL;
    ClusterBufs c;
    float4 *f = (float4 *)base;
    c.sball = f;
    c.cball = f + n;
    // every u32 array starts on a 16-byte boundary (the sort reads its keys
    // with 16-byte loads and keeps 64-bit sums in its scratch)
    const int64_t n4 = (n + 3) & ~(int64_t)3;
    uint32_t *u = (uint32_t *)(c.cball + nc);
    c.code = u;
    c.perm = u + n4;
    c.code_alt = u + 2 * n4;
    c.perm_alt = u + 3 * n4;
    c.sgid = u + 4 * n4;
    c.tmp = u + 5 * n4;
    return c;
}
}  // namespace

size_t rays_cluster_bytes(int64_t n)
{
    const int64_t nc = (n + CL - 1) / CL;
    const int64_t n4 = (n + 3) & ~(int64_t)3;
    return sizeof(float4) * (size_t)(n + nc) + sizeof(uint32_t) * (size_t)(5 * n4) +
           sizeof(uint32_t) * sort_tmp_elems((uint32_t)n) + 64;
}

cudaError_t launch_rays_bin(const float4 *ro, const float4 *rd, int64_t n_rays, const float4 *rec,
                            int64_t n, float4 *ball, float4 *part, float4 *scene, float4 *blk,
                            float4 *wblk, void *clusters, uint32_t *cnt, cudaStream_t s)
{
    const int parts = rays_ball_parts(n);
    k_balls<<<parts, CULL_BS, 0, s>>>(rec, n, ball, part);
    k_scene<<<1, 32, 0, s>>>(part, parts, scene);
    const ClusterBufs cb = carve_clusters(clusters, n);
    const int64_t nc = (n + CL - 1) / CL;
    k_morton<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ball, n, scene, cb.code, cb.perm);
    count_launches(3);
    cudaError_t e = launch_sort(cb.code, cb.perm, cb.code_alt, cb.perm_alt, (uint32_t)n, 30, cb.tmp, s);
    if (e != cudaSuccess) return e;
    k_clusters<<<(unsigned)((nc * 32 + 127) / 128), 128, 0, s>>>(ball, cb.perm, n, nc, scene, cb.sball, cb.sgid,
                                                               cb.cball);
    const int T = rays_blocks(n_rays);
    k_ray_blocks<<<T, RB, 0, s>>>(ro, rd, n_rays, scene, blk, wblk);
    k_rays_count<<<(unsigned)(((int64_t)T * 32 + BIN_BS - 1) / BIN_BS), BIN_BS, 0, s>>>(blk, wblk, cb.cball,
                                                                                       cb.sball, n, nc, T, cnt);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_rays_emit(const float4 *blk, const float4 *wblk, const void *clusters, int64_t n, int64_t b0,
                             int nb, const uint32_t *off, const uint32_t *cnt, uint32_t *gids, uint2 *ranges,
                             cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    const ClusterBufs cb = carve_clusters(const_cast<void *>(clusters), n);
    const int64_t nc = (n + CL - 1) / CL;
    k_rays_emit<<<(unsigned)(((int64_t)nb * 32 + BIN_BS - 1) / BIN_BS), BIN_BS, 0, s>>>(
        blk, wblk, cb.cball, cb.sball, cb.sgid, n, nc, b0, nb, off, cnt, gids, ranges);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rays_forward(const float4 *ro, const float4 *rd, const float2 *tof, int64_t n_rays,
                                int64_t b0, int nb, const float4 *rec, const uint32_t *gids,
                                const uint2 *ranges, float *out, int ker, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    if (ker == 1) k_rays_forward<1><<<nb, RB, 0, s>>>(ro, rd, nullptr, n_rays, b0, rec, gids, ranges, out);
    else k_rays_forward<0><<<nb, RB, 0, s>>>(ro, rd, tof, n_rays, b0, rec, gids, ranges, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rays_adjoint(const float4 *ro, const float4 *rd, const float2 *tof, int64_t n_rays,
                                int64_t b0, int nb, const float4 *rec, const uint32_t *gids,
                                const uint2 *ranges, const float *dLdI, float4 *grad, int ker,
                                cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    if (ker == 1)
        k_rays_adjoint<1><<<nb, RB, 0, s>>>(ro, rd, nullptr, n_rays, b0, rec, gids, ranges, dLdI, (float *)grad);
    else
        k_rays_adjoint<0><<<nb, RB, 0, s>>>(ro, rd, tof, n_rays, b0, rec, gids, ranges, dLdI, (float *)grad);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rgrt
