// Voxelisation: the density field of the Gaussians, sum_g rho_g
// exp(-m_g(x)/2) with m_g(x) = (x - mu_g)^T P_g (x - mu_g) <= 9 (the cut of
// the projector), sampled at voxel centres -- the reconstructed volume.
//
// The grid is cut into bricks of 8 x 8 x 16 voxels, one CTA of 256 threads per
// brick, four voxels along z per thread (the exponent is a quadratic in z:
// its xy part is computed once per Gaussian and thread); each warp holds an
// 8 x 4 x 4 block.  Binning:
// per Gaussian the box mu +- sqrt(K^2 Sigma_aa) (K^2 = 9.0625) gives a voxel
// range per axis, hence a brick range; counts, exclusive scan, emission of
// (brick, Gaussian) pairs in Gaussian order, stable radix sort by brick and
// per-brick ranges give every brick its list in ascending Gaussian order.  The
// CTA walks its list in shared-memory chunks; a warp skips a Gaussian whose box
// misses its slab (warp-uniform branch).
#include "rgrt_internal.h"

namespace rgrt {
namespace {

constexpr int VB = 256;            // threads per brick
constexpr int VZ = 4;              // voxels per thread along z
constexpr int BZ = 4 * VZ;         // brick depth: 8 x 8 x 16 voxels
constexpr int VCH = 256;           // records per chunk
constexpr float NEG_HALF_LOG2E_V = -0.721347520444481703f;
constexpr float VOX_CUT_ARG = -6.49212768400033233f;  // -9 log2(e) / 2

// one Gaussian in shared memory; P carries the exponent's scale k
// (-log2(e)/2, or -1/kappa^2 for Epanechnikov)
struct VRecord {
    float4 g0;   // mu, rho
    float4 g1;   // k P00, 2k P01, k P11, 2k P02
    float4 g2;   // 2k P12, k P22, hx, hy   (h = half-widths of the K-sigma box)
    float4 g3;   // hz
};

__device__ __forceinline__ float ex2_fast(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// voxel index range [lo, hi] of the interval [c - h, c + h] on the axis
// x_i = o + i s (i in [0, n)); empty when lo > hi
__device__ __forceinline__ void axis_range(float c, float h, float o, float s, int n, int &lo, int &hi)
{
    const float a = (c - h - o) / s, b = (c + h - o) / s;
    if (!(a <= b) || b < -1.0f || a > (float)n) {   // empty (or NaN)
        lo = 1;
        hi = 0;
        return;
    }
    // one voxel of slack on each side covers the rounding of the division
    lo = max((int)floorf(fmaxf(a, -1.0f)), 0);
    hi = min((int)ceilf(fminf(b, (float)n)), n - 1);
}

__global__ void k_vox_count(const float4 *__restrict__ crec, int64_t n, VolDev v, uint32_t *cnt,
                            uint4 *bbox)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 c0 = __ldg(crec + CREC_F4 * k), c1 = __ldg(crec + CREC_F4 * k + 1),
                 c2 = __ldg(crec + CREC_F4 * k + 2);
    const float hx = sqrtf(CULL_K2 * c1.x), hy = sqrtf(CULL_K2 * c1.w), hz = sqrtf(CULL_K2 * c2.y);
    int i0, i1, j0, j1, k0, k1;
    axis_range(c0.x, hx, v.ox, v.sx, v.nx, i0, i1);
    axis_range(c0.y, hy, v.oy, v.sy, v.ny, j0, j1);
    axis_range(c0.z, hz, v.oz, v.sz, v.nz, k0, k1);
    uint32_t c = 0;
    uint4 b = make_uint4(1u, 0u, 0u, 0u);   // empty
    if (i0 <= i1 && j0 <= j1 && k0 <= k1) {
        const int bx0 = i0 >> 3, bx1 = i1 >> 3, by0 = j0 >> 3, by1 = j1 >> 3, bz0 = k0 / BZ, bz1 = k1 / BZ;
        c = (uint32_t)((bx1 - bx0 + 1) * (by1 - by0 + 1) * (bz1 - bz0 + 1));
        b = make_uint4((uint32_t)bx0 | ((uint32_t)bx1 << 16), (uint32_t)by0 | ((uint32_t)by1 << 16),
                       (uint32_t)bz0 | ((uint32_t)bz1 << 16), 0u);
    }
    cnt[k] = c;
    bbox[k] = b;
}

__global__ void k_vox_emit(int64_t n, VolDev v, const uint32_t *__restrict__ cnt,
                           const uint32_t *__restrict__ off, const uint4 *__restrict__ bbox,
                           uint32_t *keys, uint32_t *vals, uint32_t cap)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n || cnt[k] == 0) return;
    const uint4 b = bbox[k];
    const int bx0 = b.x & 0xffff, bx1 = b.x >> 16, by0 = b.y & 0xffff, by1 = b.y >> 16,
              bz0 = b.z & 0xffff, bz1 = b.z >> 16;
    uint32_t o = off[k];
    for (int bz = bz0; bz <= bz1; bz++)
        for (int by = by0; by <= by1; by++)
            for (int bx = bx0; bx <= bx1; bx++) {
                if (o < cap) {
                    keys[o] = ((uint32_t)bz * (uint32_t)v.by + (uint32_t)by) * (uint32_t)v.bx + (uint32_t)bx;
                    vals[o] = (uint32_t)k;
                }
                o++;
            }
}

__global__ void k_vox_ranges(const uint32_t *__restrict__ keys, uint32_t nk, uint2 *ranges, uint32_t nb)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk) return;
    const uint32_t b = keys[i];
    if (b >= nb) return;
    if (i == 0 || keys[i - 1] != b) ranges[b].x = i;
    if (i == nk - 1 || keys[i + 1] != b) ranges[b].y = i + 1;
}

template <int KER>
__global__ void __launch_bounds__(VB) k_voxelize(const float4 *__restrict__ rec,
                                                 const float4 *__restrict__ crec,
                                                 const uint32_t *__restrict__ gids,
                                                 const uint2 *__restrict__ ranges, VolDev v,
                                                 float *__restrict__ out)
{
    __shared__ VRecord sr[VCH];
    const uint32_t brick = blockIdx.x;
    const int bx = (int)(brick % (uint32_t)v.bx);
    const int by = (int)((brick / (uint32_t)v.bx) % (uint32_t)v.by);
    const int bz = (int)(brick / ((uint32_t)v.bx * (uint32_t)v.by));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // warp w: x 0..7 (lane & 7), y (w & 1) * 4 + lane >> 3, z (w >> 1) * VZ + 0..VZ-1
    const int i = bx * 8 + (lane & 7);
    const int j = by * 8 + (w & 1) * 4 + (lane >> 3);
    const int k0 = bz * BZ + (w >> 1) * VZ;
    const float x = v.ox + (float)i * v.sx, y = v.oy + (float)j * v.sy, z0 = v.oz + (float)k0 * v.sz;
    // the warp's block of 8 x 4 x VZ voxels: centre and half extents
    const float i0 = (float)(bx * 8), j0 = (float)(by * 8 + (w & 1) * 4);
    const float cx = v.ox + (i0 + 3.5f) * v.sx, cy = v.oy + (j0 + 1.5f) * v.sy;
    const float cz = z0 + 0.5f * (float)(VZ - 1) * v.sz;
    const float ex = 3.5f * v.sx, ey = 1.5f * v.sy, ez = 0.5f * (float)(VZ - 1) * v.sz;
    const uint2 rg = ranges[brick];
    float acc[VZ];
#pragma unroll
    for (int q = 0; q < VZ; q++) acc[q] = 0.0f;
    for (uint32_t c = rg.x; c < rg.y; c += VCH) {
        const int cnt = (int)min((uint32_t)VCH, rg.y - c);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += VB) {
            const uint32_t gid = __ldg(gids + c + t);
            const float4 *r = rec + REC_F4 * (size_t)gid;
            const float4 c1 = __ldg(crec + CREC_F4 * (size_t)gid + 1), c2 = __ldg(crec + CREC_F4 * (size_t)gid + 2);
            const float4 r1 = __ldg(r + 1), r2 = __ldg(r + 2);
            // the exponent's scale folded into P: arg = d^T (k P) d
            const float kk = KER == 1 ? -1.0f / 7.0f : NEG_HALF_LOG2E_V;
            sr[t].g0 = __ldg(r);
            sr[t].g1 = make_float4(kk * r1.x, 2.0f * kk * r1.y, kk * r1.w, 2.0f * kk * r1.z);   // P00 2P01 P11 2P02
            sr[t].g2 = make_float4(2.0f * kk * r2.x, kk * r2.y, sqrtf(CULL_K2 * c1.x), sqrtf(CULL_K2 * c1.w));
            sr[t].g3 = make_float4(sqrtf(CULL_K2 * c2.y), 0.0f, 0.0f, 0.0f);                       // 2P12 P22 hx hy | hz
        }
        __syncthreads();
        for (int t = 0; t < cnt; t++) {
            const float4 g0 = sr[t].g0, g2 = sr[t].g2;
            const float hz = sr[t].g3.x;
            // warp-uniform: skip a Gaussian whose box misses this warp's voxels
            if (fabsf(g0.x - cx) > g2.z + ex || fabsf(g0.y - cy) > g2.w + ey || fabsf(g0.z - cz) > hz + ez)
                continue;
            const float4 g1 = sr[t].g1;
            const float dx = x - g0.x, dy = y - g0.y;
            // arg(dz) = a0 + dz (b0 + c0 dz): the xy terms once, then VZ voxels along z
            const float a0 = dx * (g1.x * dx + g1.y * dy) + g1.z * dy * dy;
            const float b0 = g1.w * dx + g2.x * dy;
            const float c0 = g2.y;
#pragma unroll
            for (int q = 0; q < VZ; q++) {
                const float dz = z0 + (float)q * v.sz - g0.z;
                const float arg = a0 + dz * (b0 + c0 * dz);
                if (KER == 1) {
                    const float cc = 1.0f + arg;                // 1 - m / kappa^2
                    acc[q] += cc > 0.0f ? g0.w * cc : 0.0f;
                } else {
                    const float f = g0.w * ex2_fast(arg);
                    acc[q] += arg >= VOX_CUT_ARG ? f : 0.0f;
                }
            }
        }
    }
    if (i < v.nx && j < v.ny) {
#pragma unroll
        for (int q = 0; q < VZ; q++)
            if (k0 + q < v.nz) out[((int64_t)(k0 + q) * v.ny + j) * v.nx + i] = acc[q];
    }
}

}  // namespace

cudaError_t launch_vox_count(const float4 *crec, int64_t n, const VolDev &v, uint32_t *cnt, uint4 *bbox,
                             cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_vox_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(crec, n, v, cnt, bbox);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_vox_emit(int64_t n, const VolDev &v, const uint32_t *cnt, const uint32_t *off,
                            const uint4 *bbox, uint32_t *keys, uint32_t *vals, uint32_t cap, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_vox_emit<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, v, cnt, off, bbox, keys, vals, cap);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_vox_ranges(const uint32_t *keys, uint32_t nk, uint2 *ranges, uint32_t nb, cudaStream_t s)
{
    if (nk == 0) return cudaSuccess;
    k_vox_ranges<<<(nk + 255) / 256, 256, 0, s>>>(keys, nk, ranges, nb);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_voxelize(const float4 *rec, const float4 *crec, const uint32_t *gids, const uint2 *ranges,
                            const VolDev &v, float *out, int ker, cudaStream_t s)
{
    const int64_t nb = (int64_t)v.bx * v.by * v.bz;
    if (nb <= 0) return cudaSuccess;
    if (ker == 1) k_voxelize<1><<<(unsigned)nb, VB, 0, s>>>(rec, crec, gids, ranges, v, out);
    else k_voxelize<0><<<(unsigned)nb, VB, 0, s>>>(rec, crec, gids, ranges, v, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rgrt
