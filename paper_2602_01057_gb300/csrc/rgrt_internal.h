// Internal declarations shared by the CUDA translation units of librgrt.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rgrt.h"

namespace rgrt {

// Geometry as the kernels see it.  kind: 0 = parallel rays (CT parallel and
// the PET ring), 1 = cone beam, 2 = 3-D PET (LORs between two rings: their
// direction e_w + kappa e_v depends on the radial bin).  pet != 0 selects the
// PET chord segment between the ring's two crystals.  The output index of
// (view, row, col) is view stride_view + row stride_row + col.
constexpr int GM_PARALLEL = 0, GM_CONE = 1, GM_PET3D = 2;
struct DevGeom {
    int kind, pet;
    int n_views, n_rows, n_cols;  // 3-D PET: n_views counts (ring difference, angle) pairs
    int tile_w, tile_h, tiles_x, tiles_y;
    int v0;                       // first view of the current chunk
    long long stride_view, stride_row;
    float dso, dsd, t_a, t_b, radius2;
    int n_ang, max_rd;            // 3-D PET: angles per ring difference, largest ring difference
    float ring_pitch;             // 3-D PET: axial distance of neighbouring rings
    // first table value and inverse spacing of utab / vtab when uniformly
    // spaced (CT, arc-corrected PET radial bins, planes and rings), else 0
    float u0, uinv, v0f, vinv;
    const float *frames;          // n_views x 9 : e_u, e_v, e_w
    const float *utab;            // n_cols pixel u coordinates
    const float *vtab;            // n_rows pixel v coordinates (3-D PET: ring heights)
    // time of flight (PET ring): n_tof bins (0: none) centred at
    // tof_t0 + k tof_h along the LOR from its midpoint, 1/sigma^2 = tof_tau,
    // sigma^2 = tof_s2; output of bin k at k stride_tof + the LOR's index
    int n_tof;
    float tof_t0, tof_h, tof_tau, tof_s2;
    long long stride_tof;
};

constexpr int TOF_MAX = RGRT_TOF_MAX_BINS;

// 3-D PET: ring difference of view `view`
__host__ __device__ inline int pet3d_delta(const DevGeom &g, int view) { return view / g.n_ang - g.max_rd; }

// Views of a description (3-D PET: one per ring difference and angle) and
// its rays.
int64_t desc_views(const rgrt_geom_desc *d);
int64_t desc_rays(const rgrt_geom_desc *d);
// Host tables of a validated description -- frames [views x 9], u [n_cols],
// v [n_rows], the binary32 rounding of the binary64 geometry -- into tab
// (9 views + n_cols + n_rows floats), and every field of dg but the table
// pointers.
void geom_tables(const rgrt_geom_desc *d, float *tab, DevGeom &dg);

// Per-Gaussian records built once per parameter version.
//   rec  : 5 float4 = (mu, rho), (P00 P01 P02 P11), (P12 P22 S00 S01),
//          (S02 S11 S12 S22), (sigma_max, 0, 0, 0);  P = Sigma^-1, S = Sigma/det Sigma
//   crec : 3 float4 = (mu, 0), (Sig00 Sig01 Sig02 Sig11), (Sig12 Sig22 0 0)
//          -- the FP32 culling record, bit-exact by specification.
constexpr int REC_F4 = 5;
constexpr int CREC_F4 = 3;

// Gradient accumulator per Gaussian: 4 float4 =
//   (dmu, drho), (GP00 GP01 GP02 GP11), (GP12 GP22 GS00 GS01), (GS02 GS11 GS12 GS22)
// GP, GS: symmetric-matrix gradients w.r.t. P and S (entry (a,b) == (b,a)).
constexpr int GRAD_F4 = 4;

// culling constant K^2 (K = 3.0104, a margin over the 3-sigma pair cut)
constexpr float CULL_K2 = 9.0625f;
// pair cut-off: m <= 9
constexpr float PAIR_CUT2 = 9.0f;

struct Stats {
    unsigned long long pairs_eval, pairs_kept;
};

// number of kernels the library has launched (all contexts, all threads)
void count_launches(int k);

// geometry validation and the thread-local error message of the C ABI
int validate_geometry(const rgrt_geom_desc *d);
int report_error(int code, const char *msg);

// ---- launchers (each returns cudaGetLastError of its launch) -------------
// bad (nullable): set to nonzero when a parameter is not finite
cudaError_t launch_records(const float *mu, const float *ls, const float *q, const float *rho,
                           int64_t n, float4 *rec, float4 *crec, uint32_t *bad, cudaStream_t s);
cudaError_t launch_cull(const DevGeom &g, int nv, const float4 *crec, int64_t n, uint32_t *cnt,
                        uint2 *rect, cudaStream_t s);
// key = tile field << 8 | position code; lbits >= 0: the tile field is
// (view << lbits) | tile within the view, for launch_sort_views; lbits < 0:
// the tile id view * tiles per view + tile
cudaError_t launch_emit(const DevGeom &g, int nv, int64_t n, const uint32_t *cnt,
                        const uint32_t *off, const uint2 *rect, uint32_t *keys, uint32_t *vals,
                        uint32_t cap, uint32_t *overflow, cudaStream_t s, int lbits = -1);
// n_dev (nullable): the number of sorted keys, read on the device (<= n_keys);
// tpv, lbits: tiles per view and the emit's lbits (the tile field decoded to
// view * tpv + tile when lbits >= 0)
cudaError_t launch_ranges(const uint32_t *keys, uint32_t n_keys, uint2 *ranges, uint32_t n_tiles,
                          cudaStream_t s, const unsigned long long *n_dev = nullptr, uint32_t tpv = 0,
                          int lbits = -1);

// exclusive scan of n u32 values; writes out[0..n) and the 64-bit total to
// *total (device).  tmp must hold scan_tmp_elems(n) u64.
size_t scan_tmp_elems(int64_t n);
cudaError_t launch_scan(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *total,
                        unsigned long long *tmp, cudaStream_t s);

// stable LSD radix sort of (keys, vals) by the low `bits` key bits; results
// end in (keys, vals) (alt buffers are scratch).  tmp must hold
// sort_tmp_elems(n) u32 (sort_tmp_elems(n, nv) for launch_sort_views).
size_t sort_tmp_elems(uint32_t n, int nv = 0);
// in_alt (nullable): set when the result is left in (keys_alt, vals_alt)
// instead of being copied back (an odd number of passes).  n_dev (nullable):
// sort only the first min(n, *n_dev) keys, the count read on the device
// (buffers and launches sized for n, e.g. inside a captured graph)
cudaError_t launch_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                        uint32_t n, int bits, uint32_t *tmp, cudaStream_t s, bool *in_alt = nullptr,
                        const unsigned long long *n_dev = nullptr);
// The same sort, view by view: the emitted keys are grouped by view (view v's
// keys start at off[v stride], the scan of the per-(view, Gaussian) counts),
// and each view's keys are sorted on their own by their low `bits` bits --
// the tile within the view and the position code, with keys emitted with
// lbits = bits - 8 -- which takes fewer passes than sorting on the view too.
cudaError_t launch_sort_views(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                              uint32_t n, int bits, const uint32_t *off, int64_t stride, int nv,
                              uint32_t *tmp, cudaStream_t s, bool *in_alt = nullptr,
                              const unsigned long long *n_dev = nullptr);

// ker: kernel of the primitives (RGRT_KERNEL_GAUSSIAN / RGRT_KERNEL_EPANECHNIKOV)
cudaError_t launch_forward(const DevGeom &g, int nv, const float4 *rec, const float4 *crec,
                           const uint32_t *gids, const uint2 *ranges, float *out, Stats *stats,
                           int ker, cudaStream_t s);
cudaError_t launch_adjoint(const DevGeom &g, int nv, const float4 *rec, const float4 *crec,
                           const uint32_t *gids, const uint2 *ranges, const float *dLdI,
                           float4 *grad, int ker, cudaStream_t s);
// one scan of a batch, as the persistent kernels see it
struct ScanDesc {
    DevGeom g;
    const float4 *rec, *crec;
    const uint32_t *gids;
    const uint2 *ranges;
    float *out;             // forward output
    const float *dLdI;      // adjoint input
    float4 *grad;           // adjoint accumulator
    uint32_t item_begin;    // first (scan, tile) work item of the scan
    uint32_t n_items;       // tiles of the scan
};
// persistent integration / adjoint over every tile of a batch of scans; the
// queue counter must be zero at launch.  tile_threads = tile_w * tile_h of
// every scan (one ray per thread in the forward).
cudaError_t launch_forward_persistent(bool cone, const ScanDesc *d, int nscan, uint32_t total,
                                      uint32_t *queue, int tile_threads, int grid, cudaStream_t s);
cudaError_t launch_adjoint_persistent(bool cone, int tile_w, const ScanDesc *d, int nscan,
                                      uint32_t total, uint32_t *queue, int grid, cudaStream_t s);
// CTAs of a persistent launch: SMs x resident CTAs per SM
int persistent_grid(bool forward, bool cone, int tile_w, int tile_threads);

cudaError_t launch_param_chain(const float *mu, const float *ls, const float *q, const float *rho,
                               int64_t n, const float4 *grad, float *g_mu, float *g_ls,
                               float *g_q, float *g_rho, cudaStream_t s);
// acc (nullable): device double the step's total is accumulated in (the
// loss of several ray ranges); loss_out then receives the running total
cudaError_t launch_loss(int kind, const float *I, const float *y, int64_t n, float kappa,
                        float eps, const float *mult, const float *add, float *dLdI, double *partial,
                        int nblk, float *loss_out, cudaStream_t s, double *acc = nullptr);
int loss_blocks(int64_t n);
// Adam; bc_dev (optional) supplies the bias corrections (1 - beta^t) from
// device memory instead of bc1, bc2; skip (optional) leaves everything
// unchanged when *skip != 0
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr,
                        float beta1, float beta2, float eps, float bc1, float bc2,
                        const float *bc_dev, const uint32_t *skip, cudaStream_t s);

// ---- explicit rays (rays.cu) ----------------------------------------------
// ro[r] = (o', t_a'), rd[r] = (unit d, t_b'), o' re-based at the point of the
// line nearest the world origin; *bad |= 1 for an invalid ray
// tof2 (nullable): per ray (t_c, sigma_T) -> tof[r] = (t_c re-based, 1/sigma_T^2 or 0)
cudaError_t launch_rays_prep(const float *o3, const float *d3, const float *t2, const float *tof2, int64_t n,
                             float4 *ro, float4 *rd, float2 *tof, uint32_t *bad, cudaStream_t s);
int rays_blocks(int64_t n_rays);       // ray blocks (128 rays each)
int rays_ball_parts(int64_t n);        // partial scene boxes of the ball pass
// balls (n float4), partial boxes (2 x parts), scene box (2), block lines
// (2 x blocks) and per-block Gaussian counts
// wblk: the same bound per 32-ray warp (4 per block, 2 float4 each)
// clusters: scratch of rays_cluster_bytes(n) bytes (the bounding balls in
// Morton order, their ids, the cluster balls and the sort's buffers)
size_t rays_cluster_bytes(int64_t n);
cudaError_t launch_rays_bin(const float4 *ro, const float4 *rd, int64_t n_rays, const float4 *rec,
                            int64_t n, float4 *ball, float4 *part, float4 *scene, float4 *blk,
                            float4 *wblk, void *clusters, uint32_t *cnt, cudaStream_t s);
// per-warp lists (RAYS_WPB per block; clusters in Morton order, members in
// order) of blocks b0 .. b0+nb-1 at offsets off[0 .. RAYS_WPB nb); cnt holds
// RAYS_WPB counts per block
constexpr int RAYS_WPB = 4;
cudaError_t launch_rays_emit(const float4 *blk, const float4 *wblk, const void *clusters, int64_t n, int64_t b0,
                             int nb, const uint32_t *off, const uint32_t *cnt, uint32_t *gids, uint2 *ranges,
                             cudaStream_t s);
// tof (nullable, Gaussian kernel only): per ray (t_c, tau)
cudaError_t launch_rays_forward(const float4 *ro, const float4 *rd, const float2 *tof, int64_t n_rays,
                                int64_t b0, int nb, const float4 *rec, const uint32_t *gids,
                                const uint2 *ranges, float *out, int ker, cudaStream_t s);
cudaError_t launch_rays_adjoint(const float4 *ro, const float4 *rd, const float2 *tof, int64_t n_rays,
                                int64_t b0, int nb, const float4 *rec, const uint32_t *gids,
                                const uint2 *ranges, const float *dLdI, float4 *grad, int ker,
                                cudaStream_t s);

// ---- voxelisation (voxel.cu) ----------------------------------------------
// voxel (i, j, k) centre = (ox + i sx, oy + j sy, oz + k sz); bricks of
// 8 x 8 x 16 voxels, bx x by x bz of them
struct VolDev {
    float ox, oy, oz, sx, sy, sz;
    int nx, ny, nz, bx, by, bz;
};
// per Gaussian: number of bricks its K-sigma box touches and their range
cudaError_t launch_vox_count(const float4 *crec, int64_t n, const VolDev &v, uint32_t *cnt, uint4 *bbox,
                             cudaStream_t s);
cudaError_t launch_vox_emit(int64_t n, const VolDev &v, const uint32_t *cnt, const uint32_t *off,
                            const uint4 *bbox, uint32_t *keys, uint32_t *vals, uint32_t cap, cudaStream_t s);
// ranges[b] = [first, last + 1) of brick b in the sorted keys (zeroed first)
cudaError_t launch_vox_ranges(const uint32_t *keys, uint32_t nk, uint2 *ranges, uint32_t nb, cudaStream_t s);
cudaError_t launch_voxelize(const float4 *rec, const float4 *crec, const uint32_t *gids, const uint2 *ranges,
                            const VolDev &v, float *out, int ker, cudaStream_t s);

}  // namespace rgrt
