/*
 * rgrt.h -- C ABI of the GB300 analytic Gaussian ray-tracing projector.
 *
 * The library projects a set of anisotropic 3D Gaussians along the rays of a
 * CT (parallel- or cone-beam) or PET (ring, arc-corrected or raw-chord)
 * geometry and back-propagates a loss to the Gaussian parameters.  It follows
 * the problem statement of "Radioactive 3D Gaussian Ray Tracing for
 * Tomographic Reconstruction", section 3:
 *   Gaussian     G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)),
 *                Sigma = R S S^T R^T                            (Eq. 2)
 *   ray          r(t) = o + t d                                  (Eq. 3)
 *   projection   I(r) = sum_i rho_i int G_i(o + t d) dt          (Eq. 4)
 *   closed form  rho sqrt(2 pi/A) exp(-1/2 (C - B^2/A))          (Eqs. 7-12)
 * with erf terms where the ray segment is finite, and Gaussians whose
 * contribution is negligible skipped (section 4.1, implementation details):
 * a pair counts when C - B^2/A <= 9 (the ray meets the 3-sigma ellipsoid).
 *
 * Parameterisation (per Gaussian, FP32):
 *   mu[3]         centre
 *   logscale[3]   l, with S = diag(exp(l))
 *   quat[4]       (w, x, y, z), normalised inside R(q); gradients are taken
 *                 with respect to the unnormalised q
 *   rho           density scale (the normalisation of Eq. 2 is absorbed in it)
 * Arrays are structure-of-arrays, contiguous: mu[n][3], logscale[n][3],
 * quat[n][4], rho[n].
 *
 * Memory: every pointer argument may be host memory (pageable or pinned) or
 * device memory of the context's device; the library detects which and
 * copies host data through its own device buffers, stream-ordered.  Device
 * buffers passed in stay owned by the caller.  The library owns the
 * Gaussians it copies (RGRT_COPY), their Adam state, and its binning scratch,
 * all counted against the context's HBM budget.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 * enqueue work on it; project_forward and project_backward read one 8-byte
 * count back from the device per binning pass (a short synchronisation on
 * that stream).  Results written to host pointers are complete on return.
 *
 * Errors: every call returns RGRT_OK (0) or a negative code; the message of
 * the last failure on the calling thread is returned by rgrt_last_error().
 * No call aborts the process or lets a C++ exception cross the ABI.
 */
#ifndef RGRT_H
#define RGRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------- */
#define RGRT_OK 0
#define RGRT_E_INVAL -1     /* bad argument: shape, null pointer, non-finite geometry */
#define RGRT_E_NOMEM -2     /* request exceeds the context's HBM budget, or cudaMalloc failed */
#define RGRT_E_CAPACITY -3  /* one view's tile lists do not fit the budget */
#define RGRT_E_CUDA -4      /* a CUDA runtime call failed (message names it) */
#define RGRT_E_TIMEOUT -5   /* a bounded device-side wait gave up */

/* ---- flags ---------------------------------------------------------- */
#define RGRT_COPY 0     /* gaussians_create: the library keeps its own device copy */
#define RGRT_BORROW 1   /* gaussians_create: wrap the caller's device arrays (must stay alive) */

#define RGRT_LOSS_L2 0       /* L = 1/2 sum (I - y)^2 */
#define RGRT_LOSS_POISSON 1  /* L = sum (k I + e - y log(k I + e)), k = kappa, e = eps */

/* kernel of the primitives (gaussians_set_kernel) */
#define RGRT_KERNEL_GAUSSIAN 0      /* rho exp(-m/2), Eq. 2; pairs with m <= 9 count */
#define RGRT_KERNEL_EPANECHNIKOV 1  /* rho (1 - m/7)_+: compact support, covariance Sigma */

#define RGRT_GEOM_CT_PARALLEL 0
#define RGRT_GEOM_CT_CONE 1
#define RGRT_GEOM_PET_RING 2
#define RGRT_GEOM_PET_3D 3

typedef struct rgrt_ctx rgrt_ctx;
typedef struct rgrt_gauss rgrt_gauss;
typedef struct rgrt_geom rgrt_geom;

/*
 * Geometry description (section 3 "Inherent limitations": cone/parallel-beam
 * CT and PET with arc correction; the constants are the caller's).
 *
 * CT frame of view k (angle th = angles[k]): e_w = (cos th, sin th, 0) from
 * source to detector, e_u = (-sin th, cos th, 0), e_v = (0, 0, 1); detector
 * pixel (row j, col i) at u_i = (i - (n_cols-1)/2) pitch_u,
 * v_j = (j - (n_rows-1)/2) pitch_v.
 *   CT_PARALLEL  ray o = u e_u + v e_v, d = e_w, t in [t_a, t_b].
 *   CT_CONE      source S = -dso e_w, pixel D = S + dsd e_w + u e_u + v e_v;
 *                the ray runs from S to D.
 * PET frame of angle k: phi = pi k / n_views (phi = angles[k] when angles
 * is not null, e.g. a subset of a sinogram's angles), e_u = (cos phi, sin phi, 0),
 * e_v = (0,0,1), e_w = (sin phi, -cos phi, 0); radial bin i at
 *   arc_mode 0 (arc-corrected): s_i = (i - c) pi radius / n_crystals
 *   arc_mode 1 (raw chords):    s_i = radius sin((i - c) pi / n_crystals)
 * with c = (n_cols-1)/2, plane j at z_j = (j - (n_rows-1)/2) pitch_v; the
 * line of response o = s e_u + z e_v, d = e_w runs over the chord
 * t in [-sqrt(radius^2 - s^2), +sqrt(radius^2 - s^2)].
 * PET_3D (fully 3-D sinograms, the oblique LORs of section 3's geometric
 * flexibility): n_rows rings at z_r = (r - (n_rows-1)/2) pitch_v, the angles
 * and radial bins of PET_RING, and one view per (ring difference delta in
 * [-max_ring_diff, max_ring_diff], angle): view = (delta + max_ring_diff)
 * n_views + angle.  Row j of a view is the ring pair (r1, r2) = (j, j +
 * delta) for delta >= 0, (j - delta, j) otherwise; the LOR runs from
 * s e_u - h e_w + z_r1 e_v to s e_u + h e_w + z_r2 e_v, h = sqrt(radius^2 -
 * s^2).  Rows j >= n_rows - |delta| have no ring pair: their output is 0 and
 * they take no gradient.
 * Output layout: CT I[view][row][col]; PET I[plane][angle][radial];
 * PET_3D I[delta][angle][ring pair][radial]
 * ((2 max_ring_diff + 1) n_views n_rows n_cols values).
 * tile_w/tile_h: binning tile in pixels (width 8, 16 or 32, height 4..32 in
 * steps of 4, 32..256 pixels; 0 = 16).
 */
typedef struct {
    int32_t kind;        /* RGRT_GEOM_* */
    int32_t n_views;     /* CT projections / PET sinogram angles (PET_3D: per ring difference) */
    int32_t n_rows;      /* CT detector rows / PET planes / PET_3D rings */
    int32_t n_cols;      /* CT detector columns / PET radial bins */
    const double *angles;/* CT: n_views angles in radians (host memory); PET: null or n_views angles */
    double pitch_u, pitch_v;
    double t_a, t_b;     /* CT_PARALLEL segment */
    double dso, dsd;     /* CT_CONE source-origin and source-detector distances */
    double radius;       /* PET ring radius */
    int32_t n_crystals;  /* PET crystals per ring */
    int32_t arc_mode;    /* PET: 0 arc-corrected, 1 raw chord positions */
    int32_t tile_w, tile_h;
    int32_t max_ring_diff; /* PET_3D: largest ring difference, 0..n_rows-1 (other kinds: ignored) */
} rgrt_geom_desc;

/* Adam hyper-parameters of loss_step (Kingma & Ba; the paper trains with
 * Adam, section 4.1, and states no values). */
typedef struct {
    float lr_mu, lr_logscale, lr_quat, lr_rho;
    float beta1, beta2, eps;
    float kappa, poisson_eps; /* RGRT_LOSS_POISSON only */
} rgrt_adam;

/* ---- context -------------------------------------------------------- */

/* Create a context on CUDA device `device` whose device allocations stay
 * within hbm_budget_bytes (0 = 90% of the free memory at creation).
 * Returns RGRT_E_INVAL for a bad device, RGRT_E_CUDA on a runtime failure. */
int rgrt_ctx_create(rgrt_ctx **out, int device, size_t hbm_budget_bytes);
/* Free every buffer of the context (Gaussians and geometries made from it
 * must be destroyed first). */
int rgrt_ctx_destroy(rgrt_ctx *ctx);

/* ---- Gaussians (Eq. 2) ---------------------------------------------- */

/* Register n Gaussians.  flags = RGRT_COPY copies the four arrays (host or
 * device) into library-owned device memory; RGRT_BORROW keeps the caller's
 * device pointers (n may be 0).  RGRT_E_INVAL for n < 0, a null array with
 * n > 0, or BORROW of host memory. */
int gaussians_create(rgrt_ctx *ctx, int64_t n, const float *mu3, const float *logscale3,
                     const float *quat4, const float *rho, int flags, rgrt_gauss **out);
int gaussians_destroy(rgrt_gauss *g);
/* Select the kernel of the primitives (RGRT_KERNEL_*; default Gaussian).
 * Section 2 names the Epanechnikov kernel as an alternative that ray tracing
 * can use: rho (1 - m(x)/kappa^2)_+ with m(x) the Mahalanobis distance
 * squared under Sigma and kappa^2 = 7 (its normalised form has covariance
 * Sigma); its line integral is rho (4 kappa/3) c^{3/2} / sqrt(A),
 * c = 1 - m/kappa^2, on a line, and a polynomial over a finite segment.
 * Every projector and voxeliser call honours it except the batch calls,
 * which reject non-Gaussian sets.  RGRT_E_INVAL for an unknown kernel. */
int gaussians_set_kernel(rgrt_gauss *g, int kernel);

/* Copy the current parameters out (host or device pointers; null skips). */
int gaussians_get(rgrt_gauss *g, float *mu3, float *logscale3, float *quat4, float *rho, void *stream);
/* Overwrite the parameters (host or device pointers; null keeps the old). */
int gaussians_set(rgrt_gauss *g, const float *mu3, const float *logscale3, const float *quat4,
                  const float *rho, void *stream);
int64_t gaussians_count(const rgrt_gauss *g);

/* ---- geometry (Eq. 3, section 3 arc correction) --------------------- */

/* Validate the description and upload its tables (view frames, pixel
 * coordinates).  RGRT_E_INVAL for non-positive sizes, non-finite or
 * degenerate constants (dsd <= dso <= 0, radius^2 < s^2 of a bin, ...). */
int geometry_set(rgrt_ctx *ctx, const rgrt_geom_desc *desc, rgrt_geom **out);
int geometry_destroy(rgrt_geom *g);
/* Explicit rays (any set of lines, e.g. a helical cone-beam trajectory or
 * list-mode events): ray r is the line through o3[3r..3r+2] along
 * d3[3r..3r+2] (any nonzero length; the library normalises it), integrated
 * over t in [t2[2r], t2[2r+1]], t measured along the unit direction from o
 * (either end may be infinite).  The arrays may be host or device memory and
 * are copied.  Projections I[n_rays] follow the rays' order; consecutive rays
 * are binned in blocks of 128, so keeping neighbouring rays close makes the
 * binning tight (incoherent rays still give the exact result, more slowly).
 * Explicit-ray geometries work with every projector call except the batch
 * calls.  RGRT_E_INVAL for n_rays <= 0, a null array, a non-finite origin, a
 * zero or non-finite direction, or a NaN or reversed segment.  This is the
 * ray-level form of Eq. 3 (o + t d) with no detector structure. */
int geometry_set_rays(rgrt_ctx *ctx, int64_t n_rays, const float *o3, const float *d3,
                      const float *t2, rgrt_geom **out);

/* Explicit rays with time of flight (TOF PET, which the paper's future-work
 * section plans): as geometry_set_rays, plus tof2[2r] = t_c, the centre of
 * ray r's Gaussian TOF kernel N(t; t_c, sigma_T^2) along the ray (t as in
 * t2) and tof2[2r + 1] = sigma_T (<= 0 or infinite: no weight for that
 * ray).  The weighted line integral keeps the closed form of Eqs. 7-12 with
 * A + 1/sigma_T^2, B - t_c/sigma_T^2, C + t_c^2/sigma_T^2 and the factor
 * 1/(sqrt(2 pi) sigma_T); a pair still counts by its spatial m <= 9.
 * Gaussian kernel only (projections of an Epanechnikov set return
 * RGRT_E_INVAL).  RGRT_E_INVAL also for a NaN width or centre. */
int geometry_set_rays_tof(rgrt_ctx *ctx, int64_t n_rays, const float *o3, const float *d3,
                          const float *t2, const float *tof2, rgrt_geom **out);

/* Largest number of time-of-flight bins per LOR of a sinogram geometry. */
#define RGRT_TOF_MAX_BINS 16

/* Time of flight on a PET ring sinogram (RGRT_GEOM_PET_RING; the paper's
 * future-work section plans TOF PET): every LOR is measured in n_tof bins
 * (1..RGRT_TOF_MAX_BINS), bin k weighting the line by the Gaussian kernel
 * N(t; t_k, sigma^2) with t measured along the LOR from its midpoint (the
 * transaxial plane's chord centre) and t_k = (k - (n_tof - 1)/2) spacing
 * (same length unit as the geometry).  The outputs become n_tof per LOR,
 * bin outermost: I[bin][plane][angle][radial] (geometry_num_rays = n_tof x
 * sinogram size), as do the losses' measurements and the measurement model's
 * arrays (set those after this call).  Tile lists are those of the sinogram
 * (one binning serves every bin).  A pair still counts by its spatial
 * m <= 9.  Gaussian kernel only (projections of an Epanechnikov set return
 * RGRT_E_INVAL).  RGRT_E_INVAL for another geometry kind, a bin count out
 * of range, or a spacing or width that is not positive and finite. */
int geometry_set_tof(rgrt_geom *g, int n_tof, float spacing, float sigma);

/* Outputs of a geometry: rays, or (time-of-flight bin, LOR) pairs. */
int64_t geometry_num_rays(const rgrt_geom *g);

/* Measurement model of the losses (the attenuation, scatter and randoms that
 * the paper's future-work section plans to model in the pipeline): per ray a
 * multiplicative factor mult[r] (attenuation, detector efficiency) and an
 * additive background add[r] (scatter + randoms, in counts), both
 * geometry_num_rays floats, host or device, copied; null = none (1 / 0).
 * loss_step, loss_grad and the batch calls then use the prediction
 * mult I + add (L2) or the mean kappa mult I + add + eps (Poisson), with
 * dL/dI carrying the factor mult.  The projector calls are unaffected.  Set
 * them before creating a batch that uses the geometry. */
int geometry_set_corrections(rgrt_geom *g, const float *mult, const float *add);

/* ---- projector (Eqs. 4, 11, 12) ------------------------------------- */

/* out_I[geometry_num_rays] = sum over Gaussians of rho sqrt(2 pi/A)
 * exp(-m/2) Phi, Phi the erf factor of the finite segment.  Overwrites. */
int project_forward(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, float *out_I,
                    void *stream);

/* Adjoint of project_forward: given dL/dI[geometry_num_rays], writes dL/dmu,
 * dL/dlogscale, dL/dquat, dL/drho (overwrite, not accumulate; a null output
 * is skipped).  The tile lists of the last project_forward of the same
 * (Gaussians, geometry) are reused when the parameters are unchanged and the
 * budget allowed keeping them; otherwise they are rebuilt. */
int project_backward(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom,
                     const float *dL_dI, float *g_mu3, float *g_logscale3, float *g_quat4,
                     float *g_rho, void *stream);

/* One optimisation step: forward, loss and dL/dI against measurements
 * y[geometry_num_rays], adjoint, and an Adam update of the Gaussians in
 * place (Adam state kept on the device with the Gaussians).  t = step
 * number (>= 1) for bias correction.  loss_out (host or device, may be
 * null) receives the loss as a float. */
int loss_step(rgrt_ctx *ctx, rgrt_gauss *g, const rgrt_geom *geom, const float *y, int loss,
              const rgrt_adam *hp, int t, float *loss_out, void *stream);

/* Loss and its gradient without an update: forward, loss against
 * y[geometry_num_rays] (only kappa and poisson_eps of hp are read), dL/dI,
 * adjoint and parameter chain; writes dL/dmu, dL/dlogscale, dL/dquat, dL/drho
 * (host or device; null skips) and the loss (host or device, may be null).
 * The Gaussians are not changed.  For callers that run their own optimiser.
 * Errors as loss_step. */
int loss_grad(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, const float *y, int loss,
              const rgrt_adam *hp, float *loss_out, float *g_mu3, float *g_logscale3,
              float *g_quat4, float *g_rho, void *stream);

/* ---- voxelisation ---------------------------------------------------- */

/* Regular voxel grid: voxel (i, j, k) has its centre at
 * origin + (i size[0], j size[1], k size[2]); dims = (nx, ny, nz). */
typedef struct {
    double origin[3];
    double size[3];      /* > 0 */
    int32_t dims[3];     /* > 0, each <= 65535 x 8 */
} rgrt_volume_desc;

/* The reconstructed volume: out[k][j][i] = sum over Gaussians of
 * rho exp(-(x - mu)^T Sigma^-1 (x - mu) / 2) at voxel centre x (the integrand
 * of Eq. 4 with the Gaussians of Eq. 2), with the projector's cut (a Gaussian
 * counts where that exponent's argument m <= 9).  out: nx ny nz floats, host
 * or device.  RGRT_E_INVAL for a bad grid, RGRT_E_NOMEM over the budget. */
int gaussians_voxelize(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_volume_desc *vol, float *out,
                       void *stream);

/* ---- batched scans ---------------------------------------------------- */

typedef struct rgrt_batch rgrt_batch;

/* A batch of n_scans independent scans (scan i = Gaussians g[i] projected
 * with geometry geom[i]); all scans share one ray kind (cone vs parallel)
 * and one tile shape.  Creation plans key capacities from one binning pass
 * per scan (it synchronises).  The handles must outlive the batch; the
 * Gaussians are updated in place by rgrt_batch_loss_step.  RGRT_E_INVAL for
 * mixed kinds or tile shapes, RGRT_E_NOMEM when the plan exceeds the budget. */
int rgrt_batch_create(rgrt_ctx *ctx, int n_scans, rgrt_gauss *const *g,
                      const rgrt_geom *const *geom, rgrt_batch **out);
int rgrt_batch_destroy(rgrt_batch *b);

/* Forward projection of every scan (binning of all scans, then one persistent
 * launch over every (scan, tile) work item of the scans too small to fill the
 * GPU for 16 waves; a larger scan is projected right after its binning by a
 * launch of its own.  Captured once in a CUDA graph and replayed).  out_I[i] receives scan i's projection (host or device; null
 * skips it).  Re-plans and repeats when the parameters have moved so far that
 * a scan's tile entries no longer fit.  Synchronises with `stream`. */
int rgrt_batch_forward(rgrt_batch *b, float *const *out_I, void *stream);

/* One optimisation step of every scan, as loss_step does for one: forward,
 * loss against y[i] (device arrays), adjoint (the small scans: one persistent
 * forward and one persistent adjoint launch over all of them; a large scan:
 * binning, forward, loss and adjoint back to back, its lists still in L2),
 * then the parameter chains and Adam (step t) of every scan.  loss_out[n_scans] (host or
 * device, may be null) receives the losses.  Captured in a CUDA graph that is
 * replayed while y, loss and hp stay the same.  Synchronises with `stream`. */
int rgrt_batch_loss_step(rgrt_batch *b, const float *const *y, int loss, const rgrt_adam *hp, int t,
                         float *loss_out, void *stream);

/* Tile lists of scan `scan` as the batch's last forward or step binned them
 * (layout as rgrt_debug_tile_lists: n_keys_out entries, tile_start[T + 1]
 * CSR offsets over the scan's T tiles, gid[cap] Gaussian ids, host or
 * device outputs).  Synchronises.  RGRT_E_INVAL for a bad scan index,
 * RGRT_E_CAPACITY if cap is smaller than the number of entries. */
int rgrt_batch_debug_tile_lists(rgrt_batch *b, int scan, int64_t *n_keys_out, uint32_t *tile_start,
                                uint32_t *gid, int64_t cap);

/* tiles of all scans, planned key capacity, re-plans so far */
int rgrt_batch_info(rgrt_batch *b, int64_t *work_items, int64_t *key_capacity, int *replans);

/* Tile-shape autotuner: times project_forward + project_backward of g on
 * `desc` (an evenly spaced subset of max_views views; max_views <= 0 keeps
 * all -- the sort's pass count depends on the total number of tiles, so a
 * subset can favour small tiles) for the tile shapes 16x16, 16x8, 8x8 and
 * 32x8, and returns the fastest (and its time in ms). */
int rgrt_autotune_tile(rgrt_ctx *ctx, rgrt_gauss *g, const rgrt_geom_desc *desc, int max_views,
                       int *tile_w, int *tile_h, double *ms_out);

/* ---- allocation-free forward projection ----------------------------- */

/* Maximum scratch, in bytes, of project_forward_noalloc (one static device
 * array per GPU that loads the library, held until the process exits). */
#define RGRT_NOALLOC_SCRATCH_BYTES (64u << 20)

/* project_forward without any memory allocation, for callers that must not
 * allocate device memory where they project (device memory owned by another
 * allocator, latency budgets that exclude cudaMalloc/cudaFree and the device
 * synchronisation they may cause, or fully reserved devices).  The paper has
 * no counterpart: this is an interface convenience.
 * All intermediate buffers come from a static device array of
 * RGRT_NOALLOC_SCRATCH_BYTES; no context is needed.  Arguments as for
 * gaussians_create + geometry_set + project_forward, but every array (mu3,
 * logscale3, quat4, rho, out_I) must be device memory of the current device;
 * desc->angles stays host memory.  Limits: at most 1024 views (PET_3D: angles
 * x ring differences) of 1024 x 1024 pixels, and the whole pipeline must fit
 * the scratch (C1-sized problems of
 * a few thousand Gaussians fit easily); otherwise RGRT_E_CAPACITY with a
 * message stating the bytes needed.  RGRT_E_INVAL for an array that is not
 * memory of the current device, and for non-finite parameters (as
 * project_forward).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); that first call should come before any
 * stream capture on the device.  Calls share the array, which keeps the last
 * call's contents: calls whose GPU work overlaps (unordered streams, several
 * host threads) race.  Every call reads the entry count and the non-finite
 * flag back from the device (16 bytes; a synchronisation of `stream`). */
int project_forward_noalloc(const rgrt_geom_desc *desc, int64_t n, const float *mu3,
                            const float *logscale3, const float *quat4, const float *rho,
                            float *out_I, void *stream);

/* ---- diagnostics ---------------------------------------------------- */

/* Message of the last failed call on this thread ("" if none). */
const char *rgrt_last_error(void);

/* Number of CUDA kernels the library has launched in this process. */
int64_t rgrt_launch_count(void);

/* The FP32 covariance records the cull uses: Sigma packed
 * (00,01,02,11,12,22), n x 6 floats (host or device). */
int rgrt_debug_records(rgrt_ctx *ctx, const rgrt_gauss *g, float *sigma6, void *stream);

/* Tile lists of views [v0, v1) (3-D PET: views count (ring difference,
 * angle) pairs, ring-difference major): n_keys_out = number of (tile,
 * Gaussian) entries; tile_start[n_tiles + 1] (CSR offsets, tile id =
 * (view - v0) * tiles_per_view + ty * tiles_x + tx) and gid[cap] (Gaussian
 * ids).  A tile's entries form a set: the projection needs no depth order
 * (paper section 2.3), and their order is the implementation's own.  Host
 * or device outputs; RGRT_E_INVAL for explicit-ray geometries or a bad view
 * range; RGRT_E_CAPACITY if cap is smaller than the number of entries
 * (n_keys_out is still set). */
int rgrt_debug_tile_lists(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, int v0,
                          int v1, int64_t *n_keys_out, uint32_t *tile_start, uint32_t *gid,
                          int64_t cap, void *stream);

/* Per-kernel timing: when enabled, every kernel launch of the library is
 * bracketed by CUDA events on its stream.  rgrt_prof_get reports for the
 * kernel named `name` the number of launches and their summed device time
 * (ms) since the last reset (it synchronises the recorded events). */
int rgrt_prof_enable(rgrt_ctx *ctx, int on);
int rgrt_prof_reset(rgrt_ctx *ctx);
int rgrt_prof_get(rgrt_ctx *ctx, const char *name, int64_t *launches, double *ms);
/* Pair counters (off by default: they cost a few instructions per pair).
 * When enabled, each project_forward counts the (ray, Gaussian) pairs it
 * evaluated and those with m <= 9; rgrt_stats_get returns the counts of the
 * last forward and its number of (tile, Gaussian) entries. */
int rgrt_stats_enable(rgrt_ctx *ctx, int on);
int rgrt_stats_get(rgrt_ctx *ctx, int64_t *pairs_evaluated, int64_t *pairs_kept, int64_t *keys);

#ifdef __cplusplus
}
#endif
#endif /* RGRT_H */
