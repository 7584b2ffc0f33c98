// Batched form: one optimisation step (or one forward pass) over many
// independent scans -- each with its own Gaussians and geometry -- as a single
// stream of work.  The scans are binned one after another.  A scan large
// enough to fill the GPU for 16 waves of tiles is projected, its loss taken
// and back-projected right after its binning, with launches of its own (its
// lists and records are still in L2 for the adjoint).  The smaller scans
// share ONE persistent launch that integrates every (scan, tile) work item,
// taken from an atomic counter (uneven scans fill the GPU together instead of
// leaving it under-filled one by one), then their losses and ONE persistent
// adjoint launch.  The parameter chains and the Adam updates of every scan
// come last.  The whole step is captured once in a CUDA graph and replayed,
// so a step costs one graph launch and one small read-back (losses and the
// key-capacity overflow flag) instead of a host round trip per scan.
//
// Key capacities are planned from a real binning pass (with 25% headroom);
// a step sorts only the entries it emits (their count is read on the
// device).  If the parameters move so far that a scan's (tile, Gaussian)
// entries no longer fit, the emit kernel raises the overflow flag, every Adam
// update of that step is skipped on the device, and the host re-plans,
// re-captures and repeats the step.  Only the sorted Gaussian ids and tile ranges of a scan
// are kept per scan; counts, keys and sort buffers are shared scratch sized
// for the largest scan.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "../../include/rgrt.h"
#include "rgrt_internal.h"
#include "rgrt_objects.h"

using namespace rgrt;

namespace {

#define BK(expr)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            char m_[300];                                                                \
            snprintf(m_, sizeof(m_), "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                     __FILE__, __LINE__);                                                \
            return report_error(RGRT_E_CUDA, m_);                                        \
        }                                                                                \
    } while (0)

#define BTRY(expr)                     \
    do {                               \
        int r_ = (expr);               \
        if (r_ != RGRT_OK) return r_;  \
    } while (0)

struct BatchScan {
    rgrt_gauss *g = nullptr;
    const rgrt_geom *geom = nullptr;
    int64_t N = 0, R = 0, E = 0;
    uint32_t T = 0, cap = 0;
    int bits = 0, nblk = 1;
    int lbits = -1;             // >= 0: keys sorted view by view (see launch_sort_views)
    bool large = false;         // projected by its own launches (not the persistent ones)
    uint32_t *vals = nullptr;   // sorted Gaussian ids [cap]
    uint2 *ranges = nullptr;    // [T]
    float *I = nullptr, *dLdI = nullptr;
    float4 *grad = nullptr;
    float *gflat = nullptr;
    double *partial = nullptr;
};

int ceil_log2_b(uint64_t x)
{
    int b = 0;
    while ((1ull << b) < x) b++;
    return b;
}

}  // namespace

struct rgrt_batch {
    rgrt_ctx *ctx = nullptr;
    int n = 0;
    bool cone = false;
    int tile_w = 16, tile_h = 16;
    std::vector<BatchScan> sc;
    // shared binning scratch
    uint32_t *cnt = nullptr, *off = nullptr, *keys = nullptr, *keys_alt = nullptr,
             *vals_alt = nullptr, *sort_tmp = nullptr;
    uint2 *rect = nullptr;
    unsigned long long *stmp = nullptr, *total = nullptr;
    // batch tables
    ScanDesc *d_desc = nullptr;
    uint32_t *d_queue = nullptr, *d_overflow = nullptr;
    float *d_loss = nullptr, *d_bc = nullptr;
    float *h_pin = nullptr;       // pinned: [2] bias corrections, [n] losses, [1] overflow bits
    uint32_t total_items = 0;     // work items of the persistent launches (small scans)
    uint64_t all_tiles = 0;       // tiles of every scan
    int n_small = 0;              // scans in the persistent descriptor table
    int grid_f = 0, grid_a = 0;
    uint64_t keys_capacity = 0;
    // graphs
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec_step = nullptr, exec_fwd = nullptr;
    long long kernels_step = 0, kernels_fwd = 0;   // kernel nodes of each graph
    std::vector<const float *> cap_y;
    int cap_loss = -1;
    rgrt_adam cap_hp{};
    std::vector<std::pair<void *, size_t>> allocs;
    int replans = 0;
};

namespace {

int balloc(rgrt_batch *b, void **p, size_t bytes)
{
    BTRY(ctx_alloc(b->ctx, p, bytes));
    b->allocs.push_back({ *p, bytes });
    return RGRT_OK;
}

void free_plan(rgrt_batch *b)
{
    for (auto &a : b->allocs) ctx_free(b->ctx, a.first, a.second);
    b->allocs.clear();
    for (auto &s : b->sc) {
        s.vals = nullptr; s.ranges = nullptr; s.I = s.dLdI = nullptr;
        s.grad = nullptr; s.gflat = nullptr; s.partial = nullptr;
    }
    b->cnt = b->off = b->keys = b->keys_alt = b->vals_alt = b->sort_tmp = nullptr;
    b->rect = nullptr;
    b->stmp = b->total = nullptr;
    b->d_desc = nullptr;
    b->d_queue = b->d_overflow = nullptr;
    b->d_loss = b->d_bc = nullptr;
    if (b->exec_step) cudaGraphExecDestroy(b->exec_step);
    if (b->exec_fwd) cudaGraphExecDestroy(b->exec_fwd);
    b->exec_step = b->exec_fwd = nullptr;
}

// measure every scan's key count with one real binning pass, size the buffers
int plan(rgrt_batch *b)
{
    free_plan(b);
    cudaStream_t s = b->stream;
    int64_t Emax = 1;
    for (auto &x : b->sc) Emax = std::max<int64_t>(Emax, x.E);
    BTRY(balloc(b, (void **)&b->cnt, sizeof(uint32_t) * Emax));
    BTRY(balloc(b, (void **)&b->off, sizeof(uint32_t) * Emax));
    BTRY(balloc(b, (void **)&b->rect, sizeof(uint2) * Emax));
    BTRY(balloc(b, (void **)&b->stmp, sizeof(unsigned long long) * scan_tmp_elems(Emax)));
    BTRY(balloc(b, (void **)&b->total, sizeof(unsigned long long) * 2));
    uint32_t capmax = 1;
    int vmax = 0;
    b->keys_capacity = 0;
    for (int i = 0; i < b->n; i++) {
        BatchScan &x = b->sc[i];
        DevGeom dg = x.geom->dg;
        dg.v0 = 0;
        BK(launch_records(x.g->mu, x.g->ls, x.g->q, x.g->rho, x.N, x.g->rec, x.g->crec, nullptr, s));
        BK(launch_cull(dg, dg.n_views, x.g->crec, x.N, b->cnt, b->rect, s));
        BK(launch_scan(b->cnt, b->off, x.E, b->total, b->stmp, s));
        unsigned long long K = 0;
        BK(cudaMemcpyAsync(&K, b->total, sizeof(K), cudaMemcpyDeviceToHost, s));
        BK(cudaStreamSynchronize(s));
        unsigned long long cap = K + K / 4 + 4096;
        if (cap >= 0xffffffffull) return report_error(RGRT_E_CAPACITY, "a scan of the batch has more than 2^32 tile entries");
        x.cap = (uint32_t)cap;
        capmax = std::max(capmax, x.cap);
        if (x.lbits >= 0) vmax = std::max(vmax, x.geom->dg.n_views);
        b->keys_capacity += cap;
        BTRY(balloc(b, (void **)&x.vals, sizeof(uint32_t) * (size_t)x.cap));
        BTRY(balloc(b, (void **)&x.ranges, sizeof(uint2) * (size_t)x.T));
        BTRY(balloc(b, (void **)&x.I, sizeof(float) * (size_t)x.R));
        BTRY(balloc(b, (void **)&x.dLdI, sizeof(float) * (size_t)x.R));
        BTRY(balloc(b, (void **)&x.grad, sizeof(float4) * GRAD_F4 * (size_t)std::max<int64_t>(x.N, 1)));
        BTRY(balloc(b, (void **)&x.gflat, sizeof(float) * 11 * (size_t)std::max<int64_t>(x.N, 1)));
        x.nblk = loss_blocks(x.R);
        BTRY(balloc(b, (void **)&x.partial, sizeof(double) * (size_t)x.nblk));
    }
    BTRY(balloc(b, (void **)&b->keys, sizeof(uint32_t) * capmax));
    BTRY(balloc(b, (void **)&b->keys_alt, sizeof(uint32_t) * capmax));
    BTRY(balloc(b, (void **)&b->vals_alt, sizeof(uint32_t) * capmax));
    BTRY(balloc(b, (void **)&b->sort_tmp, sizeof(uint32_t) * sort_tmp_elems(capmax, vmax)));
    b->grid_f = persistent_grid(true, b->cone, b->tile_w, b->tile_w * b->tile_h);
    b->grid_a = persistent_grid(false, b->cone, b->tile_w, b->tile_w * b->tile_h);
    // A scan whose tiles fill the GPU for 16 waves or more gains nothing from
    // sharing the persistent launches: it is binned, projected, and its loss
    // and adjoint taken back to back with launches of its own, while its
    // lists and records are still in L2.  The others share the persistent
    // launches (work items, scan by scan).
    std::vector<ScanDesc> hd;
    uint64_t items = 0;
    b->all_tiles = 0;
    for (int i = 0; i < b->n; i++) {
        BatchScan &x = b->sc[i];
        b->all_tiles += x.T;
        x.large = (int64_t)x.T >= 16 * (int64_t)b->grid_f;
        if (x.large) continue;
        hd.emplace_back();
        ScanDesc &d = hd.back();
        d.g = x.geom->dg;
        d.g.v0 = 0;
        d.rec = x.g->rec;
        d.crec = x.g->crec;
        d.gids = x.vals;
        d.ranges = x.ranges;
        d.out = x.I;
        d.dLdI = x.dLdI;
        d.grad = x.grad;
        d.item_begin = (uint32_t)items;
        d.n_items = x.T;
        items += x.T;
    }
    if (items >= 0xffffffffull) return report_error(RGRT_E_CAPACITY, "too many tiles in the batch");
    b->total_items = (uint32_t)items;
    b->n_small = (int)hd.size();
    BTRY(balloc(b, (void **)&b->d_desc, sizeof(ScanDesc) * std::max<size_t>(hd.size(), 1)));
    if (!hd.empty())
        BK(cudaMemcpyAsync(b->d_desc, hd.data(), sizeof(ScanDesc) * hd.size(), cudaMemcpyHostToDevice, s));
    BTRY(balloc(b, (void **)&b->d_queue, sizeof(uint32_t) * 2));
    BTRY(balloc(b, (void **)&b->d_overflow, sizeof(uint32_t)));
    BTRY(balloc(b, (void **)&b->d_loss, sizeof(float) * b->n));
    BTRY(balloc(b, (void **)&b->d_bc, sizeof(float) * 2));
    BK(cudaStreamSynchronize(s));
    return RGRT_OK;
}

// binning of scan i into its own sorted id list and tile ranges
int enqueue_bin_scan(rgrt_batch *b, int i, cudaStream_t s)
{
    {
        BatchScan &x = b->sc[i];
        DevGeom dg = x.geom->dg;
        dg.v0 = 0;
        BK(launch_records(x.g->mu, x.g->ls, x.g->q, x.g->rho, x.N, x.g->rec, x.g->crec, nullptr, s));
        BK(launch_cull(dg, dg.n_views, x.g->crec, x.N, b->cnt, b->rect, s));
        BK(launch_scan(b->cnt, b->off, x.E, b->total, b->stmp, s));
        // the scan's total (on the device) is the number of keys this step
        // emits: the sort and the ranges take only those (at most the planned
        // capacity; an item past it writes padding keys, which sort last and
        // map to no tile, and raises the overflow flag)
        BK(launch_emit(dg, dg.n_views, x.N, b->cnt, b->off, b->rect, b->keys, x.vals, x.cap,
                       b->d_overflow, s, x.lbits));
        if (x.lbits >= 0)
            BK(launch_sort_views(b->keys, x.vals, b->keys_alt, b->vals_alt, x.cap, x.bits, b->off, x.N,
                                 dg.n_views, b->sort_tmp, s, nullptr, b->total));
        else
            BK(launch_sort(b->keys, x.vals, b->keys_alt, b->vals_alt, x.cap, x.bits, b->sort_tmp, s, nullptr,
                           b->total));
        BK(cudaMemsetAsync(x.ranges, 0, sizeof(uint2) * (size_t)x.T, s));
        BK(launch_ranges(b->keys, x.cap, x.ranges, x.T, s, b->total, (uint32_t)x.geom->tiles_per_view,
                         x.lbits));
    }
    return RGRT_OK;
}

// forward of a large scan with launches of its own (all its views at once)
int enqueue_forward_large(rgrt_batch *b, int i, cudaStream_t s)
{
    BatchScan &x = b->sc[i];
    DevGeom dg = x.geom->dg;
    dg.v0 = 0;
    BK(launch_forward(dg, dg.n_views, x.g->rec, x.g->crec, x.vals, x.ranges, x.I, nullptr,
                      RGRT_KERNEL_GAUSSIAN, s));
    return RGRT_OK;
}

int enqueue_forward(rgrt_batch *b, cudaStream_t s)
{
    BK(cudaMemsetAsync(b->d_overflow, 0, sizeof(uint32_t), s));
    for (int i = 0; i < b->n; i++) {
        BTRY(enqueue_bin_scan(b, i, s));
        if (b->sc[i].large) BTRY(enqueue_forward_large(b, i, s));
    }
    if (b->n_small > 0) {
        BK(cudaMemsetAsync(b->d_queue, 0, sizeof(uint32_t), s));
        BK(launch_forward_persistent(b->cone, b->d_desc, b->n_small, b->total_items, b->d_queue,
                                     b->tile_w * b->tile_h, b->grid_f, s));
    }
    return RGRT_OK;
}

int enqueue_loss(rgrt_batch *b, int i, const float *const *y, int loss, const rgrt_adam *hp, cudaStream_t s)
{
    BatchScan &x = b->sc[i];
    BK(launch_loss(loss, x.I, y[i], x.R, hp->kappa, hp->poisson_eps, x.geom->d_mult, x.geom->d_add,
                   x.dLdI, x.partial, x.nblk, b->d_loss + i, s));
    BK(cudaMemsetAsync(x.grad, 0, sizeof(float4) * GRAD_F4 * (size_t)std::max<int64_t>(x.N, 1), s));
    return RGRT_OK;
}

int enqueue_step(rgrt_batch *b, const float *const *y, int loss, const rgrt_adam *hp, cudaStream_t s)
{
    BK(cudaMemsetAsync(b->d_overflow, 0, sizeof(uint32_t), s));
    // large scans: binning, forward, loss and adjoint back to back
    for (int i = 0; i < b->n; i++) {
        BTRY(enqueue_bin_scan(b, i, s));
        BatchScan &x = b->sc[i];
        if (!x.large) continue;
        BTRY(enqueue_forward_large(b, i, s));
        BTRY(enqueue_loss(b, i, y, loss, hp, s));
        DevGeom dg = x.geom->dg;
        dg.v0 = 0;
        BK(launch_adjoint(dg, dg.n_views, x.g->rec, x.g->crec, x.vals, x.ranges, x.dLdI, x.grad,
                          RGRT_KERNEL_GAUSSIAN, s));
    }
    // small scans: one persistent forward and one persistent adjoint
    if (b->n_small > 0) {
        BK(cudaMemsetAsync(b->d_queue, 0, sizeof(uint32_t), s));
        BK(launch_forward_persistent(b->cone, b->d_desc, b->n_small, b->total_items, b->d_queue,
                                     b->tile_w * b->tile_h, b->grid_f, s));
        for (int i = 0; i < b->n; i++)
            if (!b->sc[i].large) BTRY(enqueue_loss(b, i, y, loss, hp, s));
        BK(cudaMemsetAsync(b->d_queue + 1, 0, sizeof(uint32_t), s));
        BK(launch_adjoint_persistent(b->cone, b->tile_w, b->d_desc, b->n_small, b->total_items,
                                     b->d_queue + 1, b->grid_a, s));
    }
    // parameter chains and Adam last: an overflow flagged by any scan's
    // binning skips every update
    for (int i = 0; i < b->n; i++) {
        BatchScan &x = b->sc[i];
        if (x.N == 0) continue;
        rgrt_gauss *g = x.g;
        float *gf = x.gflat;
        const int64_t N = x.N;
        BK(launch_param_chain(g->mu, g->ls, g->q, g->rho, N, x.grad, gf, gf + 3 * N, gf + 6 * N,
                              gf + 10 * N, s));
        float *ps[4] = { g->mu, g->ls, g->q, g->rho };
        const int64_t offs[4] = { 0, 3 * N, 6 * N, 10 * N }, len[4] = { 3 * N, 3 * N, 4 * N, N };
        const float lr[4] = { hp->lr_mu, hp->lr_logscale, hp->lr_quat, hp->lr_rho };
        for (int k = 0; k < 4; k++)
            BK(launch_adam(ps[k], gf + offs[k], g->adam_m + offs[k], g->adam_v + offs[k], len[k], lr[k],
                           hp->beta1, hp->beta2, hp->eps, 1.0f, 1.0f, b->d_bc, b->d_overflow, s));
    }
    return RGRT_OK;
}

int capture(rgrt_batch *b, cudaGraphExec_t *exec, bool step, const float *const *y, int loss,
            const rgrt_adam *hp)
{
    if (*exec) {
        cudaGraphExecDestroy(*exec);
        *exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const long long before = rgrt_launch_count();
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int r = step ? enqueue_step(b, y, loss, hp, b->stream) : enqueue_forward(b, b->stream);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    // captured kernels run at each replay, not now: count them there
    const long long k = rgrt_launch_count() - before;
    count_launches((int)-k);
    (step ? b->kernels_step : b->kernels_fwd) = k;
    if (r != RGRT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    BK(e);
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    BK(e);
    return RGRT_OK;
}

// run `exec` on the batch stream, ordered after and before the caller's stream;
// returns the overflow flag
int run_graph(rgrt_batch *b, cudaGraphExec_t exec, cudaStream_t user, bool read_losses, bool *overflow)
{
    BK(cudaEventRecord(b->ev_in, user));
    BK(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    BK(cudaMemcpyAsync(b->d_bc, b->h_pin, sizeof(float) * 2, cudaMemcpyHostToDevice, b->stream));
    BK(cudaGraphLaunch(exec, b->stream));
    count_launches((int)(exec == b->exec_step ? b->kernels_step : b->kernels_fwd));
    uint32_t *h_over = (uint32_t *)(b->h_pin + 2 + b->n);
    BK(cudaMemcpyAsync(h_over, b->d_overflow, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
    if (read_losses)
        BK(cudaMemcpyAsync(b->h_pin + 2, b->d_loss, sizeof(float) * b->n, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    BK(cudaEventRecord(b->ev_out, b->stream));
    BK(cudaStreamWaitEvent(user, b->ev_out, 0));
    *overflow = *h_over != 0;
    return RGRT_OK;
}

int check_batch(rgrt_batch *b)
{
    if (!b) return report_error(RGRT_E_INVAL, "null batch");
    BK(cudaSetDevice(b->ctx->device));
    return RGRT_OK;
}

}  // namespace

extern "C" {

int rgrt_batch_create(rgrt_ctx *ctx, int n_scans, rgrt_gauss *const *g, const rgrt_geom *const *geom,
                      rgrt_batch **out)
{
    if (!ctx || !out || n_scans <= 0 || !g || !geom) return report_error(RGRT_E_INVAL, "bad batch arguments");
    *out = nullptr;
    BK(cudaSetDevice(ctx->device));
    rgrt_batch *b = new (std::nothrow) rgrt_batch();
    if (!b) return report_error(RGRT_E_NOMEM, "host allocation failed");
    b->ctx = ctx;
    b->n = n_scans;
    b->sc.resize(n_scans);
    for (int i = 0; i < n_scans; i++) {
        if (!g[i] || !geom[i] || g[i]->ctx != ctx || geom[i]->ctx != ctx) {
            delete b;
            return report_error(RGRT_E_INVAL, "batch scan with a null handle or one of another context");
        }
        if (geom[i]->rays || geom[i]->dg.kind == GM_PET3D || geom[i]->dg.n_tof) {
            delete b;
            return report_error(RGRT_E_INVAL, "explicit-ray, 3-D PET and time-of-flight geometries are not batched");
        }
        if (g[i]->kernel != RGRT_KERNEL_GAUSSIAN) {
            delete b;
            return report_error(RGRT_E_INVAL, "batches take Gaussian-kernel sets only");
        }
        const DevGeom &dg = geom[i]->dg;
        const bool cone = dg.kind == 1;
        if (i == 0) {
            b->cone = cone;
            b->tile_w = dg.tile_w;
            b->tile_h = dg.tile_h;
        } else if (cone != b->cone || dg.tile_w != b->tile_w || dg.tile_h != b->tile_h) {
            delete b;
            return report_error(RGRT_E_INVAL,
                                "all scans of a batch need the same ray kind and tile shape");
        }
        BatchScan &x = b->sc[i];
        x.g = g[i];
        x.geom = geom[i];
        x.N = g[i]->n;
        x.R = geom[i]->n_rays;
        x.T = (uint32_t)(dg.n_views * geom[i]->tiles_per_view);
        x.E = (int64_t)dg.n_views * x.N;
        if ((uint64_t)x.T >= (1ull << 24)) {
            delete b;
            return report_error(RGRT_E_CAPACITY, "a batch scan has more than 2^24 tiles");
        }
        const int lb = ceil_log2_b((uint64_t)geom[i]->tiles_per_view);
        x.lbits = ((uint64_t)dg.n_views << lb) < (1ull << 24) ? lb : -1;
        x.bits = x.lbits >= 0 ? x.lbits + 8 : ceil_log2_b(x.T) + 8;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_pin, sizeof(float) * (3 + n_scans));
    if (e != cudaSuccess) {
        rgrt_batch_destroy(b);
        return report_error(RGRT_E_CUDA, cudaGetErrorString(e));
    }
    b->h_pin[0] = b->h_pin[1] = 1.0f;
    int r = plan(b);
    if (r != RGRT_OK) {
        rgrt_batch_destroy(b);
        return r;
    }
    *out = b;
    return RGRT_OK;
}

int rgrt_batch_destroy(rgrt_batch *b)
{
    if (!b) return RGRT_OK;
    cudaSetDevice(b->ctx->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_plan(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->h_pin) cudaFreeHost(b->h_pin);
    delete b;
    return RGRT_OK;
}

int rgrt_batch_forward(rgrt_batch *b, float *const *out_I, void *stream)
{
    BTRY(check_batch(b));
    if (!out_I) return report_error(RGRT_E_INVAL, "null outputs");
    cudaStream_t user = (cudaStream_t)stream;
    for (int attempt = 0; attempt < 3; attempt++) {
        if (!b->exec_fwd) BTRY(capture(b, &b->exec_fwd, false, nullptr, 0, nullptr));
        bool over = false;
        BTRY(run_graph(b, b->exec_fwd, user, false, &over));
        if (!over) {
            for (int i = 0; i < b->n; i++)
                if (out_I[i])
                    BK(cudaMemcpyAsync(out_I[i], b->sc[i].I, sizeof(float) * (size_t)b->sc[i].R,
                                       cudaMemcpyDefault, user));
            BK(cudaStreamSynchronize(user));
            return RGRT_OK;
        }
        b->replans++;
        BTRY(plan(b));
    }
    return report_error(RGRT_E_CAPACITY, "batch key capacity overflowed after re-planning");
}

int rgrt_batch_loss_step(rgrt_batch *b, const float *const *y, int loss, const rgrt_adam *hp, int t,
                         float *loss_out, void *stream)
{
    BTRY(check_batch(b));
    if (!y || !hp) return report_error(RGRT_E_INVAL, "null argument");
    if (loss != RGRT_LOSS_L2 && loss != RGRT_LOSS_POISSON) return report_error(RGRT_E_INVAL, "loss kind");
    if (t < 1) return report_error(RGRT_E_INVAL, "Adam step t must be >= 1");
    cudaStream_t user = (cudaStream_t)stream;
    for (int i = 0; i < b->n; i++) {
        cudaPointerAttributes a;
        if (!y[i] || cudaPointerGetAttributes(&a, y[i]) != cudaSuccess ||
            !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return report_error(RGRT_E_INVAL, "batch measurements must be device arrays");
        }
        BTRY(gauss_adam(b->sc[i].g, b->stream));
    }
    bool same = b->exec_step && b->cap_loss == loss &&
                (int)b->cap_y.size() == b->n && std::equal(b->cap_y.begin(), b->cap_y.end(), y) &&
                b->cap_hp.lr_mu == hp->lr_mu && b->cap_hp.lr_logscale == hp->lr_logscale &&
                b->cap_hp.lr_quat == hp->lr_quat && b->cap_hp.lr_rho == hp->lr_rho &&
                b->cap_hp.beta1 == hp->beta1 && b->cap_hp.beta2 == hp->beta2 &&
                b->cap_hp.eps == hp->eps && b->cap_hp.kappa == hp->kappa &&
                b->cap_hp.poisson_eps == hp->poisson_eps;
    b->h_pin[0] = (float)(1.0 - pow((double)hp->beta1, (double)t));
    b->h_pin[1] = (float)(1.0 - pow((double)hp->beta2, (double)t));
    for (int attempt = 0; attempt < 3; attempt++) {
        if (!same) {
            BTRY(capture(b, &b->exec_step, true, y, loss, hp));
            b->cap_y.assign(y, y + b->n);
            b->cap_loss = loss;
            b->cap_hp = *hp;
            same = true;
        }
        bool over = false;
        BTRY(run_graph(b, b->exec_step, user, true, &over));
        if (!over) {
            for (int i = 0; i < b->n; i++) b->sc[i].g->version++;
            if (loss_out) BK(cudaMemcpy(loss_out, b->h_pin + 2, sizeof(float) * b->n, cudaMemcpyDefault));
            return RGRT_OK;
        }
        // entries did not fit: the device skipped every Adam update; re-plan and repeat
        b->replans++;
        BTRY(plan(b));
        same = false;
    }
    return report_error(RGRT_E_CAPACITY, "batch key capacity overflowed after re-planning");
}

int rgrt_autotune_tile(rgrt_ctx *ctx, rgrt_gauss *g, const rgrt_geom_desc *desc, int max_views,
                       int *tile_w, int *tile_h, double *ms_out)
{
    if (!ctx || !g || !desc || !tile_w || !tile_h) return report_error(RGRT_E_INVAL, "null argument");
    BTRY(validate_geometry(desc));
    BK(cudaSetDevice(ctx->device));
    static const int cand[][2] = { { 16, 16 }, { 16, 8 }, { 8, 8 }, { 32, 8 } };
    rgrt_geom_desc sub = *desc;
    std::vector<double> ang;
    if (max_views > 0 && max_views < desc->n_views) {
        // evenly spaced subset of the views (a PET sinogram without explicit
        // angles spaces its angles pi j / n_views)
        for (int k = 0; k < max_views; k++) {
            const int64_t j = (int64_t)k * desc->n_views / max_views;
            ang.push_back(desc->angles ? desc->angles[j]
                                       : 3.14159265358979323846 * (double)j / (double)desc->n_views);
        }
        sub.angles = ang.data();
        sub.n_views = max_views;
    }
    const int64_t R = desc_rays(&sub);
    float *I = nullptr;
    BTRY(ctx_alloc(ctx, (void **)&I, sizeof(float) * (size_t)R));
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int bw = 16, bh = 16, rc = RGRT_OK;
    for (const auto &c : cand) {
        sub.tile_w = c[0];
        sub.tile_h = c[1];
        rgrt_geom *geom = nullptr;
        if (geometry_set(ctx, &sub, &geom) != RGRT_OK) continue;
        double ms = 1e300;
        for (int rep = 0; rep < 3 && rc == RGRT_OK; rep++) {   // first repetition warms up
            cudaEventRecord(e0, s);
            rc = project_forward(ctx, g, geom, I, s);
            if (rc == RGRT_OK) rc = project_backward(ctx, g, geom, I, nullptr, nullptr, nullptr, nullptr, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, (double)t);
        }
        geometry_destroy(geom);
        if (rc != RGRT_OK) break;
        if (ms < best) {
            best = ms;
            bw = c[0];
            bh = c[1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx_free(ctx, I, sizeof(float) * (size_t)R);
    if (rc != RGRT_OK) return rc;
    *tile_w = bw;
    *tile_h = bh;
    if (ms_out) *ms_out = best;
    return RGRT_OK;
}

int rgrt_batch_debug_tile_lists(rgrt_batch *b, int scan, int64_t *n_keys_out, uint32_t *tile_start,
                                uint32_t *gid, int64_t cap)
{
    BTRY(check_batch(b));
    if (scan < 0 || scan >= b->n || !n_keys_out || !tile_start)
        return report_error(RGRT_E_INVAL, "bad scan index or null argument");
    const BatchScan &x = b->sc[scan];
    BK(cudaStreamSynchronize(b->stream));
    std::vector<uint2> rg(x.T);
    if (x.T > 0 && x.ranges)
        BK(cudaMemcpy(rg.data(), x.ranges, sizeof(uint2) * x.T, cudaMemcpyDeviceToHost));
    std::vector<uint32_t> start(x.T + 1, 0);
    uint32_t pos = 0;
    for (uint32_t t = 0; t < x.T; t++) {
        start[t] = pos;
        if (rg[t].y > rg[t].x) {
            if (rg[t].x != pos) return report_error(RGRT_E_CUDA, "batch tile ranges are not contiguous");
            pos = rg[t].y;
        }
    }
    start[x.T] = pos;
    if (pos > x.cap) return report_error(RGRT_E_CUDA, "batch tile ranges exceed the scan's capacity");
    *n_keys_out = pos;
    BK(cudaMemcpy(tile_start, start.data(), sizeof(uint32_t) * (x.T + 1), cudaMemcpyDefault));
    if ((int64_t)pos > cap) return report_error(RGRT_E_CAPACITY, "tile entries exceed the capacity given");
    if (pos > 0 && gid) BK(cudaMemcpy(gid, x.vals, sizeof(uint32_t) * pos, cudaMemcpyDefault));
    return RGRT_OK;
}

int rgrt_batch_info(rgrt_batch *b, int64_t *work_items, int64_t *key_capacity, int *replans)
{
    if (!b) return report_error(RGRT_E_INVAL, "null batch");
    if (work_items) *work_items = (int64_t)b->all_tiles;
    if (key_capacity) *key_capacity = (int64_t)b->keys_capacity;
    if (replans) *replans = b->replans;
    return RGRT_OK;
}

}  // extern "C"
