// C ABI of librgrt: contexts, Gaussians, geometries, and the stream-ordered
// orchestration of the projector pipeline (records -> cull -> scan -> emit
// -> radix sort -> tile ranges -> integrate / adjoint -> parameter chain).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <utility>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/rgrt.h"
#include "rgrt_internal.h"
#include "rgrt_objects.h"

using namespace rgrt;

namespace {
std::atomic<long long> g_launches{ 0 };
}

void rgrt::count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(expr)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(RGRT_E_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),      \
                        __FILE__, __LINE__);                                              \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        int r_ = (expr);               \
        if (r_ != RGRT_OK) return r_;  \
    } while (0)

}  // namespace

namespace {

int dev_alloc(rgrt_ctx *c, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (c->used + bytes > c->budget)
        return fail(RGRT_E_NOMEM, "allocation of %zu bytes exceeds the HBM budget (%zu of %zu used)",
                    bytes, c->used, c->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return fail(RGRT_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    c->used += bytes;
    return RGRT_OK;
}

void dev_free(rgrt_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    if (bytes == 0) bytes = 16;
    c->used -= bytes;
}

int ensure(rgrt_ctx *c, Buf &b, size_t bytes)
{
    if (b.bytes >= bytes && b.p) return RGRT_OK;
    size_t want = bytes + bytes / 8 + 256;
    if (b.p) {
        cudaFree(b.p);
        c->used -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    TRY(dev_alloc(c, &b.p, want));
    b.bytes = want;
    return RGRT_OK;
}

void release(rgrt_ctx *c, Buf &b)
{
    if (b.p) {
        cudaFree(b.p);
        c->used -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of an input array: the pointer itself, or a staged copy
int stage_input(rgrt_ctx *c, Buf &b, const void *src, size_t bytes, cudaStream_t s, const void **out)
{
    if (!src || bytes == 0 || is_device_ptr(src)) {
        *out = src;
        return RGRT_OK;
    }
    TRY(ensure(c, b, bytes));
    CK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s));
    *out = b.p;
    return RGRT_OK;
}

// device buffer for an output; returns whether a copy-back is needed
int stage_output(rgrt_ctx *c, Buf &b, void *dst, size_t bytes, void **out, bool *copy_back)
{
    *copy_back = false;
    if (!dst || bytes == 0 || is_device_ptr(dst)) {
        *out = dst;
        return RGRT_OK;
    }
    TRY(ensure(c, b, bytes));
    *out = b.p;
    *copy_back = true;
    return RGRT_OK;
}

// ---- profiling ------------------------------------------------------------

struct ProfScope {
    rgrt_ctx *c;
    const char *name;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(rgrt_ctx *c_, const char *n, cudaStream_t s_) : c(c_), name(n), s(s_)
    {
        if (c->prof && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, s);
    }
    ~ProfScope()
    {
        if (a && b) {
            cudaEventRecord(b, s);
            c->pending.push_back(ProfRec{ name, a, b });
        }
    }
};

void prof_harvest(rgrt_ctx *c)
{
    for (auto &r : c->pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &e = c->prof_acc[r.name];
        e.first += 1;
        e.second += ms;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->pending.clear();
}

#define PROF(name) ProfScope prof_scope_(ctx, name, s)

// ---- pipeline pieces ------------------------------------------------------

// records of the current parameters; total[1] collects the non-finite flag,
// which the next host read-back of the binning totals checks
int build_records(rgrt_ctx *ctx, const rgrt_gauss *g, cudaStream_t s)
{
    if (g->n == 0) return RGRT_OK;
    TRY(ensure(ctx, ctx->total, sizeof(unsigned long long) * 2));
    unsigned long long *bad = (unsigned long long *)ctx->total.p + 1;
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
    PROF("k_records");
    CK(launch_records(g->mu, g->ls, g->q, g->rho, g->n, g->rec, g->crec, (uint32_t *)bad, s));
    return RGRT_OK;
}

// the binning totals (K) and the non-finite flag, read back together
int read_totals(rgrt_ctx *ctx, cudaStream_t s, unsigned long long *K)
{
    CK(cudaMemcpyAsync(ctx->h_total, ctx->total.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->h_total[1])
        return fail(RGRT_E_INVAL, "non-finite Gaussian parameters (mu, log-scale, quaternion or rho)");
    if (K) *K = ctx->h_total[0];
    return RGRT_OK;
}

int ceil_log2(uint64_t x)
{
    int b = 0;
    while ((1ull << b) < x) b++;
    return b;
}

// cull + scan + emit + sort + ranges for views [v0, v0 + nv); RGRT_E_CAPACITY
// if the chunk's keys do not fit the budget (the caller then splits it)
int bin_views(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, int v0, int nv,
              cudaStream_t s, uint32_t *n_keys)
{
    const int64_t N = g->n;
    const int64_t E = (int64_t)nv * N;
    DevGeom dg = geom->dg;
    dg.v0 = v0;
    const uint32_t T = (uint32_t)nv * (uint32_t)geom->tiles_per_view;
    if (T >= (1u << 24))  // tile ids share the key with an 8-bit position code
        return fail(RGRT_E_CAPACITY, "views %d..%d hold %u tiles (2^24 at most)", v0, v0 + nv, T);
    TRY(ensure(ctx, ctx->cnt, sizeof(uint32_t) * (size_t)E));
    TRY(ensure(ctx, ctx->off, sizeof(uint32_t) * (size_t)E));
    TRY(ensure(ctx, ctx->rect, sizeof(uint2) * (size_t)E));
    TRY(ensure(ctx, ctx->scan_tmp, sizeof(unsigned long long) * scan_tmp_elems(E)));
    TRY(ensure(ctx, ctx->total, sizeof(unsigned long long) * 2));
    TRY(ensure(ctx, ctx->ranges, sizeof(uint2) * (size_t)T));
    {
        PROF("k_cull");
        CK(launch_cull(dg, nv, g->crec, N, (uint32_t *)ctx->cnt.p, (uint2 *)ctx->rect.p, s));
    }
    {
        PROF("scan");
        CK(launch_scan((uint32_t *)ctx->cnt.p, (uint32_t *)ctx->off.p, E,
                       (unsigned long long *)ctx->total.p, (unsigned long long *)ctx->scan_tmp.p, s));
    }
    unsigned long long K = 0;
    TRY(read_totals(ctx, s, &K));
    if (K >= 0xffffffffull)
        return fail(RGRT_E_CAPACITY, "views %d..%d produce %llu tile entries (more than 2^32)", v0,
                    v0 + nv, K);
    // the views' keys are sorted view by view (on the tile within the view and
    // the position code) when the padded tile field (view << lbits | tile)
    // fits the key's 24 bits
    const uint32_t tpv = (uint32_t)geom->tiles_per_view;
    const int lbits = ceil_log2(tpv);
    const bool by_view = ((uint64_t)nv << lbits) < (1ull << 24);
    const int nseg = by_view ? nv : 0;
    size_t need = 4 * sizeof(uint32_t) * (size_t)K + sizeof(uint32_t) * sort_tmp_elems((uint32_t)K, nseg);
    size_t have = ctx->keys.bytes + ctx->vals.bytes + ctx->keys_alt.bytes + ctx->vals_alt.bytes +
                  ctx->sort_tmp.bytes;
    if (need > have && ctx->used - have + need + need / 8 > ctx->budget)
        return fail(RGRT_E_CAPACITY, "views %d..%d produce %llu tile entries, over the budget", v0,
                    v0 + nv, K);
    TRY(ensure(ctx, ctx->keys, sizeof(uint32_t) * (size_t)K));
    TRY(ensure(ctx, ctx->vals, sizeof(uint32_t) * (size_t)K));
    TRY(ensure(ctx, ctx->keys_alt, sizeof(uint32_t) * (size_t)K));
    TRY(ensure(ctx, ctx->vals_alt, sizeof(uint32_t) * (size_t)K));
    TRY(ensure(ctx, ctx->sort_tmp, sizeof(uint32_t) * sort_tmp_elems((uint32_t)K, nseg)));
    uint32_t *keys = (uint32_t *)ctx->keys.p, *vals = (uint32_t *)ctx->vals.p;
    {
        PROF("k_emit");
        CK(launch_emit(dg, nv, N, (uint32_t *)ctx->cnt.p, (uint32_t *)ctx->off.p,
                       (uint2 *)ctx->rect.p, keys, vals, (uint32_t)K, nullptr, s, by_view ? lbits : -1));
    }
    {
        PROF("radix_sort");
        bool in_alt = false;
        if (by_view)
            CK(launch_sort_views(keys, vals, (uint32_t *)ctx->keys_alt.p, (uint32_t *)ctx->vals_alt.p,
                                 (uint32_t)K, lbits + 8, (const uint32_t *)ctx->off.p, N, nv,
                                 (uint32_t *)ctx->sort_tmp.p, s, &in_alt));
        else
            CK(launch_sort(keys, vals, (uint32_t *)ctx->keys_alt.p, (uint32_t *)ctx->vals_alt.p,
                           (uint32_t)K, ceil_log2(T) + 8, (uint32_t *)ctx->sort_tmp.p, s, &in_alt));
        if (in_alt) {   // adopt the buffers that hold the result
            std::swap(ctx->keys, ctx->keys_alt);
            std::swap(ctx->vals, ctx->vals_alt);
            keys = (uint32_t *)ctx->keys.p;
            vals = (uint32_t *)ctx->vals.p;
        }
    }
    {
        PROF("k_ranges");
        CK(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(uint2) * (size_t)T, s));
        CK(launch_ranges(keys, (uint32_t)K, (uint2 *)ctx->ranges.p, T, s, nullptr, tpv, by_view ? lbits : -1));
    }
    *n_keys = (uint32_t)K;
    ctx->last_keys += (long long)K;
    ctx->bin_g = g;
    ctx->bin_geom = geom;
    ctx->bin_version = g->version;
    ctx->bin_v0 = v0;
    ctx->bin_nv = nv;
    ctx->bin_keys = (uint32_t)K;
    ctx->bin_valid = true;
    return RGRT_OK;
}

// first chunk size: bounded per-(view, Gaussian) scratch
int initial_chunk(const rgrt_gauss *g, const rgrt_geom *geom)
{
    const int64_t max_entries = (int64_t)1 << 27;
    int64_t nv = g->n > 0 ? max_entries / g->n : geom->desc.n_views;
    if (nv < 1) nv = 1;
    if (nv > geom->desc.n_views) nv = geom->desc.n_views;
    return (int)nv;
}

// run `body(v0, nv)` over view chunks, binning each first; chunks halve on
// RGRT_E_CAPACITY.  reuse: keep the cached binning if it covers the chunk.
template <class F>
int for_chunks(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, cudaStream_t s,
               bool reuse, F body)
{
    int V = geom->desc.n_views;
    int nv = initial_chunk(g, geom);
    int v0 = 0;
    while (v0 < V) {
        int cur = nv < V - v0 ? nv : V - v0;
        uint32_t K = 0;
        bool cached = reuse && ctx->bin_valid && ctx->bin_g == g && ctx->bin_geom == geom &&
                      ctx->bin_version == g->version && ctx->bin_v0 == v0 && ctx->bin_nv == cur;
        if (!cached) {
            int r = bin_views(ctx, g, geom, v0, cur, s, &K);
            if (r == RGRT_E_CAPACITY && cur > 1) {
                ctx->bin_valid = false;
                nv = cur / 2;
                continue;
            }
            if (r != RGRT_OK) {
                ctx->bin_valid = false;
                return r;
            }
        } else {
            K = ctx->bin_keys;
        }
        TRY(body(v0, cur, K));
        v0 += cur;
    }
    return RGRT_OK;
}

int check_ctx(rgrt_ctx *c)
{
    if (!c) return fail(RGRT_E_INVAL, "null context");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(RGRT_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return RGRT_OK;
}

// ---- explicit rays --------------------------------------------------------

// balls, scene box, block lines and per-block counts, then split the blocks
// into consecutive ranges whose lists fit the budget; body(b0, nb) runs after
// each range's lists are built.  reuse: keep cached lists of a single range.
template <class F>
int for_ray_ranges(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, cudaStream_t s,
                   bool reuse, F body)
{
    const int64_t N = g->n;
    const int T = geom->n_blocks;
    if (reuse && ctx->bin_valid && ctx->bin_g == g && ctx->bin_geom == geom &&
        ctx->bin_version == g->version && ctx->bin_v0 == 0 && ctx->bin_nv == T)
        return body(0, T);
    ctx->bin_valid = false;
    const int parts = rays_ball_parts(N);
    TRY(ensure(ctx, ctx->ball, sizeof(float4) * (size_t)N));
    TRY(ensure(ctx, ctx->part, sizeof(float4) * 2 * (size_t)parts));
    TRY(ensure(ctx, ctx->scene, sizeof(float4) * 2));
    TRY(ensure(ctx, ctx->blk, sizeof(float4) * 2 * (size_t)T));
    TRY(ensure(ctx, ctx->wblk, sizeof(float4) * 8 * (size_t)T));
    const size_t TL = (size_t)T * RAYS_WPB;   // one list per warp
    TRY(ensure(ctx, ctx->cnt, sizeof(uint32_t) * TL));
    TRY(ensure(ctx, ctx->off, sizeof(uint32_t) * TL));
    TRY(ensure(ctx, ctx->ranges, sizeof(uint2) * TL));
    TRY(ensure(ctx, ctx->scan_tmp, sizeof(unsigned long long) * scan_tmp_elems((int64_t)TL)));
    TRY(ensure(ctx, ctx->total, sizeof(unsigned long long) * 2));
    TRY(ensure(ctx, ctx->clusters, rays_cluster_bytes(N)));
    {
        PROF("rays_bin");
        CK(launch_rays_bin(geom->d_ro, geom->d_rd, geom->n_rays, g->rec, N, (float4 *)ctx->ball.p,
                           (float4 *)ctx->part.p, (float4 *)ctx->scene.p, (float4 *)ctx->blk.p,
                           (float4 *)ctx->wblk.p, ctx->clusters.p, (uint32_t *)ctx->cnt.p, s));
    }
    ctx->h_cnt.resize(TL);
    CK(cudaMemcpyAsync(ctx->h_cnt.data(), ctx->cnt.p, sizeof(uint32_t) * TL, cudaMemcpyDeviceToHost, s));
    TRY(read_totals(ctx, s, nullptr));
    // list capacity: what the budget leaves (the current list buffer included)
    size_t avail = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
    avail += ctx->vals.bytes;
    avail = avail > ((size_t)1 << 20) ? avail - ((size_t)1 << 20) : 0;
    uint64_t cap = avail / sizeof(uint32_t);
    if (cap > 0x7fffffffull) cap = 0x7fffffffull;
    std::vector<std::pair<int, int>> rng;
    uint64_t acc = 0, total = 0;
    int b0 = 0;
    auto block_count = [&](int b) -> uint64_t {
        uint64_t c = 0;
        for (int w = 0; w < RAYS_WPB; w++) c += ctx->h_cnt[(size_t)b * RAYS_WPB + w];
        return c;
    };
    for (int b = 0; b < T; b++) {
        const uint64_t c = block_count(b);
        if (c > cap)
            return fail(RGRT_E_CAPACITY, "ray block %d lists %llu Gaussians, over the budget", b,
                        (unsigned long long)c);
        if (acc + c > cap) {
            rng.push_back({ b0, b - b0 });
            b0 = b;
            acc = 0;
        }
        acc += c;
        total += c;
    }
    rng.push_back({ b0, T - b0 });
    uint64_t kmax = 0;
    for (auto &r : rng) {
        uint64_t k = 0;
        for (int b = r.first; b < r.first + r.second; b++) k += block_count(b);
        kmax = k > kmax ? k : kmax;
    }
    TRY(ensure(ctx, ctx->vals, sizeof(uint32_t) * (size_t)(kmax > 0 ? kmax : 1)));
    ctx->last_keys += (long long)total;
    for (auto &r : rng) {
        {
            PROF("rays_emit");
            CK(launch_scan((const uint32_t *)ctx->cnt.p + (size_t)r.first * RAYS_WPB, (uint32_t *)ctx->off.p,
                           (int64_t)r.second * RAYS_WPB, (unsigned long long *)ctx->total.p,
                           (unsigned long long *)ctx->scan_tmp.p, s));
            CK(launch_rays_emit((const float4 *)ctx->blk.p, (const float4 *)ctx->wblk.p, ctx->clusters.p, N,
                                r.first, r.second, (const uint32_t *)ctx->off.p, (const uint32_t *)ctx->cnt.p,
                                (uint32_t *)ctx->vals.p, (uint2 *)ctx->ranges.p, s));
        }
        if (rng.size() == 1) {
            ctx->bin_g = g;
            ctx->bin_geom = geom;
            ctx->bin_version = g->version;
            ctx->bin_v0 = 0;
            ctx->bin_nv = T;
            ctx->bin_valid = true;
        }
        TRY(body(r.first, r.second));
    }
    return RGRT_OK;
}

int run_forward_rays(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, float *out,
                     cudaStream_t s)
{
    if (geom->d_tof && g->kernel != RGRT_KERNEL_GAUSSIAN)
        return fail(RGRT_E_INVAL, "time of flight takes the Gaussian kernel");
    TRY(build_records(ctx, g, s));
    ctx->last_keys = 0;
    return for_ray_ranges(ctx, g, geom, s, false, [&](int b0, int nb) -> int {
        PROF("k_rays_forward");
        CK(launch_rays_forward(geom->d_ro, geom->d_rd, geom->d_tof, geom->n_rays, b0, nb, g->rec,
                               (const uint32_t *)ctx->vals.p, (const uint2 *)ctx->ranges.p, out, g->kernel, s));
        return RGRT_OK;
    });
}

int run_forward(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, float *out,
                cudaStream_t s)
{
    if (geom->rays) {
        if (g->n == 0) {
            CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)geom->n_rays, s));
            return RGRT_OK;
        }
        return run_forward_rays(ctx, g, geom, out, s);
    }
    if (geom->dg.n_tof && g->kernel != RGRT_KERNEL_GAUSSIAN)
        return fail(RGRT_E_INVAL, "time of flight takes the Gaussian kernel");
    if (g->n == 0) {
        CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)geom->n_rays, s));
        return RGRT_OK;
    }
    TRY(build_records(ctx, g, s));
    Stats *st = nullptr;
    if (ctx->stats_on) {
        TRY(ensure(ctx, ctx->stats, sizeof(Stats)));
        CK(cudaMemsetAsync(ctx->stats.p, 0, sizeof(Stats), s));
        st = (Stats *)ctx->stats.p;
    }
    ctx->last_keys = 0;
    return for_chunks(ctx, g, geom, s, false, [&](int v0, int nv, uint32_t K) -> int {
        (void)K;
        DevGeom dg = geom->dg;
        dg.v0 = v0;
        PROF("k_forward");
        CK(launch_forward(dg, nv, g->rec, g->crec, (uint32_t *)ctx->vals.p, (uint2 *)ctx->ranges.p,
                          out, st, g->kernel, s));
        return RGRT_OK;
    });
}

// adjoint into ctx->grad (zeroed first), then the parameter chain into the
// four (device) outputs
int run_backward(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, const float *dLdI,
                 float *gm, float *gl, float *gq, float *gr, cudaStream_t s)
{
    const int64_t N = g->n;
    if (N == 0) return RGRT_OK;
    TRY(ensure(ctx, ctx->grad, sizeof(float4) * GRAD_F4 * (size_t)N));
    CK(cudaMemsetAsync(ctx->grad.p, 0, sizeof(float4) * GRAD_F4 * (size_t)N, s));
    bool reuse = ctx->bin_valid && ctx->bin_g == g && ctx->bin_geom == geom &&
                 ctx->bin_version == g->version;
    if (!reuse) TRY(build_records(ctx, g, s));
    if (geom->rays) {
        if (geom->d_tof && g->kernel != RGRT_KERNEL_GAUSSIAN)
            return fail(RGRT_E_INVAL, "time of flight takes the Gaussian kernel");
        TRY(for_ray_ranges(ctx, g, geom, s, reuse, [&](int b0, int nb) -> int {
            PROF("k_rays_adjoint");
            CK(launch_rays_adjoint(geom->d_ro, geom->d_rd, geom->d_tof, geom->n_rays, b0, nb, g->rec,
                                   (const uint32_t *)ctx->vals.p, (const uint2 *)ctx->ranges.p, dLdI,
                                   (float4 *)ctx->grad.p, g->kernel, s));
            return RGRT_OK;
        }));
        PROF("k_param_chain");
        CK(launch_param_chain(g->mu, g->ls, g->q, g->rho, N, (float4 *)ctx->grad.p, gm, gl, gq, gr, s));
        return RGRT_OK;
    }
    if (geom->dg.n_tof && g->kernel != RGRT_KERNEL_GAUSSIAN)
        return fail(RGRT_E_INVAL, "time of flight takes the Gaussian kernel");
    TRY(for_chunks(ctx, g, geom, s, reuse, [&](int v0, int nv, uint32_t K) -> int {
        (void)K;
        DevGeom dg = geom->dg;
        dg.v0 = v0;
        PROF("k_adjoint");
        CK(launch_adjoint(dg, nv, g->rec, g->crec, (uint32_t *)ctx->vals.p, (uint2 *)ctx->ranges.p,
                          dLdI, (float4 *)ctx->grad.p, g->kernel, s));
        return RGRT_OK;
    }));
    PROF("k_param_chain");
    CK(launch_param_chain(g->mu, g->ls, g->q, g->rho, N, (float4 *)ctx->grad.p, gm, gl, gq, gr, s));
    return RGRT_OK;
}

int validate_desc(const rgrt_geom_desc *d)
{
    if (!d) return fail(RGRT_E_INVAL, "null geometry description");
    if (d->kind < 0 || d->kind > 3) return fail(RGRT_E_INVAL, "unknown geometry kind %d", d->kind);
    if (d->n_views <= 0 || d->n_rows <= 0 || d->n_cols <= 0)
        return fail(RGRT_E_INVAL, "geometry sizes must be positive (%d views, %d x %d)", d->n_views,
                    d->n_rows, d->n_cols);
    int tw = d->tile_w ? d->tile_w : 16, th = d->tile_h ? d->tile_h : 16;
    if ((tw != 8 && tw != 16 && tw != 32) || th % 4 || th > 32 || tw * th > 256 || tw * th < 32)
        return fail(RGRT_E_INVAL, "tile %dx%d: width 8, 16 or 32, height a multiple of 4 up to 32, "
                    "32..256 rays", tw, th);
    if ((d->n_cols + tw - 1) / tw > 65535 || (d->n_rows + th - 1) / th > 65535)
        return fail(RGRT_E_INVAL, "too many tiles per detector axis");
    const bool pet = d->kind == RGRT_GEOM_PET_RING || d->kind == RGRT_GEOM_PET_3D;
    if (d->kind == RGRT_GEOM_PET_3D && (d->max_ring_diff < 0 || d->max_ring_diff >= d->n_rows))
        return fail(RGRT_E_INVAL, "max_ring_diff %d outside 0..%d", d->max_ring_diff, d->n_rows - 1);
    if (desc_views(d) > (1 << 30)) return fail(RGRT_E_INVAL, "too many views");
    if (desc_views(d) * ((d->n_cols + tw - 1) / tw) * ((d->n_rows + th - 1) / th) > (1 << 30))
        return fail(RGRT_E_INVAL, "too many tiles");
    if (pet && d->angles) {
        for (int v = 0; v < d->n_views; v++)
            if (!std::isfinite(d->angles[v])) return fail(RGRT_E_INVAL, "non-finite view angle %d", v);
    }
    if (!pet) {
        if (!d->angles) return fail(RGRT_E_INVAL, "CT geometry needs view angles");
        for (int v = 0; v < d->n_views; v++)
            if (!std::isfinite(d->angles[v])) return fail(RGRT_E_INVAL, "non-finite view angle %d", v);
        if (!(d->pitch_u > 0) || !(d->pitch_v > 0) || !std::isfinite(d->pitch_u) ||
            !std::isfinite(d->pitch_v))
            return fail(RGRT_E_INVAL, "detector pitch must be positive and finite");
    }
    if (d->kind == RGRT_GEOM_CT_PARALLEL) {
        if (std::isnan(d->t_a) || std::isnan(d->t_b) || !(d->t_a < d->t_b))
            return fail(RGRT_E_INVAL, "parallel-beam segment needs t_a < t_b");
    }
    if (d->kind == RGRT_GEOM_CT_CONE) {
        if (!(d->dso > 0) || !(d->dsd > d->dso) || !std::isfinite(d->dsd))
            return fail(RGRT_E_INVAL, "cone beam needs 0 < dso < dsd (finite)");
    }
    if (pet) {
        if (!(d->radius > 0) || !std::isfinite(d->radius) || d->n_crystals <= 0)
            return fail(RGRT_E_INVAL, "PET ring needs radius > 0 and crystals > 0");
        if (!(d->pitch_v > 0) || !std::isfinite(d->pitch_v))
            return fail(RGRT_E_INVAL, "PET plane / ring spacing must be positive");
        if (d->arc_mode != 0 && d->arc_mode != 1) return fail(RGRT_E_INVAL, "arc_mode must be 0 or 1");
        double c = 0.5 * (double)(d->n_cols - 1);
        double smax = d->arc_mode == 0 ? c * (M_PI * d->radius / d->n_crystals) : d->radius;
        if (d->arc_mode == 1 && c * M_PI / d->n_crystals >= M_PI / 2)
            return fail(RGRT_E_INVAL, "raw radial bins reach beyond the ring");
        if (d->arc_mode == 0 && !(smax < d->radius))
            return fail(RGRT_E_INVAL, "radial bins reach beyond the ring");
    }
    return RGRT_OK;
}

}  // namespace

int rgrt::ctx_alloc(rgrt_ctx *c, void **p, size_t bytes) { return dev_alloc(c, p, bytes); }
void rgrt::ctx_free(rgrt_ctx *c, void *p, size_t bytes) { dev_free(c, p, bytes); }

int rgrt::gauss_adam(rgrt_gauss *g, cudaStream_t s)
{
    if (g->adam_m || g->n == 0) return RGRT_OK;
    void *p = nullptr;
    TRY(dev_alloc(g->ctx, &p, sizeof(float) * 22 * (size_t)g->n));
    CK(cudaMemsetAsync(p, 0, sizeof(float) * 22 * (size_t)g->n, s));
    g->adam_m = (float *)p;
    g->adam_v = g->adam_m + 11 * g->n;
    return RGRT_OK;
}

int64_t rgrt::desc_views(const rgrt_geom_desc *d)
{
    return d->kind == RGRT_GEOM_PET_3D ? (int64_t)d->n_views * (2 * (int64_t)d->max_ring_diff + 1)
                                       : (int64_t)d->n_views;
}

int64_t rgrt::desc_rays(const rgrt_geom_desc *d)
{
    return desc_views(d) * d->n_rows * d->n_cols;
}

void rgrt::geom_tables(const rgrt_geom_desc *d, float *tab, DevGeom &dg)
{
    const int V = (int)desc_views(d), H = d->n_rows, W = d->n_cols;
    const bool pet = d->kind == RGRT_GEOM_PET_RING || d->kind == RGRT_GEOM_PET_3D;
    const int n_ang = d->n_views;   // PET angles (per ring difference for 3-D PET)
    const double PI = 3.14159265358979323846;
    for (int v = 0; v < V; v++) {
        double eu[3], ev[3], ew[3];
        if (pet) {
            const int a = v % n_ang;
            double phi = d->angles ? d->angles[a] : (PI * (double)a) / (double)n_ang;
            double c = cos(phi), s = sin(phi);
            eu[0] = c; eu[1] = s; eu[2] = 0.0;
            ew[0] = s; ew[1] = -c; ew[2] = 0.0;
        } else {
            double th_ = d->angles[v];
            double c = cos(th_), s = sin(th_);
            ew[0] = c; ew[1] = s; ew[2] = 0.0;
            eu[0] = -s; eu[1] = c; eu[2] = 0.0;
        }
        ev[0] = 0.0; ev[1] = 0.0; ev[2] = 1.0;
        for (int k = 0; k < 3; k++) {
            tab[9 * v + k] = (float)eu[k];
            tab[9 * v + 3 + k] = (float)ev[k];
            tab[9 * v + 6 + k] = (float)ew[k];
        }
    }
    float *ut = tab + 9 * (size_t)V, *vt = ut + W;
    for (int i = 0; i < W; i++) {
        double k = (double)i - 0.5 * (double)(W - 1);
        double u;
        if (pet)
            u = d->arc_mode == 0 ? k * ((PI * d->radius) / (double)d->n_crystals)
                                 : d->radius * sin((k * PI) / (double)d->n_crystals);
        else
            u = k * d->pitch_u;
        ut[i] = (float)u;
    }
    for (int j = 0; j < H; j++) vt[j] = (float)(((double)j - 0.5 * (double)(H - 1)) * d->pitch_v);

    const int tw = d->tile_w ? d->tile_w : 16, th = d->tile_h ? d->tile_h : 16;
    dg = DevGeom{};
    dg.kind = d->kind == RGRT_GEOM_CT_CONE ? GM_CONE : d->kind == RGRT_GEOM_PET_3D ? GM_PET3D : GM_PARALLEL;
    dg.pet = pet;
    dg.n_views = V; dg.n_rows = H; dg.n_cols = W;
    dg.tile_w = tw; dg.tile_h = th;
    dg.tiles_x = (W + tw - 1) / tw;
    dg.tiles_y = (H + th - 1) / th;
    dg.v0 = 0;
    if (d->kind == RGRT_GEOM_PET_RING) { dg.stride_view = W; dg.stride_row = (long long)V * W; }
    else { dg.stride_view = (long long)H * W; dg.stride_row = W; }
    dg.dso = (float)d->dso;
    dg.dsd = (float)d->dsd;
    dg.t_a = (float)d->t_a;
    dg.t_b = (float)d->t_b;
    dg.radius2 = (float)(d->radius * d->radius);
    dg.n_ang = n_ang;
    dg.max_rd = d->kind == RGRT_GEOM_PET_3D ? d->max_ring_diff : 0;
    dg.ring_pitch = (float)d->pitch_v;
    // uniform tables: the search guesses from t0 + i step (the guess only
    // starts the search; its result comes from the table comparisons)
    dg.u0 = ut[0];
    dg.uinv = (W > 1 && (!pet || d->arc_mode == 0)) ? (float)((double)(W - 1) / ((double)ut[W - 1] - (double)ut[0])) : 0.0f;
    dg.v0f = vt[0];
    dg.vinv = H > 1 ? (float)((double)(H - 1) / ((double)vt[H - 1] - (double)vt[0])) : 0.0f;
}

// validation and error reporting shared with the allocation-free entry point
int rgrt::validate_geometry(const rgrt_geom_desc *d) { return validate_desc(d); }
int rgrt::report_error(int code, const char *msg) { return fail(code, "%s", msg); }

// ===========================================================================
// exported API
// ===========================================================================

extern "C" {

const char *rgrt_last_error(void) { return g_err.c_str(); }

int64_t rgrt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int rgrt_ctx_create(rgrt_ctx **out, int device, size_t budget)
{
    if (!out) return fail(RGRT_E_INVAL, "null output");
    *out = nullptr;
    int nd = 0;
    cudaError_t e = cudaGetDeviceCount(&nd);
    if (e != cudaSuccess) return fail(RGRT_E_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= nd) return fail(RGRT_E_INVAL, "device %d of %d", device, nd);
    CK(cudaSetDevice(device));
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    rgrt_ctx *c = new (std::nothrow) rgrt_ctx();
    if (!c) return fail(RGRT_E_NOMEM, "host allocation failed");
    c->device = device;
    c->budget = budget ? budget : (size_t)(0.9 * (double)fr);
    e = cudaMallocHost((void **)&c->h_total, sizeof(unsigned long long) * 2);
    if (e != cudaSuccess) {
        delete c;
        return fail(RGRT_E_CUDA, "cudaMallocHost: %s", cudaGetErrorString(e));
    }
    *out = c;
    return RGRT_OK;
}

int rgrt_ctx_destroy(rgrt_ctx *c)
{
    if (!c) return RGRT_OK;
    cudaSetDevice(c->device);
    prof_harvest(c);
    Buf *bufs[] = { &c->cnt, &c->off, &c->rect, &c->keys, &c->vals, &c->keys_alt, &c->vals_alt,
                    &c->sort_tmp, &c->scan_tmp, &c->ranges, &c->total, &c->I, &c->dLdI, &c->y,
                    &c->grad, &c->gflat, &c->partial, &c->stats, &c->loss, &c->loss_acc, &c->ball, &c->part,
                    &c->scene, &c->blk, &c->wblk, &c->clusters };
    for (Buf *b : bufs) release(c, *b);
    for (auto &b : c->stage_in) release(c, b);
    for (auto &b : c->stage_out) release(c, b);
    if (c->h_total) cudaFreeHost(c->h_total);
    delete c;
    return RGRT_OK;
}

int gaussians_create(rgrt_ctx *ctx, int64_t n, const float *mu3, const float *ls3, const float *q4,
                     const float *rho, int flags, rgrt_gauss **out)
{
    TRY(check_ctx(ctx));
    if (!out) return fail(RGRT_E_INVAL, "null output");
    *out = nullptr;
    if (n < 0 || n > (int64_t)0x7fffffff) return fail(RGRT_E_INVAL, "Gaussian count %lld", (long long)n);
    if (n > 0 && (!mu3 || !ls3 || !q4 || !rho)) return fail(RGRT_E_INVAL, "null parameter array");
    if (flags != RGRT_COPY && flags != RGRT_BORROW) return fail(RGRT_E_INVAL, "flags %d", flags);
    if (flags == RGRT_BORROW && n > 0 &&
        !(is_device_ptr(mu3) && is_device_ptr(ls3) && is_device_ptr(q4) && is_device_ptr(rho)))
        return fail(RGRT_E_INVAL, "RGRT_BORROW needs device arrays");
    rgrt_gauss *g = new (std::nothrow) rgrt_gauss();
    if (!g) return fail(RGRT_E_NOMEM, "host allocation failed");
    g->ctx = ctx;
    g->n = n;
    g->owned = flags == RGRT_COPY;
    size_t recb = sizeof(float4) * (REC_F4 + CREC_F4) * (size_t)(n > 0 ? n : 1);
    size_t parb = g->owned ? sizeof(float) * 11 * (size_t)n : 0;
    g->bytes = recb + parb;
    void *blk = nullptr;
    int r = dev_alloc(ctx, &blk, g->bytes);
    if (r != RGRT_OK) {
        delete g;
        return r;
    }
    g->block = blk;
    g->rec = (float4 *)blk;
    g->crec = g->rec + REC_F4 * (size_t)(n > 0 ? n : 1);
    if (g->owned) {
        float *p = (float *)(g->crec + CREC_F4 * (size_t)(n > 0 ? n : 1));
        g->mu = p;
        g->ls = p + 3 * n;
        g->q = p + 6 * n;
        g->rho = p + 10 * n;
        if (n > 0) {
            cudaMemcpy(g->mu, mu3, sizeof(float) * 3 * n, cudaMemcpyDefault);
            cudaMemcpy(g->ls, ls3, sizeof(float) * 3 * n, cudaMemcpyDefault);
            cudaMemcpy(g->q, q4, sizeof(float) * 4 * n, cudaMemcpyDefault);
            cudaError_t e = cudaMemcpy(g->rho, rho, sizeof(float) * n, cudaMemcpyDefault);
            if (e != cudaSuccess) {
                dev_free(ctx, blk, g->bytes);
                delete g;
                return fail(RGRT_E_CUDA, "copying parameters: %s", cudaGetErrorString(e));
            }
        }
    } else {
        g->mu = const_cast<float *>(mu3);
        g->ls = const_cast<float *>(ls3);
        g->q = const_cast<float *>(q4);
        g->rho = const_cast<float *>(rho);
    }
    *out = g;
    return RGRT_OK;
}

int gaussians_destroy(rgrt_gauss *g)
{
    if (!g) return RGRT_OK;
    rgrt_ctx *c = g->ctx;
    cudaSetDevice(c->device);
    if (c->bin_g == g) c->bin_valid = false;
    dev_free(c, g->block, g->bytes);
    if (g->adam_m) dev_free(c, g->adam_m, sizeof(float) * 22 * (size_t)g->n);
    delete g;
    return RGRT_OK;
}

int64_t gaussians_count(const rgrt_gauss *g) { return g ? g->n : -1; }

int gaussians_set_kernel(rgrt_gauss *g, int kernel)
{
    if (!g) return fail(RGRT_E_INVAL, "null Gaussians");
    if (kernel != RGRT_KERNEL_GAUSSIAN && kernel != RGRT_KERNEL_EPANECHNIKOV)
        return fail(RGRT_E_INVAL, "unknown kernel %d", kernel);
    g->kernel = kernel;
    g->version++;
    return RGRT_OK;
}

int gaussians_get(rgrt_gauss *g, float *mu3, float *ls3, float *q4, float *rho, void *stream)
{
    if (!g) return fail(RGRT_E_INVAL, "null Gaussians");
    TRY(check_ctx(g->ctx));
    cudaStream_t s = (cudaStream_t)stream;
    size_t n = (size_t)g->n;
    if (n == 0) return RGRT_OK;
    if (mu3) CK(cudaMemcpyAsync(mu3, g->mu, sizeof(float) * 3 * n, cudaMemcpyDefault, s));
    if (ls3) CK(cudaMemcpyAsync(ls3, g->ls, sizeof(float) * 3 * n, cudaMemcpyDefault, s));
    if (q4) CK(cudaMemcpyAsync(q4, g->q, sizeof(float) * 4 * n, cudaMemcpyDefault, s));
    if (rho) CK(cudaMemcpyAsync(rho, g->rho, sizeof(float) * n, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return RGRT_OK;
}

int gaussians_set(rgrt_gauss *g, const float *mu3, const float *ls3, const float *q4,
                  const float *rho, void *stream)
{
    if (!g) return fail(RGRT_E_INVAL, "null Gaussians");
    TRY(check_ctx(g->ctx));
    cudaStream_t s = (cudaStream_t)stream;
    size_t n = (size_t)g->n;
    if (n > 0) {
        if (mu3 && mu3 != g->mu) CK(cudaMemcpyAsync(g->mu, mu3, sizeof(float) * 3 * n, cudaMemcpyDefault, s));
        if (ls3 && ls3 != g->ls) CK(cudaMemcpyAsync(g->ls, ls3, sizeof(float) * 3 * n, cudaMemcpyDefault, s));
        if (q4 && q4 != g->q) CK(cudaMemcpyAsync(g->q, q4, sizeof(float) * 4 * n, cudaMemcpyDefault, s));
        if (rho && rho != g->rho) CK(cudaMemcpyAsync(g->rho, rho, sizeof(float) * n, cudaMemcpyDefault, s));
    }
    g->version++;
    return RGRT_OK;
}

int geometry_set(rgrt_ctx *ctx, const rgrt_geom_desc *d, rgrt_geom **out)
{
    TRY(check_ctx(ctx));
    if (!out) return fail(RGRT_E_INVAL, "null output");
    *out = nullptr;
    TRY(validate_desc(d));
    rgrt_geom *g = new (std::nothrow) rgrt_geom();
    if (!g) return fail(RGRT_E_NOMEM, "host allocation failed");
    g->ctx = ctx;
    g->desc = *d;
    g->desc.angles = nullptr;
    const int V = (int)desc_views(d), H = d->n_rows, W = d->n_cols;
    std::vector<float> tab((size_t)9 * V + W + H);
    DevGeom &dg = g->dg;
    geom_tables(d, tab.data(), dg);
    g->desc.tile_w = dg.tile_w;
    g->desc.tile_h = dg.tile_h;
    // the library's views: 3-D PET has one per (ring difference, angle)
    g->desc.n_views = V;
    g->bytes = sizeof(float) * tab.size();
    int r = dev_alloc(ctx, (void **)&g->d_tables, g->bytes);
    if (r != RGRT_OK) {
        delete g;
        return r;
    }
    cudaError_t e = cudaMemcpy(g->d_tables, tab.data(), g->bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(ctx, g->d_tables, g->bytes);
        delete g;
        return fail(RGRT_E_CUDA, "uploading geometry tables: %s", cudaGetErrorString(e));
    }
    dg.frames = g->d_tables;
    dg.utab = g->d_tables + 9 * (size_t)V;
    dg.vtab = dg.utab + W;
    g->tiles_per_view = dg.tiles_x * dg.tiles_y;
    g->n_rays = (int64_t)V * H * W;
    *out = g;
    return RGRT_OK;
}

int geometry_destroy(rgrt_geom *g)
{
    if (!g) return RGRT_OK;
    rgrt_ctx *c = g->ctx;
    cudaSetDevice(c->device);
    if (c->bin_geom == g) c->bin_valid = false;
    dev_free(c, g->d_mult, sizeof(float) * (size_t)g->n_rays);
    dev_free(c, g->d_add, sizeof(float) * (size_t)g->n_rays);
    if (g->rays) {
        dev_free(c, g->d_ro, sizeof(float4) * (size_t)g->n_rays);
        dev_free(c, g->d_rd, sizeof(float4) * (size_t)g->n_rays);
        dev_free(c, g->d_tof, sizeof(float2) * (size_t)g->n_rays);
    } else {
        dev_free(c, g->d_tables, g->bytes);
    }
    delete g;
    return RGRT_OK;
}

int geometry_set_rays(rgrt_ctx *ctx, int64_t n_rays, const float *o3, const float *d3,
                      const float *t2, rgrt_geom **out)
{
    return geometry_set_rays_tof(ctx, n_rays, o3, d3, t2, nullptr, out);
}

int geometry_set_rays_tof(rgrt_ctx *ctx, int64_t n_rays, const float *o3, const float *d3,
                          const float *t2, const float *tof2, rgrt_geom **out)
{
    TRY(check_ctx(ctx));
    if (!out) return fail(RGRT_E_INVAL, "null output");
    *out = nullptr;
    if (n_rays <= 0) return fail(RGRT_E_INVAL, "n_rays must be positive (%lld)", (long long)n_rays);
    if (!o3 || !d3 || !t2) return fail(RGRT_E_INVAL, "null ray array");
    if ((n_rays + 127) / 128 > 0x7fffffffLL) return fail(RGRT_E_INVAL, "too many rays");
    rgrt_geom *g = new (std::nothrow) rgrt_geom();
    if (!g) return fail(RGRT_E_NOMEM, "host allocation failed");
    g->ctx = ctx;
    g->rays = true;
    g->n_rays = n_rays;
    g->n_blocks = rays_blocks(n_rays);
    g->desc.n_views = 1;
    g->desc.n_rows = 1;
    g->desc.n_cols = 0;
    cudaStream_t s = nullptr;
    const size_t nb = sizeof(float4) * (size_t)n_rays;
    int r = dev_alloc(ctx, (void **)&g->d_ro, nb);
    if (r == RGRT_OK) r = dev_alloc(ctx, (void **)&g->d_rd, nb);
    const void *po = nullptr, *pd = nullptr, *pt = nullptr, *pf = nullptr;
    if (r == RGRT_OK && tof2) r = dev_alloc(ctx, (void **)&g->d_tof, sizeof(float2) * (size_t)n_rays);
    if (r == RGRT_OK && tof2)
        r = stage_input(ctx, ctx->stage_in[3], tof2, 2 * sizeof(float) * (size_t)n_rays, s, &pf);
    if (r == RGRT_OK) r = stage_input(ctx, ctx->stage_in[0], o3, 3 * sizeof(float) * (size_t)n_rays, s, &po);
    if (r == RGRT_OK) r = stage_input(ctx, ctx->stage_in[1], d3, 3 * sizeof(float) * (size_t)n_rays, s, &pd);
    if (r == RGRT_OK) r = stage_input(ctx, ctx->stage_in[2], t2, 2 * sizeof(float) * (size_t)n_rays, s, &pt);
    if (r == RGRT_OK) r = ensure(ctx, ctx->total, sizeof(unsigned long long) * 2);
    if (r == RGRT_OK) {
        uint32_t bad = 0;
        cudaError_t e = cudaMemsetAsync(ctx->total.p, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess)
            e = launch_rays_prep((const float *)po, (const float *)pd, (const float *)pt, (const float *)pf,
                                 n_rays, g->d_ro, g->d_rd, g->d_tof, (uint32_t *)ctx->total.p, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, ctx->total.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            r = fail(RGRT_E_CUDA, "preparing rays: %s", cudaGetErrorString(e));
        else if (bad)
            r = fail(RGRT_E_INVAL, "a ray has a non-finite origin, a zero or non-finite direction, "
                                   "a segment with t_a > t_b or NaN, or a NaN time of flight");
    }
    for (int k = 0; k < 4; k++) release(ctx, ctx->stage_in[k]);  // staged copies are not kept
    if (r != RGRT_OK) {
        if (g->d_ro) dev_free(ctx, g->d_ro, nb);
        if (g->d_rd) dev_free(ctx, g->d_rd, nb);
        if (g->d_tof) dev_free(ctx, g->d_tof, sizeof(float2) * (size_t)n_rays);
        delete g;
        return r;
    }
    *out = g;
    return RGRT_OK;
}

int64_t geometry_num_rays(const rgrt_geom *g) { return g ? g->n_rays : -1; }

static int set_ray_array(rgrt_ctx *ctx, float **dst, const float *src, int64_t n)
{
    const size_t bytes = sizeof(float) * (size_t)n;
    if (!src) {
        dev_free(ctx, *dst, bytes);
        *dst = nullptr;
        return RGRT_OK;
    }
    if (!*dst) TRY(dev_alloc(ctx, (void **)dst, bytes));
    CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyDefault));
    return RGRT_OK;
}

int geometry_set_tof(rgrt_geom *g, int n_tof, float spacing, float sigma)
{
    if (!g) return fail(RGRT_E_INVAL, "null geometry");
    TRY(check_ctx(g->ctx));
    if (g->rays || g->desc.kind != RGRT_GEOM_PET_RING)
        return fail(RGRT_E_INVAL, "time-of-flight bins apply to PET ring sinograms");
    if (n_tof < 1 || n_tof > RGRT_TOF_MAX_BINS)
        return fail(RGRT_E_INVAL, "%d time-of-flight bins (1..%d)", n_tof, RGRT_TOF_MAX_BINS);
    if (!(spacing > 0.0f) || !std::isfinite(spacing) || !(sigma > 0.0f) || !std::isfinite(sigma))
        return fail(RGRT_E_INVAL, "time-of-flight spacing and width must be positive and finite");
    if (g->d_mult || g->d_add)
        return fail(RGRT_E_INVAL, "set the measurement model after the time-of-flight bins");
    const int64_t lors = desc_rays(&g->desc);
    g->dg.n_tof = n_tof;
    g->dg.tof_h = spacing;
    g->dg.tof_t0 = -0.5f * (float)(n_tof - 1) * spacing;
    g->dg.tof_s2 = sigma * sigma;
    g->dg.tof_tau = 1.0f / (sigma * sigma);
    g->dg.stride_tof = lors;
    g->n_rays = lors * n_tof;
    return RGRT_OK;
}

int geometry_set_corrections(rgrt_geom *g, const float *mult, const float *add)
{
    if (!g) return fail(RGRT_E_INVAL, "null geometry");
    TRY(check_ctx(g->ctx));
    TRY(set_ray_array(g->ctx, &g->d_mult, mult, g->n_rays));
    TRY(set_ray_array(g->ctx, &g->d_add, add, g->n_rays));
    return RGRT_OK;
}

int project_forward(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, float *out_I,
                    void *stream)
{
    TRY(check_ctx(ctx));
    if (!g || !geom || !out_I) return fail(RGRT_E_INVAL, "null argument");
    if (g->ctx != ctx || geom->ctx != ctx) return fail(RGRT_E_INVAL, "objects of another context");
    cudaStream_t s = (cudaStream_t)stream;
    void *dout;
    bool back;
    size_t ob = sizeof(float) * (size_t)geom->n_rays;
    TRY(stage_output(ctx, ctx->stage_out[0], out_I, ob, &dout, &back));
    TRY(run_forward(ctx, g, geom, (float *)dout, s));
    if (back) {
        CK(cudaMemcpyAsync(out_I, dout, ob, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return RGRT_OK;
}

int project_backward(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, const float *dL_dI,
                     float *g_mu3, float *g_ls3, float *g_q4, float *g_rho, void *stream)
{
    TRY(check_ctx(ctx));
    if (!g || !geom || !dL_dI) return fail(RGRT_E_INVAL, "null argument");
    if (g->ctx != ctx || geom->ctx != ctx) return fail(RGRT_E_INVAL, "objects of another context");
    cudaStream_t s = (cudaStream_t)stream;
    const void *dw;
    TRY(stage_input(ctx, ctx->stage_in[0], dL_dI, sizeof(float) * (size_t)geom->n_rays, s, &dw));
    size_t n = (size_t)g->n;
    float *outs[4] = { g_mu3, g_ls3, g_q4, g_rho };
    const size_t sz[4] = { 3 * n, 3 * n, 4 * n, n };
    void *dev[4];
    bool back[4];
    for (int k = 0; k < 4; k++)
        TRY(stage_output(ctx, ctx->stage_out[k], outs[k], sizeof(float) * sz[k], &dev[k], &back[k]));
    TRY(run_backward(ctx, g, geom, (const float *)dw, (float *)dev[0], (float *)dev[1],
                     (float *)dev[2], (float *)dev[3], s));
    bool any = false;
    for (int k = 0; k < 4; k++)
        if (back[k]) {
            CK(cudaMemcpyAsync(outs[k], dev[k], sizeof(float) * sz[k], cudaMemcpyDeviceToHost, s));
            any = true;
        }
    if (any) CK(cudaStreamSynchronize(s));
    return RGRT_OK;
}

// forward, loss and dL/dI into ctx->dLdI, adjoint and parameter chain into
// the four device gradient arrays (shared by loss_step and loss_grad)
static int run_loss_grad(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, const void *dy,
                         int loss, const rgrt_adam *hp, float *gm, float *gl, float *gq, float *gr,
                         cudaStream_t s)
{
    const int64_t R = geom->n_rays, N = g->n;
    TRY(ensure(ctx, ctx->I, sizeof(float) * (size_t)R));
    TRY(ensure(ctx, ctx->dLdI, sizeof(float) * (size_t)R));
    int nblk = loss_blocks(R);
    TRY(ensure(ctx, ctx->partial, sizeof(double) * (size_t)nblk));
    TRY(ensure(ctx, ctx->loss, sizeof(float) * 4));
    const bool view_major = !geom->rays && geom->dg.stride_row == geom->dg.n_cols &&
                            geom->dg.stride_view == (long long)geom->dg.n_rows * geom->dg.n_cols;
    if (view_major && N > 0) {
        // the loss is separable over rays, so each view chunk runs forward,
        // loss and adjoint on one binning (a geometry binned in several chunks
        // is binned once per step, not once per pass)
        TRY(ensure(ctx, ctx->loss_acc, sizeof(double)));
        TRY(ensure(ctx, ctx->grad, sizeof(float4) * GRAD_F4 * (size_t)N));
        CK(cudaMemsetAsync(ctx->loss_acc.p, 0, sizeof(double), s));
        CK(cudaMemsetAsync(ctx->grad.p, 0, sizeof(float4) * GRAD_F4 * (size_t)N, s));
        TRY(build_records(ctx, g, s));
        Stats *st = nullptr;
        if (ctx->stats_on) {
            TRY(ensure(ctx, ctx->stats, sizeof(Stats)));
            CK(cudaMemsetAsync(ctx->stats.p, 0, sizeof(Stats), s));
            st = (Stats *)ctx->stats.p;
        }
        ctx->last_keys = 0;
        const int64_t HW = (int64_t)geom->dg.n_rows * geom->dg.n_cols;
        float *I = (float *)ctx->I.p, *dLdI = (float *)ctx->dLdI.p;
        const float *y = (const float *)dy;
        TRY(for_chunks(ctx, g, geom, s, false, [&](int v0, int nv, uint32_t K) -> int {
            (void)K;
            DevGeom dg = geom->dg;
            dg.v0 = v0;
            {
                PROF("k_forward");
                CK(launch_forward(dg, nv, g->rec, g->crec, (uint32_t *)ctx->vals.p, (uint2 *)ctx->ranges.p,
                                  I, st, g->kernel, s));
            }
            const int64_t off = (int64_t)v0 * HW, n = (int64_t)nv * HW;
            {
                PROF("k_loss");
                CK(launch_loss(loss, I + off, y + off, n, hp->kappa, hp->poisson_eps,
                               geom->d_mult ? geom->d_mult + off : nullptr,
                               geom->d_add ? geom->d_add + off : nullptr, dLdI + off,
                               (double *)ctx->partial.p, loss_blocks(n), (float *)ctx->loss.p, s,
                               (double *)ctx->loss_acc.p));
            }
            {
                PROF("k_adjoint");
                CK(launch_adjoint(dg, nv, g->rec, g->crec, (uint32_t *)ctx->vals.p, (uint2 *)ctx->ranges.p,
                                  dLdI, (float4 *)ctx->grad.p, g->kernel, s));
            }
            return RGRT_OK;
        }));
        PROF("k_param_chain");
        CK(launch_param_chain(g->mu, g->ls, g->q, g->rho, N, (float4 *)ctx->grad.p, gm, gl, gq, gr, s));
        return RGRT_OK;
    }
    TRY(run_forward(ctx, g, geom, (float *)ctx->I.p, s));
    {
        PROF("k_loss");
        CK(launch_loss(loss, (float *)ctx->I.p, (const float *)dy, R, hp->kappa, hp->poisson_eps,
                       geom->d_mult, geom->d_add,
                       (float *)ctx->dLdI.p, (double *)ctx->partial.p, nblk, (float *)ctx->loss.p, s));
    }
    if (N > 0) TRY(run_backward(ctx, g, geom, (float *)ctx->dLdI.p, gm, gl, gq, gr, s));
    return RGRT_OK;
}

static int check_loss_args(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, const float *y,
                           int loss, const rgrt_adam *hp)
{
    TRY(check_ctx(ctx));
    if (!g || !geom || !y || !hp) return fail(RGRT_E_INVAL, "null argument");
    if (g->ctx != ctx || geom->ctx != ctx) return fail(RGRT_E_INVAL, "objects of another context");
    if (loss != RGRT_LOSS_L2 && loss != RGRT_LOSS_POISSON) return fail(RGRT_E_INVAL, "loss %d", loss);
    return RGRT_OK;
}

int loss_step(rgrt_ctx *ctx, rgrt_gauss *g, const rgrt_geom *geom, const float *y, int loss,
              const rgrt_adam *hp, int t, float *loss_out, void *stream)
{
    TRY(check_loss_args(ctx, g, geom, y, loss, hp));
    if (t < 1) return fail(RGRT_E_INVAL, "Adam step t must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t R = geom->n_rays, N = g->n;
    const void *dy;
    TRY(stage_input(ctx, ctx->stage_in[0], y, sizeof(float) * (size_t)R, s, &dy));
    float *gf = nullptr;
    if (N > 0) {
        TRY(ensure(ctx, ctx->gflat, sizeof(float) * 11 * (size_t)N));
        gf = (float *)ctx->gflat.p;
    }
    TRY(run_loss_grad(ctx, g, geom, dy, loss, hp, gf, gf ? gf + 3 * N : nullptr,
                      gf ? gf + 6 * N : nullptr, gf ? gf + 10 * N : nullptr, s));
    if (N > 0) {
        if (!g->adam_m) {
            void *p = nullptr;
            TRY(dev_alloc(ctx, &p, sizeof(float) * 22 * (size_t)N));
            CK(cudaMemsetAsync(p, 0, sizeof(float) * 22 * (size_t)N, s));
            g->adam_m = (float *)p;
            g->adam_v = g->adam_m + 11 * N;
        }
        float bc1 = (float)(1.0 - pow((double)hp->beta1, (double)t));
        float bc2 = (float)(1.0 - pow((double)hp->beta2, (double)t));
        float *ps[4] = { g->mu, g->ls, g->q, g->rho };
        const int64_t off[4] = { 0, 3 * N, 6 * N, 10 * N }, len[4] = { 3 * N, 3 * N, 4 * N, N };
        const float lr[4] = { hp->lr_mu, hp->lr_logscale, hp->lr_quat, hp->lr_rho };
        PROF("k_adam");
        for (int k = 0; k < 4; k++)
            CK(launch_adam(ps[k], gf + off[k], g->adam_m + off[k], g->adam_v + off[k], len[k], lr[k],
                           hp->beta1, hp->beta2, hp->eps, bc1, bc2, nullptr, nullptr, s));
        g->version++;
    }
    if (loss_out) CK(cudaMemcpyAsync(loss_out, ctx->loss.p, sizeof(float), cudaMemcpyDefault, s));
    if (loss_out && !is_device_ptr(loss_out)) CK(cudaStreamSynchronize(s));
    return RGRT_OK;
}

int loss_grad(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, const float *y, int loss,
              const rgrt_adam *hp, float *loss_out, float *g_mu3, float *g_ls3, float *g_q4,
              float *g_rho, void *stream)
{
    TRY(check_loss_args(ctx, g, geom, y, loss, hp));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t R = geom->n_rays;
    const size_t n = (size_t)g->n;
    const void *dy;
    TRY(stage_input(ctx, ctx->stage_in[0], y, sizeof(float) * (size_t)R, s, &dy));
    float *outs[4] = { g_mu3, g_ls3, g_q4, g_rho };
    const size_t sz[4] = { 3 * n, 3 * n, 4 * n, n };
    void *dev[4];
    bool back[4];
    for (int k = 0; k < 4; k++)
        TRY(stage_output(ctx, ctx->stage_out[k], outs[k], sizeof(float) * sz[k], &dev[k], &back[k]));
    TRY(run_loss_grad(ctx, g, geom, dy, loss, hp, (float *)dev[0], (float *)dev[1], (float *)dev[2],
                      (float *)dev[3], s));
    bool sync = false;
    for (int k = 0; k < 4; k++)
        if (back[k]) {
            CK(cudaMemcpyAsync(outs[k], dev[k], sizeof(float) * sz[k], cudaMemcpyDeviceToHost, s));
            sync = true;
        }
    if (loss_out) {
        CK(cudaMemcpyAsync(loss_out, ctx->loss.p, sizeof(float), cudaMemcpyDefault, s));
        sync = sync || !is_device_ptr(loss_out);
    }
    if (sync) CK(cudaStreamSynchronize(s));
    return RGRT_OK;
}

int gaussians_voxelize(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_volume_desc *vol, float *out,
                       void *stream)
{
    TRY(check_ctx(ctx));
    if (!g || !vol || !out) return fail(RGRT_E_INVAL, "null argument");
    if (g->ctx != ctx) return fail(RGRT_E_INVAL, "Gaussians of another context");
    for (int a = 0; a < 3; a++) {
        if (vol->dims[a] <= 0 || vol->dims[a] > 65535 * 8)
            return fail(RGRT_E_INVAL, "volume dimension %d out of range (%d)", a, vol->dims[a]);
        if (!(vol->size[a] > 0.0) || !std::isfinite(vol->size[a]) || !std::isfinite(vol->origin[a]))
            return fail(RGRT_E_INVAL, "voxel size must be positive and finite, origin finite");
    }
    cudaStream_t s = (cudaStream_t)stream;
    VolDev v;
    v.ox = (float)vol->origin[0]; v.oy = (float)vol->origin[1]; v.oz = (float)vol->origin[2];
    v.sx = (float)vol->size[0]; v.sy = (float)vol->size[1]; v.sz = (float)vol->size[2];
    v.nx = vol->dims[0]; v.ny = vol->dims[1]; v.nz = vol->dims[2];
    v.bx = (v.nx + 7) / 8; v.by = (v.ny + 7) / 8; v.bz = (v.nz + 15) / 16;
    const int64_t nb = (int64_t)v.bx * v.by * v.bz;
    if (nb >= 0x7fffffffLL) return fail(RGRT_E_INVAL, "too many voxel bricks (%lld)", (long long)nb);
    const size_t nvox = (size_t)v.nx * v.ny * v.nz;
    void *dout;
    bool back;
    TRY(stage_output(ctx, ctx->stage_out[0], out, sizeof(float) * nvox, &dout, &back));
    const int64_t N = g->n;
    if (N == 0) {
        CK(cudaMemsetAsync(dout, 0, sizeof(float) * nvox, s));
    } else {
        TRY(build_records(ctx, g, s));
        TRY(ensure(ctx, ctx->cnt, sizeof(uint32_t) * (size_t)N));
        TRY(ensure(ctx, ctx->off, sizeof(uint32_t) * (size_t)N));
        TRY(ensure(ctx, ctx->rect, sizeof(uint4) * (size_t)N));
        TRY(ensure(ctx, ctx->scan_tmp, sizeof(unsigned long long) * scan_tmp_elems(N)));
        TRY(ensure(ctx, ctx->total, sizeof(unsigned long long) * 2));
        TRY(ensure(ctx, ctx->ranges, sizeof(uint2) * (size_t)nb));
        {
            PROF("vox_bin");
            CK(launch_vox_count(g->crec, N, v, (uint32_t *)ctx->cnt.p, (uint4 *)ctx->rect.p, s));
            CK(launch_scan((uint32_t *)ctx->cnt.p, (uint32_t *)ctx->off.p, N,
                           (unsigned long long *)ctx->total.p, (unsigned long long *)ctx->scan_tmp.p, s));
        }
        unsigned long long K = 0;
        TRY(read_totals(ctx, s, &K));
        if (K >= 0xffffffffull)
            return fail(RGRT_E_CAPACITY, "%llu (brick, Gaussian) entries (more than 2^32)", K);
        TRY(ensure(ctx, ctx->keys, sizeof(uint32_t) * (size_t)(K ? K : 1)));
        TRY(ensure(ctx, ctx->vals, sizeof(uint32_t) * (size_t)(K ? K : 1)));
        TRY(ensure(ctx, ctx->keys_alt, sizeof(uint32_t) * (size_t)(K ? K : 1)));
        TRY(ensure(ctx, ctx->vals_alt, sizeof(uint32_t) * (size_t)(K ? K : 1)));
        TRY(ensure(ctx, ctx->sort_tmp, sizeof(uint32_t) * sort_tmp_elems((uint32_t)(K ? K : 1))));
        uint32_t *keys = (uint32_t *)ctx->keys.p, *vals = (uint32_t *)ctx->vals.p;
        {
            PROF("vox_bin");
            CK(launch_vox_emit(N, v, (const uint32_t *)ctx->cnt.p, (const uint32_t *)ctx->off.p,
                               (const uint4 *)ctx->rect.p, keys, vals, (uint32_t)K, s));
            if (K > 0)
                CK(launch_sort(keys, vals, (uint32_t *)ctx->keys_alt.p, (uint32_t *)ctx->vals_alt.p,
                               (uint32_t)K, ceil_log2((uint64_t)nb) > 0 ? ceil_log2((uint64_t)nb) : 1,
                               (uint32_t *)ctx->sort_tmp.p, s));
            CK(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(uint2) * (size_t)nb, s));
            CK(launch_vox_ranges(keys, (uint32_t)K, (uint2 *)ctx->ranges.p, (uint32_t)nb, s));
        }
        ctx->bin_valid = false;   // the shared scratch now holds brick lists
        PROF("k_voxelize");
        CK(launch_voxelize(g->rec, g->crec, vals, (const uint2 *)ctx->ranges.p, v, (float *)dout, g->kernel, s));
    }
    if (back) {
        CK(cudaMemcpyAsync(out, dout, sizeof(float) * nvox, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return RGRT_OK;
}

int rgrt_debug_records(rgrt_ctx *ctx, const rgrt_gauss *g, float *sigma6, void *stream)
{
    TRY(check_ctx(ctx));
    if (!g || !sigma6) return fail(RGRT_E_INVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    TRY(build_records(ctx, g, s));
    std::vector<float4> h((size_t)CREC_F4 * g->n);
    if (g->n > 0)
        CK(cudaMemcpyAsync(h.data(), g->crec, sizeof(float4) * h.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<float> o((size_t)6 * g->n);
    for (int64_t k = 0; k < g->n; k++) {
        float4 a = h[CREC_F4 * k + 1], b = h[CREC_F4 * k + 2];
        float v[6] = { a.x, a.y, a.z, a.w, b.x, b.y };
        memcpy(&o[6 * k], v, sizeof(v));
    }
    if (!o.empty()) CK(cudaMemcpy(sigma6, o.data(), sizeof(float) * o.size(), cudaMemcpyDefault));
    return RGRT_OK;
}

int rgrt_debug_tile_lists(rgrt_ctx *ctx, const rgrt_gauss *g, const rgrt_geom *geom, int v0, int v1,
                          int64_t *n_keys_out, uint32_t *tile_start, uint32_t *gid, int64_t cap,
                          void *stream)
{
    TRY(check_ctx(ctx));
    if (!g || !geom || !n_keys_out || !tile_start) return fail(RGRT_E_INVAL, "null argument");
    if (geom->rays) return fail(RGRT_E_INVAL, "explicit rays have no tile lists");
    if (v0 < 0 || v1 > desc_views(&geom->desc) || v0 >= v1) return fail(RGRT_E_INVAL, "view range");
    cudaStream_t s = (cudaStream_t)stream;
    int nv = v1 - v0;
    uint32_t T = (uint32_t)nv * (uint32_t)geom->tiles_per_view;
    std::vector<uint32_t> start(T + 1, 0);
    uint32_t K = 0;
    if (g->n > 0) {
        TRY(build_records(ctx, g, s));
        TRY(bin_views(ctx, g, geom, v0, nv, s, &K));
        std::vector<uint2> rg(T);
        CK(cudaMemcpyAsync(rg.data(), ctx->ranges.p, sizeof(uint2) * T, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        uint32_t pos = 0;
        for (uint32_t t = 0; t < T; t++) {
            start[t] = pos;
            if (rg[t].y > rg[t].x) {
                if (rg[t].x != pos) return fail(RGRT_E_CUDA, "tile ranges are not contiguous");
                pos = rg[t].y;
            }
        }
        start[T] = pos;
        if (pos != K) return fail(RGRT_E_CUDA, "tile ranges cover %u of %u entries", pos, K);
    }
    *n_keys_out = K;
    CK(cudaMemcpy(tile_start, start.data(), sizeof(uint32_t) * (T + 1), cudaMemcpyDefault));
    if ((int64_t)K > cap) return fail(RGRT_E_CAPACITY, "%u entries, capacity %lld", K, (long long)cap);
    if (K > 0 && gid) CK(cudaMemcpy(gid, ctx->vals.p, sizeof(uint32_t) * K, cudaMemcpyDefault));
    return RGRT_OK;
}

int rgrt_prof_enable(rgrt_ctx *ctx, int on)
{
    if (!ctx) return fail(RGRT_E_INVAL, "null context");
    ctx->prof = on != 0;
    return RGRT_OK;
}

int rgrt_prof_reset(rgrt_ctx *ctx)
{
    if (!ctx) return fail(RGRT_E_INVAL, "null context");
    prof_harvest(ctx);
    ctx->prof_acc.clear();
    return RGRT_OK;
}

int rgrt_prof_get(rgrt_ctx *ctx, const char *name, int64_t *launches, double *ms)
{
    if (!ctx || !name) return fail(RGRT_E_INVAL, "null argument");
    prof_harvest(ctx);
    auto it = ctx->prof_acc.find(name);
    if (launches) *launches = it == ctx->prof_acc.end() ? 0 : it->second.first;
    if (ms) *ms = it == ctx->prof_acc.end() ? 0.0 : it->second.second;
    return RGRT_OK;
}

int rgrt_stats_enable(rgrt_ctx *ctx, int on)
{
    if (!ctx) return fail(RGRT_E_INVAL, "null context");
    ctx->stats_on = on != 0;
    return RGRT_OK;
}

int rgrt_stats_get(rgrt_ctx *ctx, int64_t *pairs_evaluated, int64_t *pairs_kept, int64_t *keys)
{
    TRY(check_ctx(ctx));
    Stats st{ 0, 0 };
    if (ctx->stats.p) CK(cudaMemcpy(&st, ctx->stats.p, sizeof(Stats), cudaMemcpyDeviceToHost));
    if (pairs_evaluated) *pairs_evaluated = (int64_t)st.pairs_eval;
    if (pairs_kept) *pairs_kept = (int64_t)st.pairs_kept;
    if (keys) *keys = ctx->last_keys;
    return RGRT_OK;
}

}  // extern "C"
