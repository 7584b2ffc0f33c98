// project_forward_noalloc: the forward projection with no memory allocation.
//
// Some callers cannot allocate device memory at the moment they project:
// applications whose device memory belongs to another allocator (a framework
// memory pool that must not be bypassed with cudaMalloc), code on a latency
// budget that cannot afford cudaMalloc/cudaFree (both may synchronise the
// whole device), or processes that have already reserved all device memory.
// For them this entry point runs the same pipeline as project_forward (records,
// cull, scan, emit, radix sort, tile ranges, integration) with every
// intermediate buffer carved out of one statically declared device array of
// RGRT_NOALLOC_SCRATCH_BYTES.  The array exists on every GPU that loads the
// library, for the life of the process.
//
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in symbol); the address is fetched with cudaGetSymbolAddress
// once per device, with that device current, by the first call made on the
// device -- so that first call must come before any stream capture.  All calls
// share the array: calls whose GPU work overlaps (unordered streams, several
// host threads) race and corrupt each other's results.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/rgrt.h"
#include "rgrt_internal.h"

using namespace rgrt;

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)RGRT_NOALLOC_SCRATCH_BYTES;
constexpr int MAX_DEVICES = 64;
constexpr int MAX_VIEWS = 1024, MAX_SIDE = 1024;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void *g_base[MAX_DEVICES];

// device address of g_scratch on the current device (looked up once)
int scratch_base(int dev, void **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return report_error(RGRT_E_INVAL, "device id out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char msg[200];
            snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the static scratch: %s",
                     cudaGetErrorString(e));
            return report_error(RGRT_E_CUDA, msg);
        }
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return RGRT_OK;
}

// device or managed memory of device `dev` (an array on another GPU would be
// read through peer access, or fault)
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// bump allocator over the scratch array (256-byte aligned pieces)
struct Carver {
    unsigned char *base;
    size_t used = 0;
    template <class T>
    T *take(size_t count)
    {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + sizeof(T) * (count ? count : 1);
        return reinterpret_cast<T *>(base + off);
    }
};

int ceil_log2_u(uint64_t x)
{
    int b = 0;
    while ((1ull << b) < x) b++;
    return b;
}

#define NA_CK(expr)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            char m_[256];                                                              \
            snprintf(m_, sizeof(m_), "%s: %s", #expr, cudaGetErrorString(e_));         \
            return report_error(RGRT_E_CUDA, m_);                                      \
        }                                                                              \
    } while (0)

}  // namespace

extern "C" int project_forward_noalloc(const rgrt_geom_desc *d, int64_t n, const float *mu3,
                                       const float *logscale3, const float *quat4,
                                       const float *rho, float *out_I, void *stream)
{
    if (!d || !out_I) return report_error(RGRT_E_INVAL, "null argument");
    if (n < 0 || n > (int64_t)0x7fffffff) return report_error(RGRT_E_INVAL, "Gaussian count");
    if (n > 0 && (!mu3 || !logscale3 || !quat4 || !rho))
        return report_error(RGRT_E_INVAL, "null parameter array");
    int rc = validate_geometry(d);
    if (rc != RGRT_OK) return rc;
    if (desc_views(d) > MAX_VIEWS || d->n_rows > MAX_SIDE || d->n_cols > MAX_SIDE)
        return report_error(RGRT_E_CAPACITY,
                            "project_forward_noalloc handles at most 1024 views of 1024 x 1024 pixels");
    const int V = (int)desc_views(d), H = d->n_rows, W = d->n_cols;
    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    if (!on_device(out_I, dev) || (n > 0 && !(on_device(mu3, dev) && on_device(logscale3, dev) &&
                                              on_device(quat4, dev) && on_device(rho, dev)))) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "project_forward_noalloc takes arrays in the memory of the current device (%d) only", dev);
        return report_error(RGRT_E_INVAL, msg);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t R = (int64_t)V * H * W;
    if (n == 0) {
        NA_CK(cudaMemsetAsync(out_I, 0, sizeof(float) * (size_t)R, s));
        return RGRT_OK;
    }
    void *base = nullptr;
    rc = scratch_base(dev, &base);
    if (rc != RGRT_OK) return rc;

    // geometry tables (the same binary32 values geometry_set uploads)
    float tab[9 * MAX_VIEWS + 2 * MAX_SIDE];
    DevGeom dg;
    geom_tables(d, tab, dg);

    // carve the fixed-size part of the scratch
    Carver cv{ (unsigned char *)base };
    const size_t ntab = (size_t)9 * V + W + H;
    float *d_tab = cv.take<float>(ntab);
    float4 *rec = cv.take<float4>((size_t)REC_F4 * n);
    float4 *crec = cv.take<float4>((size_t)CREC_F4 * n);
    const int64_t E = (int64_t)V * n;
    const uint32_t T = (uint32_t)V * (uint32_t)(dg.tiles_x * dg.tiles_y);
    uint32_t *cnt = cv.take<uint32_t>((size_t)E);
    uint32_t *off = cv.take<uint32_t>((size_t)E);
    uint2 *rect = cv.take<uint2>((size_t)E);
    unsigned long long *stmp = cv.take<unsigned long long>(scan_tmp_elems(E));
    unsigned long long *total = cv.take<unsigned long long>(2);
    uint2 *ranges = cv.take<uint2>(T);
    if (T >= (1u << 24))
        return report_error(RGRT_E_CAPACITY, "project_forward_noalloc: more than 2^24 tiles");
    if (cv.used > SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "project_forward_noalloc: %lld Gaussians x %d views need %zu bytes before binning, "
                 "over the %zu-byte static scratch",
                 (long long)n, V, cv.used, SCRATCH_BYTES);
        return report_error(RGRT_E_CAPACITY, msg);
    }
    dg.frames = d_tab;
    dg.utab = d_tab + 9 * (size_t)V;
    dg.vtab = dg.utab + W;

    NA_CK(cudaMemcpyAsync(d_tab, tab, sizeof(float) * ntab, cudaMemcpyHostToDevice, s));
    // total[1]: the records kernel's flag for non-finite parameters (the
    // scratch keeps the last call's contents, so it is cleared first)
    NA_CK(cudaMemsetAsync(total + 1, 0, sizeof(unsigned long long), s));
    NA_CK(launch_records(mu3, logscale3, quat4, rho, n, rec, crec, (uint32_t *)(total + 1), s));
    NA_CK(launch_cull(dg, V, crec, n, cnt, rect, s));
    NA_CK(launch_scan(cnt, off, E, total, stmp, s));
    unsigned long long tot[2] = { 0, 0 };
    NA_CK(cudaMemcpyAsync(tot, total, sizeof(tot), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (tot[1])
        return report_error(RGRT_E_INVAL, "non-finite Gaussian parameters (mu, log-scale, quaternion or rho)");
    const unsigned long long K = tot[0];
    // carve the part that depends on the number of (tile, Gaussian) entries
    uint32_t *keys = cv.take<uint32_t>(K);
    uint32_t *vals = cv.take<uint32_t>(K);
    uint32_t *keys_alt = cv.take<uint32_t>(K);
    uint32_t *vals_alt = cv.take<uint32_t>(K);
    uint32_t *sort_tmp = cv.take<uint32_t>(K < 0xffffffffull ? sort_tmp_elems((uint32_t)K) : 1);
    if (K >= 0xffffffffull || cv.used > SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "project_forward_noalloc: %llu tile entries need %zu bytes, over the %zu-byte "
                 "static scratch",
                 K, cv.used, SCRATCH_BYTES);
        return report_error(RGRT_E_CAPACITY, msg);
    }
    NA_CK(launch_emit(dg, V, n, cnt, off, rect, keys, vals, (uint32_t)K, nullptr, s));
    NA_CK(launch_sort(keys, vals, keys_alt, vals_alt, (uint32_t)K, ceil_log2_u(T) + 8, sort_tmp, s));
    // tiles without entries keep the zero range: clear before filling
    NA_CK(cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)T, s));
    NA_CK(launch_ranges(keys, (uint32_t)K, ranges, T, s));
    NA_CK(launch_forward(dg, V, rec, crec, vals, ranges, out_I, nullptr, RGRT_KERNEL_GAUSSIAN, s));
    return RGRT_OK;
}
