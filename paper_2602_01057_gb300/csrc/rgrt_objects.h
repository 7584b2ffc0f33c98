// Object layouts of the C ABI handles, shared by the translation units of
// librgrt that implement calls on them.
#pragma once
#include <map>
#include <string>
#include <vector>

#include "rgrt_internal.h"

namespace rgrt {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};

}  // namespace rgrt

struct rgrt_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    // scratch
    rgrt::Buf cnt, off, rect, keys, vals, keys_alt, vals_alt, sort_tmp, scan_tmp, ranges, total;
    rgrt::Buf stage_in[4], stage_out[4], I, dLdI, y, grad, gflat, partial, stats, loss, loss_acc;
    rgrt::Buf ball, part, scene, blk, wblk, clusters;    // explicit-ray binning
    std::vector<uint32_t> h_cnt;               // per-block list lengths (explicit rays)
    unsigned long long *h_total = nullptr;  // pinned
    // binning cache
    const rgrt_gauss *bin_g = nullptr;
    const rgrt_geom *bin_geom = nullptr;
    unsigned long long bin_version = 0;
    int bin_v0 = -1, bin_nv = 0;
    uint32_t bin_keys = 0;
    bool bin_valid = false;
    // profiling
    bool prof = false;
    bool stats_on = false;
    std::vector<rgrt::ProfRec> pending;
    std::map<std::string, std::pair<long long, double>> prof_acc;
    long long last_keys = 0;
};

struct rgrt_gauss {
    rgrt_ctx *ctx = nullptr;
    int64_t n = 0;
    bool owned = false;
    float *mu = nullptr, *ls = nullptr, *q = nullptr, *rho = nullptr;
    void *block = nullptr;     // owned parameter block (COPY)
    float4 *rec = nullptr, *crec = nullptr;
    float *adam_m = nullptr, *adam_v = nullptr;
    unsigned long long version = 1;
    int kernel = RGRT_KERNEL_GAUSSIAN;   // kernel of the primitives
    size_t bytes = 0;
};

struct rgrt_geom {
    rgrt_ctx *ctx = nullptr;
    rgrt_geom_desc desc{};
    rgrt::DevGeom dg{};
    float *d_tables = nullptr;
    int64_t n_rays = 0;
    // explicit rays: per ray (o', t_a') and (unit d, t_b'); ray blocks
    bool rays = false;
    float4 *d_ro = nullptr, *d_rd = nullptr;
    float2 *d_tof = nullptr;   // explicit rays with time of flight: (t_c, 1/sigma_T^2)
    int n_blocks = 0;
    // measurement model per ray (optional): multiplicative factor, additive background
    float *d_mult = nullptr, *d_add = nullptr;
    int tiles_per_view = 0;
    size_t bytes = 0;
};


namespace rgrt {
// device allocation counted against the context's HBM budget
int ctx_alloc(rgrt_ctx *c, void **p, size_t bytes);
void ctx_free(rgrt_ctx *c, void *p, size_t bytes);
// Adam state of a Gaussian set (allocated on first use)
int gauss_adam(rgrt_gauss *g, cudaStream_t s);
}  // namespace rgrt
