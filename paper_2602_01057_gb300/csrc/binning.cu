// Binning (a2, second half): exclusive scan of per-(view, Gaussian) tile
// counts, emission of (tile, position, Gaussian) keys, a stable LSD radix
// sort on the key bits, and per-tile ranges.  Keys are emitted in (view,
// Gaussian) order and the sort is stable, so each tile's list is ordered by
// footprint position and then by Gaussian id: the lists are canonical and the
// per-ray sums deterministic.  Being emitted view by view, the keys are
// already grouped by view: the sort then orders each view's keys on their
// own (on the tile within the view and the position code), which takes
// fewer 8-bit passes than sorting on the view's bits too.
#include "rgrt_internal.h"

namespace rgrt {
namespace {

constexpr int SCAN_BS = 256;
constexpr int SCAN_IPT = 16;
constexpr int SCAN_TILE = SCAN_BS * SCAN_IPT;

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *sh)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, int64_t n, unsigned long long *part)
{
    __shared__ unsigned long long sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; i++) {
        int64_t x = base + (int64_t)i * SCAN_BS + threadIdx.x;
        if (x < n) s += in[x];
    }
    s = block_sum_u64(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// single block: exclusive scan of part[0..nb) in place, total to *total
__global__ void k_scan_top(unsigned long long *part, int64_t nb, unsigned long long *total)
{
    __shared__ unsigned long long sh[32];
    __shared__ unsigned long long carry_sh;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_sh = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t x = base + threadIdx.x;
        unsigned long long v = x < nb ? part[x] : 0ull;
        unsigned long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) sh[w] = inc;
        __syncthreads();
        if (w == 0) {
            unsigned long long s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
            unsigned long long si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long t = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o) si += t;
            }
            if (lane < (int)(blockDim.x >> 5)) sh[lane] = si - s;
        }
        __syncthreads();
        unsigned long long carry = carry_sh;
        unsigned long long excl = carry + sh[w] + inc - v;
        if (x < nb) part[x] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_sh = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_sh;
}

__global__ void k_scan_down(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                            const unsigned long long *__restrict__ part)
{
    __shared__ uint32_t sm[SCAN_TILE];
    __shared__ uint32_t wsum[SCAN_BS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; i++) {
        int64_t x = base + (int64_t)i * SCAN_BS + t;
        sm[i * SCAN_BS + t] = x < n ? in[x] : 0u;
    }
    __syncthreads();
    uint32_t loc[SCAN_IPT];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_IPT; j++) { loc[j] = sm[t * SCAN_IPT + j]; s += loc[j]; }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t v = lane < SCAN_BS / 32 ? wsum[lane] : 0u;
        uint32_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += u;
        }
        if (lane < SCAN_BS / 32) wsum[lane] = vi - v;
    }
    __syncthreads();
    uint32_t run = (uint32_t)part[blockIdx.x] + wsum[w] + inc - s;
#pragma unroll
    for (int j = 0; j < SCAN_IPT; j++) { sm[t * SCAN_IPT + j] = run; run += loc[j]; }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_IPT; i++) {
        int64_t x = base + (int64_t)i * SCAN_BS + t;
        if (x < n) out[x] = sm[i * SCAN_BS + t];
    }
}

// one thread per (view of the chunk, Gaussian): write its tiles' keys.
// key = tile id << 8 | position code, the code being the 4-bit row and
// column buckets of the centre of the Gaussian's pixel box within the tile:
// sorting by it orders each tile's list by footprint position (Gaussians of
// the same position keep ascending ids, the sort being stable).
// One thread per (view of the chunk, Gaussian) item; a CTA's 256 items own
// one contiguous output range (the offsets are their exclusive scan).  With
// STAGE the range is staged in shared memory and written out coalesced when
// it fits -- worth it when items emit several keys each (large footprints);
// with a key or two per item the direct writes are as compact and the
// staging buffer only costs occupancy.
constexpr int EMIT_BS = 256;
constexpr int EMIT_STAGE = 4096;

// lbits >= 0: the key's tile field is (view << lbits) | tile within the
// view (the views' keys then sort on their own; see launch_sort_views);
// lbits < 0: the tile id of the chunk, view * tiles per view + tile.
__device__ __forceinline__ void emit_item(const DevGeom &g, int vl, uint32_t k, uint2 r, uint32_t o,
                                          uint32_t *kd, uint32_t *vd, int lbits)
{
    const int i0 = r.x & 0xffff, i1 = r.x >> 16, j0 = r.y & 0xffff, j1 = r.y >> 16;
    const int tw = g.tile_w, th = g.tile_h;
    const int tx0 = i0 / tw, tx1 = i1 / tw, ty0 = j0 / th, ty1 = j1 / th;
    const uint32_t tbase = lbits >= 0 ? (uint32_t)vl << lbits : (uint32_t)vl * (uint32_t)(g.tiles_x * g.tiles_y);
    for (int ty = ty0; ty <= ty1; ty++) {
        const int jl = max(j0 - ty * th, 0), jh = min(j1 - ty * th, th - 1);
        const uint32_t rb = (uint32_t)(((jl + jh) * 8) / th);
        for (int tx = tx0; tx <= tx1; tx++) {
            const int il = max(i0 - tx * tw, 0), ih = min(i1 - tx * tw, tw - 1);
            const uint32_t cb = (uint32_t)(((il + ih) * 8) / tw);
            kd[o] = ((tbase + (uint32_t)ty * (uint32_t)g.tiles_x + (uint32_t)tx) << 8) | (rb << 4) | cb;
            vd[o] = k;
            o++;
        }
    }
}

template <bool STAGE>
__global__ void __launch_bounds__(EMIT_BS) k_emit(DevGeom g, int nv, int64_t n,
                                                  const uint32_t *__restrict__ cnt,
                                                  const uint32_t *__restrict__ off,
                                                  const uint2 *__restrict__ rect,
                                                  uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                  uint32_t cap, uint32_t *overflow, int lbits)
{
    __shared__ uint32_t sk[STAGE ? EMIT_STAGE : 1], sv[STAGE ? EMIT_STAGE : 1];
    const int64_t tot = (int64_t)nv * n;
    const int64_t first = (int64_t)blockIdx.x * EMIT_BS;
    const int64_t last = min(first + EMIT_BS, tot) - 1;
    const int64_t idx = first + threadIdx.x;
    const uint64_t rs = off[first], re = (uint64_t)off[last] + cnt[last];
    // staged only when the whole range fits the buffer (an item past the
    // capacity writes nothing, as in the direct path)
    const bool staged = STAGE && re - rs <= (uint64_t)EMIT_STAGE && re <= (uint64_t)cap;
    uint32_t c = 0;
    if (idx < tot) {
        c = cnt[idx];
        if (c != 0) {
            const uint32_t o = off[idx];
            if ((uint64_t)o + c > cap) {   // more entries than the buffer holds
                if (overflow) atomicOr(overflow, 1u);
                // its slots below the capacity get the padding key (sorts
                // last, maps to no tile), so that no slot is left stale
                for (uint32_t e = o; e < cap && e < o + c; e++) keys[e] = 0xffffffffu;
            } else {
                const int vl = (int)(idx / n);
                const uint32_t k = (uint32_t)(idx - (int64_t)vl * n);
                if (staged) emit_item(g, vl, k, rect[idx], o - (uint32_t)rs, sk, sv, lbits);
                else emit_item(g, vl, k, rect[idx], o, keys, vals, lbits);
            }
        }
    }
    if (!staged) return;     // uniform over the CTA
    __syncthreads();
    const uint32_t m = (uint32_t)(re - rs);
    for (uint32_t e = threadIdx.x; e < m; e += EMIT_BS) {
        keys[rs + e] = sk[e];
        vals[rs + e] = sv[e];
    }
}

constexpr int SORT_BS = 256;     // one thread per digit value
constexpr int SORT_ITEMS = 16;   // keys per thread
constexpr int SORT_TILE = SORT_BS * SORT_ITEMS;
constexpr int SORT_WARPS = SORT_BS / 32;
constexpr int SORT_WSEG = 32 * SORT_ITEMS;   // keys of one warp's segment

// Keys of a tile: warp w owns the contiguous segment [w SORT_WSEG, (w + 1)
// SORT_WSEG) of it, read lane-striped (item i of lane l is key i 32 + l), so
// walking items in order and lanes in order visits the segment in key order.

// n_dev (nullable): the number of keys to sort, read on the device (at most n;
// the grid and the histogram layout follow n)
__device__ __forceinline__ uint32_t sort_count(uint32_t n, const unsigned long long *n_dev)
{
    return n_dev ? (uint32_t)min((unsigned long long)n, *n_dev) : n;
}

// Segments (nullable tables): the keys of each segment -- one view's keys,
// contiguous in the emitted array -- are sorted on their own.  Segment s
// holds keys [seg_start[s], seg_start[s + 1]) and sort tiles [tile_start[s],
// tile_start[s + 1]); tile_start[ns] is the number of tiles in use.
struct SortSegs {
    const uint32_t *tile_start = nullptr;
    const uint32_t *seg_start = nullptr;
    const uint4 *span = nullptr;   // [nb]: every tile's (lo, hi, hb, hs), from k_sort_spans
    int ns = 0;
};

// The keys [lo, hi) of sort tile b, and where its count of digit d sits in
// the histogram: hist[hb + d hs].  Without segments tile b holds keys
// [b SORT_TILE, (b + 1) SORT_TILE) and its counts are hist[d nb + b]: one
// exclusive scan over the histogram then gives every (digit, tile) its
// output offset.  With segments, segment s's counts sit digit-major from
// 256 tile_start[s] on (the same scan then orders segment by segment, and
// within one by digit and tile); tiles past the ones in use are empty and
// own the histogram's tail [256 tile_start[ns], 256 nb), which they zero.
struct TileSpan {
    uint32_t lo, hi;
    size_t hb, hs;
};

__device__ __forceinline__ TileSpan tile_span(uint32_t b, uint32_t nb, uint32_t n, const SortSegs &sg)
{
    TileSpan t;
    if (!sg.tile_start) {
        t.lo = b * SORT_TILE;
        t.hi = t.lo < n ? min(n, t.lo + SORT_TILE) : t.lo;
        t.hb = b;
        t.hs = nb;
        return t;
    }
    if (sg.span) {
        const uint4 q = sg.span[b];
        t.lo = q.x;
        t.hi = q.y;
        t.hb = q.z;
        t.hs = q.w;
        return t;
    }
    const uint32_t used = sg.tile_start[sg.ns];
    if (b >= used) {
        t.lo = t.hi = 0;
        t.hb = (size_t)256 * b;
        t.hs = 1;
        return t;
    }
    // the segment s with tile_start[s] <= b < tile_start[s + 1]
    int a = 0, c = sg.ns;
    while (c - a > 1) {
        const int m = (a + c) >> 1;
        if (sg.tile_start[m] <= b) a = m;
        else c = m;
    }
    const uint32_t t0 = sg.tile_start[a], tl = b - t0;
    t.lo = sg.seg_start[a] + tl * SORT_TILE;
    t.hi = min(sg.seg_start[a + 1], t.lo + SORT_TILE);
    t.hb = (size_t)256 * t0 + tl;
    t.hs = sg.tile_start[a + 1] - t0;
    return t;
}

__global__ void k_sort_hist(const uint32_t *__restrict__ keys, uint32_t n, int shift,
                            uint32_t *__restrict__ hist, uint32_t nb, const unsigned long long *n_dev,
                            SortSegs sg)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    n = sort_count(n, n_dev);
    const TileSpan sp = tile_span(blockIdx.x, nb, n, sg);
    __syncthreads();
    // the tile as 16-byte loads from the 16-byte boundary at or below its
    // first key (every load issued before the counting; one more vector
    // covers the tail a misaligned start pushes out), scalar loads past its
    // last key or when the key array is not 16-byte aligned
    const bool vec = ((uintptr_t)keys & 15u) == 0;
    const uint32_t a0 = vec ? sp.lo & ~3u : sp.lo;
    constexpr int V = SORT_ITEMS / 4;
    uint4 q[V + 1];
#pragma unroll
    for (int j = 0; j <= V; j++) {
        const uint32_t k = a0 + 4 * (threadIdx.x + j * SORT_BS);
        if (vec && k + 3 < sp.hi) {
            q[j] = __ldg(reinterpret_cast<const uint4 *>(keys + k));
        } else {
            q[j].x = k < sp.hi ? keys[k] : 0u;
            q[j].y = k + 1 < sp.hi ? keys[k + 1] : 0u;
            q[j].z = k + 2 < sp.hi ? keys[k + 2] : 0u;
            q[j].w = k + 3 < sp.hi ? keys[k + 3] : 0u;
        }
    }
#pragma unroll
    for (int j = 0; j <= V; j++) {
        const uint32_t k = a0 + 4 * (threadIdx.x + j * SORT_BS);
        const uint32_t e[4] = { q[j].x, q[j].y, q[j].z, q[j].w };
#pragma unroll
        for (int c = 0; c < 4; c++)
            if (k + c >= sp.lo && k + c < sp.hi) atomicAdd(&h[(e[c] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[sp.hb + (size_t)threadIdx.x * sp.hs] = h[threadIdx.x];
}

// Scatter of one radix pass.  A CTA takes a tile of SORT_TILE keys and ranks
// them stably by digit: every warp ranks its segment with warp-private digit
// counters (items in order, lanes in order, peers of a digit from
// match_any), a per-digit scan over the warps and one over the digits give
// tile-local positions; keys and values are placed there in shared memory
// and written out in that order -- each digit's keys are consecutive there
// and land consecutively at the digit's global offset (runs, not single words).
__global__ void __launch_bounds__(SORT_BS) k_sort_scatter(const uint32_t *__restrict__ keys,
                                                          const uint32_t *__restrict__ vals,
                                                          uint32_t *__restrict__ okeys,
                                                          uint32_t *__restrict__ ovals, uint32_t n,
                                                          int shift, const uint32_t *__restrict__ hist,
                                                          const uint32_t *__restrict__ offs, uint32_t nb,
                                                          const unsigned long long *n_dev, SortSegs sg)
{
    __shared__ uint32_t sk[SORT_TILE], sv[SORT_TILE];
    __shared__ uint32_t wcnt[SORT_WARPS][256];
    __shared__ uint32_t lbase[256], gofs[256], wsum[SORT_WARPS];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    n = sort_count(n, n_dev);
    const TileSpan sp = tile_span(blockIdx.x, nb, n, sg);
    if (sp.hi <= sp.lo) return;   // uniform over the CTA: a tile with no keys
    const uint32_t base = sp.lo, end = sp.hi;
    const uint32_t seg = base + w * SORT_WSEG;
    // every global load of the tile up front: keys, values, and the tile's
    // count and global offset of every digit
    uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; i++) {
        const uint32_t k = seg + i * 32 + lane;
        key[i] = k < end ? keys[k] : 0u;
        val[i] = k < end ? vals[k] : 0u;
    }
    const uint32_t my_ofs = offs[sp.hb + (size_t)t * sp.hs];
#pragma unroll
    for (int ww = 0; ww < SORT_WARPS; ww++) wcnt[ww][t] = 0;
    gofs[t] = my_ofs;
    // tile-local start of every digit: exclusive scan of the tile's histogram
    {
        const uint32_t c = hist[sp.hb + (size_t)t * sp.hs];
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t add = 0;
        for (int ww = 0; ww < w; ww++) add += wsum[ww];
        lbase[t] = add + x - c;
    }
    // warp-local ranks
    uint32_t *cnt = wcnt[w];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; i++) {
        const bool valid = seg + i * 32 + lane < end;
        const uint32_t d = valid ? (key[i] >> shift) & 255u : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = cnt[d & 255u];
        rank[i] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0u) cnt[d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps' runs (exclusive over warps)
    {
        uint32_t acc = lbase[t];
#pragma unroll
        for (int ww = 0; ww < SORT_WARPS; ww++) {
            const uint32_t c = wcnt[ww][t];
            wcnt[ww][t] = acc;
            acc += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; i++) {
        const uint32_t k = seg + i * 32 + lane;
        if (k < end) {
            const uint32_t at = cnt[(key[i] >> shift) & 255u] + rank[i];
            if (at < SORT_TILE) {
                sk[at] = key[i];
                sv[at] = val[i];
            }
        }
    }
    __syncthreads();
    const uint32_t cnt_tile = end - base;
    for (uint32_t k = t; k < cnt_tile; k += SORT_BS) {
        const uint32_t kk = sk[k];
        const uint32_t d = (kk >> shift) & 255u;
        uint32_t dst = gofs[d] + (k - lbase[d]);
        if (dst >= n) dst = base + k;  // never taken when the histogram scan is consistent
        okeys[dst] = kk;
        ovals[dst] = sv[k];
    }
}

// Segment tables of launch_sort_views: segment v (a view) starts at key
// off[v stride] (the scan of the per-(view, Gaussian) counts) and takes
// ceil(len / SORT_TILE) sort tiles; one block scans the tile counts.
__global__ void k_sort_segments(const uint32_t *__restrict__ off, int64_t stride, int ns, uint32_t n,
                                const unsigned long long *n_dev, uint32_t *__restrict__ tile_start,
                                uint32_t *__restrict__ seg_start)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    n = sort_count(n, n_dev);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base <= ns; base += blockDim.x) {
        const int v = base + (int)threadIdx.x;
        uint32_t tiles = 0;
        if (v <= ns) {
            const uint32_t st = v < ns ? min(off[(int64_t)v * stride], n) : n;
            seg_start[v] = st;
            if (v < ns) {
                const uint32_t en = v + 1 < ns ? min(off[(int64_t)(v + 1) * stride], n) : n;
                tiles = (en - st + SORT_TILE - 1) / SORT_TILE;
            }
        }
        uint32_t inc = tiles;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t add = carry;
        for (int ww = 0; ww < w; ww++) add += wsum[ww];
        if (v <= ns) tile_start[v] = add + inc - tiles;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int ww = 0; ww < nw; ww++) tot += wsum[ww];
            carry += tot;
        }
        __syncthreads();
    }
}

// Every sort tile's span (tile_span of the segment tables, once per sort
// rather than once per tile and pass)
__global__ void k_sort_spans(uint32_t nb, uint32_t n, const unsigned long long *n_dev, SortSegs sg,
                             uint4 *__restrict__ span)
{
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    n = sort_count(n, n_dev);
    sg.span = nullptr;
    const TileSpan t = tile_span(b, nb, n, sg);
    span[b] = make_uint4(t.lo, t.hi, (uint32_t)t.hb, (uint32_t)t.hs);
}

// Tile ranges of the sorted keys: entry i opens tile k = key >> 8 if the key
// before it has another tile, and closes it if the key after it does.  A
// thread takes RANGE_ITEMS consecutive keys as 16-byte loads (scalar loads
// for a ragged end or an unaligned array) and its two neighbours.
constexpr int RANGE_ITEMS = 8;

// With lbits >= 0 the key's tile field is (view << lbits) | tile within the
// view, decoded here to view * tpv + tile.
__global__ void k_ranges(const uint32_t *__restrict__ keys, uint32_t n, uint2 *__restrict__ ranges,
                         uint32_t n_tiles, const unsigned long long *n_dev, uint32_t tpv, int lbits)
{
    n = sort_count(n, n_dev);
    const uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) * RANGE_ITEMS;
    if (i0 >= n) return;
    uint32_t k[RANGE_ITEMS + 2];
    k[0] = i0 > 0 ? keys[i0 - 1] >> 8 : 0xffffffffu;
    if (((uintptr_t)keys & 15u) == 0 && i0 + RANGE_ITEMS <= n) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(keys + i0));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(keys + i0) + 1);
        k[1] = a.x >> 8; k[2] = a.y >> 8; k[3] = a.z >> 8; k[4] = a.w >> 8;
        k[5] = b.x >> 8; k[6] = b.y >> 8; k[7] = b.z >> 8; k[8] = b.w >> 8;
    } else {
#pragma unroll
        for (int j = 0; j < RANGE_ITEMS; j++) k[j + 1] = i0 + j < n ? keys[i0 + j] >> 8 : 0xffffffffu;
    }
    k[RANGE_ITEMS + 1] = i0 + RANGE_ITEMS < n ? keys[i0 + RANGE_ITEMS] >> 8 : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < RANGE_ITEMS; j++) {
        const uint32_t i = i0 + j, f = k[j + 1];
        // keys past n read as 0xffffffff, which is no tile; emitted tile ids are < n_tiles
        uint64_t t = f;
        if (lbits >= 0) {
            const uint32_t tl = f & ((1u << lbits) - 1u);
            t = tl < tpv ? (uint64_t)(f >> lbits) * tpv + tl : ~0ull;
        }
        if (i >= n || t >= n_tiles) continue;
        if (k[j] != f) ranges[t].x = i;
        if (k[j + 2] != f) ranges[t].y = i + 1;
    }
}

}  // namespace

size_t scan_tmp_elems(int64_t n)
{
    return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 1;
}

cudaError_t launch_scan(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *total,
                        unsigned long long *tmp, cudaStream_t s)
{
    if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, n, tmp);
    k_scan_top<<<1, 1024, 0, s>>>(tmp, nb, total);
    k_scan_down<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, out, n, tmp);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_emit(const DevGeom &g, int nv, int64_t n, const uint32_t *cnt,
                        const uint32_t *off, const uint2 *rect, uint32_t *keys, uint32_t *vals,
                        uint32_t cap, uint32_t *overflow, cudaStream_t s, int lbits)
{
    int64_t tot = (int64_t)nv * n;
    if (tot <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((tot + EMIT_BS - 1) / EMIT_BS);
    if ((double)cap >= 3.0 * (double)tot)
        k_emit<true><<<grid, EMIT_BS, 0, s>>>(g, nv, n, cnt, off, rect, keys, vals, cap, overflow, lbits);
    else
        k_emit<false><<<grid, EMIT_BS, 0, s>>>(g, nv, n, cnt, off, rect, keys, vals, cap, overflow, lbits);
    count_launches(1);
    return cudaGetLastError();
}

// Scratch of a sort of n keys in ns segments (ns = 0: one): the histogram
// and its scan [256 nb] each, the scan's 64-bit scratch, and the segment
// tables [ns + 1] each.
struct SortLayout {
    uint32_t nb;
    size_t hn, stmp, stot, tiles, segs, span, total;
};

SortLayout sort_layout(uint32_t n, int ns)
{
    SortLayout L;
    L.nb = (uint32_t)(((size_t)n + SORT_TILE - 1) / SORT_TILE + (ns > 0 ? (size_t)ns + 1 : 0));
    L.hn = (size_t)256 * L.nb;
    L.stmp = (2 * L.hn + 1) & ~(size_t)1;                      // u32 index, 8-byte aligned
    L.stot = L.stmp + 2 * scan_tmp_elems((int64_t)L.hn);
    L.tiles = L.stot + 2;
    L.segs = L.tiles + (ns > 0 ? (size_t)ns + 1 : 0);
    L.span = (L.segs + (ns > 0 ? (size_t)ns + 1 : 0) + 3) & ~(size_t)3;   // 16-byte aligned
    L.total = L.span + (ns > 0 ? 4 * (size_t)L.nb : 0) + 8;
    return L;
}

size_t sort_tmp_elems(uint32_t n, int ns)
{
    return sort_layout(n, ns).total;
}

namespace {

cudaError_t sort_passes(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                        uint32_t n, int bits, uint32_t *tmp, const SortLayout &L, SortSegs sg,
                        cudaStream_t s, bool *in_alt, const unsigned long long *n_dev)
{
    uint32_t *hist = tmp;
    uint32_t *offs = tmp + L.hn;
    unsigned long long *stmp = (unsigned long long *)(tmp + L.stmp);
    unsigned long long *stot = (unsigned long long *)(tmp + L.stot);
    const uint32_t nb = L.nb;
    uint32_t *src_k = keys, *src_v = vals, *dst_k = keys_alt, *dst_v = vals_alt;
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_sort_hist<<<nb, SORT_BS, 0, s>>>(src_k, n, shift, hist, nb, n_dev, sg);
        cudaError_t e = launch_scan(hist, offs, (int64_t)L.hn, stot, stmp, s);
        if (e != cudaSuccess) return e;
        k_sort_scatter<<<nb, SORT_BS, 0, s>>>(src_k, src_v, dst_k, dst_v, n, shift, hist, offs, nb, n_dev, sg);
        count_launches(2);
        uint32_t *tk = src_k, *tv = src_v;
        src_k = dst_k; src_v = dst_v; dst_k = tk; dst_v = tv;
    }
    if (src_k != keys) {  // odd pass count: the result sits in the alternate buffers
        if (in_alt) {
            *in_alt = true;
        } else {
            cudaMemcpyAsync(keys, src_k, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(vals, src_v, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        }
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                        uint32_t n, int bits, uint32_t *tmp, cudaStream_t s, bool *in_alt,
                        const unsigned long long *n_dev)
{
    if (in_alt) *in_alt = false;
    if (n == 0) return cudaSuccess;
    return sort_passes(keys, vals, keys_alt, vals_alt, n, bits, tmp, sort_layout(n, 0), SortSegs(), s,
                       in_alt, n_dev);
}

cudaError_t launch_sort_views(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                              uint32_t n, int bits, const uint32_t *off, int64_t stride, int nv,
                              uint32_t *tmp, cudaStream_t s, bool *in_alt, const unsigned long long *n_dev)
{
    if (in_alt) *in_alt = false;
    if (n == 0 || nv <= 0) return cudaSuccess;
    const SortLayout L = sort_layout(n, nv);
    SortSegs sg;
    sg.tile_start = tmp + L.tiles;
    sg.seg_start = tmp + L.segs;
    sg.ns = nv;
    k_sort_segments<<<1, 1024, 0, s>>>(off, stride, nv, n, n_dev, tmp + L.tiles, tmp + L.segs);
    uint4 *span = reinterpret_cast<uint4 *>(tmp + L.span);
    k_sort_spans<<<(L.nb + 255) / 256, 256, 0, s>>>(L.nb, n, n_dev, sg, span);
    count_launches(2);
    sg.span = span;
    return sort_passes(keys, vals, keys_alt, vals_alt, n, bits, tmp, L, sg, s, in_alt, n_dev);
}

cudaError_t launch_ranges(const uint32_t *keys, uint32_t n_keys, uint2 *ranges, uint32_t n_tiles,
                          cudaStream_t s, const unsigned long long *n_dev, uint32_t tpv, int lbits)
{
    if (n_keys == 0) return cudaSuccess;
    const uint32_t threads = (n_keys + RANGE_ITEMS - 1) / RANGE_ITEMS;
    k_ranges<<<(threads + 255) / 256, 256, 0, s>>>(keys, n_keys, ranges, n_tiles, n_dev, tpv, lbits);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rgrt
