// a2 + a4. Binning of projected Gaussians into 16x16 tiles in front-to-back
// order (Sec. 3.4 "Differentiable Rasterization"): an exclusive scan of the
// number of tiles each (view, Gaussian) touches, emission of one
// (key = (global tile << 32) | bits(depth), value = Gaussian index) pair per
// touched tile, the onesweep radix sort (sort.cu), and each tile's [start, end).
#include "common.cuh"
#include "sort.cuh"

namespace gs {

constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;
constexpr int kEmitChunk = kEmitThreads * kEmitItems;

__device__ __forceinline__ uint64_t block_exclusive_scan_u64(uint64_t x, uint64_t *tmp /* [8] */, uint64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFullMask, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    uint64_t wbase = 0, all = 0;
    #pragma unroll
    for (int w = 0; w < kEmitThreads / 32; w++) {
        wbase += (w < warp) ? tmp[w] : 0ull;
        all += tmp[w];
    }
    __syncthreads();
    if (total) *total = all;
    return wbase + inc - x;
}

__global__ void __launch_bounds__(kEmitThreads) count_reduce_kernel(const uint32_t *__restrict__ tt, int64_t total,
                                                                    uint64_t *block_sums)
{
    __shared__ uint64_t tmp[kEmitThreads / 32];
    const int64_t first = (int64_t)blockIdx.x * kEmitChunk + threadIdx.x;
    uint64_t s = 0;
    #pragma unroll
    for (int k = 0; k < kEmitItems; k++) {
        const int64_t idx = first + k * kEmitThreads;
        if (idx < total) s += tt[idx];
    }
    uint64_t all;
    block_exclusive_scan_u64(s, tmp, &all);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = all;
}

// One block: exclusive scan of the block sums in place; the grand total is the
// pair count.
__global__ void __launch_bounds__(1024) scan_sums_kernel(uint64_t *sums, int64_t nb, int64_t cap,
                                                         uint32_t *n_pairs, uint32_t *status)
{
    __shared__ uint64_t tmp[32];
    __shared__ uint64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint64_t x = i < nb ? sums[i] : 0ull;
        uint64_t inc = x;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(kFullMask, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) tmp[warp] = inc;
        __syncthreads();
        uint64_t wbase = 0, all = 0;
        for (int w = 0; w < 32; w++) {
            wbase += (w < warp) ? tmp[w] : 0ull;
            all += tmp[w];
        }
        if (i < nb) sums[i] = carry + wbase + inc - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t total = carry;
        *n_pairs = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
        if (total > (uint64_t)cap) raise_status(status, GS_ERR_CAPACITY);
    }
}

// Load-balanced emission: the block first scans its chunk's pair counts into
// shared memory (with each record's depth bits, rectangle, view and index),
// then its threads walk the chunk's output positions in order, each finding
// its record by binary search, so consecutive threads write consecutive pairs.
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(const float *__restrict__ rec, const uint2 *__restrict__ rect,
                                                            const uint32_t *__restrict__ tt,
                                                            int64_t n, int64_t total, ViewTable vt,
                                                            const uint64_t *__restrict__ block_off, uint64_t *keys,
                                                            uint32_t *vals, int64_t cap, uint32_t *status)
{
    __shared__ uint64_t tmp[kEmitThreads / 32];
    __shared__ uint32_t s_excl[kEmitChunk + 1];
    __shared__ uint32_t s_z[kEmitChunk], s_r0[kEmitChunk], s_r1[kEmitChunk], s_g[kEmitChunk];
    __shared__ uint16_t s_v[kEmitChunk];
    const int64_t chunk = (int64_t)blockIdx.x * kEmitChunk;
    const int64_t first = chunk + (int64_t)threadIdx.x * kEmitItems;
    uint32_t c[kEmitItems];
    uint64_t sum = 0;
    #pragma unroll
    for (int k = 0; k < kEmitItems; k++) {
        const int64_t o = first + k;
        c[k] = o < total ? tt[o] : 0u;
        sum += c[k];
    }
    uint64_t block_total;
    uint64_t run = block_exclusive_scan_u64(sum, tmp, &block_total);
    #pragma unroll
    for (int k = 0; k < kEmitItems; k++) {
        const int r = threadIdx.x * kEmitItems + k;
        s_excl[r] = (uint32_t)run;
        run += c[k];
        if (c[k]) {
            const int64_t o = first + k;
            const int v = (int)(o / n);
            s_v[r] = (uint16_t)v;
            s_g[r] = (uint32_t)(o - (int64_t)v * n);
            s_z[r] = __float_as_uint(rec[12 * o + 2]);
            const uint2 rr = rect[o];
            s_r0[r] = rr.x;
            s_r1[r] = rr.y;
        }
    }
    if (threadIdx.x == 0) s_excl[kEmitChunk] = (uint32_t)block_total;
    __syncthreads();
    const uint64_t base = block_off[blockIdx.x];
    const uint32_t nq = (uint32_t)block_total;
    bool overflow = false;
    for (uint32_t q = threadIdx.x; q < nq; q += kEmitThreads) {
        // last record r with s_excl[r] <= q (records of zero count share their successor's offset)
        int lo = 0, hi = kEmitChunk;  // invariant: s_excl[lo] <= q < s_excl[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_excl[mid] <= q) lo = mid; else hi = mid;
        }
        const int r = lo;
        const uint32_t k = q - s_excl[r];
        const uint32_t r0 = s_r0[r], r1 = s_r1[r];
        const uint32_t x0 = r0 & 0xffff, y0 = r0 >> 16, x1 = r1 & 0xffff;
        const uint32_t w = x1 - x0 + 1;
        const uint32_t ty = y0 + k / w, tx = x0 + k % w;
        const ViewInfo &V = vt.v[s_v[r]];
        const uint64_t pos = base + q;
        if (pos < (uint64_t)cap) {
            keys[pos] = ((uint64_t)((uint32_t)V.tile_base + ty * (uint32_t)V.tiles_x + tx) << 32) | s_z[r];
            vals[pos] = s_g[r];
        } else {
            overflow = true;
        }
    }
    if (overflow) raise_status(status, GS_ERR_CAPACITY);
}

__global__ void ranges_kernel(const uint64_t *__restrict__ keys, const uint32_t *n_pairs_p, uint32_t cap,
                              uint32_t *ranges)
{
    const uint32_t n = min(*n_pairs_p, cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[2 * t] = i;
        if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[2 * t + 1] = i + 1;
    }
}

static int ceil_log2(int64_t x)
{
    int b = 0;
    while ((int64_t(1) << b) < x) b++;
    return b;
}

struct BinWorkspace {
    uint64_t *block_sums;
    uint64_t *alt_keys;
    uint32_t *alt_vals;
    void *sort_ws;
    size_t bytes;
};

static BinWorkspace carve(void *base, int64_t n_records, int64_t cap)
{
    BinWorkspace w;
    const int64_t nb = (n_records + kEmitChunk - 1) / kEmitChunk + 1;
    unsigned char *p = static_cast<unsigned char *>(base);
    size_t off = 0;
    w.block_sums = reinterpret_cast<uint64_t *>(p + off);
    off += align256(sizeof(uint64_t) * (size_t)nb);
    w.alt_keys = reinterpret_cast<uint64_t *>(p + off);
    off += align256(sizeof(uint64_t) * (size_t)cap);
    w.alt_vals = reinterpret_cast<uint32_t *>(p + off);
    off += align256(sizeof(uint32_t) * (size_t)cap);
    w.sort_ws = p + off;
    off += sort_workspace_bytes(cap);
    w.bytes = off;
    return w;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_bin_sort_workspace_size(int64_t n_records, int64_t pair_capacity, int64_t n_tiles_total)
{
    (void)n_tiles_total;
    if (n_records < 0 || pair_capacity < 1) return 0;
    return carve(nullptr, n_records, pair_capacity).bytes;
}

extern "C" gs_status_t gs_bin_sort(const gs_projected_t *proj, int64_t n, const gs_view_t *views, int32_t n_views,
                                   gs_bins_t *bins, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!proj || !bins || n < 0) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    const int64_t cap = bins->capacity;
    if (cap < 1 || cap >= (int64_t(1) << 30)) return GS_ERR_INVALID_ARG;
    if (!bins->keys || !bins->vals || !bins->ranges || !bins->n_pairs || !bins->status || !workspace)
        return GS_ERR_INVALID_ARG;
    const int64_t total = (int64_t)n_views * n;
    BinWorkspace w = carve(workspace, total, cap);
    if (workspace_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(bins->ranges, 0, sizeof(uint32_t) * 2 * (size_t)vt.n_tiles_total, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (total == 0) {
        if (cudaMemsetAsync(bins->n_pairs, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
        return GS_OK;
    }
    if (!proj->rec || !proj->rect || !proj->tiles_touched) return GS_ERR_INVALID_ARG;

    const int n_bits = 32 + ceil_log2(vt.n_tiles_total);
    const int P = sort_passes(n_bits);
    // emit where an odd or even number of passes leaves the result in bins
    uint64_t *ek = (P & 1) ? w.alt_keys : bins->keys;
    uint32_t *ev = (P & 1) ? w.alt_vals : bins->vals;
    uint64_t *ok = (P & 1) ? bins->keys : w.alt_keys;
    uint32_t *ov = (P & 1) ? bins->vals : w.alt_vals;

    const int64_t nb = (total + kEmitChunk - 1) / kEmitChunk;
    count_reduce_kernel<<<(unsigned)nb, kEmitThreads, 0, s>>>(proj->tiles_touched, total, w.block_sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(w.block_sums, nb, cap, bins->n_pairs, bins->status);
    emit_kernel<<<(unsigned)nb, kEmitThreads, 0, s>>>(proj->rec, reinterpret_cast<const uint2 *>(proj->rect),
                                                      proj->tiles_touched, n, total, vt, w.block_sums,
                                                      ek, ev, cap, bins->status);
    st = launch_status();
    if (st != GS_OK) return st;
    st = radix_sort_pairs(ek, ev, ok, ov, bins->n_pairs, cap, n_bits, w.sort_ws, bins->status, s);
    if (st != GS_OK) return st;
    ranges_kernel<<<num_sms() * 4, 256, 0, s>>>(bins->keys, bins->n_pairs, (uint32_t)cap, bins->ranges);
    return launch_status();
}
