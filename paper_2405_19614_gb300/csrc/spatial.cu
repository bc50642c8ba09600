// Spatial order of the map (a layout service for the Sec. 3.4 mapping; the
// paper has no counterpart).  A map grown by densification is stored in the
// order its Gaussians were created, keyframe by keyframe in pixel order, so
// Gaussians that are close in memory are close in space and are drawn in the
// same views.  Kernels that give a warp 32 consecutive Gaussians (projection
// and its backward) then do one view's work for all 32 lanes at once.  This
// entry point restores that order for any map: each Gaussian's rank in the
// Morton (Z-order) sequence of its quantised mean, ties in index order, to be
// applied with gs_compact_rows to every per-Gaussian array.
//
// Quantisation: the means' bounding box [lo, hi] per axis, then
// q = min(1023, (uint) ((m - lo) * (1024 / (hi - lo)))) in correctly rounded
// FP32 (0 on a flat axis), and the code interleaves the ten bits of x, y and z
// (x lowest).  The ranks come from four 8-bit onesweep passes over the 30-bit
// codes (stable, so equal codes keep index order).
#include "common.cuh"
#include "sort.cuh"

namespace gs {

constexpr int kSpThreads = 256;
constexpr int kSpPasses = 4;

// Float order as unsigned integers (monotone), for atomic min / max.
__device__ __forceinline__ uint32_t float_key(float x)
{
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// box[0..2] = min keys, box[3..5] = max keys (start at ~0 / 0).
__global__ void __launch_bounds__(kSpThreads) bbox_kernel(const float *__restrict__ means, int64_t n, uint32_t *box)
{
    uint32_t lo[3] = {~0u, ~0u, ~0u}, hi[3] = {0u, 0u, 0u};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        #pragma unroll
        for (int a = 0; a < 3; a++) {
            const uint32_t k = float_key(means[3 * i + a]);
            lo[a] = min(lo[a], k);
            hi[a] = max(hi[a], k);
        }
    }
    #pragma unroll
    for (int a = 0; a < 3; a++) {
        lo[a] = __reduce_min_sync(kFullMask, lo[a]);
        hi[a] = __reduce_max_sync(kFullMask, hi[a]);
    }
    if ((threadIdx.x & 31) == 0) {
        #pragma unroll
        for (int a = 0; a < 3; a++) {
            atomicMin(box + a, lo[a]);
            atomicMax(box + 3 + a, hi[a]);
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v)  // bit i -> bit 3i
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t quantise(float m, float lo, float hi)
{
    const float ext = __fsub_rn(hi, lo);
    if (!(ext > 0.0f)) return 0u;
    const float t = __fmul_rn(__fsub_rn(m, lo), __fdiv_rn(1024.0f, ext));
    return t >= 1023.0f ? 1023u : (uint32_t)t;
}

__global__ void __launch_bounds__(kSpThreads) morton_kernel(const float *__restrict__ means, int64_t n,
                                                            const uint32_t *__restrict__ box, uint32_t *keys,
                                                            uint32_t *idx, uint32_t *hist, uint32_t *n_dev)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_dev = (uint32_t)n;  // the key count of the sort passes
    __shared__ uint32_t h[kSpPasses][kRadix];
    for (int k = threadIdx.x; k < kSpPasses * kRadix; k += blockDim.x) (&h[0][0])[k] = 0;
    __syncthreads();
    float lo[3], hi[3];
    #pragma unroll
    for (int a = 0; a < 3; a++) {
        lo[a] = key_float(box[a]);
        hi[a] = key_float(box[3 + a]);
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    uint32_t code = 0;
    if (valid) {
        code = spread10(quantise(means[3 * i], lo[0], hi[0])) | (spread10(quantise(means[3 * i + 1], lo[1], hi[1])) << 1) |
               (spread10(quantise(means[3 * i + 2], lo[2], hi[2])) << 2);
        keys[i] = code;
        idx[i] = (uint32_t)i;
    }
    count_digits_warp(h, code, valid, kSpPasses);
    __syncthreads();
    for (int k = threadIdx.x; k < kSpPasses * kRadix; k += blockDim.x) {
        const uint32_t c = (&h[0][0])[k];
        if (c) atomicAdd(hist + k, c);
    }
}

__global__ void __launch_bounds__(kSpThreads) rank_kernel(const uint32_t *__restrict__ sorted_idx, int64_t n,
                                                          int32_t *new_index)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) new_index[sorted_idx[j]] = (int32_t)j;
}

struct SpWorkspace {
    uint32_t *small;  // box[6], n, counters[4], hist[4][256]
    uint32_t *keys[2], *idx[2];
    uint32_t *lb[2];
    size_t small_bytes, lb_bytes, bytes;
};

static SpWorkspace sp_carve(void *base, int64_t n)
{
    SpWorkspace w;
    unsigned char *p = static_cast<unsigned char *>(base);
    size_t off = 0;
    w.small = reinterpret_cast<uint32_t *>(p + off);
    w.small_bytes = sizeof(uint32_t) * (6 + 1 + kSpPasses + kSpPasses * kRadix);
    off += align256(w.small_bytes);
    for (int i = 0; i < 2; i++) {
        w.keys[i] = reinterpret_cast<uint32_t *>(p + off);
        off += align256(sizeof(uint32_t) * (size_t)n);
        w.idx[i] = reinterpret_cast<uint32_t *>(p + off);
        off += align256(sizeof(uint32_t) * (size_t)n);
    }
    w.lb_bytes = onesweep_lookback_bytes(n);
    for (int i = 0; i < 2; i++) {
        w.lb[i] = reinterpret_cast<uint32_t *>(p + off);
        off += w.lb_bytes;
    }
    w.bytes = off;
    return w;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_spatial_order_workspace_size(int64_t n)
{
    if (n < 1) return 0;
    return sp_carve(nullptr, n).bytes;
}

extern "C" gs_status_t gs_spatial_order(const float *means, int64_t n, int32_t *new_index, void *workspace,
                                        size_t workspace_bytes, uint32_t *status, void *stream)
{
    if (n < 0 || n >= (int64_t(1) << 31)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!means || !new_index || !workspace) return GS_ERR_INVALID_ARG;
    SpWorkspace w = sp_carve(workspace, n);
    if (workspace_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    uint32_t *box = w.small, *n_dev = w.small + 6, *counters = w.small + 7, *hist = w.small + 7 + kSpPasses;
    // box minima start at ~0, everything else at 0
    if (cudaMemsetAsync(w.small, 0, w.small_bytes, s) != cudaSuccess ||
        cudaMemsetAsync(box, 0xff, 3 * sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(w.lb[0], 0, w.lb_bytes, s) != cudaSuccess)
        return GS_ERR_CUDA;
    const unsigned blocks = (unsigned)((n + kSpThreads - 1) / kSpThreads);
    const unsigned bb = blocks < (unsigned)num_sms() * 8 ? blocks : (unsigned)num_sms() * 8;
    bbox_kernel<<<bb, kSpThreads, 0, s>>>(means, n, box);
    morton_kernel<<<blocks, kSpThreads, 0, s>>>(means, n, box, w.keys[0], w.idx[0], hist, n_dev);
    for (int p = 0; p < kSpPasses; p++) {
        const int a = p & 1;
        gs_status_t st = onesweep_pass(w.keys[a], w.idx[a], w.keys[a ^ 1], w.idx[a ^ 1], n_dev, n, hist + p * kRadix,
                                       w.lb[a], p + 1 < kSpPasses ? w.lb[a ^ 1] : nullptr, counters + p, 8 * p,
                                       kSortPlain, nullptr, status, s);
        if (st != GS_OK) return st;
    }
    rank_kernel<<<blocks, kSpThreads, 0, s>>>(w.idx[0], n, new_index);  // an even number of passes ends in 0
    return launch_status();
}
