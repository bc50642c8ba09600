// Map maintenance around the mapping iterations (Sec. 3.4 "Densification" and
// "Gaussian Pruning") and the keyframe choice of the Fusion Bridge (Sec. 3.3
// "View Point Selection").
//
// Densification: every pixel whose border mask M_b = alpha is below a
// threshold and whose sensor depth d is positive gets a new Gaussian at the
// back-projection of the pixel centre, isotropic with radius r = d / f (one
// pixel on the image plane, Eq. d: d = r f), the pixel's colour as its SH
// degree-0 band, identity rotation and a given opacity logit.
// Pruning: Gaussians whose opacity logit is below logit(tau) are removed;
// rows of every parameter (and optimiser-state) array are compacted, order
// kept.
// Both selections are compactions done with a per-block scan, so the order of
// new and surviving Gaussians is deterministic (pixel order; index order).
#include "common.cuh"

namespace gs {

constexpr int kSelThreads = 256, kSelItems = 8, kSelChunk = kSelThreads * kSelItems;
constexpr float kShC0 = 0.28209479177387814f;  // degree-0 basis value 1 / (2 sqrt(pi))

__device__ __forceinline__ uint32_t block_scan_u32(uint32_t x, uint32_t *tmp, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    uint32_t base = 0, all = 0;
    #pragma unroll
    for (int w = 0; w < kSelThreads / 32; w++) {
        base += (w < warp) ? tmp[w] : 0u;
        all += tmp[w];
    }
    __syncthreads();
    *total = all;
    return base + inc - x;
}

// Pass 1: number of selected items per chunk.  Selection is computed by SEL.
template <typename SEL>
__global__ void __launch_bounds__(kSelThreads) select_count_kernel(SEL sel, int64_t n, uint32_t *counts)
{
    __shared__ uint32_t tmp[kSelThreads / 32];
    const int64_t first = (int64_t)blockIdx.x * kSelChunk + (int64_t)threadIdx.x * kSelItems;
    uint32_t c = 0;
    #pragma unroll
    for (int k = 0; k < kSelItems; k++) c += (first + k < n && sel(first + k)) ? 1u : 0u;
    uint32_t total;
    block_scan_u32(c, tmp, &total);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// One block: exclusive scan of the chunk counts in place; the total is written
// to *total (and clamped to the capacity in *stored).
__global__ void __launch_bounds__(1024) select_scan_kernel(uint32_t *counts, int64_t nb, uint32_t *total,
                                                           uint32_t capacity_left, uint32_t *stored, uint32_t *status)
{
    __shared__ uint32_t tmp[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint32_t x = i < nb ? counts[i] : 0u;
        uint32_t inc = x;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) tmp[warp] = inc;
        __syncthreads();
        uint32_t wb = 0, all = 0;
        for (int w = 0; w < 32; w++) {
            wb += (w < warp) ? tmp[w] : 0u;
            all += tmp[w];
        }
        if (i < nb) counts[i] = carry + wb + inc - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *total = carry;
        if (stored) *stored = carry < capacity_left ? carry : capacity_left;
        if (carry > capacity_left) raise_status(status, GS_ERR_CAPACITY);
    }
}

struct DensifySel {
    const float *alpha, *depth;
    float threshold;
    __device__ bool operator()(int64_t p) const { return alpha[p] < threshold && depth[p] > 0.0f; }
};

struct DensifyArgs {
    const float *alpha, *depth, *rgb, *viewmats;
    float threshold, opacity_logit;
    float *means, *log_scales, *quats, *opac, *sh;
    int32_t sh_floats;  // 3 (deg + 1)^2
    int64_t n_old, capacity, P;
};

__global__ void __launch_bounds__(kSelThreads) densify_write_kernel(DensifyArgs a, ViewTable vt, const uint32_t *offsets)
{
    __shared__ uint32_t tmp[kSelThreads / 32];
    const int64_t first = (int64_t)blockIdx.x * kSelChunk + (int64_t)threadIdx.x * kSelItems;
    bool sel[kSelItems];
    uint32_t c = 0;
    #pragma unroll
    for (int k = 0; k < kSelItems; k++) {
        const int64_t p = first + k;
        sel[k] = p < a.P && a.alpha[p] < a.threshold && a.depth[p] > 0.0f;
        c += sel[k];
    }
    uint32_t total;
    uint32_t off = offsets[blockIdx.x] + block_scan_u32(c, tmp, &total);
    #pragma unroll 1
    for (int k = 0; k < kSelItems; k++) {
        if (!sel[k]) continue;
        const int64_t p = first + k;
        const int64_t g = a.n_old + off++;
        if (g >= a.capacity) continue;
        int v = 0;
        for (int w = 1; w < vt.n_views; w++)
            if (p >= vt.v[w].pix_base) v = w;
        const ViewInfo &V = vt.v[v];
        const int64_t lp = p - V.pix_base;
        const float px = (float)(lp % V.width) + 0.5f, py = (float)(lp / V.width) + 0.5f;
        const float d = a.depth[p];
        // camera-space point, then world = R^T (p_c - t)
        const float xc = (px - V.cx) / V.fx * d, yc = (py - V.cy) / V.fy * d, zc = d;
        const float *E = a.viewmats + 12 * v;
        const float qx = xc - E[3], qy = yc - E[7], qz = zc - E[11];
        a.means[3 * g + 0] = E[0] * qx + E[4] * qy + E[8] * qz;
        a.means[3 * g + 1] = E[1] * qx + E[5] * qy + E[9] * qz;
        a.means[3 * g + 2] = E[2] * qx + E[6] * qy + E[10] * qz;
        const float ls = logf(d / V.fx);  // one pixel on the image plane: r = d / f
        a.log_scales[3 * g + 0] = ls;
        a.log_scales[3 * g + 1] = ls;
        a.log_scales[3 * g + 2] = ls;
        a.quats[4 * g + 0] = 1.0f;
        a.quats[4 * g + 1] = 0.0f;
        a.quats[4 * g + 2] = 0.0f;
        a.quats[4 * g + 3] = 0.0f;
        a.opac[g] = a.opacity_logit;
        float *shg = a.sh + (int64_t)a.sh_floats * g;
        for (int k = 0; k < a.sh_floats; k++) shg[k] = 0.0f;
        for (int ch = 0; ch < 3; ch++) shg[ch] = (a.rgb[3 * p + ch] - 0.5f) / kShC0;
    }
}

struct PruneSel {
    const float *opacity_logit;
    float min_logit;
    __device__ bool operator()(int64_t i) const { return opacity_logit[i] >= min_logit; }
};

__global__ void __launch_bounds__(kSelThreads) prune_index_kernel(const float *opacity_logit, int64_t n, float min_logit,
                                                                   const uint32_t *offsets, int32_t *new_index)
{
    __shared__ uint32_t tmp[kSelThreads / 32];
    const int64_t first = (int64_t)blockIdx.x * kSelChunk + (int64_t)threadIdx.x * kSelItems;
    bool keep[kSelItems];
    uint32_t c = 0;
    #pragma unroll
    for (int k = 0; k < kSelItems; k++) {
        keep[k] = first + k < n && opacity_logit[first + k] >= min_logit;
        c += keep[k];
    }
    uint32_t total;
    uint32_t off = offsets[blockIdx.x] + block_scan_u32(c, tmp, &total);
    #pragma unroll
    for (int k = 0; k < kSelItems; k++)
        if (first + k < n) new_index[first + k] = keep[k] ? (int32_t)(off++) : -1;
}

struct RowArrays {
    int32_t count;
    const float *src[GS_MAX_COMPACT_ARRAYS];
    float *dst[GS_MAX_COMPACT_ARRAYS];
    int32_t width[GS_MAX_COMPACT_ARRAYS];
};

// One thread per (row, array); copies kept rows to their new index.
__global__ void compact_rows_kernel(const int32_t *__restrict__ new_index, int64_t n, RowArrays A)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (i >= n || a >= A.count) return;
    const int32_t j = new_index[i];
    if (j < 0) return;
    const int w = A.width[a];
    const float *s = A.src[a] + (int64_t)w * i;
    float *d = A.dst[a] + (int64_t)w * j;
    for (int k = 0; k < w; k++) d[k] = s[k];
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_select_workspace_size(int64_t n_items)
{
    return n_items < 0 ? 0 : sizeof(uint32_t) * (size_t)((n_items + kSelChunk - 1) / kSelChunk + 1);
}

extern "C" gs_status_t gs_densify(const float *alpha, const float *target_rgb, const float *target_depth,
                                  const gs_view_t *views, const float *viewmats, int32_t n_views, float threshold,
                                  float opacity_logit, gs_param_grads_t *params, int32_t sh_degree, int64_t n_old,
                                  int64_t capacity, uint32_t *n_added, uint32_t *status, void *workspace,
                                  size_t workspace_bytes, void *stream)
{
    if (!alpha || !target_rgb || !target_depth || !viewmats || !params || !n_added || !workspace || n_old < 0 ||
        capacity < n_old || sh_degree < 0 || sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    if (!params->means || !params->log_scales || !params->quats || !params->opacity_logit || !params->sh)
        return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    const int64_t P = vt.n_pix_total;
    if (workspace_bytes < gs_select_workspace_size(P)) return GS_ERR_INVALID_ARG;
    const int64_t left = capacity - n_old;
    if (left > 0xffffffffLL) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    uint32_t *counts = static_cast<uint32_t *>(workspace);
    const int64_t nb = (P + kSelChunk - 1) / kSelChunk;
    DensifySel sel{alpha, target_depth, threshold};
    select_count_kernel<<<(unsigned)nb, kSelThreads, 0, s>>>(sel, P, counts);
    uint32_t *total = counts + nb;
    select_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, total, (uint32_t)left, n_added, status);
    DensifyArgs a;
    a.alpha = alpha;
    a.depth = target_depth;
    a.rgb = target_rgb;
    a.viewmats = viewmats;
    a.threshold = threshold;
    a.opacity_logit = opacity_logit;
    a.means = params->means;
    a.log_scales = params->log_scales;
    a.quats = params->quats;
    a.opac = params->opacity_logit;
    a.sh = params->sh;
    a.sh_floats = 3 * (sh_degree + 1) * (sh_degree + 1);
    a.n_old = n_old;
    a.capacity = capacity;
    a.P = P;
    densify_write_kernel<<<(unsigned)nb, kSelThreads, 0, s>>>(a, vt, counts);
    return launch_status();
}

extern "C" gs_status_t gs_prune_select(const float *opacity_logit, int64_t n, float tau, int32_t *new_index,
                                       uint32_t *n_kept, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!opacity_logit || !new_index || !n_kept || !workspace || n < 0 || n > 0x7fffffffLL) return GS_ERR_INVALID_ARG;
    if (!(tau > 0.0f && tau < 1.0f)) return GS_ERR_INVALID_ARG;
    if (workspace_bytes < gs_select_workspace_size(n)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (n == 0) return cudaMemsetAsync(n_kept, 0, sizeof(uint32_t), s) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
    // opacity = sigmoid(logit) >= tau  <=>  logit >= log(tau / (1 - tau)); the cut is taken on the logit,
    // rounded once to FP32, so every implementation makes the same decision
    const float min_logit = (float)log((double)tau / (1.0 - (double)tau));
    uint32_t *counts = static_cast<uint32_t *>(workspace);
    const int64_t nb = (n + kSelChunk - 1) / kSelChunk;
    PruneSel sel{opacity_logit, min_logit};
    select_count_kernel<<<(unsigned)nb, kSelThreads, 0, s>>>(sel, n, counts);
    select_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, n_kept, 0xffffffffu, nullptr, nullptr);
    prune_index_kernel<<<(unsigned)nb, kSelThreads, 0, s>>>(opacity_logit, n, min_logit, counts, new_index);
    return launch_status();
}

extern "C" gs_status_t gs_compact_rows(const int32_t *new_index, int64_t n, const gs_rows_t *arrays,
                                       int32_t n_arrays, void *stream)
{
    if (!new_index || !arrays || n < 0 || n_arrays < 1 || n_arrays > GS_MAX_COMPACT_ARRAYS) return GS_ERR_INVALID_ARG;
    RowArrays A;
    A.count = n_arrays;
    for (int k = 0; k < GS_MAX_COMPACT_ARRAYS; k++) {
        A.src[k] = k < n_arrays ? arrays[k].src : nullptr;
        A.dst[k] = k < n_arrays ? arrays[k].dst : nullptr;
        A.width[k] = k < n_arrays ? arrays[k].row_floats : 0;
        if (k < n_arrays && (!A.src[k] || !A.dst[k] || A.width[k] < 1 || A.src[k] == A.dst[k]))
            return GS_ERR_INVALID_ARG;
    }
    if (n == 0) return GS_OK;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)n_arrays);
    compact_rows_kernel<<<grid, 256, 0, as_stream(stream)>>>(new_index, n, A);
    return launch_status();
}

// View point selection (Sec. 3.3): keyframe i is selected when
// beta <= M_{i-1,i} < alpha * T_{i-1,i}; the first keyframe is always selected.
extern "C" gs_status_t gs_select_views(const int32_t *matches, const int32_t *totals, int32_t n, float alpha,
                                       int32_t beta, int32_t *selected)
{
    if (n < 0 || (n > 0 && (!matches || !totals || !selected))) return GS_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; i++) {
        if (i == 0) {
            selected[i] = 1;
            continue;
        }
        selected[i] = (matches[i] >= beta && (double)matches[i] < (double)alpha * (double)totals[i]) ? 1 : 0;
    }
    return GS_OK;
}
