// a5. Forward compositing (Sec. 3.4: C(p) = sum_i c_i f_i prod_{j<i} (1 - f_j)
// and D(p) likewise with the depths d_i; Sec. 3.3: border mask M_b(p) =
// sum_i f_i prod_{j<i} (1 - f_j) = 1 - T_final).
//
// One persistent launch covers every (view, tile) work item of every view:
// 256-thread blocks pull items from an atomic counter, so views of different
// sizes share one launch and long tiles do not hold up a static schedule.
// Each block stages its tile's sorted splat records in batches of 256 in
// shared memory and each thread composites one pixel front to back, leaving
// the batch loop once all 256 pixels have run out of transmittance.
#include "common.cuh"

namespace gs {

struct RenderFwdArgs {
    const float4 *rec;
    int64_t n;
    const uint32_t *vals;
    const uint32_t *ranges;
    float *rgb, *depth, *alpha, *final_T;
    uint32_t *n_contrib;
    uint32_t *n_eval, *n_blend;  // STATS variant only
    uint32_t *work_counter;
};

// STATS = true counts, per pixel, the list entries evaluated and blended (the
// algorithmic work of the compositing) instead of writing the image.
template <bool STATS>
__global__ void __launch_bounds__(kTilePix) render_fwd_kernel(RenderFwdArgs a, ViewTable vt)
{
    __shared__ float4 s_pos[kTilePix];  // (u, v, z, opacity)
    __shared__ float4 s_con[kTilePix];  // (conicA, conicB, conicC, -)
    __shared__ float4 s_col[kTilePix];  // (r, g, b, -)
    __shared__ int s_item;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= vt.n_tiles_total) break;
        const int v = view_of_tile(vt, item);
        const ViewInfo &V = vt.v[v];
        const int lt = item - V.tile_base;
        const int px = (lt % V.tiles_x) * kTile + (tid & (kTile - 1));
        const int py = (lt / V.tiles_x) * kTile + (tid / kTile);
        const bool inside = px < V.width && py < V.height;
        const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
        const uint32_t b = a.ranges[2 * item], e = a.ranges[2 * item + 1];
        const int64_t rbase = (int64_t)v * a.n;

        float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, D = 0.0f;
        uint32_t last = 0, n_eval = 0, n_blend = 0;
        bool done = !inside;
        for (uint32_t start = b; start < e; start += kTilePix) {
            if (__syncthreads_count(done) == kTilePix) break;
            const uint32_t idx = start + tid;
            if (idx < e) {
                const int64_t r = rbase + a.vals[idx];
                s_pos[tid] = a.rec[3 * r];
                s_con[tid] = a.rec[3 * r + 1];
                s_col[tid] = a.rec[3 * r + 2];
            }
            __syncthreads();
            const int cnt = (int)min((uint32_t)kTilePix, e - start);
            if (!done) {
                for (int j = 0; j < cnt; j++) {
                    const float4 p = s_pos[j];
                    const float4 c = s_con[j];
                    float dx, dy;
                    const float power = splat_power(p.x, p.y, c.x, c.y, c.z, sx, sy, &dx, &dy);
                    const float alpha = fminf(kAlphaMax, __fmul_rn(p.w, __expf(power)));
                    if (STATS) n_eval++;
                    if (alpha < kAlphaMin) continue;
                    const float tT = T * (1.0f - alpha);
                    if (tT < kTMin) {
                        done = true;
                        break;
                    }
                    if (STATS) n_blend++;
                    const float w = alpha * T;
                    const float4 col = s_col[j];
                    C0 += col.x * w;
                    C1 += col.y * w;
                    C2 += col.z * w;
                    D += p.z * w;
                    T = tT;
                    last = start - b + (uint32_t)j + 1u;
                }
            }
            __syncthreads();
        }
        if (STATS && inside) {
            const int64_t pix = V.pix_base + (int64_t)py * V.width + px;
            a.n_eval[pix] = n_eval;
            a.n_blend[pix] = n_blend;
        } else if (inside) {
            const int64_t pix = V.pix_base + (int64_t)py * V.width + px;
            a.rgb[3 * pix + 0] = C0;
            a.rgb[3 * pix + 1] = C1;
            a.rgb[3 * pix + 2] = C2;
            a.depth[pix] = D;
            a.alpha[pix] = 1.0f - T;
            a.final_T[pix] = T;
            a.n_contrib[pix] = last;
        }
    }
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_render_fwd(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins,
                                     const gs_view_t *views, int32_t n_views, gs_image_t *img,
                                     uint32_t *work_counter, void *stream)
{
    if (!proj || !bins || !img || !work_counter || n < 0) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (!img->rgb || !img->depth || !img->alpha || !img->final_T || !img->n_contrib || !bins->ranges ||
        !bins->vals || (n > 0 && !proj->rec))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(work_counter, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    RenderFwdArgs a;
    a.rec = reinterpret_cast<const float4 *>(proj->rec);
    a.n = n;
    a.vals = bins->vals;
    a.ranges = bins->ranges;
    a.rgb = img->rgb;
    a.depth = img->depth;
    a.alpha = img->alpha;
    a.final_T = img->final_T;
    a.n_contrib = img->n_contrib;
    a.n_eval = a.n_blend = nullptr;
    a.work_counter = work_counter;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_fwd_kernel<false>, kTilePix, 0);
    const int64_t slots = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(slots < vt.n_tiles_total ? slots : vt.n_tiles_total);
    render_fwd_kernel<false><<<grid > 0 ? grid : 1, kTilePix, 0, s>>>(a, vt);
    return launch_status();
}

extern "C" gs_status_t gs_render_stats(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins,
                                       const gs_view_t *views, int32_t n_views, uint32_t *n_eval, uint32_t *n_blend,
                                       uint32_t *work_counter, void *stream)
{
    if (!proj || !bins || !n_eval || !n_blend || !work_counter || n < 0) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (!bins->ranges || !bins->vals || (n > 0 && !proj->rec)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(work_counter, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    RenderFwdArgs a = {};
    a.rec = reinterpret_cast<const float4 *>(proj->rec);
    a.n = n;
    a.vals = bins->vals;
    a.ranges = bins->ranges;
    a.n_eval = n_eval;
    a.n_blend = n_blend;
    a.work_counter = work_counter;
    const int grid = (int)(num_sms() * 4 < vt.n_tiles_total ? num_sms() * 4 : vt.n_tiles_total);
    render_fwd_kernel<true><<<grid > 0 ? grid : 1, kTilePix, 0, s>>>(a, vt);
    return launch_status();
}
