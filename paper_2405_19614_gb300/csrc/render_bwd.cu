// a7. Backward of the compositing (reverse mode of Sec. 3.4 C(p), D(p) and of
// the Sec. 3.3 border mask M_b(p) = 1 - T_final).
//
// The per-pixel blend state is recomputed, not stored: each pixel starts from
// its final transmittance and walks its tile's list backwards from the last
// blended entry, recovering T_i = T_{i+1} / (1 - alpha_i).  With
// s = sum over later entries k of (c_k.gC + z_k gD) alpha_k T_k:
//   dL/dc_i = gC alpha_i T_i,  dL/dz_i = gD alpha_i T_i,
//   dL/dalpha_i = T_i (c_i.gC + z_i gD) - s / (1 - alpha_i) + gA T_final / (1 - alpha_i),
// and through alpha_i = min(0.99, o_i g_i), g_i = exp(power_i), to the
// opacity, the 2D mean and the conic (no gradient where the clamp is active).
//
// Every thread of a block is at the same list entry at the same time, so the
// per-Gaussian gradients are summed across the warp with shuffles, then
// across the block's warps in shared memory, and only then added to HBM with
// 16-byte vector atomics: at most three per (Gaussian, tile).
#include "common.cuh"

namespace gs {

struct RenderBwdArgs {
    const float4 *rec;
    int64_t n;
    const uint32_t *vals;
    const uint32_t *ranges;
    const float *final_T;
    const uint32_t *n_contrib;
    const float *d_rgb, *d_depth, *d_alpha;
    float4 *grad2d;
    uint32_t *work_counter;
};

constexpr int kAcc = 10;

__global__ void __launch_bounds__(kTilePix) render_bwd_kernel(RenderBwdArgs a, ViewTable vt)
{
    __shared__ float4 s_pos[kTilePix];
    __shared__ float4 s_con[kTilePix];
    __shared__ float4 s_col[kTilePix];
    __shared__ int64_t s_rid[kTilePix];
    __shared__ float s_acc[kTilePix][kAcc + 1];
    __shared__ int s_item;
    __shared__ uint32_t s_maxlast;
    const int tid = threadIdx.x, lane = tid & 31;
    for (;;) {
        if (tid == 0) {
            s_item = (int)atomicAdd(a.work_counter, 1u);
            s_maxlast = 0;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= vt.n_tiles_total) break;
        const int v = view_of_tile(vt, item);
        const ViewInfo &V = vt.v[v];
        const int lt = item - V.tile_base;
        const int px = (lt % V.tiles_x) * kTile + (tid & (kTile - 1));
        const int py = (lt / V.tiles_x) * kTile + (tid / kTile);
        const bool inside = px < V.width && py < V.height;
        const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
        const uint32_t b = a.ranges[2 * item];
        const int64_t rbase = (int64_t)v * a.n;

        float T = 1.0f, Tf = 1.0f, gC0 = 0.0f, gC1 = 0.0f, gC2 = 0.0f, gD = 0.0f, gA = 0.0f;
        uint32_t last = 0;
        if (inside) {
            const int64_t pix = V.pix_base + (int64_t)py * V.width + px;
            Tf = T = a.final_T[pix];
            last = a.n_contrib[pix];
            if (a.d_rgb) {
                gC0 = a.d_rgb[3 * pix];
                gC1 = a.d_rgb[3 * pix + 1];
                gC2 = a.d_rgb[3 * pix + 2];
            }
            if (a.d_depth) gD = a.d_depth[pix];
            if (a.d_alpha) gA = a.d_alpha[pix];
        }
        if (last) atomicMax(&s_maxlast, last);
        __syncthreads();
        const uint32_t maxlast = s_maxlast;
        float S = 0.0f;  // suffix sum of (c.gC + z gD) alpha T over later entries

        for (uint32_t bend = maxlast; bend > 0;) {
            const uint32_t bstart = bend > (uint32_t)kTilePix ? bend - kTilePix : 0u;
            const int cnt = (int)(bend - bstart);
            if (tid < cnt) {
                const int64_t r = rbase + a.vals[b + bstart + tid];
                s_rid[tid] = r;
                s_pos[tid] = a.rec[3 * r];
                s_con[tid] = a.rec[3 * r + 1];
                s_col[tid] = a.rec[3 * r + 2];
                #pragma unroll
                for (int k = 0; k < kAcc; k++) s_acc[tid][k] = 0.0f;
            }
            __syncthreads();
            for (int j = cnt - 1; j >= 0; j--) {
                const uint32_t pos = bstart + (uint32_t)j;
                float gr[kAcc];
                #pragma unroll
                for (int k = 0; k < kAcc; k++) gr[k] = 0.0f;
                bool contrib = false;
                if (pos < last) {
                    const float4 p = s_pos[j];
                    const float4 c = s_con[j];
                    float dx, dy;
                    const float power = splat_power(p.x, p.y, c.x, c.y, c.z, sx, sy, &dx, &dy);
                    const float g = __expf(power);
                    const float araw = __fmul_rn(p.w, g);
                    const float alpha = fminf(kAlphaMax, araw);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        const float om = 1.0f - alpha;
                        const float inv_om = 1.0f / om;
                        const float Tb = T * inv_om;
                        const float w = alpha * Tb;
                        const float4 col = s_col[j];
                        gr[6] = gC0 * w;
                        gr[7] = gC1 * w;
                        gr[8] = gC2 * w;
                        gr[9] = gD * w;
                        const float wgt = col.x * gC0 + col.y * gC1 + col.z * gC2 + p.z * gD;
                        const float dalpha = Tb * wgt + (gA * Tf - S) * inv_om;
                        S += wgt * w;
                        T = Tb;
                        if (araw < kAlphaMax) {
                            gr[5] = dalpha * g;
                            const float dpow = dalpha * araw;
                            gr[0] = dpow * (-c.x * dx - c.y * dy);
                            gr[1] = dpow * (-c.z * dy - c.y * dx);
                            gr[2] = -0.5f * dx * dx * dpow;
                            gr[3] = -dx * dy * dpow;
                            gr[4] = -0.5f * dy * dy * dpow;
                        }
                    }
                }
                if (__any_sync(kFullMask, contrib)) {
                    #pragma unroll
                    for (int k = 0; k < kAcc; k++) gr[k] = warp_sum(gr[k]);
                    if (lane == 0) {
                        #pragma unroll
                        for (int k = 0; k < kAcc; k++) atomicAdd(&s_acc[j][k], gr[k]);
                    }
                }
            }
            __syncthreads();
            if (tid < cnt) {
                float r[kAcc];
                bool any = false;
                #pragma unroll
                for (int k = 0; k < kAcc; k++) {
                    r[k] = s_acc[tid][k];
                    any |= (r[k] != 0.0f);
                }
                if (any) {
                    float4 *dst = a.grad2d + 3 * s_rid[tid];
                    atomicAdd(dst, make_float4(r[0], r[1], r[2], r[3]));
                    atomicAdd(dst + 1, make_float4(r[4], r[5], r[6], r[7]));
                    atomicAdd(reinterpret_cast<float2 *>(dst + 2), make_float2(r[8], r[9]));
                }
            }
            __syncthreads();
            bend = bstart;
        }
        __syncthreads();  // every thread has read s_item and s_maxlast before they are reset
    }
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_grad2d_size(int64_t n, int32_t n_views)
{
    if (n < 0 || n_views < 0) return 0;
    return sizeof(float) * 12 * (size_t)n * (size_t)n_views;
}

extern "C" gs_status_t gs_render_bwd_splats(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins,
                                            const gs_view_t *views, int32_t n_views, const gs_image_t *img,
                                            const float *d_rgb, const float *d_depth, const float *d_alpha,
                                            float *grad2d, uint32_t *work_counter, void *stream)
{
    if (!proj || !bins || !img || !grad2d || !work_counter || n < 0) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (!img->final_T || !img->n_contrib || !bins->ranges || !bins->vals || (n > 0 && !proj->rec))
        return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(grad2d) & 15) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(work_counter, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    RenderBwdArgs a;
    a.rec = reinterpret_cast<const float4 *>(proj->rec);
    a.n = n;
    a.vals = bins->vals;
    a.ranges = bins->ranges;
    a.final_T = img->final_T;
    a.n_contrib = img->n_contrib;
    a.d_rgb = d_rgb;
    a.d_depth = d_depth;
    a.d_alpha = d_alpha;
    a.grad2d = reinterpret_cast<float4 *>(grad2d);
    a.work_counter = work_counter;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_bwd_kernel, kTilePix, 0);
    const int64_t slots = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(slots < vt.n_tiles_total ? slots : vt.n_tiles_total);
    render_bwd_kernel<<<grid > 0 ? grid : 1, kTilePix, 0, s>>>(a, vt);
    return launch_status();
}
