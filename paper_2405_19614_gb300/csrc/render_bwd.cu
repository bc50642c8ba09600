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
// Each warp owns a 16 x 2*PPT band of the tile and walks only the staged
// entries that can reach alpha = 1/255 in that band (the same conservative
// test as the forward, 32 entries at a time).  All threads of a warp are at
// the same list entry at the same time: a thread first sums the gradients of
// its PPT pixels in registers, the warp reduces the ten sums with a
// reduce-scatter butterfly (12 shuffles, one total per lane), the block adds
// its warps' totals in shared memory, and only then are they added to HBM with
// vector atomics: at most three per (Gaussian, tile).  PPT and BATCH are
// picked by the autotuner.
#include "common.cuh"
#include "render.cuh"

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

// Blocks per SM asked of the register allocator: 64 registers a thread for
// one and two pixels a thread, 80 for four, 128 for eight (no spills inside
// the entry loop at these budgets).
template <int PPT>
struct BwdOccupancy {
    static constexpr int value = PPT == 1 ? 4 : PPT == 2 ? 8 : PPT == 4 ? 12 : 16;
};

template <int PPT, int BATCH>
__global__ void __launch_bounds__(kTilePix / PPT, BwdOccupancy<PPT>::value)
    render_bwd_kernel(RenderBwdArgs a, ViewTable vt)
{
    constexpr int THREADS = kTilePix / PPT;
    constexpr int WARPS = THREADS / 32;
    constexpr int BAND = 2 * PPT;  // rows per warp
    constexpr int WORDS = BATCH / 32;
    __shared__ float4 s_pos[BATCH];
    __shared__ float4 s_con[BATCH];
    __shared__ float4 s_col[BATCH];
    __shared__ int64_t s_rid[BATCH];
    // per-warp gradient totals of the staged entries; s_hit marks the entries
    // a warp has written, so nothing needs clearing between batches
    __shared__ float s_acc[WARPS][BATCH][kAcc + 1];
    __shared__ uint32_t s_hit[WARPS][WORDS];
    __shared__ int s_item;
    __shared__ uint32_t s_maxlast;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ly0 = warp * BAND + (lane >> 4);  // this thread's rows: ly0 + 2k
    int slot;
    bool slot_valid;
    reduce10_slot(lane, &slot, &slot_valid);
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
        const int tx0 = (lt % V.tiles_x) * kTile, ty0 = (lt / V.tiles_x) * kTile;
        const int px = tx0 + (lane & (kTile - 1));
        const int py0 = ty0 + ly0;
        const float sx = (float)px + 0.5f;
        const float bx0 = (float)tx0 + 0.5f, bx1 = (float)tx0 + (kTile - 0.5f);
        const float by0 = (float)(ty0 + warp * BAND) + 0.5f, by1 = by0 + (float)(BAND - 1);
        const uint32_t b = a.ranges[2 * item];
        const int64_t rbase = (int64_t)v * a.n;

        // per pixel: T running transmittance, gC/gD upstream gradients,
        // R = gA T_final - (sum over later blended entries of (c.gC + z gD) alpha T)
        float T[PPT], gC0[PPT], gC1[PPT], gC2[PPT], gD[PPT], R[PPT];
        uint32_t last[PPT];
        uint32_t my_last = 0;
        #pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = py0 + 2 * k;
            T[k] = 1.0f;
            gC0[k] = gC1[k] = gC2[k] = gD[k] = R[k] = 0.0f;
            last[k] = 0;
            if (px < V.width && py < V.height) {
                const int64_t pix = V.pix_base + (int64_t)py * V.width + px;
                T[k] = a.final_T[pix];
                last[k] = a.n_contrib[pix];
                if (a.d_rgb) {
                    gC0[k] = a.d_rgb[3 * pix];
                    gC1[k] = a.d_rgb[3 * pix + 1];
                    gC2[k] = a.d_rgb[3 * pix + 2];
                }
                if (a.d_depth) gD[k] = a.d_depth[pix];
                if (a.d_alpha) R[k] = a.d_alpha[pix] * T[k];
            }
            my_last = max(my_last, last[k]);
        }
        if (my_last) atomicMax(&s_maxlast, my_last);
        const uint32_t warp_last = __reduce_max_sync(kFullMask, my_last);
        __syncthreads();
        const uint32_t maxlast = s_maxlast;

        for (uint32_t bend = maxlast; bend > 0;) {
            const uint32_t bstart = bend > (uint32_t)BATCH ? bend - BATCH : 0u;
            const int cnt = (int)(bend - bstart);
            for (int r = tid; r < cnt; r += THREADS) {
                const int64_t g = rbase + a.vals[b + bstart + r];
                s_rid[r] = g;
                s_pos[r] = a.rec[3 * g];
                s_con[r] = a.rec[3 * g + 1];
                s_col[r] = a.rec[3 * g + 2];
            }
            __syncthreads();
            for (int m = ((cnt - 1) >> 5) << 5; m >= 0; m -= 32) {
              const int jl = m + lane;
              uint32_t todo = __ballot_sync(kFullMask, jl < cnt && (uint32_t)(bstart + jl) < warp_last &&
                                                           !splat_misses_box(s_pos[jl], s_con[jl], bx0, bx1, by0, by1));
              uint32_t hit = 0;
              while (todo) {
                const int bit = 31 - __clz(todo);
                todo &= ~(1u << bit);
                const int j = m + bit;
                const uint32_t pos = bstart + (uint32_t)j;
                float gr[kAcc];
                #pragma unroll
                for (int k = 0; k < kAcc; k++) gr[k] = 0.0f;
                bool contrib = false;
                if (pos < my_last) {
                    const float4 p = s_pos[j];
                    const float4 c = s_con[j];
                    const float4 col = s_col[j];
                    // exponents (and offsets) of this thread's pixels, two per packed evaluation
                    float pw[PPT], dyk[PPT], dx;
                    if (PPT == 1) {
                        pw[0] = splat_power(p.x, p.y, c.w, col.w, c.x, c.y, c.z, sx, (float)py0 + 0.5f, &dx, &dyk[0]);
                    } else {
                        #pragma unroll
                        for (int k = 0; k < PPT; k += 2) {
                            float2 dy2;
                            const float2 p2 = splat_power2(p.x, p.y, c.w, col.w, c.x, c.y, c.z, sx,
                                                           f2((float)(py0 + 2 * k) + 0.5f, (float)(py0 + 2 * k + 2) + 0.5f),
                                                           &dx, &dy2);
                            pw[k] = p2.x;
                            pw[(k + 1) % PPT] = p2.y;
                            dyk[k] = dy2.x;
                            dyk[(k + 1) % PPT] = dy2.y;
                        }
                    }
                    #pragma unroll
                    for (int k = 0; k < PPT; k++) {
                        if (pos >= last[k]) continue;
                        const float dy = dyk[k];
                        const float g = __expf(pw[k]);
                        const float araw = __fmul_rn(p.w, g);
                        const float alpha = fminf(kAlphaMax, araw);
                        if (alpha < kAlphaMin) continue;
                        contrib = true;
                        // 1 - alpha >= 0.01: the fast reciprocal is within 2 ulp
                        const float inv_om = __fdividef(1.0f, 1.0f - alpha);
                        const float Tb = T[k] * inv_om;
                        const float w = alpha * Tb;
                        gr[6] += gC0[k] * w;
                        gr[7] += gC1[k] * w;
                        gr[8] += gC2[k] * w;
                        gr[9] += gD[k] * w;
                        const float wgt = col.x * gC0[k] + col.y * gC1[k] + col.z * gC2[k] + p.z * gD[k];
                        const float dalpha = Tb * wgt + R[k] * inv_om;
                        R[k] -= wgt * w;
                        T[k] = Tb;
                        if (araw < kAlphaMax) {
                            gr[5] += dalpha * g;
                            const float dpow = dalpha * araw;
                            gr[0] += dpow * (-c.x * dx - c.y * dy);
                            gr[1] += dpow * (-c.z * dy - c.y * dx);
                            gr[2] += -0.5f * dx * dx * dpow;
                            gr[3] += -dx * dy * dpow;
                            gr[4] += -0.5f * dy * dy * dpow;
                        }
                    }
                }
                if (__any_sync(kFullMask, contrib)) {
                    const float r = warp_reduce_scatter10(gr, lane);
                    if (slot_valid) s_acc[warp][j][slot] = r;
                    hit |= 1u << bit;
                }
              }
              if (lane == 0) s_hit[warp][m >> 5] = hit;
            }
            __syncthreads();
            for (int r = tid; r < cnt; r += THREADS) {
                float q[kAcc];
                #pragma unroll
                for (int k = 0; k < kAcc; k++) q[k] = 0.0f;
                bool any = false;
                #pragma unroll
                for (int w = 0; w < WARPS; w++) {
                    if (!((s_hit[w][r >> 5] >> (r & 31)) & 1u)) continue;
                    any = true;
                    #pragma unroll
                    for (int k = 0; k < kAcc; k++) q[k] += s_acc[w][r][k];
                }
                if (any) {
                    float4 *dst = a.grad2d + 3 * s_rid[r];
                    atomicAdd(dst, make_float4(q[0], q[1], q[2], q[3]));
                    atomicAdd(dst + 1, make_float4(q[4], q[5], q[6], q[7]));
                    atomicAdd(reinterpret_cast<float2 *>(dst + 2), make_float2(q[8], q[9]));
                }
            }
            __syncthreads();
            bend = bstart;
        }
        __syncthreads();  // every thread has read s_item and s_maxlast before they are reset
    }
}

template <int PPT, int BATCH>
static gs_status_t launch_bwd(const RenderBwdArgs &a, const ViewTable &vt, cudaStream_t s)
{
    auto kern = render_bwd_kernel<PPT, BATCH>;
    constexpr int threads = kTilePix / PPT;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    const int64_t slots = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(slots < vt.n_tiles_total ? slots : vt.n_tiles_total);
    kern<<<grid > 0 ? grid : 1, threads, 0, s>>>(a, vt);
    return launch_status();
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
    switch (render_variant_bwd()) {
    case 0: return launch_bwd<1, 64>(a, vt, s);
    case 1: return launch_bwd<2, 128>(a, vt, s);
    case 2: return launch_bwd<4, 64>(a, vt, s);
    case 3: return launch_bwd<4, 128>(a, vt, s);
    default: return launch_bwd<8, 64>(a, vt, s);
    }
}
