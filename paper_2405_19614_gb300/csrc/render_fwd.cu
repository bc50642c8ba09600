// a5. Forward compositing (Sec. 3.4: C(p) = sum_i c_i f_i prod_{j<i} (1 - f_j)
// and D(p) likewise with the depths d_i; Sec. 3.3: border mask M_b(p) =
// sum_i f_i prod_{j<i} (1 - f_j) = 1 - T_final).
//
// One persistent launch covers every (view, tile) work item of every view:
// blocks pull items from an atomic counter, so views of different sizes share
// one launch and long tiles do not hold up a static schedule.  A block of
// 256 / PPT threads owns one 16x16 tile at a time; each warp owns a 16 x 2*PPT
// band of it and each thread PPT pixels of that band (rows r, r + 2, ...), so
// every splat record staged in shared memory serves PPT pixels per load.
// Records are staged in batches of BATCH; each warp first drops, 32 at a time
// and in parallel, the records that provably cannot reach alpha = 1/255 in its
// band (splat_misses_box), then walks the rest.  The block leaves the batch
// loop once all its pixels have run out of transmittance.  PPT and BATCH are
// chosen per workload by the autotuner.
#include "common.cuh"
#include "render.cuh"

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
template <int PPT, int BATCH, bool STATS>
__global__ void __launch_bounds__(kTilePix / PPT) render_fwd_kernel(RenderFwdArgs a, ViewTable vt)
{
    constexpr int THREADS = kTilePix / PPT;
    constexpr int BAND = 2 * PPT;      // rows per warp
    __shared__ float4 s_pos[BATCH];    // (u, v, z, opacity)
    __shared__ float4 s_con[BATCH];    // (conicA, conicB, conicC, -)
    __shared__ float4 s_col[BATCH];    // (r, g, b, -)
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ly0 = warp * BAND + (lane >> 4);  // this thread's rows: ly0 + 2k
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= vt.n_tiles_total) break;
        const int v = view_of_tile(vt, item);
        const ViewInfo &V = vt.v[v];
        const int lt = item - V.tile_base;
        const int tx0 = (lt % V.tiles_x) * kTile, ty0 = (lt / V.tiles_x) * kTile;
        const int px = tx0 + (lane & (kTile - 1));
        const int py0 = ty0 + ly0;
        const float sx = (float)px + 0.5f;
        // the warp's band of pixel centres, for culling
        const float bx0 = (float)tx0 + 0.5f, bx1 = (float)tx0 + (kTile - 0.5f);
        const float by0 = (float)(ty0 + warp * BAND) + 0.5f, by1 = by0 + (float)(BAND - 1);
        const uint32_t b = a.ranges[2 * item], e = a.ranges[2 * item + 1];
        const int64_t rbase = (int64_t)v * a.n;

        float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT];
        uint32_t last[PPT], n_eval[PPT], n_blend[PPT];
        bool live[PPT];
        int alive = 0;
        #pragma unroll
        for (int k = 0; k < PPT; k++) {
            T[k] = 1.0f;
            C0[k] = C1[k] = C2[k] = D[k] = 0.0f;
            last[k] = n_eval[k] = n_blend[k] = 0;
            live[k] = px < V.width && (py0 + 2 * k) < V.height;
            alive += live[k];
        }
        for (uint32_t start = b; start < e; start += BATCH) {
            if (__syncthreads_count(alive > 0) == 0) break;
            #pragma unroll
            for (int r = tid; r < BATCH; r += THREADS) {
                const uint32_t idx = start + r;
                if (idx < e) {
                    const int64_t g = rbase + a.vals[idx];
                    s_pos[r] = a.rec[3 * g];
                    s_con[r] = a.rec[3 * g + 1];
                    s_col[r] = a.rec[3 * g + 2];
                }
            }
            __syncthreads();
            const int cnt = (int)min((uint32_t)BATCH, e - start);
            for (int m = 0; m < cnt && __any_sync(kFullMask, alive > 0); m += 32) {
                // entries of this chunk that may reach alpha = 1/255 in the warp's band
                const int jl = m + lane;
                uint32_t todo = __ballot_sync(
                    kFullMask, jl < cnt && (STATS || !splat_misses_box(s_pos[jl], s_con[jl], bx0, bx1, by0, by1)));
                if (alive == 0) todo = 0;
                while (todo) {
                    const int j = m + __ffs(todo) - 1;
                    todo &= todo - 1;
                    const float4 p = s_pos[j];
                    const float4 c = s_con[j];
                    const float4 col = s_col[j];
                    // alphas of this thread's pixels, two per packed evaluation
                    float al[PPT];
                    if (PPT == 1) {
                        al[0] = splat_alpha(p, c, col, sx, (float)py0 + 0.5f);
                    } else {
                        #pragma unroll
                        for (int k = 0; k < PPT; k += 2) {
                            const float2 a2 = splat_alpha2(p, c, col, sx,
                                                           f2((float)(py0 + 2 * k) + 0.5f, (float)(py0 + 2 * k + 2) + 0.5f));
                            al[k] = a2.x;
                            al[(k + 1) % PPT] = a2.y;
                        }
                    }
                    #pragma unroll
                    for (int k = 0; k < PPT; k++) {
                        if (!live[k]) continue;
                        const float alpha = al[k];
                        if (STATS) n_eval[k]++;
                        if (alpha < kAlphaMin) continue;
                        const float tT = T[k] * (1.0f - alpha);
                        if (tT < kTMin) {
                            live[k] = false;
                            alive--;
                            continue;
                        }
                        if (STATS) n_blend[k]++;
                        const float w = alpha * T[k];
                        C0[k] += col.x * w;
                        C1[k] += col.y * w;
                        C2[k] += col.z * w;
                        D[k] += p.z * w;
                        T[k] = tT;
                        last[k] = start - b + (uint32_t)j + 1u;
                    }
                    if (alive == 0) break;
                }
            }
            __syncthreads();
        }
        #pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = py0 + 2 * k;
            if (px >= V.width || py >= V.height) continue;
            const int64_t pix = V.pix_base + (int64_t)py * V.width + px;
            if (STATS) {
                a.n_eval[pix] = n_eval[k];
                a.n_blend[pix] = n_blend[k];
            } else {
                a.rgb[3 * pix + 0] = C0[k];
                a.rgb[3 * pix + 1] = C1[k];
                a.rgb[3 * pix + 2] = C2[k];
                a.depth[pix] = D[k];
                a.alpha[pix] = 1.0f - T[k];
                a.final_T[pix] = T[k];
                a.n_contrib[pix] = last[k];
            }
        }
    }
}

template <int PPT, int BATCH, bool STATS>
static gs_status_t launch_fwd(const RenderFwdArgs &a, const ViewTable &vt, cudaStream_t s)
{
    auto kern = render_fwd_kernel<PPT, BATCH, STATS>;
    constexpr int threads = kTilePix / PPT;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    const int64_t slots = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(slots < vt.n_tiles_total ? slots : vt.n_tiles_total);
    kern<<<grid > 0 ? grid : 1, threads, 0, s>>>(a, vt);
    return launch_status();
}

template <bool STATS>
static gs_status_t dispatch_fwd(const RenderFwdArgs &a, const ViewTable &vt, cudaStream_t s)
{
    switch (render_variant_fwd()) {
    case 0: return launch_fwd<1, 256, STATS>(a, vt, s);
    case 1: return launch_fwd<2, 128, STATS>(a, vt, s);
    case 2: return launch_fwd<2, 256, STATS>(a, vt, s);
    case 3: return launch_fwd<4, 64, STATS>(a, vt, s);
    case 4: return launch_fwd<4, 128, STATS>(a, vt, s);
    default: return launch_fwd<8, 64, STATS>(a, vt, s);
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
    RenderFwdArgs a = {};
    a.rec = reinterpret_cast<const float4 *>(proj->rec);
    a.n = n;
    a.vals = bins->vals;
    a.ranges = bins->ranges;
    a.rgb = img->rgb;
    a.depth = img->depth;
    a.alpha = img->alpha;
    a.final_T = img->final_T;
    a.n_contrib = img->n_contrib;
    a.work_counter = work_counter;
    return dispatch_fwd<false>(a, vt, s);
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
    return launch_fwd<1, 256, true>(a, vt, s);
}

// Compositing kernel variants in use (pixels per thread x staged batch), set by
// the autotuner; defaults suit 1200x680 views of room-scale scenes.
namespace gs {
static int g_variant_fwd = 1;
static int g_variant_bwd = 3;
int render_variant_fwd() { return g_variant_fwd; }
int render_variant_bwd() { return g_variant_bwd; }
}  // namespace gs

extern "C" gs_status_t gs_set_render_variants(int32_t fwd, int32_t bwd)
{
    if (fwd < 0 || fwd >= kFwdVariants || bwd < 0 || bwd >= kBwdVariants) return GS_ERR_INVALID_ARG;
    g_variant_fwd = fwd;
    g_variant_bwd = bwd;
    return GS_OK;
}

extern "C" gs_status_t gs_get_render_variants(int32_t *fwd, int32_t *bwd, int32_t *n_fwd, int32_t *n_bwd)
{
    if (fwd) *fwd = g_variant_fwd;
    if (bwd) *bwd = g_variant_bwd;
    if (n_fwd) *n_fwd = kFwdVariants;
    if (n_bwd) *n_bwd = kBwdVariants;
    return GS_OK;
}
