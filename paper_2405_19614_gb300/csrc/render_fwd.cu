// a5. Forward compositing (Sec. 3.4: C(p) = sum_i c_i f_i prod_{j<i} (1 - f_j)
// and D(p) likewise with the depths d_i; Sec. 3.3: border mask M_b(p) =
// sum_i f_i prod_{j<i} (1 - f_j) = 1 - T_final).
//
// One persistent launch covers every (view, tile, band) work item of every
// view: warps pull items from an atomic counter, so views of different sizes
// (and tile shapes) share one launch and long tiles do not hold up a static
// schedule.  A band is BW x PPT * 32 / BW pixels of a tile and each thread
// owns PPT pixels of it (one column, rows r, r + 32 / BW, ...).  A warp walks
// its tile's list in chunks of 32 (or 64) entries, one per lane, fetching the
// next chunk while it works on the current one (into registers, by
// asynchronous copies or by the tensor memory accelerator into shared
// memory), drops (in parallel) the entries that provably cannot reach
// alpha = 1/255 in its band (splat_misses_box), and walks the rest (records
// in the base-2 form of render.cuh), with asynchronous-copy staging four
// entries at a time; it stops once all its pixels have run out of
// transmittance.  Warps never wait for one another.  The band shape and the
// staging are chosen per workload by the autotuner.
#include "async_copy.cuh"
#include "common.cuh"
#include "render.cuh"
#include "tma.cuh"

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
    uint32_t *status;  // device error word (a bounded wait that expired), may be null
    uint32_t n_items;  // (view, tile, band) work items, set by the launcher
    // LOSS variant only: the L1 terms of a6 evaluated as each pixel finishes
    const float *trgb, *tdepth;
    float kc, kd, gamma;
    int32_t use_gate;
    float *loss, *d_rgb, *d_depth;
};

__device__ __forceinline__ float sgn(float x) { return (float)((x > 0.0f) - (x < 0.0f)); }

// The three float4 of list entry idx of a tile (zeros past the end).
__device__ __forceinline__ void load_entry(const RenderFwdArgs &a, int64_t rbase, uint32_t idx, uint32_t e,
                                           float4 &r0, float4 &r1, float4 &r2)
{
    if (idx < e) {
        const int64_t g = rbase + a.vals[idx];
        r0 = __ldg(a.rec + 3 * g);
        r1 = __ldg(a.rec + 3 * g + 1);
        r2 = __ldg(a.rec + 3 * g + 2);
    } else {
        r0 = r1 = r2 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// STATS = true counts, per pixel, the list entries evaluated and blended (the
// algorithmic work of the compositing, without culling) instead of writing the
// image.  CH list entries (32 or 64: one or two a lane) are loaded, culled and
// staged together; the next CH are loaded while they are walked: by the
// lanes' own loads into registers (TMA = false), or, with TMA, gathered four
// records at a time by the tensor memory accelerator straight into a second
// shared-memory buffer (tma.cuh), which takes the prefetch out of registers.
// ASYNC (32-entry chunks): the lanes copy the next chunk's records into a
// second shared-memory buffer with their own asynchronous copies (through L1,
// holding no registers) and load the Gaussian indices one chunk further ahead.
template <int PPT, int BW, int CH, bool TMA, bool STATS, bool LOSS, bool ASYNC = false>
__global__ void __launch_bounds__(kRenderThreads, ASYNC ? RenderOccupancy<PPT, true>::fwd_async
                                                        : RenderOccupancy<PPT, TMA>::fwd) render_fwd_kernel(
    RenderFwdArgs a, ViewTable vt, const __grid_constant__ CUtensorMap rec_map)
{
    static_assert(!(TMA && ASYNC) && (!ASYNC || CH == 32), "one staging mode; asynchronous copies of 32 entries");
    __shared__ float s_loss[kRenderThreads / 32];
    float lacc = 0.0f;  // LOSS: this thread's share of the loss
    constexpr int WARPS = kRenderThreads / 32;
    constexpr int RS = 32 / BW;   // rows between a thread's pixels
    constexpr int BH = PPT * RS;  // band height (width BW)
    constexpr int NC = CH / 32;   // entries a lane stages per chunk
    // (u, v, z, log2 o), (base-2 conic, du), (rgb, dv) of a chunk
    __shared__ float4 s_rec[TMA ? 1 : WARPS][ASYNC ? 2 : 1][3][TMA ? 1 : CH];
    constexpr int kBufBytes = (CH / kGatherRows) * kGatherSlot;
    __shared__ alignas(128) unsigned char s_tbuf[TMA ? WARPS : 1][2][TMA ? kBufBytes : 16];
    __shared__ alignas(8) uint64_t s_bar[WARPS][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t phase = 0;     // TMA: bit k = parity of barrier k's next phase
    bool tma_failed = false;
    // the tensor map's address in the parameter space (taken here, outside
    // any lambda, so that it is the parameter itself and not a copy)
    const CUtensorMap *map = &rec_map;
    if (TMA) {
        if (lane == 0) {
            mbar_init(&s_bar[warp][0], 1);
            mbar_init(&s_bar[warp][1], 1);
            fence_mbar_init();
        }
        __syncwarp();
    }
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(a.work_counter, 1u);
        wi = __shfl_sync(kFullMask, wi, 0);
        if (wi >= a.n_items) break;
        // work item -> view, tile of the view, band of the tile
        const int v = view_of_item(vt, (int)wi);
        const ViewInfo &V = vt.v[v];
        // tile sides and band sides are powers of two: the band index splits by shifts
        const int sx_shift = __ffs(V.tile_w) - __ffs(BW), sb_shift = sx_shift + __ffs(V.tile_h) - __ffs(BH);
        const int local = (int)wi - V.item_base;
        const int lt = local >> sb_shift, band = local & ((1 << sb_shift) - 1);
        const int item = V.tile_base + lt;  // global tile id
        const int bxo = (band & ((1 << sx_shift) - 1)) * BW, byo = (band >> sx_shift) * BH;  // band origin in the tile
        const int tx0 = (lt % V.tiles_x) * V.tile_w, ty0 = (lt / V.tiles_x) * V.tile_h;
        const int px = tx0 + bxo + lane % BW;
        const int py0 = ty0 + byo + lane / BW;  // this thread's rows: py0 + RS k
        const float sx = (float)px + 0.5f;
        // the warp's band of pixel centres, for culling
        const float bx0 = (float)(tx0 + bxo) + 0.5f, bx1 = bx0 + (float)(BW - 1);
        const float by0 = (float)(ty0 + byo) + 0.5f, by1 = by0 + (float)(BH - 1);
        const uint32_t b = a.ranges[2 * item], e = a.ranges[2 * item + 1];
        const int64_t rbase = (int64_t)v * a.n;

        // pixel state in pairs (pixels 2i, 2i + 1 of the thread), updated with
        // packed FP32x2 instructions; with one pixel a thread the second of
        // the pair is never live
        constexpr int NP = (PPT + 1) / 2;
        float2 T[NP], C0[NP], C1[NP], C2[NP], D[NP];
        uint32_t last[2 * NP], n_eval[2 * NP], n_blend[2 * NP];
        bool live[2 * NP];
        #pragma unroll
        for (int i = 0; i < NP; i++) {
            T[i] = f2(1.0f);
            C0[i] = C1[i] = C2[i] = D[i] = f2(0.0f);
        }
        #pragma unroll
        for (int k = 0; k < 2 * NP; k++) {
            last[k] = n_eval[k] = n_blend[k] = 0;
            live[k] = k < PPT && px < V.width && (py0 + RS * k) < V.height;
        }
        // whether any pixel of the warp has transmittance left
        auto warp_alive = [&]() {
            bool any = false;
            #pragma unroll
            for (int k = 0; k < 2 * NP; k++) any = any || live[k];
            return __any_sync(kFullMask, any);
        };
        // the walk of one staged entry (p, c, col): the thread's pixel pairs
        auto blend_entry = [&](const float4 &p, const float4 &cc, const float4 &col, uint32_t pos) {
            const SplatColumn kc = splat_column(p, cc, sx);
            // two pixels per packed evaluation and update; branch-free per
            // pixel (a skipped pixel adds exactly zero), so the chains interleave
            #pragma unroll
            for (int i = 0; i < NP; i++) {
                float2 dy;
                const float2 l2 = splat_log2a2(
                    kc, p, cc, col, f2((float)(py0 + RS * 2 * i) + 0.5f, (float)(py0 + RS * (2 * i + 1)) + 0.5f),
                    &dy);
                const float2 al = f2(alpha_of_l2(l2.x), alpha_of_l2(l2.y));
                const float2 tT = __fmul2_rn(T[i], __fadd2_rn(f2(1.0f), f2(-al.x, -al.y)));  // T (1 - alpha)
                const float2 aT = __fmul2_rn(al, T[i]);
                bool blend[2];
                #pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int k = 2 * i + h;
                    const bool hit = live[k] && (h ? l2.y : l2.x) >= kLog2AlphaMin;
                    const bool stop = hit && (h ? tT.y : tT.x) < kTMin;  // stops before this entry
                    blend[h] = hit && !stop;
                    if (STATS) {
                        n_eval[k] += live[k];
                        n_blend[k] += blend[h];
                    }
                    last[k] = blend[h] ? pos + 1u : last[k];
                    live[k] = live[k] && !stop;
                }
                const float2 w = f2(blend[0] ? aT.x : 0.0f, blend[1] ? aT.y : 0.0f);
                C0[i] = __ffma2_rn(f2(col.x), w, C0[i]);
                C1[i] = __ffma2_rn(f2(col.y), w, C1[i]);
                C2[i] = __ffma2_rn(f2(col.z), w, C2[i]);
                D[i] = __ffma2_rn(f2(p.z), w, D[i]);
                T[i] = f2(blend[0] ? tT.x : T[i].x, blend[1] ? tT.y : T[i].y);
            }
        };
        if constexpr (TMA) {
            // chunks through two shared-memory buffers: the next chunk's
            // records are gathered by the TMA while this one is walked
            auto issue = [&](uint32_t m0, int kb) {
                int row[NC];
                #pragma unroll
                for (int c = 0; c < NC; c++) {
                    const uint32_t idx = m0 + 32 * c + lane;
                    row[c] = (int)(rbase + a.vals[idx < e ? idx : m0]);  // past the end: a valid row, unused
                }
                if (lane == 0) mbar_arrive_expect_tx(&s_bar[warp][kb], CH * kRecBytes);
                __syncwarp();
                #pragma unroll
                for (int c = 0; c < NC; c++) {
                    const int r1 = __shfl_down_sync(kFullMask, row[c], 1);
                    const int r2 = __shfl_down_sync(kFullMask, row[c], 2);
                    const int r3 = __shfl_down_sync(kFullMask, row[c], 3);
                    if ((lane & 3) == 0)
                        tma_gather4(&s_tbuf[warp][kb][rec_offset(32 * c + lane)], map, row[c], r1, r2, r3,
                                    &s_bar[warp][kb]);
                }
            };
            auto wait = [&](int kb) {
                const bool ok = mbar_wait_parity(&s_bar[warp][kb], (phase >> kb) & 1u);
                phase ^= 1u << kb;
                return __all_sync(kFullMask, ok);
            };
            bool pend[2] = {false, false};
            int kb = 0;
            if (b < e) {
                issue(b, 0);
                pend[0] = true;
            }
            for (uint32_t m = b; m < e; m += CH, kb ^= 1) {
                if (!warp_alive()) break;
                if (m + CH < e) {
                    issue(m + CH, kb ^ 1);
                    pend[kb ^ 1] = true;
                }
                pend[kb] = false;
                if (!wait(kb)) {
                    tma_failed = true;
                    break;
                }
                const unsigned char *buf = s_tbuf[warp][kb];
                uint32_t todo[NC];
                #pragma unroll
                for (int c = 0; c < NC; c++) {
                    const int slot = 32 * c + lane;
                    const float4 p = *reinterpret_cast<const float4 *>(buf + rec_offset(slot));
                    const float4 cc = *reinterpret_cast<const float4 *>(buf + rec_offset(slot) + 16);
                    const bool keep = m + slot < e && (STATS || !splat_misses_box(p, cc, bx0, bx1, by0, by1));
                    todo[c] = __ballot_sync(kFullMask, keep);  // every lane takes part
                }
                #pragma unroll
                for (int c = 0; c < NC; c++) {
                    while (todo[c]) {
                        const int j = __ffs(todo[c]) - 1;
                        todo[c] &= todo[c] - 1;
                        const int slot = 32 * c + j;
                        const float4 *r = reinterpret_cast<const float4 *>(buf + rec_offset(slot));
                        blend_entry(r[0], r[1], r[2], m - b + (uint32_t)slot);
                        if (!warp_alive()) {  // the warp's pixels are done (a warp-uniform exit)
                            #pragma unroll
                            for (int c2 = 0; c2 < NC; c2++) todo[c2] = 0;
                            break;
                        }
                    }
                }
                __syncwarp();  // buffer kb is read before it is filled again
            }
            // a chunk gathered ahead of a walk that stopped early
            #pragma unroll
            for (int k2 = 0; k2 < 2; k2++)
                if (pend[k2] && !wait(k2)) tma_failed = true;
        } else if constexpr (ASYNC) {
            auto gid_at = [&](uint32_t m0) -> uint32_t {
                const uint32_t idx = m0 + lane;
                return idx < e ? a.vals[idx] : 0u;
            };
            // chunk [m0, m0 + 32) into buffer kb, its Gaussian indices g already loaded
            auto copy = [&](uint32_t m0, uint32_t g, int kb) {
                if (m0 + lane < e) {
                    const float4 *src = a.rec + 3 * (rbase + g);
                    cp_async16_ca(&s_rec[warp][kb][0][lane], src);
                    cp_async16_ca(&s_rec[warp][kb][1][lane], src + 1);
                    cp_async16_ca(&s_rec[warp][kb][2][lane], src + 2);
                }
                cp_async_commit();
            };
            int kb = 0;
            if (b < e) copy(b, gid_at(b), 0);
            uint32_t g_next = b + CH < e ? gid_at(b + CH) : 0u;  // indices of the next chunk
            for (uint32_t m = b; m < e; m += CH, kb ^= 1) {
                if (!warp_alive()) break;
                cp_async_wait<0>();
                __syncwarp();  // every lane's copies of this chunk have landed
                if (m + CH < e) {
                    copy(m + CH, g_next, kb ^ 1);
                    g_next = m + 2 * CH < e ? gid_at(m + 2 * CH) : 0u;
                }
                const bool keep = m + lane < e && (STATS || !splat_misses_box(s_rec[warp][kb][0][lane],
                                                                              s_rec[warp][kb][1][lane], bx0, bx1,
                                                                              by0, by1));
                uint32_t todo = __ballot_sync(kFullMask, keep);
                // kept entries four (or two) at a time, in one block of
                // straight-line code: a later entry's evaluation (which needs
                // no pixel state) overlaps an earlier entry's blend.  The
                // warp's liveness is tested after each group: an entry walked
                // after the warp's pixels have stopped changes nothing (no
                // pixel is live).  (The same grouping as a lambda shared with
                // the other stagings spilled here and measured 2.4 % slower.)
                // Eight pixels a thread walk one entry at a time: their four
                // pixel pairs already interleave, and grouped entries measured
                // 18 % slower at that register budget.  Groups of eight (two
                // pixels a thread) spill: 0.727 ms at nine blocks per SM, 0.716
                // at eight, against 0.718 for groups of four at nine.
                constexpr int kGroup = PPT >= 8 ? 1 : 4;
                auto blend_bit = [&](int j) {
                    blend_entry(s_rec[warp][kb][0][j], s_rec[warp][kb][1][j], s_rec[warp][kb][2][j],
                                m - b + (uint32_t)j);
                };
                auto pop = [&]() {
                    const int j = __ffs(todo) - 1;
                    todo &= todo - 1;
                    return j;
                };
                while (todo) {
                    const int n_left = __popc(todo);
                    if (kGroup >= 4 && n_left >= 4) {
                        const int j0 = pop(), j1 = pop(), j2 = pop(), j3 = pop();
                        blend_bit(j0);
                        blend_bit(j1);
                        blend_bit(j2);
                        blend_bit(j3);
                    } else if (kGroup >= 2 && n_left >= 2) {
                        const int j0 = pop(), j1 = pop();
                        blend_bit(j0);
                        blend_bit(j1);
                    } else {
                        blend_bit(pop());
                    }
                    if (!warp_alive()) break;  // the warp's pixels are done (a warp-uniform exit)
                }
                __syncwarp();  // buffer kb is read before it is filled again
            }
            cp_async_wait<0>();  // a chunk copied ahead of a walk that stopped early
        } else {
        float4 n0[NC], n1[NC], n2[NC];  // this lane's entries of the next chunk
        #pragma unroll
        for (int c = 0; c < NC; c++) load_entry(a, rbase, b + 32 * c + lane, e, n0[c], n1[c], n2[c]);
        for (uint32_t m = b; m < e; m += CH) {
            if (!warp_alive()) break;
            uint32_t todo[NC];
            __syncwarp();  // the previous chunk's records have been read
            #pragma unroll
            for (int c = 0; c < NC; c++) {
                const float4 r0 = n0[c], r1 = n1[c], r2 = n2[c];
                const bool have = m + 32 * c + lane < e;
                if (m + CH < e) load_entry(a, rbase, m + CH + 32 * c + lane, e, n0[c], n1[c], n2[c]);
                const bool keep = have && (STATS || !splat_misses_box(r0, r1, bx0, bx1, by0, by1));
                todo[c] = __ballot_sync(kFullMask, keep);
                s_rec[warp][0][0][32 * c + lane] = r0;
                s_rec[warp][0][1][32 * c + lane] = r1;
                s_rec[warp][0][2][32 * c + lane] = r2;
            }
            __syncwarp();
            #pragma unroll
            for (int c = 0; c < NC; c++) {
                while (todo[c]) {
                    const int j = __ffs(todo[c]) - 1;
                    todo[c] &= todo[c] - 1;
                    const int slot = 32 * c + j;
                    blend_entry(s_rec[warp][0][0][slot], s_rec[warp][0][1][slot], s_rec[warp][0][2][slot],
                                m - b + (uint32_t)slot);
                    if (!warp_alive()) {  // the warp's pixels are done (a warp-uniform exit)
                        #pragma unroll
                        for (int c2 = 0; c2 < NC; c2++) todo[c2] = 0;
                        break;
                    }
                }
            }
        }
        }
        #pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = py0 + RS * k;
            if (px >= V.width || py >= V.height) continue;
            const int64_t pix = V.pix_base + (int64_t)py * V.width + px;
            const int i = k >> 1;
            const bool hi = k & 1;
            if (STATS) {
                a.n_eval[pix] = n_eval[k];
                a.n_blend[pix] = n_blend[k];
            } else {
                const float t = hi ? T[i].y : T[i].x;
                a.rgb[3 * pix + 0] = hi ? C0[i].y : C0[i].x;
                a.rgb[3 * pix + 1] = hi ? C1[i].y : C1[i].x;
                a.rgb[3 * pix + 2] = hi ? C2[i].y : C2[i].x;
                a.depth[pix] = hi ? D[i].y : D[i].x;
                a.alpha[pix] = 1.0f - t;
                a.final_T[pix] = t;
                a.n_contrib[pix] = last[k];
                if (LOSS) {
                    // the a6 terms of this pixel, in the operations of gs_loss_l1
                    const float C[3] = {hi ? C0[i].y : C0[i].x, hi ? C1[i].y : C1[i].x, hi ? C2[i].y : C2[i].x};
                    const float Dp = hi ? D[i].y : D[i].x, Dt = a.tdepth[pix];
                    bool gate = true;
                    if (a.use_gate) gate = (Dt > 0.0f) && (Dp > 0.0f) && (1.0f - t > a.gamma);
                    const float g = gate ? 1.0f : 0.0f;
                    float l = 0.0f;
                    #pragma unroll
                    for (int ch = 0; ch < 3; ch++) {
                        const float r = C[ch] - a.trgb[3 * pix + ch];
                        l += a.kc * fabsf(r);
                        a.d_rgb[3 * pix + ch] = g * a.kc * sgn(r);
                    }
                    const float r = Dp - Dt;
                    l += a.kd * fabsf(r);
                    a.d_depth[pix] = g * a.kd * sgn(r);
                    lacc += g * l;
                }
            }
        }
        if (TMA && tma_failed) {  // a gather never completed: report it and stop taking work
            if (lane == 0) raise_status(a.status, GS_ERR_TIMEOUT);
            break;
        }
    }
    if (LOSS) {  // one atomic per block (every warp has left the item loop)
        lacc = warp_sum(lacc);
        if (lane == 0) s_loss[warp] = lacc;
        __syncthreads();
        if (tid == 0) {
            float sum = 0.0f;
            #pragma unroll
            for (int w = 0; w < kRenderThreads / 32; w++) sum += s_loss[w];
            atomicAdd(a.loss, sum);
        }
    }
}

template <int PPT, int BW, int CH, bool TMA, bool STATS, bool LOSS = false, bool ASYNC = false>
static gs_status_t launch_fwd(RenderFwdArgs a, ViewTable vt, const CUtensorMap &map, cudaStream_t s)
{
    // work items: the bands of every tile of every view (tile shapes are per view)
    a.n_items = render_items(&vt, BW, PPT * (32 / BW));
    auto kern = render_fwd_kernel<PPT, BW, CH, TMA, STATS, LOSS, ASYNC>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRenderThreads, 0);
    const int64_t slots = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int64_t blocks_needed = ((int64_t)a.n_items + kRenderThreads / 32 - 1) / (kRenderThreads / 32);
    const int grid = (int)(slots < blocks_needed ? slots : blocks_needed);
    kern<<<grid > 0 ? grid : 1, kRenderThreads, 0, s>>>(a, vt, map);
    return launch_status();
}

template <int CH, bool TMA, bool STATS, bool LOSS, bool ASYNC = false>
static gs_status_t dispatch_fwd_band(int base, const RenderFwdArgs &a, const ViewTable &vt, const CUtensorMap &map,
                                     cudaStream_t s)
{
    switch (base) {
    case 0: return launch_fwd<1, 8, CH, TMA, STATS, LOSS, ASYNC>(a, vt, map, s);
    case 1: return launch_fwd<2, 8, CH, TMA, STATS, LOSS, ASYNC>(a, vt, map, s);
    case 2: return launch_fwd<2, 16, CH, TMA, STATS, LOSS, ASYNC>(a, vt, map, s);
    case 3: return launch_fwd<4, 8, CH, TMA, STATS, LOSS, ASYNC>(a, vt, map, s);
    case 4: return launch_fwd<4, 16, CH, TMA, STATS, LOSS, ASYNC>(a, vt, map, s);
    default: return launch_fwd<8, 16, CH, TMA, STATS, LOSS, ASYNC>(a, vt, map, s);
    }
}

// The variant to launch and, for the gathering variants, the record tensor
// map (host work only: nothing is enqueued).  A gathering variant whose map
// cannot be made (no records) runs as the same variant with lane loads.
static int prepare_fwd(const RenderFwdArgs &a, const ViewTable &vt, int var, CUtensorMap *map)
{
    var = fitting_variant(vt, var);
    if (variant_gathers(var) && make_record_map(reinterpret_cast<const float *>(a.rec), a.n * vt.n_views, map) != GS_OK)
        var -= 2 * kBandVariants;
    return var;
}

template <bool STATS, bool LOSS = false>
static gs_status_t dispatch_fwd(int var, const RenderFwdArgs &a, const ViewTable &vt, const CUtensorMap &map,
                                cudaStream_t s)
{
    const int base = var % kBandVariants;
    switch (var / kBandVariants) {
    case 0: return dispatch_fwd_band<32, false, STATS, LOSS>(base, a, vt, map, s);
    case 1: return dispatch_fwd_band<32, false, STATS, LOSS, true>(base, a, vt, map, s);
    case 2: return dispatch_fwd_band<32, true, STATS, LOSS>(base, a, vt, map, s);
    default: return dispatch_fwd_band<64, true, STATS, LOSS>(base, a, vt, map, s);
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
    a.status = bins->status;
    CUtensorMap map = {};
    const int var = prepare_fwd(a, vt, render_variant_fwd(), &map);
    if (cudaMemsetAsync(work_counter, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    return dispatch_fwd<false>(var, a, vt, map, s);
}

extern "C" gs_status_t gs_render_fwd_l1(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins,
                                        const gs_view_t *views, int32_t n_views, gs_image_t *img,
                                        uint32_t *work_counter, const float *target_rgb, const float *target_depth,
                                        float w_c, float w_d, int32_t use_gate, float gamma, float *loss,
                                        float *d_rgb, float *d_depth, void *stream)
{
    if (!proj || !bins || !img || !work_counter || n < 0) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (!img->rgb || !img->depth || !img->alpha || !img->final_T || !img->n_contrib || !bins->ranges ||
        !bins->vals || (n > 0 && !proj->rec) || !target_rgb || !target_depth || !loss || !d_rgb || !d_depth)
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
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
    a.status = bins->status;
    // the weights of gs_loss_l1, over all pixels of the views
    a.kc = (float)((double)w_c / (3.0 * (double)vt.n_pix_total));
    a.kd = (float)((double)w_d / (double)vt.n_pix_total);
    a.trgb = target_rgb;
    a.tdepth = target_depth;
    a.use_gate = use_gate;
    a.gamma = gamma;
    a.loss = loss;
    a.d_rgb = d_rgb;
    a.d_depth = d_depth;
    CUtensorMap map = {};
    const int var = prepare_fwd(a, vt, render_variant_fwd(), &map);
    if (cudaMemsetAsync(work_counter, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    return dispatch_fwd<false, true>(var, a, vt, map, s);
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
    a.status = bins->status;
    const CUtensorMap none = {};
    return launch_fwd<1, 16, 32, false, true>(a, vt, none, s);
}

// Compositing kernel variants in use (see kFwdVariants), set by the
// autotuner; defaults suit 1200x680 views of room-scale scenes.
namespace gs {
static int g_variant_fwd = 7;  // (2, 8) bands, asynchronous-copy staging
static int g_variant_bwd = 9;  // (4, 8) bands, asynchronous-copy staging
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
