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
// With t = dL/dalpha o g (0 where the clamp is active, a decision taken on
// log2(o g) as in the forward; o g is the raw alpha the walk computes) and
// d = mean - pixel,
// power = -1/2 (A dx^2 + 2 B dx dy + C dy^2), so over a thread's pixels (one
// column: dx is common) the mean and conic gradients need only
// G = sum t, S1 = sum t dy, S2 = sum t dy^2:
//   dL/du = -(A dx G + B S1),  dL/dv = -(B dx G + C S1),
//   dL/dA = -dx^2 G / 2,  dL/dB = -dx S1,  dL/dC = -S2 / 2,  dL/do = G / o.
//
// Work items are (view, tile, band) with a band of BW x PPT * 32 / BW pixels
// (a thread's PPT pixels share a column), pulled by warps from an atomic
// counter.  A warp walks the entries up to its
// pixels' last blend backwards in chunks of 32 (next chunk prefetched),
// keeping only the entries that can reach alpha = 1/255 in its band (the same
// conservative test as the forward); warps never wait for one another.  All
// threads of a warp are at the same entry at the same time: a thread sums its
// PPT pixels' terms in registers, two pixels at a time (a pixel pair that no
// lane blends is skipped by the warp; two pairs that both blend run as one
// straight-line block, so that their chains interleave and their copies of
// the entry's values are shared), and the warp reduces the ten gradients of
// three to five entries at a time through a transposed table in shared memory
// (five paired column stores a lane per entry, then one 32-pair row sum a
// lane per batch); the lanes holding a total pair add them to HBM in one
// predicated paired atomic instruction.  Per
// warp band rather than per tile costs few extra atomics: after culling an
// entry rarely reaches more than one band.  With eight pixels a thread a band
// is a 16 x 16 item whose two halves are culled apart: an entry kept in both
// is reduced once, an entry kept in one is tested in that half only.  PPT is
// picked by the autotuner.
#include <type_traits>

#include "async_copy.cuh"
#include "common.cuh"
#include "render.cuh"
#include "tma.cuh"

namespace gs {

struct RenderBwdArgs {
    const float4 *rec;
    int64_t n;
    const uint32_t *vals;
    const uint32_t *ranges;
    const float *final_T;
    const uint32_t *n_contrib;
    const float *d_rgb, *d_depth, *d_alpha;
    float *grad2d;
    uint32_t *work_counter;
    uint32_t *status;  // device error word (a bounded wait that expired), may be null
    uint32_t n_items;  // (view, tile, band) work items, set by the launcher
};

constexpr int kAcc = 10;
// The ten sums of a batch of consecutive entries are reduced over the warp
// together: every lane stores its values as five pairs, one column of a
// (batch * 5) x 32 table of pairs in shared memory (rows padded to kRedPitch
// pairs: the 8-byte column stores and the 16-byte row loads below are free of
// bank conflicts), then lane j adds up row j and the lanes holding a total
// pair add it to HBM in one predicated paired atomic instruction (the pairs
// are 8-byte aligned: grad2d rows are 48 bytes, their base 16-byte aligned).
constexpr int kPairs = kAcc / 2;
constexpr int kRedPitch = 34;
// Entries a batch: as many as the table can hold while the block still leaves
// room in shared memory for the blocks per SM the launch bounds ask for: five
// with four pixels a thread (five blocks per SM; five entries a batch measured
// 2 % faster than four), four with eight pixels a thread (four blocks, the
// upstream gradients in shared memory as well), three with TMA staging (its
// gather buffers) or one or two pixels a thread (eight blocks).
template <int PPT, bool TMA>
struct RedBatch {
    static constexpr int value = TMA ? 3 : PPT == 4 ? 5 : PPT == 8 ? 4 : 3;
    static_assert(value * kPairs <= 32, "one row per lane");
};

// Record and index of list entry idx (zeros past the end of the walk).
__device__ __forceinline__ void load_bwd_entry(const RenderBwdArgs &a, int64_t rbase, uint32_t idx, bool valid,
                                               float4 &r0, float4 &r1, float4 &r2, uint32_t &g)
{
    if (valid) {
        g = a.vals[idx];
        const int64_t o = rbase + g;
        r0 = __ldg(a.rec + 3 * o);
        r1 = __ldg(a.rec + 3 * o + 1);
        r2 = __ldg(a.rec + 3 * o + 2);
    } else {
        g = 0;
        r0 = r1 = r2 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// CH list entries (32 or 64: one or two a lane) are loaded, culled and staged
// together, the next CH loaded while they are walked: by the lanes' own loads
// (TMA = false), or gathered four records at a time by the tensor memory
// accelerator into a second shared-memory buffer (tma.cuh).
// ASYNC (32-entry chunks): the lanes copy the next chunk's records into a
// second shared-memory buffer with their own asynchronous copies (through L1,
// like the lane loads, but holding no registers), and load the Gaussian
// indices one chunk further ahead.
template <int PPT, int BW, int CH, bool TMA, bool ASYNC = false>
__global__ void __launch_bounds__(kRenderThreads, RenderOccupancy<PPT, TMA || ASYNC>::bwd)
    render_bwd_kernel(RenderBwdArgs a, ViewTable vt, const __grid_constant__ CUtensorMap rec_map)
{
    static_assert(!(TMA && ASYNC) && (!ASYNC || CH == 32), "one staging mode; asynchronous copies of 32 entries");
    constexpr int WARPS = kRenderThreads / 32;
    constexpr int RS = 32 / BW;   // rows between a thread's pixels
    constexpr int BH = PPT * RS;  // band height (width BW)
    constexpr int NC = CH / 32;   // entries a lane stages per chunk
    constexpr int NP = (PPT + 1) / 2;  // pixel pairs a thread
    // eight pixels a thread (a 16 x 16 item): the item's upper and lower
    // halves (rows [0, BH / 2) and [BH / 2, BH), two pixel pairs each) are
    // culled apart, so an entry kept in one half costs the tests of that half
    // only, and an entry kept in both is reduced once for the whole item; the
    // upstream gradients wait in shared memory (each lane reads its own) to
    // keep the registers of four more pixels free
    constexpr bool SPLIT = PPT == 8;
    __shared__ float4 s_up[SPLIT ? WARPS : 1][SPLIT ? NP : 1][2][32];
    __shared__ float4 s_rec[TMA ? 1 : WARPS][ASYNC ? 2 : 1][3][TMA ? 1 : CH];  // (per buffer, ASYNC)
    __shared__ uint32_t s_gid[WARPS][TMA || ASYNC ? 2 : 1][CH];  // Gaussian index of each staged entry (per buffer)
    constexpr int kBatch = RedBatch<PPT, TMA>::value;
    __shared__ __align__(16) float2 s_red[WARPS][kBatch * kPairs][kRedPitch];
    __shared__ uint32_t s_bgid[WARPS][kBatch];
    constexpr int kBufBytes = (CH / kGatherRows) * kGatherSlot;
    __shared__ alignas(128) unsigned char s_tbuf[TMA ? WARPS : 1][2][TMA ? kBufBytes : 16];
    __shared__ alignas(8) uint64_t s_bar[WARPS][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t phase = 0;  // TMA: bit k = parity of barrier k's next phase
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
    const int red_entry = lane / kPairs, red_pair = lane % kPairs;  // the row this lane adds up
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
        const float bx0 = (float)(tx0 + bxo) + 0.5f, bx1 = bx0 + (float)(BW - 1);
        const float by0 = (float)(ty0 + byo) + 0.5f, by1 = by0 + (float)(BH - 1);
        const float bym = by0 + (float)(BH / 2 - 1);  // last row centre of the upper half
        const uint32_t b = a.ranges[2 * item];
        const int64_t rbase = (int64_t)v * a.n;
        // entries waiting in s_red, and their reduction
        int nb = 0;
        auto flush = [&]() {
            __syncwarp();  // every lane's columns (and lane 0's ids) are written
            if (red_entry < nb) {
                // the row's 32 pairs, two a load, in two running sums
                const float4 *row = reinterpret_cast<const float4 *>(&s_red[warp][lane][0]);
                float4 q = row[0];
                float2 even = make_float2(q.x, q.y), odd = make_float2(q.z, q.w);
                #pragma unroll
                for (int c = 1; c < 16; c++) {
                    q = row[c];
                    even = __fadd2_rn(even, make_float2(q.x, q.y));
                    odd = __fadd2_rn(odd, make_float2(q.z, q.w));
                }
                const float2 r = __fadd2_rn(even, odd);
                if (r.x != 0.0f || r.y != 0.0f)
                    atomicAdd(reinterpret_cast<float2 *>(a.grad2d + 12 * (rbase + s_bgid[warp][red_entry])) + red_pair,
                              r);
            }
            __syncwarp();  // the table may be written again
            nb = 0;
        };

        // per pixel: T running transmittance, gC/gD upstream gradients,
        // R = gA T_final - (sum over later blended entries of (c.gC + z gD) alpha T)
        // pixel state in pairs (pixels 2i, 2i + 1 of the thread) for packed
        // FP32x2 updates; with one pixel a thread the second is never blended
        float2 T[NP], gC0[NP], gC1[NP], gC2[NP], gD[NP], R[NP];
        uint32_t last[2 * NP];
        uint32_t my_last = 0;
        #pragma unroll
        for (int i = 0; i < NP; i++) {
            float t[2] = {1.0f, 1.0f}, c0[2] = {0.f, 0.f}, c1[2] = {0.f, 0.f}, c2[2] = {0.f, 0.f}, d[2] = {0.f, 0.f},
                  r[2] = {0.f, 0.f};
            #pragma unroll
            for (int h = 0; h < 2; h++) {
                const int k = 2 * i + h;
                const int py = py0 + RS * k;
                last[k] = 0;
                if (k < PPT && px < V.width && py < V.height) {
                    const int64_t pix = V.pix_base + (int64_t)py * V.width + px;
                    t[h] = a.final_T[pix];
                    last[k] = a.n_contrib[pix];
                    if (a.d_rgb) {
                        c0[h] = a.d_rgb[3 * pix];
                        c1[h] = a.d_rgb[3 * pix + 1];
                        c2[h] = a.d_rgb[3 * pix + 2];
                    }
                    if (a.d_depth) d[h] = a.d_depth[pix];
                    if (a.d_alpha) r[h] = a.d_alpha[pix] * t[h];
                }
                my_last = max(my_last, last[k]);
            }
            T[i] = f2(t[0], t[1]);
            gC0[i] = f2(c0[0], c0[1]);
            gC1[i] = f2(c1[0], c1[1]);
            gC2[i] = f2(c2[0], c2[1]);
            gD[i] = f2(d[0], d[1]);
            R[i] = f2(r[0], r[1]);
            if constexpr (SPLIT) {
                s_up[warp][i][0][lane] = make_float4(c0[0], c0[1], c1[0], c1[1]);
                s_up[warp][i][1][lane] = make_float4(c2[0], c2[1], d[0], d[1]);
            }
        }
        const uint32_t warp_last = __reduce_max_sync(kFullMask, my_last);

        // the gradients of one staged entry (p, c, col) of Gaussian gid at list
        // position pos: every pixel pair of the thread, then the warp's sums
        // halves: bit 0 = the entry is kept in the upper half, bit 1 = in the
        // lower half (both set without the split)
        auto grad_entry = [&](const float4 &p, const float4 &c, const float4 &col, uint32_t gid, uint32_t pos,
                              uint32_t halves) {
            // per pixel pair: colour (3) and depth gradients, and the sums
            // G, S1, S2 (of t = dL/dalpha o g), accumulated two pixels at a time
            float2 gc[4] = {f2(0.f), f2(0.f), f2(0.f), f2(0.f)};
            float2 G2 = f2(0.f), S12 = f2(0.f), S22 = f2(0.f);
            bool contrib = false;
            const SplatColumn kc = splat_column(p, c, sx);
            {
                // per group of pixel pairs (a half of the item with the split,
                // else all of them): the blend tests first, then the pairs
                // with a blended pixel (independent chains interleave).  No
                // test of pos against the thread's own last blend: the warp
                // walks below its largest last blend, so some thread always
                // tests, and a thread past its pixels' last blends finds no
                // blended pixel (pos >= last) without a branch of its own
                constexpr int GROUPS = SPLIT ? 2 : 1, GP = NP / GROUPS;
                #pragma unroll
                for (int h = 0; h < GROUPS; h++) {
                    // a half the entry cannot reach (the warp agrees) is not tested
                    if (SPLIT && !((halves >> h) & 1u)) continue;
                    float2 l2[GP], dy[GP];
                    bool hx[GP], hy[GP];
                    #pragma unroll
                    for (int j = 0; j < GP; j++) {
                        const int i = h * GP + j;
                        l2[j] = splat_log2a2(
                            kc, p, c, col,
                            f2((float)(py0 + RS * 2 * i) + 0.5f, (float)(py0 + RS * (2 * i + 1)) + 0.5f), &dy[j]);
                        hx[j] = pos < last[2 * i] && l2[j].x >= kLog2AlphaMin;
                        hy[j] = pos < last[2 * i + 1] && l2[j].y >= kLog2AlphaMin;
                    }
                    // the body of pair j of this group, run by every lane of
                    // the warp: a lane whose pair does not blend runs it with
                    // raw alpha 0, which changes none of its state and adds
                    // exactly zero
                    auto pair_body = [&](auto J) {
                        constexpr int j = decltype(J)::value;
                        const int i = h * GP + j;
                        // the pair's upstream gradients
                        float2 uc0 = gC0[i], uc1 = gC1[i], uc2 = gC2[i], ud = gD[i];
                        if constexpr (SPLIT) {
                            const float4 q0 = ld_shared_f4(&s_up[warp][i][0][lane]);
                            const float4 q1 = ld_shared_f4(&s_up[warp][i][1][lane]);
                            uc0 = f2(q0.x, q0.y);
                            uc1 = f2(q0.z, q0.w);
                            uc2 = f2(q1.x, q1.y);
                            ud = f2(q1.z, q1.w);
                        }
                        // a pixel of the pair that does not blend this entry takes
                        // raw alpha 0, so its w, t and sums are exactly zero
                        const float2 araw =
                            f2(hx[j] ? ex2_approx(l2[j].x) : 0.0f, hy[j] ? ex2_approx(l2[j].y) : 0.0f);
                        const float2 al = f2(fminf(kAlphaMax, araw.x), fminf(kAlphaMax, araw.y));
                        // where the clamp is in force (decided on l2) no gradient passes
                        const bool cx = l2[j].x >= kLog2AlphaMax, cy = l2[j].y >= kLog2AlphaMax;
                        const float2 om = __ffma2_rn(al, f2(-1.0f), f2(1.0f));
                        // 1 - alpha >= 0.01: the fast reciprocal is within 2 ulp
                        const float2 inv = f2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
                        const float2 Tb = __fmul2_rn(T[i], inv);
                        const float2 w = __fmul2_rn(al, Tb);
                        gc[0] = __ffma2_rn(uc0, w, gc[0]);
                        gc[1] = __ffma2_rn(uc1, w, gc[1]);
                        gc[2] = __ffma2_rn(uc2, w, gc[2]);
                        gc[3] = __ffma2_rn(ud, w, gc[3]);
                        float2 wgt = __fmul2_rn(f2(col.x), uc0);
                        wgt = __ffma2_rn(f2(col.y), uc1, wgt);
                        wgt = __ffma2_rn(f2(col.z), uc2, wgt);
                        wgt = __ffma2_rn(f2(p.z), ud, wgt);
                        const float2 dalpha = __ffma2_rn(Tb, wgt, __fmul2_rn(R[i], inv));
                        R[i] = __ffma2_rn(f2(-wgt.x, -wgt.y), w, R[i]);
                        // T of a pixel that does not blend stays exact
                        T[i] = f2(hx[j] ? Tb.x : T[i].x, hy[j] ? Tb.y : T[i].y);
                        const float2 tg = __fmul2_rn(dalpha, araw);
                        const float2 t = f2(cx ? 0.0f : tg.x, cy ? 0.0f : tg.y);
                        const float2 u = __fmul2_rn(t, dy[j]);
                        G2 = __fadd2_rn(G2, t);
                        S12 = __fadd2_rn(S12, u);
                        S22 = __ffma2_rn(u, dy[j], S22);
                    };
                    // warp-uniform skips: a pair that no lane blends is skipped by all
                    bool act[GP];
                    #pragma unroll
                    for (int j = 0; j < GP; j++) {
                        act[j] = __any_sync(kFullMask, hx[j] || hy[j]);
                        contrib = contrib || act[j];
                    }
                    if constexpr (GP == 2) {
                        // both pairs blended (about half the kept entries): one
                        // block of straight-line code, in which the two pairs'
                        // independent chains interleave
                        if (act[0] && act[1]) {
                            pair_body(std::integral_constant<int, 0>{});
                            pair_body(std::integral_constant<int, 1>{});
                        } else if (act[0]) {
                            pair_body(std::integral_constant<int, 0>{});
                        } else if (act[1]) {
                            pair_body(std::integral_constant<int, 1>{});
                        }
                    } else {
                        static_assert(GP == 1, "one or two pixel pairs a group");
                        if (act[0]) pair_body(std::integral_constant<int, 0>{});
                    }
                }
            }
            if (contrib) {  // warp-uniform: set under the warp-uniform pair skip
                // staged conic (A', B', C') = -log2(e) (A/2, B, C/2)
                const float G = G2.x + G2.y, S1 = S12.x + S12.y, S2 = S22.x + S22.y;
                const float dx = kc.dx, dxG = dx * G;
                float gr[kAcc];
                gr[0] = (2.0f * kLn2) * c.x * dxG + kLn2 * c.y * S1;  // -(A dx G + B S1)
                gr[1] = kLn2 * c.y * dxG + (2.0f * kLn2) * c.z * S1;  // -(B dx G + C S1)
                gr[2] = -0.5f * dx * dxG;
                gr[3] = -dx * S1;
                gr[4] = -0.5f * S2;
                gr[5] = G * ex2_approx(-p.w);  // dL/do = G / o
                gr[6] = gc[0].x + gc[0].y;
                gr[7] = gc[1].x + gc[1].y;
                gr[8] = gc[2].x + gc[2].y;
                gr[9] = gc[3].x + gc[3].y;
                #pragma unroll
                for (int k = 0; k < kPairs; k++) s_red[warp][nb * kPairs + k][lane] = f2(gr[2 * k], gr[2 * k + 1]);
                if (lane == 0) s_bgid[warp][nb] = gid;
                if (++nb == kBatch) flush();
            }
        };

        // the warp's cull of a staged chunk, one entry a lane: upper = the
        // entries that can reach alpha >= 1/255 in the item (in its upper half
        // with the split), lower = in its lower half (none without the split)
        auto cull = [&](const float4 &r0, const float4 &r1, bool have, uint32_t &upper, uint32_t &lower) {
            if constexpr (SPLIT) {
                upper = __ballot_sync(kFullMask, have && !splat_misses_box(r0, r1, bx0, bx1, by0, bym));
                lower = __ballot_sync(kFullMask, have && !splat_misses_box(r0, r1, bx0, bx1, bym + 1.0f, by1));
            } else {
                upper = __ballot_sync(kFullMask, have && !splat_misses_box(r0, r1, bx0, bx1, by0, by1));
                lower = 0u;
            }
        };
        auto halves_of = [&](uint32_t upper, uint32_t lower, int bit) -> uint32_t {
            return SPLIT ? ((upper >> bit) & 1u) | (((lower >> bit) & 1u) << 1) : 3u;
        };

        // chunks [lo, hi) of the list, from the warp's last blend down to 0,
        // CH entries a chunk; within a chunk the entries are taken from the
        // highest index down
        uint32_t hi = warp_last;
        uint32_t lo = hi > (uint32_t)CH ? hi - CH : 0u;
        if constexpr (TMA) {
            // the chunk [l0, h0) into buffer kb: each lane fetches its entries'
            // Gaussian indices, every fourth lane gathers four records
            auto issue = [&](uint32_t l0, uint32_t h0, int kb) {
                int row[NC];
                #pragma unroll
                for (int c = 0; c < NC; c++) {
                    const uint32_t idx = l0 + 32 * c + lane;
                    const uint32_t g = a.vals[b + (idx < h0 ? idx : l0)];  // past the end: a valid row, unused
                    s_gid[warp][kb][32 * c + lane] = g;
                    row[c] = (int)(rbase + g);
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
            if (hi > 0) {
                issue(lo, hi, 0);
                pend[0] = true;
            }
            while (hi > 0) {
                const uint32_t nlo = lo > (uint32_t)CH ? lo - CH : 0u;
                if (lo > 0) {
                    issue(nlo, lo, kb ^ 1);
                    pend[kb ^ 1] = true;
                }
                pend[kb] = false;
                if (!wait(kb)) {
                    tma_failed = true;
                    break;
                }
                const unsigned char *buf = s_tbuf[warp][kb];
                uint32_t todo[NC], upper[NC], lower[NC];
                #pragma unroll
                for (int c = 0; c < NC; c++) {
                    const int slot = 32 * c + lane;
                    const float4 r0 = *reinterpret_cast<const float4 *>(buf + rec_offset(slot));
                    const float4 r1 = *reinterpret_cast<const float4 *>(buf + rec_offset(slot) + 16);
                    cull(r0, r1, lo + slot < hi, upper[c], lower[c]);
                    todo[c] = upper[c] | lower[c];
                }
                #pragma unroll
                for (int cc = NC - 1; cc >= 0; cc--)
                    while (todo[cc]) {
                        const int bit = 31 - __clz(todo[cc]);
                        todo[cc] &= ~(1u << bit);
                        const int slot = 32 * cc + bit;
                        const float4 *r = reinterpret_cast<const float4 *>(buf + rec_offset(slot));
                        grad_entry(r[0], r[1], r[2], s_gid[warp][kb][slot], lo + (uint32_t)slot,
                                   halves_of(upper[cc], lower[cc], bit));
                    }
                __syncwarp();  // buffer kb is read before it is filled again
                hi = lo;
                lo = nlo;
                kb ^= 1;
            }
            // a chunk gathered ahead of a walk that stopped
            #pragma unroll
            for (int k2 = 0; k2 < 2; k2++)
                if (pend[k2] && !wait(k2)) tma_failed = true;
        } else if constexpr (ASYNC) {
            auto gid_at = [&](uint32_t l0, uint32_t h0) -> uint32_t {
                const uint32_t idx = l0 + lane;
                return idx < h0 ? a.vals[b + idx] : 0u;
            };
            // chunk [l0, h0) into buffer kb, the indices g already loaded
            auto copy = [&](uint32_t l0, uint32_t h0, uint32_t g, int kb) {
                s_gid[warp][kb][lane] = g;
                if (l0 + lane < h0) {
                    const float4 *src = a.rec + 3 * (rbase + g);
                    cp_async16_ca(&s_rec[warp][kb][0][lane], src);
                    cp_async16_ca(&s_rec[warp][kb][1][lane], src + 1);
                    cp_async16_ca(&s_rec[warp][kb][2][lane], src + 2);
                }
                cp_async_commit();
            };
            int kb = 0;
            if (hi > 0) copy(lo, hi, gid_at(lo, hi), 0);
            uint32_t nlo = lo > (uint32_t)CH ? lo - CH : 0u;
            uint32_t g_next = lo > 0 ? gid_at(nlo, lo) : 0u;  // indices of the next chunk
            while (hi > 0) {
                cp_async_wait<0>();
                __syncwarp();  // every lane's copies of this chunk have landed
                if (lo > 0) {
                    copy(nlo, lo, g_next, kb ^ 1);
                    const uint32_t nnlo = nlo > (uint32_t)CH ? nlo - CH : 0u;
                    g_next = nlo > 0 ? gid_at(nnlo, nlo) : 0u;
                }
                uint32_t upper, lower;
                cull(s_rec[warp][kb][0][lane], s_rec[warp][kb][1][lane], lo + lane < hi, upper, lower);
                uint32_t todo = upper | lower;
                while (todo) {
                    const int bit = 31 - __clz(todo);
                    todo &= ~(1u << bit);
                    grad_entry(s_rec[warp][kb][0][bit], s_rec[warp][kb][1][bit], s_rec[warp][kb][2][bit],
                               s_gid[warp][kb][bit], lo + (uint32_t)bit, halves_of(upper, lower, bit));
                }
                __syncwarp();  // buffer kb is read before it is filled again
                hi = lo;
                lo = nlo;
                nlo = lo > (uint32_t)CH ? lo - CH : 0u;
                kb ^= 1;
            }
        } else {
            float4 n0[NC], n1[NC], n2[NC];
            uint32_t ng[NC];
            #pragma unroll
            for (int c = 0; c < NC; c++)
                load_bwd_entry(a, rbase, b + lo + 32 * c + lane, lo + 32 * c + lane < hi, n0[c], n1[c], n2[c], ng[c]);
            while (hi > 0) {
                const uint32_t nlo = lo > (uint32_t)CH ? lo - CH : 0u;
                uint32_t todo[NC], upper[NC], lower[NC];
                __syncwarp();  // the previous chunk's records have been read
                #pragma unroll
                for (int c = 0; c < NC; c++) {
                    const float4 r0 = n0[c], r1 = n1[c], r2 = n2[c];
                    const uint32_t g_self = ng[c];
                    const bool have = lo + 32 * c + lane < hi;
                    if (lo > 0)
                        load_bwd_entry(a, rbase, b + nlo + 32 * c + lane, nlo + 32 * c + lane < lo, n0[c], n1[c],
                                       n2[c], ng[c]);
                    cull(r0, r1, have, upper[c], lower[c]);
                    todo[c] = upper[c] | lower[c];
                    s_rec[warp][0][0][32 * c + lane] = r0;
                    s_rec[warp][0][1][32 * c + lane] = r1;
                    s_rec[warp][0][2][32 * c + lane] = r2;
                    s_gid[warp][0][32 * c + lane] = g_self;
                }
                __syncwarp();
                #pragma unroll
                for (int cc = NC - 1; cc >= 0; cc--)
                    while (todo[cc]) {
                        const int bit = 31 - __clz(todo[cc]);
                        todo[cc] &= ~(1u << bit);
                        const int slot = 32 * cc + bit;
                        grad_entry(s_rec[warp][0][0][slot], s_rec[warp][0][1][slot], s_rec[warp][0][2][slot],
                                   s_gid[warp][0][slot], lo + (uint32_t)slot, halves_of(upper[cc], lower[cc], bit));
                    }
                hi = lo;
                lo = nlo;
            }
        }
        if (nb > 0) flush();
        if (TMA && tma_failed) {  // a gather never completed: report it and stop taking work
            if (lane == 0) raise_status(a.status, GS_ERR_TIMEOUT);
            break;
        }
    }
}

template <int PPT, int BW, int CH, bool TMA, bool ASYNC = false>
static gs_status_t launch_bwd(RenderBwdArgs a, ViewTable vt, const CUtensorMap &map, cudaStream_t s)
{
    // work items: the bands of every tile of every view (tile shapes are per view)
    a.n_items = render_items(&vt, BW, PPT * (32 / BW));
    auto kern = render_bwd_kernel<PPT, BW, CH, TMA, ASYNC>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRenderThreads, 0);
    const int64_t slots = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int64_t blocks_needed = ((int64_t)a.n_items + kRenderThreads / 32 - 1) / (kRenderThreads / 32);
    const int grid = (int)(slots < blocks_needed ? slots : blocks_needed);
    kern<<<grid > 0 ? grid : 1, kRenderThreads, 0, s>>>(a, vt, map);
    return launch_status();
}

template <int CH, bool TMA, bool ASYNC = false>
static gs_status_t dispatch_bwd_band(int base, const RenderBwdArgs &a, const ViewTable &vt, const CUtensorMap &map,
                                     cudaStream_t s)
{
    switch (base) {
    case 0: return launch_bwd<1, 8, CH, TMA, ASYNC>(a, vt, map, s);
    case 1: return launch_bwd<2, 8, CH, TMA, ASYNC>(a, vt, map, s);
    case 2: return launch_bwd<2, 16, CH, TMA, ASYNC>(a, vt, map, s);
    case 3: return launch_bwd<4, 8, CH, TMA, ASYNC>(a, vt, map, s);
    case 4: return launch_bwd<4, 16, CH, TMA, ASYNC>(a, vt, map, s);
    default: return launch_bwd<8, 16, CH, TMA, ASYNC>(a, vt, map, s);
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
    RenderBwdArgs a = {};
    a.rec = reinterpret_cast<const float4 *>(proj->rec);
    a.n = n;
    a.vals = bins->vals;
    a.ranges = bins->ranges;
    a.final_T = img->final_T;
    a.n_contrib = img->n_contrib;
    a.d_rgb = d_rgb;
    a.d_depth = d_depth;
    a.d_alpha = d_alpha;
    a.grad2d = grad2d;
    a.work_counter = work_counter;
    a.status = bins->status;
    // the variant and, for the gathering variants, the record tensor map (a
    // gathering variant whose map cannot be made runs with lane loads)
    int var = fitting_variant(vt, render_variant_bwd());
    CUtensorMap map = {};
    if (variant_gathers(var) && make_record_map(reinterpret_cast<const float *>(a.rec), n * vt.n_views, &map) != GS_OK)
        var -= 2 * kBandVariants;
    if (cudaMemsetAsync(work_counter, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    const int base = var % kBandVariants;
    switch (var / kBandVariants) {
    case 0: return dispatch_bwd_band<32, false>(base, a, vt, map, s);
    case 1: return dispatch_bwd_band<32, false, true>(base, a, vt, map, s);
    case 2: return dispatch_bwd_band<32, true>(base, a, vt, map, s);
    default: return dispatch_bwd_band<64, true>(base, a, vt, map, s);
    }
}
