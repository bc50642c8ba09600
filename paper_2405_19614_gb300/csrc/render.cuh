// Shared pieces of the forward and backward compositing kernels.
#pragma once

#include "common.cuh"

namespace gs {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// A 16-byte shared-memory load the compiler may not move out of a loop (the
// value stays in shared memory, not in registers, between uses).
__device__ __forceinline__ float4 ld_shared_f4(const float4 *p)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
    return v;
}

// 2^x by the approximate base-2 exponential instruction (a relative error of
// a few units in the last place; results below 2^-126 flush to zero).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The compositing evaluates alpha_i = min(0.99, o_i exp(power_i)) in base 2:
// with power = -1/2 (A dx^2 + C dy^2) - B dx dy and d = mean - pixel centre,
//   log2(o exp(power)) = log2(o) + A' dx^2 + dy (B' dx + C' dy),
//   A' = -log2(e)/2 A, B' = -log2(e) B, C' = -log2(e)/2 C,
// and the projection writes the record in that form (log2 o and A', B', C'
// by a fixed sequence of correctly rounded operations).  An entry costs two
// packed FMAs per pixel pair up to the blend test.  Both alpha decisions are
// taken on this logarithm l2, before any exponential: the entry is skipped
// when l2 < log2(1/255), and the clamp at 0.99 (which passes no gradient) is
// in force when l2 >= log2(0.99).  l2 itself is one fixed sequence of
// correctly rounded FP32 operations on the record, so the decisions are
// reproducible bit for bit (the CPU oracle takes them on the same FP32
// value).  The value blended is min(0.99, 2^l2), branch free; next to the cut
// it may differ from 0.99 by the exponential's last bits either way, which is
// a continuous difference, not a decision.  The forward and backward kernels
// go through the same helpers, so both take the same decisions and the same
// alphas.
constexpr float kLn2 = 0.6931471806f;
constexpr float kLog2AlphaMin = -0x1.ffa37cp+2f;  // FP32 value nearest log2(1/255)
constexpr float kLog2AlphaMax = -0x1.db1f34p-7f;  // FP32 value nearest log2(0.99)

// alpha of a blended entry from its l2: min(0.99, 2^l2), the exponential by
// the approximate instruction.
__device__ __forceinline__ float alpha_of_l2(float l2) { return fminf(kAlphaMax, ex2_approx(l2)); }

// The part of log2(raw alpha) that a thread's pixels share (they lie in one
// column sx): dx, log2(o) + A' dx^2 and B' dx.  The mean is u + du: u - sx is
// exact (both are close FP32 numbers) and the remainder du restores the
// mean's precision.
struct SplatColumn {
    float dx, base, bdx;
};

__device__ __forceinline__ SplatColumn splat_column(const float4 &p, const float4 &c, float sx)
{
    SplatColumn k;
    k.dx = __fadd_rn(__fsub_rn(p.x, sx), c.w);
    k.base = __fmaf_rn(__fmul_rn(c.x, k.dx), k.dx, p.w);
    k.bdx = __fmul_rn(c.y, k.dx);
    return k;
}

// log2(raw alpha) of a staged record at the two pixel centres (sx, sy.x) and
// (sx, sy.y), with dy = mean - pixel centre per pixel.
__device__ __forceinline__ float2 splat_log2a2(const SplatColumn &k, const float4 &p, const float4 &c,
                                               const float4 &col, float2 sy, float2 *dy_out)
{
    const float2 dy = __fadd2_rn(__fadd2_rn(f2(p.y), f2(-sy.x, -sy.y)), f2(col.w));
    *dy_out = dy;
    return __ffma2_rn(dy, __ffma2_rn(f2(c.z), dy, f2(k.bdx)), f2(k.base));
}

// Minimum over t in [t0, t1] of P s^2 + 2 B s t + Q t^2 for a fixed s (Q > 0):
// the unconstrained minimiser t = -B s / Q clamped to the interval.  *mag
// receives the sum of the magnitudes of the three terms at that point.
__device__ __forceinline__ float edge_min(float P, float B, float Q, float s, float t0, float t1, float *mag)
{
    // t only has to be near the minimiser: q(t) - q_min = Q (t - t*)^2 is far
    // below the margin of splat_misses_box for a 2-ulp quotient
    const float t = fminf(fmaxf(__fdividef(-B * s, Q), t0), t1);
    const float a = P * s * s, b = 2.0f * B * s * t, c = Q * t * t;
    *mag = fmaxf(*mag, a + fabsf(b) + c);
    return a + b + c;
}

// Conservative test that a splat cannot reach alpha >= 1/255 anywhere in a box
// of pixel centres [x0, x1] x [y0, y1].  With d = pixel - mean, log2 of the
// raw alpha at a pixel is log2(o) - q(d), q(d) = P dx^2 + 2 B dx dy + Q dy^2
// with (P, B, Q) = -(A', B'/2, C') from the record (positive definite).  q is
// convex with minimum 0 at the mean, so over a box not containing the mean its
// minimum lies on one of the four edges, where it is a one-dimensional
// quadratic; the box minimum bounds q at every pixel centre inside.  The entry
// is dropped when log2(o) - q_min is below log2(1/255) by more than
// 1.5e-3 + 4e-6 M, M the magnitude of the terms of q: more than the FP32
// rounding of this bound and of the per-pixel evaluation together, so a
// dropped entry is one the per-pixel test would have skipped: results are
// unchanged, only work is saved.  (A bound through the smallest eigenvalue of
// the conic is weaker and, for elongated splats, cancels badly in FP32.)
__device__ __forceinline__ bool splat_misses_box(const float4 &p, const float4 &c, float x0, float x1, float y0,
                                                 float y1)
{
    const float ex0 = x0 - p.x, ex1 = x1 - p.x, ey0 = y0 - p.y, ey1 = y1 - p.y;
    float q = 0.0f, mag = 0.0f;
    if (!(ex0 <= 0.0f && ex1 >= 0.0f && ey0 <= 0.0f && ey1 >= 0.0f)) {
        const float P = -c.x, B = -0.5f * c.y, Q = -c.z;
        q = fminf(fminf(edge_min(P, B, Q, ex0, ey0, ey1, &mag), edge_min(P, B, Q, ex1, ey0, ey1, &mag)),
                  fminf(edge_min(Q, B, P, ey0, ex0, ex1, &mag), edge_min(Q, B, P, ey1, ex0, ex1, &mag)));
    }
    return p.w - q < kLog2AlphaMin - (1.5e-3f + 4e-6f * mag);
}

// Threads per block of the compositing kernels (each warp works alone).
constexpr int kRenderThreads = 128;

// Blocks per SM asked of the register allocator, per pixels per thread:
// 64 registers a thread up to two pixels, 80 for four (102 for the backward,
// whose packed gradient state spills at 80; five blocks of four warps measured
// 1.5 % faster than four), 128 for eight.
#ifndef GS_BWD_BLOCKS_PPT4
#define GS_BWD_BLOCKS_PPT4 5
#endif
// With TMA staging or asynchronous copies the next chunk waits in shared
// memory, not registers, and four pixels a thread would fit six blocks per SM
// at 80 registers; but the interleaved bodies of a thread's two pixel pairs
// want more: five blocks (95 registers) measured 3 % faster than six, four
// (110 registers) 3.5 % slower than five.
#ifndef GS_BWD_BLOCKS_PPT4_TMA
#define GS_BWD_BLOCKS_PPT4_TMA 5
#endif
// Eight pixels a thread (upstream gradients in shared memory): about 120
// registers; at 96 (five blocks) the compiler needs 20 % more instructions.
#ifndef GS_BWD_BLOCKS_PPT8
#define GS_BWD_BLOCKS_PPT8 4
#endif
// Forward, up to two pixels a thread, asynchronous-copy staging: nine blocks
// (56 registers) measured 0.8 % faster than eight (64 registers) and 2.3 %
// faster than ten (47 registers).
#ifndef GS_FWD_BLOCKS_PPT2_ASYNC
#define GS_FWD_BLOCKS_PPT2_ASYNC 9
#endif
template <int PPT, bool TMA = false>
struct RenderOccupancy {
    static constexpr int fwd = PPT <= 2 ? 8 : PPT == 4 ? (TMA ? 7 : 6) : 4;
    // forward with asynchronous copies (no prefetch registers)
    static constexpr int fwd_async = PPT <= 2 ? GS_FWD_BLOCKS_PPT2_ASYNC : PPT == 4 ? 7 : 4;
    static constexpr int bwd = PPT <= 2 ? 8 : PPT == 4 ? (TMA ? GS_BWD_BLOCKS_PPT4_TMA : GS_BWD_BLOCKS_PPT4)
                                                         : GS_BWD_BLOCKS_PPT8;
};

// Kernel variants the autotuner picks from: a band shape as (pixels per
// thread, band width) (1, 8) (2, 8) (2, 16) (4, 8) (4, 16) (8, 16), each with a
// staged chunk of 32 list entries loaded by the lanes into registers (variants
// 0-5), of 32 copied by the lanes' asynchronous copies into a second
// shared-memory buffer (6-11), or of 32 (12-17) or 64 (18-23) gathered by the
// tensor memory accelerator.  A warp's band is BW x PPT * 32 / BW pixels; a thread's pixels
// share a column, 32 / BW rows apart.
constexpr int kBandVariants = 6;
constexpr int kFwdVariants = 4 * kBandVariants;
constexpr int kBwdVariants = 4 * kBandVariants;
inline bool variant_gathers(int var) { return var >= 2 * kBandVariants; }
constexpr int kVariantPPT[kBandVariants] = {1, 2, 2, 4, 4, 8};
constexpr int kVariantBW[kBandVariants] = {8, 8, 16, 8, 16, 16};
int render_variant_fwd();
int render_variant_bwd();

// The variant a launch uses: var when its band divides the tile of every view,
// else the (2, 8) band (8 x 8 pixels, which divides every allowed tile) with
// var's chunk size.
inline int fitting_variant(const ViewTable &vt, int var)
{
    const int base = var % kBandVariants, ch = var / kBandVariants;
    const int bw = kVariantBW[base], bh = kVariantPPT[base] * (32 / bw);
    for (int k = 0; k < vt.n_views; k++)
        if (vt.v[k].tile_w % bw || vt.v[k].tile_h % bh) return 1 + ch * kBandVariants;
    return var;
}

// Sets each view's first work item for bands of bw x bh pixels (work items
// are the bands of every tile, view by view) and returns the total.
inline uint32_t render_items(ViewTable *vt, int bw, int bh)
{
    int64_t items = 0;
    for (int k = 0; k < vt->n_views; k++) {
        ViewInfo &V = vt->v[k];
        V.item_base = (int32_t)items;
        items += (int64_t)V.tiles_x * V.tiles_y * (V.tile_w / bw) * (V.tile_h / bh);
    }
    return (uint32_t)items;
}

}  // namespace gs
