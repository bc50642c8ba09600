// Shared pieces of the forward and backward compositing kernels.
#pragma once

#include "common.cuh"

namespace gs {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

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
// so an entry costs two packed FMAs per pixel pair up to the blend test, which
// compares this logarithm with log2(1/255); the exponential is taken only
// where the entry is blended.  The forward and backward kernels go through the
// same helpers with the same explicitly rounded operations, so both take the
// same skip decisions and the same alphas bit for bit.
constexpr float kLog2e = 1.442695041f;
constexpr float kLn2 = 0.6931471806f;
constexpr float kLog2AlphaMin = -7.994353294f;  // FP32 value nearest log2(1/255), within 1e-7 relative of it

// Turns a record, as staged in shared memory for the per-pixel walk, into the
// base-2 form: p.w = log2(o), c.xyz = (A', B', C').  The mean remainders (c.w,
// col.w), depth and colour are unchanged.
__device__ __forceinline__ void stage_log2(float4 &p, float4 &c)
{
    p.w = __log2f(p.w);
    c.x = __fmul_rn(c.x, -0.5f * kLog2e);
    c.y = __fmul_rn(c.y, -kLog2e);
    c.z = __fmul_rn(c.z, -0.5f * kLog2e);
}

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
// of pixel centres [x0, x1] x [y0, y1].  With d = pixel - mean, alpha at a
// pixel is min(0.99, o exp(-q(d)/2)), q(d) = A dx^2 + 2 B dx dy + C dy^2 (the
// conic is positive definite).  q is convex with minimum 0 at the mean, so over
// a box not containing the mean its minimum lies on one of the four edges, where
// it is a one-dimensional quadratic; the box minimum bounds q at every pixel
// centre inside.  The entry is dropped when o exp(-q_min/2) is below 1/255 by a
// factor e^-(0.001 + 2e-6 M), M the magnitude of the terms of q: more than the
// FP32 rounding of this bound and of the per-pixel evaluation together, so a
// dropped entry is one the per-pixel test would have skipped: results are
// unchanged, only work is saved.  (A bound through the smallest eigenvalue of
// the conic is weaker and, for elongated splats, cancels badly in FP32.)
__device__ __forceinline__ bool splat_misses_box(const float4 &p, const float4 &c, float x0, float x1, float y0,
                                                 float y1)
{
    const float ex0 = x0 - p.x, ex1 = x1 - p.x, ey0 = y0 - p.y, ey1 = y1 - p.y;
    float q = 0.0f, mag = 0.0f;
    if (!(ex0 <= 0.0f && ex1 >= 0.0f && ey0 <= 0.0f && ey1 >= 0.0f)) {
        const float A = c.x, B = c.y, C = c.z;
        q = fminf(fminf(edge_min(A, B, C, ex0, ey0, ey1, &mag), edge_min(A, B, C, ex1, ey0, ey1, &mag)),
                  fminf(edge_min(C, B, A, ey0, ex0, ex1, &mag), edge_min(C, B, A, ey1, ex0, ex1, &mag)));
    }
    // alpha bound < (1/255) e^-margin  <=>  -q/2 < -ln(255 o) - margin
    return -0.5f * q < -__logf(255.0f * p.w) - (1e-3f + 2e-6f * mag);
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
template <int PPT>
struct RenderOccupancy {
    static constexpr int fwd = PPT <= 2 ? 8 : PPT == 4 ? 6 : 4;
    static constexpr int bwd = PPT <= 2 ? 8 : PPT == 4 ? GS_BWD_BLOCKS_PPT4 : 4;
};

// Kernel variants the autotuner picks from, as (pixels per thread, band
// width): (1, 8) (2, 8) (2, 16) (4, 8) (4, 16) (8, 16).  A warp's band is
// BW x PPT * 32 / BW pixels; a thread's pixels share a column, 32 / BW rows
// apart.
constexpr int kFwdVariants = 6;
constexpr int kBwdVariants = 6;
int render_variant_fwd();
int render_variant_bwd();

}  // namespace gs
