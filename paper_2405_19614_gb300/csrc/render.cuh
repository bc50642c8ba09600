// Shared pieces of the forward and backward compositing kernels.
#pragma once

#include "common.cuh"

namespace gs {

// alpha_i = min(0.99, o_i exp(power_i)) at the pixel centre (sx, sy).  The
// forward and backward kernels both go through splat_power and this exact
// expression, so they take the same skip decisions bit for bit.
__device__ __forceinline__ float splat_alpha(const float4 &p, const float4 &c, float sx, float sy)
{
    float dx, dy;
    const float power = splat_power(p.x, p.y, c.x, c.y, c.z, sx, sy, &dx, &dy);
    return fminf(kAlphaMax, __fmul_rn(p.w, __expf(power)));
}

// Conservative test that a splat cannot reach alpha >= 1/255 anywhere in a box
// of pixel centres [x0, x1] x [y0, y1]: for every sample s in the box,
//   power(s) = -1/2 (s - mu)^T Q (s - mu) <= -1/2 lambda_min(Q) dist(mu, box)^2,
// so alpha <= o exp(-1/2 lambda_min dist^2).  The entry is dropped when that
// bound is below 1/255 by a factor e^-0.001, a margin far larger than the FP32
// rounding of the per-pixel evaluation, so a dropped entry is one the per-pixel
// test would have skipped: results are unchanged, only work is saved.
__device__ __forceinline__ bool splat_misses_box(const float4 &p, const float4 &c, float x0, float x1, float y0,
                                                 float y1)
{
    const float dx = fmaxf(fmaxf(x0 - p.x, p.x - x1), 0.0f);
    const float dy = fmaxf(fmaxf(y0 - p.y, p.y - y1), 0.0f);
    const float h = 0.5f * (c.x - c.z);
    const float lmin = fmaxf(0.5f * (c.x + c.z) - sqrtf(h * h + c.y * c.y), 0.0f);
    // alpha bound < (1/255) e^-0.001  <=>  -1/2 lmin d^2 < -ln(255 o) - 0.001
    return -0.5f * lmin * (dx * dx + dy * dy) < -__logf(255.0f * p.w) - 1e-3f;
}

// Kernel variants (pixels per thread x staged batch) the autotuner picks from.
constexpr int kFwdVariants = 6;  // (1,256) (2,128) (2,256) (4,64) (4,128) (8,64)
constexpr int kBwdVariants = 5;  // (1,256) (2,128) (4,64) (4,128) (8,64)
int render_variant_fwd();
int render_variant_bwd();

// Sums ten values over the 32 lanes of a warp by recursive halving: at each
// step a lane keeps half of its values, sends the other half to the partner
// lane and adds what the partner sent (12 shuffles in all).  On return lane L
// holds the warp total of value index reduce10_index(L), valid where
// reduce10_valid(L).
__device__ __forceinline__ float warp_reduce_scatter10(const float (&g)[10], int lane)
{
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
    float a5[5], a3[3], a2[2];
    #pragma unroll
    for (int i = 0; i < 5; i++) {
        const float lo = g[i], hi = g[i + 5];
        a5[i] = (u16 ? hi : lo) + __shfl_xor_sync(kFullMask, u16 ? lo : hi, 16);
    }
    #pragma unroll
    for (int i = 0; i < 3; i++) {
        const float lo = a5[i], hi = (i + 3 < 5) ? a5[i + 3] : 0.0f;
        a3[i] = (u8 ? hi : lo) + __shfl_xor_sync(kFullMask, u8 ? lo : hi, 8);
    }
    #pragma unroll
    for (int i = 0; i < 2; i++) {
        const float lo = a3[i], hi = (i + 2 < 3) ? a3[i + 2] : 0.0f;
        a2[i] = (u4 ? hi : lo) + __shfl_xor_sync(kFullMask, u4 ? lo : hi, 4);
    }
    float a1 = (u2 ? a2[1] : a2[0]) + __shfl_xor_sync(kFullMask, u2 ? a2[0] : a2[1], 2);
    return a1 + __shfl_xor_sync(kFullMask, a1, 1);
}

__host__ __device__ __forceinline__ void reduce10_slot(int lane, int *index, bool *valid)
{
    int base = 0, cnt = 10;
    const int H[4] = {5, 3, 2, 1};
    const int bit[4] = {16, 8, 4, 2};
    #pragma unroll
    for (int s = 0; s < 4; s++) {
        if (lane & bit[s]) {
            base += H[s];
            cnt = cnt - H[s] > 0 ? cnt - H[s] : 0;
        } else {
            cnt = cnt < H[s] ? cnt : H[s];
        }
    }
    *index = base;
    *valid = cnt >= 1 && (lane & 1) == 0;
}

}  // namespace gs
