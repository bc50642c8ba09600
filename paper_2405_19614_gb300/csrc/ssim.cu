// SSIM term of the mapping loss (Sec. 3.4: L_m = (1 - zeta)(w4 L1(D) +
// w5 L1(C)) + zeta L_SSIM; zeta = 0.3 in Table hyper).  The paper does not
// define its SSIM; this is the usual structural similarity: per colour channel,
// local moments under an 11 x 11 Gaussian window of standard deviation 1.5
// (normalised, zero padding, same size), C1 = 0.01^2, C2 = 0.03^2,
//   s = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
// L_SSIM = weight (1 - mean s) over all pixels and channels of all views.
//
// Two kernels over 32 x 48 output tiles of all views.  The first stages the
// tile plus a 5-pixel halo of both images (all three channels, coalesced) in
// shared memory, filters the moments x, y, x^2 + y^2 and x y separably (s
// needs the two variances only through their sum) and sums s into the loss;
// per pixel and channel it writes the three partial derivatives of s with
// respect to the moments that depend on the rendered image,
//   ds/dmx = (2 my (a2 - a1) - 2 mx s (b2 - b1)) / (b1 b2),
//   ds/dE[x^2] = -s / b2,  ds/dE[xy] = 2 a1 / (b1 b2),
// as nine planar maps.  The second filters those maps with the same
// (symmetric) window and adds
//   dL/dx = g (G*ds/dmx + 2 x G*ds/dE[x^2] + y G*ds/dE[xy]),  g = -weight/(3P)
// to d_rgb.
//
// The gradient kernel stages a channel's three maps while the previous
// channel is filtered: with the tensor memory accelerator (one 4-D box per
// channel, below) where every view's width is a multiple of 4, else by
// double-buffered 4-byte asynchronous copies.  Both filters are done with
// each value read once from shared memory: the
// horizontal pass gives each thread one halo row and eight output columns
// (lanes are consecutive rows, so row pitches are odd for conflict-free
// access); the vertical pass gives each thread one column and six output rows
// and keeps the 16 input rows it needs in registers.
#include <mutex>

#include "common.cuh"
#include "async_copy.cuh"
#include "tma.cuh"

namespace gs {

constexpr int kSsimTW = 32, kSsimTH = 48, kSsimR = 5, kSsimWin = 2 * kSsimR + 1;
constexpr int kSsimRows = kSsimTH + 2 * kSsimR;  // 58 halo rows
constexpr int kSsimCols = kSsimTW + 2 * kSsimR;  // 42 halo columns
constexpr int kSsimSeg = 8;                      // output columns per thread, horizontal pass
constexpr int kSsimGrp = 6;                      // output rows per thread, vertical pass
constexpr int kSsimThreads = 256;
constexpr int kSsimInPitchXY = 3 * kSsimCols + 1;  // 127: interleaved RGB halo row
constexpr int kSsimInPitch = kSsimCols + 1;        // 43: one map's halo row
constexpr int kSsimHPitch = kSsimTW + 1;           // 33: horizontally filtered row
constexpr int kSsimOutPitch = 3 * kSsimTW + 1;     // 97: interleaved RGB output row
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;

static_assert(kSsimTW == 4 * kSsimSeg, "four column segments per halo row");
static_assert(kSsimRows <= 64, "two 32-row groups cover the halo rows");
static_assert(kSsimTH == 8 * kSsimGrp, "eight warps of row groups cover the tile");
static_assert(kSsimSeg % 2 == 0 && kSsimGrp % 2 == 0, "outputs are filtered in pairs");

constexpr size_t kSsimStatsSmem =
    sizeof(float) * (2 * kSsimRows * kSsimInPitchXY + 4 * kSsimRows * kSsimHPitch);
constexpr size_t kSsimGradSmem =
    sizeof(float) * (2 * 3 * kSsimRows * kSsimInPitch + 3 * kSsimRows * kSsimHPitch + kSsimTH * kSsimOutPitch);

struct SsimTiles {
    int32_t n_views;
    int32_t base[GS_MAX_VIEWS + 1];  // first tile of each view, running sum
    int32_t tiles_x[GS_MAX_VIEWS];
    int32_t width[GS_MAX_VIEWS], height[GS_MAX_VIEWS];
    int64_t pix_base[GS_MAX_VIEWS];
    int64_t n_pix;
    float g[kSsimWin];
    // gp[t] = (g[t], g[t - 1]) for t = 0 .. 11, zero outside the window: the
    // weights of two neighbouring outputs for one input, for packed FMAs
    float2 gp[kSsimWin + 1];
};

__device__ __forceinline__ void ssim_tile_of(const SsimTiles &T, int item, int *v, int *x0, int *y0)
{
    int vv = 0;
    #pragma unroll 1
    for (int k = 1; k < T.n_views; k++)
        if (item >= T.base[k]) vv = k;
    const int lt = item - T.base[vv];
    *v = vv;
    *x0 = (lt % T.tiles_x[vv]) * kSsimTW;
    *y0 = (lt / T.tiles_x[vv]) * kSsimTH;
}

// Both passes accumulate two neighbouring outputs (o, o + 1) per packed
// FP32x2 FMA: output o takes g[t] and output o + 1 takes g[t - 1] from input
// o + t, i.e. the weight pair gp[t].  Each output still sums its inputs in
// ascending order with single-rounded FMAs, exactly as one FMA at a time.

// Horizontal pass for NM maps: acc[p][m] = (out(2p), out(2p + 1)) with
// out(o) = sum_t g[t] f_m(column o + t), for the eight output columns of this
// thread's segment; load(i, f) gives the NM map values at the segment's halo
// column i = 0..17 of this thread's row.
template <int NM, typename Load>
__device__ __forceinline__ void ssim_hpass(const SsimTiles &T, Load load, float2 (&acc)[kSsimSeg / 2][NM])
{
    float2 w[kSsimWin + 1];  // weight pairs held in registers for the packed FMAs
    #pragma unroll
    for (int t = 0; t <= kSsimWin; t++) w[t] = T.gp[t];
    #pragma unroll
    for (int p = 0; p < kSsimSeg / 2; p++)
        #pragma unroll
        for (int m = 0; m < NM; m++) acc[p][m] = make_float2(0.0f, 0.0f);
    #pragma unroll
    for (int i = 0; i < kSsimSeg + kSsimWin - 1; i++) {
        float f[NM];
        load(i, f);
        #pragma unroll
        for (int p = 0; p < kSsimSeg / 2; p++) {
            const int t = i - 2 * p;
            if (t < 0 || t > kSsimWin) continue;
            #pragma unroll
            for (int m = 0; m < NM; m++) acc[p][m] = __ffma2_rn(w[t], make_float2(f[m], f[m]), acc[p][m]);
        }
    }
}

// Vertical pass for NM maps: thread column c, output rows r0 .. r0+5 (as pairs
// out[p] = rows (2p, 2p + 1)) from filtered rows r0 .. r0+15 of h[m][row][c].
template <int NM>
__device__ __forceinline__ void ssim_vpass(const SsimTiles &T, const float *h, int c, int r0,
                                           float2 (&out)[kSsimGrp / 2][NM])
{
    float2 w[kSsimWin + 1];
    #pragma unroll
    for (int t = 0; t <= kSsimWin; t++) w[t] = T.gp[t];
    #pragma unroll
    for (int p = 0; p < kSsimGrp / 2; p++)
        #pragma unroll
        for (int m = 0; m < NM; m++) out[p][m] = make_float2(0.0f, 0.0f);
    #pragma unroll
    for (int i = 0; i < kSsimGrp + kSsimWin - 1; i++) {
        float f[NM];
        #pragma unroll
        for (int m = 0; m < NM; m++) f[m] = h[(m * kSsimRows + r0 + i) * kSsimHPitch + c];
        #pragma unroll
        for (int p = 0; p < kSsimGrp / 2; p++) {
            const int t = i - 2 * p;
            if (t < 0 || t > kSsimWin) continue;
            #pragma unroll
            for (int m = 0; m < NM; m++) out[p][m] = __ffma2_rn(w[t], make_float2(f[m], f[m]), out[p][m]);
        }
    }
}

// Gradient kernels, end of a channel: the vertical pass of the three filtered
// maps and dL/dx = G*ds/dmx + 2 x G*ds/dE[x^2] + y G*ds/dE[xy] into s_out.
__device__ __forceinline__ void ssim_grad_channel_out(const SsimTiles &T, const float *s_h, float *s_out, int vc,
                                                      int vr0, int ch, const float (&xs)[kSsimGrp],
                                                      const float (&ys)[kSsimGrp])
{
    float2 fp[kSsimGrp / 2][3];
    ssim_vpass<3>(T, s_h, vc, vr0, fp);
    #pragma unroll
    for (int o = 0; o < kSsimGrp; o++) {
        float f[3];
        #pragma unroll
        for (int m = 0; m < 3; m++) f[m] = (o & 1) ? fp[o >> 1][m].y : fp[o >> 1][m].x;
        s_out[(vr0 + o) * kSsimOutPitch + 3 * vc + ch] = f[0] + 2.f * xs[o] * f[1] + ys[o] * f[2];
    }
}

// Gradient kernels, end of the tile: d_rgb += gsc * s_out.  The tile's rows of
// d_rgb are contiguous runs of 3 * 32 floats; all reads are issued before the
// writes.
__device__ __forceinline__ void ssim_grad_write(const float *s_out, float *__restrict__ d_rgb, float gsc, int tid,
                                                int x0, int y0, int W, int H, int64_t pb)
{
    constexpr int kPer = kSsimTH * 3 * kSsimTW / kSsimThreads;
    static_assert(kPer * kSsimThreads == kSsimTH * 3 * kSsimTW, "whole rounds");
    int64_t idx[kPer];
    float cur[kPer];
    #pragma unroll
    for (int i = 0; i < kPer; i++) {
        const int e = tid + i * kSsimThreads;
        const int r = e / (3 * kSsimTW), q = e - r * (3 * kSsimTW);
        const int gy = y0 + r, gx = x0 + q / 3;
        idx[i] = (gx < W && gy < H) ? 3 * (pb + (int64_t)gy * W + x0) + q : -1;
        cur[i] = idx[i] >= 0 ? d_rgb[idx[i]] : 0.0f;
    }
    #pragma unroll
    for (int i = 0; i < kPer; i++) {
        const int e = tid + i * kSsimThreads;
        const int r = e / (3 * kSsimTW), q = e - r * (3 * kSsimTW);
        if (idx[i] >= 0) d_rgb[idx[i]] = cur[i] + gsc * s_out[r * kSsimOutPitch + q];
    }
}

__global__ void __launch_bounds__(kSsimThreads) ssim_stats_kernel(const float *__restrict__ x,
                                                                  const float *__restrict__ y, SsimTiles T,
                                                                  float *__restrict__ partial, float *loss,
                                                                  float scale, float constant)
{
    extern __shared__ float smem[];
    float *s_in = smem;                                   // [2][rows][127]: x, y halo, RGB interleaved
    float *s_h = smem + 2 * kSsimRows * kSsimInPitchXY;  // [4][rows][33]
    __shared__ float red[kSsimThreads / 32];
    int v, x0, y0;
    ssim_tile_of(T, blockIdx.x, &v, &x0, &y0);
    const int W = T.width[v], H = T.height[v];
    const int64_t pb = T.pix_base[v];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // stage: halo rows of 42 pixels x 3 channels (126 floats) are contiguous
    // in both images; a warp copies whole rows and a lane the same four
    // positions of every row, whose column bounds are tested once; every copy
    // is in flight at once
    constexpr int kRowFloats = 3 * kSsimCols;
    bool col_in[4];
    #pragma unroll
    for (int j = 0; j < 4; j++) {
        const int q = lane + 32 * j, gx = x0 - kSsimR + q / 3;
        col_in[j] = q < kRowFloats && gx >= 0 && gx < W;
    }
    for (int r = warp; r < kSsimRows; r += kSsimThreads / 32) {
        const int gy = y0 - kSsimR + r;
        const bool row_in = gy >= 0 && gy < H;
        const int64_t row = 3 * (pb + (int64_t)(row_in ? gy : 0) * W + (x0 - kSsimR));
        #pragma unroll
        for (int j = 0; j < 4; j++) {
            const int q = lane + 32 * j;
            if (q < kRowFloats) {
                const bool in = row_in && col_in[j];
                const int64_t idx = in ? row + q : 0;
                cp_async4(s_in + r * kSsimInPitchXY + q, x + idx, in);
                cp_async4(s_in + (kSsimRows + r) * kSsimInPitchXY + q, y + idx, in);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    float acc_s = 0.0f;
    const int hrow = (warp >> 2) * 32 + lane, hseg = warp & 3;  // horizontal pass: row, column segment
    const int vc = lane, vr0 = warp * kSsimGrp;                // vertical pass: column, first output row
    for (int ch = 0; ch < 3; ch++) {
        if (hrow < kSsimRows) {
            const float *rx = s_in + hrow * kSsimInPitchXY + 3 * hseg * kSsimSeg + ch;
            const float *ry = rx + kSsimRows * kSsimInPitchXY;
            // s needs the two variances only through their sum, so four maps do:
            // x, y, x^2 + y^2 and x y
            float2 acc[kSsimSeg / 2][4];
            ssim_hpass<4>(T, [&](int i, float (&f)[4]) {
                const float a = rx[3 * i], b = ry[3 * i];
                f[0] = a;
                f[1] = b;
                f[2] = fmaf(a, a, b * b);
                f[3] = a * b;
            }, acc);
            #pragma unroll
            for (int p = 0; p < kSsimSeg / 2; p++)
                #pragma unroll
                for (int m = 0; m < 4; m++) {
                    float *dst = s_h + (m * kSsimRows + hrow) * kSsimHPitch + hseg * kSsimSeg + 2 * p;
                    dst[0] = acc[p][m].x;
                    dst[1] = acc[p][m].y;
                }
        }
        __syncthreads();
        float2 mp[kSsimGrp / 2][4];
        ssim_vpass<4>(T, s_h, vc, vr0, mp);
        const int gx = x0 + vc;
        #pragma unroll
        for (int o = 0; o < kSsimGrp; o++) {
            const int gy = y0 + vr0 + o;
            if (gx >= W || gy >= H) continue;
            float mo[4];
            #pragma unroll
            for (int m = 0; m < 4; m++) mo[m] = (o & 1) ? mp[o >> 1][m].y : mp[o >> 1][m].x;
            const float mx = mo[0], my = mo[1];
            const float m2 = mx * mx + my * my, sxy = mo[3] - mx * my;
            const float a1 = 2.f * mx * my + kSsimC1, a2 = 2.f * sxy + kSsimC2;
            const float b1 = m2 + kSsimC1, b2 = (mo[2] - m2) + kSsimC2;
            const float ib = __fdividef(1.0f, b1 * b2);  // b1 b2 >= C1 C2: in the fast quotient's range
            const float s = a1 * a2 * ib;
            acc_s += s;
            const int64_t p = pb + (int64_t)gy * W + gx;
            float *pl = partial + (int64_t)(3 * ch) * T.n_pix + p;
            pl[0] = (2.f * my * (a2 - a1) - 2.f * mx * s * (b2 - b1)) * ib;
            pl[T.n_pix] = -s * b1 * ib;
            pl[2 * T.n_pix] = 2.f * a1 * ib;
        }
        __syncthreads();
    }
    acc_s = warp_sum(acc_s);
    if (lane == 0) red[warp] = acc_s;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int w = 0; w < kSsimThreads / 32; w++) s += red[w];
        atomicAdd(loss, scale * s + (blockIdx.x == 0 ? constant : 0.0f));
    }
}

__global__ void __launch_bounds__(kSsimThreads) ssim_grad_kernel(const float *__restrict__ x,
                                                                 const float *__restrict__ y, SsimTiles T,
                                                                 const float *__restrict__ partial,
                                                                 float *__restrict__ d_rgb, float gsc)
{
    extern __shared__ float smem[];
    constexpr int kBuf = 3 * kSsimRows * kSsimInPitch;
    float *s_in = smem;                                 // [2][3][rows][43]: a channel's three maps, double-buffered
    float *s_h = smem + 2 * kBuf;                       // [3][rows][33]
    float *s_out = s_h + 3 * kSsimRows * kSsimHPitch;  // [48][97]: dL/dx, RGB interleaved
    int v, x0, y0;
    ssim_tile_of(T, blockIdx.x, &v, &x0, &y0);
    const int W = T.width[v], H = T.height[v];
    const int64_t pb = T.pix_base[v];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int hrow = (warp >> 2) * 32 + lane, hseg = warp & 3;
    const int vc = lane, vr0 = warp * kSsimGrp;
    // copies of channel ch's three maps (halo included) into buffer ch & 1: a
    // warp copies whole halo rows of 42 values, a lane the same two columns of
    // every row (bounds tested once)
    bool col_in[2];
    #pragma unroll
    for (int j = 0; j < 2; j++) {
        const int c = lane + 32 * j, gx = x0 - kSsimR + c;
        col_in[j] = c < kSsimCols && gx >= 0 && gx < W;
    }
    auto stage = [&](int ch) {
        float *dst = s_in + (ch & 1) * kBuf;
        for (int mr = warp; mr < 3 * kSsimRows; mr += kSsimThreads / 32) {
            const int m = mr / kSsimRows, r = mr - m * kSsimRows;
            const int gy = y0 - kSsimR + r;
            const bool row_in = gy >= 0 && gy < H;
            const int64_t row = (int64_t)(3 * ch + m) * T.n_pix + pb + (int64_t)(row_in ? gy : 0) * W + (x0 - kSsimR);
            #pragma unroll
            for (int j = 0; j < 2; j++) {
                const int c = lane + 32 * j;
                if (c < kSsimCols) {
                    const bool in = row_in && col_in[j];
                    cp_async4(dst + (m * kSsimRows + r) * kSsimInPitch + c, partial + (in ? row + c : 0), in);
                }
            }
        }
        cp_async_commit();
    };
    stage(0);
    for (int ch = 0; ch < 3; ch++) {
        if (ch < 2) {
            stage(ch + 1);  // in flight while this channel is filtered
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // this channel's image values for the output pixels, loaded ahead of the filtering
        const int gx = x0 + vc;
        float xs[kSsimGrp], ys[kSsimGrp];
        #pragma unroll
        for (int o = 0; o < kSsimGrp; o++) {
            const int gy = y0 + vr0 + o;
            xs[o] = ys[o] = 0.0f;
            if (gx < W && gy < H) {
                const int64_t p = pb + (int64_t)gy * W + gx;
                xs[o] = x[3 * p + ch];
                ys[o] = y[3 * p + ch];
            }
        }
        if (hrow < kSsimRows) {
            const float *r0 = s_in + (ch & 1) * kBuf + hrow * kSsimInPitch + hseg * kSsimSeg;
            float2 acc[kSsimSeg / 2][3];
            ssim_hpass<3>(T, [&](int i, float (&f)[3]) {
                f[0] = r0[i];
                f[1] = r0[kSsimRows * kSsimInPitch + i];
                f[2] = r0[2 * kSsimRows * kSsimInPitch + i];
            }, acc);
            #pragma unroll
            for (int p = 0; p < kSsimSeg / 2; p++)
                #pragma unroll
                for (int m = 0; m < 3; m++) {
                    float *dst = s_h + (m * kSsimRows + hrow) * kSsimHPitch + hseg * kSsimSeg + 2 * p;
                    dst[0] = acc[p][m].x;
                    dst[1] = acc[p][m].y;
                }
        }
        __syncthreads();
        ssim_grad_channel_out(T, s_h, s_out, vc, vr0, ch, xs, ys);
        __syncthreads();
    }
    ssim_grad_write(s_out, d_rgb, gsc, tid, x0, y0, W, H, pb);
}

// TMA staging of the gradient kernel: a view's nine partial maps are one 4-D
// tensor (4 floats, W / 4 groups of 4, H rows, 9 maps), and a channel's three
// maps over the tile and its halo are one box of 13 groups (image columns
// x0 - 8 .. x0 + 43, of which x0 - 5 .. x0 + 36 are used) x 58 rows x 3 maps.
// It lands in shared memory with a row pitch of 52 floats, 13 16-byte groups:
// in the horizontal pass a lane reads its row 16 bytes at a time, and the
// eight rows of each quarter-warp then fall on eight different bank groups.
// Rows and columns outside the view read as zero: the window's zero padding.
constexpr int kSsimTmaGroups = 13;
constexpr int kSsimTmaPitch = 4 * kSsimTmaGroups;  // 52 floats
constexpr int kSsimTmaLead = 8;                    // staged columns left of the tile (x0 - 8: 16-byte aligned)
constexpr uint32_t kSsimTmaBytes = sizeof(float) * 3 * kSsimRows * kSsimTmaPitch;
constexpr size_t kSsimGradTmaSmem = kSsimTmaBytes + sizeof(float) * 3 * kSsimRows * kSsimHPitch;
static_assert(kSsimTmaPitch >= kSsimTmaLead + kSsimTW + kSsimR, "a staged row covers the window");
static_assert(kSsimTW % 4 == 0 && kSsimTmaLead % 4 == 0 && kSsimSeg % 4 == 0, "16-byte aligned groups");

struct SsimMaps {
    CUtensorMap m[GS_MAX_VIEWS];
};

// Its outputs stay in registers (a thread's six pixels of one column, all
// three channels) instead of a shared-memory tile: 59 KB of shared memory a
// block, three blocks per SM (80 registers, a few bytes of spill; two blocks
// at 93 registers without spill measured 0.6 % slower).
#ifndef GS_SSIM_GRAD_TMA_BLOCKS
#define GS_SSIM_GRAD_TMA_BLOCKS 3
#endif
__global__ void __launch_bounds__(kSsimThreads, GS_SSIM_GRAD_TMA_BLOCKS) ssim_grad_tma_kernel(const float *__restrict__ x,
                                                                     const float *__restrict__ y, SsimTiles T,
                                                                     const __grid_constant__ SsimMaps maps,
                                                                     float *__restrict__ d_rgb, float gsc,
                                                                     uint32_t *status, uint32_t extra_tx)
{
    extern __shared__ __align__(128) float smem[];
    float *s_in = smem;                                 // [3][rows][52]: a channel's three maps (TMA box)
    float *s_h = smem + 3 * kSsimRows * kSsimTmaPitch;  // [3][rows][33]
    __shared__ alignas(8) uint64_t s_bar;
    int v, x0, y0;
    ssim_tile_of(T, blockIdx.x, &v, &x0, &y0);
    const int W = T.width[v], H = T.height[v];
    const int64_t pb = T.pix_base[v];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int hrow = (warp >> 2) * 32 + lane, hseg = warp & 3;
    const int vc = lane, vr0 = warp * kSsimGrp;
    const CUtensorMap *map = &maps.m[v];
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // channel ch's box into s_in, by one thread, after every earlier read of
    // s_in (extra_tx > 0 makes the barrier wait for bytes that never come)
    auto issue = [&](int ch) {
        if (tid == 0) {
            fence_proxy_async_shared();
            mbar_arrive_expect_tx(&s_bar, kSsimTmaBytes + extra_tx);  // extra_tx: 0 but in the timeout check
            tma_load_4d(s_in, map, 0, (x0 - kSsimTmaLead) / 4, y0 - kSsimR, 3 * ch, &s_bar);
        }
    };
    issue(0);
    uint32_t parity = 0;
    const int gx = x0 + vc;
    float g_out[kSsimGrp][3];  // dL/dx of the thread's pixels, per channel
    for (int ch = 0; ch < 3; ch++) {
        // this channel's image values for the output pixels, loaded ahead of the filtering
        float xs[kSsimGrp], ys[kSsimGrp];
        #pragma unroll
        for (int o = 0; o < kSsimGrp; o++) {
            const int gy = y0 + vr0 + o;
            xs[o] = ys[o] = 0.0f;
            if (gx < W && gy < H) {
                const int64_t p = pb + (int64_t)gy * W + gx;
                xs[o] = x[3 * p + ch];
                ys[o] = y[3 * p + ch];
            }
        }
        const bool ok = mbar_wait_parity(&s_bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            // the box never arrived: report it, give the copy one more bounded
            // wait (it must not land in a later block's shared memory), stop
            if (tid == 0) raise_status(status, GS_ERR_TIMEOUT);
            mbar_wait_parity(&s_bar, parity ^ 1u);
            return;
        }
        if (hrow < kSsimRows) {
            // staged column j holds image column x0 - 8 + j; halo column i of
            // this segment (image column x0 - 5 + 8 hseg + i) is j = 3 + i
            const float *r0 = s_in + hrow * kSsimTmaPitch + hseg * kSsimSeg;
            float2 acc[kSsimSeg / 2][3];
            ssim_hpass<3>(T, [&](int i, float (&f)[3]) {
                const int j = kSsimTmaLead - kSsimR + i;
                #pragma unroll
                for (int m = 0; m < 3; m++) {
                    const float4 q =
                        *reinterpret_cast<const float4 *>(r0 + m * kSsimRows * kSsimTmaPitch + (j & ~3));
                    f[m] = (j & 3) == 0 ? q.x : (j & 3) == 1 ? q.y : (j & 3) == 2 ? q.z : q.w;
                }
            }, acc);
            #pragma unroll
            for (int p = 0; p < kSsimSeg / 2; p++)
                #pragma unroll
                for (int m = 0; m < 3; m++) {
                    float *dst = s_h + (m * kSsimRows + hrow) * kSsimHPitch + hseg * kSsimSeg + 2 * p;
                    dst[0] = acc[p][m].x;
                    dst[1] = acc[p][m].y;
                }
        }
        __syncthreads();
        if (ch < 2) issue(ch + 1);  // in flight while this channel is finished
        float2 fp[kSsimGrp / 2][3];
        ssim_vpass<3>(T, s_h, vc, vr0, fp);
        #pragma unroll
        for (int o = 0; o < kSsimGrp; o++) {
            float f[3];
            #pragma unroll
            for (int m = 0; m < 3; m++) f[m] = (o & 1) ? fp[o >> 1][m].y : fp[o >> 1][m].x;
            #pragma unroll
            for (int c = 0; c < 3; c++)
                if (c == ch) g_out[o][c] = f[0] + 2.f * xs[o] * f[1] + ys[o] * f[2];
        }
        __syncthreads();  // s_h is read before the next channel's horizontal pass writes it
    }
    // d_rgb += gsc * dL/dx: a warp's pixels of one row are 32 consecutive RGB
    // triples; all reads are issued before the writes
    float cur[kSsimGrp][3];
    #pragma unroll
    for (int o = 0; o < kSsimGrp; o++) {
        const int gy = y0 + vr0 + o;
        #pragma unroll
        for (int c = 0; c < 3; c++) cur[o][c] = 0.0f;
        if (gx < W && gy < H) {
            const int64_t p = pb + (int64_t)gy * W + gx;
            #pragma unroll
            for (int c = 0; c < 3; c++) cur[o][c] = d_rgb[3 * p + c];
        }
    }
    #pragma unroll
    for (int o = 0; o < kSsimGrp; o++) {
        const int gy = y0 + vr0 + o;
        if (gx < W && gy < H) {
            const int64_t p = pb + (int64_t)gy * W + gx;
            #pragma unroll
            for (int c = 0; c < 3; c++) d_rgb[3 * p + c] = cur[o][c] + gsc * g_out[o][c];
        }
    }
}

static gs_status_t make_ssim_tiles(const gs_view_t *views, int32_t n_views, SsimTiles *T)
{
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    T->n_views = n_views;
    int64_t tiles = 0;
    for (int v = 0; v < n_views; v++) {
        T->base[v] = (int32_t)tiles;
        T->tiles_x[v] = (views[v].width + kSsimTW - 1) / kSsimTW;
        T->width[v] = views[v].width;
        T->height[v] = views[v].height;
        T->pix_base[v] = vt.v[v].pix_base;
        tiles += (int64_t)T->tiles_x[v] * ((views[v].height + kSsimTH - 1) / kSsimTH);
    }
    if (tiles >= (int64_t(1) << 31)) return GS_ERR_INVALID_ARG;
    T->base[n_views] = (int32_t)tiles;
    T->n_pix = vt.n_pix_total;
    // window: exp(-i^2 / (2 * 1.5^2)), i = -5..5, normalised to sum 1
    double g[kSsimWin], sum = 0.0;
    for (int i = 0; i < kSsimWin; i++) {
        const double d = i - kSsimR;
        g[i] = exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[i];
    }
    for (int i = 0; i < kSsimWin; i++) T->g[i] = (float)(g[i] / sum);
    for (int t = 0; t <= kSsimWin; t++)
        T->gp[t] = make_float2(t < kSsimWin ? T->g[t] : 0.0f, t >= 1 ? T->g[t - 1] : 0.0f);
    return GS_OK;
}

// Both kernels take more than 48 KB of dynamic shared memory, which has to be
// allowed once per device.
static gs_status_t ssim_set_smem_limits()
{
    static std::mutex mu;
    static bool done[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return GS_OK;
    if (cudaFuncSetAttribute(ssim_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsimStatsSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(ssim_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsimGradSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(ssim_grad_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSsimGradTmaSmem) != cudaSuccess)
        return GS_ERR_CUDA;
    done[dev] = true;
    return GS_OK;
}

// The per-view tensor maps of the partial maps at `partial` ([9][n_pix]
// floats), or false when a view's rows are not 16-byte aligned (its width or
// first pixel not a multiple of 4) or a map cannot be made.
static bool make_ssim_maps(const SsimTiles &T, const float *partial, SsimMaps *maps)
{
    if (T.n_pix % 4 || (reinterpret_cast<uintptr_t>(partial) & 15)) return false;
    for (int v = 0; v < T.n_views; v++) {
        if (T.width[v] % 4 || T.pix_base[v] % 4) return false;
        const uint64_t dims[4] = {4, (uint64_t)T.width[v] / 4, (uint64_t)T.height[v], 9};
        const uint64_t strides[3] = {16, 4 * (uint64_t)T.width[v], 4 * (uint64_t)T.n_pix};
        const uint32_t box[4] = {4, kSsimTmaGroups, kSsimRows, 3};
        if (make_tensor_map_4d(partial + T.pix_base[v], dims, strides, box, &maps->m[v]) != GS_OK) return false;
    }
    return true;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_ssim_workspace_size(int64_t n_pixels)
{
    return n_pixels < 0 ? 0 : sizeof(float) * 9 * (size_t)n_pixels;
}

// Both passes; extra_tx > 0 (the timeout check) requires the staged pass.
static gs_status_t ssim_launch(const float *rgb, const float *target_rgb, const gs_view_t *views, int32_t n_views,
                               float weight, float *loss, float *d_rgb, void *workspace, size_t workspace_bytes,
                               uint32_t *status, uint32_t extra_tx, void *stream)
{
    if (!rgb || !target_rgb || !loss || !d_rgb || !workspace) return GS_ERR_INVALID_ARG;
    SsimTiles T;
    gs_status_t st = make_ssim_tiles(views, n_views, &T);
    if (st != GS_OK) return st;
    const int64_t P = T.n_pix;
    if (workspace_bytes < gs_ssim_workspace_size(P)) return GS_ERR_INVALID_ARG;
    if (ssim_set_smem_limits() != GS_OK) return GS_ERR_CUDA;
    cudaStream_t s = as_stream(stream);
    const int blocks = T.base[n_views];
    float *partial = static_cast<float *>(workspace);
    const float scale = (float)(-(double)weight / (3.0 * (double)P));
    // weight * (1 - mean s): block 0 adds the constant weight, every block -weight/(3P) times its sum of s
    ssim_stats_kernel<<<blocks, kSsimThreads, kSsimStatsSmem, s>>>(rgb, target_rgb, T, partial, loss, scale, weight);
    static SsimMaps maps;  // 8 KB: static, not on the stack; copied into the launch's parameters
    static std::mutex maps_mu;
    std::lock_guard<std::mutex> lock(maps_mu);
    if (make_ssim_maps(T, partial, &maps))
        ssim_grad_tma_kernel<<<blocks, kSsimThreads, kSsimGradTmaSmem, s>>>(rgb, target_rgb, T, maps, d_rgb, scale,
                                                                            status, extra_tx);
    else if (extra_tx == 0)
        ssim_grad_kernel<<<blocks, kSsimThreads, kSsimGradSmem, s>>>(rgb, target_rgb, T, partial, d_rgb, scale);
    else
        return GS_ERR_UNSUPPORTED;
    return launch_status();
}

extern "C" gs_status_t gs_loss_ssim(const float *rgb, const float *target_rgb, const gs_view_t *views,
                                    int32_t n_views, float weight, float *loss, float *d_rgb, void *workspace,
                                    size_t workspace_bytes, uint32_t *status, void *stream)
{
    return ssim_launch(rgb, target_rgb, views, n_views, weight, loss, d_rgb, workspace, workspace_bytes, status, 0,
                       stream);
}

extern "C" gs_status_t gs_check_ssim_timeout(const float *rgb, const float *target_rgb, const gs_view_t *views,
                                             int32_t n_views, float *loss, float *d_rgb, void *workspace,
                                             size_t workspace_bytes, uint32_t *status, void *stream)
{
    if (!status) return GS_ERR_INVALID_ARG;
    return ssim_launch(rgb, target_rgb, views, n_views, 1.0f, loss, d_rgb, workspace, workspace_bytes, status, 16,
                       stream);
}
