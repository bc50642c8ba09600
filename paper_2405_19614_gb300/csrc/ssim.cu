// SSIM term of the mapping loss (Sec. 3.4: L_m = (1 - zeta)(w4 L1(D) +
// w5 L1(C)) + zeta L_SSIM; zeta = 0.3 in Table hyper).  The paper does not
// define its SSIM; this is the usual structural similarity: per colour channel,
// local moments under an 11 x 11 Gaussian window of standard deviation 1.5
// (normalised, zero padding, same size), C1 = 0.01^2, C2 = 0.03^2,
//   s = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
// L_SSIM = weight (1 - mean s) over all pixels and channels of all views.
//
// Two kernels over 32 x 16 output tiles of all views.  The first stages each
// tile plus a 5-pixel halo in shared memory, filters the five moments
// separably (rows, then columns), sums s into the loss and writes, per pixel
// and channel, the three partial derivatives of s with respect to the moments
// that depend on the rendered image:
//   ds/dmx = (2 my (a2 - a1) - 2 mx s (b2 - b1)) / (b1 b2),
//   ds/dE[x^2] = -s / b2,  ds/dE[xy] = 2 a1 / (b1 b2).
// The second filters those maps with the same (symmetric) window and forms
//   dL/dx = g (G*ds/dmx + 2 x G*ds/dE[x^2] + y G*ds/dE[xy]),  g = -weight/(3P),
// which it adds to d_rgb.
#include "common.cuh"

namespace gs {

constexpr int kSsimTW = 32, kSsimTH = 16, kSsimR = 5, kSsimWin = 2 * kSsimR + 1;
constexpr int kSsimHW = kSsimTW + 2 * kSsimR, kSsimHH = kSsimTH + 2 * kSsimR;  // 42 x 26 with halo
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;

struct SsimTiles {
    int32_t n_views;
    int32_t base[GS_MAX_VIEWS + 1];  // first tile of each view, running sum
    int32_t tiles_x[GS_MAX_VIEWS];
    int32_t width[GS_MAX_VIEWS], height[GS_MAX_VIEWS];
    int64_t pix_base[GS_MAX_VIEWS];
    float g[kSsimWin];
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

__global__ void __launch_bounds__(256) ssim_stats_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                         SsimTiles T, float *__restrict__ partial, float *loss,
                                                         float scale, float constant)
{
    __shared__ float sx[kSsimHH][kSsimHW], sy[kSsimHH][kSsimHW];
    __shared__ float hs[5][kSsimHH][kSsimTW];
    __shared__ float red[8];
    int v, x0, y0;
    ssim_tile_of(T, blockIdx.x, &v, &x0, &y0);
    const int W = T.width[v], H = T.height[v];
    const int64_t pb = T.pix_base[v];
    const int tid = threadIdx.x;
    float acc = 0.0f;
    for (int ch = 0; ch < 3; ch++) {
        for (int k = tid; k < kSsimHH * kSsimHW; k += 256) {
            const int r = k / kSsimHW, c = k % kSsimHW;
            const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + c;
            float xv = 0.0f, yv = 0.0f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const int64_t p = pb + (int64_t)gy * W + gx;
                xv = x[3 * p + ch];
                yv = y[3 * p + ch];
            }
            sx[r][c] = xv;
            sy[r][c] = yv;
        }
        __syncthreads();
        for (int k = tid; k < kSsimHH * kSsimTW; k += 256) {
            const int r = k / kSsimTW, c = k % kSsimTW;
            float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
            #pragma unroll
            for (int t = 0; t < kSsimWin; t++) {
                const float w = T.g[t], a = sx[r][c + t], b = sy[r][c + t];
                m0 += w * a;
                m1 += w * b;
                m2 += w * a * a;
                m3 += w * b * b;
                m4 += w * a * b;
            }
            hs[0][r][c] = m0;
            hs[1][r][c] = m1;
            hs[2][r][c] = m2;
            hs[3][r][c] = m3;
            hs[4][r][c] = m4;
        }
        __syncthreads();
        for (int k = tid; k < kSsimTH * kSsimTW; k += 256) {
            const int r = k / kSsimTW, c = k % kSsimTW;
            const int gy = y0 + r, gx = x0 + c;
            float mx = 0.f, my = 0.f, ex2 = 0.f, ey2 = 0.f, exy = 0.f;
            #pragma unroll
            for (int t = 0; t < kSsimWin; t++) {
                const float w = T.g[t];
                mx += w * hs[0][r + t][c];
                my += w * hs[1][r + t][c];
                ex2 += w * hs[2][r + t][c];
                ey2 += w * hs[3][r + t][c];
                exy += w * hs[4][r + t][c];
            }
            if (gx >= W || gy >= H) continue;
            const float sx2 = ex2 - mx * mx, sy2 = ey2 - my * my, sxy = exy - mx * my;
            const float a1 = 2.f * mx * my + kSsimC1, a2 = 2.f * sxy + kSsimC2;
            const float b1 = mx * mx + my * my + kSsimC1, b2 = sx2 + sy2 + kSsimC2;
            const float ib = 1.0f / (b1 * b2);
            const float s = a1 * a2 * ib;
            acc += s;
            const int64_t p = pb + (int64_t)gy * W + gx;
            partial[9 * p + 3 * ch + 0] = (2.f * my * (a2 - a1) - 2.f * mx * s * (b2 - b1)) * ib;
            partial[9 * p + 3 * ch + 1] = -s / b2;
            partial[9 * p + 3 * ch + 2] = 2.f * a1 * ib;
        }
        __syncthreads();
    }
    acc = warp_sum(acc);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; w++) s += red[w];
        atomicAdd(loss, scale * s + (blockIdx.x == 0 ? constant : 0.0f));
    }
}

__global__ void __launch_bounds__(256) ssim_grad_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                        SsimTiles T, const float *__restrict__ partial,
                                                        float *__restrict__ d_rgb, float gsc)
{
    __shared__ float sp[3][kSsimHH][kSsimHW];
    __shared__ float hs[3][kSsimHH][kSsimTW];
    int v, x0, y0;
    ssim_tile_of(T, blockIdx.x, &v, &x0, &y0);
    const int W = T.width[v], H = T.height[v];
    const int64_t pb = T.pix_base[v];
    const int tid = threadIdx.x;
    for (int ch = 0; ch < 3; ch++) {
        for (int k = tid; k < kSsimHH * kSsimHW; k += 256) {
            const int r = k / kSsimHW, c = k % kSsimHW;
            const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + c;
            float a = 0.f, b = 0.f, d = 0.f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const int64_t p = pb + (int64_t)gy * W + gx;
                a = partial[9 * p + 3 * ch + 0];
                b = partial[9 * p + 3 * ch + 1];
                d = partial[9 * p + 3 * ch + 2];
            }
            sp[0][r][c] = a;
            sp[1][r][c] = b;
            sp[2][r][c] = d;
        }
        __syncthreads();
        for (int k = tid; k < kSsimHH * kSsimTW; k += 256) {
            const int r = k / kSsimTW, c = k % kSsimTW;
            float m0 = 0.f, m1 = 0.f, m2 = 0.f;
            #pragma unroll
            for (int t = 0; t < kSsimWin; t++) {
                const float w = T.g[t];
                m0 += w * sp[0][r][c + t];
                m1 += w * sp[1][r][c + t];
                m2 += w * sp[2][r][c + t];
            }
            hs[0][r][c] = m0;
            hs[1][r][c] = m1;
            hs[2][r][c] = m2;
        }
        __syncthreads();
        for (int k = tid; k < kSsimTH * kSsimTW; k += 256) {
            const int r = k / kSsimTW, c = k % kSsimTW;
            const int gy = y0 + r, gx = x0 + c;
            if (gx >= W || gy >= H) continue;
            float f0 = 0.f, f1 = 0.f, f2 = 0.f;
            #pragma unroll
            for (int t = 0; t < kSsimWin; t++) {
                const float w = T.g[t];
                f0 += w * hs[0][r + t][c];
                f1 += w * hs[1][r + t][c];
                f2 += w * hs[2][r + t][c];
            }
            const int64_t p = pb + (int64_t)gy * W + gx;
            d_rgb[3 * p + ch] += gsc * (f0 + 2.f * x[3 * p + ch] * f1 + y[3 * p + ch] * f2);
        }
        __syncthreads();
    }
}

static gs_status_t make_ssim_tiles(const gs_view_t *views, int32_t n_views, SsimTiles *T, int64_t *n_pix)
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
    // window: exp(-i^2 / (2 * 1.5^2)), i = -5..5, normalised to sum 1
    double g[kSsimWin], sum = 0.0;
    for (int i = 0; i < kSsimWin; i++) {
        const double d = i - kSsimR;
        g[i] = exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[i];
    }
    for (int i = 0; i < kSsimWin; i++) T->g[i] = (float)(g[i] / sum);
    *n_pix = vt.n_pix_total;
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_ssim_workspace_size(int64_t n_pixels)
{
    return n_pixels < 0 ? 0 : sizeof(float) * 9 * (size_t)n_pixels;
}

extern "C" gs_status_t gs_loss_ssim(const float *rgb, const float *target_rgb, const gs_view_t *views,
                                    int32_t n_views, float weight, float *loss, float *d_rgb, void *workspace,
                                    size_t workspace_bytes, void *stream)
{
    if (!rgb || !target_rgb || !loss || !d_rgb || !workspace) return GS_ERR_INVALID_ARG;
    SsimTiles T;
    int64_t P = 0;
    gs_status_t st = make_ssim_tiles(views, n_views, &T, &P);
    if (st != GS_OK) return st;
    if (workspace_bytes < gs_ssim_workspace_size(P)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int blocks = T.base[n_views];
    float *partial = static_cast<float *>(workspace);
    const float scale = (float)(-(double)weight / (3.0 * (double)P));
    // weight * (1 - mean s): block 0 adds the constant weight, every block -weight/(3P) times its sum of s
    ssim_stats_kernel<<<blocks, 256, 0, s>>>(rgb, target_rgb, T, partial, loss, scale, weight);
    ssim_grad_kernel<<<blocks, 256, 0, s>>>(rgb, target_rgb, T, partial, d_rgb, scale);
    return launch_status();
}
