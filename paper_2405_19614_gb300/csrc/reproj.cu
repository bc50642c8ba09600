// a9. Keypoint re-projection loss of the tracking-centred encoder (Sec. 3.2
// Eq. lba, used in the Sec. 3.3 joint loss with weight w1):
//   L = (weight / n) sum_i || u_i - pi(K_v, E_v, P_i) ||_2,
// pi(K, E, P) = (fx X/Z + cx, fy Y/Z + cy) with (X, Y, Z) = R P + t, and its
// gradient with respect to the twist xi of the pose Exp(xi) E at xi = 0:
//   dp/drho = I, dp/dphi = -[p]x.
#include "common.cuh"

namespace gs {

__global__ void __launch_bounds__(256) reproj_kernel(const float *__restrict__ pts, const float *__restrict__ obs,
                                                     const int32_t *__restrict__ view_ids, int64_t n,
                                                     const float *__restrict__ viewmats, ViewTable vt, float scale,
                                                     float near_z, float *loss, float *d_twist)
{
    __shared__ float s_acc[GS_MAX_VIEWS][7];
    for (int k = threadIdx.x; k < vt.n_views * 7; k += blockDim.x) s_acc[k / 7][k % 7] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps step through the keypoints together (the sums below are
    // warp-wide), a lane past the end or behind the camera adding nothing
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
        const int64_t i = i0 + lane;
        float c[7] = {0, 0, 0, 0, 0, 0, 0};
        int v = i < n ? (view_ids ? view_ids[i] : 0) : -1;
        if (v >= vt.n_views) v = -1;
        if (v >= 0) {
            const float *E = viewmats + 12 * v;
            const float X = pts[3 * i], Y = pts[3 * i + 1], Z = pts[3 * i + 2];
            const float x = E[0] * X + E[1] * Y + E[2] * Z + E[3];
            const float y = E[4] * X + E[5] * Y + E[6] * Z + E[7];
            const float z = E[8] * X + E[9] * Y + E[10] * Z + E[11];
            if (z > near_z) {
                const ViewInfo &V = vt.v[v];
                const float rz = 1.0f / z;
                const float rx = obs[2 * i] - (V.fx * x * rz + V.cx);
                const float ry = obs[2 * i + 1] - (V.fy * y * rz + V.cy);
                const float nr = sqrtf(rx * rx + ry * ry);
                c[0] = scale * nr;
                if (nr > 0.0f) {
                    const float gu = -scale * rx / nr, gw = -scale * ry / nr;
                    const float gx = gu * V.fx * rz, gy = gw * V.fy * rz;
                    const float gz = -(gu * V.fx * x + gw * V.fy * y) * rz * rz;
                    c[1] = gx;
                    c[2] = gy;
                    c[3] = gz;
                    c[4] = y * gz - z * gy;
                    c[5] = z * gx - x * gz;
                    c[6] = x * gy - y * gx;
                }
            } else {
                v = -1;
            }
        }
        // keypoints come grouped by view: when every contributing lane has the
        // same view the warp adds up its terms and one lane adds them to the
        // block's sums, else each lane adds its own
        const int vmax = __reduce_max_sync(kFullMask, v);
        if (vmax < 0) continue;
        if (__all_sync(kFullMask, v == vmax || v < 0)) {
            #pragma unroll
            for (int k = 0; k < 7; k++) {
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(kFullMask, c[k], o);
            }
            if (lane == 0) {
                #pragma unroll
                for (int k = 0; k < 7; k++) atomicAdd(&s_acc[vmax][k], c[k]);
            }
        } else if (v >= 0) {
            #pragma unroll
            for (int k = 0; k < 7; k++) atomicAdd(&s_acc[v][k], c[k]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < vt.n_views * 7; k += blockDim.x) {
        const float r = s_acc[k / 7][k % 7];
        if (r == 0.0f) continue;
        if (k % 7 == 0) {
            if (loss) atomicAdd(loss, r);
        } else if (d_twist) {
            atomicAdd(d_twist + 6 * (k / 7) + (k % 7 - 1), r);
        }
    }
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_reproj_loss_grad(const float *points, const float *obs, const int32_t *view_ids, int64_t n,
                                           const gs_view_t *views, const float *viewmats, int32_t n_views,
                                           float weight, float near_z, float *loss, float *d_twist, void *stream)
{
    if (n < 0 || !viewmats) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (n == 0) return GS_OK;
    if (!points || !obs) return GS_ERR_INVALID_ARG;
    const float scale = (float)((double)weight / (double)n);
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < num_sms() * 2 ? want : num_sms() * 2);
    reproj_kernel<<<grid, 256, 0, as_stream(stream)>>>(points, obs, view_ids, n, viewmats, vt, scale, near_z, loss,
                                                       d_twist);
    return launch_status();
}
