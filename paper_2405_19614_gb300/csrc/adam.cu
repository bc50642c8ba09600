// a10. Adam step over the flat parameter buffer (Sec. 3.4: the Gaussian
// parameters are "iteratively refined using gradient-based optimization"; the
// optimiser is not named), and the on-device pose update of the tracking loop.
#include "common.cuh"

namespace gs {

struct AdamGroups {
    int32_t n;
    int64_t off[GS_MAX_ADAM_GROUPS];
    int64_t cnt[GS_MAX_ADAM_GROUPS];
    float lr[GS_MAX_ADAM_GROUPS];
};

__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float b1, float b2, float eps,
                                         float lr, float ibc1, float ibc2)
{
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    p -= lr * (m * ibc1) / (sqrtf(v * ibc2) + eps);
}

__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ param, const float *__restrict__ grad,
                                                   float *__restrict__ m, float *__restrict__ v, AdamGroups gr,
                                                   float b1, float b2, float eps, int32_t *step)
{
    const int t = step[0] + 1;
    const float ibc1 = 1.0f / (1.0f - powf(b1, (float)t));
    const float ibc2 = 1.0f / (1.0f - powf(b2, (float)t));
    const int gi = blockIdx.y;
    const int64_t off = gr.off[gi], cnt = gr.cnt[gi];
    const float lr = gr.lr[gi];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // scalar head up to a 16-byte boundary, float4 body, scalar tail
    int64_t head = (4 - (off & 3)) & 3;
    if (head > cnt) head = cnt;
    const int64_t body = (cnt - head) / 4;
    for (int64_t k = tid; k < head; k += stride)
        adam_one(param[off + k], grad[off + k], m[off + k], v[off + k], b1, b2, eps, lr, ibc1, ibc2);
    float4 *p4 = reinterpret_cast<float4 *>(param + off + head);
    const float4 *g4 = reinterpret_cast<const float4 *>(grad + off + head);
    float4 *m4 = reinterpret_cast<float4 *>(m + off + head);
    float4 *v4 = reinterpret_cast<float4 *>(v + off + head);
    for (int64_t k = tid; k < body; k += stride) {
        float4 P = p4[k], G = g4[k], M = m4[k], Vv = v4[k];
        adam_one(P.x, G.x, M.x, Vv.x, b1, b2, eps, lr, ibc1, ibc2);
        adam_one(P.y, G.y, M.y, Vv.y, b1, b2, eps, lr, ibc1, ibc2);
        adam_one(P.z, G.z, M.z, Vv.z, b1, b2, eps, lr, ibc1, ibc2);
        adam_one(P.w, G.w, M.w, Vv.w, b1, b2, eps, lr, ibc1, ibc2);
        p4[k] = P;
        m4[k] = M;
        v4[k] = Vv;
    }
    for (int64_t k = head + 4 * body + tid; k < cnt; k += stride)
        adam_one(param[off + k], grad[off + k], m[off + k], v[off + k], b1, b2, eps, lr, ibc1, ibc2);
    // the last block to finish publishes the step number
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y;
        const unsigned ticket = atomicAdd(reinterpret_cast<unsigned *>(step + 1), 1u);
        if (ticket == total - 1) {
            step[0] = t;
            step[1] = 0;
        }
    }
}

// E <- Exp(xi) E, xi <- 0 (xi = (rho, phi); closed-form SE(3) exponential).
__global__ void pose_update_kernel(float *viewmats, float *twist, int n_views)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    double rho[3], ph[3];
    for (int k = 0; k < 3; k++) {
        rho[k] = twist[6 * v + k];
        ph[k] = twist[6 * v + 3 + k];
    }
    const double th2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2], th = sqrt(th2);
    double A, B, C;
    if (th < 1e-5) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
        C = 1.0 / 6.0 - th2 / 120.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    const double Kx[3][3] = {{0, -ph[2], ph[1]}, {ph[2], 0, -ph[0]}, {-ph[1], ph[0], 0}};
    double K2[3][3], R[3][3], Vm[3][3], t[3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) K2[i][j] = Kx[i][0] * Kx[0][j] + Kx[i][1] * Kx[1][j] + Kx[i][2] * Kx[2][j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            const double I = i == j ? 1.0 : 0.0;
            R[i][j] = I + A * Kx[i][j] + B * K2[i][j];
            Vm[i][j] = I + B * Kx[i][j] + C * K2[i][j];
        }
    for (int i = 0; i < 3; i++) t[i] = Vm[i][0] * rho[0] + Vm[i][1] * rho[1] + Vm[i][2] * rho[2];
    float *E = viewmats + 12 * v;
    double out[12];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 4; j++) {
            double acc = R[i][0] * E[j] + R[i][1] * E[4 + j] + R[i][2] * E[8 + j];
            if (j == 3) acc += t[i];
            out[4 * i + j] = acc;
        }
    for (int k = 0; k < 12; k++) E[k] = (float)out[k];
    for (int k = 0; k < 6; k++) twist[6 * v + k] = 0.0f;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_adam_step(float *param, const float *grad, float *m, float *v, const gs_adam_group_t *groups,
                                    int32_t n_groups, float beta1, float beta2, float eps, int32_t *step, void *stream)
{
    if (!param || !grad || !m || !v || !groups || !step) return GS_ERR_INVALID_ARG;
    if (n_groups < 1 || n_groups > GS_MAX_ADAM_GROUPS) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(param) | reinterpret_cast<uintptr_t>(grad) | reinterpret_cast<uintptr_t>(m) |
         reinterpret_cast<uintptr_t>(v)) & 15)
        return GS_ERR_INVALID_ARG;
    AdamGroups g;
    g.n = n_groups;
    int64_t maxcnt = 0;
    for (int k = 0; k < GS_MAX_ADAM_GROUPS; k++) {
        g.off[k] = k < n_groups ? groups[k].offset : 0;
        g.cnt[k] = k < n_groups ? groups[k].count : 0;
        g.lr[k] = k < n_groups ? groups[k].lr : 0.0f;
        if (k < n_groups && (g.off[k] < 0 || g.cnt[k] < 0)) return GS_ERR_INVALID_ARG;
        if (g.cnt[k] > maxcnt) maxcnt = g.cnt[k];
    }
    int64_t want = (maxcnt / 4 + 255) / 256;
    const int64_t cap = num_sms() * 4;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    dim3 grid((unsigned)want, (unsigned)n_groups);
    adam_kernel<<<grid, 256, 0, as_stream(stream)>>>(param, grad, m, v, g, beta1, beta2, eps, step);
    return launch_status();
}

extern "C" gs_status_t gs_pose_update(float *viewmats, float *twist, int32_t n_views, void *stream)
{
    if (!viewmats || !twist || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    pose_update_kernel<<<1, 64, 0, as_stream(stream)>>>(viewmats, twist, n_views);
    return launch_status();
}
