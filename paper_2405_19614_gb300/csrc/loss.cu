// a6. L1 rendering losses with the optional filter gate (Sec. 3.3: gate
// G(p) = [D_c(p) > 0][D_g(p) > 0][M_b(p) > gamma] and the joint loss terms
// w2 L_c + w3 L_d; Sec. 3.4: the L1 terms of the mapping loss L_m).
//   L = w_c / (3P) sum_p G(p) |C(p) - C^(p)|_1 + w_d / P sum_p G(p) |D(p) - D^(p)|
// over all P pixels of the batch; writes dL/dC, dL/dD (sign(0) = 0).
#include "common.cuh"

namespace gs {

__device__ __forceinline__ float sgn(float x) { return (float)((x > 0.0f) - (x < 0.0f)); }

__global__ void __launch_bounds__(256) loss_l1_kernel(const float *__restrict__ rgb, const float *__restrict__ depth,
                                                      const float *__restrict__ alpha, const float *__restrict__ trgb,
                                                      const float *__restrict__ tdepth, int64_t P, float kc, float kd,
                                                      int use_gate, float gamma, float *loss, float *d_rgb,
                                                      float *d_depth)
{
    __shared__ float part[8];
    float acc = 0.0f;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        const float D = depth[p], Dt = tdepth[p];
        bool gate = true;
        if (use_gate) gate = (Dt > 0.0f) && (D > 0.0f) && (alpha[p] > gamma);
        const float g = gate ? 1.0f : 0.0f;
        float l = 0.0f;
        #pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            const float r = rgb[3 * p + ch] - trgb[3 * p + ch];
            l += kc * fabsf(r);
            d_rgb[3 * p + ch] = g * kc * sgn(r);
        }
        const float r = D - Dt;
        l += kd * fabsf(r);
        d_depth[p] = g * kd * sgn(r);
        acc += g * l;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
        if (loss) atomicAdd(loss, s);
    }
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_loss_l1(const float *rgb, const float *depth, const float *alpha, const float *target_rgb,
                                  const float *target_depth, int64_t n_pixels, float w_c, float w_d,
                                  int32_t use_gate, float gamma, float *loss, float *d_rgb, float *d_depth,
                                  void *stream)
{
    if (n_pixels < 0) return GS_ERR_INVALID_ARG;
    if (n_pixels == 0) return GS_OK;
    if (!rgb || !depth || !target_rgb || !target_depth || !d_rgb || !d_depth || (use_gate && !alpha))
        return GS_ERR_INVALID_ARG;
    const float kc = (float)((double)w_c / (3.0 * (double)n_pixels));
    const float kd = (float)((double)w_d / (double)n_pixels);
    const int64_t want = (n_pixels + 255) / 256;
    const int grid = (int)(want < num_sms() * 8 ? want : num_sms() * 8);
    loss_l1_kernel<<<grid, 256, 0, as_stream(stream)>>>(rgb, depth, alpha, target_rgb, target_depth, n_pixels, kc, kd,
                                                        use_gate, gamma, loss, d_rgb, d_depth);
    return launch_status();
}
