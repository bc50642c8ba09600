// Keyframe decoding: the RGB-D frames of the experiments (Sec. 4: TUM RGB-D
// sequences, 8-bit colour and 16-bit depth images) arrive from the host in
// their sensor format, five bytes a pixel, and are widened on the device to
// the FP32 targets of the losses: colour c / 255, depth d * depth_scale
// (metres per depth unit; 0 stays 0, the sensor's "no reading").  Both are one
// correctly rounded FP32 operation, so the result equals the same expression
// evaluated in FP32 anywhere.
#include "common.cuh"

namespace gs {

// Four pixels a thread: 12 colour bytes (three 4-byte words) and four depth
// values (one 8-byte word) in, three float4 of colour and one of depth out.
__global__ void __launch_bounds__(256) decode_kernel(const uint32_t *__restrict__ rgb8w,
                                                     const uint2 *__restrict__ depth16w, int64_t n_quads,
                                                     float depth_scale, float4 *__restrict__ rgb,
                                                     float4 *__restrict__ depth)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_quads;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w[3] = {rgb8w[3 * q], rgb8w[3 * q + 1], rgb8w[3 * q + 2]};
        float c[12];
        #pragma unroll
        for (int k = 0; k < 12; k++) c[k] = __fdiv_rn((float)((w[k >> 2] >> (8 * (k & 3))) & 0xffu), 255.0f);
        rgb[3 * q] = make_float4(c[0], c[1], c[2], c[3]);
        rgb[3 * q + 1] = make_float4(c[4], c[5], c[6], c[7]);
        rgb[3 * q + 2] = make_float4(c[8], c[9], c[10], c[11]);
        const uint2 d = depth16w[q];
        depth[q] = make_float4(__fmul_rn((float)(d.x & 0xffffu), depth_scale), __fmul_rn((float)(d.x >> 16), depth_scale),
                               __fmul_rn((float)(d.y & 0xffffu), depth_scale), __fmul_rn((float)(d.y >> 16), depth_scale));
    }
}

// The last n mod 4 pixels, one a thread.
__global__ void decode_tail_kernel(const uint8_t *__restrict__ rgb8, const uint16_t *__restrict__ depth16, int64_t p0,
                                   int64_t n, float depth_scale, float *__restrict__ rgb, float *__restrict__ depth)
{
    const int64_t p = p0 + threadIdx.x;
    if (p >= n) return;
    for (int ch = 0; ch < 3; ch++) rgb[3 * p + ch] = __fdiv_rn((float)rgb8[3 * p + ch], 255.0f);
    depth[p] = __fmul_rn((float)depth16[p], depth_scale);
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_decode_keyframes(const uint8_t *rgb8, const uint16_t *depth16, int64_t n_pixels,
                                           float depth_scale, float *rgb, float *depth, void *stream)
{
    if (n_pixels < 0) return GS_ERR_INVALID_ARG;
    if (n_pixels == 0) return GS_OK;
    if (!rgb8 || !depth16 || !rgb || !depth) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(rgb8) & 3) || (reinterpret_cast<uintptr_t>(depth16) & 7) ||
        (reinterpret_cast<uintptr_t>(rgb) & 15) || (reinterpret_cast<uintptr_t>(depth) & 15))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int64_t quads = n_pixels / 4;
    if (quads > 0) {
        int64_t blocks = (quads + 255) / 256;
        const int64_t cap = (int64_t)num_sms() * 8;
        if (blocks > cap) blocks = cap;
        decode_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(rgb8),
                                                        reinterpret_cast<const uint2 *>(depth16), quads, depth_scale,
                                                        reinterpret_cast<float4 *>(rgb), reinterpret_cast<float4 *>(depth));
    }
    if (4 * quads < n_pixels) decode_tail_kernel<<<1, 4, 0, s>>>(rgb8, depth16, 4 * quads, n_pixels, depth_scale, rgb, depth);
    return launch_status();
}
