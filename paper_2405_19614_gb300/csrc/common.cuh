// Internal helpers of the sm_103a splatting library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kTile = GS_TILE;              // default tile width and height
constexpr uint32_t kFullMask = 0xffffffffu;

// Per-view constants passed by value to kernels.
struct ViewInfo {
    float fx, fy, cx, cy;
    int32_t width, height, tiles_x, tiles_y;
    int32_t tile_base;
    int16_t tile_w, tile_h;  // tile shape in pixels
    int64_t pix_base;
    int32_t item_base;  // first compositing work item of the view (set by the launcher)
    int32_t pad;
};

struct ViewTable {
    int32_t n_views;
    int32_t n_tiles_total;
    int64_t n_pix_total;
    ViewInfo v[GS_MAX_VIEWS];
};

static_assert(sizeof(ViewTable) <= 3700, "view table must fit in kernel parameters with the other arguments");

// A tile side: 8, 16, 32 or 64 pixels (0 means the default).
inline bool valid_tile_side(int32_t t) { return t == 8 || t == 16 || t == 32 || t == 64; }

inline gs_status_t make_view_table(const gs_view_t *views, int32_t n_views, ViewTable *vt)
{
    if (!views || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    vt->n_views = n_views;
    int64_t tiles = 0, pix = 0;
    for (int i = 0; i < n_views; i++) {
        const gs_view_t &s = views[i];
        if (s.width <= 0 || s.height <= 0 || s.width > (1 << 20) || s.height > (1 << 20)) return GS_ERR_INVALID_ARG;
        if (!(s.fx > 0.0f) || !(s.fy > 0.0f)) return GS_ERR_INVALID_ARG;
        const int32_t tw = s.tile_w ? s.tile_w : kTile, th = s.tile_h ? s.tile_h : kTile;
        if (!valid_tile_side(tw) || !valid_tile_side(th) || tw * th > 2048) return GS_ERR_INVALID_ARG;
        ViewInfo &d = vt->v[i];
        d.fx = s.fx;
        d.fy = s.fy;
        d.cx = s.cx;
        d.cy = s.cy;
        d.width = s.width;
        d.height = s.height;
        d.tile_w = (int16_t)tw;
        d.tile_h = (int16_t)th;
        d.tiles_x = (s.width + tw - 1) / tw;
        d.tiles_y = (s.height + th - 1) / th;
        d.tile_base = (int32_t)tiles;
        d.item_base = 0;
        d.pad = 0;
        d.pix_base = pix;
        tiles += (int64_t)d.tiles_x * d.tiles_y;
        pix += (int64_t)s.width * s.height;
        if (tiles >= (int64_t(1) << 31) || pix >= (int64_t(1) << 35)) return GS_ERR_INVALID_ARG;
    }
    vt->n_tiles_total = (int32_t)tiles;
    vt->n_pix_total = pix;
    return GS_OK;
}

// View that owns a global tile id (views are few; a linear scan is enough).
__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int tile)
{
    int v = 0;
    #pragma unroll 1
    for (int k = 1; k < vt.n_views; k++)
        if (tile >= vt.v[k].tile_base) v = k;
    return v;
}

// View that owns a compositing work item.
__device__ __forceinline__ int view_of_item(const ViewTable &vt, int item)
{
    int v = 0;
    #pragma unroll 1
    for (int k = 1; k < vt.n_views; k++)
        if (item >= vt.v[k].item_base) v = k;
    return v;
}

__device__ __forceinline__ void raise_status(uint32_t *status, gs_status_t code)
{
    if (status) atomicOr(status, 1u << (unsigned)code);
}

inline gs_status_t launch_status()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Warp-wide sum.
__device__ __forceinline__ float warp_sum(float x)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFullMask, x, o);
    return x;
}

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;

}  // namespace gs
