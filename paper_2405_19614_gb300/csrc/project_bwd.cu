// a8. Backward of the projection (reverse of Sec. 3.4 "Projection"; the pose
// gradient serves the Sec. 3.3 joint optimisation, the parameter gradients the
// Sec. 3.4 mapping).
//
// Forward map being differentiated, per view:
//   conic = Sigma2D^-1,  Sigma2D = J Sc J^T + blur I,  Sc = W S W^T,
//   S = M M^T,  M = R(q / |q|) diag(exp(log_scale)),
//   mu2D = (fx x/z + cx, fy y/z + cy),  depth = z,  p = (x, y, z) = W mu + t,
//   J = [[fx/z, 0, -fx tx/z^2], [0, fy/z, -fy ty/z^2]] with tx = clamp(x/z) z,
//   opacity = sigmoid(logit),  colour = max(0, SH(dir) + 1/2),
//   dir = (mu - c) / |mu - c|,  c = -W^T t.
// Twist xi = (rho, phi) with pose Exp(xi) E at xi = 0: p -> p + rho + phi x p,
// Sc -> Exp(phi) Sc Exp(phi)^T, c -> c - W^T rho.
//
// Two kernels, one thread per Gaussian, each looping over all views so that
// gradients summed over views reach HBM once.  The colour kernel keeps the
// Gaussian's SH coefficients and their gradients in registers (the basis and
// its direction gradient are evaluated once per view for all three channels)
// and propagates the view-direction gradient to the mean and to the twist.
// The geometry kernel then does the mean, covariance, opacity and pose paths
// and clears the 2D gradient entries it consumed.  Keeping the SH state out of
// the geometry kernel keeps it at a register count that lets many warps hide
// latency.
#include "common.cuh"
#include "async_copy.cuh"
#include "sh.cuh"

namespace gs {

struct ProjectBwdArgs {
    const float *means, *log_scales, *quats, *opacity_logit, *sh;
    const float *viewmats;
    int64_t n;
    float blur;
    const int32_t *radii;
    float4 *grad2d;
    float *g_means, *g_log_scales, *g_quats, *g_opacity_logit, *g_sh;  // all NULL: pose only
    float *d_twist;
    bool overwrite;          // write (=) the parameter gradients instead of adding (+=)
    bool color_wrote_means;  // the colour kernel has written g_means (SH degree > 0)
};

// dst = v (overwrite) or dst += v
__device__ __forceinline__ void put_grad(float *dst, float v, bool overwrite) { *dst = overwrite ? v : *dst + v; }

__device__ __forceinline__ void flush_twist(float *d_twist, int n_views, float (*s_tw)[6])
{
    __syncthreads();
    for (int k = threadIdx.x; k < n_views * 6; k += blockDim.x) {
        const float r = s_tw[k / 6][k % 6];
        if (r != 0.0f) atomicAdd(d_twist + k, r);
    }
}

// Twist terms of a warp, reduced once per kTwGroup views instead of one warp
// reduction per view and term: lane l stores its NV terms of view v in column
// l of rows (v mod kTwGroup) * NV + k of the warp's table; after the group's
// last view each lane sums whole rows (32 terms, 16-byte loads; the 36-float
// pitch keeps both access patterns free of bank conflicts) into the block's
// s_tw.  Every view of a group stores its rows, zeros included.
constexpr int kTwGroup = 8;
constexpr int kTwPitch = 36;
constexpr int kPbwdWarps = 4;  // 128-thread blocks

template <int NV>
__device__ __forceinline__ void twist_put(float (*tab)[kTwPitch], int v, const float (&tw)[NV], int lane, int n_views,
                                          float (*s_tw)[6])
{
    const int slot = v % kTwGroup;
    #pragma unroll
    for (int k = 0; k < NV; k++) tab[slot * NV + k][lane] = tw[k];
    if (slot != kTwGroup - 1 && v != n_views - 1) return;
    __syncwarp();
    const int v0 = v - slot;
    for (int r = lane; r < (slot + 1) * NV; r += 32) {
        const float4 *row = reinterpret_cast<const float4 *>(tab[r]);
        float4 q = row[0];
        float2 lo = make_float2(q.x, q.y), hi = make_float2(q.z, q.w);
        #pragma unroll
        for (int c = 1; c < 8; c++) {
            q = row[c];
            lo = __fadd2_rn(lo, make_float2(q.x, q.y));
            hi = __fadd2_rn(hi, make_float2(q.z, q.w));
        }
        const float sum = (lo.x + lo.y) + (hi.x + hi.y);
        if (sum != 0.0f) atomicAdd(&s_tw[v0 + r / NV][r % NV], sum);
    }
    __syncwarp();
}

// Bit v of the result is set when Gaussian i is drawn in view v.  All radii are
// loaded up front (independent loads, eight at a time), so the view loops that
// follow carry no load whose address depends on an earlier load.
__device__ __forceinline__ uint64_t visible_views(const int32_t *radii, int64_t n, int64_t i, bool active, int n_views)
{
    uint64_t mask = 0;
    if (!active) return 0;
    for (int v0 = 0; v0 < n_views; v0 += 8) {
        int r[8];
        #pragma unroll
        for (int k = 0; k < 8; k++) r[k] = (v0 + k < n_views) ? __ldg(radii + (int64_t)(v0 + k) * n + i) : 0;
        #pragma unroll
        for (int k = 0; k < 8; k++)
            if (r[k] > 0) mask |= 1ull << (v0 + k);
    }
    return mask;
}

// Colour path: one thread per Gaussian, holding its 3K SH coefficients and
// their gradients in registers for the whole walk over the views.  A block's
// coefficients travel through shared memory both ways, so that every global
// access is a contiguous run over the block's rows: row r of the tile is
// Gaussian i0 + r, its 3K floats (coefficient-major, channel-minor) at pitch
// ShTile::pitch.  With 3K a multiple of 4 (degrees 1 and 3) the copies and the
// row reads are 16-byte, and the pitch is four times an odd number, so the
// eight rows a quarter warp reads fall on distinct bank groups; otherwise they
// are 4-byte with an odd pitch.
template <int DEG>
struct ShTile {
    static constexpr int K = ShCount<DEG>::value;
    static constexpr int row = 3 * K;
    static constexpr bool vec = row % 4 == 0;
    static constexpr int pitch = vec ? ((row / 4) % 2 ? row : row + 4) : (row % 2 ? row : row + 1);
};

// tile <- rows [0, rows) of the block's coefficients at src, as asynchronous
// copies (vec4: src is 16-byte aligned); complete after cp_async_wait_all
template <int DEG>
__device__ __forceinline__ void sh_tile_load_async(const float *src, int rows, bool vec4, float *tile)
{
    using T = ShTile<DEG>;
    const int total = rows * T::row;
    if (T::vec && vec4) {
        for (int u = threadIdx.x; u < total / 4; u += blockDim.x) {
            const int f = 4 * u, r = f / T::row;
            cp_async16(tile + r * T::pitch + (f - r * T::row), src + f);
        }
    } else {
        for (int f = threadIdx.x; f < total; f += blockDim.x) {
            const int r = f / T::row;
            cp_async4(tile + r * T::pitch + (f - r * T::row), src + f, true);
        }
    }
}

// dst = tile (overwrite) or dst += tile, rows [0, rows)
template <int DEG>
__device__ __forceinline__ void sh_tile_store(float *dst, int rows, bool vec4, const float *tile, bool overwrite)
{
    using T = ShTile<DEG>;
    const int total = rows * T::row;
    if (T::vec && vec4) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (int u = threadIdx.x; u < total / 4; u += blockDim.x) {
            const int f = 4 * u, r = f / T::row;
            float4 g = *reinterpret_cast<const float4 *>(tile + r * T::pitch + (f - r * T::row));
            if (!overwrite) {
                const float4 o = d4[u];
                g = make_float4(o.x + g.x, o.y + g.y, o.z + g.z, o.w + g.w);
            }
            d4[u] = g;
        }
    } else {
        for (int f = threadIdx.x; f < total; f += blockDim.x) {
            const int r = f / T::row;
            put_grad(dst + f, tile[r * T::pitch + (f - r * T::row)], overwrite);
        }
    }
}

// this thread's row of the tile <-> registers
template <int DEG>
__device__ __forceinline__ void sh_row_read(const float *row, float (&x)[3 * ShCount<DEG>::value])
{
    using T = ShTile<DEG>;
    if constexpr (T::vec) {
        #pragma unroll
        for (int q = 0; q < T::row / 4; q++) {
            const float4 w = reinterpret_cast<const float4 *>(row)[q];
            x[4 * q] = w.x;
            x[4 * q + 1] = w.y;
            x[4 * q + 2] = w.z;
            x[4 * q + 3] = w.w;
        }
    } else {
        #pragma unroll
        for (int f = 0; f < T::row; f++) x[f] = row[f];
    }
}

template <int DEG>
__device__ __forceinline__ void sh_row_write(float *row, const float (&x)[3 * ShCount<DEG>::value])
{
    using T = ShTile<DEG>;
    if constexpr (T::vec) {
        #pragma unroll
        for (int q = 0; q < T::row / 4; q++)
            reinterpret_cast<float4 *>(row)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    } else {
        #pragma unroll
        for (int f = 0; f < T::row; f++) row[f] = x[f];
    }
}

constexpr int kColorThreads = 32 * kPbwdWarps;

// Three blocks per SM: at most 168 registers a thread, of which the SH
// coefficients and their gradients take 96 at degree 3.
template <int DEG>
__global__ void __launch_bounds__(kColorThreads, 3) project_bwd_color_kernel(ProjectBwdArgs a, ViewTable vt)
{
    using T = ShTile<DEG>;
    constexpr int K = T::K;
    __shared__ float s_E[GS_MAX_VIEWS][12];
    __shared__ float s_c[GS_MAX_VIEWS][3];
    __shared__ float s_tw[GS_MAX_VIEWS][6];
    __shared__ __align__(16) float s_twt[kPbwdWarps][kTwGroup * 3][kTwPitch];
    __shared__ __align__(16) float s_sh[kColorThreads * T::pitch];

    const int64_t i0 = (int64_t)blockIdx.x * kColorThreads;
    const int rows = a.n - i0 < kColorThreads ? (int)(a.n - i0) : kColorThreads;
    const int64_t i = i0 + threadIdx.x;
    const bool active = threadIdx.x < rows;
    const bool vec4 = (reinterpret_cast<uintptr_t>(a.sh) & 15) == 0 &&
                      (!a.g_sh || (reinterpret_cast<uintptr_t>(a.g_sh) & 15) == 0);
    // Prologue: every global load that depends on no other is put in flight
    // at once (the tile and the view matrices as asynchronous copies, then the
    // radii and the mean), so that a block waits on one load latency here
    // instead of a chain of them.  (Issuing the first group's colour gradients
    // here as well spills at three blocks per SM and measured slower.)
    for (int k = threadIdx.x; k < vt.n_views * 12; k += kColorThreads)
        cp_async4(&s_E[k / 12][k % 12], a.viewmats + k, true);
    sh_tile_load_async<DEG>(a.sh + (int64_t)T::row * i0, rows, vec4, s_sh);
    for (int k = threadIdx.x; k < vt.n_views * 6; k += kColorThreads) s_tw[k / 6][k % 6] = 0.0f;
    const uint64_t vis_mask = visible_views(a.radii, a.n, i, active, vt.n_views);
    float m[3] = {0.0f, 0.0f, 0.0f};
    if (active) {
        #pragma unroll
        for (int k = 0; k < 3; k++) m[k] = a.means[3 * i + k];
    }
    // The colour gradients (entries 6..8 of the 2D records) of a group of views
    // are fetched together, by independent loads, and parked in this thread's
    // own row of the tile (free once the coefficients are in registers), so
    // that the walk over the group's views waits on one load latency instead
    // of one per view.
    constexpr int kSlot = T::vec ? 4 : 3;
    constexpr int kGroup = T::pitch / kSlot < 8 ? T::pitch / kSlot : 8;
    const float *g2 = reinterpret_cast<const float *>(a.grad2d);
    float gq[kGroup][3];
    auto fetch_group = [&](int v0) {
        #pragma unroll
        for (int j = 0; j < kGroup; j++) {
            const int v = v0 + j;
            const bool on = v < vt.n_views && ((vis_mask >> v) & 1ull);
            const int64_t o = 12 * ((int64_t)v * a.n + i) + 6;
            #pragma unroll
            for (int c = 0; c < 3; c++) gq[j][c] = on ? g2[o + c] : 0.0f;
        }
    };
    cp_async_wait_all();
    __syncthreads();
    for (int v = threadIdx.x; v < vt.n_views; v += kColorThreads) {
        const float *E = s_E[v];
        #pragma unroll
        for (int k = 0; k < 3; k++) s_c[v][k] = -(E[k] * E[3] + E[4 + k] * E[7] + E[8 + k] * E[11]);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const bool want_twist = a.d_twist != nullptr;
    float sh[3 * K], gsh[3 * K];
    if (active) {
        sh_row_read<DEG>(s_sh + threadIdx.x * T::pitch, sh);
    } else {
        #pragma unroll
        for (int f = 0; f < 3 * K; f++) sh[f] = 0.0f;
    }
    #pragma unroll
    for (int f = 0; f < 3 * K; f++) gsh[f] = 0.0f;
    float gm[3] = {0.0f, 0.0f, 0.0f};
    float *slots = s_sh + threadIdx.x * T::pitch;

    float(*twt)[kTwPitch] = s_twt[threadIdx.x >> 5];
    const bool put_twist = want_twist && DEG > 0;  // the colour depends on the view direction
    #pragma unroll 1
    for (int v0 = 0; v0 < vt.n_views; v0 += kGroup) {
        fetch_group(v0);
        #pragma unroll
        for (int j = 0; j < kGroup; j++) {
            if constexpr (T::vec) {
                reinterpret_cast<float4 *>(slots)[j] = make_float4(gq[j][0], gq[j][1], gq[j][2], 0.0f);
            } else {
                #pragma unroll
                for (int c = 0; c < 3; c++) slots[3 * j + c] = gq[j][c];
            }
        }
        #pragma unroll 1
        for (int j = 0; j < kGroup && v0 + j < vt.n_views; j++) {
            const int v = v0 + j;
            const bool vis = (vis_mask >> v) & 1ull;
            float tw[3] = {0.0f, 0.0f, 0.0f};
            if (!__any_sync(kFullMask, vis)) {
                if (put_twist) twist_put<3>(twt, v, tw, lane, vt.n_views, s_tw);
                continue;
            }
            if (vis) {
                float gc[3];
                if constexpr (T::vec) {
                    const float4 q = reinterpret_cast<const float4 *>(slots)[j];
                    gc[0] = q.x;
                    gc[1] = q.y;
                    gc[2] = q.z;
                } else {
                    #pragma unroll
                    for (int c = 0; c < 3; c++) gc[c] = slots[3 * j + c];
                }
                if (gc[0] != 0.0f || gc[1] != 0.0f || gc[2] != 0.0f) {
                    const float vx = m[0] - s_c[v][0], vy = m[1] - s_c[v][1], vz = m[2] - s_c[v][2];
                    const float rn = rsqrtf(vx * vx + vy * vy + vz * vz);
                    const float dx = vx * rn, dy = vy * rn, dz = vz * rn;
                    float Y[K];
                    sh_basis<DEG>(dx, dy, dz, Y);
                    float col[3] = {0.5f, 0.5f, 0.5f};
                    #pragma unroll
                    for (int k = 0; k < K; k++)
                        #pragma unroll
                        for (int c = 0; c < 3; c++) col[c] += sh[3 * k + c] * Y[k];
                    // colour = max(0, SH + 1/2): no gradient where it is clamped
                    #pragma unroll
                    for (int c = 0; c < 3; c++)
                        if (!(col[c] >= 0.0f)) gc[c] = 0.0f;
                    #pragma unroll
                    for (int k = 0; k < K; k++)
                        #pragma unroll
                        for (int c = 0; c < 3; c++) gsh[3 * k + c] += Y[k] * gc[c];
                    if constexpr (DEG > 0) {
                        float wk[K];
                        #pragma unroll
                        for (int k = 0; k < K; k++) wk[k] = sh[3 * k] * gc[0] + sh[3 * k + 1] * gc[1] + sh[3 * k + 2] * gc[2];
                        float gdir[3];
                        sh_basis_grad<DEG>(dx, dy, dz, wk, gdir);
                        const float dd = gdir[0] * dx + gdir[1] * dy + gdir[2] * dz;
                        const float gvx = (gdir[0] - dx * dd) * rn, gvy = (gdir[1] - dy * dd) * rn,
                                    gvz = (gdir[2] - dz * dd) * rn;
                        gm[0] += gvx;
                        gm[1] += gvy;
                        gm[2] += gvz;
                        const float *E = s_E[v];
                        tw[0] = E[0] * gvx + E[1] * gvy + E[2] * gvz;
                        tw[1] = E[4] * gvx + E[5] * gvy + E[6] * gvz;
                        tw[2] = E[8] * gvx + E[9] * gvy + E[10] * gvz;
                    }
                }
            }
            if (put_twist) twist_put<3>(twt, v, tw, lane, vt.n_views, s_tw);
        }
    }
    if (a.g_sh) {
        // (each thread has used only its own row since the tile was loaded)
        if (active) sh_row_write<DEG>(s_sh + threadIdx.x * T::pitch, gsh);
        __syncthreads();
        sh_tile_store<DEG>(a.g_sh + (int64_t)T::row * i0, rows, vec4, s_sh, a.overwrite);
        if (active && DEG > 0) {
            #pragma unroll
            for (int k = 0; k < 3; k++) put_grad(a.g_means + 3 * i + k, gm[k], a.overwrite);
        }
    }
    if (want_twist) flush_twist(a.d_twist, vt.n_views, s_tw);
}

// Geometry path: one thread per Gaussian.  Five blocks per SM (96 registers,
// a few bytes of spill): the kernel waits on loads, and the fifth block's
// warps hide more of them than the spill costs.
__global__ void __launch_bounds__(128, 5) project_bwd_geom_kernel(ProjectBwdArgs a, ViewTable vt)
{
    __shared__ float s_E[GS_MAX_VIEWS][12];
    __shared__ float s_tw[GS_MAX_VIEWS][6];
    __shared__ __align__(16) float s_twt[kPbwdWarps][kTwGroup * 6][kTwPitch];
    // prologue as in the colour kernel: the view matrices as asynchronous
    // copies, then the parameters, the radii and the first visible view's 2D
    // gradients, all in flight before the block waits
    for (int k = threadIdx.x; k < vt.n_views * 12; k += blockDim.x)
        cp_async4(&s_E[k / 12][k % 12], a.viewmats + k, true);
    for (int k = threadIdx.x; k < vt.n_views * 6; k += blockDim.x) s_tw[k / 6][k % 6] = 0.0f;

    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < a.n;
    const int lane = threadIdx.x & 31;
    const bool want_twist = a.d_twist != nullptr;

    float m[3] = {0, 0, 0}, ls[3] = {0, 0, 0}, q[4] = {1, 0, 0, 0}, ol = 0.0f;
    if (active) {
        #pragma unroll
        for (int k = 0; k < 3; k++) {
            m[k] = a.means[3 * i + k];
            ls[k] = a.log_scales[3 * i + k];
        }
        const float4 q4 = reinterpret_cast<const float4 *>(a.quats)[i];
        q[0] = q4.x;
        q[1] = q4.y;
        q[2] = q4.z;
        q[3] = q4.w;
        ol = a.opacity_logit[i];
    }
    const uint64_t vis_mask = visible_views(a.radii, a.n, i, active, vt.n_views);
    // 2D gradients of the first visible view, then always one visible view ahead
    float4 N0 = make_float4(0.f, 0.f, 0.f, 0.f), N1 = N0, N2 = N0;
    if (vis_mask) {
        const int64_t o = (int64_t)(__ffsll((long long)vis_mask) - 1) * a.n + i;
        N0 = a.grad2d[3 * o];
        N1 = a.grad2d[3 * o + 1];
        N2 = a.grad2d[3 * o + 2];
    }
    cp_async_wait_all();
    __syncthreads();
    const float qn2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    const float qinv = rsqrtf(fmaxf(qn2, 1e-30f));
    const float w = q[0] * qinv, qa = q[1] * qinv, qb = q[2] * qinv, qc = q[3] * qinv;
    float Rq[3][3];
    Rq[0][0] = 1.f - 2.f * (qb * qb + qc * qc);
    Rq[0][1] = 2.f * (qa * qb - w * qc);
    Rq[0][2] = 2.f * (qa * qc + w * qb);
    Rq[1][0] = 2.f * (qa * qb + w * qc);
    Rq[1][1] = 1.f - 2.f * (qa * qa + qc * qc);
    Rq[1][2] = 2.f * (qb * qc - w * qa);
    Rq[2][0] = 2.f * (qa * qc - w * qb);
    Rq[2][1] = 2.f * (qb * qc + w * qa);
    Rq[2][2] = 1.f - 2.f * (qa * qa + qb * qb);
    const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
    float M[3][3], S[3][3];
    #pragma unroll
    for (int r = 0; r < 3; r++)
        #pragma unroll
        for (int c = 0; c < 3; c++) M[r][c] = Rq[r][c] * s[c];
    #pragma unroll
    for (int r = 0; r < 3; r++)
        #pragma unroll
        for (int c = 0; c < 3; c++) S[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
    const float opac = 1.0f / (1.0f + expf(-ol));

    float gm[3] = {0, 0, 0}, Gw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gol = 0.0f;
    float(*twt)[kTwPitch] = s_twt[threadIdx.x >> 5];
    #pragma unroll 1
    for (int v = 0; v < vt.n_views; v++) {
        float tw[6] = {0, 0, 0, 0, 0, 0};
        const bool vis = (vis_mask >> v) & 1ull;
        if (!__any_sync(kFullMask, vis)) {
            if (want_twist) twist_put<6>(twt, v, tw, lane, vt.n_views, s_tw);
            continue;
        }
        if (vis) {
            const int64_t o = (int64_t)v * a.n + i;
            const float4 G0 = N0, G1 = N1, G2v = N2;
            const uint64_t rest = vis_mask & ~((2ull << v) - 1ull);
            if (rest) {
                const int64_t on = (int64_t)(__ffsll((long long)rest) - 1) * a.n + i;
                N0 = a.grad2d[3 * on];
                N1 = a.grad2d[3 * on + 1];
                N2 = a.grad2d[3 * on + 2];
            }
            const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
            a.grad2d[3 * o] = zero4;
            a.grad2d[3 * o + 1] = zero4;
            a.grad2d[3 * o + 2] = zero4;
            const float gu = G0.x, gv = G0.y, gA = G0.z, gB = G0.w, gC = G1.x, gop = G1.y, gz = G2v.y;
            const float *E = s_E[v];
            const ViewInfo &V = vt.v[v];
            const float W[3][3] = {{E[0], E[1], E[2]}, {E[4], E[5], E[6]}, {E[8], E[9], E[10]}};
            const float x = W[0][0] * m[0] + W[0][1] * m[1] + W[0][2] * m[2] + E[3];
            const float y = W[1][0] * m[0] + W[1][1] * m[1] + W[1][2] * m[2] + E[7];
            const float z = W[2][0] * m[0] + W[2][1] * m[1] + W[2][2] * m[2] + E[11];
            float WS[3][3], Sc[3][3];
            #pragma unroll
            for (int r = 0; r < 3; r++)
                #pragma unroll
                for (int c = 0; c < 3; c++) WS[r][c] = W[r][0] * S[0][c] + W[r][1] * S[1][c] + W[r][2] * S[2][c];
            #pragma unroll
            for (int r = 0; r < 3; r++)
                #pragma unroll
                for (int c = 0; c < 3; c++) Sc[r][c] = WS[r][0] * W[c][0] + WS[r][1] * W[c][1] + WS[r][2] * W[c][2];
            const float limx = 1.3f * (0.5f * (float)V.width / V.fx);
            const float limy = 1.3f * (0.5f * (float)V.height / V.fy);
            const float rz = 1.0f / z, rz2 = rz * rz;
            const float xz = x * rz, yz = y * rz;
            const bool clx = xz < -limx || xz > limx, cly = yz < -limy || yz > limy;
            const float Lx = xz < 0.f ? -limx : limx, Ly = yz < 0.f ? -limy : limy;
            const float tx = (clx ? Lx : xz) * z, ty = (cly ? Ly : yz) * z;
            const float J00 = V.fx * rz, J02 = -V.fx * tx * rz2, J11 = V.fy * rz, J12 = -V.fy * ty * rz2;
            float JS0[3], JS1[3];
            #pragma unroll
            for (int c = 0; c < 3; c++) {
                JS0[c] = J00 * Sc[0][c] + J02 * Sc[2][c];
                JS1[c] = J11 * Sc[1][c] + J12 * Sc[2][c];
            }
            const float ca = JS0[0] * J00 + JS0[2] * J02 + a.blur;
            const float cb = JS0[1] * J11 + JS0[2] * J12;
            const float cc = JS1[1] * J11 + JS1[2] * J12 + a.blur;
            const float det = ca * cc - cb * cb;
            const float id2 = 1.0f / (det * det);
            // conic (A, B, C) = (c, -b, a) / det  ->  covariance (a, b, c)
            const float ga = (-gA * cc * cc + gB * cb * cc - gC * cb * cb) * id2;
            const float gb = (2.f * gA * cb * cc - gB * (det + 2.f * cb * cb) + 2.f * gC * ca * cb) * id2;
            const float gc = (-gA * cb * cb + gB * ca * cb - gC * ca * ca) * id2;
            const float hb = 0.5f * gb;
            // Gc = J^T G2 J with G2 = [[ga, hb], [hb, gc]]
            const float u0 = ga * J02 + hb * J12, u1 = hb * J02 + gc * J12;
            float Gc[3][3];
            Gc[0][0] = J00 * ga * J00;
            Gc[0][1] = J00 * hb * J11;
            Gc[0][2] = J00 * u0;
            Gc[1][1] = J11 * gc * J11;
            Gc[1][2] = J11 * u1;
            Gc[2][2] = J02 * u0 + J12 * u1;
            Gc[1][0] = Gc[0][1];
            Gc[2][0] = Gc[0][2];
            Gc[2][1] = Gc[1][2];
            // dL/dJ = 2 G2 J Sc
            const float gJ00 = 2.f * (ga * JS0[0] + hb * JS1[0]);
            const float gJ02 = 2.f * (ga * JS0[2] + hb * JS1[2]);
            const float gJ11 = 2.f * (hb * JS0[1] + gc * JS1[1]);
            const float gJ12 = 2.f * (hb * JS0[2] + gc * JS1[2]);
            float gpx = gu * V.fx * rz, gpy = gv * V.fy * rz;
            float gpz = -(gu * V.fx * x + gv * V.fy * y) * rz2 + gz;
            gpz -= (gJ00 * V.fx + gJ11 * V.fy) * rz2;
            if (!clx) {
                gpx -= gJ02 * V.fx * rz2;
                gpz += gJ02 * 2.f * V.fx * x * rz2 * rz;
            } else {
                gpz += gJ02 * V.fx * Lx * rz2;
            }
            if (!cly) {
                gpy -= gJ12 * V.fy * rz2;
                gpz += gJ12 * 2.f * V.fy * y * rz2 * rz;
            } else {
                gpz += gJ12 * V.fy * Ly * rz2;
            }
            #pragma unroll
            for (int c = 0; c < 3; c++) gm[c] += W[0][c] * gpx + W[1][c] * gpy + W[2][c] * gpz;
            // world covariance gradient W^T Gc W, accumulated over views
            float GcW[3][3];
            #pragma unroll
            for (int r = 0; r < 3; r++)
                #pragma unroll
                for (int c = 0; c < 3; c++) GcW[r][c] = Gc[r][0] * W[0][c] + Gc[r][1] * W[1][c] + Gc[r][2] * W[2][c];
            #pragma unroll
            for (int r = 0; r < 3; r++)
                #pragma unroll
                for (int c = 0; c < 3; c++) Gw[r][c] += W[0][r] * GcW[0][c] + W[1][r] * GcW[1][c] + W[2][r] * GcW[2][c];
            gol += gop * opac * (1.0f - opac);
            if (want_twist) {
                tw[0] = gpx;
                tw[1] = gpy;
                tw[2] = gpz;
                // (Sc Gc - Gc Sc) entries (1,2), (2,0), (0,1)
                float A12 = 0.f, A20 = 0.f, A01 = 0.f;
                #pragma unroll
                for (int k = 0; k < 3; k++) {
                    A12 += Sc[1][k] * Gc[k][2] - Gc[1][k] * Sc[k][2];
                    A20 += Sc[2][k] * Gc[k][0] - Gc[2][k] * Sc[k][0];
                    A01 += Sc[0][k] * Gc[k][1] - Gc[0][k] * Sc[k][1];
                }
                tw[3] = y * gpz - z * gpy + 2.f * A12;
                tw[4] = z * gpx - x * gpz + 2.f * A20;
                tw[5] = x * gpy - y * gpx + 2.f * A01;
            }
        }
        if (want_twist) twist_put<6>(twt, v, tw, lane, vt.n_views, s_tw);
    }

    if (active && a.g_means) {
        // M = Rq diag(s):  dL/dM = 2 Gw M
        float gM[3][3];
        #pragma unroll
        for (int r = 0; r < 3; r++)
            #pragma unroll
            for (int c = 0; c < 3; c++) gM[r][c] = 2.f * (Gw[r][0] * M[0][c] + Gw[r][1] * M[1][c] + Gw[r][2] * M[2][c]);
        float gR[3][3];
        #pragma unroll
        for (int c = 0; c < 3; c++) {
            float gsv = 0.f;
            #pragma unroll
            for (int r = 0; r < 3; r++) {
                gsv += gM[r][c] * Rq[r][c];
                gR[r][c] = gM[r][c] * s[c];
            }
            put_grad(a.g_log_scales + 3 * i + c, gsv * s[c], a.overwrite);
        }
        float gq[4];
        gq[0] = 2.f * (-qc * gR[0][1] + qb * gR[0][2] + qc * gR[1][0] - qa * gR[1][2] - qb * gR[2][0] + qa * gR[2][1]);
        gq[1] = 2.f * (qb * gR[0][1] + qc * gR[0][2] + qb * gR[1][0] - w * gR[1][2] + qc * gR[2][0] + w * gR[2][1]) -
                4.f * qa * (gR[1][1] + gR[2][2]);
        gq[2] = 2.f * (qa * gR[0][1] + w * gR[0][2] + qa * gR[1][0] + qc * gR[1][2] - w * gR[2][0] + qc * gR[2][1]) -
                4.f * qb * (gR[0][0] + gR[2][2]);
        gq[3] = 2.f * (-w * gR[0][1] + qa * gR[0][2] + w * gR[1][0] + qb * gR[1][2] + qa * gR[2][0] + qb * gR[2][1]) -
                4.f * qc * (gR[0][0] + gR[1][1]);
        const float qd = gq[0] * w + gq[1] * qa + gq[2] * qb + gq[3] * qc;
        const float qn[4] = {w, qa, qb, qc};
        #pragma unroll
        for (int k = 0; k < 4; k++) put_grad(a.g_quats + 4 * i + k, (gq[k] - qn[k] * qd) * qinv, a.overwrite);
        #pragma unroll
        for (int k = 0; k < 3; k++) put_grad(a.g_means + 3 * i + k, gm[k], a.overwrite && !a.color_wrote_means);
        put_grad(a.g_opacity_logit + i, gol, a.overwrite);
    }
    if (want_twist) flush_twist(a.d_twist, vt.n_views, s_tw);
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_project_bwd(const gs_params_t *params, const gs_view_t *views, const float *viewmats,
                                      int32_t n_views, const gs_options_t *opt, const gs_projected_t *proj,
                                      float *grad2d, gs_param_grads_t *grads, float *d_twist, void *stream)
{
    if (!params || !viewmats || !opt || !proj || !grad2d) return GS_ERR_INVALID_ARG;
    if (!grads && !d_twist) return GS_ERR_INVALID_ARG;
    if (params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (params->n == 0) return GS_OK;
    if (!params->means || !params->log_scales || !params->quats || !params->opacity_logit || !params->sh ||
        !proj->radii)
        return GS_ERR_INVALID_ARG;
    if (grads && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logit || !grads->sh))
        return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(grad2d) & 15) || (reinterpret_cast<uintptr_t>(params->quats) & 15))
        return GS_ERR_INVALID_ARG;
    ProjectBwdArgs a;
    a.means = params->means;
    a.log_scales = params->log_scales;
    a.quats = params->quats;
    a.opacity_logit = params->opacity_logit;
    a.sh = params->sh;
    a.viewmats = viewmats;
    a.n = params->n;
    a.blur = opt->blur;
    a.radii = proj->radii;
    a.grad2d = reinterpret_cast<float4 *>(grad2d);
    a.g_means = grads ? grads->means : nullptr;  // NULL grads: pose-only (twist gradients only)
    a.g_log_scales = grads ? grads->log_scales : nullptr;
    a.g_quats = grads ? grads->quats : nullptr;
    a.g_opacity_logit = grads ? grads->opacity_logit : nullptr;
    a.g_sh = grads ? grads->sh : nullptr;
    a.d_twist = d_twist;
    a.overwrite = opt->overwrite_grads != 0;
    a.color_wrote_means = params->sh_degree > 0;
    const int threads = 128;
    cudaStream_t s = as_stream(stream);
    // colour first: the geometry kernel clears the 2D gradients after use
    const unsigned cblocks = (unsigned)((params->n + kColorThreads - 1) / kColorThreads);
    switch (params->sh_degree) {
    case 0: project_bwd_color_kernel<0><<<cblocks, kColorThreads, 0, s>>>(a, vt); break;
    case 1: project_bwd_color_kernel<1><<<cblocks, kColorThreads, 0, s>>>(a, vt); break;
    case 2: project_bwd_color_kernel<2><<<cblocks, kColorThreads, 0, s>>>(a, vt); break;
    default: project_bwd_color_kernel<3><<<cblocks, kColorThreads, 0, s>>>(a, vt); break;
    }
    const unsigned gblocks = (unsigned)((params->n + threads - 1) / threads);
    project_bwd_geom_kernel<<<gblocks, threads, 0, s>>>(a, vt);
    return launch_status();
}

extern "C" gs_status_t gs_render_bwd(const gs_params_t *params, const gs_view_t *views, const float *viewmats,
                                     int32_t n_views, const gs_options_t *opt, const gs_projected_t *proj,
                                     const gs_bins_t *bins, const gs_image_t *img, const float *d_rgb,
                                     const float *d_depth, const float *d_alpha, float *grad2d,
                                     gs_param_grads_t *grads, float *d_twist, uint32_t *work_counter, void *stream)
{
    if (!params) return GS_ERR_INVALID_ARG;
    gs_status_t st = gs_render_bwd_splats(proj, params->n, bins, views, n_views, img, d_rgb, d_depth, d_alpha,
                                          grad2d, work_counter, stream);
    if (st != GS_OK) return st;
    return gs_project_bwd(params, views, viewmats, n_views, opt, proj, grad2d, grads, d_twist, stream);
}
