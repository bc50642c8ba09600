// a1. Projection of every Gaussian into every view (Sec. 3.4 "Projection":
// mu2D = K E_t mu / d, r2D = f r / d, generalised to the EWA footprint of the
// rasteriser used in Sec. 4.1).
//
// One thread per Gaussian loops over all views, so the structure-of-arrays
// parameters are read from HBM once per launch however many views there are.
// The radius, tile rectangle and depth follow a fixed sequence of correctly
// rounded FP32 operations (explicit __f*_rn intrinsics, never contracted) so
// that the tile keys are reproducible bit for bit.  So does every quantity the
// compositing takes a decision on: the record carries log2(o) and the conic
// scaled to base 2, and the 2D mean's double-FP32 remainder, so that
// log2(alpha) at a pixel (render.cuh) and with it the alpha skip and clamp
// decisions are reproducible bit for bit too.  Colour is ordinary FP32.
#include "common.cuh"
#include "sh.cuh"

namespace gs {

#define MUL __fmul_rn
#define ADD __fadd_rn
#define SUB __fsub_rn
#define DIV __fdiv_rn

// exp for the geometry: Cody-Waite reduction (ln 2 split into a 15-bit head
// and a tail), degree-7 Taylor polynomial of e^r in Horner form with fused
// multiply-adds, exact scaling by 2^k; argument clamped to [-80, 80].  Each
// step is one correctly rounded operation, so the result is reproducible on
// any IEEE machine that runs the same steps.
__device__ __forceinline__ float geom_expf(float x)
{
    x = (x > 80.0f) ? 80.0f : x;
    x = (x < -80.0f) ? -80.0f : x;
    float k = rintf(MUL(x, 0x1.715476p+0f));
    float r = __fmaf_rn(-k, 0x1.62e4p-1f, x);
    r = __fmaf_rn(-k, 0x1.7f7d1cp-20f, r);
    float p = 0x1.a01a02p-13f;
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
    p = __fmaf_rn(p, r, 0x1.111112p-7f);
    p = __fmaf_rn(p, r, 0x1.555556p-5f);
    p = __fmaf_rn(p, r, 0x1.555556p-3f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    if (p != p) return p;
    int ki = (int)k;
    return MUL(p, __int_as_float((ki + 127) << 23));
}

// log2 for the decision record, y >= 1: y = m 2^e with m in (sqrt(1/2),
// sqrt(2)], then log2 m = (2 / ln 2) atanh(s), s = (m - 1) / (m + 1), by the
// odd series s (C1 + s^2 (C3 + s^2 (C5 + s^2 (C7 + s^2 C9)))), C_k = 2 / (k ln 2)
// (|s| <= 0.172, so the next term is below 1e-9 relative), Horner with fused
// multiply-adds.  Each step is one correctly rounded operation.
__device__ __forceinline__ float geom_log2f(float y)
{
    const uint32_t bits = __float_as_uint(y);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) {
        m = MUL(m, 0.5f);
        e += 1;
    }
    const float s = DIV(SUB(m, 1.0f), ADD(m, 1.0f));
    const float s2 = MUL(s, s);
    float p = 0x1.484b14p-2f;
    p = __fmaf_rn(p, s2, 0x1.a61762p-2f);
    p = __fmaf_rn(p, s2, 0x1.2776c6p-1f);
    p = __fmaf_rn(p, s2, 0x1.ec709ep-1f);
    p = __fmaf_rn(p, s2, 0x1.715476p+1f);
    return ADD((float)e, MUL(s, p));
}

// log2 of the opacity sigmoid(l) = 1 / (1 + e^-l): -log2(1 + e^-l).
__device__ __forceinline__ float geom_log2_opacity(float l)
{
    return -geom_log2f(ADD(1.0f, geom_expf(-l)));
}

struct Geom {
    float u, v, z;
    float ca, cb, cc;   // 2D covariance including the blur
    float det;
    int32_t radius;
    int32_t x0, y0, x1, y1;
};

// The FP32 geometry contract, in two parts: the world covariance S (symmetric,
// view-independent, so computed once per Gaussian; false for a degenerate
// quaternion, which no view draws), then per view the projection.
__device__ __forceinline__ bool world_covariance(const float ls[3], const float q[4], float S[3][3])
{
    float nq = ADD(ADD(ADD(MUL(q[0], q[0]), MUL(q[1], q[1])), MUL(q[2], q[2])), MUL(q[3], q[3]));
    if (!(nq > 0.0f)) return false;
    float sq = __fsqrt_rn(nq);
    float w = DIV(q[0], sq), a = DIV(q[1], sq), b = DIV(q[2], sq), c = DIV(q[3], sq);
    float R[3][3];
    R[0][0] = SUB(1.0f, MUL(2.0f, ADD(MUL(b, b), MUL(c, c))));
    R[0][1] = MUL(2.0f, SUB(MUL(a, b), MUL(w, c)));
    R[0][2] = MUL(2.0f, ADD(MUL(a, c), MUL(w, b)));
    R[1][0] = MUL(2.0f, ADD(MUL(a, b), MUL(w, c)));
    R[1][1] = SUB(1.0f, MUL(2.0f, ADD(MUL(a, a), MUL(c, c))));
    R[1][2] = MUL(2.0f, SUB(MUL(b, c), MUL(w, a)));
    R[2][0] = MUL(2.0f, SUB(MUL(a, c), MUL(w, b)));
    R[2][1] = MUL(2.0f, ADD(MUL(b, c), MUL(w, a)));
    R[2][2] = SUB(1.0f, MUL(2.0f, ADD(MUL(a, a), MUL(b, b))));

    float s[3] = {geom_expf(ls[0]), geom_expf(ls[1]), geom_expf(ls[2])};
    float M[3][3];
    #pragma unroll
    for (int i = 0; i < 3; i++)
        #pragma unroll
        for (int j = 0; j < 3; j++) M[i][j] = MUL(R[i][j], s[j]);
    #pragma unroll
    for (int i = 0; i < 3; i++)
        #pragma unroll
        for (int j = i; j < 3; j++) {
            S[i][j] = ADD(ADD(MUL(M[i][0], M[j][0]), MUL(M[i][1], M[j][1])), MUL(M[i][2], M[j][2]));
            S[j][i] = S[i][j];
        }
    return true;
}

// The per-view part.  Returns false when the Gaussian touches no tile.  lim:
// the view's (limx, limy) = 1.3 (0.5 width / fx, 0.5 height / fy).
__device__ __forceinline__ bool geometry(const float m[3], const float S[3][3], const float *E, const ViewInfo &V,
                                         const float *lim, float near_z, float blur, Geom &g)
{
    float x = ADD(ADD(ADD(MUL(E[0], m[0]), MUL(E[1], m[1])), MUL(E[2], m[2])), E[3]);
    float y = ADD(ADD(ADD(MUL(E[4], m[0]), MUL(E[5], m[1])), MUL(E[6], m[2])), E[7]);
    float z = ADD(ADD(ADD(MUL(E[8], m[0]), MUL(E[9], m[1])), MUL(E[10], m[2])), E[11]);
    if (!(z > near_z)) return false;

    const float limx = lim[0], limy = lim[1];
    float xz = DIV(x, z), yz = DIV(y, z);
    xz = fminf(limx, fmaxf(-limx, xz));
    yz = fminf(limy, fmaxf(-limy, yz));
    float tx = MUL(xz, z), ty = MUL(yz, z);
    float z2 = MUL(z, z);
    float J00 = DIV(V.fx, z), J02 = -DIV(MUL(V.fx, tx), z2);
    float J11 = DIV(V.fy, z), J12 = -DIV(MUL(V.fy, ty), z2);

    float T[2][3];
    #pragma unroll
    for (int j = 0; j < 3; j++) {
        T[0][j] = ADD(MUL(J00, E[0 + j]), MUL(J02, E[8 + j]));
        T[1][j] = ADD(MUL(J11, E[4 + j]), MUL(J12, E[8 + j]));
    }
    float U[2][3];
    #pragma unroll
    for (int i = 0; i < 2; i++)
        #pragma unroll
        for (int j = 0; j < 3; j++)
            U[i][j] = ADD(ADD(MUL(T[i][0], S[0][j]), MUL(T[i][1], S[1][j])), MUL(T[i][2], S[2][j]));
    float ca = ADD(ADD(ADD(MUL(U[0][0], T[0][0]), MUL(U[0][1], T[0][1])), MUL(U[0][2], T[0][2])), blur);
    float cb = ADD(ADD(MUL(U[0][0], T[1][0]), MUL(U[0][1], T[1][1])), MUL(U[0][2], T[1][2]));
    float cc = ADD(ADD(ADD(MUL(U[1][0], T[1][0]), MUL(U[1][1], T[1][1])), MUL(U[1][2], T[1][2])), blur);

    float det = SUB(MUL(ca, cc), MUL(cb, cb));
    if (!(det > 0.0f)) return false;
    float mid = MUL(0.5f, ADD(ca, cc));
    float disc = SUB(MUL(mid, mid), det);
    float lam = ADD(mid, __fsqrt_rn(fmaxf(disc, 0.0f)));
    float rad = ceilf(MUL(3.0f, __fsqrt_rn(lam)));

    float u = ADD(DIV(MUL(V.fx, x), z), V.cx);
    float v = ADD(DIV(MUL(V.fy, y), z), V.cy);
    if (!(fabsf(u) < 0x1p24f && fabsf(v) < 0x1p24f && rad < 0x1p24f)) return false;

    // tile sides are powers of two, so these quotients are exact
    const float tw = (float)V.tile_w, th = (float)V.tile_h;
    float fx0 = floorf(DIV(SUB(u, rad), tw)), fx1 = floorf(DIV(ADD(u, rad), tw));
    float fy0 = floorf(DIV(SUB(v, rad), th)), fy1 = floorf(DIV(ADD(v, rad), th));
    fx0 = fmaxf(fx0, 0.0f);
    fy0 = fmaxf(fy0, 0.0f);
    fx1 = fminf(fx1, (float)(V.tiles_x - 1));
    fy1 = fminf(fy1, (float)(V.tiles_y - 1));
    if (!(fx0 <= fx1 && fy0 <= fy1)) return false;

    g.u = u;
    g.v = v;
    g.z = z;
    g.ca = ca;
    g.cb = cb;
    g.cc = cc;
    g.det = det;
    g.radius = (int32_t)rad;
    g.x0 = (int32_t)fx0;
    g.y0 = (int32_t)fy0;
    g.x1 = (int32_t)fx1;
    g.y1 = (int32_t)fy1;
    return true;
}

// Error-free transformations for double-FP32 arithmetic (hi + lo).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = ADD(a, b);
    const float bb = SUB(s, a);
    e = ADD(SUB(a, SUB(s, bb)), SUB(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = MUL(a, b);
    e = __fmaf_rn(a, b, -p);
}

// r0 m0 + r1 m1 + r2 m2 + t as hi + lo (compensated dot product); hi is the
// geometry's camera coordinate, bit for bit.
__device__ __forceinline__ void dot3_plus(const float *r, const float *m, float t, float &hi, float &lo)
{
    float p, e, s, es;
    two_prod(r[0], m[0], s, lo);
    two_prod(r[1], m[1], p, e);
    two_sum(s, p, s, es);
    lo = ADD(lo, ADD(e, es));
    two_prod(r[2], m[2], p, e);
    two_sum(s, p, s, es);
    lo = ADD(lo, ADD(e, es));
    two_sum(s, t, s, es);
    lo = ADD(lo, es);
    hi = s;
}

// Remainder (f * x / z + c) - ref of the pixel coordinate, with x and z given
// as hi + lo pairs, in double-FP32 arithmetic.
__device__ __forceinline__ float pixel_remainder(float f, float xh, float xl, float zh, float zl, float c, float ref)
{
    const float q = DIV(xh, zh);
    // x - q z, exactly for the hi parts, then the lo parts
    const float r = ADD(__fmaf_rn(-q, zh, xh), SUB(xl, MUL(q, zl)));
    const float ql = DIV(r, zh);
    float m, me;
    two_prod(f, q, m, me);
    const float ml = ADD(me, MUL(f, ql));
    float s, se;
    two_sum(m, c, s, se);
    return ADD(SUB(s, ref), ADD(se, ml));
}

// Base-2 conic of a 2D covariance (a, b, c) with determinant det:
// (A', B', C') = (-log2(e)/2 c, log2(e) b, -log2(e)/2 a) / det, so that
// log2(o exp(-1/2 d^T conic d)) = log2(o) + A' dx^2 + B' dx dy + C' dy^2.
constexpr float kNegHalfLog2e = -0x1.715476p-1f;
constexpr float kLog2eF = 0x1.715476p+0f;

// Tiles of a rectangle of at most 64 tiles (w x h, row-major bits from tile
// (x0, y0)) that a splat can reach with alpha >= 1/255.  With d = pixel -
// mean (mean u + du, v + dv) and q(d) = P dx^2 + 2 B dx dy + Q dy^2,
// (P, B, Q) = -(A', B'/2, C') of the record, log2 of the raw alpha is
// log2 o - q(d), so the pixels that can blend lie in the ellipse q <= K,
// K = log2 o - log2(1/255) + margin.  The margin, 1.5e-3 + 3.2e-5
// (sqrt(PQ) + |B|)^2 / (PQ - B^2), is twice the bound on the FP32 evaluation
// error of the per-pixel test inside that ellipse (whose terms are at most
// K (sqrt(PQ) + |B|)^2 / (PQ - B^2) in magnitude).  For each tile row, a
// horizontal band of pixel centres y in [a, b], the ellipse's points in the
// band form an x-interval: an end is the ellipse's own extreme point x = +-X,
// X = sqrt(K Q / (PQ - B^2)) at y = -+B X / Q, when that lies in the band, else
// where the band's edge y = c crosses the ellipse, x = (-B c +- sqrt(PK -
// (PQ - B^2) c^2)) / P.  A tile is kept when its pixel centres' x-range meets
// the interval widened by 2e-3 + 2e-5 X (more than the rounding of the ends).
// So a dropped tile is one where every pixel would skip the splat.  One fixed
// sequence of correctly rounded operations, so the tile lists are
// reproducible bit for bit.
__device__ __forceinline__ unsigned long long tile_keep_mask(float u, float v, float du, float dv, float log2o,
                                                             float A2, float B2, float C2, int x0, int y0, int w,
                                                             int h, int tw, int th)
{
    constexpr float kCut = -0x1.ffa37cp+2f;  // log2(1/255) rounded to FP32
    const float P = -A2, Q = -C2, B = MUL(-0.5f, B2);
    const float D = SUB(MUL(P, Q), MUL(B, B));
    if (!(D > 0.0f)) return ~0ull >> (64 - w * h);  // degenerate: keep every tile
    const float r = ADD(__fsqrt_rn(MUL(P, Q)), fabsf(B));
    const float K = ADD(SUB(log2o, kCut), ADD(1.5e-3f, DIV(MUL(3.2e-5f, MUL(r, r)), D)));
    if (!(K > 0.0f)) return 0ull;  // no pixel reaches the cut
    const float X = __fsqrt_rn(DIV(MUL(K, Q), D));
    const float yR = DIV(MUL(-B, X), Q), yL = -yR;  // heights of the rightmost and leftmost points
    const float delta = ADD(2e-3f, MUL(2e-5f, X));
    const float PK = MUL(P, K);
    unsigned long long mask = 0ull;
    #pragma unroll 1
    for (int j = 0; j < h; j++) {
        const float cy0 = (float)((y0 + j) * th) + 0.5f, cy1 = ADD(cy0, (float)(th - 1));
        const float a = SUB(SUB(cy0, v), dv), b = SUB(SUB(cy1, v), dv);
        float xr, xl;
        if (yR >= a && yR <= b) {
            xr = X;
        } else {
            const float c = yR > b ? b : a;
            const float disc = SUB(PK, MUL(MUL(D, c), c));
            if (!(disc >= 0.0f)) continue;  // the band misses the ellipse
            xr = DIV(ADD(MUL(-B, c), __fsqrt_rn(disc)), P);
        }
        if (yL >= a && yL <= b) {
            xl = -X;
        } else {
            const float c = yL > b ? b : a;
            const float disc = SUB(PK, MUL(MUL(D, c), c));
            if (!(disc >= 0.0f)) continue;
            xl = DIV(SUB(MUL(-B, c), __fsqrt_rn(disc)), P);
        }
        const float lo = SUB(xl, delta), hi = ADD(xr, delta);
        #pragma unroll 1
        for (int i = 0; i < w; i++) {
            const float cx0 = (float)((x0 + i) * tw) + 0.5f, cx1 = ADD(cx0, (float)(tw - 1));
            const float e0 = SUB(SUB(cx0, u), du), e1 = SUB(SUB(cx1, u), du);
            if (lo <= e1 && e0 <= hi) mask |= 1ull << (j * w + i);
        }
    }
    return mask;
}

#undef MUL
#undef ADD
#undef SUB
#undef DIV

struct ProjectArgs {
    const float *means, *log_scales, *quats, *opacity_logit, *sh;
    const float *viewmats;
    int64_t n;
    float near_z, blur;
    float4 *rec;
    uint2 *rect;
    int32_t *radii;
    uint32_t *tiles_touched;
    unsigned long long *tile_mask;
};

template <int DEG>
__global__ void __launch_bounds__(128) project_kernel(ProjectArgs a, ViewTable vt)
{
    constexpr int K = ShCount<DEG>::value;
    __shared__ float s_E[GS_MAX_VIEWS][12];
    __shared__ float s_c[GS_MAX_VIEWS][3];
    __shared__ float s_lim[GS_MAX_VIEWS][2];
    for (int k = threadIdx.x; k < vt.n_views * 12; k += blockDim.x) s_E[k / 12][k % 12] = a.viewmats[k];
    __syncthreads();
    for (int v = threadIdx.x; v < vt.n_views; v += blockDim.x) {
        // camera centre c = -R^T t
        const float *E = s_E[v];
        #pragma unroll
        for (int i = 0; i < 3; i++) s_c[v][i] = -(E[i] * E[3] + E[4 + i] * E[7] + E[8 + i] * E[11]);
        // the view's clamp of x/z and y/z (in the geometry contract's operations)
        const ViewInfo &V = vt.v[v];
        s_lim[v][0] = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)V.width), V.fx));
        s_lim[v][1] = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)V.height), V.fy));
    }
    __syncthreads();

    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float m[3], ls[3], q[4];
    #pragma unroll
    for (int k = 0; k < 3; k++) {
        m[k] = __ldg(a.means + 3 * i + k);
        ls[k] = __ldg(a.log_scales + 3 * i + k);
    }
    const float4 q4 = __ldg(reinterpret_cast<const float4 *>(a.quats) + i);
    q[0] = q4.x;
    q[1] = q4.y;
    q[2] = q4.z;
    q[3] = q4.w;
    const float log2o = geom_log2_opacity(__ldg(a.opacity_logit + i));
    float S[3][3];
    const bool cov_ok = world_covariance(ls, q, S);
    // the SH coefficients are read only for the views the Gaussian is drawn
    // in (they come from L1 after the first): 48 registers fewer a thread than
    // holding them across the view loop, and no read for a Gaussian no view draws
    float sh[K * 3];
    const float *shp = a.sh + (int64_t)K * 3 * i;
    auto load_sh = [&]() {
        if constexpr ((K * 3) % 4 == 0) {
            #pragma unroll
            for (int k = 0; k < K * 3 / 4; k++) {
                float4 t = __ldg(reinterpret_cast<const float4 *>(shp) + k);
                sh[4 * k] = t.x;
                sh[4 * k + 1] = t.y;
                sh[4 * k + 2] = t.z;
                sh[4 * k + 3] = t.w;
            }
        } else {
            #pragma unroll
            for (int k = 0; k < K * 3; k++) sh[k] = __ldg(shp + k);
        }
    };

    #pragma unroll 1
    for (int v = 0; v < vt.n_views; v++) {
        const int64_t o = (int64_t)v * a.n + i;
        Geom g;
        if (!cov_ok || !geometry(m, S, s_E[v], vt.v[v], s_lim[v], a.near_z, a.blur, g)) {
            a.radii[o] = 0;
            a.tiles_touched[o] = 0;
            continue;
        }
        float dx = m[0] - s_c[v][0], dy = m[1] - s_c[v][1], dz = m[2] - s_c[v][2];
        const float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= rn;
        dy *= rn;
        dz *= rn;
        load_sh();
        float Y[K];
        sh_basis<DEG>(dx, dy, dz, Y);
        float col[3];
        #pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            float acc = 0.5f;
            #pragma unroll
            for (int k = 0; k < K; k++) acc += sh[3 * k + ch] * Y[k];
            col[ch] = fmaxf(acc, 0.0f);
        }
        // the 2D mean to ~1e-7 px: camera point and projection in double-FP32
        const float *E = s_E[v];
        float xh, xl, yh, yl, zh, zl;
        dot3_plus(E + 0, m, E[3], xh, xl);
        dot3_plus(E + 4, m, E[7], yh, yl);
        dot3_plus(E + 8, m, E[11], zh, zl);
        const ViewInfo &V = vt.v[v];
        const float du = pixel_remainder(V.fx, xh, xl, zh, zl, V.cx, g.u);
        const float dv = pixel_remainder(V.fy, yh, yl, zh, zl, V.cy, g.v);
        const uint32_t r0 = (uint32_t)g.x0 | ((uint32_t)g.y0 << 16);
        const uint32_t r1 = (uint32_t)g.x1 | ((uint32_t)g.y1 << 16);
        const float A2 = __fdiv_rn(__fmul_rn(kNegHalfLog2e, g.cc), g.det);
        const float B2 = __fdiv_rn(__fmul_rn(kLog2eF, g.cb), g.det);
        const float C2 = __fdiv_rn(__fmul_rn(kNegHalfLog2e, g.ca), g.det);
        a.rec[3 * o + 0] = make_float4(g.u, g.v, g.z, log2o);
        a.rec[3 * o + 1] = make_float4(A2, B2, C2, du);
        a.rec[3 * o + 2] = make_float4(col[0], col[1], col[2], dv);
        a.rect[o] = make_uint2(r0, r1);
        a.radii[o] = g.radius;
        // the tiles the splat can reach: the kept bits of a rectangle of up to
        // 64 tiles (written only for drawn records), else the whole rectangle
        const int w = g.x1 - g.x0 + 1, h = g.y1 - g.y0 + 1;
        uint32_t touched = (uint32_t)(w * h);
        if (w * h <= 64) {
            const unsigned long long mask =
                tile_keep_mask(g.u, g.v, du, dv, log2o, A2, B2, C2, g.x0, g.y0, w, h, vt.v[v].tile_w, vt.v[v].tile_h);
            a.tile_mask[o] = mask;
            touched = (uint32_t)__popcll(mask);
        }
        a.tiles_touched[o] = touched;
    }
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_project(const gs_params_t *params, const gs_view_t *views, const float *viewmats,
                                  int32_t n_views, const gs_options_t *opt, gs_projected_t *out, void *stream)
{
    if (!params || !viewmats || !opt || !out) return GS_ERR_INVALID_ARG;
    if (params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (params->n == 0) return GS_OK;
    if (!params->means || !params->log_scales || !params->quats || !params->opacity_logit || !params->sh ||
        !out->rec || !out->rect || !out->radii || !out->tiles_touched || !out->tile_mask)
        return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(out->rect) & 7) || (reinterpret_cast<uintptr_t>(out->tile_mask) & 7))
        return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(out->rec) & 15) || (reinterpret_cast<uintptr_t>(params->quats) & 15))
        return GS_ERR_INVALID_ARG;
    if ((params->sh_degree == 1 || params->sh_degree == 3) && (reinterpret_cast<uintptr_t>(params->sh) & 15))
        return GS_ERR_INVALID_ARG;
    ProjectArgs a;
    a.means = params->means;
    a.log_scales = params->log_scales;
    a.quats = params->quats;
    a.opacity_logit = params->opacity_logit;
    a.sh = params->sh;
    a.viewmats = viewmats;
    a.n = params->n;
    a.near_z = opt->near_z;
    a.blur = opt->blur;
    a.rec = reinterpret_cast<float4 *>(out->rec);
    a.rect = reinterpret_cast<uint2 *>(out->rect);
    a.radii = out->radii;
    a.tiles_touched = out->tiles_touched;
    a.tile_mask = reinterpret_cast<unsigned long long *>(out->tile_mask);
    const int threads = 128;
    const unsigned blocks = (unsigned)((params->n + threads - 1) / threads);
    cudaStream_t s = as_stream(stream);
    switch (params->sh_degree) {
    case 0: project_kernel<0><<<blocks, threads, 0, s>>>(a, vt); break;
    case 1: project_kernel<1><<<blocks, threads, 0, s>>>(a, vt); break;
    case 2: project_kernel<2><<<blocks, threads, 0, s>>>(a, vt); break;
    default: project_kernel<3><<<blocks, threads, 0, s>>>(a, vt); break;
    }
    return launch_status();
}

extern "C" gs_status_t gs_layout(const gs_view_t *views, int32_t n_views, int64_t *n_tiles_total,
                                 int64_t *n_pixels_total)
{
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    if (n_tiles_total) *n_tiles_total = vt.n_tiles_total;
    if (n_pixels_total) *n_pixels_total = vt.n_pix_total;
    return GS_OK;
}

extern "C" const char *gs_version(void) { return "gs-sm103a 0.2"; }

extern "C" gs_status_t gs_get_device_status(const uint32_t *status_dev, uint32_t *status_host, void *stream)
{
    if (!status_dev || !status_host) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (cudaMemcpyAsync(status_host, status_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GS_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" size_t gs_workspace_size(int32_t op, int64_t n, int32_t n_views, int64_t pair_capacity, int64_t n_pixels)
{
    if (n < 0 || n_views < 0 || pair_capacity < 0 || n_pixels < 0) return 0;
    switch (op) {
    case GS_OP_BIN_SORT: return gs_bin_sort_workspace_size(n * n_views, pair_capacity, 0);
    case GS_OP_GRAD2D: return gs_grad2d_size(n, n_views);
    case GS_OP_SSIM: return gs_ssim_workspace_size(n_pixels);
    case GS_OP_SELECT: return gs_select_workspace_size(n);
    case GS_OP_SPATIAL_ORDER: return gs_spatial_order_workspace_size(n);
    case GS_OP_CHECK_LOOKBACK: return gs_check_lookback_timeout_workspace_size();
    default: return 0;
    }
}

extern "C" const char *gs_status_string(gs_status_t s)
{
    switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_CAPACITY: return "pair capacity exceeded";
    case GS_ERR_TIMEOUT: return "bounded wait expired";
    case GS_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}
