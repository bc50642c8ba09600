/*
 * gs_oracle.c -- plain, slow CPU oracle for the differentiable Gaussian
 * splatting hot path of TAMBRIDGE (arXiv 2405.19614).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path; both are
 * written independently from the paper's equations and the readings of them
 * listed in the design notes.
 *
 * What it computes (paper sections / equations cited per function):
 *   - FP32 geometry (the binning contract): camera transform, EWA 2D
 *     covariance, support radius, tile rectangle, depth key.  Sec. 3.4
 *     "Projection" (mu2D = K E_t mu / d, r2D = f r / d), generalised to the
 *     anisotropic EWA footprint of the rasteriser the paper uses (Sec. 4.1).
 *   - Binning: per-tile lists in front-to-back order (Sec. 3.4,
 *     "Differentiable Rasterization": Gaussians sorted front to back).
 *   - FP64 compositing of colour, depth and border mask: the C(p), D(p) and
 *     M_b(p) equations of Sec. 3.4 and Sec. 3.3.
 *   - FP64 reverse mode of the above, down to means, log-scales, quaternions,
 *     opacity logits, SH coefficients and the camera's SE(3) twist.
 *   - L1 rendering losses and the filter gate G(p) (Sec. 3.3, Sec. 3.4 L_m).
 *   - The keypoint re-projection loss L_rpj (Eq. lba, Sec. 3.2).
 *   - Adam (the gradient-based optimiser; Sec. 3.4 leaves it unnamed).
 *   - The SE(3) exponential used for the pose twist.
 *
 * Precision: FP64 everywhere except what decides tile membership and order
 * (the FP32 operation order written out in orc_geom_one()) and the alpha skip
 * and clamp decisions (the FP32 operation order of orc_blend_records() and
 * orc_blend_l2()): round to nearest, no contraction (build with
 * -ffp-contract=off).  Single threaded on purpose.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* A camera: pinhole intrinsics, image size and the world -> camera pose.
 * Inputs arrive as FP64; the FP32 geometry rounds them to float (exact for
 * float32-valued inputs, which is what the CUDA path receives). */
typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
    double viewmat[12]; /* row-major 3x4 world -> camera [R | t] */
} orc_view_t;

/* ------------------------------------------------------------------------ */
/* FP32 geometry                                                            */
/* ------------------------------------------------------------------------ */

/* exp used inside the FP32 geometry: Cody-Waite reduction by ln2 split into a
 * 15-bit head and a tail, then the degree-7 Taylor polynomial of e^r in Horner
 * form with fused multiply-adds, then an exact scaling by 2^k.  The argument
 * is clamped to [-80, 80] so the result stays a normal float.  Every step is a
 * single correctly rounded FP32 operation, so any IEEE implementation of the
 * same steps returns the same bits. */
float orc_geom_expf(float x)
{
    if (x > 80.0f) x = 80.0f;
    if (x < -80.0f) x = -80.0f;
    float k = rintf(x * 0x1.715476p+0f);
    float r = fmaf(-k, 0x1.62e4p-1f, x);
    r = fmaf(-k, 0x1.7f7d1cp-20f, r);
    float p = 0x1.a01a02p-13f;       /* 1/7! */
    p = fmaf(p, r, 0x1.6c16c2p-10f); /* 1/6! */
    p = fmaf(p, r, 0x1.111112p-7f);  /* 1/5! */
    p = fmaf(p, r, 0x1.555556p-5f);  /* 1/4! */
    p = fmaf(p, r, 0x1.555556p-3f);  /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    if (p != p) return p;
    int ki = (int)k;
    union { uint32_t u; float f; } s;
    s.u = (uint32_t)(ki + 127) << 23;
    return p * s.f;
}

typedef struct {
    int32_t radius;
    int32_t x0, y0, x1, y1; /* inclusive tile rectangle */
    float u, v, z;
    float ca, cb, cc, det; /* 2D covariance (with the blur) and its determinant */
    int footprint;         /* u, v, z, ca, cb, cc, det are set (touching a tile or not) */
} orc_geom_t;

/* Geometry of one Gaussian in one view, FP32.  Returns 1 if the Gaussian
 * touches at least one tile, else 0.  The operation order below is the
 * contract; parentheses show the order of every addition. */
static int orc_geom_one(const double md[3], const double lsd[3], const double qd[4],
                        const orc_view_t *V, float near_z, float blur, int tw,
                        int th, orc_geom_t *g)
{
    float m[3], ls[3], q[4], E[12];
    g->footprint = 0;
    for (int i = 0; i < 3; i++) {
        m[i] = (float)md[i];
        ls[i] = (float)lsd[i];
    }
    for (int i = 0; i < 4; i++) q[i] = (float)qd[i];
    for (int i = 0; i < 12; i++) E[i] = (float)V->viewmat[i];
    const float Vfx = (float)V->fx, Vfy = (float)V->fy, Vcx = (float)V->cx, Vcy = (float)V->cy;
    /* camera-space mean p = R mu + t */
    float x = ((E[0] * m[0] + E[1] * m[1]) + E[2] * m[2]) + E[3];
    float y = ((E[4] * m[0] + E[5] * m[1]) + E[6] * m[2]) + E[7];
    float z = ((E[8] * m[0] + E[9] * m[1]) + E[10] * m[2]) + E[11];
    if (!(z > near_z)) return 0;

    /* normalised quaternion (w, x, y, z) */
    float nq = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(nq > 0.0f)) return 0;
    float sq = sqrtf(nq);
    float w = q[0] / sq, a = q[1] / sq, b = q[2] / sq, c = q[3] / sq;

    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (b * b + c * c);
    R[0][1] = 2.0f * (a * b - w * c);
    R[0][2] = 2.0f * (a * c + w * b);
    R[1][0] = 2.0f * (a * b + w * c);
    R[1][1] = 1.0f - 2.0f * (a * a + c * c);
    R[1][2] = 2.0f * (b * c - w * a);
    R[2][0] = 2.0f * (a * c - w * b);
    R[2][1] = 2.0f * (b * c + w * a);
    R[2][2] = 1.0f - 2.0f * (a * a + b * b);

    float s[3] = {orc_geom_expf(ls[0]), orc_geom_expf(ls[1]), orc_geom_expf(ls[2])};
    float M[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[i][j] = R[i][j] * s[j];
    float S[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++) {
            S[i][j] = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2];
            S[j][i] = S[i][j];
        }

    /* perspective Jacobian with the tangent clamped to 1.3x the half field of view */
    float limx = 1.3f * ((0.5f * (float)V->width) / Vfx);
    float limy = 1.3f * ((0.5f * (float)V->height) / Vfy);
    float xz = x / z, yz = y / z;
    xz = fminf(limx, fmaxf(-limx, xz));
    yz = fminf(limy, fmaxf(-limy, yz));
    float tx = xz * z, ty = yz * z;
    float z2 = z * z;
    float J00 = Vfx / z, J02 = -((Vfx * tx) / z2);
    float J11 = Vfy / z, J12 = -((Vfy * ty) / z2);

    /* T = J W, W = camera rotation */
    float T[2][3];
    for (int j = 0; j < 3; j++) {
        T[0][j] = J00 * E[0 + j] + J02 * E[8 + j];
        T[1][j] = J11 * E[4 + j] + J12 * E[8 + j];
    }
    /* U = T S */
    float U[2][3];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++)
            U[i][j] = (T[i][0] * S[0][j] + T[i][1] * S[1][j]) + T[i][2] * S[2][j];
    float ca = ((U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2]) + blur;
    float cb = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2];
    float cc = ((U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2]) + blur;

    float det = ca * cc - cb * cb;
    if (!(det > 0.0f)) return 0;
    float mid = 0.5f * (ca + cc);
    float disc = mid * mid - det;
    float lam = mid + sqrtf(fmaxf(disc, 0.0f));
    float rad = ceilf(3.0f * sqrtf(lam));

    float u = (Vfx * x) / z + Vcx;
    float v = (Vfy * y) / z + Vcy;
    if (!(fabsf(u) < 0x1p24f && fabsf(v) < 0x1p24f && rad < 0x1p24f)) return 0;
    g->u = u;
    g->v = v;
    g->z = z;
    g->ca = ca;
    g->cb = cb;
    g->cc = cc;
    g->det = det;
    g->footprint = 1;

    int ntx = (V->width + tw - 1) / tw, nty = (V->height + th - 1) / th;
    float fx0 = floorf((u - rad) / (float)tw), fx1 = floorf((u + rad) / (float)tw);
    float fy0 = floorf((v - rad) / (float)th), fy1 = floorf((v + rad) / (float)th);
    fx0 = fmaxf(fx0, 0.0f);
    fy0 = fmaxf(fy0, 0.0f);
    fx1 = fminf(fx1, (float)(ntx - 1));
    fy1 = fminf(fy1, (float)(nty - 1));
    if (!(fx0 <= fx1 && fy0 <= fy1)) return 0;

    g->radius = (int32_t)rad;
    g->x0 = (int32_t)fx0;
    g->y0 = (int32_t)fy0;
    g->x1 = (int32_t)fx1;
    g->y1 = (int32_t)fy1;
    return 1;
}

/* Batched geometry: out arrays are [n_views * n].  rect = (x0, y0, x1, y1) or
 * (0, 0, -1, -1) for an untouched Gaussian; radius 0 marks it. */
void orc_project_geom(int32_t n_views, const orc_view_t *views, int64_t n,
                      const double *means, const double *log_scales,
                      const double *quats, float near_z, float blur, int32_t tw,
                      int32_t th, int32_t *radius, int32_t *rect, float *uvz,
                      uint32_t *tiles_touched)
{
    for (int32_t v = 0; v < n_views; v++)
        for (int64_t i = 0; i < n; i++) {
            int64_t o = (int64_t)v * n + i;
            orc_geom_t g;
            if (orc_geom_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, &views[v],
                             near_z, blur, tw, th, &g)) {
                radius[o] = g.radius;
                rect[4 * o + 0] = g.x0;
                rect[4 * o + 1] = g.y0;
                rect[4 * o + 2] = g.x1;
                rect[4 * o + 3] = g.y1;
                uvz[3 * o + 0] = g.u;
                uvz[3 * o + 1] = g.v;
                uvz[3 * o + 2] = g.z;
                tiles_touched[o] = (uint32_t)((g.x1 - g.x0 + 1) * (g.y1 - g.y0 + 1));
            } else {
                radius[o] = 0;
                rect[4 * o + 0] = 0;
                rect[4 * o + 1] = 0;
                rect[4 * o + 2] = -1;
                rect[4 * o + 3] = -1;
                uvz[3 * o + 0] = uvz[3 * o + 1] = uvz[3 * o + 2] = 0.0f;
                tiles_touched[o] = 0;
            }
        }
}

/* ------------------------------------------------------------------------ */
/* FP32 alpha decisions                                                     */
/* ------------------------------------------------------------------------ */

/* The compositing's two alpha decisions (skip an entry when alpha < 1/255,
 * clamp alpha at 0.99) are taken, on both sides, on one FP32 value: the
 * base-2 logarithm of the raw alpha o exp(-1/2 d^T conic d) of Eq. gauss,
 *   l2 = log2 o + A' dx^2 + dy (B' dx + C' dy),
 *   (A', B', C') = -log2(e) (A/2, B, C/2),  d = 2D mean - pixel centre,
 * evaluated by the fixed sequence of correctly rounded FP32 operations below
 * from a per-(view, Gaussian) record that is itself such a sequence on the
 * FP32 geometry: the decisions are then reproducible bit for bit, and the
 * FP64 image takes them from here, as it takes tile membership from the FP32
 * geometry.  The values blended stay FP64. */

/* log2 of y >= 1: y = m 2^e with m in (sqrt(1/2), sqrt(2)], log2 m =
 * (2/ln 2) atanh(s) with s = (m - 1)/(m + 1), by the odd series
 * s (C1 + s^2 (C3 + s^2 (C5 + s^2 (C7 + s^2 C9)))), C_k = 2/(k ln 2), in Horner
 * form with fused multiply-adds (|s| <= 0.172: the next term is below 1e-9
 * relative). */
float orc_geom_log2f(float y)
{
    union { float f; uint32_t u; } b;
    b.f = y;
    int e = (int)((b.u >> 23) & 0xffu) - 127;
    b.u = (b.u & 0x7fffffu) | 0x3f800000u;
    float m = b.f;
    if (m > 0x1.6a09e6p+0f) { /* sqrt(2) rounded to FP32 */
        m = m * 0.5f;
        e += 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = 0x1.484b14p-2f;       /* 2/(9 ln 2) */
    p = fmaf(p, s2, 0x1.a61762p-2f); /* 2/(7 ln 2) */
    p = fmaf(p, s2, 0x1.2776c6p-1f); /* 2/(5 ln 2) */
    p = fmaf(p, s2, 0x1.ec709ep-1f); /* 2/(3 ln 2) */
    p = fmaf(p, s2, 0x1.715476p+1f); /* 2/ln 2 */
    return (float)e + s * p;
}

/* Error-free transformations: a + b = s + e and a b = p + e exactly. */
static void orc_two_sum(float a, float b, float *s, float *e)
{
    float ss = a + b;
    float bb = ss - a;
    *e = (a - (ss - bb)) + (b - bb);
    *s = ss;
}

static void orc_two_prod(float a, float b, float *p, float *e)
{
    float pp = a * b;
    *e = fmaf(a, b, -pp);
    *p = pp;
}

/* r0 m0 + r1 m1 + r2 m2 + t as hi + lo; hi equals the geometry's coordinate. */
static void orc_dot3_plus(const float *r, const float *m, float t, float *hi, float *lo)
{
    float s, l, p, e, es;
    orc_two_prod(r[0], m[0], &s, &l);
    orc_two_prod(r[1], m[1], &p, &e);
    orc_two_sum(s, p, &s, &es);
    l = l + (e + es);
    orc_two_prod(r[2], m[2], &p, &e);
    orc_two_sum(s, p, &s, &es);
    l = l + (e + es);
    orc_two_sum(s, t, &s, &es);
    l = l + es;
    *hi = s;
    *lo = l;
}

/* (f x / z + c) - ref for x = xh + xl, z = zh + zl, in double-FP32. */
static float orc_pixel_remainder(float f, float xh, float xl, float zh, float zl, float c, float ref)
{
    float q = xh / zh;
    float r = fmaf(-q, zh, xh) + (xl - q * zl);
    float ql = r / zh;
    float m, me, s, se;
    orc_two_prod(f, q, &m, &me);
    float ml = me + f * ql;
    orc_two_sum(m, c, &s, &se);
    return (s - ref) + (se + ml);
}

#define ORC_NEG_HALF_LOG2E (-0x1.715476p-1f) /* -log2(e)/2 rounded to FP32 */
#define ORC_LOG2E_F (0x1.715476p+0f)         /* log2(e) rounded to FP32 */
#define ORC_L2_ALPHA_MIN (-0x1.ffa37cp+2f)   /* log2(1/255) rounded to FP32 */
#define ORC_L2_ALPHA_MAX (-0x1.db1f34p-7f)   /* log2(0.99) rounded to FP32 */

/* Decision records [n_views * n, 8] of every (view, Gaussian) with a 2D
 * footprint (in front of the near plane, positive definite covariance; drawn
 * or not): (u, v, du, dv, log2 o, A', B', C'), zeros elsewhere.  u, v are the
 * geometry's; du, dv the remainders of the 2D mean in double-FP32 (camera
 * point by compensated dot products, then f x / z + c); log2 o =
 * -log2(1 + exp(-logit)) with the geometry's exp and the log2 above;
 * A' = (-log2(e)/2 c) / det, B' = (log2(e) b) / det, C' = (-log2(e)/2 a) / det
 * for the 2D covariance (a, b, c) and its determinant. */
void orc_blend_records(int32_t n_views, const orc_view_t *views, int64_t n, const double *means,
                       const double *log_scales, const double *quats, const double *opacity_logit,
                       float near_z, float blur, int32_t tw, int32_t th, float *drec)
{
    for (int32_t v = 0; v < n_views; v++) {
        const orc_view_t *V = &views[v];
        float E[12];
        for (int k = 0; k < 12; k++) E[k] = (float)V->viewmat[k];
        for (int64_t i = 0; i < n; i++) {
            float *r = drec + 8 * ((int64_t)v * n + i);
            for (int k = 0; k < 8; k++) r[k] = 0.0f;
            orc_geom_t g;
            orc_geom_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, V, near_z, blur, tw, th, &g);
            if (!g.footprint) continue;
            float m[3] = {(float)means[3 * i], (float)means[3 * i + 1], (float)means[3 * i + 2]};
            float xh, xl, yh, yl, zh, zl;
            orc_dot3_plus(E + 0, m, E[3], &xh, &xl);
            orc_dot3_plus(E + 4, m, E[7], &yh, &yl);
            orc_dot3_plus(E + 8, m, E[11], &zh, &zl);
            r[0] = g.u;
            r[1] = g.v;
            r[2] = orc_pixel_remainder((float)V->fx, xh, xl, zh, zl, (float)V->cx, g.u);
            r[3] = orc_pixel_remainder((float)V->fy, yh, yl, zh, zl, (float)V->cy, g.v);
            float l = (float)opacity_logit[i];
            r[4] = -orc_geom_log2f(1.0f + orc_geom_expf(-l));
            r[5] = (ORC_NEG_HALF_LOG2E * g.cc) / g.det;
            r[6] = (ORC_LOG2E_F * g.cb) / g.det;
            r[7] = (ORC_NEG_HALF_LOG2E * g.ca) / g.det;
        }
    }
}

/* Keep-mask of the w x h <= 64 tiles of a rectangle from (x0, y0) for a
 * decision record r: bit j * w + i is set when the splat may reach alpha >=
 * 1/255 at a pixel of tile (x0 + i, y0 + j).  With d = pixel - mean and
 * q = P dx^2 + 2 B dx dy + Q dy^2, (P, B, Q) = -(A', B'/2, C'), log2 of the raw
 * alpha is log2 o - q, so such pixels lie in the ellipse q <= K, K = log2 o -
 * log2(1/255) + margin, margin = 1.5e-3 + 3.2e-5 (sqrt(PQ) + |B|)^2 / D,
 * D = PQ - B^2 (twice the FP32 error bound of the per-pixel evaluation inside
 * the ellipse).  Per tile row (pixel centres y in [a, b]) the ellipse's points
 * form an x-interval, whose ends are the ellipse's extreme points x = +-X,
 * X = sqrt(K Q / D), at y = -+B X / Q when those lie in [a, b], else the
 * crossings of the band's edge y = c: x = (-B c +- sqrt(P K - D c^2)) / P.  A
 * tile is kept when its pixel centres' x-range meets the interval widened by
 * 2e-3 + 2e-5 X.  FP32, in this operation order. */
uint64_t orc_tile_mask(const float *r, int x0, int y0, int w, int h, int tw, int th)
{
    float u = r[0], v = r[1], du = r[2], dv = r[3], l2o = r[4];
    float P = -r[5], Q = -r[7], B = -0.5f * r[6];
    float D = P * Q - B * B;
    if (!(D > 0.0f)) return ~(uint64_t)0 >> (64 - w * h);
    float rr = sqrtf(P * Q) + fabsf(B);
    float K = (l2o - ORC_L2_ALPHA_MIN) + (1.5e-3f + (3.2e-5f * (rr * rr)) / D);
    if (!(K > 0.0f)) return 0;
    float X = sqrtf((K * Q) / D);
    float yR = (-B * X) / Q, yL = -yR;
    float delta = 2e-3f + 2e-5f * X;
    float PK = P * K;
    uint64_t mask = 0;
    for (int j = 0; j < h; j++) {
        float cy0 = (float)((y0 + j) * th) + 0.5f, cy1 = cy0 + (float)(th - 1);
        float a = (cy0 - v) - dv, b = (cy1 - v) - dv;
        float xr, xl;
        if (yR >= a && yR <= b) {
            xr = X;
        } else {
            float c = yR > b ? b : a;
            float disc = PK - (D * c) * c;
            if (!(disc >= 0.0f)) continue;
            xr = ((-B * c) + sqrtf(disc)) / P;
        }
        if (yL >= a && yL <= b) {
            xl = -X;
        } else {
            float c = yL > b ? b : a;
            float disc = PK - (D * c) * c;
            if (!(disc >= 0.0f)) continue;
            xl = ((-B * c) - sqrtf(disc)) / P;
        }
        float lo = xl - delta, hi = xr + delta;
        for (int i = 0; i < w; i++) {
            float cx0 = (float)((x0 + i) * tw) + 0.5f, cx1 = cx0 + (float)(tw - 1);
            float e0 = (cx0 - u) - du, e1 = (cx1 - u) - du;
            if (lo <= e1 && e0 <= hi) mask |= (uint64_t)1 << (j * w + i);
        }
    }
    return mask;
}

/* Tiles each drawn (view, Gaussian) keeps: for rectangles of up to 64 tiles
 * the set bits of orc_tile_mask, else every tile (mask 0); kept [.] receives
 * the number kept.  rect, drec as orc_project_geom and orc_blend_records give
 * them. */
void orc_tile_cull(int32_t n_views, const orc_view_t *views, int64_t n, const float *drec, const int32_t *rect,
                   int32_t tw, int32_t th, uint64_t *mask, uint32_t *kept)
{
    (void)views;
    for (int64_t o = 0; o < (int64_t)n_views * n; o++) {
        int32_t x0 = rect[4 * o], y0 = rect[4 * o + 1], x1 = rect[4 * o + 2], y1 = rect[4 * o + 3];
        mask[o] = 0;
        if (x1 < x0 || y1 < y0) {
            kept[o] = 0;
            continue;
        }
        int w = x1 - x0 + 1, h = y1 - y0 + 1;
        if (w * h <= 64) {
            mask[o] = orc_tile_mask(drec + 8 * o, x0, y0, w, h, tw, th);
            uint32_t c = 0;
            for (uint64_t m = mask[o]; m; m &= m - 1) c++;
            kept[o] = c;
        } else {
            kept[o] = (uint32_t)(w * h);
        }
    }
}

/* l2 of a decision record at pixel (px, py), sampled at its centre. */
static float orc_blend_l2(const float *r, int px, int py)
{
    float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
    float dx = (r[0] - sx) + r[2];
    float base = fmaf(r[5] * dx, dx, r[4]);
    float bdx = r[6] * dx;
    float dy = (r[1] - sy) + r[3];
    return fmaf(dy, fmaf(r[7], dy, bdx), base);
}

/* l2 for m (record, pixel) pairs, for the tests of this arithmetic. */
void orc_blend_l2_many(int64_t m, const float *drec, const int32_t *px, const int32_t *py, float *out)
{
    for (int64_t k = 0; k < m; k++) out[k] = orc_blend_l2(drec + 8 * k, px[k], py[k]);
}

/* ------------------------------------------------------------------------ */
/* Binning: per-tile lists, front to back                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t key;
    uint32_t val;
} orc_pair_t;

static int orc_pair_cmp(const void *pa, const void *pb)
{
    const orc_pair_t *a = (const orc_pair_t *)pa, *b = (const orc_pair_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

/* Number of (Gaussian, tile) pairs. */
int64_t orc_count_pairs(int64_t total, const uint32_t *tiles_touched)
{
    int64_t k = 0;
    for (int64_t i = 0; i < total; i++) k += tiles_touched[i];
    return k;
}

/* Builds every (Gaussian, tile) pair with key (global tile id << 32) | bits(z)
 * and value = Gaussian index, then orders them by (key, Gaussian index): tiles
 * ascending, and within a tile front to back with ties broken by index.  The
 * tiles of a rectangle of up to 64 tiles are those its mask keeps (every tile
 * when mask is NULL).
 * ranges[2t], ranges[2t+1] = [start, end) of global tile t.
 * tile_base[v] = global id of view v's first tile. */
void orc_bin(int32_t n_views, const orc_view_t *views, int64_t n, int32_t tw,
             int32_t th, const int32_t *rect, const uint64_t *mask, const float *uvz,
             const int32_t *tile_base, int64_t n_tiles_total, uint64_t *keys,
             uint32_t *vals, uint32_t *ranges)
{
    (void)th; /* rectangles are already in tile units */
    int64_t total = (int64_t)n_views * n, k = 0;
    for (int64_t o = 0; o < total; o++) {
        int32_t x0 = rect[4 * o], y0 = rect[4 * o + 1], x1 = rect[4 * o + 2], y1 = rect[4 * o + 3];
        if (x1 >= x0 && y1 >= y0) k += (int64_t)(x1 - x0 + 1) * (y1 - y0 + 1);
    }
    orc_pair_t *pairs = (orc_pair_t *)malloc(sizeof(orc_pair_t) * (size_t)(k > 0 ? k : 1));
    int64_t w = 0;
    for (int32_t v = 0; v < n_views; v++) {
        int ntx = (views[v].width + tw - 1) / tw;
        for (int64_t i = 0; i < n; i++) {
            int64_t o = (int64_t)v * n + i;
            int32_t x0 = rect[4 * o], y0 = rect[4 * o + 1], x1 = rect[4 * o + 2], y1 = rect[4 * o + 3];
            if (x1 < x0 || y1 < y0) continue;
            union { float f; uint32_t u; } zb;
            zb.f = uvz[3 * o + 2];
            int rw = x1 - x0 + 1, rh = y1 - y0 + 1;
            int masked = mask != NULL && rw * rh <= 64;
            for (int32_t ty = y0; ty <= y1; ty++)
                for (int32_t tx = x0; tx <= x1; tx++) {
                    if (masked && !((mask[o] >> ((ty - y0) * rw + (tx - x0))) & 1)) continue;
                    uint64_t tile = (uint64_t)(tile_base[v] + ty * ntx + tx);
                    pairs[w].key = (tile << 32) | (uint64_t)zb.u;
                    pairs[w].val = (uint32_t)i;
                    w++;
                }
        }
    }
    qsort(pairs, (size_t)w, sizeof(orc_pair_t), orc_pair_cmp);
    for (int64_t t = 0; t < n_tiles_total; t++) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (int64_t i = 0; i < w; i++) {
        keys[i] = pairs[i].key;
        vals[i] = pairs[i].val;
        uint32_t tile = (uint32_t)(pairs[i].key >> 32);
        if (i == 0 || (uint32_t)(pairs[i - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)i;
        if (i == w - 1 || (uint32_t)(pairs[i + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(i + 1);
    }
    free(pairs);
}

/* ------------------------------------------------------------------------ */
/* FP64 projection                                                          */
/* ------------------------------------------------------------------------ */

/* Real spherical harmonics up to degree 3 on the unit sphere (no Condon-
 * Shortley phase), normalised so that each function has unit L2 norm over the
 * sphere.  Constants are evaluated from their closed forms.  dY[k][c] is the
 * derivative of the polynomial form with respect to direction component c. */
static void orc_sh_basis(const double d[3], int deg, double Y[16], double dY[16][3])
{
    const double PI = 3.14159265358979323846;
    const double c0 = 0.5 / sqrt(PI);
    const double c1 = sqrt(3.0 / (4.0 * PI));
    const double c2a = 0.5 * sqrt(15.0 / PI), c2b = 0.25 * sqrt(5.0 / PI), c2c = 0.25 * sqrt(15.0 / PI);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * PI)), c3b = 0.5 * sqrt(105.0 / PI);
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * PI)), c3d = 0.25 * sqrt(7.0 / PI);
    const double c3e = 0.25 * sqrt(105.0 / PI);
    double x = d[0], y = d[1], z = d[2];
    memset(dY, 0, sizeof(double) * 16 * 3);
    Y[0] = c0;
    if (deg < 1) return;
    Y[1] = c1 * y; dY[1][1] = c1;
    Y[2] = c1 * z; dY[2][2] = c1;
    Y[3] = c1 * x; dY[3][0] = c1;
    if (deg < 2) return;
    Y[4] = c2a * x * y; dY[4][0] = c2a * y; dY[4][1] = c2a * x;
    Y[5] = c2a * y * z; dY[5][1] = c2a * z; dY[5][2] = c2a * y;
    Y[6] = c2b * (3.0 * z * z - 1.0); dY[6][2] = 6.0 * c2b * z;
    Y[7] = c2a * x * z; dY[7][0] = c2a * z; dY[7][2] = c2a * x;
    Y[8] = c2c * (x * x - y * y); dY[8][0] = 2.0 * c2c * x; dY[8][1] = -2.0 * c2c * y;
    if (deg < 3) return;
    Y[9] = c3a * y * (3.0 * x * x - y * y);
    dY[9][0] = 6.0 * c3a * x * y; dY[9][1] = c3a * (3.0 * x * x - 3.0 * y * y);
    Y[10] = c3b * x * y * z;
    dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
    Y[11] = c3c * y * (5.0 * z * z - 1.0);
    dY[11][1] = c3c * (5.0 * z * z - 1.0); dY[11][2] = 10.0 * c3c * y * z;
    Y[12] = c3d * z * (5.0 * z * z - 3.0);
    dY[12][2] = c3d * (15.0 * z * z - 3.0);
    Y[13] = c3c * x * (5.0 * z * z - 1.0);
    dY[13][0] = c3c * (5.0 * z * z - 1.0); dY[13][2] = 10.0 * c3c * x * z;
    Y[14] = c3e * z * (x * x - y * y);
    dY[14][0] = 2.0 * c3e * x * z; dY[14][1] = -2.0 * c3e * y * z; dY[14][2] = c3e * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3.0 * y * y);
    dY[15][0] = c3a * (3.0 * x * x - 3.0 * y * y); dY[15][1] = -6.0 * c3a * x * y;
}

void orc_sh_eval(const double *dirs, int64_t n, int32_t deg, double *Y_out)
{
    double Y[16], dY[16][3];
    int K = (deg + 1) * (deg + 1);
    for (int64_t i = 0; i < n; i++) {
        orc_sh_basis(dirs + 3 * i, deg, Y, dY);
        for (int k = 0; k < K; k++) Y_out[i * K + k] = Y[k];
    }
}

typedef struct {
    double p[3];
    double qn[4], qnorm;
    double Rq[3][3];
    double s[3];
    double M[3][3];
    double Sc[3][3]; /* camera-space 3D covariance W S W^T */
    int clampx, clampy;
    double limx, limy;
    double J[2][3];
    double cov[3]; /* a, b, c (including the blur) */
    double det;
    double conic[3];
    double uv[2];
    double opacity;
    double dirv[3], dirn, dir[3];
    double Y[16], dY[16][3];
    double color[3];
    int col_clamped[3];
} orc_p64_t;

static void orc_proj64(const double *m, const double *ls, const double *q, double ol,
                       const double *sh, int deg, const orc_view_t *V, double blur,
                       orc_p64_t *P)
{
    const double *E = V->viewmat;
    double W[3][3], t[3];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) W[i][j] = E[4 * i + j];
        t[i] = E[4 * i + 3];
    }
    double mu[3] = {m[0], m[1], m[2]};
    for (int i = 0; i < 3; i++) P->p[i] = W[i][0] * mu[0] + W[i][1] * mu[1] + W[i][2] * mu[2] + t[i];

    double qq[4] = {q[0], q[1], q[2], q[3]};
    P->qnorm = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    for (int i = 0; i < 4; i++) P->qn[i] = qq[i] / P->qnorm;
    double w = P->qn[0], a = P->qn[1], b = P->qn[2], c = P->qn[3];
    double (*R)[3] = P->Rq;
    R[0][0] = 1 - 2 * (b * b + c * c); R[0][1] = 2 * (a * b - w * c); R[0][2] = 2 * (a * c + w * b);
    R[1][0] = 2 * (a * b + w * c); R[1][1] = 1 - 2 * (a * a + c * c); R[1][2] = 2 * (b * c - w * a);
    R[2][0] = 2 * (a * c - w * b); R[2][1] = 2 * (b * c + w * a); R[2][2] = 1 - 2 * (a * a + b * b);
    for (int j = 0; j < 3; j++) P->s[j] = exp((double)ls[j]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) P->M[i][j] = R[i][j] * P->s[j];
    double S[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            S[i][j] = P->M[i][0] * P->M[j][0] + P->M[i][1] * P->M[j][1] + P->M[i][2] * P->M[j][2];
    double WS[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) WS[i][j] = W[i][0] * S[0][j] + W[i][1] * S[1][j] + W[i][2] * S[2][j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) P->Sc[i][j] = WS[i][0] * W[j][0] + WS[i][1] * W[j][1] + WS[i][2] * W[j][2];

    double x = P->p[0], y = P->p[1], z = P->p[2];
    P->limx = 1.3 * (0.5 * V->width / V->fx);
    P->limy = 1.3 * (0.5 * V->height / V->fy);
    double xz = x / z, yz = y / z;
    P->clampx = (xz < -P->limx || xz > P->limx);
    P->clampy = (yz < -P->limy || yz > P->limy);
    double tx = (P->clampx ? (xz < 0 ? -P->limx : P->limx) : xz) * z;
    double ty = (P->clampy ? (yz < 0 ? -P->limy : P->limy) : yz) * z;
    memset(P->J, 0, sizeof(P->J));
    P->J[0][0] = V->fx / z;
    P->J[0][2] = -V->fx * tx / (z * z);
    P->J[1][1] = V->fy / z;
    P->J[1][2] = -V->fy * ty / (z * z);
    double JS[2][3];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++)
            JS[i][j] = P->J[i][0] * P->Sc[0][j] + P->J[i][1] * P->Sc[1][j] + P->J[i][2] * P->Sc[2][j];
    double C2[2][2];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            C2[i][j] = JS[i][0] * P->J[j][0] + JS[i][1] * P->J[j][1] + JS[i][2] * P->J[j][2];
    P->cov[0] = C2[0][0] + blur;
    P->cov[1] = C2[0][1];
    P->cov[2] = C2[1][1] + blur;
    P->det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    P->conic[0] = P->cov[2] / P->det;
    P->conic[1] = -P->cov[1] / P->det;
    P->conic[2] = P->cov[0] / P->det;
    P->uv[0] = V->fx * x / z + V->cx;
    P->uv[1] = V->fy * y / z + V->cy;
    P->opacity = 1.0 / (1.0 + exp(-(double)ol));

    /* view direction from the camera centre c = -W^T t to the mean */
    double cc[3];
    for (int i = 0; i < 3; i++) cc[i] = -(W[0][i] * t[0] + W[1][i] * t[1] + W[2][i] * t[2]);
    for (int i = 0; i < 3; i++) P->dirv[i] = mu[i] - cc[i];
    P->dirn = sqrt(P->dirv[0] * P->dirv[0] + P->dirv[1] * P->dirv[1] + P->dirv[2] * P->dirv[2]);
    for (int i = 0; i < 3; i++) P->dir[i] = P->dirv[i] / P->dirn;
    orc_sh_basis(P->dir, deg, P->Y, P->dY);
    int K = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0;
        for (int k = 0; k < K; k++) acc += (double)sh[3 * k + ch] * P->Y[k];
        acc += 0.5;
        P->col_clamped[ch] = acc < 0.0;
        P->color[ch] = acc < 0.0 ? 0.0 : acc;
    }
}

/* FP64 per-(view, Gaussian) 2D quantities for every Gaussian that touches a
 * tile in that view.  Row layout of out [n_views*n, 16]:
 *   u, v, z, conicA, conicB, conicC, opacity, r, g, b, cov_a, cov_b, cov_c,
 *   clampx, clampy, valid. */
void orc_project64(int32_t n_views, const orc_view_t *views, int64_t n,
                   const double *means, const double *log_scales, const double *quats,
                   const double *opacity_logit, const double *sh, int32_t deg,
                   double blur, const int32_t *radius, double *out)
{
    int K = (deg + 1) * (deg + 1);
    for (int32_t v = 0; v < n_views; v++)
        for (int64_t i = 0; i < n; i++) {
            int64_t o = (int64_t)v * n + i;
            double *r = out + 16 * o;
            memset(r, 0, sizeof(double) * 16);
            if (radius[o] == 0) continue;
            orc_p64_t P;
            orc_proj64(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity_logit[i],
                       sh + (int64_t)3 * K * i, deg, &views[v], blur, &P);
            r[0] = P.uv[0]; r[1] = P.uv[1]; r[2] = P.p[2];
            r[3] = P.conic[0]; r[4] = P.conic[1]; r[5] = P.conic[2];
            r[6] = P.opacity;
            r[7] = P.color[0]; r[8] = P.color[1]; r[9] = P.color[2];
            r[10] = P.cov[0]; r[11] = P.cov[1]; r[12] = P.cov[2];
            r[13] = P.clampx; r[14] = P.clampy; r[15] = 1.0;
        }
}

/* ------------------------------------------------------------------------ */
/* FP64 compositing                                                         */
/* ------------------------------------------------------------------------ */

#define ORC_ALPHA_MAX 0.99
#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_T_MIN 1e-4

/* Flag bits for pixels whose result depends on a decision taken too close to
 * its threshold for FP32 and FP64 to be sure to agree. */
#define ORC_FLAG_ALPHA_MIN 1
#define ORC_FLAG_T_MIN 2
#define ORC_FLAG_ALPHA_MAX 4

typedef struct {
    double margin_alpha; /* test knob: also flag FP64 alphas within this relative margin of 1/255 or 0.99 */
    double margin_T;     /* extra relative band around 1e-4 added to the computed one */
} orc_margins_t;

static void orc_view_tiles(const orc_view_t *V, int tw, int th, int *ntx, int *nty)
{
    *ntx = (V->width + tw - 1) / tw;
    *nty = (V->height + th - 1) / th;
}

/* Bound on the relative error of the kernel's approximate 2^x (the GPU's
 * ex2.approx.ftz.f32): two units in the last place of FP32, 2^-22.  Measured
 * over every FP32 input in [-8, 0): at most 2^-22.73. */
#define ORC_EX2_REL 0x1p-22
/* The kernel rounds T (1 - alpha) to FP32 (relative error at most 2^-24) and
 * 1 - alpha, which is exact for alpha >= 1/2 and otherwise lies in (1/2, 1],
 * so that its rounding error is at most 2^-25 absolute. */
static double orc_t_round(double a) { return 0x1p-24 + (a < 0.5 ? 0x1p-25 / (1.0 - a) : 0.0); }
/* The kernel compares with 1e-4 rounded to FP32 (2.6e-9 relative below). */
#define ORC_T_CUT_REL 3e-9

/* Composites every pixel of every view front to back over its tile's list:
 *   alpha_i = min(0.99, o_i exp(-1/2 d^T conic d)), skipped if < 1/255;
 *   stop before blending i when T (1 - alpha_i) < 1e-4;
 *   C += c_i alpha_i T, D += z_i alpha_i T, T *= (1 - alpha_i); A = 1 - T.
 * Pixel (px, py) is sampled at (px + 0.5, py + 0.5).  Images are stored per
 * view at pix_base[v] + py * width + px.  n_contrib = number of list entries
 * consumed up to and including the last blended one.
 * The skip and clamp decisions are taken on the FP32 l2 of the decision
 * records drec (orc_blend_records); the alphas blended are the FP64 values.
 * The stop decision compares the FP64 T (1 - alpha) with 1e-4; a kernel that
 * computes T in FP32 from alphas min(0.99, 2^l2) (approximate exponential,
 * relative error below ORC_EX2_REL) may decide it the other way only when the
 * FP64 product lies within the relative deviation its alphas can accumulate:
 * per blended entry, alpha / (1 - alpha) times the known |l2 ln 2 - ln alpha|
 * of that evaluation (|ln(0.99f / 0.99)| where the clamp is in force) plus
 * ORC_EX2_REL, and the roundings of 1 - alpha and of the product
 * (orc_t_round).  Such pixels are flagged (ORC_FLAG_T_MIN) and slack [P, 4]
 * receives the blend weight alpha T of the entry at that decision, times its
 * largest colour channel and times its depth (a result that stops one entry
 * earlier or later differs by exactly that entry's contribution), and, for
 * every pixel, the accumulated relative band of its final T. */
void orc_render(int32_t n_views, const orc_view_t *views, int64_t n,
                const double *proj, const float *drec, int32_t tw, int32_t th, const int32_t *tile_base,
                const int64_t *pix_base, const uint32_t *vals, const uint32_t *ranges,
                orc_margins_t mg, double *rgb, double *depth, double *alpha,
                double *final_T, int32_t *n_contrib, int32_t *flags, double *slack)
{
    const double ln2 = 0.69314718055994530942;
    const double dev_clamp = fabs(log((double)0.99f / ORC_ALPHA_MAX));
    for (int32_t v = 0; v < n_views; v++) {
        const orc_view_t *V = &views[v];
        int ntx, nty;
        orc_view_tiles(V, tw, th, &ntx, &nty);
        for (int py = 0; py < V->height; py++)
            for (int px = 0; px < V->width; px++) {
                int64_t pix = pix_base[v] + (int64_t)py * V->width + px;
                int64_t tile = tile_base[v] + (py / th) * ntx + (px / tw);
                uint32_t b = ranges[2 * tile], e = ranges[2 * tile + 1];
                double T = 1.0, C[3] = {0, 0, 0}, D = 0.0, lnT_unc = 0.0;
                int32_t last = 0, fl = 0;
                double sx = px + 0.5, sy = py + 0.5;
                slack[4 * pix] = slack[4 * pix + 1] = slack[4 * pix + 2] = 0.0;
                for (uint32_t k = b; k < e; k++) {
                    int64_t o = (int64_t)v * n + vals[k];
                    const double *r = proj + 16 * o;
                    float l2 = orc_blend_l2(drec + 8 * o, px, py);
                    double dx = r[0] - sx, dy = r[1] - sy;
                    double power = -0.5 * (r[3] * dx * dx + r[5] * dy * dy) - r[4] * dx * dy;
                    double araw = r[6] * exp(power);
                    if (mg.margin_alpha > 0.0) {
                        if (fabs(log(araw / ORC_ALPHA_MAX)) <= mg.margin_alpha) fl |= ORC_FLAG_ALPHA_MAX;
                        double a0 = araw < ORC_ALPHA_MAX ? araw : ORC_ALPHA_MAX;
                        if (fabs(log(a0 / ORC_ALPHA_MIN)) <= mg.margin_alpha) fl |= ORC_FLAG_ALPHA_MIN;
                    }
                    if (l2 < ORC_L2_ALPHA_MIN) continue;
                    int clamp = l2 >= ORC_L2_ALPHA_MAX;
                    double a = clamp ? ORC_ALPHA_MAX : araw;
                    double dev = (clamp ? dev_clamp : fabs((double)l2 * ln2 - log(araw))) + ORC_EX2_REL;
                    double step_unc = a / (1.0 - a) * dev + orc_t_round(a);
                    double tT = T * (1.0 - a);
                    if (fabs(log(tT / ORC_T_MIN)) <= mg.margin_T + lnT_unc + step_unc + ORC_T_CUT_REL) {
                        fl |= ORC_FLAG_T_MIN;
                        double w = a * T, cm = r[7];
                        if (r[8] > cm) cm = r[8];
                        if (r[9] > cm) cm = r[9];
                        slack[4 * pix] = w;
                        slack[4 * pix + 1] = w * cm;
                        slack[4 * pix + 2] = w * r[2];
                    }
                    if (tT < ORC_T_MIN) break;
                    for (int ch = 0; ch < 3; ch++) C[ch] += r[7 + ch] * a * T;
                    D += r[2] * a * T;
                    T = tT;
                    lnT_unc += step_unc;
                    last = (int32_t)(k - b + 1);
                }
                for (int ch = 0; ch < 3; ch++) rgb[3 * pix + ch] = C[ch];
                depth[pix] = D;
                alpha[pix] = 1.0 - T;
                final_T[pix] = T;
                n_contrib[pix] = last;
                flags[pix] = fl;
                slack[4 * pix + 3] = lnT_unc;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* FP64 reverse mode                                                        */
/* ------------------------------------------------------------------------ */


/* Reverse mode of orc_render for given dL/dC [P,3], dL/dD [P], dL/dA [P].
 * Accumulates per-(view, Gaussian) 2D gradients into g2d [n_views*n, 10] with
 * columns: d u, d v, d conicA, d conicB, d conicC, d opacity, d r, d g, d b,
 * d z.  The blend weights are alpha_i T_i with T_i = prod_{j<i} (1 - alpha_j),
 * so with s = sum over later blended entries k of (c_k.gC + z_k gD) alpha_k T_k:
 *   dL/dalpha_i = T_i (c_i.gC + z_i gD) - s / (1 - alpha_i)
 *                 + gA T_final / (1 - alpha_i).
 * The skip and clamp decisions are orc_render's (on the FP32 l2 of drec); the
 * clamp alpha = min(0.99, o g) passes no gradient where it is active. */
void orc_render_bwd(int32_t n_views, const orc_view_t *views, int64_t n,
                    const double *proj, const float *drec, int32_t tw, int32_t th, const int32_t *tile_base,
                    const int64_t *pix_base, const uint32_t *vals, const uint32_t *ranges,
                    const double *dC, const double *dD, const double *dA, double *g2d)
{
    int64_t maxlen = 1;
    for (int32_t v = 0; v < n_views; v++) {
        int ntx, nty;
        orc_view_tiles(&views[v], tw, th, &ntx, &nty);
        for (int64_t t = tile_base[v]; t < tile_base[v] + (int64_t)ntx * nty; t++) {
            int64_t len = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
            if (len > maxlen) maxlen = len;
        }
    }
    uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)maxlen);
    double *al = (double *)malloc(sizeof(double) * (size_t)maxlen);
    double *Ti = (double *)malloc(sizeof(double) * (size_t)maxlen);
    double *gv = (double *)malloc(sizeof(double) * (size_t)maxlen);
    int *clp = (int *)malloc(sizeof(int) * (size_t)maxlen);
    for (int32_t v = 0; v < n_views; v++) {
        const orc_view_t *V = &views[v];
        int ntx, nty;
        orc_view_tiles(V, tw, th, &ntx, &nty);
        for (int py = 0; py < V->height; py++)
            for (int px = 0; px < V->width; px++) {
                int64_t pix = pix_base[v] + (int64_t)py * V->width + px;
                int64_t tile = tile_base[v] + (py / th) * ntx + (px / tw);
                uint32_t b = ranges[2 * tile], e = ranges[2 * tile + 1];
                double sx = px + 0.5, sy = py + 0.5;
                /* forward again, remembering the blended entries */
                int64_t nb = 0;
                double T = 1.0;
                for (uint32_t k = b; k < e; k++) {
                    int64_t o = (int64_t)v * n + vals[k];
                    const double *r = proj + 16 * o;
                    float l2 = orc_blend_l2(drec + 8 * o, px, py);
                    if (l2 < ORC_L2_ALPHA_MIN) continue;
                    double dx = r[0] - sx, dy = r[1] - sy;
                    double power = -0.5 * (r[3] * dx * dx + r[5] * dy * dy) - r[4] * dx * dy;
                    double g = exp(power);
                    double araw = r[6] * g;
                    int c = l2 >= ORC_L2_ALPHA_MAX;
                    double a = c ? ORC_ALPHA_MAX : araw;
                    double tT = T * (1.0 - a);
                    if (tT < ORC_T_MIN) break;
                    ids[nb] = vals[k];
                    al[nb] = a;
                    Ti[nb] = T;
                    gv[nb] = g;
                    clp[nb] = c;
                    nb++;
                    T = tT;
                }
                double Tf = T;
                double gC[3] = {dC[3 * pix], dC[3 * pix + 1], dC[3 * pix + 2]};
                double gD = dD[pix], gA = dA[pix];
                double s = 0.0;
                for (int64_t j = nb - 1; j >= 0; j--) {
                    int64_t o = (int64_t)v * n + ids[j];
                    const double *r = proj + 16 * o;
                    double *G = g2d + 10 * o;
                    double a = al[j], Tj = Ti[j];
                    double wgt = r[7] * gC[0] + r[8] * gC[1] + r[9] * gC[2] + r[2] * gD;
                    double da = Tj * wgt - s / (1.0 - a) + gA * Tf / (1.0 - a);
                    s += wgt * a * Tj;
                    for (int ch = 0; ch < 3; ch++) G[6 + ch] += gC[ch] * a * Tj;
                    G[9] += gD * a * Tj;
                    if (clp[j]) continue;
                    double g = gv[j];
                    G[5] += da * g;                 /* d opacity */
                    double dpow = da * r[6] * g;    /* dL/d power */
                    double dx = r[0] - sx, dy = r[1] - sy;
                    G[0] += dpow * (-r[3] * dx - r[4] * dy);
                    G[1] += dpow * (-r[5] * dy - r[4] * dx);
                    G[2] += -0.5 * dx * dx * dpow;  /* d conicA */
                    G[3] += -dx * dy * dpow;        /* d conicB */
                    G[4] += -0.5 * dy * dy * dpow;  /* d conicC */
                }
            }
    }
    free(ids);
    free(al);
    free(Ti);
    free(gv);
    free(clp);
}

static void m3_mul(const double A[3][3], const double B[3][3], double C[3][3])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) C[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
}

static void m3_transpose(const double A[3][3], double B[3][3])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) B[i][j] = A[j][i];
}

/* Reverse mode of the projection of one Gaussian in one view.  G = the 10 2D
 * gradients of orc_render_bwd.  Accumulates into the parameter gradients of
 * this Gaussian and into the view's twist gradient (rho, phi), taken at
 * xi = 0 for the pose Exp(xi) E_t. */
static void orc_proj64_bwd(const orc_p64_t *P, const double *sh, int deg,
                           const orc_view_t *V, const double G[10], double *g_mean,
                           double *g_ls, double *g_quat, double *g_ol, double *g_sh,
                           double *g_twist)
{
    const double *E = V->viewmat;
    double W[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) W[i][j] = E[4 * i + j];
    double x = P->p[0], y = P->p[1], z = P->p[2];
    double fx = V->fx, fy = V->fy;

    /* conic (A, B, C) = (c, -b, a) / det  ->  covariance (a, b, c) */
    double a = P->cov[0], b = P->cov[1], c = P->cov[2], det = P->det, d2 = det * det;
    double gA = G[2], gB = G[3], gCn = G[4];
    double ga = gA * (-c * c / d2) + gB * (b * c / d2) + gCn * (-b * b / d2);
    double gb = gA * (2.0 * b * c / d2) + gB * (-(det + 2.0 * b * b) / d2) + gCn * (2.0 * a * b / d2);
    double gc = gA * (-b * b / d2) + gB * (a * b / d2) + gCn * (-a * a / d2);

    /* Sigma2D = J Sc J^T + blur I */
    double G2[2][2] = {{ga, 0.5 * gb}, {0.5 * gb, gc}};
    const double (*J)[3] = P->J;
    double Gc[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 2; k++)
                for (int l = 0; l < 2; l++) acc += J[k][i] * G2[k][l] * J[l][j];
            Gc[i][j] = acc;
        }
    double gJ[2][3];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 2; k++)
                for (int l = 0; l < 3; l++) acc += G2[i][k] * J[k][l] * P->Sc[l][j];
            gJ[i][j] = 2.0 * acc;
        }

    /* camera-space point gradient */
    double gp[3] = {0.0, 0.0, 0.0};
    gp[2] += gJ[0][0] * (-fx / (z * z)) + gJ[1][1] * (-fy / (z * z));
    if (!P->clampx) {
        gp[0] += gJ[0][2] * (-fx / (z * z));
        gp[2] += gJ[0][2] * (2.0 * fx * x / (z * z * z));
    } else {
        double L = (x / z < 0) ? -P->limx : P->limx;
        gp[2] += gJ[0][2] * (fx * L / (z * z));
    }
    if (!P->clampy) {
        gp[1] += gJ[1][2] * (-fy / (z * z));
        gp[2] += gJ[1][2] * (2.0 * fy * y / (z * z * z));
    } else {
        double L = (y / z < 0) ? -P->limy : P->limy;
        gp[2] += gJ[1][2] * (fy * L / (z * z));
    }
    gp[0] += G[0] * fx / z;
    gp[2] += G[0] * (-fx * x / (z * z));
    gp[1] += G[1] * fy / z;
    gp[2] += G[1] * (-fy * y / (z * z));
    gp[2] += G[9];

    for (int i = 0; i < 3; i++) g_mean[i] += W[0][i] * gp[0] + W[1][i] * gp[1] + W[2][i] * gp[2];

    /* world covariance S = M M^T, M = Rq diag(s): Gw = W^T Gc W, dL/dM = 2 Gw M */
    double Wt[3][3], tmp[3][3], Gw[3][3], gM[3][3];
    m3_transpose(W, Wt);
    m3_mul(Wt, Gc, tmp);
    m3_mul(tmp, W, Gw);
    m3_mul(Gw, P->M, gM);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) gM[i][j] *= 2.0;
    double gR[3][3];
    for (int j = 0; j < 3; j++) {
        double gs = 0.0;
        for (int i = 0; i < 3; i++) {
            gs += gM[i][j] * P->Rq[i][j];
            gR[i][j] = gM[i][j] * P->s[j];
        }
        g_ls[j] += gs * P->s[j];
    }
    double w = P->qn[0], qa = P->qn[1], qb = P->qn[2], qc = P->qn[3];
    double gq[4];
    gq[0] = 2.0 * (-qc * gR[0][1] + qb * gR[0][2] + qc * gR[1][0] - qa * gR[1][2] - qb * gR[2][0] + qa * gR[2][1]);
    gq[1] = 2.0 * (qb * gR[0][1] + qc * gR[0][2] + qb * gR[1][0] - w * gR[1][2] + qc * gR[2][0] + w * gR[2][1])
            - 4.0 * qa * (gR[1][1] + gR[2][2]);
    gq[2] = 2.0 * (qa * gR[0][1] + w * gR[0][2] + qa * gR[1][0] + qc * gR[1][2] - w * gR[2][0] + qc * gR[2][1])
            - 4.0 * qb * (gR[0][0] + gR[2][2]);
    gq[3] = 2.0 * (-w * gR[0][1] + qa * gR[0][2] + w * gR[1][0] + qb * gR[1][2] + qa * gR[2][0] + qb * gR[2][1])
            - 4.0 * qc * (gR[0][0] + gR[1][1]);
    double dot = gq[0] * w + gq[1] * qa + gq[2] * qb + gq[3] * qc;
    for (int i = 0; i < 4; i++) g_quat[i] += (gq[i] - P->qn[i] * dot) / P->qnorm;

    /* opacity = sigmoid(logit) */
    *g_ol += G[5] * P->opacity * (1.0 - P->opacity);

    /* colour = max(0, sum_k sh_k Y_k(dir) + 0.5) */
    int K = (deg + 1) * (deg + 1);
    double gdir[3] = {0.0, 0.0, 0.0};
    for (int ch = 0; ch < 3; ch++) {
        if (P->col_clamped[ch]) continue;
        double gcol = G[6 + ch];
        for (int k = 0; k < K; k++) {
            g_sh[3 * k + ch] += P->Y[k] * gcol;
            for (int d = 0; d < 3; d++) gdir[d] += (double)sh[3 * k + ch] * gcol * P->dY[k][d];
        }
    }
    double dd = gdir[0] * P->dir[0] + gdir[1] * P->dir[1] + gdir[2] * P->dir[2];
    double gv[3];
    for (int i = 0; i < 3; i++) {
        gv[i] = (gdir[i] - P->dir[i] * dd) / P->dirn;
        g_mean[i] += gv[i];
    }

    if (!g_twist) return;
    /* p(xi) = p + rho + phi x p */
    g_twist[0] += gp[0];
    g_twist[1] += gp[1];
    g_twist[2] += gp[2];
    g_twist[3] += y * gp[2] - z * gp[1];
    g_twist[4] += z * gp[0] - x * gp[2];
    g_twist[5] += x * gp[1] - y * gp[0];
    /* Sc(xi) = Exp(phi) Sc Exp(phi)^T: dL/dphi = 2 (A23, A31, A12), A = Sc Gc - Gc Sc */
    double SG[3][3], GS[3][3];
    m3_mul(P->Sc, Gc, SG);
    m3_mul(Gc, P->Sc, GS);
    g_twist[3] += 2.0 * (SG[1][2] - GS[1][2]);
    g_twist[4] += 2.0 * (SG[2][0] - GS[2][0]);
    g_twist[5] += 2.0 * (SG[0][1] - GS[0][1]);
    /* camera centre c(xi) = c - W^T rho, and the SH direction depends on mu - c */
    for (int i = 0; i < 3; i++) g_twist[i] += W[i][0] * gv[0] + W[i][1] * gv[1] + W[i][2] * gv[2];
}

/* Chains per-(view, Gaussian) 2D gradients g2d [n_views*n, 10] to parameter
 * gradients (accumulated, +=) summed over views, and to each view's twist
 * gradient g_twist [n_views, 6] (+=, may be NULL). */
void orc_project_bwd(int32_t n_views, const orc_view_t *views, int64_t n,
                     const double *means, const double *log_scales, const double *quats,
                     const double *opacity_logit, const double *sh, int32_t deg, double blur,
                     const int32_t *radius, const double *g2d, double *g_means,
                     double *g_log_scales, double *g_quats, double *g_opacity_logit,
                     double *g_sh, double *g_twist)
{
    int K = (deg + 1) * (deg + 1);
    for (int32_t v = 0; v < n_views; v++)
        for (int64_t i = 0; i < n; i++) {
            int64_t o = (int64_t)v * n + i;
            if (radius[o] == 0) continue;
            orc_p64_t P;
            const double *shi = sh + (int64_t)3 * K * i;
            orc_proj64(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity_logit[i], shi, deg,
                       &views[v], blur, &P);
            orc_proj64_bwd(&P, shi, deg, &views[v], g2d + 10 * o, g_means + 3 * i,
                           g_log_scales + 3 * i, g_quats + 4 * i, g_opacity_logit + i,
                           g_sh + (int64_t)3 * K * i, g_twist ? g_twist + 6 * v : NULL);
        }
}

/* ------------------------------------------------------------------------ */
/* Losses                                                                   */
/* ------------------------------------------------------------------------ */

/* L = w_c/(3P) sum G |C - C^| + w_d/P sum G |D - D^| over all P pixels of the
 * batch, where the gate G(p) = [D^(p) > 0][D(p) > 0][A(p) > gamma] when
 * use_gate, else 1 (Sec. 3.3 filter gates, Sec. 3.4 L1 terms).  Writes
 * dL/dC, dL/dD (sign(0) = 0) and returns L. */
double orc_loss_l1(int64_t P, const double *rgb, const double *depth, const double *alpha,
                   const double *t_rgb, const double *t_depth, double w_c, double w_d,
                   int32_t use_gate, double gamma, double *dC, double *dD)
{
    double L = 0.0;
    for (int64_t p = 0; p < P; p++) {
        int gate = 1;
        if (use_gate) gate = (t_depth[p] > 0.0) && (depth[p] > 0.0) && (alpha[p] > gamma);
        for (int ch = 0; ch < 3; ch++) {
            double r = rgb[3 * p + ch] - (double)t_rgb[3 * p + ch];
            double sg = (r > 0) - (r < 0);
            L += gate ? w_c * fabs(r) / (3.0 * P) : 0.0;
            dC[3 * p + ch] = gate ? w_c * sg / (3.0 * P) : 0.0;
        }
        double r = depth[p] - (double)t_depth[p];
        double sg = (r > 0) - (r < 0);
        L += gate ? w_d * fabs(r) / (double)P : 0.0;
        dD[p] = gate ? w_d * sg / (double)P : 0.0;
    }
    return L;
}

/* Keypoint re-projection loss (Eq. lba): for map points P_i (world) observed at
 * u_i (pixels, same convention as the splat means), with the pose
 * Exp(xi) E_t:  L = (w/n) sum_i || u_i - pi(K, E_t, P_i) ||_2.  Points with
 * camera depth <= near_z are left out.  Writes dL/dxi at xi = 0 (+=) and
 * returns L.  view_ids (may be NULL) picks each point's view. */
double orc_reproj(int64_t n, const double *pts, const double *obs, const int32_t *view_ids,
                  const orc_view_t *views, double weight, double near_z, double *g_twist)
{
    double L = 0.0;
    for (int64_t i = 0; i < n; i++) {
        int32_t v = view_ids ? view_ids[i] : 0;
        const orc_view_t *V = &views[v];
        const double *E = V->viewmat;
        double p[3];
        for (int r = 0; r < 3; r++)
            p[r] = (double)E[4 * r] * pts[3 * i] + (double)E[4 * r + 1] * pts[3 * i + 1] +
                   (double)E[4 * r + 2] * pts[3 * i + 2] + (double)E[4 * r + 3];
        if (!(p[2] > near_z)) continue;
        double u = V->fx * p[0] / p[2] + V->cx, w = V->fy * p[1] / p[2] + V->cy;
        double rx = obs[2 * i] - u, ry = obs[2 * i + 1] - w;
        double nr = sqrt(rx * rx + ry * ry);
        L += weight * nr / (double)n;
        if (nr == 0.0 || !g_twist) continue;
        /* dL/dpi = -(w/n) r/|r|;  dpi/dp = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] */
        double gu = -weight * rx / (nr * n), gw = -weight * ry / (nr * n);
        double gp[3];
        gp[0] = gu * V->fx / p[2];
        gp[1] = gw * V->fy / p[2];
        gp[2] = -gu * V->fx * p[0] / (p[2] * p[2]) - gw * V->fy * p[1] / (p[2] * p[2]);
        double *g = g_twist + 6 * v;
        g[0] += gp[0];
        g[1] += gp[1];
        g[2] += gp[2];
        g[3] += p[1] * gp[2] - p[2] * gp[1];
        g[4] += p[2] * gp[0] - p[0] * gp[2];
        g[5] += p[0] * gp[1] - p[1] * gp[0];
    }
    return L;
}

/* ------------------------------------------------------------------------ */
/* Optimiser and pose                                                       */
/* ------------------------------------------------------------------------ */

/* One Adam step at step number t (1-based), in FP64. */
void orc_adam(int64_t n, double *param, const double *grad, double *m, double *v, double lr,
              double b1, double b2, double eps, int32_t t)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        param[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* SE(3) exponential of xi = (rho, phi): R = I + A [phi]x + B [phi]x^2,
 * t = (I + B [phi]x + C [phi]x^2) rho with A = sin th / th,
 * B = (1 - cos th) / th^2, C = (th - sin th) / th^3 (series near 0).
 * Writes out = Exp(xi) * E as a row-major 3x4 matrix. */
void orc_se3_exp_apply(const double *xi, const double *E, double *out)
{
    double rho[3] = {xi[0], xi[1], xi[2]}, ph[3] = {xi[3], xi[4], xi[5]};
    double th2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2], th = sqrt(th2);
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
    double K[3][3] = {{0, -ph[2], ph[1]}, {ph[2], 0, -ph[0]}, {-ph[1], ph[0], 0}};
    double K2[3][3];
    m3_mul(K, K, K2);
    double R[3][3], Vm[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double I = i == j ? 1.0 : 0.0;
            R[i][j] = I + A * K[i][j] + B * K2[i][j];
            Vm[i][j] = I + B * K[i][j] + C * K2[i][j];
        }
    double t[3];
    for (int i = 0; i < 3; i++) t[i] = Vm[i][0] * rho[0] + Vm[i][1] * rho[1] + Vm[i][2] * rho[2];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 4; j++) {
            double acc = R[i][0] * E[j] + R[i][1] * E[4 + j] + R[i][2] * E[8 + j];
            if (j == 3) acc += t[i];
            out[4 * i + j] = acc;
        }
    }
}
