// Real spherical harmonics up to degree 3 for view-dependent colour.
//
// Basis: real SH without the Condon-Shortley phase, each function of unit L2
// norm on the sphere, evaluated on a unit direction (x, y, z).  Order: l = 0;
// l = 1: y, z, x; l = 2: xy, yz, 3z^2-1, xz, x^2-y^2; l = 3: y(3x^2-y^2), xyz,
// y(5z^2-1), z(5z^2-3), x(5z^2-1), z(x^2-y^2), x(x^2-3y^2).  Constants are the
// closed-form normalisations:
//   c0 = 1/(2 sqrt(pi)), c1 = sqrt(3/(4 pi)),
//   c2a = sqrt(15/pi)/2, c2b = sqrt(5/pi)/4, c2c = sqrt(15/pi)/4,
//   c3a = sqrt(35/(2 pi))/4, c3b = sqrt(105/pi)/2, c3c = sqrt(21/(2 pi))/4,
//   c3d = sqrt(7/pi)/4, c3e = sqrt(105/pi)/4.
#pragma once

namespace gs {

constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.48860251190291992f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.54627421529603959f;
constexpr float kC3a = 0.59004358992664352f;
constexpr float kC3b = 2.8906114426405538f;
constexpr float kC3c = 0.45704579946446572f;
constexpr float kC3d = 0.37317633259011540f;
constexpr float kC3e = 1.4453057213202769f;

template <int DEG>
struct ShCount {
    static constexpr int value = (DEG + 1) * (DEG + 1);
};

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
    Y[0] = kC0;
    if (DEG < 1) return;
    Y[1] = kC1 * y;
    Y[2] = kC1 * z;
    Y[3] = kC1 * x;
    if (DEG < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;
    Y[5] = kC2a * y * z;
    Y[6] = kC2b * (3.0f * zz - 1.0f);
    Y[7] = kC2a * x * z;
    Y[8] = kC2c * (xx - yy);
    if (DEG < 3) return;
    Y[9] = kC3a * y * (3.0f * xx - yy);
    Y[10] = kC3b * x * y * z;
    Y[11] = kC3c * y * (5.0f * zz - 1.0f);
    Y[12] = kC3d * z * (5.0f * zz - 3.0f);
    Y[13] = kC3c * x * (5.0f * zz - 1.0f);
    Y[14] = kC3e * z * (xx - yy);
    Y[15] = kC3a * x * (xx - 3.0f * yy);
}

// Gradient of sum_k w_k Y_k with respect to the (unnormalised) direction
// components, given per-basis weights w_k.
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, const float *w, float *g)
{
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
    if (DEG >= 1) {
        gy += kC1 * w[1];
        gz += kC1 * w[2];
        gx += kC1 * w[3];
    }
    if (DEG >= 2) {
        gx += kC2a * (y * w[4] + z * w[7]) + 2.0f * kC2c * x * w[8];
        gy += kC2a * (x * w[4] + z * w[5]) - 2.0f * kC2c * y * w[8];
        gz += kC2a * (y * w[5] + x * w[7]) + 6.0f * kC2b * z * w[6];
    }
    if (DEG >= 3) {
        float xx = x * x, yy = y * y, zz = z * z;
        gx += 6.0f * kC3a * x * y * w[9] + kC3b * y * z * w[10] + kC3c * (5.0f * zz - 1.0f) * w[13] +
              2.0f * kC3e * x * z * w[14] + kC3a * (3.0f * xx - 3.0f * yy) * w[15];
        gy += kC3a * (3.0f * xx - 3.0f * yy) * w[9] + kC3b * x * z * w[10] + kC3c * (5.0f * zz - 1.0f) * w[11] -
              2.0f * kC3e * y * z * w[14] - 6.0f * kC3a * x * y * w[15];
        gz += kC3b * x * y * w[10] + 10.0f * kC3c * y * z * w[11] + kC3d * (15.0f * zz - 3.0f) * w[12] +
              10.0f * kC3c * x * z * w[13] + kC3e * (xx - yy) * w[14];
    }
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

}  // namespace gs
