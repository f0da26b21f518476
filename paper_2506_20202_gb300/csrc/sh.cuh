// Real spherical harmonics up to degree 3 (orthonormal, standard (l, m) basis with positive
// polynomials: Y_{1,-1} = c1 y, Y_{1,0} = c1 z, Y_{1,1} = c1 x, ...), coefficient index
// k = l*l + l + m, evaluated as polynomials of a unit direction (x, y, z), and the
// vector-Jacobian product of those polynomials with respect to x, y, z.
#pragma once

namespace rara {

constexpr float kY00 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;    // (1/2) sqrt(15 / pi)
constexpr float kY20 = 0.31539156525252005f;   // (1/4) sqrt(5 / pi)
constexpr float kY22 = 0.54627421529603959f;   // (1/4) sqrt(15 / pi)
constexpr float kY33 = 0.59004358992664352f;   // (1/4) sqrt(35 / (2 pi))
constexpr float kY32 = 2.8906114426405538f;    // (1/2) sqrt(105 / pi)
constexpr float kY31 = 0.45704579946446572f;   // (1/4) sqrt(21 / (2 pi))
constexpr float kY30 = 0.37317633259011540f;   // (1/4) sqrt(7 / pi)
constexpr float kY32b = 1.4453057213202769f;   // (1/4) sqrt(105 / pi)

__device__ __forceinline__ int sh_count(int degree) { return (degree + 1) * (degree + 1); }

__device__ __forceinline__ void sh_basis(int degree, float x, float y, float z, float b[16])
{
    b[0] = kY00;
    if (degree >= 1) {
        b[1] = kY1 * y;
        b[2] = kY1 * z;
        b[3] = kY1 * x;
    }
    if (degree >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        b[4] = kY2a * x * y;
        b[5] = kY2a * y * z;
        b[6] = kY20 * (3.0f * zz - 1.0f);
        b[7] = kY2a * x * z;
        b[8] = kY22 * (xx - yy);
        if (degree >= 3) {
            b[9] = kY33 * y * (3.0f * xx - yy);
            b[10] = kY32 * x * y * z;
            b[11] = kY31 * y * (5.0f * zz - 1.0f);
            b[12] = kY30 * z * (5.0f * zz - 3.0f);
            b[13] = kY31 * x * (5.0f * zz - 1.0f);
            b[14] = kY32b * z * (xx - yy);
            b[15] = kY33 * x * (xx - 3.0f * yy);
        }
    }
}

// Vector-Jacobian product of the basis: g = sum_k s_k * d b_k / d(x, y, z) over
// k < sh_count(degree), for the polynomials as written (the direction's normalisation is
// the caller's).
__device__ __forceinline__ void sh_basis_vjp(int degree, float x, float y, float z, const float s[16], float g[3])
{
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
    if (degree >= 1) {
        gy += kY1 * s[1];
        gz += kY1 * s[2];
        gx += kY1 * s[3];
    }
    if (degree >= 2) {
        gx += kY2a * (y * s[4] + z * s[7]) + 2.0f * kY22 * x * s[8];
        gy += kY2a * (x * s[4] + z * s[5]) - 2.0f * kY22 * y * s[8];
        gz += kY2a * (y * s[5] + x * s[7]) + 6.0f * kY20 * z * s[6];
        if (degree >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            gx += 6.0f * kY33 * x * y * s[9] + kY32 * y * z * s[10] + kY31 * (5.0f * zz - 1.0f) * s[13] +
                  2.0f * kY32b * x * z * s[14] + 3.0f * kY33 * (xx - yy) * s[15];
            gy += 3.0f * kY33 * (xx - yy) * s[9] + kY32 * x * z * s[10] + kY31 * (5.0f * zz - 1.0f) * s[11] -
                  2.0f * kY32b * y * z * s[14] - 6.0f * kY33 * x * y * s[15];
            gz += kY32 * x * y * s[10] + 10.0f * kY31 * y * z * s[11] + kY30 * (15.0f * zz - 3.0f) * s[12] +
                  10.0f * kY31 * x * z * s[13] + kY32b * (xx - yy) * s[14];
        }
    }
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

}  // namespace rara
