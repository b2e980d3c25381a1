// kspace.cuh -- the reciprocal-space tensor of Eq. (M2) for one wave vector,
// shared by the k-vector table of the dense assembly and the influence
// function of the spectral (mesh) product.
#pragma once

namespace bd {

// M2(k) = (a - a^3 k^2/3)(1 + k^2/(4 alpha^2) + k^4/(8 alpha^4))
//         (6 pi/(k^2 V)) exp(-k^2/(4 alpha^2)) (I - khat khat)
// for one k (not folded with -k); components xx, xy, xz, yy, yz, zz
__host__ __device__ inline void m2_tensor(const double k[3], double a, double alpha, double L,
                                          double m[6])
{
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double al2 = alpha * alpha;
    const double V = L * L * L;
    const double f = (a - a * a * a * k2 / 3.0) * (1.0 + k2 / (4.0 * al2) + k2 * k2 / (8.0 * al2 * al2))
                   * (6.0 * 3.14159265358979323846 / (k2 * V)) * exp(-k2 / (4.0 * al2));
    m[0] = f * (1.0 - k[0] * k[0] / k2);
    m[1] = f * (-k[0] * k[1] / k2);
    m[2] = f * (-k[0] * k[2] / k2);
    m[3] = f * (1.0 - k[1] * k[1] / k2);
    m[4] = f * (-k[1] * k[2] / k2);
    m[5] = f * (1.0 - k[2] * k[2] / k2);
}

}  // namespace bd
