// pair_bound.cuh -- the pair estimate of the smallest eigenvalue of D.
//
// Sec. IV asks for d_min <= lambda_min(D).  Every diagonal block of D is the
// same multiple of the identity, d_s I (the self term plus the lattice sums
// of the bead's own images and of the k-vectors, both isotropic by the cubic
// symmetry of the lattice), so the 6 x 6 principal submatrix of D on a pair
// (nu, mu) is [[d_s I, B], [B, d_s I]] with B = D_{nu mu} symmetric, and its
// eigenvalues are d_s -+ the eigenvalues of B.  Its smallest eigenvalue,
// d_s - rho(B) (rho = spectral radius), is >= lambda_min(D) by Cauchy
// interlacing.  The pair estimate is therefore
//   theta_pair = d_s - max over pairs nu != mu of rho(D_{nu mu}).
// In dense solutions the lowest modes of D are the relative motions of the
// closest overlapping pairs (almost all of such an eigenvector sits on two
// beads: the overlap-corrected mobility of beads at r << a differs from the
// self term by O(r/a)), and theta_pair lands within a few per cent of
// lambda_min, where Lanczos from a random start needs far more steps than
// the products of one step provide.
#pragma once
#include <math.h>

namespace bd {

// pairs whose Gershgorin bound on rho(B) stays at or below this are reported
// by that bound (an upper bound on rho, so the estimate only gets safer);
// above it rho is computed exactly
constexpr float kPairExactAbove = 0.5f;

// rho(B) of the symmetric 3 x 3 block (xx, xy, xz, yy, yz, zz), or its
// Gershgorin bound where that is <= kPairExactAbove.  The exact value comes
// from the trigonometric solution of the characteristic cubic of
// (B - q I)/p with q = tr B / 3 (O. K. Smith, Commun. ACM 4 (1961) 168).
// Returns NaN for a non-finite block (fmaxf drops it in the reductions).
__device__ __forceinline__ float pair_block_radius(float a00, float a01, float a02, float a11,
                                                   float a12, float a22)
{
    const float g0 = fabsf(a00) + fabsf(a01) + fabsf(a02);
    const float g1 = fabsf(a01) + fabsf(a11) + fabsf(a12);
    const float g2 = fabsf(a02) + fabsf(a12) + fabsf(a22);
    const float g = fmaxf(g0, fmaxf(g1, g2));
    if (!(g > kPairExactAbove)) return g;          // also NaN -> NaN (g is NaN)
    const float q = (a00 + a11 + a22) * (1.f / 3.f);
    const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const float off = a01 * a01 + a02 * a02 + a12 * a12;
    const float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.f * off;
    if (!(p2 > 0.f)) return fabsf(q);              // B = q I
    const float p = sqrtf(p2 * (1.f / 6.f));
    const float det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
                      a02 * (a01 * a12 - b11 * a02);
    float r = det / (2.f * p * p * p);
    r = fminf(1.f, fmaxf(-1.f, r));
    // phi in [0, pi/3]: the fast sine/cosine (absolute error ~1e-6 on this
    // range) keep the slow-path argument reduction and its stack frame out of
    // the assembly kernel; 2 p cos is then good to ~1e-6 p
    const float phi = acosf(r) * (1.f / 3.f);
    float sp, cp;
    __sincosf(phi, &sp, &cp);
    const float lmax = q + 2.f * p * cp;
    // cos(phi + 2 pi/3) = -cos(phi)/2 - sin(phi) sqrt(3)/2
    const float lmin = q - p * (cp + 1.73205080756887729f * sp);
    return fmaxf(fabsf(lmax), fabsf(lmin));
}

// max of v over the warp (NaN lanes dropped), then one atomicMax of its bit
// pattern into *word (non-negative floats order like their bit patterns) by
// lane 0, only when it exceeds the value already there.  Every lane of the
// warp must call it.
__device__ __forceinline__ void warp_max_to_word(float v, unsigned *word)
{
    v = fmaxf(v, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > __uint_as_float(*(volatile unsigned *)word))
        atomicMax(word, __float_as_uint(v));
}

}  // namespace bd
