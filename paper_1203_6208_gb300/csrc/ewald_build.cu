// ewald_build.cu -- assembly of the dense periodic RPY diffusion matrix D(R)
// (Eq. DFmodified): self term + real-space image sum of M1 (Eq. M1) +
// reciprocal sum of M2(k) cos(k.(r_nu - r_mu)) (Eq. M2) + overlap correction
// M* (Eq. cor5) for the image of a pair closer than 2a.
//
// One CTA owns a 16 x 16 tile of bead pairs (I <= J); one thread owns one
// pair and walks that pair's own list of periodic images with a per-thread
// cursor, so a warp runs max(images) iterations instead of the union of 32
// different candidate shells.  The 3x3 blocks are staged in shared memory
// and written as the tile and its mirror with coalesced row stores (D is
// symmetric and each 3x3 block is a symmetric tensor).  The same template
// runs in FP64 (BD_FP64) and FP32 (mixed plans, which also write the 16-bit
// tensor-core copy of D).
#include <limits.h>
#include <math.h>
#include <string.h>

#include "bd_internal.cuh"
#include "pair_common.cuh"
#include "pair_bound.cuh"
#include "recip_tc.cuh"
#include "kspace.cuh"
#include "spectral.cuh"
#include "tc_gemm.cuh"

namespace bd {



// ---------------------------------------------------------------------------
// Plan-time tables (FP64, on the device)

__global__ void k_ewald_coef(double a, double alpha, double L, double rc, EwaldCoef *out)
{
    const double rpi = 0.56418958354775628695;  // 1/sqrt(pi)
    EwaldCoef c;
    double a3 = a * a * a, al = alpha, al2 = al * al, al3 = al2 * al, al5 = al3 * al2,
           al7 = al5 * al2;
    c.alpha = al; c.alpha2 = al2; c.a = a; c.L = L; c.invL = 1.0 / L; c.rc2 = rc * rc;
    c.four_a2 = 4.0 * a * a;
    c.A1 = 0.75 * a; c.A3 = 0.5 * a3;
    c.P0 = (-4.5 * a * al + 14.0 * a3 * al3) * rpi;
    c.P1 = (3.0 * a * al3 - 20.0 * a3 * al5) * rpi;
    c.P2 = 4.0 * a3 * al7 * rpi;
    c.Q = a3 * al * rpi;
    c.R0 = (1.5 * a * al - 2.0 * a3 * al3) * rpi;
    c.R1 = (-3.0 * a * al3 + 16.0 * a3 * al5) * rpi;
    c.R2 = -4.0 * a3 * al7 * rpi;
    c.S = -3.0 * a3 * al * rpi;
    c.self = 1.0 - 6.0 * a * al * rpi + 40.0 * a3 * al3 * rpi / 3.0;
    c.g1a = a * al * rpi; c.g1b = a3 * al3 * rpi;
    c.g2a = a * al3 * rpi; c.g2b = a3 * al5 * rpi;
    c.inv_a = 1.0 / a;
    *out = c;
}

template <typename T>
__device__ void fill_ewt(const EwaldCoef &c, EwaldT<T> *o)
{
    o->alpha = (T)c.alpha; o->alpha2 = (T)c.alpha2; o->A1 = (T)c.A1; o->A3 = (T)c.A3;
    o->P0 = (T)c.P0; o->P1 = (T)c.P1; o->P2 = (T)c.P2; o->Q = (T)c.Q;
    o->R0 = (T)c.R0; o->R1 = (T)c.R1; o->R2 = (T)c.R2; o->S = (T)c.S;
    o->g1a = (T)c.g1a; o->g1b = (T)c.g1b; o->g2a = (T)c.g2a; o->g2b = (T)c.g2b;
    o->inv_a = (T)c.inv_a; o->rc2 = (T)c.rc2; o->four_a2 = (T)c.four_a2; o->self = (T)c.self;
    o->L = (T)c.L;
    o->Llo = (T)(c.L - (double)(T)c.L);
    o->halfL = (T)(0.5 * c.L);
    o->Lf = (float)c.L;
    o->invLf = (float)c.invL;
}

__global__ void k_ewald_typed(const EwaldCoef *c, EwaldT<double> *o64, EwaldT<float> *o32)
{
    fill_ewt<double>(*c, o64);
    if (o32) fill_ewt<float>(*c, o32);
}

// positions wrapped into [0, L): FP64, and as FP32 hi/lo words.  fmod is
// exact (the remainder of a binary64 division is representable), so an
// unwrapped coordinate of any finite magnitude lands in [0, L); x - L floor(x/L)
// would leave a residual many box lengths long once x/L is not exact.
__global__ void k_wrap(const double *R, int n3, double L, double *pw, float *pw32)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    double x = fmod(R[i], L);
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    pw[i] = x;
    if (pw32) {
        float h = (float)x;
        pw32[i] = h;
        pw32[n3 + i] = (float)(x - (double)h);
    }
}

// M2(k) of Eq. (M2) for the half-space vectors n (integers from the host),
// folded with the -k partner (factor 2).
__global__ void k_kvec(const int *nvec, int nk, double a, double alpha, double L, KVec *out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nk) return;
    const double two_pi = 6.283185307179586476925;
    KVec kv;
    for (int i = 0; i < 3; i++) kv.k[i] = two_pi * nvec[3 * t + i] / L;
    double m[6];
    m2_tensor(kv.k, a, alpha, L, m);
    for (int i = 0; i < 6; i++) kv.m[i] = 2.0 * m[i];      // folded with -k
    out[t] = kv;
}

// Eq. (M1) coefficient pair (c1(u), c2(u)/u) at u = r^2, FP64, for the table fit
__device__ void m1_pair(const EwaldCoef &c, double u, double *f1, double *f2)
{
    double rinv = rsqrt(u), r = u * rinv, uinv = rinv * rinv;
    double ec = erfc(c.alpha * r) * rinv;
    double ex = exp(-c.alpha2 * u);
    *f1 = ec * (c.A1 + c.A3 * uinv) + ex * ((c.P2 * u + c.P1) * u + c.P0 + c.Q * uinv);
    double c2 = ec * (c.A1 - 3.0 * c.A3 * uinv) + ex * ((c.R2 * u + c.R1) * u + c.R0 + c.S * uinv);
    *f2 = c2 * uinv;
}

// One thread per (interval, function): interpolate at the DEG+1 Chebyshev
// nodes of the interval and solve for the monomial coefficients in t in
// [-1, 1] (Gaussian elimination with partial pivoting, FP64), stored in the
// table's precision.
template <typename T>
__global__ void k_m1_table(const EwaldCoef *ewc, int i0, int ntab, T *tab)
{
    constexpr int DEG = TabFmt<T>::DEG, SHIFT = TabFmt<T>::SHIFT, STRIDE = TabFmt<T>::STRIDE;
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 2 * ntab) return;
    const int i = id >> 1, which = id & 1;
    const int N = DEG + 1;
    const EwaldCoef &c = *ewc;
    double lo = (double)__uint_as_float((unsigned)(i0 + i) << SHIFT);
    double hi = (double)__uint_as_float((unsigned)(i0 + i + 1) << SHIFT);
    double mid = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
    double A[DEG + 1][DEG + 2];
    for (int j = 0; j < N; j++) {
        double t = cos(3.14159265358979323846 * (j + 0.5) / N);
        double f1, f2;
        m1_pair(c, mid + hw * t, &f1, &f2);
        double p = 1.0;
        for (int k = 0; k < N; k++) { A[j][k] = p; p *= t; }
        A[j][N] = which ? f2 : f1;
    }
    for (int col = 0; col < N; col++) {
        int piv = col;
        for (int r = col + 1; r < N; r++)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k <= N; k++) { double tt = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = tt; }
        for (int r = col + 1; r < N; r++) {
            double f = A[r][col] / A[col][col];
            for (int k = col; k <= N; k++) A[r][k] -= f * A[col][k];
        }
    }
    double x[DEG + 1];
    for (int r = N - 1; r >= 0; r--) {
        double acc = A[r][N];
        for (int k = r + 1; k < N; k++) acc -= A[r][k] * x[k];
        x[r] = acc / A[r][r];
    }
    T *row = tab + (size_t)i * STRIDE;
    if (which == 0) { row[0] = (T)mid; row[1] = (T)(1.0 / hw); }
    for (int k = 0; k < N; k++) row[2 + which * N + k] = (T)x[k];
}

// per k in the working precision, [nk][12]: the six folded tensor components
// (xx xy xz yy yz zz), then k (x y z), then padding
__global__ void k_kvec_m(const KVec *kv, int nk, double *m64, float *m32)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nk) return;
    for (int i = 0; i < 12; i++) {
        double v = i < 6 ? kv[t].m[i] : (i < 9 ? kv[t].k[i - 6] : 0.0);
        m64[12 * t + i] = v;
        if (m32) m32[12 * t + i] = (float)v;
    }
}

// cos/sin(k_t . r_nu) per bead and half-space k (FP64 plans; FP32 copies if
// cs32 is given).  The pair factor cos(k.(r_nu - r_mu)) is then
// c_nu c_mu + s_nu s_mu.
__global__ void k_trig(const double *R, int n, const KVec *kv, int nk, double *cs, double *sn,
                       float *cs32, float *sn32)
{
    int nu = blockIdx.x * blockDim.x + threadIdx.x;
    int t = blockIdx.y;
    if (nu >= n || t >= nk) return;
    double ph = kv[t].k[0] * R[3 * nu] + kv[t].k[1] * R[3 * nu + 1] + kv[t].k[2] * R[3 * nu + 2];
    double s, c;
    sincos(ph, &s, &c);
    cs[(size_t)t * n + nu] = c;
    sn[(size_t)t * n + nu] = s;
    if (cs32) {
        cs32[(size_t)t * n + nu] = (float)c;
        sn32[(size_t)t * n + nu] = (float)s;
    }
}

template <typename T> struct Math;
template <> struct Math<double> {
    __device__ static double rsqrt_(double x) { return rsqrt(x); }
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double erfc_(double x) { return erfc(x); }
    __device__ static double exp_(double x) { return exp(x); }
};
template <> struct Math<float> {
    __device__ static float rsqrt_(float x) { return rsqrtf(x); }
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float erfc_(float x) { return erfcf(x); }
    __device__ static float exp_(float x) { return expf(x); }
};

// Eq. (M1) for one image vector v (u = |v|^2 > 0); accumulates the six
// independent components (xx, xy, xz, yy, yz, zz).
template <typename T>
__device__ __forceinline__ void add_m1(T vx, T vy, T vz, T u, const EwaldT<T> &c, T acc[6])
{
    T rinv = Math<T>::rsqrt_(u);
    T r = u * rinv;
    T uinv = rinv * rinv;
    T ec = Math<T>::erfc_(c.alpha * r) * rinv;
    T ex = Math<T>::exp_(-c.alpha2 * u);
    T c1 = ec * (c.A1 + c.A3 * uinv) + ex * ((c.P2 * u + c.P1) * u + c.P0 + c.Q * uinv);
    T c2 = ec * (c.A1 - (T)3 * c.A3 * uinv) + ex * ((c.R2 * u + c.R1) * u + c.R0 + c.S * uinv);
    T g = c2 * uinv;
    T gx = g * vx, gy = g * vy;
    acc[0] += c1 + gx * vx;
    acc[1] += gx * vy;
    acc[2] += gx * vz;
    acc[3] += c1 + gy * vy;
    acc[4] += gy * vz;
    acc[5] += c1 + g * vz * vz;
}

// Eq. (M1) for one image from the piecewise-polynomial table (4a^2 <= u <= r_c^2)
// one table row (mid, 1/half-width, 9 + 9 coefficients) with 16-byte loads
template <typename T> struct TabRow;
template <> struct TabRow<float> {
    float v[TabFmt<float>::STRIDE];
    __device__ __forceinline__ TabRow(const float *row)
    {
        const float4 *q = (const float4 *)row;
#pragma unroll
        for (int k = 0; k < TabFmt<float>::STRIDE / 4; k++) {
            float4 x = __ldg(q + k);
            v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
        }
    }
};
template <> struct TabRow<double> {
    double v[TabFmt<double>::STRIDE];
    __device__ __forceinline__ TabRow(const double *row)
    {
        const double2 *q = (const double2 *)row;
#pragma unroll
        for (int k = 0; k < TabFmt<double>::STRIDE / 2; k++) {
            double2 x = __ldg(q + k);
            v[2 * k] = x.x; v[2 * k + 1] = x.y;
        }
    }
};

template <typename T>
__device__ __forceinline__ void add_m1_tab(T vx, T vy, T vz, T u, const T *__restrict__ tab,
                                           int i0, int ntab, T acc[6])
{
    constexpr int DEG = TabFmt<T>::DEG;
    int i = (int)(__float_as_uint((float)u) >> TabFmt<T>::SHIFT) - i0;
    i = i < 0 ? 0 : (i >= ntab ? ntab - 1 : i);
    const TabRow<T> r(tab + (size_t)i * TabFmt<T>::STRIDE);
    T t = (u - r.v[0]) * r.v[1];
    const T *a = r.v + 2, *b = r.v + 2 + (DEG + 1);
    T c1 = a[DEG], g = b[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; k--) {
        c1 = c1 * t + a[k];
        g = g * t + b[k];
    }
    T gx = g * vx, gy = g * vy;
    acc[0] += c1 + gx * vx;
    acc[1] += gx * vy;
    acc[2] += gx * vz;
    acc[3] += c1 + gy * vy;
    acc[4] += gy * vz;
    acc[5] += c1 + g * vz * vz;
}

// The same for the image loop of the FP32 dense assembly, where the caller
// has already checked 4a^2 <= u <= r_c^2: the interval index then lies in
// [0, ntab) without a clamp (the table range is built from the same FP32
// values, 4a^2 and r_c^2 (1 + 1e-6)).  The intervals split each binade into
// 2^BITS equal parts, so the low 23 - BITS fraction bits of u are its offset
// in its interval: 1 + offset / 2^(23 - BITS) is built as a float f in
// [1, 2) and t = 2 f - 3 equals (u - mid) / hw exactly, so only the row's ten
// coefficients are loaded (40 of its 48 bytes).  The isotropic part c1 is
// summed into c1sum (added to the three diagonal components once per pair).
__device__ __forceinline__ void add_m1_tab_in_range(float vx, float vy, float vz, float u,
                                                    const float *__restrict__ tab, int i0,
                                                    float acc[6], float &c1sum)
{
    constexpr int BITS = TabFmt<float>::BITS, SHIFT = TabFmt<float>::SHIFT;
    static_assert(TabFmt<float>::DEG == 4 && TabFmt<float>::STRIDE == 12,
                  "row layout: mid, 1/hw, a0 .. a4, b0 .. b4");
    const unsigned ub = __float_as_uint(u);
    const float *row = tab + (size_t)((int)(ub >> SHIFT) - i0) * TabFmt<float>::STRIDE;
    const float2 q0 = __ldg((const float2 *)(row + 2));      // a0 a1
    const float4 q1 = __ldg((const float4 *)(row + 4));      // a2 a3 a4 b0
    const float4 q2 = __ldg((const float4 *)(row + 8));      // b1 b2 b3 b4
    const float t = fmaf(2.f, __uint_as_float(0x3F800000u | ((ub << BITS) & 0x7FFFFFu)), -3.f);
    float c1 = q1.z, g = q2.w;
    c1 = c1 * t + q1.y; g = g * t + q2.z;
    c1 = c1 * t + q1.x; g = g * t + q2.y;
    c1 = c1 * t + q0.y; g = g * t + q2.x;
    c1 = c1 * t + q0.x; g = g * t + q1.w;
    const float gx = g * vx, gy = g * vy, gz = g * vz;
    acc[0] += gx * vx;
    acc[1] += gx * vy;
    acc[2] += gx * vz;
    acc[3] += gy * vy;
    acc[4] += gy * vz;
    acc[5] += gz * vz;
    c1sum += c1;
}

template <typename T>
__device__ __forceinline__ T horner(const double *cf, T x)
{
    T y = (T)cf[kNT - 1];
#pragma unroll
    for (int j = kNT - 2; j >= 0; j--) y = y * x + (T)cf[j];
    return y;
}

// M1 + M* for the image closer than 2a (Eqs. M1, cor5 with the rr
// coefficient 3(x^2-4)^2/(32x^3)), evaluated as Omega_B(r) - G(r) with G the
// smooth remainder Omega_A - M1 from its Taylor series in s = alpha r; this
// avoids the (a/r)^3 cancellation between M1 and M*.  For s^2 > 1 (only
// reachable with alpha > 1/(2a)) the direct sum M1 + M* is used instead.
template <typename T>
__device__ void add_overlap(T vx, T vy, T vz, T u, const EwaldT<T> &c, T acc[6])
{
    T s2 = c.alpha2 * u;
    T d1, d2;
    T r = Math<T>::sqrt_(u);
    if (s2 <= (T)1) {
        T G1 = c.g1a * horner(c_A1, s2) + c.g1b * horner(c_B1, s2);
        T G2u = c.g2a * horner(c_A2s, s2) + c.g2b * horner(c_B2s, s2);
        T x = r * c.inv_a;
        d1 = (T)1 - (T)(9.0 / 32.0) * x - G1;
        d2 = (u > (T)0) ? ((T)(3.0 / 32.0) * c.inv_a / r - G2u) : (T)0;
    } else {
        T rinv = (T)1 / r, uinv = rinv * rinv;
        T ec = Math<T>::erfc_(c.alpha * r) * rinv;
        T ex = Math<T>::exp_(-c.alpha2 * u);
        T c1 = ec * (c.A1 + c.A3 * uinv) + ex * ((c.P2 * u + c.P1) * u + c.P0 + c.Q * uinv);
        T c2 = ec * (c.A1 - (T)3 * c.A3 * uinv) + ex * ((c.R2 * u + c.R1) * u + c.R0 + c.S * uinv);
        T x = r * c.inv_a, x2 = x * x, x3 = x2 * x;
        T q = (T)0.75 * x2 + (T)1;
        T m1 = (T)1 - q * q / ((T)2 * x3);
        T m2 = (T)3 * (x2 - (T)4) * (x2 - (T)4) / ((T)32 * x3);
        d1 = c1 + m1;
        d2 = (c2 + m2) * uinv;
    }
    acc[0] += d1 + d2 * vx * vx;
    acc[1] += d2 * vx * vy;
    acc[2] += d2 * vx * vz;
    acc[3] += d1 + d2 * vy * vy;
    acc[4] += d2 * vy * vz;
    acc[5] += d1 + d2 * vz * vz;
}


constexpr int TB = 16;                 // beads per tile side
static_assert(TB == 16, "the assembly's warp layout takes 16 x 16 pairs per CTA");
constexpr int TS = 3 * TB;             // matrix rows per tile side
constexpr int TSP = TS + 1;            // padded smem row

template <typename T> struct Store;
template <> struct Store<double> {
    __device__ static void put(double *D, void *, size_t idx, double v, int) { D[idx] = v; }
    // four consecutive elements, idx a multiple of 4 (32-byte aligned rows)
    __device__ static void put4(double *D, void *, size_t idx, const double v[4], int)
    {
        double2 *d = (double2 *)(D + idx);
        d[0] = make_double2(v[0], v[1]);
        d[1] = make_double2(v[2], v[3]);
    }
};
template <> struct Store<float> {
    __device__ static void put(float *D, void *D16, size_t idx, float v, int is_bf16)
    {
        D[idx] = v;
        if (is_bf16) ((__nv_bfloat16 *)D16)[idx] = __float2bfloat16_rn(v);
        else ((__half *)D16)[idx] = __float2half_rn(v);
    }
    // four consecutive elements: one 16-byte FP32 store and one 8-byte 16-bit store
    __device__ static void put4(float *D, void *D16, size_t idx, const float v[4], int is_bf16)
    {
        *(float4 *)(D + idx) = make_float4(v[0], v[1], v[2], v[3]);
        uint2 h;
        if (is_bf16) {
            __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
            h.x = *(const unsigned *)&a;
            h.y = *(const unsigned *)&b;
        } else {
            __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
            h.x = *(const unsigned *)&a;
            h.y = *(const unsigned *)&b;
        }
        *(uint2 *)((__half *)D16 + idx) = h;
    }
};

template <typename T> struct Sep;
template <> struct Sep<double> {
    __device__ static void get(const double *pw, const float *, long, int nu, int mu,
                               const EwaldT<double> &c, double d[3])
    {
#pragma unroll
        for (int s = 0; s < 3; s++) {
            double x = pw[3 * nu + s] - pw[3 * mu + s];
            x = x > c.halfL ? x - c.L : (x < -c.halfL ? x + c.L : x);
            d[s] = x;
        }
    }
};
template <> struct Sep<float> {
    __device__ static void get(const double *, const float *pw32, long n3, int nu, int mu,
                               const EwaldT<float> &c, float d[3])
    {
#pragma unroll
        for (int s = 0; s < 3; s++) {
            float a = pw32[3 * nu + s], b = -pw32[3 * mu + s];
            float hs = a + b;                                  // TwoSum(a, b)
            float bb = hs - a;
            float he = (a - (hs - bb)) + (b - bb);
            he += pw32[n3 + 3 * nu + s] - pw32[n3 + 3 * mu + s];
            if (hs > c.halfL) { hs -= c.L; he -= c.Llo; }
            else if (hs < -c.halfL) { hs += c.L; he += c.Llo; }
            d[s] = hs + he;
        }
    }
};

// real-space images, overlap branch and self term of the block D_{nu mu}
// (Eqs. DF, M1, DFmodified): the six components xx, xy, xz, yy, yz, zz are
// added to acc
template <typename T>
__device__ __forceinline__ void pair_real(const double *__restrict__ pw,
                                          const float *__restrict__ pw32, long n3, int nu, int mu,
                                          const EwaldT<T> &c, const T *__restrict__ tab, int tab_i0,
                                          int ntab, int overlap_corr, float rc, T acc[6])
{
    T d[3];
    Sep<T>::get(pw, pw32, n3, nu, mu, c, d);
    const bool same = (nu == mu);
    T c1sum = 0;
    ImageCursor cur;
    cur.start((float)d[0], (float)d[1], (float)d[2], c.Lf, c.invLf, rc);
    while (!cur.done) {
        T vx = d[0] + (T)cur.nx * c.L, vy = d[1] + (T)cur.ny * c.L, vz = d[2] + (T)cur.nz * c.L;
        T u = vx * vx + vy * vy + vz * vz;
        // the bead's own zero image (nu = mu, n = 0) is the one image of a
        // diagonal pair with u = 0 (its separation is exactly zero)
        const bool zero_image = same && u == (T)0;
        if (u <= c.rc2 && !zero_image) {
            // FP32: the leaner table step (the FP64 kernel keeps the plain one,
            // whose registers fit its 4 CTAs per SM without spills)
            if (u >= c.four_a2) {
                if constexpr (sizeof(T) == 4) add_m1_tab_in_range(vx, vy, vz, u, tab, tab_i0, acc, c1sum);
                else add_m1_tab<T>(vx, vy, vz, u, tab, tab_i0, ntab, acc);
            }
            else if (!same && overlap_corr) add_overlap<T>(vx, vy, vz, u, c, acc);
            else add_m1<T>(vx, vy, vz, u, c, acc);
        }
        cur.advance();
    }
    if constexpr (sizeof(T) == 4) {
        acc[0] += c1sum; acc[3] += c1sum; acc[5] += c1sum;
    }
    if (same) {
        acc[0] += c.self; acc[3] += c.self; acc[5] += c.self;
    }
}

// M1 (or M1 + M* for an overlapping pair) of one image closer than 2a, for
// the warp loop below: rare, and kept out of line so that its registers (the
// series and erfc/exp evaluation) do not weigh on the loop's allocation
struct Six {
    float v[6];
};
__device__ __noinline__ Six near_image(float vx, float vy, float vz, float u, const EwaldT<float> &c,
                                       bool overlap)
{
    float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (overlap) add_overlap<float>(vx, vy, vz, u, c, a);
    else add_m1<float>(vx, vy, vz, u, c, a);
    Six r;
#pragma unroll
    for (int k = 0; k < 6; k++) r.v[k] = a[k];
    return r;
}

// The same sum for the FP32 dense assembly, taken by the 32 pairs of a warp
// together: the lanes walk one common set of lattice candidates n (the union
// of their per-axis ranges, FP32 bounds widened by a margin as in the image
// cursor) in lockstep, skip the rows and candidates that no lane keeps (a
// vote), and a lane evaluates only the images inside its own sphere
// |d + nL| <= r_c.  The per-lane cursor's nested loops put the lanes of a warp
// at different loop levels (row set-up on some, image evaluation on others);
// here the control flow is uniform and only the evaluation is masked.  Every
// lane of the warp must call this (it holds warp votes); lanes without images
// (inactive, or with a non-finite or farther than 2^20 L separation) pass
// active = false and take no candidate.
__device__ __forceinline__ void pair_real_warp(const float *__restrict__ pw32, long n3, int nu, int mu,
                                               bool active, const EwaldT<float> &c,
                                               const float *__restrict__ tab, int tab_i0,
                                               int overlap_corr, float rc, float acc[6])
{
    constexpr unsigned kAll = 0xffffffffu;
    float d[3] = {0.f, 0.f, 0.f};
    if (active) Sep<float>::get(nullptr, pw32, n3, nu, mu, c, d);
    const bool same = (nu == mu);
    const float L = c.Lf, invL = c.invLf, rc2 = c.rc2;
    const bool ok = active && isfinite(d[0] + d[1] + d[2]) &&
                    fabsf(d[0]) + fabsf(d[1]) + fabsf(d[2]) <= 0x1p20f * L;
    int lo[3], hi[3];
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const float l = ok ? ceilf((-rc - d[s]) * invL - 1e-4f) : 0.f;
        const float h = ok ? floorf((rc - d[s]) * invL + 1e-4f) : 0.f;
        lo[s] = __reduce_min_sync(kAll, ok ? (int)l : INT_MAX);
        hi[s] = __reduce_max_sync(kAll, ok ? (int)h : INT_MIN);
    }
    float c1sum = 0.f;
    for (int ix = lo[0]; ix <= hi[0]; ix++) {
        const float vx = fmaf((float)ix, L, d[0]);
        const float rx = vx * vx;
        if (!__any_sync(kAll, ok && rx <= rc2)) continue;
        for (int iy = lo[1]; iy <= hi[1]; iy++) {
            const float vy = fmaf((float)iy, L, d[1]);
            const float rxy = fmaf(vy, vy, rx);
            if (!__any_sync(kAll, ok && rxy <= rc2)) continue;
            for (int iz = lo[2]; iz <= hi[2]; iz++) {
                const float vz = fmaf((float)iz, L, d[2]);
                const float u = fmaf(vz, vz, rxy);
                // the bead's own zero image (nu = mu, n = 0) is the one
                // image of a diagonal pair with u = 0
                const bool take = ok && u <= rc2 && !(same && u == 0.f);
                if (!__any_sync(kAll, take)) continue;
                if (take) {
                    if (u >= c.four_a2) {
                        add_m1_tab_in_range(vx, vy, vz, u, tab, tab_i0, acc, c1sum);
                    } else {
                        const Six r = near_image(vx, vy, vz, u, c, !same && overlap_corr);
#pragma unroll
                        for (int k = 0; k < 6; k++) acc[k] += r.v[k];
                    }
                }
            }
        }
    }
    acc[0] += c1sum; acc[3] += c1sum; acc[5] += c1sum;
    if (same && active) {
        acc[0] += c.self; acc[3] += c.self; acc[5] += c.self;
    }
}

constexpr int KC = 64;                 // k-vectors per shared-memory chunk

// FP32: 48 registers and 5 CTAs per SM (issue-bound; 4 CTAs took 6 % longer, 6 no
// better); FP64: 4 CTAs (fewer registers spill)
template <typename T>
__global__ void __launch_bounds__(TB *TB, sizeof(T) == 4 ? 5 : 4)
k_build_D(const double *__restrict__ pw, const float *__restrict__ pw32, int n,
          const __grid_constant__ EwaldT<T> c, const EwaldCoef *__restrict__ ewc,
          const T *__restrict__ tab, int tab_i0, int ntab, const T *__restrict__ km, int nk,
          const T *__restrict__ cs, const T *__restrict__ sn, int overlap_corr, float rc,
          T *__restrict__ D, void *__restrict__ D16, int is_bf16, long ld, int recip_in_D,
          int upper_only, unsigned *__restrict__ pairw)
{
    __shared__ T tile[TS * TSP];
    __shared__ T s_tr[4][KC][TB];      // cos nu, sin nu, cos mu, sin mu for one k chunk
    __shared__ T s_km[KC][6];
    // tile pair (I <= J) from the linear index over the upper triangle (FP32
    // estimate, integer correction: no FP64 instruction)
    long idx = blockIdx.x;
    int J = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
    while ((long)J * (J + 1) / 2 > idx) J--;
    while ((long)(J + 1) * (J + 2) / 2 <= idx) J++;
    int I = (int)(idx - (long)J * (J + 1) / 2);
    (void)ewc;
    // each warp takes 4 consecutive beads nu x 8 consecutive beads mu (beads
    // in chain order, so the warp's separations are close together and their
    // periodic images overlap: fewer candidates for the warp image loop)
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int ty = 4 * (w & 3) + (l >> 3), tx = 8 * (w >> 2) + (l & 7);
    int nu = I * TB + ty, mu = J * TB + tx;
    T acc[6] = {0, 0, 0, 0, 0, 0};
    // diagonal tiles compute nu <= mu only; the rest is mirrored on write,
    // which keeps D exactly symmetric
    const bool active = nu < n && mu < n && !(I == J && ty > tx);
    const long n3 = 3L * n;
    if (active && recip_in_D) {
        // the reciprocal sum is already in D (row <= column for every
        // component read: this tile is on or above the diagonal)
        const T *b = D + (size_t)(3 * nu) * ld + 3 * mu;
        acc[0] = b[0]; acc[1] = b[1]; acc[2] = b[2];
        acc[3] = b[ld + 1]; acc[4] = b[ld + 2]; acc[5] = b[2 * ld + 2];
    }
    if constexpr (sizeof(T) == 4)
        pair_real_warp(pw32, n3, nu, mu, active, c, tab, tab_i0, overlap_corr, rc, acc);
    else if (active)
        pair_real<T>(pw, pw32, n3, nu, mu, c, tab, tab_i0, ntab, overlap_corr, rc, acc);
    // reciprocal sum over half-space k (each folded with -k), staged per chunk
    for (int t0 = 0; t0 < nk; t0 += KC) {
        const int kc = min(KC, nk - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < 4 * kc * TB; e += TB * TB) {
            int w = e / (kc * TB), r = e % (kc * TB), t = r / TB, b = r % TB;
            int bead = (w < 2 ? I : J) * TB + b;
            const T *src = (w & 1) ? sn : cs;
            s_tr[w][t][b] = bead < n ? src[(size_t)(t0 + t) * n + bead] : (T)0;
        }
        for (int e = threadIdx.x; e < 6 * kc; e += TB * TB)
            s_km[e / 6][e % 6] = km[12 * (t0 + e / 6) + e % 6];
        __syncthreads();
        if (active) {
            for (int t = 0; t < kc; t++) {
                T cf = s_tr[0][t][ty] * s_tr[2][t][tx] + s_tr[1][t][ty] * s_tr[3][t][tx];
#pragma unroll
                for (int i = 0; i < 6; i++) acc[i] += s_km[t][i] * cf;
            }
        }
    }
    // the pair estimate of lambda_min (pair_bound.cuh): pairw[0] = max over
    // nu != mu of the spectral radius of the block, pairw[1] = d_s (the
    // diagonal block of bead 0)
    {
        const float rho = (active && nu != mu)
            ? pair_block_radius((float)acc[0], (float)acc[1], (float)acc[2], (float)acc[3],
                                (float)acc[4], (float)acc[5])
            : 0.f;
        warp_max_to_word(rho, pairw);
        if (active && nu == 0 && mu == 0) pairw[1] = __float_as_uint((float)acc[0]);
    }
    if (D == nullptr) return;           // pair estimate only (matrix-free steps)
    __syncthreads();
    // stage the 3x3 block: rows 3ty+a, cols 3tx+b.  In a diagonal tile the
    // block below the diagonal (ty > tx) is the mirror of (tx, ty): the block
    // is symmetric, so the thread of (tx, ty) writes the same six values there
    {
        auto put_block = [&](int by, int bx) {
            T *b = &tile[(3 * by) * TSP + 3 * bx];
            b[0] = acc[0]; b[1] = acc[1]; b[2] = acc[2];
            b[TSP] = acc[1]; b[TSP + 1] = acc[3]; b[TSP + 2] = acc[4];
            b[2 * TSP] = acc[2]; b[2 * TSP + 1] = acc[4]; b[2 * TSP + 2] = acc[5];
        };
        if (I != J || ty <= tx) put_block(ty, tx);
        if (I == J && ty < tx) put_block(tx, ty);
    }
    __syncthreads();
    // four consecutive columns per thread and store (rows start 256-byte
    // aligned, tile columns at multiples of 48 elements); a ragged last group
    // of columns goes element by element
    const long r0 = 3L * TB * I, c0 = 3L * TB * J;
    constexpr int NQ = TS / 4;
    static_assert(TS % 4 == 0, "tile width");
    for (int e = threadIdx.x; e < TS * NQ; e += TB * TB) {
        const int r = e / NQ, cc = 4 * (e - (e / NQ) * NQ);
        if (r0 + r >= n3) continue;
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = tile[r * TSP + cc + k];
        const size_t idx = (size_t)((r0 + r) * ld + c0 + cc);
        if (c0 + cc + 4 <= n3) Store<T>::put4(D, D16, idx, v, is_bf16);
        else
            for (int k = 0; k < 4; k++)
                if (c0 + cc + k < n3) Store<T>::put(D, D16, idx + k, v[k], is_bf16);
    }
    // the mirror block (rows c0.., columns r0..) is skipped for the symmetric
    // product's D when it lies wholly below the diagonal 128 x 128 tiles (those
    // tiles are read whole; the rest of the lower triangle is never read)
    const bool mirror = I != J && !(upper_only && c0 / 128 > (r0 + TS - 1) / 128);
    if (mirror) {
        for (int e = threadIdx.x; e < TS * NQ; e += TB * TB) {
            // mirror: row c0 + r, columns r0 + cc .. r0 + cc + 3 = tile[cc + k][r]
            const int r = e / NQ, cc = 4 * (e - (e / NQ) * NQ);
            if (c0 + r >= n3) continue;
            T v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] = tile[(cc + k) * TSP + r];
            const size_t idx = (size_t)((c0 + r) * ld + r0 + cc);
            if (r0 + cc + 4 <= n3) Store<T>::put4(D, D16, idx, v, is_bf16);
            else
                for (int k = 0; k < 4; k++)
                    if (r0 + cc + k < n3) Store<T>::put(D, D16, idx + k, v[k], is_bf16);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers

// interval range of the M1 table for u in [4a^2, r_c^2] (integer bit patterns only)
void m1_table_range(const bd_params &p, int bits, int *i0, int *ntab)
{
    const int shift = 23 - bits;
    float lo = (float)(4.0 * p.a * p.a), hi = (float)(p.r_c * p.r_c * (1.0 + 1e-6));
    if (!(lo > 0.f) || !(hi > lo)) { *i0 = 0; *ntab = 0; return; }
    unsigned blo, bhi;
    memcpy(&blo, &lo, 4);
    memcpy(&bhi, &hi, 4);
    *i0 = (int)(blo >> shift);
    *ntab = (int)(bhi >> shift) - *i0 + 1;
}

void launch_kvec_table(Plan &P, cudaStream_t s)
{
    // integer half-space vectors (no arithmetic of the method here)
    int K = 0;
    while ((K + 1) * (K + 1) <= P.p.n2max) K++;
    int *hn = (int *)malloc(sizeof(int) * 3 * (size_t)kMaxKvec);
    int nk = 0;
    for (int nx = 0; nx <= K; nx++)
        for (int ny = -K; ny <= K; ny++)
            for (int nz = -K; nz <= K; nz++) {
                int nn = nx * nx + ny * ny + nz * nz;
                if (nn == 0 || nn > P.p.n2max) continue;
                bool half = nx > 0 || (nx == 0 && ny > 0) || (nx == 0 && ny == 0 && nz > 0);
                if (!half) continue;
                if (nk < kMaxKvec) {
                    hn[3 * nk] = nx; hn[3 * nk + 1] = ny; hn[3 * nk + 2] = nz;
                }
                nk++;
            }
    P.nk = nk;
    k_ewald_coef<<<1, 1, 0, s>>>(P.p.a, P.p.alpha, P.p.box_L, P.p.r_c, P.d_ewc);
    count_launches(1);
    k_ewald_typed<<<1, 1, 0, s>>>(P.d_ewc, P.d_ew64, P.d_ew32);
    count_launches(1);
    cudaMemcpyAsync(&P.h_ew64, P.d_ew64, sizeof(EwaldT<double>), cudaMemcpyDeviceToHost, s);
    if (P.d_ew32)
        cudaMemcpyAsync(&P.h_ew32, P.d_ew32, sizeof(EwaldT<float>), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (P.ntab > 0) {
        k_m1_table<double><<<(2 * P.ntab + 63) / 64, 64, 0, s>>>(P.d_ewc, P.tab_i0, P.ntab, P.d_tab);
        count_launches(1);
    }
    if (P.d_tab32 && P.ntab32 > 0) {
        k_m1_table<float><<<(2 * P.ntab32 + 63) / 64, 64, 0, s>>>(P.d_ewc, P.tab32_i0, P.ntab32,
                                                                 P.d_tab32);
        count_launches(1);
    }
    if (nk > kMaxKvec || nk == 0) {
        free(hn);
        return;
    }
    int *dn = nullptr;
    cudaMalloc(&dn, sizeof(int) * 3 * nk);
    cudaMemcpyAsync(dn, hn, sizeof(int) * 3 * nk, cudaMemcpyHostToDevice, s);
    k_kvec<<<(nk + 127) / 128, 128, 0, s>>>(dn, nk, P.p.a, P.p.alpha, P.p.box_L, P.d_kvec);
    count_launches(1);
    k_kvec_m<<<(nk + 127) / 128, 128, 0, s>>>(P.d_kvec, nk, P.d_km64, P.d_km32);
    count_launches(1);
    cudaStreamSynchronize(s);
    cudaFree(dn);
    free(hn);
}

// FP32 tables only (mixed plans): the phase k.r is formed in FP64 and reduced
// to the fraction f of a turn, f = k.r / 2 pi - rint(k.r / 2 pi) (exact
// subtraction); 2 f is split into FP32 words x + x_lo and sin, cos of pi x
// come from the FP32 sincospif, corrected to first order in x_lo (|pi x_lo|
// <= 2e-7, the dropped term ~1e-14).  Seven FP64 instructions per entry
// instead of an FP64 sincos on this GPU's slow FP64 pipe.
__global__ void k_trig32(const double *R, int n, const KVec *kv, int nk, float *cs32, float *sn32)
{
    int nu = blockIdx.x * blockDim.x + threadIdx.x;
    int t = blockIdx.y;
    if (nu >= n || t >= nk) return;
    constexpr double kInv2Pi = 0.15915494309189533577;
    const double ph = kv[t].k[0] * R[3 * nu] + kv[t].k[1] * R[3 * nu + 1] + kv[t].k[2] * R[3 * nu + 2];
    const double f = ph * kInv2Pi;
    const double tf = 2.0 * (f - rint(f));                 // in [-1, 1]
    const float x = (float)tf;
    const float xl = (float)(tf - (double)x);
    float sp, cp;
    sincospif(x, &sp, &cp);
    const float d = 3.14159265358979f * xl;
    cs32[(size_t)t * n + nu] = fmaf(-d, sp, cp);
    sn32[(size_t)t * n + nu] = fmaf(d, cp, sp);
}

static void launch_wrap(Plan &P, const double *R, cudaStream_t s)
{
    k_wrap<<<(P.n3 + 255) / 256, 256, 0, s>>>(R, P.n3, P.p.box_L, P.d_pw64, P.d_pw32);
    count_launches(1);
}

// wrapped positions (P.d_pw64, P.d_pw32), then the per-bead cos/sin tables
// from them: the phases k.r of coordinates reduced exactly into [0, L) keep
// their digits however far the unwrapped chains have travelled
void launch_trig_tables(Plan &P, const double *R, cudaStream_t s)
{
    launch_wrap(P, R, s);
    if (P.nk == 0) return;
    dim3 g((P.n + 127) / 128, P.nk);
    if (is_mixed(P))
        k_trig32<<<g, 128, 0, s>>>(P.d_pw64, P.n, P.d_kvec, P.nk, P.d_cos32, P.d_sin32);
    else
        k_trig<<<g, 128, 0, s>>>(P.d_pw64, P.n, P.d_kvec, P.nk, P.d_cos, P.d_sin, nullptr,
                                 nullptr);
    count_launches(1);
}

static long tile_pairs(int n)
{
    long T = (n + TB - 1) / TB;
    return T * (T + 1) / 2;
}

void launch_build_D_f64(Plan &P, const double *R, double *D, cudaStream_t s)
{
    launch_trig_tables(P, R, s);
    launch_zero_i32((int32_t *)P.d_pairw, 2, s);
    long nb = tile_pairs(P.n);
    k_build_D<double><<<(unsigned)nb, TB * TB, 0, s>>>(
        P.d_pw64, P.d_pw32, P.n, P.h_ew64, P.d_ewc, P.d_tab, P.tab_i0, P.ntab, P.d_km64, P.nk,
        P.d_cos, P.d_sin, P.p.overlap_corr,
        (float)P.p.r_c, D, nullptr, 0, P.ld, 0, 0, P.d_pairw);
    count_launches(1);
}

bd_status launch_build_D_f32(Plan &P, const double *R, float *D32, void *D16, int is_bf16,
                        cudaStream_t s)
{
    launch_trig_tables(P, R, s);
    int nk = P.nk;
    if (P.recip_tc) {
        bd_status st = launch_recip_tc(P, D32, s);
        if (st != BD_OK) return st;
        nk = 0;
    }
    launch_zero_i32((int32_t *)P.d_pairw, 2, s);
    long nb = tile_pairs(P.n);
    k_build_D<float><<<(unsigned)nb, TB * TB, 0, s>>>(
        P.d_pw64, P.d_pw32, P.n, P.h_ew32, P.d_ewc, P.d_tab32, P.tab32_i0, P.ntab32, P.d_km32, nk,
        P.d_cos32, P.d_sin32, P.p.overlap_corr,
        (float)P.p.r_c, D32, D16, is_bf16, P.ld, P.recip_tc, P.tc_split == kSymShape ? 1 : 0,
        P.d_pairw);
    count_launches(1);
    return BD_OK;
}

// the pair estimate of D(R) without storing D (matrix-free steps): the
// assembly kernel with no output, the reciprocal sum per pair from the trig
// tables (launch_matfree_tables must have run for R)
void launch_pair_estimate(Plan &P, cudaStream_t s)
{
    launch_zero_i32((int32_t *)P.d_pairw, 2, s);
    long nb = tile_pairs(P.n);
    if (is_mixed(P))
        k_build_D<float><<<(unsigned)nb, TB * TB, 0, s>>>(
            P.d_pw64, P.d_pw32, P.n, P.h_ew32, P.d_ewc, P.d_tab32, P.tab32_i0, P.ntab32,
            P.d_km32, P.nk, P.d_cos32, P.d_sin32, P.p.overlap_corr, (float)P.p.r_c, nullptr,
            nullptr, 0, P.ld, 0, 0, P.d_pairw);
    else
        k_build_D<double><<<(unsigned)nb, TB * TB, 0, s>>>(
            P.d_pw64, P.d_pw32, P.n, P.h_ew64, P.d_ewc, P.d_tab, P.tab_i0, P.ntab, P.d_km64,
            P.nk, P.d_cos, P.d_sin, P.p.overlap_corr, (float)P.p.r_c, nullptr, nullptr, 0,
            P.ld, 0, 0, P.d_pairw);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Matrix-free product Y = D(R) X (the paper's LMA: D is never stored).
//
// Real space: one thread per row bead nu; a block of kMfRows threads walks all
// beads mu in tiles, evaluates the block B_{nu mu} with the same pair code as
// the assembly (images, overlap branch, self term) and accumulates
// y_nu += B_{nu mu} x_mu for every column in shared memory (per-thread
// slots, written back once: deterministic, no atomics).  Every unordered
// pair is evaluated twice (once per row), which keeps the sum per row in a
// fixed order.
// Reciprocal space: structure factors S_k = sum_mu (cos, sin)(k.r_mu) x_mu
// per half-space k and column, then y_nu += sum_k m_k (cos_nu S^c_k +
// sin_nu S^s_k) with the folded tensors m_k = 2 f(k)(I - khat khat).
constexpr int kMfRows = 128;

template <typename T>
__global__ void __launch_bounds__(kMfRows)
k_pair_apply(const double *__restrict__ pw, const float *__restrict__ pw32, int n,
             const __grid_constant__ EwaldT<T> c, const T *__restrict__ tab, int tab_i0, int ntab,
             int overlap_corr, float rc, const double *__restrict__ X, int m,
             double *__restrict__ Y, int nchunk, double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char mf_smem[];
    T *ys = (T *)mf_smem;                          // [3m][kMfRows]
    T *xs = ys + (size_t)3 * m * kMfRows;          // [kMfRows][3m]
    const int tid = threadIdx.x;
    const int nu = blockIdx.x * kMfRows + tid;
    const long n3 = 3L * n;
    const int w = 3 * m;
    // this block's share of the beads mu (chunk blockIdx.y of nchunk)
    const int mlo = (int)((long)n * blockIdx.y / nchunk), mhi = (int)((long)n * (blockIdx.y + 1) / nchunk);
    for (int i = tid; i < w * kMfRows; i += kMfRows) ys[i] = (T)0;
    for (int j0 = mlo; j0 < mhi; j0 += kMfRows) {
        __syncthreads();
        for (int e = tid; e < kMfRows * w; e += kMfRows) {
            const int j = e / w, r = e % w, col = r / 3, b = r % 3, mu = j0 + j;
            xs[e] = mu < mhi ? (T)X[(long)col * n3 + 3L * mu + b] : (T)0;
        }
        __syncthreads();
        if (nu < n) {
            const int jn = min(kMfRows, mhi - j0);
            for (int j = 0; j < jn; j++) {
                T acc[6] = {0, 0, 0, 0, 0, 0};
                pair_real<T>(pw, pw32, n3, nu, j0 + j, c, tab, tab_i0, ntab, overlap_corr, rc, acc);
                const T *x = xs + (size_t)j * w;
                for (int col = 0; col < m; col++) {
                    const T x0 = x[3 * col], x1 = x[3 * col + 1], x2 = x[3 * col + 2];
                    T *y = ys + (size_t)(3 * col) * kMfRows + tid;
                    y[0] += acc[0] * x0 + acc[1] * x1 + acc[2] * x2;
                    y[kMfRows] += acc[1] * x0 + acc[3] * x1 + acc[4] * x2;
                    y[2 * kMfRows] += acc[2] * x0 + acc[4] * x1 + acc[5] * x2;
                }
            }
        }
    }
    double *out = nchunk > 1 ? part + (size_t)blockIdx.y * n3 * m : Y;
    if (nu < n)
        for (int col = 0; col < m; col++)
            for (int a = 0; a < 3; a++)
                out[(long)col * n3 + 3L * nu + a] = (double)ys[(size_t)(3 * col + a) * kMfRows + tid];
}

// Y = sum over chunks of the partial products, in chunk order (deterministic)
__global__ void k_sum_chunks(const double *__restrict__ part, int nchunk, long len,
                             double *__restrict__ Y)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double v = 0.0;
    for (int c = 0; c < nchunk; c++) v += part[(size_t)c * len + i];
    Y[i] = v;
}

// S[(t m + col) 6 + {0,1,2}] = sum_mu cos_t(mu) x_mu[b], {3,4,5}: the sine sums;
// one block per (k, column), fixed-order block reduction
template <typename T>
__global__ void k_struct_factor(const T *__restrict__ cs, const T *__restrict__ sn, int n,
                                const double *__restrict__ X, int m, T *__restrict__ S)
{
    __shared__ T red[6][8];
    const int t = blockIdx.x, col = blockIdx.y;
    const long n3 = 3L * n;
    T v[6] = {0, 0, 0, 0, 0, 0};
    for (int mu = threadIdx.x; mu < n; mu += blockDim.x) {
        const T cm = cs[(size_t)t * n + mu], sm = sn[(size_t)t * n + mu];
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const T x = (T)X[(long)col * n3 + 3L * mu + b];
            v[b] += cm * x;
            v[3 + b] += sm * x;
        }
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; q++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) red[q][wp] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        T a = (T)0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) a += red[threadIdx.x][i];
        S[((size_t)t * m + col) * 6 + threadIdx.x] = a;
    }
}

// Y[col][3 nu + a] += sum_k sum_b m_k[ab] (cos_nu S^c_k[col][b] + sin_nu S^s_k[col][b])
template <typename T>
__global__ void k_recip_apply(const T *__restrict__ cs, const T *__restrict__ sn,
                              const T *__restrict__ km, int nk, const T *__restrict__ S, int m,
                              int n, double *__restrict__ Y)
{
    const int nu = blockIdx.x * blockDim.x + threadIdx.x, col = blockIdx.y;
    if (nu >= n) return;
    T y0 = 0, y1 = 0, y2 = 0;
    for (int t = 0; t < nk; t++) {
        const T cn = cs[(size_t)t * n + nu], sv = sn[(size_t)t * n + nu];
        const T *sf = S + ((size_t)t * m + col) * 6;
        const T q0 = cn * sf[0] + sv * sf[3], q1 = cn * sf[1] + sv * sf[4],
                q2 = cn * sf[2] + sv * sf[5];
        const T *mk = km + 12 * (size_t)t;
        y0 += mk[0] * q0 + mk[1] * q1 + mk[2] * q2;
        y1 += mk[1] * q0 + mk[3] * q1 + mk[4] * q2;
        y2 += mk[2] * q0 + mk[4] * q1 + mk[5] * q2;
    }
    const long n3 = 3L * n;
    double *out = Y + (long)col * n3 + 3L * nu;
    out[0] += (double)y0;
    out[1] += (double)y1;
    out[2] += (double)y2;
}

size_t matfree_smem(const Plan &P, int m)
{
    return (size_t)6 * m * kMfRows * (is_mixed(P) ? sizeof(float) : sizeof(double));
}

// mu chunks of the matrix-free product: enough blocks for ~4 per SM
static int matfree_chunks(const Plan &P)
{
    const int rows = (P.n + kMfRows - 1) / kMfRows;
    int c = (4 * (P.num_sms > 0 ? P.num_sms : 152) + rows - 1) / rows;
    const int cap = P.n / kMfRows;               // at least one row tile of beads per chunk
    if (c > cap) c = cap;
    if (c > 32) c = 32;
    return c < 1 ? 1 : c;
}

bd_status matfree_init(Plan &P)
{
    if (P.d_sfac) return BD_OK;
    if (P.num_sms <= 0) cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device);
    P.mf_chunks = matfree_chunks(P);
    if (P.mf_chunks > 1) {
        size_t pc = (size_t)P.mf_chunks * P.n3 * (P.p.max_rhs + 3);
        cudaError_t e = cudaMalloc(&P.d_mfpart, pc * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(BD_ERR_OOM, "matrix-free partials: %s", cudaGetErrorString(e));
        }
        P.scratch_bytes += (int64_t)(pc * sizeof(double));
    }
    size_t cnt = (size_t)(P.nk > 0 ? P.nk : 1) * (P.p.max_rhs + 3) * 6 + 8;
    size_t wn = (size_t)P.n3 * P.p.max_rhs;
    cudaError_t e = cudaMalloc(&P.d_sfac, cnt * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_mfW, wn * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BD_ERR_OOM, "matrix-free scratch: %s", cudaGetErrorString(e));
    }
    P.scratch_bytes += (int64_t)((cnt + wn) * sizeof(double));
    cudaFuncSetAttribute(k_pair_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    cudaFuncSetAttribute(k_pair_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    return check_launch("matrix-free init");
}

bd_status launch_matfree_tables(Plan &P, const double *R, cudaStream_t s)
{
    if (P.pme) {
        launch_wrap(P, R, s);
        return spectral_tables(P, s);
    }
    launch_trig_tables(P, R, s);
    return BD_OK;
}

bd_status matfree_product(Plan &P, const double *X, int m, double *Y, cudaStream_t s)
{
    if (P.pme) return launch_apply_spectral(P, X, m, Y, s);
    return launch_apply_matfree(P, X, m, Y, s);
}

bd_status launch_apply_matfree(Plan &P, const double *X, int m, double *Y, cudaStream_t s)
{
    bd_status st = matfree_init(P);
    if (st != BD_OK) return st;
    const size_t sm = matfree_smem(P, m);
    if (sm > 227 * 1024)
        return set_error(BD_ERR_UNSUPPORTED, "matrix-free product: m = %d columns need %zu bytes "
                         "of shared memory", m, sm);
    const dim3 nb((unsigned)((P.n + kMfRows - 1) / kMfRows), (unsigned)P.mf_chunks);
    const long len = (long)P.n3 * m;
    if (!is_mixed(P)) {
        k_pair_apply<double><<<nb, kMfRows, sm, s>>>(P.d_pw64, P.d_pw32, P.n, P.h_ew64, P.d_tab,
                                                     P.tab_i0, P.ntab, P.p.overlap_corr,
                                                     (float)P.p.r_c, X, m, Y, P.mf_chunks,
                                                     P.d_mfpart);
        count_launches(1);
        if (P.mf_chunks > 1) {
            k_sum_chunks<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(P.d_mfpart, P.mf_chunks, len, Y);
            count_launches(1);
        }
        if (P.nk > 0) {
            double *S = (double *)P.d_sfac;
            k_struct_factor<double><<<dim3(P.nk, m), 256, 0, s>>>(P.d_cos, P.d_sin, P.n, X, m, S);
            k_recip_apply<double><<<dim3((P.n + 127) / 128, m), 128, 0, s>>>(
                P.d_cos, P.d_sin, P.d_km64, P.nk, S, m, P.n, Y);
            count_launches(2);
        }
    } else {
        k_pair_apply<float><<<nb, kMfRows, sm, s>>>(P.d_pw64, P.d_pw32, P.n, P.h_ew32, P.d_tab32,
                                                    P.tab32_i0, P.ntab32, P.p.overlap_corr,
                                                    (float)P.p.r_c, X, m, Y, P.mf_chunks,
                                                    P.d_mfpart);
        count_launches(1);
        if (P.mf_chunks > 1) {
            k_sum_chunks<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(P.d_mfpart, P.mf_chunks, len, Y);
            count_launches(1);
        }
        if (P.nk > 0) {
            float *S = (float *)P.d_sfac;
            k_struct_factor<float><<<dim3(P.nk, m), 256, 0, s>>>(P.d_cos32, P.d_sin32, P.n, X, m, S);
            k_recip_apply<float><<<dim3((P.n + 127) / 128, m), 128, 0, s>>>(
                P.d_cos32, P.d_sin32, P.d_km32, P.nk, S, m, P.n, Y);
            count_launches(2);
        }
    }
    return check_launch("matrix-free product");
}

// ---------------------------------------------------------------------------
// Real-space part of the spectral product as a neighbour table (the Verlet
// tables of the paper's outlook, Sec. VIII).  With r_c < L/2 a pair has at
// most its minimum image within r_c, and only beads of the cells within
// `span` cells of a bead's cell (cell edge >= r_c / span) can be that close.
// The positions are fixed through a step, so for every row (bead in cell
// order) the table holds the rows within r_c -- itself included, with the
// self term -- and the six components of their block of Eqs. (M1) and
// (DFmodified), built once per position set; each product is then a sparse
// 3x3-block product over the table.  Entries are ordered by neighbour cell and
// then by row, and a row's sum is reduced in a fixed order: deterministic.

// minimum-image separation from split positions (hi + lo; lo = 0 for FP64)
template <typename T>
__device__ __forceinline__ void sep_split(const T *ah, const T *al, const T *bh, const T *bl,
                                          const EwaldT<T> &c, T d[3])
{
#pragma unroll
    for (int s = 0; s < 3; s++) {
        T a = ah[s], b = -bh[s];
        T hs = a + b;                                      // TwoSum(a, b)
        T bb = hs - a;
        T he = (a - (hs - bb)) + (b - bb);
        he += al[s] - bl[s];
        if (hs > c.halfL) { hs -= c.L; he -= c.Llo; }
        else if (hs < -c.halfL) { hs += c.L; he += c.Llo; }
        d[s] = hs + he;
    }
}

template <typename T> struct PosSplit;
template <> struct PosSplit<double> {
    __device__ static void get(const double *pw, const float *, long, int i, double h[3], double l[3])
    {
        for (int s = 0; s < 3; s++) { h[s] = pw[3 * i + s]; l[s] = 0.0; }
    }
};
template <> struct PosSplit<float> {
    __device__ static void get(const double *, const float *pw32, long n3, int i, float h[3], float l[3])
    {
        for (int s = 0; s < 3; s++) { h[s] = pw32[3 * i + s]; l[s] = pw32[n3 + 3 * i + s]; }
    }
};

// positions in cell order (row r is bead cell_beads[r]): 32 bytes a row, the
// working-precision split (hi, lo) of the wrapped position
struct __align__(32) RowPos64 { double x, y, z, w; };

template <typename T> struct RowPos;
template <> struct RowPos<double> {
    using V = RowPos64;
    __device__ static void get(const V *rp, int r, double h[3], double l[3])
    {
        const RowPos64 v = rp[r];
        h[0] = v.x; h[1] = v.y; h[2] = v.z;
        l[0] = l[1] = l[2] = 0.0;
    }
};
template <> struct RowPos<float> {
    using V = float4;   // two per row: hi, lo
    __device__ static void get(const float4 *rp, int r, float h[3], float l[3])
    {
        const float4 a = rp[2 * r], b = rp[2 * r + 1];
        h[0] = a.x; h[1] = a.y; h[2] = a.z;
        l[0] = b.x; l[1] = b.y; l[2] = b.z;
    }
};

__global__ void k_row_positions(const double *__restrict__ pw, const float *__restrict__ pw32,
                                int n, const int *__restrict__ cell_beads, int dbl,
                                void *__restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int nu = cell_beads[r];
    if (dbl) {
        ((RowPos64 *)out)[r] = RowPos64{pw[3 * nu], pw[3 * nu + 1], pw[3 * nu + 2], 0.0};
    } else {
        const long n3 = 3L * n;
        float4 *o = (float4 *)out;
        o[2 * r] = make_float4(pw32[3 * nu], pw32[3 * nu + 1], pw32[3 * nu + 2], 0.f);
        o[2 * r + 1] = make_float4(pw32[n3 + 3 * nu], pw32[n3 + 3 * nu + 1], pw32[n3 + 3 * nu + 2], 0.f);
    }
}

// one warp per row: the candidate rows of the row's (2 span + 1)^3 cells are
// taken 32 at a time in a fixed order (cells in offset order, rows ascending
// inside a cell).  FILL = false counts those within r_c (the row itself
// included) into row_start[r]; FILL = true writes them, in that order, to nbr
// (and the row to prow) from row_start[r] on.  The two passes take the same
// decisions (u is formed with explicit fused operations); the fill still stops
// at the next row's start and pads a short row (prow = -1: a zero block), so a
// row never writes outside its own entries.
constexpr int kMaxNbrCells = 125;
constexpr int kPairWarps = 8;

template <typename T, bool FILL>
__global__ void __launch_bounds__(32 * kPairWarps)
k_real_pairs(const typename RowPos<T>::V *__restrict__ rp, int n,
             const __grid_constant__ EwaldT<T> c, const int *__restrict__ cell_start,
             const int *__restrict__ cell_beads, const int *__restrict__ cell_of, int nc, int span,
             int *__restrict__ row_start, int *__restrict__ nbr, int *__restrict__ prow)
{
    __shared__ int s_lo[kPairWarps][kMaxNbrCells];       // first candidate row of each cell
    __shared__ int s_pre[kPairWarps][kMaxNbrCells + 1];  // candidates before each cell
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int r = blockIdx.x * kPairWarps + wid;
    if (r >= n) return;                                  // the whole warp
    const int cell = cell_of[cell_beads[r]];
    const int cx = cell / (nc * nc), cy = (cell / nc) % nc, cz = cell % nc;
    const int w = 2 * span + 1, ncells = w * w * w;
    int *lo = s_lo[wid], *pre = s_pre[wid];
    for (int t = lane; t < ncells; t += 32) {
        const int dx = t / (w * w) - span, dy = (t / w) % w - span, dz = t % w - span;
        const int c2 = (((cx + dx + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cz + dz + nc) % nc;
        lo[t] = cell_start[c2];
        pre[t + 1] = cell_start[c2 + 1] - cell_start[c2];
    }
    __syncwarp();
    if (lane == 0) {
        pre[0] = 0;
        for (int t = 1; t <= ncells; t++) pre[t] += pre[t - 1];
    }
    __syncwarp();
    const int total = pre[ncells];
    T mh[3], ml[3];
    RowPos<T>::get(rp, r, mh, ml);
    long k = FILL ? (long)row_start[r] : 0;
    const long kend = FILL ? (long)row_start[r + 1] : 0;
    int cnt = 0, cc = 0;
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        bool in = false;
        int j = 0;
        if (t < total) {
            while (pre[cc + 1] <= t) cc++;               // t grows: the cell cursor only advances
            j = lo[cc] + (t - pre[cc]);
            if (j == r) {
                in = true;
            } else {
                T h[3], l[3], d[3];
                RowPos<T>::get(rp, j, h, l);
                sep_split<T>(mh, ml, h, l, c, d);
                const T u = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
                in = u <= c.rc2;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (FILL) {
            if (in) {
                const long kk = k + __popc(bal & ((1u << lane) - 1u));
                if (kk < kend) {
                    nbr[kk] = j;
                    prow[kk] = r;
                }
            }
            k += __popc(bal);
        } else {
            cnt += __popc(bal);
        }
    }
    if (FILL) {
        for (long kk = k + lane; kk < kend; kk += 32) {
            nbr[kk] = r;
            prow[kk] = -1;
        }
    } else if (lane == 0) {
        row_start[r] = cnt;
    }
}

// the 3x3 blocks of the table, one thread per entry: real-space image,
// overlap branch or the self term (Eqs. M1, DFmodified, DF)
template <typename T>
__global__ void k_pair_blocks(const typename RowPos<T>::V *__restrict__ rp,
                              const __grid_constant__ EwaldT<T> c, const T *__restrict__ tab,
                              int tab_i0, int ntab, int overlap_corr, const int *__restrict__ prow,
                              const int *__restrict__ nbr, long np, T *__restrict__ tens, long cap)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int r = prow[k];
    T acc[6] = {0, 0, 0, 0, 0, 0};
    if (r >= 0) {
        const int j = nbr[k];
        if (j == r) {
            acc[0] = c.self; acc[3] = c.self; acc[5] = c.self;
        } else {
            T mh[3], ml[3], h[3], l[3], d[3];
            RowPos<T>::get(rp, r, mh, ml);
            RowPos<T>::get(rp, j, h, l);
            sep_split<T>(mh, ml, h, l, c, d);
            const T u = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
            if (u >= c.four_a2) add_m1_tab<T>(d[0], d[1], d[2], u, tab, tab_i0, ntab, acc);
            else if (overlap_corr) add_overlap<T>(d[0], d[1], d[2], u, c, acc);
            else add_m1<T>(d[0], d[1], d[2], u, c, acc);
        }
    }
#pragma unroll
    for (int q = 0; q < 6; q++) tens[q * cap + k] = acc[q];
}

// operand rows in cell order, by column chunk: xr[(ch n + r) ldx + i] =
// X[ch cw + i / 3][3 cell_beads[r] + i % 3] for i < 3 cw (zero padding up to
// ldx and past the last column)
template <typename T>
__global__ void k_pack_rows(const double *__restrict__ X, int n, int m, int cw, int ldx,
                            long len, const int *__restrict__ cell_beads, T *__restrict__ xr)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= len) return;
    const long per = (long)n * ldx;
    const int ch = (int)(idx / per);
    const long rem = idx - ch * per;
    const int r = (int)(rem / ldx), i = (int)(rem - (long)r * ldx);
    const int col = ch * cw + i / 3;
    double v = 0.0;
    if (i < 3 * cw && col < m) v = X[(long)col * 3 * n + 3L * cell_beads[r] + i % 3];
    xr[idx] = (T)v;
}

// Y[col][3 nu + a] = sum over the row's entries of block(nu, mu) x_mu: one warp
// per row, lanes over the entries, a butterfly sum over the lanes (every
// lane ends with the same, order-fixed sum); CC columns per pass
template <typename T, int CC>
__global__ void __launch_bounds__(256)
k_real_pairs_apply(int n, const int *__restrict__ cell_beads, const int *__restrict__ row_start,
                   const int *__restrict__ nbr, const T *__restrict__ tens, long cap,
                   const T *__restrict__ xr, int ldx, int m, int cw, double *__restrict__ Y)
{
    constexpr int VW = 16 / sizeof(T);
    constexpr int NV = (3 * CC + VW - 1) / VW;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    const int k0 = row_start[r], k1 = row_start[r + 1];
    const int nu = cell_beads[r];
    const long n3 = 3L * n;
    for (int c0 = 0, ch = 0; c0 < m; c0 += cw, ch++) {
        const int nx = 3 * min(cw, m - c0);
        const T *xc = xr + (size_t)ch * n * ldx;
        T acc[3 * CC];
#pragma unroll
        for (int i = 0; i < 3 * CC; i++) acc[i] = (T)0;
        for (int k = k0 + lane; k < k1; k += 32) {
            const T t0 = tens[k], t1 = tens[cap + k], t2 = tens[2 * cap + k];
            const T t3 = tens[3 * cap + k], t4 = tens[4 * cap + k], t5 = tens[5 * cap + k];
            const T *xj = xc + (size_t)nbr[k] * ldx;
            T xv[NV * VW];
#pragma unroll
            for (int v = 0; v < NV; v++) {
                if (v * VW < ldx) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(xj + v * VW);
                    memcpy(&xv[v * VW], &u, 16);
                } else {
#pragma unroll
                    for (int e = 0; e < VW; e++) xv[v * VW + e] = (T)0;
                }
            }
#pragma unroll
            for (int q = 0; q < 3 * CC; q += 3) {
                if (q < nx) {
                    const T x0 = xv[q], x1 = xv[q + 1], x2 = xv[q + 2];
                    acc[q] += t0 * x0 + t1 * x1 + t2 * x2;
                    acc[q + 1] += t1 * x0 + t3 * x1 + t4 * x2;
                    acc[q + 2] += t2 * x0 + t4 * x1 + t5 * x2;
                }
            }
        }
        T mine = (T)0;
#pragma unroll
        for (int i = 0; i < 3 * CC; i++) {
            T v = acc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == i) mine = v;
        }
        if (lane < nx) Y[(long)(c0 + lane / 3) * n3 + 3L * nu + lane % 3] = (double)mine;
    }
}

static void chunk_shape(int m, int cc, int vw, int *nchunk, int *cw, int *ldx)
{
    *nchunk = (m + cc - 1) / cc;
    *cw = (m + *nchunk - 1) / *nchunk;
    *ldx = (3 * *cw + vw - 1) / vw * vw;
}

static bd_status pairs_oom(const char *what, cudaError_t e)
{
    cudaGetLastError();
    return set_error(BD_ERR_OOM, "spectral product %s: %s", what, cudaGetErrorString(e));
}

template <typename T>
static void pairs_pass(Plan &P, const EwaldT<T> &c, bool fill, cudaStream_t s)
{
    PmeState *S = P.pme;
    const unsigned nb = (unsigned)((P.n + kPairWarps - 1) / kPairWarps);
    const auto *rp = (const typename RowPos<T>::V *)S->d_rowpos;
    if (fill)
        k_real_pairs<T, true><<<nb, 32 * kPairWarps, 0, s>>>(
            rp, P.n, c, S->d_cell_start, S->d_cell_beads, S->d_cell_of, S->nc, S->span,
            S->d_row_start, S->d_nbr, S->d_prow);
    else
        k_real_pairs<T, false><<<nb, 32 * kPairWarps, 0, s>>>(
            rp, P.n, c, S->d_cell_start, S->d_cell_beads, S->d_cell_of, S->nc, S->span,
            S->d_row_start, nullptr, nullptr);
    count_launches(1);
}

bd_status build_real_pairs(Plan &P, cudaStream_t s)
{
    PmeState *S = P.pme;
    if (S->span > 2) return set_error(BD_ERR_INVALID, "cell search span %d > 2", S->span);
    const bool dbl = !is_mixed(P);
    const size_t ts = dbl ? sizeof(double) : sizeof(float);
    k_row_positions<<<(P.n + 255) / 256, 256, 0, s>>>(P.d_pw64, P.d_pw32, P.n, S->d_cell_beads,
                                                      dbl ? 1 : 0, S->d_rowpos);
    count_launches(1);
    if (dbl) pairs_pass<double>(P, P.h_ew64, false, s);
    else pairs_pass<float>(P, P.h_ew32, false, s);
    // counts -> starts (the counts array doubles as the cursor array of the scan)
    launch_scan_counts(S->d_row_start, P.n, S->d_row_start, s);
    count_launches(1);
    cudaMemcpyAsync(S->h_npair, S->d_row_start + P.n, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(BD_ERR_CUDA, "neighbour count: %s", cudaGetErrorString(e));
    const long np = (long)*(const int *)S->h_npair;
    const size_t per = 2 * sizeof(int) + 6 * ts;
    if (np > S->pair_cap) {
        void *old[] = {S->d_nbr, S->d_prow, S->d_tens};
        for (void *q : old)
            if (q) cudaFree(q);
        S->d_nbr = S->d_prow = nullptr;
        S->d_tens = nullptr;
        P.scratch_bytes -= (int64_t)(S->pair_cap * per);
        const long cap = np + np / 8 + 1024;
        e = cudaMalloc((void **)&S->d_nbr, sizeof(int) * cap);
        if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_prow, sizeof(int) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&S->d_tens, 6 * ts * cap);
        if (e != cudaSuccess) {
            S->pair_cap = 0;
            return pairs_oom("neighbour table", e);
        }
        S->pair_cap = cap;
        P.scratch_bytes += (int64_t)(cap * per);
    }
    S->npair = np;
    const unsigned nbp = (unsigned)((np + 255) / 256);
    if (dbl) {
        pairs_pass<double>(P, P.h_ew64, true, s);
        k_pair_blocks<double><<<nbp, 256, 0, s>>>((const RowPos64 *)S->d_rowpos, P.h_ew64, P.d_tab,
                                                   P.tab_i0, P.ntab, P.p.overlap_corr, S->d_prow,
                                                   S->d_nbr, np, (double *)S->d_tens, S->pair_cap);
    } else {
        pairs_pass<float>(P, P.h_ew32, true, s);
        k_pair_blocks<float><<<nbp, 256, 0, s>>>((const float4 *)S->d_rowpos, P.h_ew32, P.d_tab32,
                                                  P.tab32_i0, P.ntab32, P.p.overlap_corr, S->d_prow,
                                                  S->d_nbr, np, (float *)S->d_tens, S->pair_cap);
    }
    count_launches(1);
    return check_launch("neighbour table");
}

template <typename T, int CC>
static bd_status real_pairs_apply(Plan &P, const double *X, int m, double *Y, cudaStream_t s)
{
    PmeState *S = P.pme;
    int nchunk, cw, ldx;
    chunk_shape(m, CC, 16 / (int)sizeof(T), &nchunk, &cw, &ldx);
    const long len = (long)nchunk * P.n * ldx;
    if (len > S->xrows_len)
        return set_error(BD_ERR_INVALID, "operand rows: %ld elements > %ld", len, S->xrows_len);
    T *xr = (T *)S->d_xrows;
    k_pack_rows<T><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(X, P.n, m, cw, ldx, len,
                                                                  S->d_cell_beads, xr);
    k_real_pairs_apply<T, CC><<<(unsigned)((P.n + 7) / 8), 256, 0, s>>>(
        P.n, S->d_cell_beads, S->d_row_start, S->d_nbr, (const T *)S->d_tens, S->pair_cap, xr, ldx,
        m, cw, Y);
    count_launches(2);
    return check_launch("real-space pairs");
}

long real_pairs_rows_len(int n, int mcap, bool dbl)
{
    int nchunk, cw, ldx;
    if (dbl) {
        chunk_shape(mcap, kPairCols64, 2, &nchunk, &cw, &ldx);
        ldx = (3 * kPairCols64 + 1) / 2 * 2;
    } else {
        chunk_shape(mcap, kPairCols32, 4, &nchunk, &cw, &ldx);
        ldx = (3 * kPairCols32 + 3) / 4 * 4;
    }
    return (long)nchunk * n * ldx;
}

bd_status launch_real_pairs(Plan &P, const double *X, int m, double *Y, cudaStream_t s)
{
    if (!P.pme->d_nbr) return set_error(BD_ERR_INVALID, "spectral product without its tables");
    if (!is_mixed(P)) return real_pairs_apply<double, kPairCols64>(P, X, m, Y, s);
    return real_pairs_apply<float, kPairCols32>(P, X, m, Y, s);
}

}  // namespace bd
