// adjoint.cu -- reverse mode of the drift product D(R).F and of the
// Chebyshev series dS = P(D) dW with respect to the bead positions R.
//
// D_{nu mu} = B(r_nu - r_mu) for nu != mu (Eq. DFmodified; the diagonal
// blocks do not depend on R).  When dL/dD = sum_q x_q y_q^T, the gradient is
// a pair sum
//   dL/dr_nu^c = sum_{mu != nu} sum_ab dB_ab/dd_c (d_{nu mu}) S_ab,
//   S = (W + W^T)/2,  W_ab = sum_q x_q[nu a] y_q[mu b] + x_q[mu a] y_q[nu b],
// and the contribution of a pair enters r_nu with + and r_mu with - (dB/dd is
// odd in d).  The kernel recomputes each pair's image sum instead of storing
// dD: per image, the radial form f1(u) I + f2(u) v v^T gives
//   dB:S = 2 v (f1' tr S + f2' v.S.v) + 2 f2 S v,
// with f1, f2 and their u-derivatives from the same M1 table as the forward
// assembly (derivative by Horner), from the Taylor series of the smooth
// Ewald remainder on the overlap branch, and from the reciprocal sum
//   -sum_k (m_k : S) k sin(k.d),  sin(k.d) = s_nu c_mu - c_nu s_mu.
// Contributions are reduced per tile row / column in shared memory and
// added to gR with atomics (order-dependent in the last bits).
#include <math.h>

#include "adjoint.cuh"
#include "pair_common.cuh"

namespace bd {

constexpr int ATB = 16;

template <typename T> struct AMath;
template <> struct AMath<double> {
    __device__ static double rsqrt_(double x) { return rsqrt(x); }
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double erfc_(double x) { return erfc(x); }
    __device__ static double exp_(double x) { return exp(x); }
};
template <> struct AMath<float> {
    __device__ static float rsqrt_(float x) { return rsqrtf(x); }
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float erfc_(float x) { return erfcf(x); }
    __device__ static float exp_(float x) { return expf(x); }
};


template <typename T>
__device__ __forceinline__ void horner_d(const double *cf, int n, T x, T &p, T &dp)
{
    p = (T)cf[n - 1];
    dp = (T)0;
    for (int j = n - 2; j >= 0; j--) {
        dp = dp * x + p;
        p = p * x + (T)cf[j];
    }
}

// dB:S for one image of the radial form f1(u) I + f2(u) v v^T
template <typename T>
__device__ __forceinline__ void radial_contract(T vx, T vy, T vz, T f1p, T f2, T f2p,
                                                const T S[6], T g[3])
{
    // S: xx xy xz yy yz zz
    T Sv0 = S[0] * vx + S[1] * vy + S[2] * vz;
    T Sv1 = S[1] * vx + S[3] * vy + S[4] * vz;
    T Sv2 = S[2] * vx + S[4] * vy + S[5] * vz;
    T trS = S[0] + S[3] + S[5];
    T vSv = vx * Sv0 + vy * Sv1 + vz * Sv2;
    T a = (T)2 * (f1p * trS + f2p * vSv), b = (T)2 * f2;
    g[0] += a * vx + b * Sv0;
    g[1] += a * vy + b * Sv1;
    g[2] += a * vz + b * Sv2;
}

template <typename T>
__global__ void __launch_bounds__(ATB *ATB)
k_pair_adjoint(const double *__restrict__ R, int n, const EwaldCoef *__restrict__ ewc,
               const T *__restrict__ tab, int tab_i0, int ntab, const T *__restrict__ km, int nk,
               const T *__restrict__ cs, const T *__restrict__ sn, int overlap_corr, float rc,
               const double *__restrict__ X, const double *__restrict__ Y, int Q, long n3,
               double *__restrict__ gR)
{
    __shared__ double red_row[ATB][ATB][3];
    __shared__ double red_col[ATB][ATB][3];
    long idx = blockIdx.x;
    int J = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while ((long)J * (J + 1) / 2 > idx) J--;
    while ((long)(J + 1) * (J + 2) / 2 <= idx) J++;
    int I = (int)(idx - (long)J * (J + 1) / 2);
    int ty = threadIdx.x / ATB, tx = threadIdx.x % ATB;
    int nu = I * ATB + ty, mu = J * ATB + tx;
    const EwaldCoef &c = *ewc;
    T gacc[3] = {0, 0, 0};
    if (nu < n && mu < n && !(I == J && ty >= tx)) {
        // symmetric source S from the Q outer products
        T S[6] = {0, 0, 0, 0, 0, 0};
        {
            double W[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int q = 0; q < Q; q++) {
                const double *xq = X + (long)q * n3, *yq = Y + (long)q * n3;
                double xn[3] = {xq[3 * nu], xq[3 * nu + 1], xq[3 * nu + 2]};
                double xm[3] = {xq[3 * mu], xq[3 * mu + 1], xq[3 * mu + 2]};
                double yn[3] = {yq[3 * nu], yq[3 * nu + 1], yq[3 * nu + 2]};
                double ym[3] = {yq[3 * mu], yq[3 * mu + 1], yq[3 * mu + 2]};
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) W[3 * a + b] += xn[a] * ym[b] + xm[a] * yn[b];
            }
            S[0] = (T)W[0];
            S[1] = (T)(0.5 * (W[1] + W[3]));
            S[2] = (T)(0.5 * (W[2] + W[6]));
            S[3] = (T)W[4];
            S[4] = (T)(0.5 * (W[5] + W[7]));
            S[5] = (T)W[8];
        }
        const double L = c.L, invL = c.invL;
        double d[3];
        for (int s = 0; s < 3; s++) {
            double x = R[3 * nu + s] - R[3 * mu + s];
            d[s] = remainder(x, L);      // exact, in [-L/2, L/2] for any finite x
        }
        const T rc2 = (T)c.rc2, four_a2 = (T)c.four_a2, Lt = (T)L;
        const T dx = (T)d[0], dy = (T)d[1], dz = (T)d[2];
        const T alpha = (T)c.alpha, alpha2 = (T)c.alpha2, inv_a = (T)c.inv_a;
        ImageCursor cur;
        cur.start((float)d[0], (float)d[1], (float)d[2], (float)L, (float)invL, rc);
        while (!cur.done) {
            T vx = dx + (T)cur.nx * Lt, vy = dy + (T)cur.ny * Lt, vz = dz + (T)cur.nz * Lt;
            T u = vx * vx + vy * vy + vz * vz;
            if (u <= rc2 && u > (T)0) {
                T f1p, f2, f2p;
                if (u >= four_a2) {
                    constexpr int DEG = TabFmt<T>::DEG;
                    int i = (int)(__float_as_uint((float)u) >> TabFmt<T>::SHIFT) - tab_i0;
                    i = i < 0 ? 0 : (i >= ntab ? ntab - 1 : i);
                    const T *row = tab + (size_t)i * TabFmt<T>::STRIDE;
                    T ihw = __ldg(row + 1);
                    T t = (u - __ldg(row)) * ihw;
                    const T *a1 = row + 2, *b1 = row + 2 + (DEG + 1);
                    T p1 = __ldg(a1 + DEG), d1 = (T)0, p2 = __ldg(b1 + DEG), d2 = (T)0;
#pragma unroll
                    for (int k = DEG - 1; k >= 0; k--) {
                        d1 = d1 * t + p1;
                        p1 = p1 * t + __ldg(a1 + k);
                        d2 = d2 * t + p2;
                        p2 = p2 * t + __ldg(b1 + k);
                    }
                    f1p = d1 * ihw;
                    f2 = p2;
                    f2p = d2 * ihw;
                } else if (overlap_corr) {
                    // Omega_B - G (Eq. cor5 reading): e1 = 1 - 9 r/(32a) - G1, e2 = 3/(32 a r) - G2/r^2
                    T s2 = alpha2 * u, r = AMath<T>::sqrt_(u);
                    T A1, dA1, B1, dB1, A2, dA2, B2, dB2;
                    horner_d(c_A1, kNT, s2, A1, dA1);
                    horner_d(c_B1, kNT, s2, B1, dB1);
                    horner_d(c_A2s, kNT, s2, A2, dA2);
                    horner_d(c_B2s, kNT, s2, B2, dB2);
                    (void)A1; (void)B1;
                    T dG1 = alpha2 * ((T)c.g1a * dA1 + (T)c.g1b * dB1);
                    T G2u = (T)c.g2a * A2 + (T)c.g2b * B2;
                    T dG2u = alpha2 * ((T)c.g2a * dA2 + (T)c.g2b * dB2);
                    f1p = -(T)(9.0 / 64.0) * inv_a / r - dG1;
                    f2 = (T)(3.0 / 32.0) * inv_a / r - G2u;
                    f2p = -(T)(3.0 / 64.0) * inv_a / (u * r) - dG2u;
                    (void)alpha;
                } else {
                    // Eq. (M1) directly (Beenakker's form inside 2a, no correction)
                    T rinv = AMath<T>::rsqrt_(u), r = u * rinv, uinv = rinv * rinv;
                    T ec = AMath<T>::erfc_(alpha * r), ex = AMath<T>::exp_(-alpha2 * u);
                    T A1 = (T)c.A1, A3 = (T)c.A3;
                    T q1 = rinv * (A1 + A3 * uinv), q2 = rinv * (A1 - (T)3 * A3 * uinv);
                    T p1 = (((T)c.P2 * u + (T)c.P1) * u + (T)c.P0 + (T)c.Q * uinv);
                    T p2 = (((T)c.R2 * u + (T)c.R1) * u + (T)c.R0 + (T)c.S * uinv);
                    // d/du of erfc(alpha sqrt u) = -alpha e^{-alpha^2 u} / (sqrt(pi) r)
                    T dec = -alpha * ex * (T)0.56418958354775628695 * rinv;
                    T dq1 = -(T)0.5 * rinv * uinv * (A1 + (T)3 * A3 * uinv);
                    T dq2 = -(T)0.5 * rinv * uinv * (A1 - (T)9 * A3 * uinv);
                    T dex = -alpha2 * ex;
                    T dp1 = (T)2 * (T)c.P2 * u + (T)c.P1 - (T)c.Q * uinv * uinv;
                    T dp2 = (T)2 * (T)c.R2 * u + (T)c.R1 - (T)c.S * uinv * uinv;
                    T c2 = ec * q2 + ex * p2;
                    T c2p = dec * q2 + ec * dq2 + dex * p2 + ex * dp2;
                    f1p = dec * q1 + ec * dq1 + dex * p1 + ex * dp1;
                    f2 = c2 * uinv;
                    f2p = c2p * uinv - c2 * uinv * uinv;
                }
                radial_contract<T>(vx, vy, vz, f1p, f2, f2p, S, gacc);
            }
            cur.advance();
        }
        // reciprocal part: -sum_k (m_k : S) k sin(k.d)
        for (int t = 0; t < nk; t++) {
            T snd = sn[(size_t)t * n + nu] * cs[(size_t)t * n + mu]
                  - cs[(size_t)t * n + nu] * sn[(size_t)t * n + mu];
            const T *mk = km + 12 * t;
            T mS = __ldg(mk) * S[0] + __ldg(mk + 3) * S[3] + __ldg(mk + 5) * S[5]
                 + (T)2 * (__ldg(mk + 1) * S[1] + __ldg(mk + 2) * S[2] + __ldg(mk + 4) * S[4]);
            T w = mS * snd;
            gacc[0] -= w * __ldg(mk + 6);
            gacc[1] -= w * __ldg(mk + 7);
            gacc[2] -= w * __ldg(mk + 8);
        }
    }
    for (int s = 0; s < 3; s++) {
        red_row[ty][tx][s] = (double)gacc[s];
        red_col[tx][ty][s] = (double)gacc[s];
    }
    __syncthreads();
    // thread (ty, tx): tx < 3 sums row ty (bead nu); 3 <= tx < 6 sums column ty (bead mu)
    if (tx < 3) {
        int b = I * ATB + ty;
        if (b < n) {
            double v = 0.0;
            for (int k = 0; k < ATB; k++) v += red_row[ty][k][tx];
            atomicAdd(&gR[3 * b + tx], v);
        }
    } else if (tx < 6) {
        int s = tx - 3, b = J * ATB + ty;
        if (b < n) {
            double v = 0.0;
            for (int k = 0; k < ATB; k++) v += red_col[ty][k][s];
            atomicAdd(&gR[3 * b + s], -v);
        }
    }
}

void launch_pair_adjoint(Plan &P, const double *R, const double *X, const double *Y, int Q,
                         double *gR, cudaStream_t s)
{
    launch_trig_tables(P, R, s);
    cudaMemsetAsync(gR, 0, sizeof(double) * P.n3, s);
    long T = (P.n + ATB - 1) / ATB;
    long nb = T * (T + 1) / 2;
    if (P.p.precision == BD_FP64) {
        k_pair_adjoint<double><<<(unsigned)nb, ATB * ATB, 0, s>>>(
            R, P.n, P.d_ewc, P.d_tab, P.tab_i0, P.ntab, P.d_km64, P.nk, P.d_cos, P.d_sin,
            P.p.overlap_corr, (float)P.p.r_c, X, Y, Q, P.n3, gR);
    } else {
        k_pair_adjoint<float><<<(unsigned)nb, ATB * ATB, 0, s>>>(
            R, P.n, P.d_ewc, P.d_tab32, P.tab32_i0, P.ntab32, P.d_km32, P.nk, P.d_cos32, P.d_sin32,
            P.p.overlap_corr, (float)P.p.r_c, X, Y, Q, P.n3, gR);
    }
    count_launches(1);
}

// ---------------------------------------------------------------------------
// elementwise pieces of the Chebyshev forward (stored history) and adjoint

// V_p = a (s DV - t V_{p-1}) - b V_{p-2}   (a = 1, b = 0 for V_1; a = 2, b = 1 after)
__global__ void k_cheb_hist(const double *DV, const double *V1, const double *V2, long len,
                            const double *bounds, double a, double b, double *out)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double dmin = bounds[0], dmax = bounds[1];
    double ys = 2.0 / (dmax - dmin), yt = (dmax + dmin) / (dmax - dmin);
    out[i] = a * (ys * DV[i] - yt * V1[i]) - (V2 ? b * V2[i] : 0.0);
}

// U_p = c_p h + a (s DU - t U_{p+1}) - U_{p+2} (a = 2; the U_0 step uses a = 1
// and c_0/2), and the outer-product factors X_q = k s U_p
__global__ void k_cheb_adj(const double *h, const double *DU, const double *U1, const double *U2,
                           long len, const double *bounds, const double *coef, int p, double a,
                           double cscale, double *out)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double dmin = bounds[0], dmax = bounds[1];
    double ys = 2.0 / (dmax - dmin), yt = (dmax + dmin) / (dmax - dmin);
    double v = cscale * coef[p] * h[i];
    if (DU) v += a * (ys * DU[i] - yt * U1[i]);
    if (U2) v -= U2[i];
    out[i] = v;
}

__global__ void k_scale_copy(const double *src, long len, const double *bounds, double k,
                             double *dst)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double ys = 2.0 / (bounds[1] - bounds[0]);
    dst[i] = k * ys * src[i];
}

void launch_cheb_hist(const double *DV, const double *V1, const double *V2, long len,
                      const double *bounds, double a, double b, double *out, cudaStream_t s)
{
    k_cheb_hist<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(DV, V1, V2, len, bounds, a, b, out);
    count_launches(1);
}

void launch_cheb_adj(const double *h, const double *DU, const double *U1, const double *U2,
                     long len, const double *bounds, const double *coef, int p, double a,
                     double cscale, double *out, cudaStream_t s)
{
    k_cheb_adj<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(h, DU, U1, U2, len, bounds, coef, p,
                                                             a, cscale, out);
    count_launches(1);
}

void launch_scale_copy(const double *src, long len, const double *bounds, double k, double *dst,
                       cudaStream_t s)
{
    k_scale_copy<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(src, len, bounds, k, dst);
    count_launches(1);
}

}  // namespace bd
