// vec_kernels.cu -- the O(N) and O(N m) parts of the step: forces (Sec. II A),
// Chebyshev coefficients and first term (Eqs. cheb1-cheb3), the error
// estimate E_f (Sec. IV), Lanczos bounds (FP64 recurrence, bisection on the
// tridiagonal matrix), the device Wiener generator (Philox4x32-10 + Box-
// Muller) and the Euler update with FENE rejection (Eq. sde, Sec. VII).
#include <math.h>

#include "bd_internal.cuh"
#include "pair_bound.cuh"

namespace bd {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum, result valid in thread 0
__device__ double block_sum(double v)
{
    __shared__ double sh[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// ---------------------------------------------------------------------------
// Forces

// springs: F^c(Q_mu) - F^c(Q_{mu-1}), Hookean F^c = Q, FENE F^c = Q/(1-Q^2/b)
__global__ void k_springs(const double *R, int n, int nb, int fene, double b, double *F,
                          int32_t *n_bad)
{
    int nu = blockIdx.x * blockDim.x + threadIdx.x;
    if (nu >= n) return;
    int j = nu % nb;
    double f[3] = {0.0, 0.0, 0.0};
    int bad = 0;
    if (j + 1 < nb) {            // spring to the next bead: +F^c(Q_nu)
        double Q[3], q2 = 0.0;
        for (int s = 0; s < 3; s++) { Q[s] = R[3 * (nu + 1) + s] - R[3 * nu + s]; q2 += Q[s] * Q[s]; }
        double g = 1.0;
        if (fene) {
            if (q2 >= b) { g = NAN; bad = 1; }
            else g = 1.0 / (1.0 - q2 / b);
        }
        for (int s = 0; s < 3; s++) f[s] += g * Q[s];
    }
    if (j > 0) {                 // spring from the previous bead: -F^c(Q_{nu-1})
        double Q[3], q2 = 0.0;
        for (int s = 0; s < 3; s++) { Q[s] = R[3 * nu + s] - R[3 * (nu - 1) + s]; q2 += Q[s] * Q[s]; }
        double g = 1.0;
        if (fene) g = (q2 >= b) ? NAN : 1.0 / (1.0 - q2 / b);
        for (int s = 0; s < 3; s++) f[s] -= g * Q[s];
    }
    for (int s = 0; s < 3; s++) F[3 * nu + s] = f[s];
    if (bad && n_bad) atomicAdd(n_bad, 1);
}

// narrow-Gaussian excluded volume over all pairs and periodic images with
// |r| <= r_ev: F_nu += (z*/d*^5) r exp(-r^2/(2 d*^2)).  One warp per bead nu,
// its lanes over the other beads mu (coalesced position loads), the images of
// each pair's minimum-image separation (exact remainder) within r_ev; the
// lanes' partial forces are then combined by a butterfly of shuffles, the
// same order on every run.
constexpr int kEvWarps = 4;

__global__ void __launch_bounds__(32 * kEvWarps)
k_ev(const double *__restrict__ R, int n, double L, double pref, double inv2d2, double rev2,
     int nmax, double *__restrict__ F)
{
    const int nu = blockIdx.x * kEvWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (nu >= n) return;                           // the whole warp leaves together
    const double rn0 = R[3 * nu], rn1 = R[3 * nu + 1], rn2 = R[3 * nu + 2];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int mu = lane; mu < n; mu += 32) {
        if (mu == nu) continue;
        const double d0 = remainder(rn0 - R[3 * mu], L);      // exact minimum image
        const double d1 = remainder(rn1 - R[3 * mu + 1], L);
        const double d2 = remainder(rn2 - R[3 * mu + 2], L);
        for (int ix = -nmax; ix <= nmax; ix++) {
            const double vx = d0 + ix * L;
            if (vx * vx > rev2) continue;
            for (int iy = -nmax; iy <= nmax; iy++) {
                const double vy = d1 + iy * L;
                if (vx * vx + vy * vy > rev2) continue;
                for (int iz = -nmax; iz <= nmax; iz++) {
                    const double vz = d2 + iz * L;
                    const double u = vx * vx + vy * vy + vz * vz;
                    if (u > rev2) continue;
                    const double w = pref * exp(-u * inv2d2);
                    acc[0] += w * vx; acc[1] += w * vy; acc[2] += w * vz;
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 3; s++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], o);
    if (lane == 0)
        for (int s = 0; s < 3; s++) F[3 * nu + s] += acc[s];
}

void launch_forces(Plan &P, const double *R, double *F, int32_t *n_bad, cudaStream_t s)
{
    int n = P.n;
    k_springs<<<(n + 127) / 128, 128, 0, s>>>(R, n, P.p.beads_per_chain, P.p.spring == 1,
                                               P.p.fene_b, F, n_bad);
    count_launches(1);
    if (P.p.ev_on) {
        double d = P.p.d_star;
        double pref = P.p.z_star / (d * d * d * d * d);
        int nmax = (int)floor(P.p.r_ev / P.p.box_L + 0.5) + 1;
        k_ev<<<(n + kEvWarps - 1) / kEvWarps, 32 * kEvWarps, 0, s>>>(
            R, n, P.p.box_L, pref, 1.0 / (2.0 * d * d), P.p.r_ev * P.p.r_ev, nmax, F);
        count_launches(1);
    }
}

// ---------------------------------------------------------------------------
// Chebyshev (Sec. IV)

// c_p = (2/N) sum_j sqrt(h cos t_j + mid) cos(p t_j), t_j = pi (j + 1/2)/N:
// the coefficients of the Chebyshev interpolant of sqrt on [d_min, d_max].
// c_p = (2/N) sum_j f(cos t_j) cos(p t_j), t_j = pi (j + 1/2)/N: one block per
// p, the terms summed in a fixed order (each thread a strided subset, then a
// fixed tree)
__global__ void k_cheb_coeffs(const double *bounds, int nch, double *c)
{
    __shared__ double red[64];
    const int p = blockIdx.x;
    const double dmin = bounds[0], dmax = bounds[1];
    const double h = 0.5 * (dmax - dmin), mid = 0.5 * (dmax + dmin);
    double v = 0.0;
    for (int j = threadIdx.x; j < nch; j += blockDim.x) {
        double t = kPi * (j + 0.5) / nch;
        v += sqrt(h * cos(t) + mid) * cos(p * t);
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 32; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) c[p] = 2.0 * red[0] / nch;
    if (p == 0 && threadIdx.x == 0) {
        c[kChebMapS] = 2.0 / (dmax - dmin);
        c[kChebMapT] = (dmax + dmin) / (dmax - dmin);
    }
}

void launch_cheb_coeffs(Plan &P, const double *bounds, int nch, cudaStream_t s)
{
    k_cheb_coeffs<<<nch, 64, 0, s>>>(bounds, nch, P.d_coef);
    count_launches(1);
}

// V0 = dW, V1 = Y V0 = s (D dW) - t dW, dS = (c0/2) dW + c1 V1
__global__ void k_cheb_first(const double *dW, const double *DW, long len, const double *bounds,
                             const double *coef, double *V0, double *V1, double *dS)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    (void)bounds;
    const double ys = coef[kChebMapS], yt = coef[kChebMapT];
    double w = dW[i];
    double v1 = ys * DW[i] - yt * w;
    V0[i] = w;
    V1[i] = v1;
    dS[i] = coef[0] * w - 0.5 * coef[0] * w + coef[1] * v1;
}

void launch_cheb_first(Plan &P, const double *bounds, const double *dW, const double *DW, int m,
                       double *V0, double *V1, double *dS, cudaStream_t s)
{
    long len = (long)P.n3 * m;
    k_cheb_first<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(dW, DW, len, bounds, P.d_coef, V0,
                                                               V1, dS);
    count_launches(1);
}

// one Chebyshev term from a plain product W = D V_{p-1} (matrix-free steps):
// V_p = 2 (s W - t V_{p-1}) - V_{p-2} over V_{p-2}, dS += c_p V_p
__global__ void k_cheb_term(const double *W, const double *V1, double *V2, long len,
                            const double *bounds, const double *coef, int p, double *dS)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    (void)bounds;
    const double ys = coef[kChebMapS], yt = coef[kChebMapT];
    double v = 2.0 * (ys * W[i] - yt * V1[i]) - V2[i];
    V2[i] = v;
    dS[i] += coef[p] * v;
}

void launch_cheb_term(Plan &P, const double *W, const double *V1, double *V2, int m,
                      const double *bounds, int p, double *dS, cudaStream_t s)
{
    long len = (long)P.n3 * m;
    k_cheb_term<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(W, V1, V2, len, bounds, P.d_coef, p,
                                                              dS);
    count_launches(1);
}

// Deterministic column dot products: block b writes its partial sum of
// column j to part[j * kRedBlocks + b]; one warp per column then adds the
// partials in block order.  No atomics, so every run gives the same bits.

__global__ void k_dot_cols_part(const double *A, const double *B, int n3, double *part)
{
    int j = blockIdx.y;
    double v = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (long)gridDim.x * blockDim.x)
        v += A[(long)j * n3 + i] * B[(long)j * n3 + i];
    v = block_sum(v);
    if (threadIdx.x == 0) part[j * kRedBlocks + blockIdx.x] = v;
}

__global__ void k_sum_parts(const double *part, int nparts, double *out)
{
    int j = blockIdx.x;
    double v = 0.0;
    for (int b = threadIdx.x; b < nparts; b += 32) v += part[j * kRedBlocks + b];
    // fixed-shape warp tree
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[j] = v;
}

void launch_dot_cols(const double *A, const double *B, int n3, int m, double *out, double *part,
                     cudaStream_t s)
{
    int bx = min(kRedBlocks, (n3 + 255) / 256);
    k_dot_cols_part<<<dim3(bx, m), 256, 0, s>>>(A, B, n3, part);
    count_launches(1);
    k_sum_parts<<<m, 32, 0, s>>>(part, bx, out);
    count_launches(1);
}

// E_f = sqrt(|dS.dS - dW.D.dW| / dW.D.dW) per column; stats->ef_max
__global__ void k_ef(const double *ss, const double *wdw, int m, double *Ef, bd_step_stats *st)
{
    if (threadIdx.x != 0) return;
    double mx = 0.0;
    for (int j = 0; j < m; j++) {
        double e = sqrt(fabs(ss[j] - wdw[j]) / wdw[j]);
        if (Ef) Ef[j] = e;
        mx = fmax(mx, e);
    }
    if (st) st->ef_max = mx;
}

void launch_ef(Plan &P, const double *dW, const double *DW, const double *dS, int m, double *Ef,
               bd_step_stats *stats, cudaStream_t s)
{
    launch_dot_cols(dW, DW, P.n3, m, P.d_wdw, P.d_redpart, s);
    launch_dot_cols(dS, dS, P.n3, m, P.d_red, P.d_redpart, s);
    k_ef<<<1, 32, 0, s>>>(P.d_red, P.d_wdw, m, Ef, stats);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        uint32_t y0 = hi1 ^ c[1] ^ k0, y2 = hi0 ^ c[3] ^ k1;
        c[0] = y0; c[1] = lo1; c[2] = y2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

__global__ void k_wiener(uint64_t seed, uint64_t step, int64_t count, double sdt, double *out,
                         const unsigned long long *step_dev)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * q >= count) return;
    if (step_dev) step = *step_dev;
    uint32_t c[4] = {(uint32_t)q, (uint32_t)((uint64_t)q >> 32), (uint32_t)step,
                     (uint32_t)(step >> 32)};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    uint64_t b1 = ((uint64_t)c[0] << 32) | c[1];
    uint64_t b2 = ((uint64_t)c[2] << 32) | c[3];
    double u1 = ((double)(b1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = ((double)(b2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double rr = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[2 * q] = sdt * rr * cs;
    if (2 * q + 1 < count) out[2 * q + 1] = sdt * rr * sn;
}

void launch_wiener(Plan &P, uint64_t seed, uint64_t step, int64_t count, double *out,
                   cudaStream_t s, const unsigned long long *step_dev)
{
    int64_t pairs = (count + 1) / 2;
    k_wiener<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(seed, step, count, sqrt(P.p.dt), out,
                                                             step_dev);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Lanczos: q_1 from a fixed Philox stream, then
//   w = D q_j; alpha_j = q_j.w; w -= alpha_j q_j + beta_{j-1} q_{j-1};
//   beta_j = |w|; q_{j+1} = w / beta_j.
// d_lq[0] = q_{j-1}, d_lq[1] = q_j, d_lq[2] = w;  d_lab = {alpha[], beta[]}
// d_red[0] = q_j.w, d_red[1] = |w|^2 (after the update)

__global__ void k_lanczos_start(double *q, double *qprev, int n3)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    uint32_t c[4] = {(uint32_t)i, 0u, 0x4C414E43u, 0u};
    philox4x32_10(c, 0x5EEDu, 0xB0u);
    q[i] = ((double)c[0] + 0.5) * (1.0 / 4294967296.0) - 0.5;
    qprev[i] = 0.0;
}

__global__ void k_scale_by_inv_sqrt(double *q, int n3, const double *nrm2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) q[i] *= rsqrt(*nrm2);
}

void launch_lanczos_init(Plan &P, cudaStream_t s)
{
    int n3 = P.n3;
    k_lanczos_start<<<(n3 + 255) / 256, 256, 0, s>>>(P.d_lq[1], P.d_lq[0], n3);
    count_launches(1);
    launch_dot_cols(P.d_lq[1], P.d_lq[1], n3, 1, P.d_red + 2, P.d_redpart, s);
    k_scale_by_inv_sqrt<<<(n3 + 255) / 256, 256, 0, s>>>(P.d_lq[1], n3, P.d_red + 2);
    count_launches(1);
}

// w -= alpha q - beta_prev qprev; per-block partial |w|^2 (ordered sum after)
__global__ void k_lanczos_orth(double *w, const double *q, const double *qprev, int n3,
                               const double *alpha, const double *beta_prev, double *part)
{
    double a = *alpha, b = beta_prev ? *beta_prev : 0.0;
    double v = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (long)gridDim.x * blockDim.x) {
        double x = w[i] - a * q[i] - b * qprev[i];
        w[i] = x;
        v += x * x;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// beta_j = sqrt(nrm2); qprev <- q; q <- w / beta_j
__global__ void k_lanczos_shift(double *qprev, double *q, const double *w, int n3,
                                const double *nrm2, double *beta)
{
    double bj = sqrt(*nrm2);
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *beta = bj;
    if (i >= n3) return;
    qprev[i] = q[i];
    q[i] = bj > 0.0 ? w[i] / bj : 0.0;
}

// called after w = D q_j (w: d_lq[2] unless given; it is overwritten)
void launch_lanczos_update(Plan &P, int j, cudaStream_t s, double *w)
{
    int n3 = P.n3;
    if (!w) w = P.d_lq[2];
    double *alpha = P.d_lab + j, *beta = P.d_lab + kMaxLanczos + j;
    double *beta_prev = j > 0 ? P.d_lab + kMaxLanczos + j - 1 : nullptr;
    launch_dot_cols(P.d_lq[1], w, n3, 1, alpha, P.d_redpart, s);
    double *part = P.d_redpart;
    int bx = min(kRedBlocks, (n3 + 255) / 256);
    k_lanczos_orth<<<bx, 256, 0, s>>>(w, P.d_lq[1], P.d_lq[0], n3, alpha, beta_prev, part);
    count_launches(1);
    k_sum_parts<<<1, 32, 0, s>>>(part, bx, P.d_red + 1);
    count_launches(1);
    k_lanczos_shift<<<(n3 + 255) / 256, 256, 0, s>>>(P.d_lq[0], P.d_lq[1], w, n3,
                                                     P.d_red + 1, beta);
    count_launches(1);
}

// number of eigenvalues of the k x k tridiagonal (alpha, beta^2) below x: sign
// changes of the Sturm sequence p_0 = 1, p_i = (alpha_i - x) p_{i-1} -
// beta_{i-1}^2 p_{i-2} (leading principal minors of T - x I).  FP32 (the FP64
// pipe of this GPU issues 2 operations per clock per SM; the bounds need a
// few digits, and FP32 resolves the Ritz values to ~1e-6 of |T|).  No
// division: the pair (p_{i-1}, p_i) is rescaled by a power of two when it
// grows or shrinks too far, which changes no sign.  A zero p_i keeps the
// sign of p_{i-1}.
__device__ int sturm_count(const float *al, const float *b2, int k, float x)
{
    float pm = 1.f, p = al[0] - x;
    bool neg = p < 0.f;
    int cnt = neg ? 1 : 0;
    for (int i = 1; i < k; i++) {
        float pn = (al[i] - x) * p - b2[i - 1] * pm;
        bool nn = pn < 0.f || (pn == 0.f && neg);
        cnt += (nn != neg) ? 1 : 0;
        neg = nn;
        pm = p;
        p = pn;
        float mx = fmaxf(fabsf(p), fabsf(pm));
        if (mx > 0x1p+60f || (mx < 0x1p-60f && mx > 0.f)) {
            int e;
            frexpf(mx, &e);
            p = ldexpf(p, -e);
            pm = ldexpf(pm, -e);
        }
    }
    return cnt;
}

// Extreme Ritz values of the k x k tridiagonal matrix by multisection on
// Sturm counts: 128 threads per end test 128 interior points of the current
// bracket (Gershgorin at the start), which shrinks it 129-fold per round,
// until it is 1e-6 of the value wide (at most 6 rounds).
// Then the widened bounds {d_min, d_max} and a status word.  Launched with
// 256 threads.
__global__ void k_lanczos_finish(const double *lab, int k, double smax, double fmin_,
                                 double *bounds, int32_t *status)
{
    __shared__ double br[2][2];
    __shared__ int first[2];
    __shared__ int kk;
    __shared__ float alf[kMaxLanczos], b2f[kMaxLanczos];
    const int g = threadIdx.x >> 7, t = threadIdx.x & 127;
    const double *al = lab, *be = lab + kMaxLanczos;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        alf[i] = (float)al[i];
        b2f[i] = (float)(be[i] * be[i]);
    }
    if (threadIdx.x == 0) {
        // stop at a breakdown (beta ~ 0: the Krylov space became invariant)
        double scale = 0.0;
        for (int i = 0; i < k; i++) scale = fmax(scale, fabs(al[i]));
        int kt = k;
        for (int i = 0; i + 1 < k; i++)
            if (!(fabs(be[i]) > 1e-13 * scale)) { kt = i + 1; break; }
        double lo = 1e300, hi = -1e300;
        for (int i = 0; i < kt; i++) {
            double rad = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < kt ? fabs(be[i]) : 0.0);
            lo = fmin(lo, al[i] - rad);
            hi = fmax(hi, al[i] + rad);
        }
        kk = kt;
        br[0][0] = br[1][0] = lo;
        br[0][1] = br[1][1] = hi;
    }
    __syncthreads();
    const int kt = kk;
    const int target = (g == 0) ? 1 : kt;        // smallest x with count(x) >= target
    for (int it = 0; it < 6; it++) {
        const double a = br[g][0], b = br[g][1];
        const bool done = !(b - a > 1e-6 * fmax(fabs(a), fabs(b)));
        if (t == 0) first[g] = 128;
        __syncthreads();
        if (!done) {
            double x = a + (b - a) * (t + 1) / 129.0;
            if (sturm_count(alf, b2f, kt, (float)x) >= target) atomicMin(&first[g], t);
        }
        __syncthreads();
        if (t == 0 && !done) {
            const int f = first[g];
            br[g][0] = f == 0 ? a : a + (b - a) * f / 129.0;
            br[g][1] = f == 128 ? b : a + (b - a) * (f + 1) / 129.0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double th0 = 0.5 * (br[0][0] + br[0][1]), th1 = 0.5 * (br[1][0] + br[1][1]);
        double dmin = fmin_ * th0, dmax = (1.0 + smax) * th1;
        bounds[0] = dmin;
        bounds[1] = dmax;
        if (status) *status = (dmin > 0.0 && dmax > dmin) ? BD_OK : BD_ERR_NOT_PD;
    }
}

void launch_lanczos_finish(Plan &P, int k, double safety_max, double dmin_fraction,
                           double *bounds, int32_t *status, cudaStream_t s)
{
    k_lanczos_finish<<<1, 256, 0, s>>>(P.d_lab, k, safety_max, dmin_fraction, bounds, status);
    count_launches(1);
}

// Fixman's estimates (Sec. IV): U+ (all ones) and U- (alternating +1, -1)
// as two columns of the first product
__global__ void k_fixman_fill(double *X, int n3)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    X[i] = 1.0;
    X[n3 + i] = (i & 1) ? -1.0 : 1.0;
}

// q = {U+.D.U+, U-.D.U-}; lambda^F = q / 3N (Eq. lmax-lmin-dilute), then the
// dilute bounds (2 lambda^F_max, lambda^F_min / 2) or the semidilute ones of
// Eqs. (fmax), (fmin): lambda_max = 0.35 N^0.6 lambda^F_max,
// lambda_min = lambda_max / (C N^0.6)
__global__ void k_fixman_bounds(const double *q, int n3, int nbeads, int mode, double C,
                                double *bounds, int32_t *status)
{
    const double lmaxF = q[0] / n3, lminF = q[1] / n3;
    double dmin, dmax;
    if (mode == BD_BOUNDS_FIXMAN_DILUTE) {
        dmax = 2.0 * lmaxF;
        dmin = 0.5 * lminF;
    } else {
        const double n06 = pow((double)nbeads, 0.6);
        dmax = 0.35 * n06 * lmaxF;
        dmin = dmax / (C * n06);
    }
    bounds[0] = dmin;
    bounds[1] = dmax;
    if (status) *status = (dmin > 0.0 && dmax > dmin) ? BD_OK : BD_ERR_NOT_PD;
}

void launch_fixman_fill(double *X, int n3, cudaStream_t s)
{
    k_fixman_fill<<<(n3 + 255) / 256, 256, 0, s>>>(X, n3);
    count_launches(1);
}

void launch_fixman_bounds(Plan &P, const double *X2, const double *Y2, int mode, double C,
                          double *bounds, int32_t *status, cudaStream_t s)
{
    launch_dot_cols(X2, Y2, P.n3, 2, P.d_red + 2 * kMaxRhs, P.d_redpart, s);
    k_fixman_bounds<<<1, 1, 0, s>>>(P.d_red + 2 * kMaxRhs, P.n3, P.n, mode, C, bounds, status);
    count_launches(1);
}

// status of given bounds (lagged mode)

// the pair estimate from a stored D: one thread per block (nu, mu), nu < mu
// (the strictly upper blocks, which every layout of D holds), block rows nu =
// blockIdx.y + k gridDim.y; the symmetric part of the block is used
template <typename T>
__global__ void k_pair_radius_scan(const T *__restrict__ D, int n, long ld, unsigned *word)
{
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    float rho = 0.f;
    for (int nu = blockIdx.y; nu < n - 1; nu += gridDim.y) {
        if (mu > nu && mu < n) {
            const T *b = D + (size_t)3 * nu * ld + 3 * mu;
            const float a00 = (float)b[0], a11 = (float)b[ld + 1], a22 = (float)b[2 * ld + 2];
            const float a01 = 0.5f * ((float)b[1] + (float)b[ld]);
            const float a02 = 0.5f * ((float)b[2] + (float)b[2 * ld]);
            const float a12 = 0.5f * ((float)b[ld + 2] + (float)b[2 * ld + 1]);
            rho = fmaxf(rho, pair_block_radius(a00, a01, a02, a11, a12, a22));
        }
    }
    warp_max_to_word(rho, word);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) word[1] = __float_as_uint((float)D[0]);
}

void launch_pair_radius_scan(const void *D, int f32, int n, long ld, unsigned *word,
                             cudaStream_t s)
{
    launch_zero_i32((int32_t *)word, 2, s);
    dim3 g((unsigned)((n + 255) / 256), (unsigned)(n - 1 < 1 ? 1 : (n - 1 < 65535 ? n - 1 : 65535)));
    if (f32) k_pair_radius_scan<float><<<g, 256, 0, s>>>((const float *)D, n, ld, word);
    else k_pair_radius_scan<double><<<g, 256, 0, s>>>((const double *)D, n, ld, word);
    count_launches(1);
}

// d_min = min(d_min, f theta_pair), theta_pair = d_s - rho_max (pair_bound.cuh).
// theta_pair <= 0 means a 6 x 6 principal submatrix of D is not positive
// definite, and then neither is D: the status says so.
__global__ void k_bounds_pair(double *b, const unsigned *word, double f, int32_t *status)
{
    const double ds = (double)__uint_as_float(word[1]);
    const double rho = (double)__uint_as_float(word[0]);
    const double th = ds - rho;
    const double dmin = th > 0.0 ? fmin(b[0], f * th) : f * th;
    b[0] = dmin;
    if (status) *status = (dmin > 0.0 && b[1] > dmin) ? BD_OK : BD_ERR_NOT_PD;
}

void launch_bounds_pair(double *bounds, const unsigned *word, double dmin_fraction,
                        int32_t *status, cudaStream_t s)
{
    k_bounds_pair<<<1, 1, 0, s>>>(bounds, word, dmin_fraction, status);
    count_launches(1);
}

// stats bookkeeping for bd_step
__global__ void k_stats_bounds(bd_step_stats *st, const double *bounds, const int32_t *bstatus)
{
    st->d_min = bounds[0];
    st->d_max = bounds[1];
    if (*bstatus != BD_OK) st->status = *bstatus;
}

// the start of a step in one launch: the statistics record and the plan's
// eight status words
__global__ void k_step_begin(bd_step_stats *st, int nch, int32_t *status)
{
    if (threadIdx.x == 0) {
        st->d_min = 0.0; st->d_max = 0.0; st->ef_max = 0.0;
        st->n_cheb = nch; st->n_overstretched = 0; st->accepted = 0; st->status = BD_OK;
    }
    if (threadIdx.x < 8) status[threadIdx.x] = 0;
}

void launch_step_begin(bd_step_stats *st, int nch, int32_t *status, cudaStream_t s)
{
    k_step_begin<<<1, 32, 0, s>>>(st, nch, status);
    count_launches(1);
}

// the lagged bounds of a step in one launch: the previous step's Lanczos
// interval, d_min tightened by this step's pair estimate (as k_bounds_pair),
// and the statistics record
__global__ void k_bounds_lagged(double *b, const double *lag, const unsigned *word, double f,
                                int32_t *status, bd_step_stats *st)
{
    const double ds = (double)__uint_as_float(word[1]);
    const double rho = (double)__uint_as_float(word[0]);
    const double th = ds - rho;
    const double dmin = th > 0.0 ? fmin(lag[0], f * th) : f * th;
    const double dmax = lag[1];
    b[0] = dmin;
    b[1] = dmax;
    const int32_t bs = (dmin > 0.0 && dmax > dmin) ? BD_OK : BD_ERR_NOT_PD;
    *status = bs;
    st->d_min = dmin;
    st->d_max = dmax;
    if (bs != BD_OK) st->status = bs;
}

void launch_bounds_lagged(double *bounds, const double *lag, const unsigned *word,
                          double dmin_fraction, int32_t *status, bd_step_stats *st, cudaStream_t s)
{
    k_bounds_lagged<<<1, 1, 0, s>>>(bounds, lag, word, dmin_fraction, status, st);
    count_launches(1);
}

void launch_stats_bounds(bd_step_stats *st, const double *bounds, const int32_t *bstatus,
                         cudaStream_t s)
{
    k_stats_bounds<<<1, 1, 0, s>>>(st, bounds, bstatus);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Euler update, Eq. (sde) with kappa = 0, and FENE rejection

__global__ void k_euler_propose(const double *R, const double *DF, const double *dS, int n3,
                                double dt, double *Rn)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    Rn[i] = R[i] + 0.25 * dt * DF[i] + dS[i] * 0.70710678118654752440;
}

__global__ void k_fene_check(const double *Rn, int n, int nb, double b, int32_t *over)
{
    int nu = blockIdx.x * blockDim.x + threadIdx.x;
    if (nu >= n || (nu % nb) + 1 >= nb) return;
    double q2 = 0.0;
    for (int s = 0; s < 3; s++) {
        double q = Rn[3 * (nu + 1) + s] - Rn[3 * nu + s];
        q2 += q * q;
    }
    if (q2 >= b) atomicAdd(over, 1);
}

__global__ void k_commit(double *R, const double *Rn, int n3, const int32_t *over,
                         const int32_t *in_bad, bd_step_stats *st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t timeout = in_bad[4];           // status word 6: a bounded wait gave up
    bool ok = (*over == 0) && (*in_bad == 0) && timeout == 0;
    if (ok && i < n3) R[i] = Rn[i];
    if (i == 0 && st) {
        st->n_overstretched = *over;
        st->accepted = ok ? 1 : 0;
        if (timeout) st->status = BD_ERR_TIMEOUT;
        else if (!ok) st->status = BD_ERR_FENE_STRETCH;
    }
}

void launch_euler(Plan &P, double *R, const double *DF, const double *dS, bd_step_stats *stats,
                  cudaStream_t s)
{
    int n3 = P.n3;
    k_euler_propose<<<(n3 + 255) / 256, 256, 0, s>>>(R, DF, dS, n3, P.p.dt, P.d_Rnew);
    count_launches(1);
    int32_t *over = P.d_status + 1;
    launch_zero_i32(over, 1, s);
    if (P.p.spring == 1) {
        k_fene_check<<<(P.n + 127) / 128, 128, 0, s>>>(P.d_Rnew, P.n, P.p.beads_per_chain,
                                                      P.p.fene_b, over);
        count_launches(1);
    }
    k_commit<<<(n3 + 255) / 256, 256, 0, s>>>(R, P.d_Rnew, n3, over, P.d_status + 2, stats);
    count_launches(1);
}

__global__ void k_counter_add(unsigned long long *c) { *c += 1ull; }

void launch_counter_add(unsigned long long *ctr, cudaStream_t s)
{
    k_counter_add<<<1, 1, 0, s>>>(ctr);
    count_launches(1);
}

__global__ void k_zero_i32(int32_t *p, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

void launch_zero_i32(int32_t *p, int n, cudaStream_t s)
{
    k_zero_i32<<<(n + 255) / 256, 256, 0, s>>>(p, n);
    count_launches(1);
}

// device-to-device copies of the step as kernels: in a captured step they
// are kernel nodes, where copy nodes would queue on the copy engines (a batch
// of replicas issues several small copies per replica and step)
__global__ void k_copy_f64(double *__restrict__ dst, const double *__restrict__ src, long n)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// dst = [a (na) | b (nb) | c (nc)]: up to three contiguous copies in one launch
__global__ void k_copy3_f64(double *__restrict__ dst, const double *__restrict__ a, long na,
                            const double *__restrict__ b, long nb, const double *__restrict__ c, long nc)
{
    const long n = na + nb + nc;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = i < na ? a[i] : (i < na + nb ? b[i - na] : c[i - na - nb]);
}

void launch_copy3_f64(double *dst, const double *a, size_t na, const double *b, size_t nb,
                      const double *c, size_t nc, cudaStream_t s)
{
    const long blocks = ((long)(na + nb + nc) + 255) / 256;
    k_copy3_f64<<<(unsigned)(blocks < 1216 ? (blocks > 0 ? blocks : 1) : 1216), 256, 0, s>>>(
        dst, a, (long)na, b, (long)nb, c, (long)nc);
    count_launches(1);
}

void launch_copy_f64(double *dst, const double *src, size_t n, cudaStream_t s)
{
    const long blocks = ((long)n + 255) / 256;
    k_copy_f64<<<(unsigned)(blocks < 1216 ? (blocks > 0 ? blocks : 1) : 1216), 256, 0, s>>>(dst, src, (long)n);
    count_launches(1);
}

}  // namespace bd
