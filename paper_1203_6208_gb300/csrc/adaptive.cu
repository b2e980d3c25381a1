// adaptive.cu -- Chebyshev series with an adaptive number of terms (Sec. IV):
// N_Ch starts from Eq. (nint) with the bounds as eigenvalue estimates,
//   N_0 = nint(sqrt(d_max / d_min)) + 1,
// and grows one term at a time until E_f < tol (or N_Ch = max_cheb).
//
// Growing N_Ch changes every coefficient c_p of Eq. (cheb1), so the series
// cannot be extended term by term.  Instead the recurrence vectors V_p of
// Eqs. (cheb2)-(cheb3) are kept (they do not depend on N_Ch) and E_f of
// every candidate N comes from the Chebyshev moments
//   mu_j = dW . T_j(A) dW,   A = (D - sigma I)/h,
// through T_p T_q = (T_{p+q} + T_{|p-q|})/2:
//   |dS(N)|^2 = sum_{p,q<N} c^_p c^_q (mu_{p+q} + mu_{|p-q|})/2,  c^_0 = c_0/2,
//   dW.D.dW  = h mu_1 + sigma mu_0.
// Two dot products per new vector give two new moments,
//   mu_{2p} = 2 V_p.V_p - mu_0,   mu_{2p-1} = 2 V_p.V_{p-1} - mu_1,
// so after V_{N-1} every E_f(N') with N' <= N is known.  The final dS is the
// combination of the stored V_p with the coefficients of the chosen N, and
// E_f is then recomputed directly from it.  The host reads one number per
// candidate N (the stream is synchronised), so this path is not for capture.
#include <math.h>

#include "adaptive.cuh"
#include "adjoint.cuh"
#include "tc_gemm.cuh"

namespace bd {

constexpr int kEfRun = 8;            // consecutive N whose E_f estimates one host wait reads

// partial sums of a.a, a.b and b.b per column (block b of kRedBlocks)
__global__ void k_moment_part(const double *A, const double *B, int n3, double *part)
{
    __shared__ double sh[3][32];
    const int j = blockIdx.y;
    double t[3] = {0.0, 0.0, 0.0};
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (long)gridDim.x * blockDim.x) {
        double a = A[(long)j * n3 + i], b = B[(long)j * n3 + i];
        t[0] += a * a;
        t[1] += a * b;
        t[2] += b * b;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
        if (lane == 0) sh[k][w] = t[k];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) v += sh[threadIdx.x][i];
        part[((size_t)j * kRedBlocks + blockIdx.x) * 3 + threadIdx.x] = v;
    }
}

// one warp per column: sums the partials in block order and stores the new
// moments of V_p (a = V_p, b = V_{p-1}); p = 1 also stores mu_0 and mu_1
__global__ void k_moment_update(const double *part, int nparts, int m, int p, double *mom)
{
    const int j = blockIdx.x, lane = threadIdx.x;
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = lane; b < nparts; b += 32)
        for (int k = 0; k < 3; k++) t[k] += part[((size_t)j * kRedBlocks + b) * 3 + k];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
    if (lane != 0) return;
    if (p == 1) {
        mom[0 * m + j] = t[2];                      // V_0 . V_0
        mom[1 * m + j] = t[1];                      // V_1 . V_0
        mom[2 * m + j] = 2.0 * t[0] - t[2];
    } else {
        mom[(size_t)(2 * p - 1) * m + j] = 2.0 * t[1] - mom[1 * m + j];
        mom[(size_t)(2 * p) * m + j] = 2.0 * t[0] - mom[0 * m + j];
    }
}

// E_f(N) of one column from the moments: block (j, b) takes column j at
// N = N0 + b (N <= 256, 256 threads), so one launch gives the estimates of a
// run of N values for every column.  The interpolant's c_t = (2/N) sum_k f_k
// cos(pi t (k + 1/2) / N), f_k = sqrt(h cos(pi (k + 1/2) / N) + mid): the f_k
// once per block, the cosines of thread t by rotating (cos, sin) through
// the N nodes (four FP64 multiply-adds a node instead of a cosine; the FP64
// pipe of this GPU runs at 1/64 of FP32), then the quadratic form above and
// est[b m + j] = E_f.
__global__ void k_ef_estimate(const double *mom, int m, const double *bounds, int N0, double *est)
{
    __shared__ double c[kMaxCheb];
    __shared__ double f[kMaxCheb];
    __shared__ double red[256];
    const int t = threadIdx.x, j = blockIdx.x, N = N0 + (int)blockIdx.y;
    const double dmin = bounds[0], dmax = bounds[1];
    const double h = 0.5 * (dmax - dmin), mid = 0.5 * (dmax + dmin);
    if (t < N) f[t] = sqrt(h * cospi((t + 0.5) / N) + mid);
    __syncthreads();
    if (t < N) {
        double cd, sd, cr, sr;
        sincospi((double)t / N, &sd, &cd);              // the step between nodes
        sincospi(0.5 * t / N, &sr, &cr);                // the first node
        double s = 0.0;
        for (int k = 0; k < N; k++) {
            s += f[k] * cr;
            const double cn = cr * cd - sr * sd;
            sr = fma(sr, cd, cr * sd);
            cr = cn;
        }
        c[t] = (t == 0 ? 1.0 : 2.0) * s / N;            // c_0 halved in the series
    }
    __syncthreads();
    double v = 0.0;
    if (t < N) {
        for (int q = 0; q < N; q++) {
            const int d = t > q ? t - q : q - t;
            v += c[q] * 0.5 * (mom[(size_t)(t + q) * m + j] + mom[(size_t)d * m + j]);
        }
        v *= c[t];
    }
    red[t] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) {
        const double wdw = h * mom[1 * m + j] + mid * mom[0 * m + j];
        est[(size_t)blockIdx.y * m + j] = sqrt(fabs(red[0] - wdw) / wdw);
    }
}

// dS = (c_0/2) V_0 + c_1 V_1 + sum_{p>=2} c_p V_p, the terms added in the
// order of the fixed-N series
__global__ void k_cheb_combine(const double *V0, const double *hist, long blk, const double *coef,
                               int N, long len, double *dS)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double w = V0[i];
    double d = coef[0] * w - 0.5 * coef[0] * w + coef[1] * hist[i];
    for (int p = 2; p < N; p++) d += coef[p] * hist[(long)(p - 1) * blk + i];
    dS[i] = d;
}

__global__ void k_stats_adaptive(bd_step_stats *st, int nch, int converged)
{
    st->n_cheb = nch;
    if (!converged && st->status == BD_OK) st->status = BD_ERR_CHEB_NOCONV;
}

static bd_status ensure_adaptive_scratch(Plan &P)
{
    if (!P.d_vhist) {
        size_t hist = (size_t)(P.p.max_cheb - 1) * P.n3 * P.p.max_rhs;
        cudaError_t e = cudaMalloc(&P.d_vhist, hist * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(BD_ERR_OOM, "Chebyshev history (%zu doubles): %s", hist,
                             cudaGetErrorString(e));
        }
        P.scratch_bytes += (int64_t)(hist * sizeof(double));
    }
    if (!P.d_mom) {
        size_t nm = (size_t)2 * kMaxCheb * kMaxRhs, np = (size_t)3 * kRedBlocks * kMaxRhs;
        size_t nw = (size_t)P.n3 * P.p.max_rhs;
        cudaError_t e = cudaMalloc(&P.d_mom, (nm + np + kEfRun * kMaxRhs + nw) * sizeof(double));
        if (e == cudaSuccess) e = cudaMallocHost(&P.h_est, kEfRun * kMaxRhs * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(BD_ERR_OOM, "adaptive Chebyshev scratch: %s", cudaGetErrorString(e));
        }
        P.scratch_bytes += (int64_t)((nm + np + kEfRun * kMaxRhs + nw) * sizeof(double));
    }
    return BD_OK;
}

bd_status cheb_adaptive_core(Plan &P, const void *D, const double *bounds, double tol,
                             const double *dW, const double *W, int m, double *dS, double *Ef,
                             bd_step_stats *stats, cudaStream_t s, int *n_used, int *converged)
{
    bd_status st = ensure_adaptive_scratch(P);
    if (st != BD_OK) return st;
    const int n3 = P.n3, nmax = P.p.max_cheb;
    const long blk = (long)n3 * m;
    double *mom = P.d_mom;
    double *part = mom + (size_t)2 * kMaxCheb * kMaxRhs;
    double *est = part + (size_t)3 * kRedBlocks * kMaxRhs;   // [kEfRun][m]
    double *Wp = est + (size_t)kEfRun * kMaxRhs;        // D V_{p-1}, 3N x m
    auto V = [&](int p) -> const double * { return p == 0 ? dW : P.d_vhist + (long)(p - 1) * blk; };
    const unsigned gl = (unsigned)((blk + 255) / 256);
    const int nparts = kRedBlocks < (n3 + 255) / 256 ? kRedBlocks : (n3 + 255) / 256;
    auto moments = [&](int p) {
        k_moment_part<<<dim3(nparts, m), 256, 0, s>>>(V(p), V(p - 1), n3, part);
        k_moment_update<<<m, 32, 0, s>>>(part, nparts, m, p, mom);
        count_launches(2);
    };
    // the bounds decide N_0 (Eq. nint with d_max / d_min for the eigenvalue ratio)
    cudaMemcpyAsync(P.h_est, bounds, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch("adaptive Chebyshev bounds");
    const double dmin = P.h_est[0], dmax = P.h_est[1];
    int N = 2;
    if (dmin > 0.0 && dmax > dmin) N = (int)floor(sqrt(dmax / dmin) + 0.5) + 1;
    if (N < 2) N = 2;
    if (N > nmax) N = nmax;
    // V_1 = (W - sigma dW)/h
    launch_cheb_hist(W, dW, nullptr, blk, bounds, 1.0, 1.0, P.d_vhist, s);
    moments(1);
    int p = 1;                       // highest V computed
    int conv = 0;
    // N grows by one until E_f < tol; the estimates of a run of up to kEfRun
    // consecutive N are taken in one launch and read with one host wait, and
    // the first N of the run below tol is the answer (the same N as one
    // check per term; the few extra terms of the run are left unused)
    for (;;) {
        const int Nhi = N + kEfRun - 1 < nmax ? N + kEfRun - 1 : nmax;
        while (p < Nhi - 1) {        // V_p = 2 (D V_{p-1} - sigma V_{p-1})/h - V_{p-2}
            p++;
            st = apply_dense(P, D, V(p - 1), m, Wp, s);
            if (st != BD_OK) return st;
            launch_cheb_hist(Wp, V(p - 1), V(p - 2), blk, bounds, 2.0, 1.0,
                               P.d_vhist + (long)(p - 1) * blk, s);
            moments(p);
        }
        const int run = Nhi - N + 1;
        k_ef_estimate<<<dim3(m, run), 256, 0, s>>>(mom, m, bounds, N, est);
        count_launches(1);
        cudaMemcpyAsync(P.h_est, est, sizeof(double) * run * m, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch("adaptive Chebyshev");
        int hit = -1;
        for (int b = 0; b < run && hit < 0; b++) {
            double mx = 0.0;
            for (int j = 0; j < m; j++) mx = fmax(mx, P.h_est[b * m + j]);
            if (mx < tol) hit = b;
        }
        if (hit >= 0) {
            N += hit;
            conv = 1;
            break;
        }
        if (Nhi >= nmax) {
            N = nmax;
            break;
        }
        N = Nhi + 1;
    }
    launch_cheb_coeffs(P, bounds, N, s);
    k_cheb_combine<<<gl, 256, 0, s>>>(dW, P.d_vhist, blk, P.d_coef, N, blk, dS);
    count_launches(1);
    launch_ef(P, dW, W, dS, m, Ef, stats, s);
    if (stats) {
        k_stats_adaptive<<<1, 1, 0, s>>>(stats, N, conv);
        count_launches(1);
    }
    if (n_used) *n_used = N;
    if (converged) *converged = conv;
    return check_launch("adaptive Chebyshev");
}

}  // namespace bd
