// spectral.cu -- the spectral matrix-free product Y = D(R) X.
//
// The paper's outlook (Sec. VIII) names the two ways past its O(N^2) Ewald
// sums: Verlet tables for the real-space part and fast Fourier transforms for
// the Fourier part.  This file is that path for the matrix-free product:
//   * real space with r_c < L/2 (every pair has at most one image within
//     r_c, the minimum image) over a cell list of cells no smaller than
//     r_c / 2, searched two cells deep;
//   * the reciprocal sum of the same truncated k-sphere as the dense D by
//     smooth particle-mesh Ewald: the operand is spread onto a K^3 mesh with
//     cardinal B-splines of order p, transformed (cuFFT, batched R2C), each
//     mesh wave vector m multiplied by G(m) |b(m)|^2 with G = M2(2 pi m / L)
//     of Eq. (M2) for |m|^2 <= n2max (zero otherwise and at m = 0) and b the
//     Euler exponential-spline factors, transformed back and interpolated
//     with the same splines.
// The mesh sum approximates the k-sum by spline interpolation; its error
// falls as (k_max L / (2 pi K))^p.  Spreading accumulates in 64-bit fixed
// point (integer atomics commute, so the mesh is the same on every run); the
// cell lists are ordered by bead index inside each cell, so the real-space
// sums are too.
#include <math.h>

#include <vector>

#include "kspace.cuh"
#include "spectral.cuh"

namespace bd {

constexpr int kMaxOrder = 10;

// a[j] = M_p(f + j), j = 0 .. p-1, for 0 <= f < 1 (cardinal B-spline of order p)
template <typename T>
__host__ __device__ inline void bspline_weights(T f, int p, T *a)
{
    a[0] = f;
    a[1] = (T)1 - f;
    for (int j = 2; j < p; j++) a[j] = (T)0;
    for (int n = 2; n < p; n++) {
        // order n -> n + 1: M_{n+1}(x) = (x M_n(x) + (n + 1 - x) M_n(x - 1)) / n
        const T inv = (T)1 / (T)n;
        for (int j = n; j >= 0; j--) {
            const T x = f + (T)j;
            const T cur = j < n ? a[j] : (T)0;
            const T prev = j > 0 ? a[j - 1] : (T)0;
            a[j] = (x * cur + ((T)(n + 1) - x) * prev) * inv;
        }
    }
}

// |b_d(m)|^2 = 1 / |sum_{j=0}^{p-2} M_p(j + 1) exp(2 pi i m j / K)|^2
static double bspline_mod2(int m, int K, int p)
{
    double a[kMaxOrder];
    bspline_weights<double>(0.0, p, a);       // a[j] = M_p(j)
    double re = 0.0, im = 0.0;
    for (int j = 0; j <= p - 2; j++) {
        const double w = a[j + 1];
        const double ph = 2.0 * 3.14159265358979323846 * m * j / K;
        re += w * cos(ph);
        im += w * sin(ph);
    }
    const double d = re * re + im * im;
    return d > 1e-30 ? 1.0 / d : 0.0;
}

template <typename T>
__global__ void k_pme_influence(int K, int n2max, double a, double alpha, double L,
                                const double *__restrict__ bmod, T *__restrict__ infl)
{
    const long Kh = (long)K * K * (K / 2 + 1);
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Kh) return;
    const int m3 = (int)(idx % (K / 2 + 1));
    const int m2 = (int)((idx / (K / 2 + 1)) % K);
    const int m1 = (int)(idx / ((long)(K / 2 + 1) * K));
    const int s1 = m1 <= K / 2 ? m1 : m1 - K, s2 = m2 <= K / 2 ? m2 : m2 - K, s3 = m3;
    const long n2 = (long)s1 * s1 + (long)s2 * s2 + (long)s3 * s3;
    T *out = infl + 6 * idx;
    if (n2 == 0 || n2 > n2max) {
        for (int i = 0; i < 6; i++) out[i] = (T)0;
        return;
    }
    const double two_pi = 6.283185307179586476925;
    const double k[3] = {two_pi * s1 / L, two_pi * s2 / L, two_pi * s3 / L};
    double m[6];
    m2_tensor(k, a, alpha, L, m);
    const double b2 = bmod[m1] * bmod[K + m2] * bmod[2 * K + m3];
    for (int i = 0; i < 6; i++) out[i] = (T)(m[i] * b2);
}

static bd_status oom(const char *what, cudaError_t e)
{
    cudaGetLastError();
    return set_error(BD_ERR_OOM, "spectral product %s: %s", what, cudaGetErrorString(e));
}

bd_status spectral_init(Plan &P)
{
    if (P.pme) return BD_OK;
    const bd_params &p = P.p;
    PmeState *S = new PmeState();
    memset(S, 0, sizeof(*S));
    P.pme = S;
    S->K = p.pme_grid;
    S->p = p.pme_order;
    // cells of edge >= r_c / 2 searched two deep when the box holds 5 or more
    // of them (5 distinct offsets -2..2), else the whole box as one cell
    const int nc2 = (int)floor(2.0 * p.box_L / p.r_c);
    if (nc2 >= 5) { S->nc = nc2; S->span = 2; }
    else { S->nc = 1; S->span = 0; }
    S->ncell = (long)S->nc * S->nc * S->nc;
    S->K3 = (long)S->K * S->K * S->K;
    S->Kh = (long)S->K * S->K * (S->K / 2 + 1);
    S->mcap = p.max_rhs + 3;
    const bool dbl = !is_mixed(P);
    const size_t ts = dbl ? sizeof(double) : sizeof(float);
    const size_t grids = (size_t)3 * S->mcap;
    cudaError_t e = cudaSuccess;
    size_t bytes = 0;
#define ALLOC(ptr, n)                                                        \
    do {                                                                     \
        if (e == cudaSuccess) {                                              \
            e = cudaMalloc((void **)&(ptr), (n));                            \
            bytes += (n);                                                    \
        }                                                                    \
    } while (0)
    ALLOC(S->d_cell_of, sizeof(int) * P.n);
    ALLOC(S->d_cell_count, sizeof(int) * S->ncell);
    ALLOC(S->d_cell_start, sizeof(int) * (S->ncell + 1));
    ALLOC(S->d_cell_beads, sizeof(int) * P.n);
    ALLOC(S->d_cell_tmp, sizeof(int) * P.n);
    ALLOC(S->d_rpart, sizeof(double) * (2 * S->span + 1) * P.n3 * S->mcap);
    ALLOC(S->d_infl, ts * 6 * S->Kh);
    ALLOC(S->d_qfix, sizeof(unsigned long long) * grids * S->K3);
    ALLOC(S->d_qreal, ts * grids * S->K3);
    ALLOC(S->d_qhat, 2 * ts * grids * S->Kh);
    ALLOC(S->d_xmax, sizeof(unsigned long long) * 4);
#undef ALLOC
    if (e != cudaSuccess) return oom("mesh", e);
    P.scratch_bytes += (int64_t)bytes;
    // influence function (plan constant)
    std::vector<double> bm(3 * (size_t)S->K);
    for (int d = 0; d < 3; d++)
        for (int m = 0; m < S->K; m++) bm[(size_t)d * S->K + m] = bspline_mod2(m, S->K, S->p);
    double *d_bm = nullptr;
    e = cudaMalloc(&d_bm, sizeof(double) * bm.size());
    if (e != cudaSuccess) return oom("spline factors", e);
    cudaMemcpy(d_bm, bm.data(), sizeof(double) * bm.size(), cudaMemcpyHostToDevice);
    const unsigned nb = (unsigned)((S->Kh + 255) / 256);
    if (dbl)
        k_pme_influence<double><<<nb, 256>>>(S->K, p.n2max, p.a, p.alpha, p.box_L, d_bm,
                                            (double *)S->d_infl);
    else
        k_pme_influence<float><<<nb, 256>>>(S->K, p.n2max, p.a, p.alpha, p.box_L, d_bm,
                                           (float *)S->d_infl);
    count_launches(1);
    cudaDeviceSynchronize();
    cudaFree(d_bm);
    return check_launch("spectral init");
}

void spectral_free(Plan &P)
{
    PmeState *S = P.pme;
    if (!S) return;
    void *ptrs[] = {S->d_cell_of, S->d_cell_count, S->d_cell_start, S->d_cell_beads, S->d_cell_tmp,
                    S->d_rpart, S->d_infl,
                    S->d_qfix, S->d_qreal, S->d_qhat, S->d_xmax};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (S->plan_m) {
        cufftDestroy(S->fwd);
        cufftDestroy(S->inv);
    }
    delete S;
    P.pme = nullptr;
}

// ---------------------------------------------------------------------------
// cell list of the wrapped positions (cells of edge L / nc >= r_c)

__global__ void k_cell_assign(const double *__restrict__ pw, int n, int nc, double L,
                              int *__restrict__ cell_of, int *__restrict__ count)
{
    const int nu = blockIdx.x * blockDim.x + threadIdx.x;
    if (nu >= n) return;
    int ci[3];
    for (int s = 0; s < 3; s++) {
        int c = (int)floor(pw[3 * nu + s] * nc / L);
        ci[s] = c < 0 ? 0 : (c >= nc ? nc - 1 : c);
    }
    const int c = (ci[0] * nc + ci[1]) * nc + ci[2];
    cell_of[nu] = c;
    atomicAdd(&count[c], 1);
}

// exclusive prefix sum of the cell counts (one block; each thread a
// contiguous chunk, then the chunk totals in order); the counts become the
// scatter cursors (= start)
__global__ void k_cell_scan(int *__restrict__ count, long ncell, int *__restrict__ start)
{
    __shared__ long tot[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const long per = (ncell + T - 1) / T, lo = t * per, hi = lo + per < ncell ? lo + per : ncell;
    long s = 0;
    for (long i = lo; i < hi; i++) s += count[i];
    tot[t] = s;
    __syncthreads();
    if (t == 0) {
        long run = 0;
        for (int i = 0; i < T; i++) {
            long v = tot[i];
            tot[i] = run;
            run += v;
        }
        start[ncell] = (int)run;
    }
    __syncthreads();
    long run = tot[t];
    for (long i = lo; i < hi; i++) {
        const int v = count[i];
        start[i] = (int)run;
        count[i] = (int)run;      // cursor
        run += v;
    }
}

__global__ void k_cell_scatter(const int *__restrict__ cell_of, int n, int *__restrict__ cursor,
                               int *__restrict__ beads)
{
    const int nu = blockIdx.x * blockDim.x + threadIdx.x;
    if (nu >= n) return;
    const int pos = atomicAdd(&cursor[cell_of[nu]], 1);
    beads[pos] = nu;
}

// ascending bead order inside each cell (fixed summation order): one block per
// cell, every bead's rank is the count of smaller indices in its cell
__global__ void k_cell_sort(const int *__restrict__ start, long ncell, const int *__restrict__ in,
                            int *__restrict__ out)
{
    const long c = blockIdx.x;
    if (c >= ncell) return;
    const int lo = start[c], hi = start[c + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int v = in[i];
        int rank = 0;
        for (int j = lo; j < hi; j++) rank += in[j] < v ? 1 : 0;
        out[lo + rank] = v;
    }
}

void spectral_tables(Plan &P, cudaStream_t s)
{
    PmeState *S = P.pme;
    cudaMemsetAsync(S->d_cell_count, 0, sizeof(int) * S->ncell, s);
    k_cell_assign<<<(P.n + 255) / 256, 256, 0, s>>>(P.d_pw64, P.n, S->nc, P.p.box_L, S->d_cell_of,
                                                   S->d_cell_count);
    k_cell_scan<<<1, 1024, 0, s>>>(S->d_cell_count, S->ncell, S->d_cell_start);
    k_cell_scatter<<<(P.n + 255) / 256, 256, 0, s>>>(S->d_cell_of, P.n, S->d_cell_count,
                                                    S->d_cell_tmp);
    k_cell_sort<<<(unsigned)S->ncell, 128, 0, s>>>(S->d_cell_start, S->ncell, S->d_cell_tmp,
                                                   S->d_cell_beads);
    count_launches(4);
}

// ---------------------------------------------------------------------------
// mesh reciprocal sum

__global__ void k_absmax_all(const double *__restrict__ X, long len, unsigned long long *out)
{
    double v = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (long)gridDim.x * blockDim.x)
        v = fmax(v, fabs(X[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// fixed-point scale 2^E / max|x| with E such that n terms of magnitude
// <= 2^E cannot overflow a signed 64-bit word; xmax[1], xmax[2] receive the
// scale and its inverse (as double bits)
__global__ void k_fix_scale(unsigned long long *xmax, int n)
{
    const double mx = __longlong_as_double((long long)xmax[0]);
    int lg = 0;
    while ((1L << lg) <= (long)n) lg++;
    const double sc = mx > 0.0 ? ldexp(1.0, 61 - lg) / mx : 1.0;
    xmax[1] = (unsigned long long)__double_as_longlong(sc);
    xmax[2] = (unsigned long long)__double_as_longlong(1.0 / sc);
}

__device__ __forceinline__ double fix_scale(const unsigned long long *xmax, int)
{
    return __longlong_as_double((long long)xmax[1]);
}

template <typename T>
__global__ void k_pme_spread(const double *__restrict__ pw, int n, double L, int K, int p,
                             const double *__restrict__ X, int m,
                             const unsigned long long *__restrict__ xmax,
                             unsigned long long *__restrict__ qfix)
{
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long)n * m) return;
    const int nu = (int)(tid % n), col = (int)(tid / n);
    const long n3 = 3L * n, K3 = (long)K * K * K;
    const double scale = fix_scale(xmax, n);
    T w[3][kMaxOrder];
    int g0[3];
    for (int d = 0; d < 3; d++) {
        const double u = pw[3 * nu + d] * K / L;
        double fl = floor(u);
        bspline_weights<T>((T)(u - fl), p, w[d]);
        g0[d] = (int)fl;
    }
    const double x[3] = {X[(long)col * n3 + 3L * nu] * scale, X[(long)col * n3 + 3L * nu + 1] * scale,
                         X[(long)col * n3 + 3L * nu + 2] * scale};
    unsigned long long *q0 = qfix + (size_t)(3 * col) * K3;
    for (int j1 = 0; j1 < p; j1++) {
        const int a1 = ((g0[0] - j1) % K + K) % K;
        for (int j2 = 0; j2 < p; j2++) {
            const int a2 = ((g0[1] - j2) % K + K) % K;
            const double w12 = (double)w[0][j1] * (double)w[1][j2];
            for (int j3 = 0; j3 < p; j3++) {
                const int a3 = ((g0[2] - j3) % K + K) % K;
                const long g = ((long)a1 * K + a2) * K + a3;
                const double ww = w12 * (double)w[2][j3];
                for (int b = 0; b < 3; b++)
                    atomicAdd(q0 + (size_t)b * K3 + g, (unsigned long long)llrint(ww * x[b]));
            }
        }
    }
}

template <typename T>
__global__ void k_pme_unfix(const unsigned long long *__restrict__ qfix, long len,
                            const unsigned long long *__restrict__ xmax, int n, T *__restrict__ q)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    (void)n;
    const double inv = __longlong_as_double((long long)xmax[2]);
    q[i] = (T)((double)(long long)qfix[i] * inv);
}

// Yhat(m) = G(m) |b(m)|^2 Qhat(m) for every column (3 x 3 real symmetric
// tensor on the three component meshes)
template <typename T, typename C>
__global__ void k_pme_influence_apply(const T *__restrict__ infl, long Kh, int m, C *__restrict__ qh)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kh * m) return;
    const long pt = i % Kh;
    const int col = (int)(i / Kh);
    const T *g = infl + 6 * pt;
    C *q = qh + (size_t)(3 * col) * Kh + pt;
    const C a = q[0], b = q[Kh], c = q[2 * Kh];
    C r0, r1, r2;
    r0.x = g[0] * a.x + g[1] * b.x + g[2] * c.x;
    r0.y = g[0] * a.y + g[1] * b.y + g[2] * c.y;
    r1.x = g[1] * a.x + g[3] * b.x + g[4] * c.x;
    r1.y = g[1] * a.y + g[3] * b.y + g[4] * c.y;
    r2.x = g[2] * a.x + g[4] * b.x + g[5] * c.x;
    r2.y = g[2] * a.y + g[4] * b.y + g[5] * c.y;
    q[0] = r0;
    q[Kh] = r1;
    q[2 * Kh] = r2;
}

// Y[col][3 nu + b] += sum_g W(u_nu - g) Ymesh[3 col + b][g]
template <typename T>
__global__ void k_pme_gather(const double *__restrict__ pw, int n, double L, int K, int p,
                             const T *__restrict__ q, int m, double *__restrict__ Y)
{
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long)n * m) return;
    const int nu = (int)(tid % n), col = (int)(tid / n);
    const long n3 = 3L * n, K3 = (long)K * K * K;
    T w[3][kMaxOrder];
    int g0[3];
    for (int d = 0; d < 3; d++) {
        const double u = pw[3 * nu + d] * K / L;
        double fl = floor(u);
        bspline_weights<T>((T)(u - fl), p, w[d]);
        g0[d] = (int)fl;
    }
    const T *q0 = q + (size_t)(3 * col) * K3;
    T y[3] = {0, 0, 0};
    for (int j1 = 0; j1 < p; j1++) {
        const int a1 = ((g0[0] - j1) % K + K) % K;
        for (int j2 = 0; j2 < p; j2++) {
            const int a2 = ((g0[1] - j2) % K + K) % K;
            const T w12 = w[0][j1] * w[1][j2];
            for (int j3 = 0; j3 < p; j3++) {
                const int a3 = ((g0[2] - j3) % K + K) % K;
                const long g = ((long)a1 * K + a2) * K + a3;
                const T ww = w12 * w[2][j3];
                for (int b = 0; b < 3; b++) y[b] += ww * q0[(size_t)b * K3 + g];
            }
        }
    }
    double *out = Y + (long)col * n3 + 3L * nu;
    for (int b = 0; b < 3; b++) out[b] += (double)y[b];
}

static bd_status cufft_plans(Plan &P, int m)
{
    PmeState *S = P.pme;
    if (S->plan_m == m) return BD_OK;
    if (S->plan_m) {
        cufftDestroy(S->fwd);
        cufftDestroy(S->inv);
        S->plan_m = 0;
    }
    int dims[3] = {S->K, S->K, S->K};
    const bool dbl = !is_mixed(P);
    cufftResult r1 = cufftPlanMany(&S->fwd, 3, dims, nullptr, 1, (int)S->K3, nullptr, 1, (int)S->Kh,
                                   dbl ? CUFFT_D2Z : CUFFT_R2C, 3 * m);
    cufftResult r2 = cufftPlanMany(&S->inv, 3, dims, nullptr, 1, (int)S->Kh, nullptr, 1, (int)S->K3,
                                   dbl ? CUFFT_Z2D : CUFFT_C2R, 3 * m);
    if (r1 != CUFFT_SUCCESS || r2 != CUFFT_SUCCESS) {
        if (r1 == CUFFT_SUCCESS) cufftDestroy(S->fwd);
        if (r2 == CUFFT_SUCCESS) cufftDestroy(S->inv);
        return set_error(BD_ERR_CUDA, "cuFFT plan for a %d^3 mesh x %d failed (%d, %d)", S->K, 3 * m,
                         (int)r1, (int)r2);
    }
    S->plan_m = m;
    return BD_OK;
}

bd_status launch_apply_spectral(Plan &P, const double *X, int m, double *Y, cudaStream_t s)
{
    PmeState *S = P.pme;
    if (!S) return set_error(BD_ERR_INVALID, "plan has no mesh (pme_grid = 0)");
    if (m > S->mcap) return set_error(BD_ERR_INVALID, "m = %d exceeds the mesh capacity %d", m, S->mcap);
    bd_status st = launch_real_cells(P, X, m, Y, s);
    if (st != BD_OK) return st;
    if (P.p.n2max <= 0) return BD_OK;
    st = cufft_plans(P, m);
    if (st != BD_OK) return st;
    const long n3 = (long)P.n3;
    const long grid_len = (long)3 * m * S->K3;
    cudaMemsetAsync(S->d_xmax, 0, sizeof(unsigned long long), s);
    k_absmax_all<<<256, 256, 0, s>>>(X, n3 * m, S->d_xmax);
    k_fix_scale<<<1, 1, 0, s>>>(S->d_xmax, P.n);
    count_launches(1);
    cudaMemsetAsync(S->d_qfix, 0, sizeof(unsigned long long) * grid_len, s);
    const unsigned nbm = (unsigned)(((long)P.n * m + 127) / 128);
    const unsigned ng = (unsigned)((grid_len + 255) / 256);
    const unsigned nh = (unsigned)((S->Kh * m + 255) / 256);
    cufftSetStream(S->fwd, s);
    cufftSetStream(S->inv, s);
    cufftResult r1, r2;
    if (!is_mixed(P)) {
        k_pme_spread<double><<<nbm, 128, 0, s>>>(P.d_pw64, P.n, P.p.box_L, S->K, S->p, X, m,
                                                S->d_xmax, S->d_qfix);
        k_pme_unfix<double><<<ng, 256, 0, s>>>(S->d_qfix, grid_len, S->d_xmax, P.n,
                                              (double *)S->d_qreal);
        r1 = cufftExecD2Z(S->fwd, (cufftDoubleReal *)S->d_qreal, (cufftDoubleComplex *)S->d_qhat);
        k_pme_influence_apply<double, cufftDoubleComplex><<<nh, 256, 0, s>>>(
            (const double *)S->d_infl, S->Kh, m, (cufftDoubleComplex *)S->d_qhat);
        r2 = cufftExecZ2D(S->inv, (cufftDoubleComplex *)S->d_qhat, (cufftDoubleReal *)S->d_qreal);
        k_pme_gather<double><<<nbm, 128, 0, s>>>(P.d_pw64, P.n, P.p.box_L, S->K, S->p,
                                                (const double *)S->d_qreal, m, Y);
    } else {
        k_pme_spread<float><<<nbm, 128, 0, s>>>(P.d_pw64, P.n, P.p.box_L, S->K, S->p, X, m,
                                               S->d_xmax, S->d_qfix);
        k_pme_unfix<float><<<ng, 256, 0, s>>>(S->d_qfix, grid_len, S->d_xmax, P.n,
                                             (float *)S->d_qreal);
        r1 = cufftExecR2C(S->fwd, (cufftReal *)S->d_qreal, (cufftComplex *)S->d_qhat);
        k_pme_influence_apply<float, cufftComplex><<<nh, 256, 0, s>>>(
            (const float *)S->d_infl, S->Kh, m, (cufftComplex *)S->d_qhat);
        r2 = cufftExecC2R(S->inv, (cufftComplex *)S->d_qhat, (cufftReal *)S->d_qreal);
        k_pme_gather<float><<<nbm, 128, 0, s>>>(P.d_pw64, P.n, P.p.box_L, S->K, S->p,
                                               (const float *)S->d_qreal, m, Y);
    }
    count_launches(6);
    if (r1 != CUFFT_SUCCESS || r2 != CUFFT_SUCCESS)
        return set_error(BD_ERR_CUDA, "cuFFT execution failed (%d, %d)", (int)r1, (int)r2);
    return check_launch("spectral product");
}

}  // namespace bd
