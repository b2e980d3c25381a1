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
//     cardinal B-splines of order p, transformed (fft.cu, real to half
//     complex), each
//     mesh wave vector m multiplied by G(m) |b(m)|^2 with G = M2(2 pi m / L)
//     of Eq. (M2) for |m|^2 <= n2max (zero otherwise and at m = 0) and b the
//     Euler exponential-spline factors, transformed back and interpolated
//     with the same splines.
// The mesh sum approximates the k-sum by spline interpolation; its error
// falls as (k_max L / (2 pi K))^p.  Spreading is mesh-centric: each mesh
// point sums its beads in a fixed order (no atomics), and the cell lists are
// ordered by bead index inside each cell, so every product is the same on
// every run.
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
    S->tpd = S->K / kMeshTile;
    S->ntile = (long)S->tpd * S->tpd * S->tpd;
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
    ALLOC(S->d_row_start, sizeof(int) * (P.n + 1));
    ALLOC(S->d_rowpos, (size_t)32 * P.n);
    S->xrows_len = real_pairs_rows_len(P.n, S->mcap, dbl);
    ALLOC(S->d_xrows, ts * S->xrows_len);
    ALLOC(S->d_infl, ts * 6 * S->Kh);
    ALLOC(S->d_tile_of, sizeof(int) * P.n);
    ALLOC(S->d_tile_count, sizeof(int) * S->ntile);
    ALLOC(S->d_tile_start, sizeof(int) * (S->ntile + 1));
    ALLOC(S->d_tile_beads, sizeof(int) * P.n);
    ALLOC(S->d_bfl, sizeof(int) * 3 * P.n);
    ALLOC(S->d_bw, ts * 3 * S->p * P.n);
    ALLOC(S->d_qreal, ts * grids * S->K3);
    ALLOC(S->d_qhat, 2 * ts * grids * S->Kh);
#undef ALLOC
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->h_npair, sizeof(long long));
    if (e != cudaSuccess) return oom("mesh", e);
    P.scratch_bytes += (int64_t)bytes;
    bd_status fst = fft_plan_init(S->fft, S->K);
    if (fst != BD_OK) return fst;
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
                    S->d_row_start, S->d_rowpos, S->d_nbr, S->d_prow, S->d_tens, S->d_xrows, S->d_infl, S->d_tile_of, S->d_tile_count, S->d_tile_start,
                    S->d_tile_beads, S->d_bfl, S->d_bw, S->d_qreal, S->d_qhat};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (S->h_npair) cudaFreeHost(S->h_npair);
    fft_free(S->fft);
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
        const double v = pw[3 * nu + s] * nc / L;
        const int c = (v >= 0.0 && v < (double)nc) ? (int)v : 0;     // non-finite: cell 0
        ci[s] = c >= nc ? nc - 1 : c;
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

// spline base index floor(u_d) mod K and weights of every bead (u_d = K x_d / L
// of the wrapped position), and the mesh tile holding the base index
template <typename T>
__global__ void k_tile_assign(const double *__restrict__ pw, int n, double L, int K, int p, int tpd,
                              int *__restrict__ bfl, T *__restrict__ bw, int *__restrict__ tile_of,
                              int *__restrict__ count)
{
    const int nu = blockIdx.x * blockDim.x + threadIdx.x;
    if (nu >= n) return;
    int ti[3];
    for (int d = 0; d < 3; d++) {
        double u = pw[3 * nu + d] * K / L;
        if (!(u >= 0.0 && u < (double)K)) u = 0.0;        // non-finite position: a valid mesh cell
        const double fl = floor(u);
        T w[kMaxOrder];
        bspline_weights<T>((T)(u - fl), p, w);
        for (int j = 0; j < p; j++) bw[((size_t)nu * 3 + d) * p + j] = w[j];
        int g = (int)fl;
        g = g < 0 ? g + K : (g >= K ? g - K : g);
        bfl[3 * nu + d] = g;
        ti[d] = g / kMeshTile;
    }
    const int t = (ti[0] * tpd + ti[1]) * tpd + ti[2];
    tile_of[nu] = t;
    atomicAdd(&count[t], 1);
}

// beads grouped by bin, ascending inside a bin: count, scan, scatter, sort
static void bin_sort(const int *bin_of, int n, int *count, long nbin, int *start, int *tmp,
                     int *out, cudaStream_t s)
{
    k_cell_scan<<<1, 1024, 0, s>>>(count, nbin, start);
    k_cell_scatter<<<(n + 255) / 256, 256, 0, s>>>(bin_of, n, count, tmp);
    k_cell_sort<<<(unsigned)nbin, 128, 0, s>>>(start, nbin, tmp, out);
    count_launches(3);
}

void launch_scan_counts(int *count, long len, int *start, cudaStream_t s)
{
    k_cell_scan<<<1, 1024, 0, s>>>(count, len, start);
}

bd_status spectral_tables(Plan &P, cudaStream_t s)
{
    PmeState *S = P.pme;
    const unsigned nb = (unsigned)((P.n + 255) / 256);
    cudaMemsetAsync(S->d_cell_count, 0, sizeof(int) * S->ncell, s);
    k_cell_assign<<<nb, 256, 0, s>>>(P.d_pw64, P.n, S->nc, P.p.box_L, S->d_cell_of,
                                     S->d_cell_count);
    count_launches(1);
    bin_sort(S->d_cell_of, P.n, S->d_cell_count, S->ncell, S->d_cell_start, S->d_cell_tmp,
             S->d_cell_beads, s);
    bd_status st = build_real_pairs(P, s);
    if (st != BD_OK || P.p.n2max <= 0) return st;
    cudaMemsetAsync(S->d_tile_count, 0, sizeof(int) * S->ntile, s);
    if (is_mixed(P))
        k_tile_assign<float><<<nb, 256, 0, s>>>(P.d_pw64, P.n, P.p.box_L, S->K, S->p, S->tpd,
                                                S->d_bfl, (float *)S->d_bw, S->d_tile_of,
                                                S->d_tile_count);
    else
        k_tile_assign<double><<<nb, 256, 0, s>>>(P.d_pw64, P.n, P.p.box_L, S->K, S->p, S->tpd,
                                                 S->d_bfl, (double *)S->d_bw, S->d_tile_of,
                                                 S->d_tile_count);
    count_launches(1);
    bin_sort(S->d_tile_of, P.n, S->d_tile_count, S->ntile, S->d_tile_start, S->d_cell_tmp,
             S->d_tile_beads, s);
    return check_launch("spectral tables");
}

// ---------------------------------------------------------------------------
// mesh reciprocal sum

// Mesh-centric spreading, Q[3 col + b][g] = sum_nu W(u_nu - g) X[col][3 nu + b]:
// one block per tile of kMeshTile^3 mesh points, one thread per point.  A
// bead with base index f_d = floor(u_d) reaches the points f_d - j, j < p,
// so the tile's beads are those binned in tiles t_d .. t_d + 1 + (p-2)/E per
// dimension (mod tpd).  The block stages them (bins in a fixed order, beads
// ascending inside a bin) with their base indices, weights and operand rows.
// Each warp covers a 2 x 4 x 4 brick of points and first compacts (ballot)
// the staged beads that reach its brick, keeping their order; each thread
// then adds w1[j1] w2[j2] w3[j3] x over those beads with
// j_d = (f_d - g_d) mod K < p.  Every mesh point is written once and summed in
// a fixed order: no atomics.  The columns go in balanced chunks of <= CC.
template <typename T> struct SpreadStage { static constexpr int value = 128; };
template <> struct SpreadStage<double> { static constexpr int value = 64; };

template <typename T, int CC>
__global__ void __launch_bounds__(kMeshTile *kMeshTile *kMeshTile)
k_pme_spread(int n, int K, int p, int tpd, const int *__restrict__ tile_start,
             const int *__restrict__ tile_beads, const int *__restrict__ bfl,
             const T *__restrict__ bw, const double *__restrict__ X, int m, T *__restrict__ q)
{
    constexpr int E = kMeshTile;
    constexpr int NW = E * E * E / 32;                     // warps: 4 x 2 x 2 bricks
    constexpr int ST = SpreadStage<T>::value;
    constexpr int VW = 16 / sizeof(T);                     // T per 16-byte shared load
    constexpr int XW = (3 * CC + VW - 1) / VW * VW;        // staged operand row
    __shared__ int s_bin0[27], s_off[28];
    __shared__ int s_mu[ST];
    __shared__ int4 s_fl[ST];
    __shared__ T s_w[ST][3 * kMaxOrder];
    __shared__ __align__(16) T s_x[ST][XW];
    __shared__ unsigned char s_list[NW][ST];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int t[3] = {b / (tpd * tpd), (b / tpd) % tpd, b % tpd};
    // brick origin of this warp and the thread's point inside it
    const int w0[3] = {t[0] * E + 2 * (wid >> 2), t[1] * E + 4 * ((wid >> 1) & 1), t[2] * E + 4 * (wid & 1)};
    const int g[3] = {w0[0] + (lane >> 4), w0[1] + ((lane >> 2) & 3), w0[2] + (lane & 3)};
    const int reach[3] = {p, p + 2, p + 2};                // (f - w0) mod K <= p + extent - 2
    const int nbd = min(2 + (p - 2) / E, tpd);
    const int nbins = nbd * nbd * nbd;
    if (tid < nbins) {
        const int i0 = tid / (nbd * nbd), i1 = (tid / nbd) % nbd, i2 = tid % nbd;
        const int bin = (((t[0] + i0) % tpd) * tpd + (t[1] + i1) % tpd) * tpd + (t[2] + i2) % tpd;
        s_bin0[tid] = tile_start[bin];
        s_off[tid + 1] = tile_start[bin + 1] - tile_start[bin];
    }
    __syncthreads();
    if (tid == 0) {
        s_off[0] = 0;
        for (int i = 1; i <= nbins; i++) s_off[i] += s_off[i - 1];
    }
    __syncthreads();
    const int total = s_off[nbins];
    const int w3 = 3 * p;
    const long n3 = 3L * n, K3 = (long)K * K * K;
    const long gi = ((long)g[0] * K + g[1]) * K + g[2];
    const int nchunk = (m + CC - 1) / CC, cw = (m + nchunk - 1) / nchunk;
    for (int c0 = 0; c0 < m; c0 += cw) {
        const int ncol = min(cw, m - c0), nx = 3 * ncol;
        T acc[3 * CC];
#pragma unroll
        for (int i = 0; i < 3 * CC; i++) acc[i] = (T)0;
        for (int j0 = 0; j0 < total; j0 += ST) {
            const int jn = min(ST, total - j0);
            __syncthreads();
            if (tid < jn) {
                const int e = j0 + tid;
                int k = 0;
                while (s_off[k + 1] <= e) k++;
                const int mu = tile_beads[s_bin0[k] + (e - s_off[k])];
                s_mu[tid] = mu;
                s_fl[tid] = make_int4(bfl[3 * mu], bfl[3 * mu + 1], bfl[3 * mu + 2], 0);
            }
            __syncthreads();
            for (int e = tid; e < jn * w3; e += blockDim.x) {
                const int i = e / w3, r = e - i * w3;
                s_w[i][r] = bw[(size_t)s_mu[i] * w3 + r];
            }
            for (int e = tid; e < jn * nx; e += blockDim.x) {
                const int i = e / nx, r = e - i * nx;
                const int c = r / 3, bb = r - 3 * c;
                s_x[i][r] = (T)X[(long)(c0 + c) * n3 + 3L * s_mu[i] + bb];
            }
            // this warp's beads, in staging order
            int cnt = 0;
            for (int jj = 0; jj < jn; jj += 32) {
                const int j = jj + lane;
                bool in = false;
                if (j < jn) {
                    const int4 f = s_fl[j];
                    int d0 = f.x - w0[0], d1 = f.y - w0[1], d2 = f.z - w0[2];
                    d0 += d0 < 0 ? K : 0;
                    d1 += d1 < 0 ? K : 0;
                    d2 += d2 < 0 ? K : 0;
                    in = d0 <= reach[0] && d1 <= reach[1] && d2 <= reach[2];
                }
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (in) s_list[wid][cnt + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)j;
                cnt += __popc(bal);
            }
            __syncthreads();
            for (int l = 0; l < cnt; l++) {
                const int j = s_list[wid][l];
                const int4 f = s_fl[j];
                int v0 = f.x - g[0], v1 = f.y - g[1], v2 = f.z - g[2];
                v0 += v0 < 0 ? K : 0;
                v1 += v1 < 0 ? K : 0;
                v2 += v2 < 0 ? K : 0;
                if (v0 < p && v1 < p && v2 < p) {
                    const T ww = s_w[j][v0] * s_w[j][p + v1] * s_w[j][2 * p + v2];
#pragma unroll
                    for (int v = 0; v < XW / VW; v++) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(&s_x[j][v * VW]);
                        T xv[VW];
                        memcpy(xv, &u, 16);
#pragma unroll
                        for (int e = 0; e < VW; e++) {
                            const int i = v * VW + e;
                            if (i < 3 * CC && i < nx) acc[i] += ww * xv[e];
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 3 * CC; i++)
            if (i < nx) q[(size_t)(3 * c0 + i) * K3 + gi] = acc[i];
    }
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

// Y[col][3 nu + b] += sum_g W(u_nu - g) Ymesh[3 col + b][g]: one warp per
// bead (beads in mesh-tile order, so a block's warps read the same
// neighbourhood of the mesh), the lanes over the P^2 (j2, j3) spline points
// of a plane -- one load instruction reads a few contiguous mesh rows -- the
// planes j1 in order, one column at a time (the block's working set is one
// column's neighbourhood), then a butterfly sum over the lanes (every lane
// ends with the same, order-fixed sum)
template <typename T, int P>
__global__ void __launch_bounds__(256)
k_pme_gather(int n, int K, const int *__restrict__ tile_beads, const int *__restrict__ bfl,
             const T *__restrict__ bw, const T *__restrict__ q, int m, double *__restrict__ Y)
{
    constexpr int NP = P * P, PER = (NP + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int nu = tile_beads[i];
    const T *wb = bw + (size_t)nu * 3 * P;
    const int g0 = bfl[3 * nu], g1 = bfl[3 * nu + 1], g2 = bfl[3 * nu + 2];
    const long K3 = (long)K * K * K, n3 = 3L * n;
    int off[PER];
    T w23[PER];
#pragma unroll
    for (int h = 0; h < PER; h++) {
        const int c = lane + 32 * h;
        const int j2 = c / P, j3 = c - (c / P) * P;
        const bool ok = c < NP;
        const int a2 = g1 - j2 < 0 ? g1 - j2 + K : g1 - j2;
        const int a3 = g2 - j3 < 0 ? g2 - j3 + K : g2 - j3;
        off[h] = ok ? a2 * K + a3 : 0;
        w23[h] = ok ? wb[P + j2] * wb[2 * P + j3] : (T)0;
    }
    for (int col = 0; col < m; col++) {
        const T *qc = q + (size_t)(3 * col) * K3;
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 2
        for (int j1 = 0; j1 < P; j1++) {
            const int r1 = g0 - j1 < 0 ? g0 - j1 + K : g0 - j1;
            const T *pl = qc + (long)r1 * K * K;
            const T w1 = wb[j1];
#pragma unroll
            for (int h = 0; h < PER; h++) {
                if (lane + 32 * h < NP) {
                    const T ww = w1 * w23[h];
                    const T *pt = pl + off[h];
                    a0 += ww * pt[0];
                    a1 += ww * pt[K3];
                    a2 += ww * pt[2 * K3];
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane < 3) Y[(long)col * n3 + 3L * nu + lane] += (double)(lane == 0 ? a0 : (lane == 1 ? a1 : a2));
    }
}

template <typename T>
static void launch_gather(const PmeState *S, int n, int m, double *Y, cudaStream_t s)
{
    const unsigned nb = (unsigned)((n + 7) / 8);
    const T *bw = (const T *)S->d_bw, *q = (const T *)S->d_qreal;
#define GATHER(PP)                                                                      \
    case PP:                                                                            \
        k_pme_gather<T, PP><<<nb, 256, 0, s>>>(n, S->K, S->d_tile_beads, S->d_bfl, bw, q, m, Y); \
        break;
    switch (S->p) {
        GATHER(4) GATHER(5) GATHER(6) GATHER(7) GATHER(8) GATHER(9) GATHER(10)
    }
#undef GATHER
}

bd_status launch_apply_spectral(Plan &P, const double *X, int m, double *Y, cudaStream_t s)
{
    PmeState *S = P.pme;
    if (!S) return set_error(BD_ERR_INVALID, "plan has no mesh (pme_grid = 0)");
    if (m > S->mcap) return set_error(BD_ERR_INVALID, "m = %d exceeds the mesh capacity %d", m, S->mcap);
    bd_status st = launch_real_pairs(P, X, m, Y, s);
    if (st != BD_OK) return st;
    if (P.p.n2max <= 0) return BD_OK;
    const unsigned ntiles = (unsigned)S->ntile;
    const unsigned nh = (unsigned)((S->Kh * m + 255) / 256);
    constexpr int kTileThreads = kMeshTile * kMeshTile * kMeshTile;
    const int B = 3 * m;                 // three component meshes per column
    if (!is_mixed(P)) {
        k_pme_spread<double, 6><<<ntiles, kTileThreads, 0, s>>>(
            P.n, S->K, S->p, S->tpd, S->d_tile_start, S->d_tile_beads, S->d_bfl,
            (const double *)S->d_bw, X, m, (double *)S->d_qreal);
        st = fft3_r2c<double>(S->fft, (const double *)S->d_qreal, S->d_qhat, B, s);
        if (st != BD_OK) return st;
        k_pme_influence_apply<double, double2><<<nh, 256, 0, s>>>(
            (const double *)S->d_infl, S->Kh, m, (double2 *)S->d_qhat);
        st = fft3_c2r<double>(S->fft, S->d_qhat, (double *)S->d_qreal, B, s);
        if (st != BD_OK) return st;
        launch_gather<double>(S, P.n, m, Y, s);
    } else {
        k_pme_spread<float, 9><<<ntiles, kTileThreads, 0, s>>>(
            P.n, S->K, S->p, S->tpd, S->d_tile_start, S->d_tile_beads, S->d_bfl,
            (const float *)S->d_bw, X, m, (float *)S->d_qreal);
        st = fft3_r2c<float>(S->fft, (const float *)S->d_qreal, S->d_qhat, B, s);
        if (st != BD_OK) return st;
        k_pme_influence_apply<float, float2><<<nh, 256, 0, s>>>(
            (const float *)S->d_infl, S->Kh, m, (float2 *)S->d_qhat);
        st = fft3_c2r<float>(S->fft, S->d_qhat, (float *)S->d_qreal, B, s);
        if (st != BD_OK) return st;
        launch_gather<float>(S, P.n, m, Y, s);
    }
    count_launches(3);
    return check_launch("spectral product");
}

}  // namespace bd
