// rows_gemm.cu -- launch shape 5 of the mixed products (few columns): the
// 16-bit D streamed row by row on the CUDA cores, and the Chebyshev loop of
// any number of replicas in one persistent launch.
//
// With m + 1 <= 8 columns (one or a few Wiener vectors and the Lanczos
// vector) a product Y = D16 X does at most 16 flops per 2-byte entry of D, so
// it is bound by the stream of D from HBM, not by arithmetic, and the FP32
// pipe keeps up; X then needs no 16-bit quantisation (it is used in FP32).
// Work item: 64 consecutive rows of one replica in the Chebyshev loop (8 per
// warp, up to 5 columns), 32 rows (4 per warp, up to 8 columns) in a plain
// product; the lanes of a warp walk the rows in chunks of 8 entries (16-byte
// loads, two chunks in flight) and each lane keeps one FP32 sum per (row,
// column); the 32 lane sums are combined by a butterfly of shuffles.  The order of every sum depends only on the row, so
// a replica gives the same bits alone or in a batch, whichever CTA takes it.
//
// Batched Chebyshev loop (Eqs. cheb2, cheb3 with the lagged Lanczos column):
// one cooperative launch runs terms p = 2 .. N_Ch - 1 of every replica.  Per
// term: phase A, every item's product and its epilogue (V_p, dS, the next
// FP32 operand, the Lanczos product w and its per-item dot partials); a
// grid barrier; phase B (with the Lanczos column), every item's rows of
// q_{j+1}, with alpha_j, beta_j reduced from the replica's partials in a
// fixed order; a grid barrier.  In phase A the CTAs claim items from a
// per-term counter (an item's rows cost as much as its replica's row length,
// 600 to 6000 entries in a batch; the item table lists the largest replicas
// first); which CTA takes an item does not change its result.  The barriers spin with a bound: a CTA that
// gives up records BD_ERR_TIMEOUT and goes on (the results are then invalid,
// nothing hangs).
#include <math.h>

#include "rows_gemm.cuh"

namespace bd {

namespace rw {

constexpr int THREADS = 256;       // 8 warps
constexpr int WR = 4;              // rows per warp, plain products (up to 8 columns)
constexpr int RB = 8 * WR;         // rows per CTA, plain products
constexpr int WRC = 8;             // rows per warp, Chebyshev loop (up to 5 columns)
constexpr int RBC = 8 * WRC;       // rows per work item of the Chebyshev loop
constexpr uint32_t kBarrierLimit = 1u << 21;

__device__ __forceinline__ void cvt8(uint4 d, int is_bf16, float f[8])
{
    const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 v;
        if (is_bf16) v = __bfloat1622float2(*(const __nv_bfloat162 *)&w[i]);
        else v = __half22float2(*(const __half2 *)&w[i]);
        f[2 * i] = v.x;
        f[2 * i + 1] = v.y;
    }
}

__device__ __forceinline__ float cvt1(uint16_t h, int is_bf16)
{
    return is_bf16 ? __bfloat162float(*(const __nv_bfloat16 *)&h) : __half2float(*(const __half *)&h);
}

// sums[r][c] = sum_k D16[row0 + r][k] X[c][k] for the W rows of each warp of
// the CTA (row0 = the warp's first row; rows at or beyond n3 give 0); every
// lane ends with every sum.  X: FP32 columns of stride xs (>= n3, a multiple
// of 8, zero-padded), staged in shared memory KC entries at a time (sx holds
// C x KC floats), so the CTA reads each operand entry from L2 once and its
// warps share it (the operand may have been written by other CTAs of the
// same launch: L2 loads, never L1).  Every thread of the CTA must call it.
constexpr int KC = 1024;

template <int C, int W>
__device__ __forceinline__ void rows_dot(const uint16_t *__restrict__ D, long ld, int n3,
                                         const float *__restrict__ X, int xs, int row0,
                                         int is_bf16, float sums[W][C], float *sx)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < W; r++)
#pragma unroll
        for (int c = 0; c < C; c++) sums[r][c] = 0.f;
    for (int kb = 0; kb < n3; kb += KC) {
        __syncthreads();                         // the previous chunk is consumed
        for (int i = threadIdx.x; i < C * (KC / 4); i += blockDim.x) {
            const int c = i / (KC / 4), k4 = 4 * (i - c * (KC / 4));
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kb + k4 < xs) v = __ldcg((const float4 *)(X + (size_t)c * xs + kb + k4));
            *(float4 *)(sx + c * KC + k4) = v;
        }
        __syncthreads();
        const int kend = min(KC, n3 - kb), kfull = kend & ~7;
        for (int k = 8 * lane; k < kfull; k += 256) {
            uint4 d[W];
#pragma unroll
            for (int r = 0; r < W; r++)
                d[r] = row0 + r < n3 ? __ldcs((const uint4 *)(D + (size_t)(row0 + r) * ld + kb + k))
                                     : make_uint4(0u, 0u, 0u, 0u);
            float x[C][8];
#pragma unroll
            for (int c = 0; c < C; c++) {
                const float4 a = *(const float4 *)(sx + c * KC + k);
                const float4 b = *(const float4 *)(sx + c * KC + k + 4);
                x[c][0] = a.x; x[c][1] = a.y; x[c][2] = a.z; x[c][3] = a.w;
                x[c][4] = b.x; x[c][5] = b.y; x[c][6] = b.z; x[c][7] = b.w;
            }
#pragma unroll
            for (int r = 0; r < W; r++) {
                float f[8];
                cvt8(d[r], is_bf16, f);
#pragma unroll
                for (int c = 0; c < C; c++)
#pragma unroll
                    for (int j = 0; j < 8; j++) sums[r][c] = fmaf(f[j], x[c][j], sums[r][c]);
            }
        }
        // ragged end of the rows (the padding columns of D are never read)
        const int k = kfull + lane;
        if (k < kend) {
#pragma unroll
            for (int r = 0; r < W; r++) {
                if (row0 + r >= n3) continue;
                const float f = cvt1(D[(size_t)(row0 + r) * ld + kb + k], is_bf16);
#pragma unroll
                for (int c = 0; c < C; c++) sums[r][c] = fmaf(f, sx[c * KC + k], sums[r][c]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < W; r++)
#pragma unroll
        for (int c = 0; c < C; c++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                sums[r][c] += __shfl_xor_sync(0xffffffffu, sums[r][c], o);
}

template <int C, int W>
__device__ __forceinline__ float pick(const float sums[W][C], int r, int c)
{
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < W; i++)
#pragma unroll
        for (int j = 0; j < C; j++)
            if (i == r && j == c) v = sums[i][j];
    return v;
}

// plain product Y = D16 X (C columns), one item per CTA
template <int C>
__global__ void __launch_bounds__(THREADS)
k_rows_plain(const uint16_t *__restrict__ D, long ld, int n3, const float *__restrict__ X, int xs,
             int is_bf16, double *__restrict__ Y)
{
    __shared__ __align__(16) float sx[C * KC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * RB + warp * WR;
    float sums[WR][C];
    rows_dot<C, WR>(D, ld, n3, X, xs, row0, is_bf16, sums, sx);
    if (lane < WR * C) {
        const int r = lane / C, c = lane % C;
        const int row = row0 + r;
        if (row < n3) Y[(size_t)c * n3 + row] = (double)pick<C, WR>(sums, r, c);
    }
}

// FP64 columns to the FP32 operand [c][xs] (padding stays zero)
__global__ void k_to32(const double *__restrict__ X, int n3, int m, float *__restrict__ X32, int xs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (i < n3 && c < m) X32[(size_t)c * xs + i] = (float)X[(size_t)c * n3 + i];
}

// ---------------------------------------------------------------------------
// the batched Chebyshev loop

// a CTA that gives up waiting marks every replica's step as timed out
__device__ void grid_barrier(unsigned *bar, unsigned nblocks, const RowsRep *reps, int nreps)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = atomicAdd(&bar[1], 0u);
        __threadfence();
        if (atomicAdd(&bar[0], 1u) == nblocks - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            uint32_t it = 0;
            while (atomicAdd(&bar[1], 0u) == g) {
                if (++it > kBarrierLimit) {
                    for (int i = 0; i < nreps; i++) atomicExch(reps[i].err, (int32_t)BD_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// the replica's Lanczos step j from its per-item partials (q_j.w, q_{j-1}.w,
// w.w), summed in a fixed order whichever CTA runs it (block-wide):
//   alpha_j = q_j.w,  |w'|^2 = w.w - alpha_j^2 - 2 beta_{j-1} q_{j-1}.w + beta_{j-1}^2
// (q_j, q_{j-1} orthonormal), beta_j = |w'|; written to lab
__device__ void lanczos_scalars(const RowsRep &R, int j)
{
    __shared__ double red[THREADS][3];
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < R.nitems; b += THREADS)
#pragma unroll
        for (int k = 0; k < 3; k++) t[k] += __ldcg(R.lan_part + 3 * b + k);
#pragma unroll
    for (int k = 0; k < 3; k++) red[threadIdx.x][k] = t[k];
    __syncthreads();
    for (int w = THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 3; k++) red[threadIdx.x][k] += red[threadIdx.x + w][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double alpha = red[0][0];
        const double bprev = j > 0 ? R.lab[kMaxLanczos + j - 1] : 0.0;
        const double n2 = red[0][2] - alpha * alpha - 2.0 * bprev * red[0][1] + bprev * bprev;
        R.lab[j] = alpha;
        R.lab[kMaxLanczos + j] = n2 > 0.0 ? sqrt(n2) : 0.0;
    }
    __syncthreads();
}

// terms p_first .. p_end - 1 of every replica; lan_from >= 0: the Lanczos
// vector rides as column m and term p takes Lanczos step j = lan_from + p - 1
template <int C>
__global__ void __launch_bounds__(THREADS)
k_rows_cheb(const RowsRep *__restrict__ reps, int nreps, const int *__restrict__ item_rep,
            int nitems, int p_first, int p_end, int lan_from, unsigned *bar)
{
    __shared__ double s_lan[RBC][3];
    __shared__ int s_last, s_item;
    __shared__ __align__(16) float sx[C * KC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned *work = bar + kRowsBarWords;          // one item counter per term, zeroed per launch
    for (int p = p_first; p < p_end; p++) {
        const int j = lan_from + p - 1;
        // ---- phase A: products and their epilogues, items claimed in turn
        for (;;) {
            if (threadIdx.x == 0) s_item = (int)atomicAdd(&work[p], 1u);
            __syncthreads();
            const int it = s_item;
            __syncthreads();
            if (it >= nitems) break;
            const RowsRep &R = reps[item_rep[it]];
            const int loc = it - R.item0;
            const int row0 = loc * RBC + warp * WRC;
            const float *X = R.X32[p & 1];
            float *Xn = R.X32[(p + 1) & 1];
            double *V2 = (p & 1) ? R.VB : R.VA;          // in V_{p-2}, out V_p
            const double *V1 = (p & 1) ? R.VA : R.VB;
            float sums[WRC][C];
            rows_dot<C, WRC>(R.D16, R.ld, R.n3, X, R.xs, row0, R.is_bf16, sums, sx);
            const double ys = R.coef[kChebMapS], yt = R.coef[kChebMapT];
            const double cp = R.coef[p];
            for (int e = lane; e < WRC * C; e += 32) {
                const int r = e / C, c = e % C;
                const int row = row0 + r;
                const double w = (double)pick<C, WRC>(sums, r, c);
                double lq[3] = {0.0, 0.0, 0.0};
                if (row < R.n3) {
                    if (c < R.m) {
                        const size_t o = (size_t)c * R.n3 + row;
                        const double v = 2.0 * (ys * w - yt * V1[o]) - V2[o];
                        V2[o] = v;
                        R.dS[o] += cp * v;
                        Xn[(size_t)c * R.xs + row] = (float)v;
                    } else if (R.lan) {
                        R.lq[2][row] = w;
                        lq[0] = __ldcg(R.lq[1] + row) * w;
                        lq[1] = __ldcg(R.lq[0] + row) * w;
                        lq[2] = w * w;
                    }
                }
                if (R.lan && c == R.m)
#pragma unroll
                    for (int k = 0; k < 3; k++) s_lan[warp * WRC + r][k] = lq[k];
            }
            if (R.lan) {
                // the item's dot partials, then the last item of the replica
                // to arrive takes the Lanczos step's scalars
                __syncthreads();
                if (threadIdx.x < 3) {
                    double t = 0.0;
                    for (int i = 0; i < RBC; i++) t += s_lan[i][threadIdx.x];
                    R.lan_part[3 * loc + threadIdx.x] = t;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    const unsigned done = atomicAdd(R.lan_count, 1u) + 1u;
                    s_last = done == (unsigned)R.nitems;
                    if (s_last) {
                        atomicExch(R.lan_count, 0u);
                        __threadfence();
                    }
                }
                __syncthreads();
                if (s_last) lanczos_scalars(R, j);
            }
        }
        if (lan_from < 0 && p + 1 == p_end) break;
        grid_barrier(bar, gridDim.x, reps, nreps);
        if (lan_from < 0) continue;
        // ---- phase B: q_{j+1} = (w - alpha_j q_j - beta_{j-1} q_{j-1}) / beta_j,
        // also into the next operand's Lanczos column
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            const RowsRep &R = reps[item_rep[it]];
            const int row = (it - R.item0) * RBC + threadIdx.x;
            if (!R.lan || threadIdx.x >= RBC || row >= R.n3) continue;
            const double alpha = __ldcg(R.lab + j), beta = __ldcg(R.lab + kMaxLanczos + j);
            const double bprev = j > 0 ? __ldcg(R.lab + kMaxLanczos + j - 1) : 0.0;
            const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
            const double q1 = __ldcg(R.lq[1] + row);
            const double qn = (__ldcg(R.lq[2] + row) - alpha * q1 - bprev * __ldcg(R.lq[0] + row)) * ib;
            R.lq[0][row] = q1;
            R.lq[1][row] = qn;
            R.X32[(p + 1) & 1][(size_t)R.m * R.xs + row] = (float)qn;
        }
        if (p + 1 < p_end) grid_barrier(bar, gridDim.x, reps, nreps);
    }
}

// one replica's table entry, written on the device (the pointers a call
// passes become kernel arguments, which a captured graph keeps by value)
__global__ void k_rep_set(RowsRep *dst, RowsRep v) { *dst = v; }

}  // namespace rw

using namespace rw;

int rows_items(int n3) { return (n3 + RBC - 1) / RBC; }

bd_status rows_plan_init(Plan &P)
{
    if (P.d_x32) return BD_OK;
    P.x32_stride = (P.n3 + 7) & ~7;
    const size_t nx = (size_t)2 * kRowsMaxCols * P.x32_stride;
    const int items = rows_items(P.n3);
    cudaError_t e = cudaMalloc(&P.d_x32, nx * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_rows_part, (size_t)3 * items * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_rows_rep, sizeof(RowsRep));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_rows_items, (size_t)items * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_rows_bar, kRowsBarAlloc * sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BD_ERR_OOM, "row-streamed product scratch: %s", cudaGetErrorString(e));
    }
    P.scratch_bytes += (int64_t)(nx * sizeof(float) + 3 * items * sizeof(double) +
                                 sizeof(RowsRep) + items * sizeof(int) + kRowsBarAlloc * sizeof(unsigned));
    cudaMemset(P.d_x32, 0, nx * sizeof(float));
    cudaMemset(P.d_rows_items, 0, (size_t)items * sizeof(int));
    cudaMemset(P.d_rows_bar, 0, kRowsBarAlloc * sizeof(unsigned));
    return check_launch("row-streamed product init");
}

bd_status rows_apply(Plan &P, const void *D16, const double *X, int m, double *Y, cudaStream_t s)
{
    if (m < 1 || m > kRowsMaxCols)
        return set_error(BD_ERR_UNSUPPORTED, "launch shape 5 takes at most %d columns", kRowsMaxCols);
    bd_status st = rows_plan_init(P);
    if (st != BD_OK) return st;
    const int xs = P.x32_stride;
    k_to32<<<dim3((P.n3 + 255) / 256, m), 256, 0, s>>>(X, P.n3, m, P.d_x32, xs);
    const unsigned g = (unsigned)((P.n3 + RB - 1) / RB);
    const uint16_t *D = (const uint16_t *)D16;
    const int bf = P.p.precision == BD_MIXED_BF16;
    switch (m) {
#define RP(CC) case CC: k_rows_plain<CC><<<g, THREADS, 0, s>>>(D, P.ld, P.n3, P.d_x32, xs, bf, Y); break;
        RP(1) RP(2) RP(3) RP(4) RP(5) RP(6) RP(7) RP(8)
#undef RP
    }
    count_launches(2);
    return check_launch("row-streamed product");
}

RowsRep rows_rep(Plan &P, const void *D16, const double *coef, const double *bounds, int m,
                 int lan, double *dS)
{
    RowsRep r{};
    r.D16 = (const uint16_t *)D16;
    r.ld = P.ld;
    r.n3 = P.n3;
    r.xs = P.x32_stride;
    r.m = m;
    r.lan = lan;
    r.is_bf16 = P.p.precision == BD_MIXED_BF16;
    r.coef = coef;
    r.bounds = bounds;
    r.VA = P.d_V[0];
    r.VB = P.d_V[1];
    r.dS = dS;
    r.X32[0] = P.d_x32;
    r.X32[1] = P.d_x32 + (size_t)kRowsMaxCols * P.x32_stride;
    for (int i = 0; i < 3; i++) r.lq[i] = P.d_lq[i];
    r.lab = P.d_lab;
    r.lan_part = P.d_rows_part;
    r.lan_count = P.d_rows_bar + 2;
    r.err = P.d_status + 6;
    r.nitems = rows_items(P.n3);
    return r;
}

void rows_cheb_prepare(Plan &P, const RowsRep &rep, RowsRep *dst, const double *V1, int lan,
                       cudaStream_t s)
{
    // the operand of term 2: V_1 (and q_j) in FP32
    k_to32<<<dim3((P.n3 + 255) / 256, rep.m), 256, 0, s>>>(V1, P.n3, rep.m, P.d_x32, P.x32_stride);
    if (lan)
        k_to32<<<dim3((P.n3 + 255) / 256, 1), 256, 0, s>>>(P.d_lq[1], P.n3, 1,
                                                          P.d_x32 + (size_t)rep.m * P.x32_stride,
                                                          P.x32_stride);
    k_rep_set<<<1, 1, 0, s>>>(dst, rep);
    launch_zero_i32((int32_t *)rep.lan_count, 1, s);
    count_launches(lan ? 3 : 2);
}

bd_status rows_cheb_launch(const RowsRep *reps, int nreps, const int *item_rep, int nitems, int cols,
                           int nch, int lan_from, unsigned *bar, int device, cudaStream_t s)
{
    if (nch <= 2) return BD_OK;
    if (cols < 1 || cols > kRowsMaxLoopCols)
        return set_error(BD_ERR_UNSUPPORTED, "the row-streamed Chebyshev loop takes at most %d columns",
                         kRowsMaxLoopCols);
    const void *fn = nullptr;
    switch (cols) {
#define RF(CC) case CC: fn = (const void *)k_rows_cheb<CC>; break;
        RF(1) RF(2) RF(3) RF(4) RF(5)
#undef RF
    }
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int grid = per_sm * sms;
    if (grid > nitems) grid = nitems;
    if (grid < 1) return set_error(BD_ERR_CUDA, "no resident CTA for the batched Chebyshev loop");
    launch_zero_i32((int32_t *)bar, 1, s);      // arrival count (a timed-out launch may leave it)
    launch_zero_i32((int32_t *)(bar + kRowsBarWords), kMaxCheb, s);   // per-term item counters
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    const int p_first = 2, p_end = nch;
    switch (cols) {
#define RL(CC) case CC: e = cudaLaunchKernelEx(&cfg, k_rows_cheb<CC>, reps, nreps, item_rep, nitems, \
                                               p_first, p_end, lan_from, bar); break;
        RL(1) RL(2) RL(3) RL(4) RL(5)
#undef RL
    }
    count_launches(1);
    if (e != cudaSuccess) return set_error(BD_ERR_CUDA, "batched Chebyshev launch: %s", cudaGetErrorString(e));
    return check_launch("batched Chebyshev loop");
}

}  // namespace bd
