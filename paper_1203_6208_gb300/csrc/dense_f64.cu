// dense_f64.cu -- FP64 multi-right-hand-side product Y = D X with the dense
// diffusion matrix (the drift D.F of Eq. sde and every D.V_p of Eqs.
// cheb2/cheb3), FP64 throughout.
//
// On GB300 the FP64 pipe (about 1.2 TFLOP/s) and not HBM bounds this product
// once X has more than one column (intensity 2m/8 flop per byte of D), so the
// kernel is organised for DFMA issue: a CTA owns BM rows and all K, stages a
// BM x BK tile of D and a BK x MC tile of X in shared memory, and each thread
// keeps CPT columns of one row (and, for narrow X, a slice of K) in registers.
// Owning all of K lets the Chebyshev recurrence run in the epilogue:
//   V_p = 2 (s (D V_{p-1}) - t V_{p-1}) - V_{p-2},  dS += c_p V_p,
// with s = 2/(d_max - d_min), t = (d_max + d_min)/(d_max - d_min).
#include "bd_internal.cuh"

namespace bd {

constexpr int BM = 32;
constexpr int BK = 32;
constexpr int NT = 128;

template <int MC>
struct Shape {
    static constexpr int CG = MC >= 4 ? 4 : MC;      // column groups
    static constexpr int CPT = MC / CG;              // columns per thread
    static constexpr int KG = NT / (BM * CG);        // k groups
};

// -- kernel begin: k_gemm_f64
template <int MC, bool CHEB>
__global__ void __launch_bounds__(NT)
k_gemm_f64(const double *__restrict__ D, long ld, int n3, const double *__restrict__ X, int m,
           double *__restrict__ Y, ChebEpi e)
{
    using S = Shape<MC>;
    __shared__ double sD[BM][BK + 1];
    __shared__ double sX[MC][BK + 1];
    __shared__ double sR[S::KG > 1 ? NT * S::CPT : 1];

    const int tid = threadIdx.x;
    const int r = tid % BM;
    const int cg = (tid / BM) % S::CG;
    const int kg = tid / (BM * S::CG);
    const long row0 = (long)blockIdx.x * BM;

    double acc[S::CPT];
#pragma unroll
    for (int c = 0; c < S::CPT; c++) acc[c] = 0.0;

    for (int k0 = 0; k0 < n3; k0 += BK) {
        // D tile: BM rows x BK cols, coalesced along the row
        for (int i = tid; i < BM * BK; i += NT) {
            int rr = i / BK, kk = i % BK;
            long gr = row0 + rr;
            int gk = k0 + kk;
            sD[rr][kk] = (gr < n3 && gk < n3) ? __ldg(&D[gr * ld + gk]) : 0.0;
        }
        // X tile: column-major X, BK consecutive entries per column
        for (int i = tid; i < MC * BK; i += NT) {
            int j = i / BK, kk = i % BK;
            int gk = k0 + kk;
            sX[j][kk] = (j < m && gk < n3) ? __ldg(&X[(long)j * n3 + gk]) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = kg; kk < BK; kk += S::KG) {
            double dv = sD[r][kk];
#pragma unroll
            for (int c = 0; c < S::CPT; c++) acc[c] = fma(dv, sX[cg * S::CPT + c][kk], acc[c]);
        }
        __syncthreads();
    }
    if (S::KG > 1) {
#pragma unroll
        for (int c = 0; c < S::CPT; c++) sR[tid * S::CPT + c] = acc[c];
        __syncthreads();
        if (kg != 0) return;
        for (int g = 1; g < S::KG; g++)
#pragma unroll
            for (int c = 0; c < S::CPT; c++) acc[c] += sR[(tid + g * BM * S::CG) * S::CPT + c];
    }
    const long gr = row0 + r;
    if (gr >= n3) return;
    if (!CHEB) {
#pragma unroll
        for (int c = 0; c < S::CPT; c++) {
            int j = cg * S::CPT + c;
            if (j < m) Y[(long)j * n3 + gr] = acc[c];
        }
    } else {
        const double dmin = e.bounds[0], dmax = e.bounds[1];
        const double ys = 2.0 / (dmax - dmin), yt = (dmax + dmin) / (dmax - dmin);
        const double cp = e.coef[e.p];
#pragma unroll
        for (int c = 0; c < S::CPT; c++) {
            int j = cg * S::CPT + c;
            if (j < m) {
                long o = (long)j * n3 + gr;
                double v = 2.0 * (ys * acc[c] - yt * e.Vprev1[o]) - e.Vprev2[o];
                e.Vprev2[o] = v;
                e.dS[o] += cp * v;
            }
        }
    }
}

// -- kernel end: k_gemm_f64

// m = 1 (Lanczos and single products): one warp per row, each lane streams
// a strided slice of the row with two independent FP64 accumulators; the
// FP64 pipe (one FMA per 8 bytes) and HBM are then both near their limits
__global__ void __launch_bounds__(256)
k_gemv_f64(const double *__restrict__ D, long ld, int n3, const double *__restrict__ x,
           double *__restrict__ y)
{
    const long row = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n3) return;
    const double *d = D + row * ld;
    double a0 = 0.0, a1 = 0.0;
    int k = lane;
    for (; k + 32 < n3; k += 64) {
        a0 = fma(__ldg(d + k), __ldg(x + k), a0);
        a1 = fma(__ldg(d + k + 32), __ldg(x + k + 32), a1);
    }
    if (k < n3) a0 = fma(__ldg(d + k), __ldg(x + k), a0);
    double a = a0 + a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) y[row] = a;
}

template <bool CHEB>
static void dispatch(const Plan &P, const double *D, const double *X, int m, double *Y,
                     const ChebEpi &e, cudaStream_t s)
{
    dim3 g((P.n3 + BM - 1) / BM);
#define BD_GEMM_CASE(MC)                                                                    \
    k_gemm_f64<MC, CHEB><<<g, NT, 0, s>>>(D, P.ld, P.n3, X, m, Y, e)
    if (m <= 1) BD_GEMM_CASE(1);
    else if (m <= 2) BD_GEMM_CASE(2);
    else if (m <= 4) BD_GEMM_CASE(4);
    else if (m <= 8) BD_GEMM_CASE(8);
    else if (m <= 16) BD_GEMM_CASE(16);
    else BD_GEMM_CASE(32);
    count_launches(1);
#undef BD_GEMM_CASE
}

void launch_gemm_f64(const Plan &P, const double *D, const double *X, int m, double *Y,
                     cudaStream_t s)
{
    if (m == 1) {
        long threads = (long)P.n3 * 32;
        k_gemv_f64<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(D, P.ld, P.n3, X, Y);
        count_launches(1);
        return;
    }
    ChebEpi e{};
    dispatch<false>(P, D, X, m, Y, e, s);
}

void launch_gemm_f64_cheb(const Plan &P, const double *D, int m, const ChebEpi &e,
                          cudaStream_t s)
{
    prod_mark(const_cast<Plan &>(P), 0, s);
    dispatch<true>(P, D, e.Vprev1, m, nullptr, e, s);
    prod_mark(const_cast<Plan &>(P), 1, s);
}

}  // namespace bd
