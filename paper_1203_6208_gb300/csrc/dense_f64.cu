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
        const double ys = e.coef[kChebMapS], yt = e.coef[kChebMapT];
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

// ---------------------------------------------------------------------------
// The same products in double-float on the FP32 pipe (FP64 plans, launch
// shape 4): the FP64 pipe of this GPU runs at 1/64 of FP32, so each FP64 word
// is split into two FP32 words d = dh + dl (48 significant bits), every
// product dh xh is formed exactly as (p, fma(dh, xh, -p)), the cross terms
// dh xl + dl xh are added to that error, and the products are summed as a
// double-float (TwoSum): ~12 FP32 operations per multiply-add, ~1e-14 relative
// to sum |d x|.  The D words are split with integer operations (conversions
// also run on the FP64 pipe here).  The products of one k tile are summed into
// a pair started at zero, whose error word is not renormalised, and each tile
// sum is added to the running pair with renormalisation: the error word never
// collects more than a tile's worth of rounding errors, so its own FP32
// rounding stays far below 2^-48 of the sum.

// d = hi + lo with hi = d truncated to 24 significant bits and lo the
// remaining 29 bits rounded to 24, from 32-bit integer operations and three
// FP32 additions (the leading-zero count and 64-bit shifts would run on the
// slow conversion path).  With s the sign, e the binary exponent and r the low
// 29 mantissa bits (d = hi + r 2^(e-52)), r is cut into r >> 6 and r & 63; a
// float whose exponent is e - 23 (resp. e - 29) and whose mantissa field holds
// that piece equals 2^(e-23) (resp. 2^(e-29)) plus the piece times 2^(e-46)
// (resp. 2^(e-52)), so subtracting the bare power of two is exact (Sterbenz)
// and leaves the piece; their sum is lo.  Exact for e in [-97, 127] (every
// word normal).  Below, the entry counts as zero (|d| < 2^-97); above, hi is
// an infinity of d's sign (FP32 overflow): D and X must lie in that range.
// No FP64 instruction is issued, not even a predicated one.
__device__ __forceinline__ void split_df(double d, float &hi, float &lo)
{
    const unsigned w1 = (unsigned)__double2hiint(d), w0 = (unsigned)__double2loint(d);
    const unsigned sign = w1 & 0x80000000u;
    const int e = (int)((w1 >> 20) & 0x7ff) - 1023;
    if (e < -97) { hi = 0.f; lo = 0.f; return; }                  // +-0, subnormal, tiny
    if (e > 127) { hi = __uint_as_float(sign | 0x7F800000u); lo = 0.f; return; }
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((w1 & 0xFFFFFu) << 3) | (w0 >> 29));
    const unsigned r = w0 & 0x1FFFFFFFu;
    const unsigned ba = sign | ((unsigned)(e - 23 + 127) << 23);
    const unsigned bb = sign | ((unsigned)(e - 29 + 127) << 23);
    const float la = __uint_as_float(ba | (r >> 6)) - __uint_as_float(ba);
    const float lb = __uint_as_float(bb | (r & 63u)) - __uint_as_float(bb);
    lo = la + lb;
}

struct DFAcc {
    float s, c;
};

__device__ __forceinline__ void df_fma(DFAcc &a, float dh, float dl, float xh, float xl)
{
    const float p = dh * xh;
    float e = fmaf(dh, xh, -p);
    e = fmaf(dh, xl, e);
    e = fmaf(dl, xh, e);
    const float t = a.s + p, z = t - a.s;
    a.c += ((a.s - (t - z)) + (p - z)) + e;
    a.s = t;
}

// a += b for two pairs, renormalised (|a.c| <= ulp(a.s) / 2 afterwards)
__device__ __forceinline__ void df_join(DFAcc &a, const DFAcc &b)
{
    const float t = a.s + b.s, z = t - a.s;
    const float e = ((a.s - (t - z)) + (b.s - z)) + (a.c + b.c);
    a.s = t + e;
    a.c = e - (a.s - t);
}

// the operand's columns split once per product: xs[0][j][i] = hi, xs[1][j][i] = lo
__global__ void k_split_cols(const double *__restrict__ X, long len, float *__restrict__ xs)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const double v = X[i];
    const float h = (float)v;
    xs[i] = h;
    xs[len + i] = (float)(v - (double)h);
}

// -- kernel begin: k_gemm_df
// D staged as (hi, lo) pairs, one 8-byte load per row and k; X staged k-major
// with each thread's CPT columns contiguous (broadcast vector loads)
template <int CPT>
__device__ __forceinline__ void load_cols(const float *p, float (&v)[CPT])
{
    if constexpr (CPT % 4 == 0) {
#pragma unroll
        for (int c = 0; c < CPT; c += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(p + c);
            v[c] = q.x; v[c + 1] = q.y; v[c + 2] = q.z; v[c + 3] = q.w;
        }
    } else if constexpr (CPT == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else {
#pragma unroll
        for (int c = 0; c < CPT; c++) v[c] = p[c];
    }
}

// 256 threads: BM rows x CG column groups x KG k groups; the next tile of D
// and X is loaded into registers while the current one is multiplied
constexpr int NTD = 256;

template <int MC>
struct ShapeDF {
    static constexpr int CG = MC >= 4 ? 4 : MC;
    static constexpr int CPT = MC / CG;
    static constexpr int KG = NTD / (BM * CG);
    static constexpr int DPT = BM * BK / NTD;                 // D entries staged per thread
    static constexpr int XPT = (MC * BK + NTD - 1) / NTD;     // X entries staged per thread
};

template <int MC, bool CHEB>
__global__ void __launch_bounds__(NTD)
k_gemm_df(const double *__restrict__ D, long ld, int n3, const float *__restrict__ xs, int m,
          double *__restrict__ Y, ChebEpi e)
{
    using S = ShapeDF<MC>;
    // row stride MC + 4: 16-byte aligned rows, and the fill below (8 k x 4
    // columns per warp) lands on 32 distinct banks for MC = 8, 16, 24 and 32
    // (one warp's 32 addresses enumerated: XS = 12, 20, 28, 36); MC = 4 takes
    // two words per bank.  MC = 24 gives CPT = 6 columns per thread, which
    // load_cols reads element by element (no 16-byte vector of 6)
    constexpr int XS = MC >= 4 ? MC + 4 : MC;
    constexpr int JG = MC >= 4 ? 4 : MC;
    __shared__ float2 sD[BM][BK + 1];
    __shared__ __align__(16) float sXh[BK][XS];
    __shared__ __align__(16) float sXl[BK][XS];
    __shared__ DFAcc sR[S::KG > 1 ? NTD * S::CPT : 1];

    const int tid = threadIdx.x;
    const int r = tid % BM;
    const int cg = (tid / BM) % S::CG;
    const int kg = tid / (BM * S::CG);
    const long row0 = (long)blockIdx.x * BM;
    const long len = (long)m * n3;

    double dreg[S::DPT];
    float xhr[S::XPT], xlr[S::XPT];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < S::DPT; q++) {
            const int i = tid + q * NTD, rr = i / BK, kk = i % BK;
            const long gr = row0 + rr;
            const int gk = k0 + kk;
            dreg[q] = (gr < n3 && gk < n3) ? __ldg(&D[gr * ld + gk]) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < S::XPT; q++) {
            const int i = tid + q * NTD;
            const int rest = i / (8 * JG);
            const int kk = (i % 8) + 8 * (rest % (BK / 8));
            const int j = (i / 8) % JG + JG * (rest / (BK / 8));
            const int gk = k0 + kk;
            const bool ok = i < MC * BK && j < m && gk < n3;
            xhr[q] = ok ? __ldg(&xs[(long)j * n3 + gk]) : 0.f;
            xlr[q] = ok ? __ldg(&xs[len + (long)j * n3 + gk]) : 0.f;
        }
    };

    DFAcc acc[S::CPT];
#pragma unroll
    for (int c = 0; c < S::CPT; c++) acc[c] = DFAcc{0.f, 0.f};

    fetch(0);
    for (int k0 = 0; k0 < n3; k0 += BK) {
        __syncthreads();                       // the previous tile is consumed
#pragma unroll
        for (int q = 0; q < S::DPT; q++) {
            const int i = tid + q * NTD;
            float h, l;
            split_df(dreg[q], h, l);
            sD[i / BK][i % BK] = make_float2(h, l);
        }
#pragma unroll
        for (int q = 0; q < S::XPT; q++) {
            const int i = tid + q * NTD;
            if (i < MC * BK) {
                const int rest = i / (8 * JG);
                const int kk = (i % 8) + 8 * (rest % (BK / 8));
                const int j = (i / 8) % JG + JG * (rest / (BK / 8));
                sXh[kk][j] = xhr[q];
                sXl[kk][j] = xlr[q];
            }
        }
        __syncthreads();
        if (k0 + BK < n3) fetch(k0 + BK);
        DFAcc t[S::CPT];
#pragma unroll
        for (int c = 0; c < S::CPT; c++) t[c] = DFAcc{0.f, 0.f};
#pragma unroll 4
        for (int kk = kg; kk < BK; kk += S::KG) {
            const float2 d = sD[r][kk];
            float xh[S::CPT], xl[S::CPT];
            load_cols<S::CPT>(&sXh[kk][cg * S::CPT], xh);
            load_cols<S::CPT>(&sXl[kk][cg * S::CPT], xl);
#pragma unroll
            for (int c = 0; c < S::CPT; c++) df_fma(t[c], d.x, d.y, xh[c], xl[c]);
        }
#pragma unroll
        for (int c = 0; c < S::CPT; c++) df_join(acc[c], t[c]);
    }
    if (S::KG > 1) {
#pragma unroll
        for (int c = 0; c < S::CPT; c++) sR[tid * S::CPT + c] = acc[c];
        __syncthreads();
        if (kg != 0) return;
        for (int g = 1; g < S::KG; g++)
#pragma unroll
            for (int c = 0; c < S::CPT; c++) df_join(acc[c], sR[(tid + g * BM * S::CG) * S::CPT + c]);
    }
    const long gr = row0 + r;
    if (gr >= n3) return;
    if (!CHEB) {
#pragma unroll
        for (int c = 0; c < S::CPT; c++) {
            int j = cg * S::CPT + c;
            if (j < m) Y[(long)j * n3 + gr] = (double)acc[c].s + (double)acc[c].c;
        }
    } else {
        const double ys = e.coef[kChebMapS], yt = e.coef[kChebMapT];
        const double cp = e.coef[e.p];
#pragma unroll
        for (int c = 0; c < S::CPT; c++) {
            int j = cg * S::CPT + c;
            if (j < m) {
                long o = (long)j * n3 + gr;
                const double w = (double)acc[c].s + (double)acc[c].c;
                double v = 2.0 * (ys * w - yt * e.Vprev1[o]) - e.Vprev2[o];
                e.Vprev2[o] = v;
                e.dS[o] += cp * v;
            }
        }
    }
}
// -- kernel end: k_gemm_df

// m = 1: one warp per row, the lanes over a strided slice of the row, 8
// loads of D in flight per lane; each group of 8 products is summed into an
// unnormalised pair and joined into the running sum
__global__ void __launch_bounds__(256)
k_gemv_df(const double *__restrict__ D, long ld, int n3, const float *__restrict__ xs,
          double *__restrict__ y)
{
    const long row = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n3) return;
    const double *d = D + row * ld;
    const float *xh = xs, *xl = xs + n3;
    DFAcc a0{0.f, 0.f};
    int k = lane;
    for (; k + 7 * 32 < n3; k += 8 * 32) {
        double v[8];
        float h[8], l[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = __ldg(d + k + 32 * u);
#pragma unroll
        for (int u = 0; u < 8; u++) {
            h[u] = __ldg(xh + k + 32 * u);
            l[u] = __ldg(xl + k + 32 * u);
        }
        DFAcc t{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 8; u++) {
            float dh, dl;
            split_df(v[u], dh, dl);
            df_fma(t, dh, dl, h[u], l[u]);
        }
        df_join(a0, t);
    }
    DFAcc t{0.f, 0.f};
    for (; k < n3; k += 32) {
        float dh, dl;
        split_df(__ldg(d + k), dh, dl);
        df_fma(t, dh, dl, __ldg(xh + k), __ldg(xl + k));
    }
    df_join(a0, t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DFAcc b{__shfl_xor_sync(0xffffffffu, a0.s, o), __shfl_xor_sync(0xffffffffu, a0.c, o)};
        // the same two values in the same order on both lanes of a pair
        DFAcc lo = (lane & o) ? b : a0, hi = (lane & o) ? a0 : b;
        df_join(lo, hi);
        a0 = lo;
    }
    if (lane == 0) y[row] = (double)a0.s + (double)a0.c;
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
    else if (m <= 24) BD_GEMM_CASE(24);      // a step's first product: 16 + 1 columns
    else BD_GEMM_CASE(32);
    count_launches(1);
#undef BD_GEMM_CASE
}

template <bool CHEB>
static void dispatch_df(const Plan &P, const double *D, const double *X, int m, double *Y,
                        const ChebEpi &e, cudaStream_t s)
{
    const long len = (long)m * P.n3;
    k_split_cols<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(X, len, P.d_xdf);
    count_launches(1);
    if (m == 1 && !CHEB) {
        long threads = (long)P.n3 * 32;
        k_gemv_df<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(D, P.ld, P.n3, P.d_xdf, Y);
        count_launches(1);
        return;
    }
    dim3 g((P.n3 + BM - 1) / BM);
#define BD_GEMM_DF_CASE(MC)                                                                   \
    k_gemm_df<MC, CHEB><<<g, NTD, 0, s>>>(D, P.ld, P.n3, P.d_xdf, m, Y, e)
    if (m <= 1) BD_GEMM_DF_CASE(1);
    else if (m <= 2) BD_GEMM_DF_CASE(2);
    else if (m <= 4) BD_GEMM_DF_CASE(4);
    else if (m <= 8) BD_GEMM_DF_CASE(8);
    else if (m <= 16) BD_GEMM_DF_CASE(16);
    else if (m <= 24) BD_GEMM_DF_CASE(24);
    else BD_GEMM_DF_CASE(32);
    count_launches(1);
#undef BD_GEMM_DF_CASE
}

void launch_gemm_f64(const Plan &P, const double *D, const double *X, int m, double *Y,
                     cudaStream_t s)
{
    if (P.tc_split == kF64DoubleFloat && P.d_xdf && m <= kMaxRhs) {
        ChebEpi e{};
        dispatch_df<false>(P, D, X, m, Y, e, s);
        return;
    }
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
    if (P.tc_split == kF64DoubleFloat && P.d_xdf && m <= kMaxRhs) dispatch_df<true>(P, D, e.Vprev1, m, nullptr, e, s);
    else dispatch<true>(P, D, e.Vprev1, m, nullptr, e, s);
    prod_mark(const_cast<Plan &>(P), 1, s);
}

}  // namespace bd
