// tc_gemm.cu -- mixed-precision products Y = D16 X on the 5th-generation
// tensor cores (tcgen05, sm_103a), and the FP64-residual refinement of D.F.
//
// With m <= 32 right-hand sides the product reads the whole 16-bit copy of D
// once per call at ~m flop per byte, so it is bound by HBM, not by the tensor
// pipe.  The kernel is a TMA -> shared memory -> tcgen05.mma -> TMEM stream:
//   * a CTA owns a 128-row block of D and one K-split; warp 0 issues TMA
//     loads of 128 x 64 tiles of D16 (128-byte swizzle) and 64 x BN tiles of
//     the scaled 16-bit operand X^T into a ST-deep ring; warp 1 issues
//     tcgen05.mma (M = 128, N = BN, K = 16, FP32 accumulator in TMEM);
//     warps 2-5 drain TMEM and write an FP32 partial;
//   * the last CTA of a row block to finish (arrival counter) sums the
//     partials of its row block in FP64 in split order (deterministic) and
//     runs the epilogue: either a plain store of Y (FP64, column scales
//     undone) or the Chebyshev term of Eqs. (cheb2)/(cheb3)
//       V_p = 2 (s W - t V_{p-1}) - V_{p-2},  dS += c_p V_p,
//     which also writes the scaled 16-bit V_p as the next product's operand.
// Every wait on an mbarrier is bounded; a wait that gives up records
// BD_ERR_TIMEOUT in a device status word, drains what is in flight, frees its
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "sym_gemm.cuh"
#include "tc_common.cuh"
#include "tc_gemm.cuh"
#include "rows_gemm.cuh"

namespace bd {

namespace tc {

// -- kernel begin: k_tc_gemm
// Stream-K schedule: the product is cut into units (row block mb, K tile kt),
// u = mb * ktiles + kt, and CTA c of the G resident CTAs owns the contiguous
// range [c U / G, (c + 1) U / G) of the U units.  A CTA's range crosses row
// blocks; each run of units inside one row block (a segment) accumulates in
// one of two TMEM buffers, so the MMA warp starts the next segment while the
// epilogue warps drain the previous one.  A segment's FP32 partial goes to
// slot (c - first CTA of mb) of its row block; the CTA that completes a row
// block (arrival counter) sums the slots in slot order in FP64
// (deterministic for a given G) and runs the epilogue, then resets the
// counter for the next launch.  No CTA ever waits on another.
__device__ __forceinline__ int cta_of_unit(long u, long U, int G)
{
    return (int)(((u + 1) * (long)G + U - 1) / U) - 1;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int BN, int ST>
__global__ void __launch_bounds__(THREADS, (ST > 8 ? 1 : 2))
k_tc_gemm(const __grid_constant__ CUtensorMap mapD, const __grid_constant__ CUtensorMap mapX,
          int n3, int ktiles, int mblk, int maxslots, float *__restrict__ part,
          int32_t *__restrict__ counters, int32_t *__restrict__ err, Epi e)
{
    constexpr int B_BYTES = BN * BK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;          // multiple of 1024
    static_assert(STAGE % 1024 == 0, "stage alignment");
    constexpr uint32_t IDESC_F16 = idesc_f16(BN, 0), IDESC_BF16 = idesc_f16(BN, 1);
    constexpr uint32_t TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[ST], empty_bar[ST];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;
    __shared__ int is_last_sh;
    __shared__ double lan_red[4][3];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, c = blockIdx.x;
    const long U = (long)mblk * ktiles;
    const long u0 = (long)c * U / G, u1 = (long)(c + 1) * U / G;
    const int nunits = (int)(u1 - u0);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < ST; s++) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), 128);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    int issued = 0;                      // the producer's loads, for the drain after an abort
    if (warp == 0 && lane == 0) {
        // ---- TMA producer: every unit of the range, in order
        int mb = (int)(u0 / ktiles), kt = (int)(u0 % ktiles);
        for (int i = 0; i < nunits; i++, kt = (kt + 1 == ktiles) ? 0 : kt + 1, mb += (kt == 0)) {
            int s = i % ST;
            uint32_t ph = (uint32_t)(i / ST) & 1u;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, &abort_flag)) break;
            uint32_t a = smem_u32(smem + s * STAGE), b = a + A_BYTES;
            uint32_t fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, STAGE);
            tma_load_2d(a, &mapD, kt * BK, mb * BM, fb);
            tma_load_2d(b, &mapX, kt * BK, 0, fb);
            issued = i + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: segment j accumulates in TMEM buffer j & 1
        const uint32_t idesc = e.is_bf16 ? IDESC_BF16 : IDESC_F16;
        bool ok = true;
        int j = -1, cur_mb = -1;
        int mb = (int)(u0 / ktiles), kt = (int)(u0 % ktiles);
        for (int i = 0; i < nunits && ok; i++, kt = (kt + 1 == ktiles) ? 0 : kt + 1, mb += (kt == 0)) {
            const bool first = (mb != cur_mb);
            if (first) {
                cur_mb = mb;
                j++;
                if (j >= 2 &&
                    !mbar_wait(smem_u32(&acc_empty[j & 1]), (uint32_t)((j >> 1) - 1) & 1u, &abort_flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint32_t acc = tmem + (uint32_t)((j & 1) * BN);
            int s = i % ST;
            uint32_t ph = (uint32_t)(i / ST) & 1u;
            if (!mbar_wait(smem_u32(&full_bar[s]), ph, &abort_flag)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t a = smem_u32(smem + s * STAGE), b = a + A_BYTES;
            uint64_t da = sw128_desc(a), db = sw128_desc(b);
#pragma unroll
            for (int k = 0; k < BK / 16; k++) {
                // advance 16 elements (32 bytes) along K inside the swizzled rows
                mma_f16(acc, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc,
                        (!first || k > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&empty_bar[s]));
            const bool last = (i + 1 == nunits) || (kt + 1 == ktiles);
            if (last) mma_commit(smem_u32(&acc_full[j & 1]));
        }
        if (!ok) {
            mma_commit(smem_u32(&drain_bar));
            for (uint32_t t = 0; t < kWaitLimit && !mbar_try(smem_u32(&drain_bar), 0); t++) {}
        }
    } else if (warp >= 2) {
        // ---- epilogue warps: each segment in order
        const int q = warp & 3;                      // TMEM lane quadrant of this warp
        const int r = q * 32 + lane;                 // row within the block
        long u = u0;
        for (int j = 0; u < u1; j++) {
            const int mb = (int)(u / ktiles);
            const long ue = ((long)(mb + 1) * ktiles < u1) ? (long)(mb + 1) * ktiles : u1;
            u = ue;
            float acc[BN];
            if (!mbar_wait_sleep(smem_u32(&acc_full[j & 1]), (uint32_t)(j >> 1) & 1u, &abort_flag))
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int cc = 0; cc < BN; cc += 16)
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((j & 1) * BN + cc), acc + cc);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&acc_empty[j & 1]));
            const int c0 = cta_of_unit((long)mb * ktiles, U, G);
            const int c1 = cta_of_unit((long)mb * ktiles + ktiles - 1, U, G);
            const int nslots = c1 - c0 + 1;
            float4 *dst = (float4 *)(part + (((size_t)mb * maxslots + (c - c0)) * BM + r) * BN);
#pragma unroll
            for (int cc = 0; cc < BN / 4; cc++)
                dst[cc] = make_float4(acc[4 * cc], acc[4 * cc + 1], acc[4 * cc + 2], acc[4 * cc + 3]);
            __threadfence();
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (threadIdx.x == 64) {
                int old = atomicAdd(&counters[mb], 1);
                is_last_sh = (old == nslots - 1);
                if (old == nslots - 1) counters[mb] = 0;   // every slot is in: ready for the next launch
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (!is_last_sh) continue;
            __threadfence();
            const long row = (long)mb * BM + r;
            double y[BN];
#pragma unroll
            for (int cc = 0; cc < BN; cc++) y[cc] = 0.0;
            for (int sp0 = 0; sp0 < nslots; sp0 += 2) {
                // two slots per round, all loads of a round issued together
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int sp = sp0 + h;
                    if (sp < nslots) {
                        const float4 *src =
                            (const float4 *)(part + (((size_t)mb * maxslots + sp) * BM + r) * BN);
#pragma unroll
                        for (int cc = 0; cc < BN / 4; cc++) {
                            float4 v = __ldcg(src + cc);
                            y[4 * cc] += v.x; y[4 * cc + 1] += v.y;
                            y[4 * cc + 2] += v.z; y[4 * cc + 3] += v.w;
                        }
                    }
                }
            }
            double lw = 0.0;                          // this row of D q_j (Lanczos column)
            if (row < n3) {
                if (e.mode == 0) {
#pragma unroll
                    for (int cc = 0; cc < BN; cc++)
                        if (cc < e.m) e.Y[(long)cc * n3 + row] = y[cc] * (double)e.inv_scale[cc];
                } else {
                    const double ys = e.coef[kChebMapS], yt = e.coef[kChebMapT];
                    const double cp = e.coef[e.p];
                    // columns in chunks of 8: every load of a chunk is issued
                    // before its stores (the vectors may alias as far as the
                    // compiler knows, so loads do not move above earlier stores)
                    constexpr int CH = 8;
#pragma unroll
                    for (int c0 = 0; c0 < BN; c0 += CH) {
                        double p1[CH], p2[CH], d0[CH];
#pragma unroll
                        for (int q = 0; q < CH; q++) {
                            const int cc = c0 + q;
                            if (cc < e.m) {
                                const long o = (long)cc * n3 + row;
                                p1[q] = __ldcg(e.Vprev1 + o);
                                p2[q] = __ldcg(e.Vprev2 + o);
                                d0[q] = __ldcg(e.dS + o);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < CH; q++) {
                            const int cc = c0 + q;
                            // a select, not a branch: a branch on cc == lan_col
                            // becomes y[lan_col] and sends y to local memory
                            const double yv = y[cc];
                            lw = (cc == e.lan_col) ? yv * (double)e.inv_scale[cc] : lw;
                            if (cc < e.m) {
                                const long o = (long)cc * n3 + row;
                                const double w = y[cc] * (double)e.inv_scale[cc];
                                const double v = 2.0 * (ys * w - yt * p1[q]) - p2[q];
                                e.Vprev2[o] = v;
                                e.dS[o] = d0[q] + cp * v;
                                float sv = (float)(v * (double)e.scale[cc]);
                                size_t xo = (size_t)cc * e.ldx + row;
                                if (e.is_bf16) ((__nv_bfloat16 *)e.X16next)[xo] = __float2bfloat16_rn(sv);
                                else ((__half *)e.X16next)[xo] = __float2half_rn(sv);
                            }
                        }
                    }
                }
            }
            if (e.mode == 1 && e.lan_col >= 0 && row < n3) e.lan_w[row] = lw;
            if (e.mode == 1 && e.lan_col >= 0) {
                // this row block's share of q_j.w, q_{j-1}.w and w.w, reduced in
                // a fixed order (deterministic)
                double t[3] = {row < n3 ? e.lan_q[row] * lw : 0.0,
                               row < n3 ? e.lan_qp[row] * lw : 0.0, lw * lw};
#pragma unroll
                for (int k = 0; k < 3; k++)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
                if (lane == 0)
                    for (int k = 0; k < 3; k++) lan_red[q][k] = t[k];
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (r == 0)
                    for (int k = 0; k < 3; k++)
                        e.lan_part[3 * mb + k] =
                            ((lan_red[0][k] + lan_red[1][k]) + lan_red[2][k]) + lan_red[3][k];
            }
        }
    }
    // ---- teardown.  Every role has left its loop once all threads are here,
    // so abort_flag is final: after an abort the producer lets every load it
    // issued land before the CTA exits, and the status word records it.
    __syncthreads();
    if (abort_flag) {
        if (warp == 0 && lane == 0)
            for (int i = (issued > ST ? issued - ST : 0); i < issued; i++) {
                int s = i % ST;
                uint32_t ph = (uint32_t)(i / ST) & 1u;
                for (uint32_t t = 0; t < kWaitLimit && !mbar_try(smem_u32(&full_bar[s]), ph); t++) {}
            }
        if (threadIdx.x == 0) atomicExch(err, (int32_t)BD_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

// -- kernel end: k_tc_gemm

template <int BN, int ST>
constexpr int smem_bytes()
{
    return ST * (A_BYTES + BN * BK * 2) + 1024;
}

}  // namespace tc

// ---------------------------------------------------------------------------
// operand preparation: per-column power-of-two scale and 16-bit X^T

// scale_j = 2^-e with 2^(e-1) < max|X_j| <= 2^e (max scaled magnitude 1)
__global__ void k_col_absmax(const double *X, int n3, int m, unsigned long long *bits)
{
    int j = blockIdx.y;
    double v = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (long)gridDim.x * blockDim.x)
        v = fmax(v, fabs(X[(long)j * n3 + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&bits[j], (unsigned long long)__double_as_longlong(v));
}

__global__ void k_col_scale(const unsigned long long *bits, int m, int bn, float *scale,
                            float *inv_scale)
{
    int j = threadIdx.x;
    if (j >= bn) return;
    float s = 1.f;
    if (j < m) {
        double mx = __longlong_as_double((long long)bits[j]);
        if (mx > 0.0 && isfinite(mx)) {
            int e;
            frexp(mx, &e);                       // mx = f 2^e, 0.5 <= f < 1
            s = ldexpf(1.f, -e);
        }
    }
    scale[j] = s;
    inv_scale[j] = 1.f / s;
}

// X16[j][i] = X[i][j] * scale_j for j < m, zero rows for m <= j < bn
__global__ void k_to16(const double *X, int n3, int m, int bn, const float *scale, void *X16,
                       int ldx, int is_bf16)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= n3 || j >= bn) return;
    float v = j < m ? (float)(X[(long)j * n3 + i] * (double)scale[j]) : 0.f;
    size_t o = (size_t)j * ldx + i;
    if (is_bf16) ((__nv_bfloat16 *)X16)[o] = __float2bfloat16_rn(v);
    else ((__half *)X16)[o] = __float2half_rn(v);
}

// ---------------------------------------------------------------------------
// host side

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bd_status get_encoder()
{
    if (g_encode) return BD_OK;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return set_error(BD_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return BD_OK;
}

static bd_status make_map(CUtensorMap *map, const void *base, int is_bf16, uint64_t inner,
                          uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer)
{
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(map, is_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                          2, const_cast<void *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(BD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return BD_OK;
}

// ring depths of the four launch shapes (BN x resident CTAs per SM)
constexpr int S16_2 = tc::stages_for<16>(2), S32_2 = tc::stages_for<32>(2);
constexpr int S16_1 = tc::stages_for<16>(1), S32_1 = tc::stages_for<32>(1);
static_assert(S16_2 >= 4 && S32_2 >= 4, "ring too shallow");
static_assert(tc::smem_bytes<16, S16_1>() <= 227 * 1024 && tc::smem_bytes<32, S32_1>() <= 227 * 1024,
              "one-CTA ring exceeds shared memory");
static_assert(2 * (tc::smem_bytes<16, S16_2>() + 2048) <= 228 * 1024 &&
              2 * (tc::smem_bytes<32, S32_2>() + 2048) <= 228 * 1024,
              "two CTAs per SM do not fit");

static int mblocks(const Plan &P) { return (P.n3 + tc::BM - 1) / tc::BM; }
static int ktiles_of(const Plan &P) { return (P.n3 + tc::BK - 1) / tc::BK; }

// resident CTAs of the stream-K product: ctas_per_sm per SM, at most one per unit
static int sk_grid(const Plan &P, int ctas_per_sm)
{
    long U = (long)mblocks(P) * ktiles_of(P);
    long g = (long)ctas_per_sm * P.num_sms;
    return (int)(g < U ? g : U);
}

// most CTAs sharing one row block for grid G (partial slots per row block)
static int sk_maxslots(const Plan &P, int G)
{
    const long KT = ktiles_of(P), MB = mblocks(P), U = MB * KT;
    auto cta_of = [&](long u) { return (int)(((u + 1) * G + U - 1) / U) - 1; };
    int mx = 1;
    for (long mb = 0; mb < MB; mb++) {
        int ns = cta_of(mb * KT + KT - 1) - cta_of(mb * KT) + 1;
        if (ns > mx) mx = ns;
    }
    return mx;
}

bd_status tc_plan_init(Plan &P)
{
    bd_status st = get_encoder();
    if (st != BD_OK) return st;
    if (cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device) != cudaSuccess ||
        P.num_sms < 1)
        return set_error(BD_ERR_CUDA, "SM count unavailable");
    P.ldx = (P.n3 + kLdAlign - 1) / kLdAlign * kLdAlign;
    size_t x16 = (size_t)2 * kMaxRhs * P.ldx * 2;               // two operand buffers
    size_t mbk = (size_t)mblocks(P);
    P.tc_maxslots = 1;
    for (int cps = 1; cps <= tc::kMaxCtasPerSm; cps++) {
        int ms = sk_maxslots(P, sk_grid(P, cps));
        if (ms > P.tc_maxslots) P.tc_maxslots = ms;
    }
    const size_t part = (size_t)P.tc_maxslots * mbk * tc::BM * kMaxRhs * sizeof(float);
    cudaError_t e = cudaMalloc(&P.d_x16, x16);
    if (e == cudaSuccess) e = cudaMalloc(&P.d_xscale, 4 * kMaxRhs * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_part, part);
    if (e == cudaSuccess) e = cudaMalloc(&P.d_counters, (mbk + 64) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_lanpart, 3 * mbk * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BD_ERR_OOM, "mixed-precision scratch: %s", cudaGetErrorString(e));
    }
    P.scratch_bytes += (int64_t)(x16 + 4 * kMaxRhs * sizeof(float) + part +
                                 (mbk + 64) * sizeof(int32_t) + 3 * mbk * sizeof(double));
    cudaMemset(P.d_x16, 0, x16);
    cudaMemset(P.d_counters, 0, (mbk + 64) * sizeof(int32_t));
    cudaError_t a[4] = {
        cudaFuncSetAttribute(tc::k_tc_gemm<16, S16_2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::smem_bytes<16, S16_2>()),
        cudaFuncSetAttribute(tc::k_tc_gemm<32, S32_2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::smem_bytes<32, S32_2>()),
        cudaFuncSetAttribute(tc::k_tc_gemm<16, S16_1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::smem_bytes<16, S16_1>()),
        cudaFuncSetAttribute(tc::k_tc_gemm<32, S32_1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::smem_bytes<32, S32_1>())};
    for (cudaError_t x : a)
        if (x != cudaSuccess) return set_error(BD_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(x));
    return BD_OK;
}

static void *x16_buf(Plan &P, int which)
{
    return (char *)P.d_x16 + (size_t)which * kMaxRhs * P.ldx * 2;
}

// column scales of X (rows 0..m-1 of the (m, 3N) block) and the 16-bit copy
static void prepare_operand(Plan &P, const double *X, int m, int bn, void *X16, cudaStream_t s)
{
    unsigned long long *bits = (unsigned long long *)(P.d_xscale + 2 * kMaxRhs);
    launch_zero_i32((int32_t *)bits, 2 * kMaxRhs, s);
    k_col_absmax<<<dim3(64, m), 256, 0, s>>>(X, P.n3, m, bits);
    count_launches(1);
    k_col_scale<<<1, 32, 0, s>>>(bits, m, bn, P.d_xscale, P.d_xscale + kMaxRhs);
    count_launches(1);
    k_to16<<<dim3((P.n3 + 255) / 256, bn), 256, 0, s>>>(X, P.n3, m, bn, P.d_xscale, X16, P.ldx,
                                                       P.p.precision == BD_MIXED_BF16);
    count_launches(1);
}

static bd_status launch_tc(Plan &P, const void *D16, const void *X16, int bn, const tc::Epi &e,
                           cudaStream_t s)
{
    const int is_bf16 = P.p.precision == BD_MIXED_BF16;
    CUtensorMap mapD, mapX;
    bd_status st = make_map(&mapD, D16, is_bf16, P.n3, P.n3, (uint64_t)P.ld * 2, tc::BK, tc::BM);
    if (st != BD_OK) return st;
    st = make_map(&mapX, X16, is_bf16, P.n3, bn, (uint64_t)P.ldx * 2, tc::BK, bn);
    if (st != BD_OK) return st;
    if (P.tc_split == kSymShape) {
        if (e.mode == 1) prod_mark(P, 0, s);
        st = sym_launch(P, mapD, mapX, bn, e, s);
        if (e.mode == 1) prod_mark(P, 1, s);
        return st;
    }
    const int ktiles = ktiles_of(P), mbk = mblocks(P);
    const int G = sk_grid(P, P.tc_split > 0 ? P.tc_split : tc::kMaxCtasPerSm);
    // the arrival counters reset themselves; a plain product (the first of
    // every step) also clears them in case an earlier launch gave up
    if (e.mode == 0) launch_zero_i32(P.d_counters, mbk, s);
    int32_t *err = P.d_status + 6;
    if (e.mode == 1) prod_mark(P, 0, s);
    const bool two = (P.tc_split > 0 ? P.tc_split : tc::kMaxCtasPerSm) == 2;
#define TC_LAUNCH(BNV, STV)                                                                   \
    tc::k_tc_gemm<BNV, STV><<<G, tc::THREADS, tc::smem_bytes<BNV, STV>(), s>>>(              \
        mapD, mapX, P.n3, ktiles, mbk, P.tc_maxslots, P.d_part, P.d_counters, err, e)
    if (bn == 16) {
        if (two) TC_LAUNCH(16, S16_2);
        else TC_LAUNCH(16, S16_1);
    } else {
        if (two) TC_LAUNCH(32, S32_2);
        else TC_LAUNCH(32, S32_1);
    }
#undef TC_LAUNCH
    count_launches(1);
    if (e.mode == 1) prod_mark(P, 1, s);
    return check_launch("tc_gemm");
}

bd_status tc_apply(Plan &P, const void *D16, const double *X, int m, double *Y, cudaStream_t s)
{
    const int bn = m <= 16 ? 16 : 32;
    void *X16 = x16_buf(P, 0);
    prepare_operand(P, X, m, bn, X16, s);
    tc::Epi e{};
    e.mode = 0;
    e.m = m;
    e.Y = Y;
    e.lan_col = -1;
    e.inv_scale = P.d_xscale + kMaxRhs;
    e.is_bf16 = P.p.precision == BD_MIXED_BF16;
    return launch_tc(P, D16, X16, bn, e, s);
}

// Autotuner of the product's launch shape: time Y = D16 X with the column
// count of a lagged Chebyshev product (max_rhs + 1, the Lanczos vector riding
// along) with 2 resident CTAs per SM (shallower ring), 1 (ring twice as
// deep), the symmetric product over the upper triangle (shape 3) and, for
// plans with max_rhs <= 4, the row-streamed CUDA-core product (shape 5), on
// this plan's own matrix, and keep the fastest.  Synchronous.
bd_status tc_autotune(Plan &P, const void *D16, cudaStream_t s, int *best_out, float *ms_out)
{
    const int m = P.p.max_rhs + 1 < kMaxRhs ? P.p.max_rhs + 1 : kMaxRhs;
    double *X = P.d_X0, *Y = P.d_Y0;
    cudaMemsetAsync(X, 0, sizeof(double) * (size_t)P.n3 * m, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 1e30f;
    const int saved = P.tc_split;
    const bool rows_ok = P.p.max_rhs + 4 <= kRowsMaxCols;
    for (int cps = 1; cps <= kRowsShape; cps++) {
        if (cps == kF64DoubleFloat || (cps == kRowsShape && !rows_ok)) continue;
        P.tc_split = cps;
        auto product = [&]() {
            return cps == kRowsShape ? rows_apply(P, D16, X, m, Y, s) : tc_apply(P, D16, X, m, Y, s);
        };
        bd_status st = product();                          // warm-up
        if (st != BD_OK) { P.tc_split = saved; cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; r++) product();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = cps; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P.tc_split = best;
    if (best_out) *best_out = best;
    if (ms_out) *ms_out = best_ms / 3.f;
    return check_launch("tc_autotune");
}

// Lanczos vector as an extra operand column: fixed scale 64 (|q_i| <= 1 for a
// unit vector, so the 16-bit copy cannot overflow)
constexpr float kLanScale = 64.f;

__global__ void k_lan_column(const double *q, int n3, float *scale, float *inv_scale, void *X16col,
                             int is_bf16)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *scale = kLanScale;
        *inv_scale = 1.f / kLanScale;
    }
    if (i >= n3) return;
    float v = (float)(q[i] * (double)kLanScale);
    if (is_bf16) ((__nv_bfloat16 *)X16col)[i] = __float2bfloat16_rn(v);
    else ((__half *)X16col)[i] = __float2half_rn(v);
}

// One Lanczos step after a product that carried q_j: from the row-block
// partials of q_j.w, q_{j-1}.w and w.w (every block sums them in the same
// order, so all blocks agree bit for bit)
//   alpha_j = q_j.w,  |w'|^2 = w.w - alpha_j^2 - 2 beta_{j-1} (q_{j-1}.w) + beta_{j-1}^2,
//   w' = w - alpha_j q_j - beta_{j-1} q_{j-1},  beta_j = |w'|,  q_{j+1} = w' / beta_j
// (the expansion takes q_j, q_{j-1} orthonormal), then q_{j-1} <- q_j,
// q_j <- q_{j+1} and the 16-bit copy of q_{j+1} into the next operand.
__global__ void k_lanczos_step(double *qprev, double *q, const double *w, int n3,
                               const double *part, int nparts, double *lab, int j, void *X16col,
                               int is_bf16)
{
    // a programmatic dependent of the product's last kernel (see tc_cheb)
    tc::grid_dep_launch();
    tc::grid_dep_wait();
    __shared__ double sh[3];
    if (threadIdx.x < 32) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int i = threadIdx.x; i < nparts; i += 32)
            for (int k = 0; k < 3; k++) t[k] += part[3 * i + k];
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; k++) sh[k] = t[k];
    }
    __syncthreads();
    const double alpha = sh[0];
    const double bprev = j > 0 ? lab[kMaxLanczos + j - 1] : 0.0;
    const double n2 = sh[2] - alpha * alpha - 2.0 * bprev * sh[1] + bprev * bprev;
    const double beta = n2 > 0.0 ? sqrt(n2) : 0.0;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        lab[j] = alpha;
        lab[kMaxLanczos + j] = beta;
    }
    if (i >= n3) return;
    // one reciprocal, not a division per element (FP64 divisions run on this
    // GPU's slow FP64 pipe)
    const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
    double x = w[i] - alpha * q[i] - bprev * qprev[i];
    double qn = x * ib;
    qprev[i] = q[i];
    q[i] = qn;
    float v = (float)qn * kLanScale;
    if (is_bf16) ((__nv_bfloat16 *)X16col)[i] = __float2bfloat16_rn(v);
    else ((__half *)X16col)[i] = __float2half_rn(v);
}

bd_status tc_cheb(Plan &P, const void *D16, int m, const double *coef, const double *bounds, int p,
                  double *Vprev2, const double *Vprev1, double *dS, cudaStream_t s, int lan_step)
{
    const bool lan = lan_step >= 0;
    const int cols = m + (lan ? 1 : 0);
    const int bn = cols <= 16 ? 16 : 32;
    const int is_bf16 = P.p.precision == BD_MIXED_BF16;
    // operand of V_{p-1}: buffer (p & 1); the epilogue writes V_p into the other
    void *cur = x16_buf(P, p & 1), *nxt = x16_buf(P, (p + 1) & 1);
    if (p == 2) {
        // scales from V_1's block (kept for the whole recurrence); 16-bit V_1
        prepare_operand(P, Vprev1, m, bn, cur, s);
        if (lan) {
            k_lan_column<<<(P.n3 + 255) / 256, 256, 0, s>>>(
                P.d_lq[1], P.n3, P.d_xscale + m, P.d_xscale + kMaxRhs + m,
                (char *)cur + (size_t)m * P.ldx * 2, is_bf16);
            count_launches(1);
        }
    }
    tc::Epi e{};
    e.mode = 1;
    e.m = m;
    e.inv_scale = P.d_xscale + kMaxRhs;
    e.scale = P.d_xscale;
    e.coef = coef;
    e.bounds = bounds;
    e.p = p;
    e.Vprev2 = Vprev2;
    e.Vprev1 = Vprev1;
    e.dS = dS;
    e.X16next = nxt;
    e.ldx = P.ldx;
    e.is_bf16 = is_bf16;
    e.lan_col = lan ? m : -1;
    e.lan_w = P.d_lq[2];
    e.lan_q = P.d_lq[1];
    e.lan_qp = P.d_lq[0];
    e.lan_part = P.d_lanpart;
    bd_status st = launch_tc(P, D16, cur, bn, e, s);
    if (st != BD_OK || !lan) return st;
    // launched as a programmatic dependent: scheduled while the product
    // finishes, it reads the product's outputs after its dependency wait, and
    // the next product may in turn be scheduled while it runs
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cl = {};
    cl.gridDim = dim3((P.n3 + 255) / 256);
    cl.blockDim = dim3(256);
    cl.stream = s;
    cl.attrs = attr;
    cl.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cl, k_lanczos_step, P.d_lq[0], P.d_lq[1],
                                              (const double *)P.d_lq[2], P.n3,
                                              (const double *)P.d_lanpart, mblocks(P), P.d_lab,
                                              lan_step, (void *)((char *)nxt + (size_t)m * P.ldx * 2),
                                              is_bf16);
    count_launches(1);
    if (le != cudaSuccess)
        return set_error(BD_ERR_CUDA, "lanczos step launch: %s", cudaGetErrorString(le));
    return check_launch("lanczos step");
}

// One FP64-residual refinement step y += (D32 x - y) for one column.  The
// FP32 matrix times x is accumulated exactly enough without the FP64 pipe
// (1/60 of FP32 on this GPU): x is split once into FP32 words x = xh + xl,
// each lane forms d*xh exactly as the pair (p, fma(d, xh, -p)) and keeps a
// double-float running sum (TwoSum), and only the 32 lane totals of a row
// are combined in FP64.  Accuracy of the residual ~1e-12 of sum |d x|; the
// kernel streams D32 once (HBM bound).
__global__ void k_split_x(const double *x, int n3, float *xs)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    double v = x[i];
    float h = (float)v;
    xs[i] = h;
    xs[n3 + i] = (float)(v - (double)h);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__global__ void __launch_bounds__(256)
k_refine(const float *__restrict__ D32, long ld, int n3, const float *__restrict__ xs,
         double *__restrict__ y)
{
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n3) return;
    const float *d = D32 + (long)row * ld;
    const float *xh = xs, *xl = xs + n3;
    float s = 0.f, c = 0.f;
    auto term = [&](float dq, float h, float l) {
        float p = dq * h;
        float pe = fmaf(dq, h, -p);
        pe = fmaf(dq, l, pe);
        float t, e;
        two_sum(s, p, t, e);
        s = t;
        c += e + pe;
    };
    // rows start 256-byte aligned (ld multiple of 64) and n3 is a multiple of
    // 3; x is split in two arrays of n3 floats, read as float4 where n3 % 4 == 0
    int k = lane * 4;
    if ((n3 & 3) == 0) {
        const float4 *xh4 = (const float4 *)xh, *xl4 = (const float4 *)xl;
        // two float4 of D per lane in flight
        for (; k + 128 + 3 < n3; k += 256) {
            float4 d0 = __ldcs((const float4 *)(d + k)), d1 = __ldcs((const float4 *)(d + k + 128));
            float4 h0 = __ldg(xh4 + (k >> 2)), l0 = __ldg(xl4 + (k >> 2));
            float4 h1 = __ldg(xh4 + ((k + 128) >> 2)), l1 = __ldg(xl4 + ((k + 128) >> 2));
            term(d0.x, h0.x, l0.x); term(d0.y, h0.y, l0.y); term(d0.z, h0.z, l0.z); term(d0.w, h0.w, l0.w);
            term(d1.x, h1.x, l1.x); term(d1.y, h1.y, l1.y); term(d1.z, h1.z, l1.z); term(d1.w, h1.w, l1.w);
        }
        for (; k + 3 < n3; k += 128) {
            float4 d0 = __ldcs((const float4 *)(d + k));
            float4 h0 = __ldg(xh4 + (k >> 2)), l0 = __ldg(xl4 + (k >> 2));
            term(d0.x, h0.x, l0.x); term(d0.y, h0.y, l0.y); term(d0.z, h0.z, l0.z); term(d0.w, h0.w, l0.w);
        }
    } else {
        for (; k + 3 < n3; k += 128) {
            float4 dv = __ldcs((const float4 *)(d + k));
            term(dv.x, __ldg(xh + k), __ldg(xl + k));
            term(dv.y, __ldg(xh + k + 1), __ldg(xl + k + 1));
            term(dv.z, __ldg(xh + k + 2), __ldg(xl + k + 2));
            term(dv.w, __ldg(xh + k + 3), __ldg(xl + k + 3));
        }
    }
    for (; k < n3; k++) term(d[k], xh[k], xl[k]);   // tail (at most 3 elements per lane)
    double acc = (double)s + (double)c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        double y0 = y[row];
        double r = acc - y0;
        y[row] = y0 + r;
    }
}

void launch_refine_f32(Plan &P, const float *D32, const double *X, int m, double *Y,
                       cudaStream_t s)
{
    long threads = (long)P.n3 * 32;
    if (P.tc_split == kSymShape) {
        // the symmetric shape's D holds the tiles on and above the diagonal only
        for (int j = 0; j < m; j++) {
            k_split_x<<<(P.n3 + 255) / 256, 256, 0, s>>>(X + (long)j * P.n3, P.n3, P.d_xsplit);
            count_launches(1);
            sym_refine(P, D32, P.d_xsplit, Y + (long)j * P.n3, s);
        }
        return;
    }
    for (int j = 0; j < m; j++) {
        k_split_x<<<(P.n3 + 255) / 256, 256, 0, s>>>(X + (long)j * P.n3, P.n3, P.d_xsplit);
        count_launches(1);
        k_refine<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(D32, P.ld, P.n3, P.d_xsplit,
                                                                   Y + (long)j * P.n3);
        count_launches(1);
    }
}

}  // namespace bd
