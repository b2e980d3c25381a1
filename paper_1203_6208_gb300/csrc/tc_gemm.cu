// tc_gemm.cu -- mixed-precision products Y = D16 X on the 5th-generation
// tensor cores (tcgen05, sm_103a), and the FP64-residual refinement of D.F.
//
// With m <= 32 right-hand sides the product reads the whole 16-bit copy of D
// once per call at ~m flop per byte, so it is bound by HBM, not by the tensor
// pipe.  The kernel is a TMA -> shared memory -> tcgen05.mma -> TMEM stream:
//   * a CTA owns a 128-row block of D and one K-split; warp 0 issues TMA
//     loads of 128 x 64 tiles of D16 (128-byte swizzle) and 64 x BN tiles of
//     the scaled 16-bit operand X^T into a STAGES-deep ring; warp 1 issues
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

#include "tc_gemm.cuh"

namespace bd {

namespace tc {

constexpr int BM = 128;          // rows of D per CTA (TMEM lanes)
constexpr int BK = 64;           // K elements per stage (128 bytes of 16-bit)
constexpr int STAGES = 5;
constexpr int THREADS = 192;     // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int A_BYTES = BM * BK * 2;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kMaxSplit = 16;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; returns false (and flags the CTA) when the limit is hit or
// another role of the CTA already gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    for (uint32_t i = 0; i < kWaitLimit; i++) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 1023u) == 1023u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1 (tcgen05)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)1 << 16;                            // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                  // SBO
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // SWIZZLE_128B
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, K-major A and B
__host__ __device__ constexpr uint32_t idesc_f16(int bn, int is_bf16)
{
    return (1u << 4)                                   // D format F32
         | ((uint32_t)is_bf16 << 7)                   // A format F16/BF16
         | ((uint32_t)is_bf16 << 10)                  // B format
         | ((uint32_t)(bn >> 3) << 17)                // N >> 3
         | ((uint32_t)(BM >> 4) << 24);               // M >> 4
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

struct Epi {
    int mode;                   // 0: plain store, 1: Chebyshev term
    int m;                      // valid columns
    double *Y;                  // mode 0 output, 3N x m column-major
    const float *inv_scale;     // per-column 1/scale of the 16-bit operand
    const float *scale;         // per-column scale (mode 1, next operand)
    const double *coef, *bounds;
    int p;
    double *Vprev2;             // in V_{p-2}, out V_p
    const double *Vprev1;
    double *dS;
    void *X16next;              // next operand (mode 1), [BN][ldx]
    int ldx;
    int is_bf16;
    int lan_col;                // mode 1: column carrying an extra vector (-1: none)
    double *lan_w;              // its product, FP64
};

// -- kernel begin: k_tc_gemm
template <int BN>
__global__ void __launch_bounds__(THREADS, 2)
k_tc_gemm(const __grid_constant__ CUtensorMap mapD, const __grid_constant__ CUtensorMap mapX,
          int n3, int ktiles, int nsplit, float *__restrict__ part, int32_t *__restrict__ counters,
          int32_t *__restrict__ err, Epi e)
{
    constexpr int B_BYTES = BN * BK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;          // multiple of 1024
    static_assert(STAGE % 1024 == 0, "stage alignment");
    constexpr uint32_t IDESC_F16 = idesc_f16(BN, 0), IDESC_BF16 = idesc_f16(BN, 1);

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accum_bar, drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;
    __shared__ int is_last_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mb = blockIdx.x, split = blockIdx.y;
    const int kt0 = (int)((long)ktiles * split / nsplit);
    const int kt1 = (int)((long)ktiles * (split + 1) / nsplit);
    const int nkt = kt1 - kt0;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; s++) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&accum_bar), 1);
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int issued = 0;
        for (int i = 0; i < nkt; i++) {
            int s = i % STAGES;
            uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, &abort_flag)) break;
            uint32_t a = smem_u32(smem + s * STAGE), b = a + A_BYTES;
            uint32_t fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, STAGE);
            int kx = (kt0 + i) * BK;
            tma_load_2d(a, &mapD, kx, mb * BM, fb);
            tma_load_2d(b, &mapX, kx, 0, fb);
            issued = i + 1;
        }
        if (abort_flag) {
            // let every load issued land before the CTA can exit
            for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; i++) {
                int s = i % STAGES;
                uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                for (uint32_t t = 0; t < kWaitLimit && !mbar_try(smem_u32(&full_bar[s]), ph); t++) {}
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = e.is_bf16 ? IDESC_BF16 : IDESC_F16;
        bool ok = true;
        for (int i = 0; i < nkt && ok; i++) {
            int s = i % STAGES;
            uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(smem_u32(&full_bar[s]), ph, &abort_flag)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t a = smem_u32(smem + s * STAGE), b = a + A_BYTES;
            uint64_t da = sw128_desc(a), db = sw128_desc(b);
#pragma unroll
            for (int k = 0; k < BK / 16; k++) {
                // advance 16 elements (32 bytes) along K inside the swizzled rows
                mma_f16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc,
                        (i > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&empty_bar[s]));
        }
        mma_commit(smem_u32(&accum_bar));
        if (!ok) {
            mma_commit(smem_u32(&drain_bar));
            for (uint32_t t = 0; t < kWaitLimit && !mbar_try(smem_u32(&drain_bar), 0); t++) {}
        }
    } else if (warp >= 2) {
        // ---- epilogue: TMEM -> FP32 partial
        const int q = warp & 3;                      // TMEM lane quadrant of this warp
        const int r = q * 32 + lane;                 // row within the block
        const long row = (long)mb * BM + r;
        float acc[BN];
        bool ok = (nkt == 0) || mbar_wait(smem_u32(&accum_bar), 0, &abort_flag);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok && nkt > 0) {
#pragma unroll
            for (int c = 0; c < BN; c += 16) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + c, acc + c);
        } else {
#pragma unroll
            for (int c = 0; c < BN; c++) acc[c] = 0.f;
        }
        float4 *dst = (float4 *)(part + ((size_t)split * gridDim.x * BM + (size_t)mb * BM + r) * BN);
#pragma unroll
        for (int c = 0; c < BN / 4; c++)
            dst[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
        __threadfence();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (threadIdx.x == 64) {
            int old = atomicAdd(&counters[mb], 1);
            is_last_sh = (old == nsplit - 1);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (is_last_sh) {
            __threadfence();
            double y[BN];
#pragma unroll
            for (int c = 0; c < BN; c++) y[c] = 0.0;
            for (int sp = 0; sp < nsplit; sp++) {
                const float4 *src =
                    (const float4 *)(part + ((size_t)sp * gridDim.x * BM + (size_t)mb * BM + r) * BN);
#pragma unroll
                for (int c = 0; c < BN / 4; c++) {
                    float4 v = __ldcg(src + c);
                    y[4 * c] += v.x; y[4 * c + 1] += v.y; y[4 * c + 2] += v.z; y[4 * c + 3] += v.w;
                }
            }
            if (row < n3) {
                if (e.mode == 0) {
#pragma unroll
                    for (int c = 0; c < BN; c++)
                        if (c < e.m) e.Y[(long)c * n3 + row] = y[c] * (double)e.inv_scale[c];
                } else {
                    const double dmin = e.bounds[0], dmax = e.bounds[1];
                    const double ys = 2.0 / (dmax - dmin), yt = (dmax + dmin) / (dmax - dmin);
                    const double cp = e.coef[e.p];
#pragma unroll
                    for (int c = 0; c < BN; c++) {
                        if (c == e.lan_col) e.lan_w[row] = y[c] * (double)e.inv_scale[c];
                        if (c < e.m) {
                            long o = (long)c * n3 + row;
                            double w = y[c] * (double)e.inv_scale[c];
                            double v = 2.0 * (ys * w - yt * e.Vprev1[o]) - e.Vprev2[o];
                            e.Vprev2[o] = v;
                            e.dS[o] += cp * v;
                            float sv = (float)(v * (double)e.scale[c]);
                            size_t xo = (size_t)c * e.ldx + row;
                            if (e.is_bf16) ((__nv_bfloat16 *)e.X16next)[xo] = __float2bfloat16_rn(sv);
                            else ((__half *)e.X16next)[xo] = __float2half_rn(sv);
                        }
                    }
                }
            }
        }
    }
    // ---- teardown
    if (threadIdx.x == 0 && abort_flag) atomicExch(err, (int32_t)BD_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32)
                     : "memory");
    }
}

// -- kernel end: k_tc_gemm

template <int BN>
constexpr int smem_bytes()
{
    return STAGES * (A_BYTES + BN * BK * 2) + 1024;
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

static int mblocks(const Plan &P) { return (P.n3 + tc::BM - 1) / tc::BM; }

bd_status tc_plan_init(Plan &P)
{
    bd_status st = get_encoder();
    if (st != BD_OK) return st;
    P.ldx = (P.n3 + kLdAlign - 1) / kLdAlign * kLdAlign;
    size_t x16 = (size_t)2 * kMaxRhs * P.ldx * 2;               // two operand buffers
    size_t mbk = (size_t)mblocks(P);
    cudaError_t e = cudaMalloc(&P.d_x16, x16);
    if (e == cudaSuccess) e = cudaMalloc(&P.d_xscale, 4 * kMaxRhs * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&P.d_part, (size_t)tc::kMaxSplit * mbk * tc::BM * kMaxRhs * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_counters, (mbk + 64) * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BD_ERR_OOM, "mixed-precision scratch: %s", cudaGetErrorString(e));
    }
    P.scratch_bytes += (int64_t)(x16 + 4 * kMaxRhs * sizeof(float) +
                                 (size_t)tc::kMaxSplit * mbk * tc::BM * kMaxRhs * sizeof(float) +
                                 (mbk + 64) * sizeof(int32_t));
    cudaMemset(P.d_x16, 0, x16);
    for (int bn : {16, 32}) {
        int sm = bn == 16 ? tc::smem_bytes<16>() : tc::smem_bytes<32>();
        cudaError_t a = bn == 16
            ? cudaFuncSetAttribute(tc::k_tc_gemm<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
            : cudaFuncSetAttribute(tc::k_tc_gemm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (a != cudaSuccess) return set_error(BD_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(a));
    }
    return BD_OK;
}

static void *x16_buf(Plan &P, int which)
{
    return (char *)P.d_x16 + (size_t)which * kMaxRhs * P.ldx * 2;
}

static int n_split(const Plan &P, int ktiles)
{
    // enough CTAs for ~5 waves of two CTAs per SM on 152 SMs, unless the
    // autotuner measured a better split for this plan
    int mbk = mblocks(P);
    int s = P.tc_split > 0 ? P.tc_split : (5 * 2 * 152 + mbk - 1) / mbk;
    if (s > tc::kMaxSplit) s = tc::kMaxSplit;
    if (s > ktiles) s = ktiles;
    return s < 1 ? 1 : s;
}

// column scales of X (rows 0..m-1 of the (m, 3N) block) and the 16-bit copy
static void prepare_operand(Plan &P, const double *X, int m, int bn, void *X16, cudaStream_t s)
{
    unsigned long long *bits = (unsigned long long *)(P.d_xscale + 2 * kMaxRhs);
    cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * kMaxRhs, s);
    k_col_absmax<<<dim3(64, m), 256, 0, s>>>(X, P.n3, m, bits);
    count_launches(1);
    k_col_scale<<<1, 32, 0, s>>>(bits, m, bn, P.d_xscale, P.d_xscale + kMaxRhs);
    count_launches(1);
    k_to16<<<dim3((P.n3 + 255) / 256, bn), 256, 0, s>>>(X, P.n3, m, bn, P.d_xscale, X16, P.ldx,
                                                       P.p.precision == BD_MIXED_BF16);
    count_launches(1);
}

// one extra column: scale from its own max and the 16-bit copy in row `col`
__global__ void k_scale_one(const unsigned long long *bits, float *scale, float *inv_scale)
{
    float sc = 1.f;
    double mx = __longlong_as_double((long long)*bits);
    if (mx > 0.0 && isfinite(mx)) {
        int e;
        frexp(mx, &e);
        sc = ldexpf(1.f, -e);
    }
    *scale = sc;
    *inv_scale = 1.f / sc;
}

static void prepare_column(Plan &P, const double *x, int col, void *X16, cudaStream_t s)
{
    unsigned long long *bits = (unsigned long long *)(P.d_xscale + 2 * kMaxRhs) + col;
    cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s);
    k_col_absmax<<<dim3(64, 1), 256, 0, s>>>(x, P.n3, 1, bits);
    count_launches(1);
    k_scale_one<<<1, 1, 0, s>>>(bits, P.d_xscale + col, P.d_xscale + kMaxRhs + col);
    count_launches(1);
    // k_to16 converts column 0 of x into row 0 of the buffer it is given: offset
    // the destination to row `col` and the scale to entry `col`
    k_to16<<<dim3((P.n3 + 255) / 256, 1), 256, 0, s>>>(
        x, P.n3, 1, 1, P.d_xscale + col, (char *)X16 + (size_t)col * P.ldx * 2, P.ldx,
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
    int ktiles = (P.n3 + tc::BK - 1) / tc::BK;
    int ns = n_split(P, ktiles);
    dim3 grid(mblocks(P), ns);
    cudaMemsetAsync(P.d_counters, 0, sizeof(int32_t) * mblocks(P), s);
    int32_t *err = P.d_status + 6;
    if (e.mode == 1) prod_mark(P, 0, s);
    if (bn == 16)
        tc::k_tc_gemm<16><<<grid, tc::THREADS, tc::smem_bytes<16>(), s>>>(
            mapD, mapX, P.n3, ktiles, ns, P.d_part, P.d_counters, err, e);
    else
        tc::k_tc_gemm<32><<<grid, tc::THREADS, tc::smem_bytes<32>(), s>>>(
            mapD, mapX, P.n3, ktiles, ns, P.d_part, P.d_counters, err, e);
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

// Autotuner of the product's tile decomposition: time Y = D16 X (m = the
// plan's max_rhs, up to 16 columns) for K-split counts 1, 2, 4, 8, 16 on this
// plan's own matrix and keep the fastest.  Synchronous.
bd_status tc_autotune(Plan &P, const void *D16, cudaStream_t s, int *best_out, float *ms_out)
{
    const int m = P.p.max_rhs < 16 ? P.p.max_rhs : 16;
    double *X = P.d_V[0], *Y = P.d_V[1];
    cudaMemsetAsync(X, 0, sizeof(double) * (size_t)P.n3 * m, s);
    const int ktiles = (P.n3 + tc::BK - 1) / tc::BK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 1e30f;
    const int saved = P.tc_split;
    for (int sp : {1, 2, 4, 8, 16}) {
        if (sp > ktiles) break;
        P.tc_split = sp;
        bd_status st = tc_apply(P, D16, X, m, Y, s);      // warm-up
        if (st != BD_OK) { P.tc_split = saved; cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; r++) tc_apply(P, D16, X, m, Y, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = sp; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P.tc_split = best;
    if (best_out) *best_out = best;
    if (ms_out) *ms_out = best_ms / 3.f;
    return check_launch("tc_autotune");
}

bd_status tc_cheb(Plan &P, const void *D16, int m, const double *coef, const double *bounds, int p,
                  double *Vprev2, const double *Vprev1, double *dS, cudaStream_t s,
                  const double *lan_q, double *lan_w)
{
    const int cols = m + (lan_q ? 1 : 0);
    const int bn = cols <= 16 ? 16 : 32;
    // operand of V_{p-1}: buffer (p & 1); the epilogue writes V_p into the other
    void *cur = x16_buf(P, p & 1), *nxt = x16_buf(P, (p + 1) & 1);
    if (p == 2) {
        // scales from V_1's block (kept for the whole recurrence); 16-bit V_1
        prepare_operand(P, Vprev1, m, bn, cur, s);
    }
    if (lan_q) prepare_column(P, lan_q, m, cur, s);
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
    e.is_bf16 = P.p.precision == BD_MIXED_BF16;
    e.lan_col = lan_q ? m : -1;
    e.lan_w = lan_w;
    return launch_tc(P, D16, cur, bn, e, s);
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
    // n3 is a multiple of 3, rows start 256-byte aligned (ld multiple of 64)
    int k = lane * 4;
    for (; k + 3 < n3; k += 128) {
        float4 dv = __ldg((const float4 *)(d + k));
        float dd[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float h = __ldg(xh + k + q), l = __ldg(xl + k + q);
            float p = dd[q] * h;
            float pe = fmaf(dd[q], h, -p);
            pe = fmaf(dd[q], l, pe);
            float t, e;
            two_sum(s, p, t, e);
            s = t;
            c += e + pe;
        }
    }
    for (; k < n3; k++) {             // tail (at most 3 elements per lane)
        float p = d[k] * xh[k];
        float pe = fmaf(d[k], xh[k], -p);
        pe = fmaf(d[k], xl[k], pe);
        float t, e;
        two_sum(s, p, t, e);
        s = t;
        c += e + pe;
    }
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
    for (int j = 0; j < m; j++) {
        k_split_x<<<(P.n3 + 255) / 256, 256, 0, s>>>(X + (long)j * P.n3, P.n3, P.d_xsplit);
        count_launches(1);
        k_refine<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(D32, P.ld, P.n3, P.d_xsplit,
                                                                   Y + (long)j * P.n3);
        count_launches(1);
    }
}

}  // namespace bd
