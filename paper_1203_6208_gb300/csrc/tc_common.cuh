// tc_common.cuh -- building blocks of the tensor-core (tcgen05) products:
// mbarrier waits with bounded spins, TMA tile loads, shared-memory and
// instruction descriptors, TMEM loads, and the epilogue arguments.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "bd_internal.cuh"

namespace bd {

namespace tc {

constexpr int BM = 128;          // rows of D per CTA (TMEM lanes)
constexpr int BK = 64;           // K elements per stage (128 bytes of 16-bit)
// ring depth: as many stages as fit the CTA's share of shared memory (two
// CTAs per SM, or one CTA per SM with a ring twice as deep); a stage is
// released only when its MMAs have completed, so the bytes in flight per SM,
// not the MMA rate, set the streaming rate
template <int BN> constexpr int stages_for(int ctas_per_sm)
{
    return (ctas_per_sm == 1 ? 224 * 1024 : 110 * 1024) / (BM * BK * 2 + BN * BK * 2);
}
constexpr int THREADS = 192;     // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int A_BYTES = BM * BK * 2;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kMaxCtasPerSm = 2;

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

// bounded wait for roles that wait long (the epilogue waits for a whole
// segment): backs off between polls so the spinning warps do not take issue
// slots from the TMA and MMA threads on the same SM sub-partitions
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity,
                                                volatile int *abort_flag)
{
    for (uint32_t i = 0; i < kWaitLimit; i++) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        __nanosleep(200);
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

// the same with an L2 cache policy (createpolicy): the products stream D once
// per product, so its tiles are loaded evict-first and leave L2 to the
// vectors and partial sums that the next kernel reads back
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap *map, int x,
                                                 int y, uint32_t bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// FP32 <-> FP64 conversions on the integer pipe.  On this GPU the hardware
// conversions issue on the FP64 pipe (1/64 of the FP32 rate), where the
// products' epilogues are short of throughput.  The IEEE binary32 fields are
// moved into the binary64 fields (exponent rebiased by 1023 - 127 = 896):
// exact for every normal FP32 value and for zero; other inputs (subnormal,
// infinite, NaN) take the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xFFu;
    if (ex == 0u && (u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    if (ex == 0u || ex == 0xFFu) return (double)f;
    const unsigned hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// FP64 -> FP32 rounded toward zero (the 29 low fraction bits dropped), for
// values in the normal FP32 range; others take the hardware conversion.  Used
// where the result is rounded again to 16 bits.
__device__ __forceinline__ float f64_to_f32_rz(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned ex = (hi >> 20) & 0x7FFu;
    if (ex < 897u || ex > 1150u) return (float)d;
    return __uint_as_float((hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) |
                           (lo >> 29));
}

// programmatic dependent launch: wait for the grids this one depends on
// (and their memory) before touching their outputs; let the next grid be
// scheduled once every CTA of this one has run this far
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
    int lan_col;                // mode 1: column carrying the Lanczos vector (-1: none)
    double *lan_w;              // its product w = D q_j, FP64
    const double *lan_q, *lan_qp;  // q_j and q_{j-1}
    double *lan_part;           // per row block: q_j.w, q_{j-1}.w, w.w (FP64)
};

}  // namespace tc

}  // namespace bd
