// recip_tc.cu -- the reciprocal part of D (Eq. DF, Eq. M2) for the mixed
// (FP32) assembly as a tensor-core product.
//
// The folded tensor of a half-space vector k is 2 f(k) (I - khat khat) =
// 2 f(k) (u1 u1^T + u2 u2^T) with u1, u2 orthonormal and perpendicular to k,
// so with cos(k.(r_nu - r_mu)) = c_nu c_mu + s_nu s_mu the whole reciprocal sum
// is one symmetric product D_rec = U U^T,
//   U[3 nu + a][4 t + 2 (c-1) + s] = sqrt(2 f_t) u_c^a(k_t) {cos, sin}(k_t . r_nu),
// a rank-4 N_k contraction over all bead pairs -- dense work for the tensor
// cores.  U is split into two words U = Uh + Ul of 11 significant bits each
// (Uh the TF32 rounding of U, Ul that of the remainder), stored as IEEE half
// scaled by 2^8 (both words are exact in half over the range of U, which is
// below 1; words under 2^-14 / 2^8 lose bits as subnormals, an absolute error
// ~1e-10), and D_rec = Uh Uh^T + Uh Ul^T + Ul Uh^T is accumulated in FP32 in
// TMEM (kind::f16, M = 128, N = 256, K = 16 per MMA -- twice the TF32 rate) and
// scaled by 2^-16 on the way out: about 2^-21 relative per term, below the
// FP32 assembly's own rounding.  The product fills the 128 x 256 blocks of
// D32 that reach the diagonal (128 x 128 tiles on and above it); the pair kernel reads the
// six components (a <= b) of each 3 x 3 block it owns there (always row <=
// column), adds the real-space, self and overlap terms and writes the final
// D32 / D16 over them.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "recip_tc.cuh"

namespace bd {

namespace rt {

constexpr int BM = 128, BN = 256, BK = 64;     // BK in half elements (128 bytes)
constexpr int STAGES = 4;
// largest padded k width K_p (4 columns per half-space k) of the tensor-core path
constexpr int kRecipTcMaxKp = 1024;
constexpr int THREADS = 192;
constexpr int A_BYTES = BM * BK * 2;           // 16 KB: 128 rows of U
constexpr int B_BYTES = BN * BK * 2;           // 32 KB: 256 rows of U
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 2 * BN;         // two accumulators
constexpr float kUScale = 256.f;               // U words stored as half(U 2^8)
constexpr float kDUnscale = 1.f / (256.f * 256.f);
constexpr uint32_t kWaitLimit = 1u << 22;

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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    for (uint32_t i = 0; i < kWaitLimit; i++) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 1023u) == 1023u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}
// long waits (the epilogue waits for the whole K loop) back off between polls
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
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// kind::f16: F32 accumulator, F16 A and B, K-major, M = 128, N = 256
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
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

// -- kernel begin: k_recip_syrk
// Persistent: CTA c takes the blocks c, c + G, c + 2G, ... of the block list
// (128 rows ti x 256 columns tj2, the column block reaching the diagonal).
// Per block the K loop runs over three segments (Uh.Uh, Uh.Ul, Ul.Uh) of nkt
// k-tiles each into one of two TMEM accumulators, so the epilogue warps drain
// one block while the MMA warp fills the next.
__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
k_recip_syrk(const __grid_constant__ CUtensorMap mapH, const __grid_constant__ CUtensorMap mapL,
             const __grid_constant__ CUtensorMap mapHB, const __grid_constant__ CUtensorMap mapLB,
             const int2 *__restrict__ blocks, int nblocks, int n3, int nkt, float *__restrict__ D32,
             long ld, int32_t *__restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_full[2], acc_empty[2],
        drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x, G = gridDim.x;
    const int nsteps = 3 * nkt;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int st = 0; st < STAGES; st++) {
            mbar_init(smem_u32(&full_bar[st]), 1);
            mbar_init(smem_u32(&empty_bar[st]), 1);
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
        // ---- TMA producer
        int it = 0;
        for (int bi = c; bi < nblocks && !abort_flag; bi += G) {
            const int2 t2 = blocks[bi];
            for (int i = 0; i < nsteps; i++, it++) {
                const int st = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1u, &abort_flag)) break;
                const int seg = i / nkt, kk = i % nkt;
                const CUtensorMap *ma = seg == 2 ? &mapL : &mapH;     // Ul.Uh in segment 2
                const CUtensorMap *mb = seg == 1 ? &mapLB : &mapHB;   // Uh.Ul in segment 1
                const uint32_t a = smem_u32(smem + st * STAGE_BYTES), b = a + A_BYTES;
                const uint32_t fb = smem_u32(&full_bar[st]);
                mbar_expect_tx(fb, STAGE_BYTES);
                tma_load_2d(a, ma, kk * BK, t2.x * BM, fb);
                tma_load_2d(b, mb, kk * BK, t2.y * BN, fb);
                issued = it + 1;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: block k accumulates in TMEM buffer k & 1
        bool ok = true;
        int it = 0, k = 0;
        for (int bi = c; bi < nblocks && ok; bi += G, k++) {
            const int buf = k & 1;
            if (k >= 2 &&
                !mbar_wait(smem_u32(&acc_empty[buf]), (uint32_t)((k >> 1) - 1) & 1u, &abort_flag)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(buf * BN);
            for (int i = 0; i < nsteps; i++, it++) {
                const int st = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(smem_u32(&full_bar[st]), ph, &abort_flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a = smem_u32(smem + st * STAGE_BYTES), b = a + A_BYTES;
                const uint64_t da = sw128_desc(a), db = sw128_desc(b);
#pragma unroll
                for (int kq = 0; kq < BK / 16; kq++)      // 16 halves = 32 bytes per MMA along K
                    mma_f16(acc, da + (uint64_t)(2 * kq), db + (uint64_t)(2 * kq),
                            (i > 0 || kq > 0) ? 1u : 0u);
                mma_commit(smem_u32(&empty_bar[st]));
            }
            if (ok) mma_commit(smem_u32(&acc_full[buf]));
        }
        if (!ok) {
            mma_commit(smem_u32(&drain_bar));
            for (uint32_t t = 0; t < kWaitLimit && !mbar_try(smem_u32(&drain_bar), 0); t++) {}
        }
    } else if (warp >= 2) {
        // ---- epilogue warps: TMEM lane quadrant q, row r of the block
        const int q = warp & 3;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        int k = 0;
        for (int bi = c; bi < nblocks; bi += G, k++) {
            const int buf = k & 1;
            if (!mbar_wait_sleep(smem_u32(&acc_full[buf]), (uint32_t)(k >> 1) & 1u, &abort_flag))
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int2 t2 = blocks[bi];
            const long row = (long)t2.x * BM + q * 32 + lane;
            // the first 128 columns lie below the diagonal when 2 tj2 < ti
            const int cstart = (2 * t2.y < t2.x) ? BM : 0;
            for (int c0 = cstart; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + lane_off + (uint32_t)(buf * BN + c0), v);
#pragma unroll
                for (int cc = 0; cc < 16; cc++) v[cc] *= kDUnscale;     // undo the 2^8 word scales
                const long col = (long)t2.y * BN + c0;
                if (row < n3) {
                    float *dst = D32 + row * ld + col;
                    if (col + 16 <= n3) {
#pragma unroll
                        for (int cc = 0; cc < 16; cc += 4)
                            *(float4 *)(dst + cc) = make_float4(v[cc], v[cc + 1], v[cc + 2], v[cc + 3]);
                    } else {
                        for (int cc = 0; cc < 16; cc++)
                            if (col + cc < n3) dst[cc] = v[cc];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive_cta(smem_u32(&acc_empty[buf]));
        }
    }
    // teardown: abort_flag is final once every thread is here; after an abort
    // the producer lets every load it issued land before the CTA exits
    __syncthreads();
    if (abort_flag) {
        if (warp == 0 && lane == 0)
            for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; i++) {
                const int st = i % STAGES;
                const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                for (uint32_t t = 0; t < kWaitLimit && !mbar_try(smem_u32(&full_bar[st]), ph); t++) {}
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
// -- kernel end: k_recip_syrk

}  // namespace rt

// U = Uh + Ul for one bead and one half-space k: the columns (c, s) of Eq. DF
// written as a product; u1, u2 from the k vector (FP64).  Uh is U rounded to
// 11 significant bits (TF32 rounding, cvt.rna) and Ul the same rounding of
// U - Uh; both are stored as half(word 2^8), exact in the normal range.
__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// per half-space k: w u1 and w u2 (w = sqrt(2 f), u1, u2 orthonormal and
// perpendicular to k), computed once per plan in FP64 and kept in FP32:
// basis[8 t + a] = w u1_a, basis[8 t + 3 + a] = w u2_a
__global__ void k_kbasis(const KVec *__restrict__ kv, int nk, float *__restrict__ basis)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nk) return;
    const KVec &K = kv[t];
    double k2 = K.k[0] * K.k[0] + K.k[1] * K.k[1] + K.k[2] * K.k[2];
    double kn = sqrt(k2);
    double kh[3] = {K.k[0] / kn, K.k[1] / kn, K.k[2] / kn};
    // 2f = trace(m)/2, m = 2 f (I - khat khat)
    double twof = 0.5 * (K.m[0] + K.m[3] + K.m[5]);
    double w = sqrt(twof > 0.0 ? twof : 0.0);
    // u1 = normalise(e x khat) with e the axis least aligned with khat; u2 = khat x u1
    int ax = fabs(kh[0]) <= fabs(kh[1]) ? (fabs(kh[0]) <= fabs(kh[2]) ? 0 : 2)
                                        : (fabs(kh[1]) <= fabs(kh[2]) ? 1 : 2);
    double e[3] = {0, 0, 0};
    e[ax] = 1.0;
    double u1[3] = {e[1] * kh[2] - e[2] * kh[1], e[2] * kh[0] - e[0] * kh[2], e[0] * kh[1] - e[1] * kh[0]};
    double n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    for (int i = 0; i < 3; i++) u1[i] /= n1;
    double u2[3] = {kh[1] * u1[2] - kh[2] * u1[1], kh[2] * u1[0] - kh[0] * u1[2], kh[0] * u1[1] - kh[1] * u1[0]};
    for (int i = 0; i < 3; i++) {
        basis[8 * t + i] = (float)(w * u1[i]);
        basis[8 * t + 3 + i] = (float)(w * u2[i]);
    }
    basis[8 * t + 6] = 0.f;
    basis[8 * t + 7] = 0.f;
}

// U rows of one bead for one k group (4 columns): all FP32 -- the split keeps
// 22 bits of U, within FP32's 24
__device__ __forceinline__ uint2 pack4(float a, float b, float c, float d)
{
    __half2 x = __floats2half2_rn(a * rt::kUScale, b * rt::kUScale);
    __half2 y = __floats2half2_rn(c * rt::kUScale, d * rt::kUScale);
    return make_uint2(*(uint32_t *)&x, *(uint32_t *)&y);
}

// One CTA per kUBeads beads: their cos/sin values for a chunk of kUChunk k
// groups are staged in shared memory (bead-major), then the CTA writes that
// chunk of its 3 kUBeads rows of Uh and Ul with consecutive threads on
// consecutive k groups, so that each warp stores 256 contiguous bytes of a row
// (a thread per (bead, k group) would scatter 8-byte stores 6 Kp bytes apart).
constexpr int kUBeads = 8;
constexpr int kUThreads = 256;
constexpr int kUChunk = 128;

__global__ void __launch_bounds__(kUThreads)
k_build_U(const float *__restrict__ cs, const float *__restrict__ sn,
          const float *__restrict__ basis, int n, int nk, int Kp,
          __half *__restrict__ Uh, __half *__restrict__ Ul)
{
    __shared__ float s_c[kUBeads][kUChunk], s_s[kUBeads][kUChunk];
    const int nu0 = blockIdx.x * kUBeads;
    const int nb = min(kUBeads, n - nu0);
    const int ng = Kp / 4;                        // k groups (>= nk, the rest zero)
    for (int t0 = 0; t0 < ng; t0 += kUChunk) {
        const int tn = min(kUChunk, ng - t0);
        __syncthreads();                          // the previous chunk is written
        for (int i = threadIdx.x; i < kUBeads * tn; i += kUThreads) {
            const int tt = i / kUBeads, b = i % kUBeads;     // 8 consecutive beads per k
            const bool in = b < nb && t0 + tt < nk;
            s_c[b][tt] = in ? cs[(size_t)(t0 + tt) * n + nu0 + b] : 0.f;
            s_s[b][tt] = in ? sn[(size_t)(t0 + tt) * n + nu0 + b] : 0.f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * nb * tn; i += kUThreads) {
            const int row = i / tn, tt = i - row * tn, t = t0 + tt;
            const int b = row / 3, a = row - 3 * b;
            const size_t o = (size_t)(3 * (nu0 + b) + a) * Kp + 4 * t;
            if (t >= nk) {
                *(uint2 *)(Uh + o) = make_uint2(0u, 0u);
                *(uint2 *)(Ul + o) = make_uint2(0u, 0u);
                continue;
            }
            const float c = s_c[b][tt], sv = s_s[b][tt];
            const float *bs = basis + 8 * t;
            const float v[4] = {bs[a] * c, bs[a] * sv, bs[3 + a] * c, bs[3 + a] * sv};
            float h[4], l[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                h[j] = to_tf32(v[j]);
                l[j] = to_tf32(v[j] - h[j]);            // exact difference
            }
            *(uint2 *)(Uh + o) = pack4(h[0], h[1], h[2], h[3]);
            *(uint2 *)(Ul + o) = pack4(l[0], l[1], l[2], l[3]);
        }
    }
}

// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;

// blocks of 128 rows x 256 columns reaching the diagonal (column block j2
// covers 128-row tiles 2 j2 and 2 j2 + 1), column-major so that the CTAs
// running together share their column block of U in L2
static int upper_blocks(int T, std::vector<int2> *out)
{
    int cnt = 0;
    const int T2 = (T + 1) / 2;
    for (int j2 = 0; j2 < T2; j2++)
        for (int i = 0; i <= 2 * j2 + 1 && i < T; i++) {
            if (out) out->push_back(make_int2(i, j2));
            cnt++;
        }
    return cnt;
}

bd_status recip_tc_init(Plan &P)
{
    P.recip_tc = 0;
    if (P.p.precision == BD_FP64 || P.nk == 0) return BD_OK;
    // needs f(k) >= 0 on every k (a - a^3 k^2/3 > 0): k_max^2 = (2 pi/L)^2 n2max < 3/a^2
    double kmax2 = (2.0 * 3.14159265358979323846 / P.p.box_L) *
                   (2.0 * 3.14159265358979323846 / P.p.box_L) * P.p.n2max;
    if (!(kmax2 * P.p.a * P.p.a < 3.0)) return BD_OK;
    // The tensor-core accumulator loses up to about half an ulp of the running
    // sum at each of the 3 K_p / 16 MMA steps, always towards zero: on the
    // positive diagonal sums the error grows with K_p (measured, 800 beads:
    // 1.8e-6 of max|D| at K_p = 960, 3.4e-6 at 1856, 9.0e-6 at 3200).  Above
    // K_p = 1024 the per-pair FP32 sum keeps D32 within 2e-6.
    if (4 * P.nk > rt::kRecipTcMaxKp) return BD_OK;
    if (!g_enc) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess || !fn)
            return set_error(BD_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        g_enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    P.recip_kp = (4 * P.nk + rt::BK - 1) / rt::BK * rt::BK;
    const int T = (P.n3 + rt::BM - 1) / rt::BM;
    std::vector<int2> tiles;
    P.recip_ntiles = upper_blocks(T, &tiles);
    size_t ub = (size_t)P.n3 * P.recip_kp * sizeof(__half);
    cudaError_t e = cudaMalloc(&P.d_Uh, ub);
    if (e == cudaSuccess) e = cudaMalloc(&P.d_Ul, ub);
    if (e == cudaSuccess) e = cudaMalloc(&P.d_kbasis, (size_t)8 * P.nk * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&P.d_rtiles, tiles.size() * sizeof(int2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BD_ERR_OOM, "reciprocal product scratch: %s", cudaGetErrorString(e));
    }
    P.scratch_bytes += (int64_t)(2 * ub + tiles.size() * sizeof(int2) + 8 * P.nk * sizeof(float));
    k_kbasis<<<(P.nk + 127) / 128, 128>>>(P.d_kvec, P.nk, P.d_kbasis);
    count_launches(1);
    cudaMemcpy(P.d_rtiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice);
    const int sm = rt::STAGES * rt::STAGE_BYTES + 1024;
    if (cudaFuncSetAttribute(rt::k_recip_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) !=
        cudaSuccess)
        return set_error(BD_ERR_CUDA, "smem attribute (reciprocal product)");
    P.recip_tc = 1;
    return BD_OK;
}

static bd_status map_U(CUtensorMap *m, const __half *base, int Kp, int n3, int rows)
{
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)n3};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {rt::BK, (cuuint32_t)rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half *>(base), dims,
                       strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(BD_ERR_CUDA, "tensor map for U (%d)", (int)r);
    return BD_OK;
}

// D32 (band tiles) = U U^T, after the per-bead trig tables of this R are built
bd_status launch_recip_tc(Plan &P, float *D32, cudaStream_t s)
{
    k_build_U<<<(P.n + kUBeads - 1) / kUBeads, kUThreads, 0, s>>>(
        P.d_cos32, P.d_sin32, P.d_kbasis, P.n, P.nk, P.recip_kp, P.d_Uh, P.d_Ul);
    count_launches(1);
    CUtensorMap mh, ml, mhb, mlb;
    bd_status st = map_U(&mh, P.d_Uh, P.recip_kp, P.n3, rt::BM);
    if (st == BD_OK) st = map_U(&ml, P.d_Ul, P.recip_kp, P.n3, rt::BM);
    if (st == BD_OK) st = map_U(&mhb, P.d_Uh, P.recip_kp, P.n3, rt::BN);
    if (st == BD_OK) st = map_U(&mlb, P.d_Ul, P.recip_kp, P.n3, rt::BN);
    if (st != BD_OK) return st;
    const int sm = rt::STAGES * rt::STAGE_BYTES + 1024;
    int nsm = P.num_sms;
    if (nsm <= 0) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P.device);
    const int G = P.recip_ntiles < nsm ? P.recip_ntiles : nsm;
    rt::k_recip_syrk<<<G, rt::THREADS, sm, s>>>(mh, ml, mhb, mlb, P.d_rtiles, P.recip_ntiles,
                                               P.n3, P.recip_kp / rt::BK, D32, P.ld,
                                               P.d_status + 6);
    count_launches(1);
    return check_launch("reciprocal product");
}

}  // namespace bd
