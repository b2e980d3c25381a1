// sym_gemm.cu -- the mixed-precision product Y = D16 X from the tiles on and
// above the diagonal of D16 only.
//
// D is symmetric (Eq. DF: the 3 x 3 block of (mu, nu) is the transpose of
// that of (nu, mu); the 16-bit copy is written mirrored), so one 128 x 128
// tile (I, J), I < J, serves both products Y_I += D_IJ X_J and
// Y_J += D_IJ^T X_I, and the product streams half of D16 from HBM.  Both
// products run on the 5th-generation tensor cores from the same staged tile:
// the first with the tile as a K-major A operand, the second with the same
// shared memory read as an MN-major A operand (its rows are the K dimension).
//
// Schedule.  The tile rows are grouped in bands of R; band b takes its tiles
// with J outer (J = r0 .. T-1) and I inner (I = r0 .. min(J, r1 - 1)), and
// the bands follow one another: a single sequence of U units that CTA c of
// the G resident CTAs cuts at [c U / G, (c + 1) U / G) (stream-K).  A CTA
// keeps one TMEM accumulator per band row (D_IJ X_J summed over its J) and
// two for the columns (D_IJ^T X_I summed over the band's rows of one J,
// double-buffered so the epilogue drains one while the next J accumulates).
// The band's operand rows X_I stay in shared memory; each stage of the ring
// holds one tile and X_J.  One warp issues the TMA loads, two issue the MMAs
// (the row products and the column products), four drain TMEM.  Partial sums
// leave the CTA as FP32 slots: one per
// (band, CTA) for the rows and one per (J-step, CTA) for the columns.  A
// second kernel sums, for each 128-row block, its row slots and then its
// column slots, band by band, in a fixed order (double-float, deterministic), and
// runs the epilogue of the product (plain store, or the Chebyshev term with
// the Lanczos column).  Every mbarrier wait is bounded; a CTA that gives up
// records BD_ERR_TIMEOUT, drains its copies in flight, frees its TMEM and
// returns.
#include <math.h>

#include <vector>

#include "sym_gemm.cuh"

namespace bd {

namespace sy {

using tc::BK;
using tc::BM;
using tc::kWaitLimit;

constexpr int R = 8;               // tile rows per band
constexpr int THREADS = 224;       // warp 0 TMA, warps 1 and 6 MMA, warps 2-5 epilogue
constexpr int A_TILE = 2 * BM * BK * 2;   // one 128 x 128 tile: two 64-column boxes
template <int BN> __host__ __device__ constexpr int xbox() { return BN * BK * 2; }   // 64 operand rows
template <int BN> __host__ __device__ constexpr int stage_bytes() { return A_TILE + 2 * xbox<BN>(); }
template <int BN> __host__ __device__ constexpr int vband_bytes() { return R * 2 * xbox<BN>(); }
template <int BN> __host__ __device__ constexpr int stages()
{
    return (226 * 1024 - vband_bytes<BN>() - 1024) / stage_bytes<BN>();
}
template <int BN> __host__ __device__ constexpr int smem_bytes()
{
    return stages<BN>() * stage_bytes<BN>() + vband_bytes<BN>() + 1024;
}

// schedule geometry, shared by the product and the reduction
struct Geo {
    int T;                 // 128-row tiles per side
    int nb;                // bands
    long U;                // units (tiles on and above the diagonal)
    int G;                 // CTAs of the product
    int rslots;            // row slots per band
    int cslots;            // column slots per J-step
    const long *boff;      // [nb + 1] first unit of each band
    const int *jbase;      // [nb + 1] first J-step of each band
    long colbase;          // first column slot in the partial pool (after the row slots)
    const int *xstart;     // [T + 1] first entry of each 128-row block in xlist
    const int *xlist;      // partial slots of each block, in summation order
};

__host__ __device__ inline int band_rows(int b, int T) { return T - b * R < R ? T - b * R : R; }

// units of band b before its J-step J
__host__ __device__ inline long jstep_off(int b, int J, int T)
{
    const int rb = band_rows(b, T), d = J - b * R;
    if (d < rb) return (long)d * (d + 1) / 2;
    return (long)rb * (rb + 1) / 2 + (long)(d - rb) * rb;
}

// CTA owning unit u: the c with c U / G <= u < (c + 1) U / G (integer division)
__host__ __device__ inline int cta_of(long u, long U, int G)
{
    return (int)(((u + 1) * (long)G + U - 1) / U) - 1;
}

struct It {
    int b, J, I;
};

__device__ inline void it_seek(It &t, long u, const long *boff, int nb, int T)
{
    int b = 0;
    while (b + 1 < nb && boff[b + 1] <= u) b++;
    long rem = u - boff[b];
    const int r0 = b * R, rb = band_rows(b, T);
    int d = 0;
    while (d < rb && rem >= d + 1) {
        rem -= d + 1;
        d++;
    }
    t.b = b;
    if (d < rb) {
        t.J = r0 + d;
        t.I = r0 + (int)rem;
    } else {
        t.J = r0 + rb + (int)(rem / rb);
        t.I = r0 + (int)(rem % rb);
    }
}

__device__ inline void it_next(It &t, int T)
{
    const int r0 = t.b * R, r1 = r0 + band_rows(t.b, T);
    t.I++;
    if (t.I > t.J || t.I >= r1) {
        t.J++;
        t.I = r0;
        if (t.J >= T) {
            t.b++;
            t.J = t.b * R;
            t.I = t.J;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// MN-major operand, 128-byte swizzle: 64-element chunks along M lbo bytes
// apart, 8-row groups along K 1024 bytes apart (SBO), version 1
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t addr, uint32_t lbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// -- kernel begin: k_sym_gemm
template <int BN>
__global__ void __launch_bounds__(THREADS, 1)
k_sym_gemm(const __grid_constant__ CUtensorMap mapD, const __grid_constant__ CUtensorMap mapX,
           Geo g, int m, int is_bf16, float *__restrict__ part, int32_t *__restrict__ err,
           int stall_cta, int pre_d)
{
    constexpr int ST = stages<BN>();
    constexpr int XB = xbox<BN>();
    constexpr int STAGE = stage_bytes<BN>();
    constexpr uint32_t TMEM_COLS = 512;
    static_assert((R + 2) * BN <= (int)TMEM_COLS, "accumulators exceed TMEM");
    static_assert(STAGE % 1024 == 0 && XB % 1024 == 0, "stage alignment");
    static_assert(ST >= 3, "ring too shallow");
    const uint32_t idesc_k = tc::idesc_f16(BN, is_bf16);
    const uint32_t idesc_mn = idesc_k | (1u << 15);          // A read MN-major

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *vband = smem + ST * STAGE;
    __shared__ __align__(8) uint64_t full_bar[ST], empty_bar[ST];
    __shared__ __align__(8) uint64_t vb_full, vb_empty, row_full, row_empty, col_full[2],
        col_empty[2], drain_bar, drain_bar2, stall_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x;
    const long u0 = (long)c * g.U / g.G, u1 = (long)(c + 1) * g.U / g.G;
    const int nunits = (int)(u1 - u0);
    const int T = g.T;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < ST; s++) {
            tc::mbar_init(tc::smem_u32(&full_bar[s]), 1);
            tc::mbar_init(tc::smem_u32(&empty_bar[s]), 2);
        }
        tc::mbar_init(tc::smem_u32(&vb_full), 1);
        tc::mbar_init(tc::smem_u32(&vb_empty), 1);
        tc::mbar_init(tc::smem_u32(&row_full), 1);
        tc::mbar_init(tc::smem_u32(&row_empty), 128);
        for (int q = 0; q < 2; q++) {
            tc::mbar_init(tc::smem_u32(&col_full[q]), 1);
            tc::mbar_init(tc::smem_u32(&col_empty[q]), 128);
        }
        tc::mbar_init(tc::smem_u32(&drain_bar), 1);
        tc::mbar_init(tc::smem_u32(&drain_bar2), 1);
        tc::mbar_init(tc::smem_u32(&stall_bar), 1);          // never completed
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    // launched as a programmatic dependent of the kernel before it: the set-up
    // above overlapped that kernel's tail; its outputs (the operand X, and the
    // partial slots this kernel overwrites) are used only after this wait.
    // The producer waits later, after its first D tiles (below).
    const bool producer = warp == 0 && lane == 0;
    if (!producer) tc::grid_dep_wait();
    if (threadIdx.x == 32) tc::grid_dep_launch();
    // the producer's record of its loads, for the drain after an abort: stages
    // issued, band segments, and the first stages' D tiles loaded ahead
    // (npre, their J in pre_j) of which the first xdone have their X_J too
    int issued = 0, pseg = 0, npre = 0, xdone = 0;
    int pre_j[ST];
    bool vb_pending = false;

    if (producer) {
        // ---- TMA producer
        const uint64_t pol_d = tc::l2_evict_first_policy();
        It t;
        it_seek(t, u0, g.boff, g.nb, T);
        if (pre_d) {
            // D was complete before the previous kernel started (the products
            // of a Chebyshev series): the D tiles of the first stages stream in
            // while that kernel finishes; each stage's barrier expects the
            // whole stage, so it completes only once X_J lands as well
            It tp = t;
            for (; npre < ST && npre < nunits; npre++) {
                const uint32_t a = tc::smem_u32(smem + npre * STAGE);
                const uint32_t fb = tc::smem_u32(&full_bar[npre]);
                tc::mbar_expect_tx(fb, STAGE);
                tc::tma_load_2d_hint(a, &mapD, tp.J * BM, tp.I * BM, fb, pol_d);
                tc::tma_load_2d_hint(a + BM * BK * 2, &mapD, tp.J * BM + BK, tp.I * BM, fb, pol_d);
                pre_j[npre] = tp.J;
                it_next(tp, T);
            }
            issued = npre;
        }
        tc::grid_dep_wait();
        int seg = 0, pb = -1;
        for (int i = 0; i < nunits; i++) {
            if (t.b != pb) {
                // the band's operand rows X_I, once the previous band's MMAs are done
                if (seg > 0 &&
                    !tc::mbar_wait(tc::smem_u32(&vb_empty), (uint32_t)(seg - 1) & 1u, &abort_flag))
                    break;
                const int r0 = t.b * R, rb = band_rows(t.b, T);
                const uint32_t vf = tc::smem_u32(&vb_full);
                tc::mbar_expect_tx(vf, (uint32_t)(rb * 2 * XB));
                for (int rr = 0; rr < rb; rr++)
                    for (int h = 0; h < 2; h++)
                        tc::tma_load_2d(tc::smem_u32(vband + (rr * 2 + h) * XB), &mapX,
                                        (r0 + rr) * BM + h * BK, 0, vf);
                vb_pending = true;
                seg++;
                pb = t.b;
            }
            const int s = i % ST;
            const uint32_t ph = (uint32_t)(i / ST) & 1u;
            const uint32_t a = tc::smem_u32(smem + s * STAGE);
            const uint32_t fb = tc::smem_u32(&full_bar[s]);
            if (i < npre) {
                // D already on its way: X_J completes the stage
                tc::tma_load_2d(a + A_TILE, &mapX, t.J * BM, 0, fb);
                tc::tma_load_2d(a + A_TILE + XB, &mapX, t.J * BM + BK, 0, fb);
                xdone = i + 1;
                it_next(t, T);
                continue;
            }
            if (!tc::mbar_wait(tc::smem_u32(&empty_bar[s]), ph ^ 1u, &abort_flag)) break;
            tc::mbar_expect_tx(fb, STAGE);
            tc::tma_load_2d_hint(a, &mapD, t.J * BM, t.I * BM, fb, pol_d);
            tc::tma_load_2d_hint(a + BM * BK * 2, &mapD, t.J * BM + BK, t.I * BM, fb, pol_d);
            tc::tma_load_2d(a + A_TILE, &mapX, t.J * BM, 0, fb);
            tc::tma_load_2d(a + A_TILE + XB, &mapX, t.J * BM + BK, 0, fb);
            issued = i + 1;
            it_next(t, T);
        }
        pseg = seg;
    } else if ((warp == 1 || warp == 6) && lane == 0) {
        // ---- MMA issuers: warp 1 the row products D_IJ X_J (K-major tile),
        // warp 6 the column products D_IJ^T X_I (the same tile MN-major);
        // each commits every ring stage (its empty barrier counts two), the
        // row issuer the band's row accumulators, the column issuer the
        // J-step's column accumulator and the band's operand rows X_I.  Two
        // issuers overlap the per-instruction issue cost of the 16 small MMAs
        // of a tile (2.5 % on the product)
        const bool rows = warp == 1;
        It t;
        it_seek(t, u0, g.boff, g.nb, T);
        bool ok = true;
        int seg = 0, jsteps = 0, pb = -1, pJ = -1;
        uint32_t started = 0;
        bool col_on = false;
        if (rows && (int)blockIdx.x == stall_cta) {
            // test hook (bd_plan_test_stall): a wait on a barrier that nothing
            // completes, given up after a bounded spin like any wait that ran
            // out; the CTA then takes the abort path below
            for (uint32_t k = 0; k < 4096u && !tc::mbar_try(tc::smem_u32(&stall_bar), 0); k++) {}
            abort_flag = 1;
            ok = false;
        }
        for (int i = 0; i < nunits && ok; i++) {
            It nx = t;
            it_next(nx, T);
            const bool first_band = (t.b != pb);
            const bool last_band = (i + 1 == nunits) || (nx.b != t.b);
            const bool first_j = first_band || (t.J != pJ);
            const bool last_j = last_band || (nx.J != t.J);
            if (first_band) {
                if (rows) {
                    if (seg > 0 &&
                        !tc::mbar_wait(tc::smem_u32(&row_empty), (uint32_t)(seg - 1) & 1u, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    started = 0;
                } else if (!tc::mbar_wait(tc::smem_u32(&vb_full), (uint32_t)seg & 1u, &abort_flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                seg++;
            }
            if (first_j) col_on = false;
            const int s = i % ST;
            const uint32_t ph = (uint32_t)(i / ST) & 1u;
            if (!tc::mbar_wait(tc::smem_u32(&full_bar[s]), ph, &abort_flag)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int rr = t.I - t.b * R;
            const uint32_t a = tc::smem_u32(smem + s * STAGE);
            if (rows) {
                const uint32_t xj = a + A_TILE;
                const uint32_t acc_r = tmem + (uint32_t)(rr * BN);
                const bool racc = (started >> rr) & 1u;
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint64_t da = tc::sw128_desc(a + (k >> 2) * (BM * BK * 2)) + (uint64_t)(2 * (k & 3));
                    const uint64_t db = tc::sw128_desc(xj + (k >> 2) * XB) + (uint64_t)(2 * (k & 3));
                    tc::mma_f16(acc_r, da, db, idesc_k, (racc || k > 0) ? 1u : 0u);
                }
                started |= 1u << rr;
            } else if (t.I != t.J) {
                if (!col_on && jsteps >= 2 &&
                    !tc::mbar_wait(tc::smem_u32(&col_empty[jsteps & 1]),
                                   (uint32_t)((jsteps >> 1) - 1) & 1u, &abort_flag)) {
                    ok = false;
                    break;
                }
                if (!col_on) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc_c = tmem + (uint32_t)((R + (jsteps & 1)) * BN);
                const uint32_t xi = tc::smem_u32(vband + rr * 2 * XB);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint64_t da = sw128_desc_mn(a + k * 2048, BM * BK * 2);
                    const uint64_t db = tc::sw128_desc(xi + (k >> 2) * XB) + (uint64_t)(2 * (k & 3));
                    tc::mma_f16(acc_c, da, db, idesc_mn, (col_on || k > 0) ? 1u : 0u);
                }
                col_on = true;
            }
            tc::mma_commit(tc::smem_u32(&empty_bar[s]));
            if (!rows && last_j && col_on) {
                tc::mma_commit(tc::smem_u32(&col_full[jsteps & 1]));
                jsteps++;
            }
            if (last_band) tc::mma_commit(tc::smem_u32(rows ? &row_full : &vb_empty));
            pb = t.b;
            pJ = t.J;
            t = nx;
        }
        if (!ok) {
            uint64_t *db = rows ? &drain_bar : &drain_bar2;
            tc::mma_commit(tc::smem_u32(db));
            for (uint32_t k = 0; k < kWaitLimit && !tc::mbar_try(tc::smem_u32(db), 0); k++) {}
        }
    } else if (warp >= 2 && warp <= 5) {
        // ---- epilogue warps: TMEM lane quadrant q, row r of the tile
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        It t;
        it_seek(t, u0, g.boff, g.nb, T);
        int seg = 0, jsteps = 0, pb = -1, pJ = -1;
        uint32_t started = 0;
        bool col_on = false;
        for (int i = 0; i < nunits; i++) {
            It nx = t;
            it_next(nx, T);
            const bool first_band = (t.b != pb);
            const bool last_band = (i + 1 == nunits) || (nx.b != t.b);
            const bool first_j = first_band || (t.J != pJ);
            const bool last_j = last_band || (nx.J != t.J);
            if (first_band) started = 0;
            if (first_j) col_on = false;
            started |= 1u << (t.I - t.b * R);
            if (t.I != t.J) col_on = true;
            if (last_j && col_on) {
                const int qb = jsteps & 1;
                if (!tc::mbar_wait_sleep(tc::smem_u32(&col_full[qb]), (uint32_t)(jsteps >> 1) & 1u,
                                         &abort_flag))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float acc[BN];
#pragma unroll
                for (int cc = 0; cc < BN; cc += 16)
                    tc::tmem_ld16(tmem + lane_off + (uint32_t)((R + qb) * BN + cc), acc + cc);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(tc::smem_u32(&col_empty[qb]));
                const long uf = g.boff[t.b] + jstep_off(t.b, t.J, T);
                const int slot = c - cta_of(uf, g.U, g.G);
                const long jid = (long)g.jbase[t.b] + (t.J - t.b * R);
                float *dst = part + ((g.colbase + jid * g.cslots + slot) * BN) * BM + r;
#pragma unroll
                for (int cc = 0; cc < BN; cc++)
                    if (cc < m) dst[(size_t)cc * BM] = acc[cc];
                jsteps++;
            }
            if (last_band) {
                if (!tc::mbar_wait_sleep(tc::smem_u32(&row_full), (uint32_t)seg & 1u, &abort_flag))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int rb = band_rows(t.b, T);
                const int slot = c - cta_of(g.boff[t.b], g.U, g.G);
                for (int rr = 0; rr < rb; rr++) {
                    float acc[BN];
                    if ((started >> rr) & 1u) {
#pragma unroll
                        for (int cc = 0; cc < BN; cc += 16)
                            tc::tmem_ld16(tmem + lane_off + (uint32_t)(rr * BN + cc), acc + cc);
                    } else {
#pragma unroll
                        for (int cc = 0; cc < BN; cc++) acc[cc] = 0.f;
                    }
                    float *dst = part + ((((long)t.b * g.rslots + slot) * R + rr) * BN) * BM + r;
#pragma unroll
                    for (int cc = 0; cc < BN; cc++)
                        if (cc < m) dst[(size_t)cc * BM] = acc[cc];
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(tc::smem_u32(&row_empty));
                seg++;
            }
            pb = t.b;
            pJ = t.J;
            t = nx;
        }
    }
    // ---- teardown.  Every role has left its loop once all threads are here,
    // so abort_flag is final: after an abort (which may come after the
    // producer issued its last load) the producer lets every load it issued
    // land before the CTA exits, and the status word records the timeout.
    __syncthreads();
    if (abort_flag) {
        if (warp == 0 && lane == 0) {
            // stages loaded ahead whose X_J was never issued: issue it (the
            // dependency wait is behind the producer whenever it can abort) so
            // that their barriers complete and the drain below can see the D
            // tiles land
            for (int i = xdone; i < npre; i++) {
                const uint32_t a = tc::smem_u32(smem + i * STAGE);
                const uint32_t fb = tc::smem_u32(&full_bar[i]);
                tc::tma_load_2d(a + A_TILE, &mapX, pre_j[i] * BM, 0, fb);
                tc::tma_load_2d(a + A_TILE + XB, &mapX, pre_j[i] * BM + BK, 0, fb);
            }
            for (int i = (issued > ST ? issued - ST : 0); i < issued; i++) {
                const int s = i % ST;
                const uint32_t ph = (uint32_t)(i / ST) & 1u;
                for (uint32_t k = 0; k < kWaitLimit && !tc::mbar_try(tc::smem_u32(&full_bar[s]), ph); k++) {}
            }
            if (vb_pending)
                for (uint32_t k = 0;
                     k < kWaitLimit && !tc::mbar_try(tc::smem_u32(&vb_full), (uint32_t)(pseg - 1) & 1u); k++) {}
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
// -- kernel end: k_sym_gemm

// ---------------------------------------------------------------------------
// For the 128-row block X (blockIdx.x) and one column (blockIdx.y): its row
// slots (band bX, every CTA whose range met the band, in CTA order) and then
// its column slots (bands b = 0 .. bX with rows above X, each J-step's CTAs
// in order) -- the list the plan built for X -- summed in that order;
// then that column's part of the product's epilogue (the Lanczos column also
// reduces its row block's dot partials).
template <int BN>
__global__ void __launch_bounds__(128)
k_sym_reduce(Geo g, const float *__restrict__ part, int n3, tc::Epi e)
{
    constexpr int kList = 256;
    __shared__ double lan_red[4][3];
    __shared__ int s_list[kList];
    // a programmatic dependent of the product kernel: scheduled while the
    // product's CTAs finish, it reads their partial slots only after this
    // wait; the kernel after it may be scheduled as soon as every CTA of this
    // one has started (it waits for this one's results itself)
    tc::grid_dep_launch();
    tc::grid_dep_wait();
    const int X = blockIdx.x, cc = blockIdx.y, r = threadIdx.x;
    const int q = r >> 5, lane = r & 31;
    const long row = (long)X * BM + r;
    const float *base = part + (size_t)cc * BM + r;
    const int i0 = g.xstart[X], i1 = g.xstart[X + 1];
    // FP32 partials summed as a double-float (TwoSum: the running sum and its
    // exact rounding errors), in list order: as exact as an FP64 sum of FP32
    // values for these lengths, at FP32 issue rate (the FP64 pipe of this GPU
    // runs at 1/64 of it)
    float sh = 0.f, sl = 0.f;
    auto add = [&](float v) {
        const float t = sh + v, bp = t - sh;
        sl += (sh - (t - bp)) + (v - bp);
        sh = t;
    };
    for (int c0 = i0; c0 < i1; c0 += kList) {
        const int cn = min(kList, i1 - c0);
        __syncthreads();
        for (int k = r; k < cn; k += 128) s_list[k] = g.xlist[c0 + k];
        __syncthreads();
        int k = 0;
        for (; k + 8 <= cn; k += 8) {
            float v[8];
#pragma unroll
            for (int h = 0; h < 8; h++) v[h] = __ldcg(base + (size_t)s_list[k + h] * (BN * BM));
#pragma unroll
            for (int h = 0; h < 8; h++) add(v[h]);
        }
        for (; k < cn; k++) add(__ldcg(base + (size_t)s_list[k] * (BN * BM)));
    }
    // the operand's column scales are powers of two: undone exactly in FP32
    const float isc = e.inv_scale[cc];
    if (e.mode == 0) {
        if (row < n3) e.Y[(long)cc * n3 + row] = tc::f32_to_f64(sh * isc) + tc::f32_to_f64(sl * isc);
        return;
    }
    if (cc == e.lan_col) {
        // the Lanczos column: w = D q_j and this row block's share of q_j.w,
        // q_{j-1}.w and w.w, reduced in a fixed order (deterministic)
        const double lw = tc::f32_to_f64(sh * isc) + tc::f32_to_f64(sl * isc);
        if (row < n3) e.lan_w[row] = lw;
        double t[3] = {row < n3 ? e.lan_q[row] * lw : 0.0, row < n3 ? e.lan_qp[row] * lw : 0.0,
                       row < n3 ? lw * lw : 0.0};
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
        if (lane == 0)
            for (int k = 0; k < 3; k++) lan_red[q][k] = t[k];
        __syncthreads();
        if (r == 0)
            for (int k = 0; k < 3; k++)
                e.lan_part[3 * X + k] = ((lan_red[0][k] + lan_red[1][k]) + lan_red[2][k]) + lan_red[3][k];
        return;
    }
    // Chebyshev term of Eqs. (cheb2)/(cheb3): V_p = 2 (s W - t V_{p-1}) - V_{p-2},
    // dS += c_p V_p, and the scaled 16-bit V_p as the next product's operand.
    // The interval map s, t (formed once per series beside the coefficients)
    // is folded with the factor 2 and the column's inverse scale (a power of
    // two) so that each element costs four FP64 fused multiply-adds:
    // V_p = 2s isc (sh + sl) - (2t V_{p-1} + V_{p-2}).
    if (row >= n3) return;
    const double ya = 2.0 * e.coef[kChebMapS] * (double)isc, yb = 2.0 * e.coef[kChebMapT];
    const double cp = e.coef[e.p];
    const long o = (long)cc * n3 + row;
    const double p1 = e.Vprev1[o], p2 = e.Vprev2[o], d0 = e.dS[o];
    const double v = fma(ya, tc::f32_to_f64(sh), fma(ya, tc::f32_to_f64(sl), -fma(yb, p1, p2)));
    e.Vprev2[o] = v;
    e.dS[o] = fma(cp, v, d0);
    const float sv = tc::f64_to_f32_rz(v) * e.scale[cc];
    const size_t xo = (size_t)cc * e.ldx + row;
    if (e.is_bf16) ((__nv_bfloat16 *)e.X16next)[xo] = __float2bfloat16_rn(sv);
    else ((__half *)e.X16next)[xo] = __float2half_rn(sv);
}

// ---------------------------------------------------------------------------
// FP64-residual refinement of one column from the FP32 D on and above the
// diagonal (the symmetric shape's D carries no lower triangle): y = D x with
// x = xh + xl split into FP32 words and every product d xh formed exactly as
// the pair (p, fma(d, xh, -p)) plus d xl, summed as double-float (TwoSum).
// One CTA per 128 x 128 tile (I, J), I <= J, each thread an 8 x 8 block;
// a tile gives the row partial D_IJ x_J and, off the diagonal, the
// column partial D_IJ^T x_I, both in FP32 pairs; a second kernel sums a row
// block's partials in a fixed order (its row partials J = X .. T-1, then its
// column partials I = 0 .. X-1).
struct DF {
    float s, c;
};

__device__ __forceinline__ void df_add(DF &a, float p, float e)
{
    const float t = a.s + p, z = t - a.s;
    a.c += ((a.s - (t - z)) + (p - z)) + e;
    a.s = t;
}

__device__ __forceinline__ void df_madd(DF &a, float d, float xh, float xl)
{
    const float p = d * xh;
    const float e = fmaf(d, xl, fmaf(d, xh, -p));
    df_add(a, p, e);
}

__device__ __forceinline__ void df_merge(DF &a, DF b)
{
    df_add(a, b.s, b.c);
}

__host__ __device__ inline void tile_of_index(long t, int *I, int *J)
{
    int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((long)j * (j + 1) / 2 > t) j--;
    while ((long)(j + 1) * (j + 2) / 2 <= t) j++;
    *J = j;
    *I = (int)(t - (long)j * (j + 1) / 2);
}

__global__ void __launch_bounds__(256, 4)
k_sym_refine_tiles(const float *__restrict__ D32, long ld, int n3, const float *__restrict__ xs,
                   float2 *__restrict__ part)
{
    // thread (tr, tc) owns rows 8 tr .. 8 tr + 7 and columns 8 tc .. 8 tc + 7
    // of the tile; its row and column sums stay in registers, then 16 partials
    // per row (and per column) are combined in shared memory in a fixed order
    __shared__ float2 s_xi[BM], s_xj[BM];
    __shared__ float2 s_red[16][BM + 1];
    const long t = blockIdx.x;
    int I, J;
    tile_of_index(t, &I, &J);
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const float *xh = xs, *xl = xs + n3;
    if (tid < BM) {
        const long gi = (long)I * BM + tid, gj = (long)J * BM + tid;
        s_xi[tid] = gi < n3 ? make_float2(xh[gi], xl[gi]) : make_float2(0.f, 0.f);
        s_xj[tid] = gj < n3 ? make_float2(xh[gj], xl[gj]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const bool off = I != J;
    const long c0 = (long)J * BM + 8 * tc;
    float2 xj[8];
#pragma unroll
    for (int k = 0; k < 8; k++) xj[k] = s_xj[8 * tc + k];
    DF rs[8], cs[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        rs[k] = DF{0.f, 0.f};
        cs[k] = DF{0.f, 0.f};
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int r = 8 * tr + i;
        const long gr = (long)I * BM + r;
        float d[8];
#pragma unroll
        for (int k = 0; k < 8; k++) d[k] = 0.f;
        if (gr < n3) {
            const float *src = D32 + gr * ld + c0;
            if (c0 + 7 < n3) {
                const float4 v0 = __ldcs((const float4 *)src), v1 = __ldcs((const float4 *)(src + 4));
                d[0] = v0.x; d[1] = v0.y; d[2] = v0.z; d[3] = v0.w;
                d[4] = v1.x; d[5] = v1.y; d[6] = v1.z; d[7] = v1.w;
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    if (c0 + k < n3) d[k] = src[k];
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) df_madd(rs[i], d[k], xj[k].x, xj[k].y);
        if (off) {
            const float2 xi = s_xi[r];
#pragma unroll
            for (int k = 0; k < 8; k++) df_madd(cs[k], d[k], xi.x, xi.y);
        }
    }
    // row sums: 16 column groups per row
#pragma unroll
    for (int i = 0; i < 8; i++) s_red[tc][8 * tr + i] = make_float2(rs[i].s, rs[i].c);
    __syncthreads();
    if (tid < BM) {
        DF a = {s_red[0][tid].x, s_red[0][tid].y};
        for (int q = 1; q < 16; q++) df_merge(a, DF{s_red[q][tid].x, s_red[q][tid].y});
        part[(t * 2) * BM + tid] = make_float2(a.s, a.c);
    }
    if (!off) return;
    __syncthreads();
    // column sums: 16 row groups per column
#pragma unroll
    for (int k = 0; k < 8; k++) s_red[tr][8 * tc + k] = make_float2(cs[k].s, cs[k].c);
    __syncthreads();
    if (tid < BM) {
        DF a = {s_red[0][tid].x, s_red[0][tid].y};
        for (int q = 1; q < 16; q++) df_merge(a, DF{s_red[q][tid].x, s_red[q][tid].y});
        part[(t * 2 + 1) * BM + tid] = make_float2(a.s, a.c);
    }
}

// y[row] += (D x)[row] - y[row] for the 128-row block X, the row block's
// partials in a fixed order (deterministic)
__global__ void __launch_bounds__(BM)
k_sym_refine_reduce(const float2 *__restrict__ part, int T, int n3, double *__restrict__ y)
{
    const int X = blockIdx.x, r = threadIdx.x;
    const long row = (long)X * BM + r;
    DF a = {0.f, 0.f};
    // row partials of tiles (X, J), J = X .. T-1: tile index J (J + 1) / 2 + X
    int J = X;
    for (; J + 4 <= T; J += 4) {
        float2 v[4];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const long tt = (long)(J + h) * (J + h + 1) / 2 + X;
            v[h] = __ldcg(part + (tt * 2) * BM + r);
        }
#pragma unroll
        for (int h = 0; h < 4; h++) df_merge(a, DF{v[h].x, v[h].y});
    }
    for (; J < T; J++) {
        const long tt = (long)J * (J + 1) / 2 + X;
        const float2 v = __ldcg(part + (tt * 2) * BM + r);
        df_merge(a, DF{v.x, v.y});
    }
    // column partials of tiles (I, X), I = 0 .. X-1: tile index X (X + 1) / 2 + I
    const long base = (long)X * (X + 1) / 2;
    int I = 0;
    for (; I + 4 <= X; I += 4) {
        float2 v[4];
#pragma unroll
        for (int h = 0; h < 4; h++) v[h] = __ldcg(part + ((base + I + h) * 2 + 1) * BM + r);
#pragma unroll
        for (int h = 0; h < 4; h++) df_merge(a, DF{v[h].x, v[h].y});
    }
    for (; I < X; I++) {
        const float2 v = __ldcg(part + ((base + I) * 2 + 1) * BM + r);
        df_merge(a, DF{v.x, v.y});
    }
    if (row >= n3) return;
    const double acc = (double)a.s + (double)a.c;
    const double y0 = y[row];
    y[row] = y0 + (acc - y0);
}

}  // namespace sy

// ---------------------------------------------------------------------------
// host side

struct SymState {
    sy::Geo geo;            // device pointers filled in
    long *d_boff;
    int *d_jbase;
    int *d_xstart, *d_xlist;
    float *d_part;
    float2 *d_rpart;        // refinement partials [tiles][2][128]
};

static bd_status sym_oom(cudaError_t e)
{
    cudaGetLastError();
    return set_error(BD_ERR_OOM, "symmetric product scratch: %s", cudaGetErrorString(e));
}

bd_status sym_plan_init(Plan &P)
{
    if (P.sym) return BD_OK;
    using namespace sy;
    const int T = (P.n3 + BM - 1) / BM;
    const int nb = (T + R - 1) / R;
    std::vector<long> boff(nb + 1);
    std::vector<int> jbase(nb + 1);
    boff[0] = 0;
    jbase[0] = 0;
    for (int b = 0; b < nb; b++) {
        const int rb = band_rows(b, T);
        boff[b + 1] = boff[b] + (long)rb * (rb + 1) / 2 + (long)(T - b * R - rb) * rb;
        jbase[b + 1] = jbase[b] + (T - b * R);
    }
    const long U = boff[nb];
    const int G = (int)((long)P.num_sms < U ? P.num_sms : U);
    // CTAs meeting each band (row slots) and each J-step's column units
    // (column slots; none for the band's first J-step, its diagonal tile only)
    std::vector<int> bsl(nb), jsl(jbase[nb], 0);
    int rs = 1, cs = 1;
    for (int b = 0; b < nb; b++) {
        const int n = cta_of(boff[b + 1] - 1, U, G) - cta_of(boff[b], U, G) + 1;
        bsl[b] = n;
        rs = n > rs ? n : rs;
        const int r0 = b * R, r1 = r0 + band_rows(b, T);
        for (int J = r0 + 1; J < T; J++) {
            const int ncol = (J < r1 ? J : r1) - r0;
            const long uf = boff[b] + jstep_off(b, J, T);
            const int k = cta_of(uf + ncol - 1, U, G) - cta_of(uf, U, G) + 1;
            jsl[jbase[b] + (J - r0)] = k;
            cs = k > cs ? k : cs;
        }
    }
    // the summation list of each 128-row block: its band's row slots, then
    // the column slots of its J-step in every band above it, in band order
    const long colbase = (long)nb * rs * R;
    std::vector<int> xstart(T + 1), xlist;
    for (int X = 0; X < T; X++) {
        xstart[X] = (int)xlist.size();
        const int bX = X / R;
        for (int sl = 0; sl < bsl[bX]; sl++)
            xlist.push_back((int)(((long)bX * rs + sl) * R + (X - bX * R)));
        for (int b = 0; b <= bX && b * R < X; b++) {
            const long jid = (long)jbase[b] + (X - b * R);
            for (int sl = 0; sl < jsl[jid]; sl++) xlist.push_back((int)(colbase + jid * cs + sl));
        }
    }
    xstart[T] = (int)xlist.size();
    SymState *S = new SymState();
    memset(S, 0, sizeof(*S));
    P.sym = S;
    const size_t nslots = (size_t)colbase + (size_t)jbase[nb] * cs;
    const size_t pool = nslots * kMaxRhs * BM;
    cudaError_t e = cudaMalloc((void **)&S->d_boff, sizeof(long) * (nb + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_jbase, sizeof(int) * (nb + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_xstart, sizeof(int) * (T + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_xlist, sizeof(int) * (xlist.size() + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_part, sizeof(float) * pool);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_rpart, sizeof(float2) * 2 * BM * U);
    if (e != cudaSuccess) return sym_oom(e);
    P.scratch_bytes += (int64_t)(sizeof(float2) * 2 * BM * U);
    P.scratch_bytes += (int64_t)(sizeof(long) * (nb + 1) + sizeof(int) * (nb + 1 + T + 1 + xlist.size()) +
                                 sizeof(float) * pool);
    cudaMemcpy(S->d_boff, boff.data(), sizeof(long) * (nb + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(S->d_jbase, jbase.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(S->d_xstart, xstart.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice);
    if (!xlist.empty())
        cudaMemcpy(S->d_xlist, xlist.data(), sizeof(int) * xlist.size(), cudaMemcpyHostToDevice);
    S->geo = Geo{T, nb, U, G, rs, cs, S->d_boff, S->d_jbase, colbase, S->d_xstart, S->d_xlist};
    cudaError_t a[2] = {
        cudaFuncSetAttribute(k_sym_gemm<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<16>()),
        cudaFuncSetAttribute(k_sym_gemm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<32>())};
    for (cudaError_t x : a)
        if (x != cudaSuccess)
            return set_error(BD_ERR_CUDA, "smem attribute (symmetric product): %s",
                             cudaGetErrorString(x));
    return check_launch("symmetric product init");
}

void sym_plan_free(Plan &P)
{
    SymState *S = P.sym;
    if (!S) return;
    void *ptrs[] = {S->d_boff, S->d_jbase, S->d_xstart, S->d_xlist, S->d_part, S->d_rpart};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete S;
    P.sym = nullptr;
}

bd_status sym_refine(Plan &P, const float *D32, const float *xs, double *y, cudaStream_t s)
{
    bd_status st = sym_plan_init(P);
    if (st != BD_OK) return st;
    const SymState *S = P.sym;
    sy::k_sym_refine_tiles<<<(unsigned)S->geo.U, 256, 0, s>>>(D32, P.ld, P.n3, xs, S->d_rpart);
    sy::k_sym_refine_reduce<<<S->geo.T, sy::BM, 0, s>>>(S->d_rpart, S->geo.T, P.n3, y);
    count_launches(2);
    return check_launch("symmetric refinement");
}

bd_status sym_launch(Plan &P, const CUtensorMap &mapD, const CUtensorMap &mapX, int bn,
                     const tc::Epi &e, cudaStream_t s)
{
    bd_status st = sym_plan_init(P);
    if (st != BD_OK) return st;
    const SymState *S = P.sym;
    const sy::Geo &g = S->geo;
    const int cols = e.m + (e.lan_col >= 0 ? 1 : 0);
    int32_t *err = P.d_status + 6;
    // the stall hook (one-shot): armed for this product unless it waits for
    // a later product of a Chebyshev series
    int stall = -1;
    if (P.test_stall > 0) {
        if (P.test_stall_term > 0 && e.mode == 1) P.test_stall_term--;
        if (P.test_stall_term == 0) {
            stall = P.test_stall - 1;
            P.test_stall = 0;
        }
    }
    // a Chebyshev series' product follows kernels that do not write D, and D
    // was complete before they started: its first D tiles may be loaded
    // before the dependency wait.  A plain product may follow the kernel that
    // wrote D, so it loads nothing before that wait.
    const int pre_d = e.mode == 1 ? 1 : 0;
    // both kernels are programmatic dependents of the kernel before them:
    // each is scheduled while its predecessor's CTAs drain and waits
    // (griddepcontrol.wait) before it reads anything that kernel wrote
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cg = {};
    cg.gridDim = dim3(g.G);
    cg.blockDim = dim3(sy::THREADS);
    cg.stream = s;
    cg.attrs = attr;
    cg.numAttrs = 1;
    cudaLaunchConfig_t cr = cg;
    cr.gridDim = dim3(g.T, cols);
    cr.blockDim = dim3(128);
    cr.dynamicSmemBytes = 0;
    cudaError_t le;
    if (bn == 16) {
        cg.dynamicSmemBytes = sy::smem_bytes<16>();
        le = cudaLaunchKernelEx(&cg, sy::k_sym_gemm<16>, mapD, mapX, g, cols, e.is_bf16,
                                S->d_part, err, stall, pre_d);
        if (le == cudaSuccess)
            le = cudaLaunchKernelEx(&cr, sy::k_sym_reduce<16>, g, (const float *)S->d_part, P.n3, e);
    } else {
        cg.dynamicSmemBytes = sy::smem_bytes<32>();
        le = cudaLaunchKernelEx(&cg, sy::k_sym_gemm<32>, mapD, mapX, g, cols, e.is_bf16,
                                S->d_part, err, stall, pre_d);
        if (le == cudaSuccess)
            le = cudaLaunchKernelEx(&cr, sy::k_sym_reduce<32>, g, (const float *)S->d_part, P.n3, e);
    }
    count_launches(2);
    if (le != cudaSuccess) return set_error(BD_ERR_CUDA, "symmetric product launch: %s",
                                            cudaGetErrorString(le));
    return check_launch("symmetric product");
}

}  // namespace bd
