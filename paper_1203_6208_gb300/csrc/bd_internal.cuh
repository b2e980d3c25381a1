// bd_internal.cuh -- internal declarations shared by the CUDA translation
// units of libbdgb (plan layout, launch helpers, error plumbing).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/bd.h"

namespace bd {

// Half-space reciprocal vector with its M2 tensor folded with the +/-k pair:
// m[0..5] = 2 f(k) (delta_ab - khat_a khat_b) for ab = xx, xy, xz, yy, yz, zz.
struct KVec {
    double k[3];
    double m[6];
};

// Ewald coefficients of Eq. (M1) with 1/sqrt(pi) folded in, in the form
//   c1 = erfc(alpha r)/r (A1 + A3/r^2) + e^{-alpha^2 r^2} (P0 + P1 r^2 + P2 r^4 + Q/r^2)
//   c2 = erfc(alpha r)/r (A1 - 3 A3/r^2) + e^{-alpha^2 r^2} (R0 + R1 r^2 + R2 r^4 + S/r^2)
// computed once per plan on the device in FP64.
struct EwaldCoef {
    double alpha, alpha2, a, L, invL, rc2, four_a2;
    double A1, A3, P0, P1, P2, Q, R0, R1, R2, S;
    double self;                 // 1 - 6 a alpha/sqrt(pi) + 40 a^3 alpha^3/(3 sqrt(pi))
    double g1a, g1b, g2a, g2b;   // a alpha, a^3 alpha^3, a alpha^3, a^3 alpha^5 (each / sqrt(pi))
    double inv_a;
};

// Piecewise-polynomial table of the Eq. (M1) coefficients for images with
// 4a^2 <= u = |r|^2 <= r_c^2: interval i covers the u whose FP32 bit pattern
// has (bits >> SHIFT) == i0 + i, i.e. 2^BITS intervals per octave of u.
// Per interval: mid, 1/half-width, then DEG+1 monomial coefficients in
// t = (u - mid)/half-width of c1(u) and of c2(u)/u.  The FP64 table (degree 8
// on 16 intervals per octave) interpolates to ~1e-12 of the local value; the
// FP32 table (degree 4 on 64 intervals per octave, 48-byte rows) to ~3e-9,
// below FP32 rounding, with half the loads and FMAs per image.
template <typename T> struct TabFmt;
template <> struct TabFmt<double> {
    static constexpr int BITS = 4, DEG = 8, SHIFT = 23 - BITS, STRIDE = 2 + 2 * (DEG + 1);
};
template <> struct TabFmt<float> {
    static constexpr int BITS = 6, DEG = 4, SHIFT = 23 - BITS, STRIDE = 2 + 2 * (DEG + 1);
};
static_assert(TabFmt<double>::STRIDE % 2 == 0 && TabFmt<float>::STRIDE % 4 == 0,
              "table rows must be 16-byte multiples");
constexpr int kTabMax = 2048;

// the Eq. (M1) coefficients and the box constants in the working precision of
// a pair kernel (converted once per plan: on this GPU a double-to-float
// conversion issues on the FP64 pipe, which must stay out of FP32 loops)
template <typename T> struct EwaldT {
    T alpha, alpha2, A1, A3, P0, P1, P2, Q, R0, R1, R2, S;
    T g1a, g1b, g2a, g2b, inv_a, rc2, four_a2, self;
    T L, Llo, halfL;     // box edge as T plus its low-order remainder (FP32: L - (float)L)
    float Lf, invLf;     // box edge and its inverse for the FP32 image cursor
};

constexpr int kMaxKvec = 4096;        // half-space k-vectors a plan may use
constexpr int kMaxRhs = 32;           // Wiener columns per product
constexpr int kMaxCheb = 256;         // Chebyshev terms
// The interval map of a Chebyshev series (Eq. cheb2: y = s x - t with
// s = 2 / (d_max - d_min), t = (d_max + d_min) / (d_max - d_min)), formed once
// per series beside its coefficients: coef[kChebMapS], coef[kChebMapT].  FP64
// divisions are long sequences on this GPU's slow FP64 pipe; the products'
// epilogues read the two values instead of dividing per CTA or per element.
constexpr int kChebMapS = kMaxCheb, kChebMapT = kMaxCheb + 1;
constexpr int kMaxLanczos = 128;      // Lanczos steps
constexpr int kLdAlign = 64;          // D leading dimension multiple (elements)

struct PmeState;
struct SymState;

// what a step's front part leaves for its back part (the batched loop runs
// in between)
struct StepCtx {
    double *R;
    const void *D;
    const double *w, *Wcols;
    double *dSd;
    bd_step_stats *st_dev;
    const double *DFd;
    double *DF;
    int m, nch, lag;
    double bound_safety, dmin_fraction;
};

struct Plan {
    bd_params p;
    int device;
    int n, n3, ld;
    int nk;                            // half-space k-vectors in use
    double self_coeff;                 // self term of Eq. (DF)
    KVec *d_kvec;                      // [nk], device
    double *d_km64;                    // folded M2 tensors and k: [nk][12] (6 tensor, 3 k, pad)
    float *d_km32;                     // the same in FP32 (mixed plans)
    EwaldCoef *d_ewc;                  // Eq. (M1) coefficients, device
    EwaldT<double> *d_ew64;            // the same per working precision
    EwaldT<float> *d_ew32;
    EwaldT<double> h_ew64;             // host copies (passed to the pair kernels by value)
    EwaldT<float> h_ew32;
    double *d_pw64;                    // positions wrapped into [0, L), FP64 [3N]
    float *d_pw32;                     // the same as FP32 hi/lo words [2][3N]
    double *d_tab;                     // M1 table [ntab][TabFmt<double>::STRIDE] (FP64)
    float *d_tab32;                    // FP32 table [ntab32][TabFmt<float>::STRIDE] (mixed plans)
    int tab_i0, ntab;                  // first interval index, interval count (FP64 table)
    int tab32_i0, ntab32;              // the same for the FP32 table (mixed plans)
    // per-bead trig tables for the reciprocal sum: cos/sin(k_t . r_nu),
    // stored [t][nu] (FP64) for the current R
    double *d_cos, *d_sin;
    float *d_cos32, *d_sin32;
    // scratch vectors (3N x max_rhs, column-major, FP64)
    double *d_F, *d_DF;                // forces and drift (3N)
    double *d_Rnew;                    // proposed positions (3N)
    double *d_V[3];                    // Chebyshev recurrence buffers (3N x max_rhs)
    double *d_X0, *d_Y0;               // first product [F, dW, extra] and its image (3N x (max_rhs+3))
    double *d_dS;                      // noise when the caller passes no dS
    double *d_dW;                      // Wiener block when generated on device
    double *d_coef;                    // Chebyshev coefficients [kMaxCheb], then the interval map
    double *d_wdw;                     // dW.D.dW per column [kMaxRhs]
    double *d_red;                     // reduction results [4*kMaxRhs]
    double *d_redpart;                 // per-block partial sums [kRedBlocks * kMaxRhs]
    double *d_bounds;                  // {d_min, d_max}
    int32_t *d_status;                 // device status words [8]
    // Lanczos
    double *d_lq[3];                   // q_{j-1}, q_j, w (3N each)
    double *d_lab;                     // alpha_j [kMaxLanczos], beta_j [kMaxLanczos]
    // mixed precision operand scratch: X^T in 16 bits, [kMaxRhsPad][ldx]
    void *d_x16;
    float *d_xscale;                   // per-column power-of-two scale
    float *d_part;                     // split-K partial sums
    int32_t *d_counters;               // stream-K arrival counters (per row block)
    double *d_lanpart;                 // Lanczos dot partials per row block [3 * blocks]
    int ldx;                           // leading dimension of d_x16 (elements)
    int tc_split;                      // resident CTAs per SM of the tensor-core product (0: 2)
    int test_stall_term;               // bd_plan_test_stall: Chebyshev-series products to let pass
    int test_stall;                    // bd_plan_test_stall: CTA + 1 of the next symmetric
                                       //   product that stalls (0: none; one-shot)
    int tc_maxslots;                   // partial slots per row block (stream-K schedule)
    SymState *sym;                     // symmetric product schedule (mixed plans)
    float *d_xdf;                      // FP64 plans, shape 4: split operand [2][kMaxRhs][3N]
    cudaGraph_t step_graph;            // a captured bd_step (bd_step_capture)
    cudaGraphExec_t step_exec;
    int num_sms;                       // SM count of the plan's device
    int64_t scratch_bytes;
    bd_step_stats *d_stats_scratch;
    cudaEvent_t phase_ev[BD_PHASE_EVENTS];
    cudaEvent_t *prod_ev;              // product timing: event pairs around each
    int prod_cap, prod_n, prod_on;     //   Chebyshev-product kernel launch
    double *d_lag_bounds;              // bounds from the previous step's lagged Lanczos
    unsigned *d_pairw;                 // pair estimate words (pair_bound.cuh), float bits:
                                       //   [0] max over pairs of the block spectral radius,
                                       //   [1] d_s; written by the last assembly
    unsigned long long *d_step_ctr;    // device step counter (BD_STEP_DEVICE_COUNTER)
    int lag_valid;                     // host flag: d_lag_bounds was produced
    int phase_on;
    float *d_y32;                      // FP32 product scratch (mixed plans)
    float *d_xsplit;                   // refinement operand: hi/lo FP32 words [2][3N]
    // reverse mode (allocated by the first backward call)
    double *d_vhist;                   // V_0..V_{N_Ch-2}, [max_cheb-1][max_rhs][3N]
    double *d_xhist;                   // scaled adjoints X_q, same shape
    double *d_ubuf[4];                 // rolling adjoint vectors and D U products
    // matrix-free products (allocated by the first one)
    void *d_sfac;                      // structure factors [nk][max_rhs + 3][6] (working precision)
    double *d_mfW;                     // product scratch of matrix-free Chebyshev terms (3N x max_rhs)
    double *d_mfpart;                  // per-chunk partial products [chunks][3N x (max_rhs + 3)]
    int mf_chunks;                     // chunks of the bead loop in one matrix-free product
    const double *matfree_R;           // set inside a matrix-free step: products recompute D(R)
    PmeState *pme;                     // spectral product state (pme_grid > 0)
    int dense_off;                     // 1: no dense D (k-sphere beyond the dense tables)
    // adaptive N_Ch (allocated by the first adaptive call)
    double *d_mom;                     // moments, dot partials, estimates, D V scratch
    double *h_est;                     // pinned host words read back per candidate N
    // reciprocal sum as a tensor-core product (mixed plans, recip_tc.cu)
    int recip_tc;                      // 1: D32's upper tiles are filled by U U^T first
    int recip_kp;                      // columns of U (4 per k-vector, padded to 64)
    int recip_ntiles;                  // 128 x 256 blocks reaching the diagonal
    __half *d_Uh, *d_Ul;               // U as hi/lo words, half(word 2^8) [3N][recip_kp]
    int2 *d_rtiles;                    // block list (128-row tile, 256-column block)
    float *d_kbasis;                   // per k: w u1, w u2 (FP32) [nk][8]
    // launch shape 5 (rows_gemm.cu): row-streamed products of a few columns
    float *d_x32;                      // FP32 operand, 2 x [kRowsMaxCols][x32_stride]
    int x32_stride;                    // 3N rounded up to 8
    double *d_rows_part;               // Lanczos dot partials per 64-row item
    void *d_rows_rep;                  // the plan's one-replica table (RowsRep)
    int *d_rows_items;                 // item -> replica (all 0 for a single plan)
    unsigned *d_rows_bar;              // grid barrier {count, generation}, Lanczos item count
    StepCtx step_ctx;                  // kept between the parts of a batched step
};

inline bool is_mixed(const Plan &P) { return P.p.precision != BD_FP64; }

// host-side count of kernel launches (bd_kernel_launches)
void count_launches(int k);
// product timing marks (end = 0 before the launch, 1 after)
void prod_mark(Plan &P, int end, cudaStream_t s);

// error plumbing (thread-local message)
bd_status set_error(bd_status st, const char *fmt, ...);
bd_status check_launch(const char *what);

// ---- launchers (defined in the .cu files) ---------------------------------
// ewald_build.cu
void m1_table_range(const bd_params &p, int bits, int *i0, int *ntab);
void launch_kvec_table(Plan &P, cudaStream_t s);
void launch_trig_tables(Plan &P, const double *R, cudaStream_t s);
void launch_build_D_f64(Plan &P, const double *R, double *D, cudaStream_t s);
bd_status launch_build_D_f32(Plan &P, const double *R, float *D32, void *D16, int is_bf16,
                        cudaStream_t s);

// matrix-free Y = D(R) X (ewald_build.cu); the tables of R must be current
bd_status launch_matfree_tables(Plan &P, const double *R, cudaStream_t s);
// pair estimate words of D(R) without storing D (after launch_matfree_tables)
void launch_pair_estimate(Plan &P, cudaStream_t s);
bd_status matfree_init(Plan &P);
bd_status launch_apply_matfree(Plan &P, const double *X, int m, double *Y, cudaStream_t s);
// the matrix-free product of the plan: spectral (pme_grid > 0) or pair sums
bd_status matfree_product(Plan &P, const double *X, int m, double *Y, cudaStream_t s);

// dense_f64.cu : Y = D X (FP64), epilogue variants
// FP64 plans: launch shape of the double-float products on the FP32 pipe
constexpr int kF64DoubleFloat = 4;

struct ChebEpi {
    const double *coef;       // device coefficients
    const double *bounds;     // device {dmin, dmax}
    int p;                    // term index being produced (>= 2)
    double *Vprev2;           // in: V_{p-2}, out: V_p (in place)
    const double *Vprev1;     // V_{p-1} (also the B operand)
    double *dS;               // accumulated sum
};
void launch_gemm_f64(const Plan &P, const double *D, const double *X, int m, double *Y,
                     cudaStream_t s);
void launch_gemm_f64_cheb(const Plan &P, const double *D, int m, const ChebEpi &e,
                          cudaStream_t s);

// vec_kernels.cu
void launch_forces(Plan &P, const double *R, double *F, int32_t *n_bad, cudaStream_t s);
void launch_cheb_coeffs(Plan &P, const double *bounds, int nch, cudaStream_t s);
void launch_cheb_first(Plan &P, const double *bounds, const double *dW, const double *DW, int m,
                       double *V0, double *V1, double *dS, cudaStream_t s);
void launch_cheb_term(Plan &P, const double *W, const double *V1, double *V2, int m,
                      const double *bounds, int p, double *dS, cudaStream_t s);
void launch_ef(Plan &P, const double *dW, const double *DW, const double *dS, int m,
               double *Ef, bd_step_stats *stats, cudaStream_t s);
void launch_wiener(Plan &P, uint64_t seed, uint64_t step, int64_t count, double *out,
                   cudaStream_t s, const unsigned long long *step_dev = nullptr);
void launch_counter_add(unsigned long long *ctr, cudaStream_t s);
void launch_lanczos_init(Plan &P, cudaStream_t s);
void launch_lanczos_update(Plan &P, int j, cudaStream_t s, double *w = nullptr);
void launch_lanczos_finish(Plan &P, int k, double safety_max, double dmin_fraction,
                           double *bounds, int32_t *status, cudaStream_t s);
void launch_step_begin(bd_step_stats *st, int nch, int32_t *status, cudaStream_t s);
void launch_bounds_lagged(double *bounds, const double *lag, const unsigned *word,
                          double dmin_fraction, int32_t *status, bd_step_stats *st, cudaStream_t s);
// the pair estimate (pair_bound.cuh): word[0] = max over pairs of rho(D_{nu mu})
// read from a stored D (FP64, or the FP32 D32 when f32), upper triangle only;
// word[1] = d_s = D[0][0]
void launch_pair_radius_scan(const void *D, int f32, int n, long ld, unsigned *word,
                             cudaStream_t s);
// bounds[0] = min(bounds[0], dmin_fraction (d_s - rho_max)) from word;
// status (may be NULL) = BD_OK, or BD_ERR_NOT_PD when d_min <= 0 or d_max <= d_min
void launch_bounds_pair(double *bounds, const unsigned *word, double dmin_fraction,
                        int32_t *status, cudaStream_t s);
// Fixman estimates: U+, U- into two columns of X; bounds from X2 . Y2 (Y2 = D X2)
void launch_fixman_fill(double *X, int n3, cudaStream_t s);
void launch_fixman_bounds(Plan &P, const double *X2, const double *Y2, int mode, double C,
                          double *bounds, int32_t *status, cudaStream_t s);
void launch_stats_bounds(bd_step_stats *st, const double *bounds, const int32_t *bstatus,
                         cudaStream_t s);
void launch_euler(Plan &P, double *R, const double *DF, const double *dS, bd_step_stats *stats,
                  cudaStream_t s);
// deterministic column dots: out[j] = A_j . B_j; part holds kRedBlocks x m partials
constexpr int kRedBlocks = 64;
void launch_dot_cols(const double *A, const double *B, int n3, int m, double *out, double *part,
                     cudaStream_t s);
void launch_zero_i32(int32_t *p, int n, cudaStream_t s);
void launch_copy_f64(double *dst, const double *src, size_t n, cudaStream_t s);
void launch_copy3_f64(double *dst, const double *a, size_t na, const double *b, size_t nb,
                      const double *c, size_t nc, cudaStream_t s);

}  // namespace bd
