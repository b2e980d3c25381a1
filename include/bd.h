/*
 * bd.h -- C ABI of libbdgb: one periodic Brownian-dynamics Euler step for
 * bead-spring polymer solutions with Ewald-summed Rotne-Prager-Yamakawa
 * hydrodynamics, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Jain, Sunthar, Duenweg & Prakash, "Optimisation of a Brownian
 * dynamics algorithm for semidilute polymer solutions" (paper sections and
 * equations are cited per entry point below).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  * Plain pointers and sizes only.  "dev" pointers are CUDA device pointers
 *    on the device that was current when the plan was created; "host"
 *    pointers are ordinary host memory.
 *  * Vectors of 3N numbers use the bead-major index 3*nu + s (s = x, y, z):
 *    positions R, forces F, Wiener increments dW, drift D.F, noise dS.
 *    A block of m such vectors is stored column-major, column j starting at
 *    element j*3N.
 *  * The diffusion matrix D (3N x 3N, symmetric) is stored row-major with the
 *    leading dimension bd_plan_info.ld (>= 3N).  Its storage depends on the
 *    plan precision:
 *      BD_FP64        : double D[3N][ld]
 *      BD_MIXED_F16 /
 *      BD_MIXED_BF16  : float  D32[3N][ld] followed (at byte offset
 *                       3N*ld*4) by a 16-bit copy D16[3N][ld] (IEEE half or
 *                       bfloat16) that feeds the tensor cores.
 *    The caller allocates bd_plan_info.d_bytes bytes for it (device memory,
 *    256-byte aligned) and owns them.
 *  * Ownership: every argument buffer is caller-owned; nothing is freed
 *    across the ABI.  The plan owns its constant tables and its scratch.
 *  * Asynchrony: compute entry points enqueue work on the given stream and
 *    return without synchronising, unless stated otherwise.  A plan may be
 *    used by one stream at a time (its scratch is shared by its calls).
 *  * Errors: every entry point returns a bd_status; no C++ exception crosses
 *    the ABI.  On an error the text is available from bd_last_error()
 *    (thread-local).  Argument errors are detected before any work is
 *    enqueued.  Errors that only the device can detect (FENE over-stretch,
 *    non-positive bounds, a bounded wait that ran out) are written to
 *    device-side status words that the caller reads when convenient.
 */
#ifndef BD_H
#define BD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *bd_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    BD_OK = 0,
    BD_ERR_INVALID = 1,       /* bad argument or plan/argument mismatch            */
    BD_ERR_OOM = 2,           /* device allocation failed (plan creation; the
                                 neighbour table of a spectral matrix-free call)  */
    BD_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed                 */
    BD_ERR_NOT_PD = 4,        /* eigenvalue bound <= 0: D not positive definite    */
    BD_ERR_FENE_STRETCH = 5,  /* a FENE spring reached |Q|^2 >= b                  */
    BD_ERR_CHEB_NOCONV = 6,   /* adaptive Chebyshev did not reach the tolerance    */
    BD_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                */
    BD_ERR_UNSUPPORTED = 8    /* request outside the library's supported range     */
} bd_status;

typedef enum {
    BD_FP64 = 0,        /* FP64 everywhere                                          */
    BD_MIXED_F16 = 1,   /* FP32 D assembly; products on tensor cores with IEEE-half
                           operands and FP32 accumulation; FP64 vectors/scalars     */
    BD_MIXED_BF16 = 2   /* as BD_MIXED_F16 with bfloat16 operands.  bfloat16 keeps 8
                           significant bits (IEEE half 11): the Brownian term lands
                           near 5e-3 of the FP64 result, above the 1e-3 bound the
                           half-precision mode meets; kept for comparison only    */
} bd_precision;

/* Model and method parameters.  Units: lengths in l_H = sqrt(kT/H), time in
 * lambda_H = zeta/(4H) (Sec. II A). */
typedef struct {
    int32_t n_beads;          /* N; chains are contiguous in the bead index       */
    int32_t beads_per_chain;  /* N_b (N % N_b == 0)                               */
    double  box_L;            /* periodic cube edge L                             */
    double  a;                /* bead radius a = sqrt(pi) h* (Sec. II A)           */
    double  alpha;            /* Ewald splitting parameter alpha (Eq. DF)          */
    double  r_c;              /* real-space cutoff: images with |r| <= r_c (Eq. rparameter) */
    int32_t n2max;            /* reciprocal cutoff: k = 2 pi n / L, n.n <= n2max (Eq. kparameter) */
    int32_t overlap_corr;     /* 1: add the overlap correction M* for |r| < 2a (Eq. DFmodified) */
    int32_t spring;           /* 0 Hookean, 1 FENE (Sec. II A)                      */
    double  fene_b;           /* FENE extensibility b                             */
    int32_t ev_on;            /* 1: narrow-Gaussian excluded volume               */
    double  z_star, d_star;   /* EV strength and range: U/kT = (z_star/d_star^3) exp(-r^2/(2 d_star^2)) */
    double  r_ev;             /* EV cutoff over periodic images                   */
    double  dt;               /* time step Delta t (Eq. sde)                      */
    int32_t precision;        /* bd_precision                                     */
    int32_t max_rhs;          /* largest m (Wiener columns) any call will use, 1..32 */
    int32_t max_cheb;         /* largest number of Chebyshev terms N_Ch, 2..256   */
    int32_t pme_grid;         /* > 0: matrix-free products use the spectral path:
                                 real space over cell lists (needs r_c < L/2) and the
                                 reciprocal sum on a pme_grid^3 mesh (a multiple
                                 of 8 with no prime factor above 5, >= 2
                                 ceil(sqrt(n2max)) + 2, <= 512); 0: off        */
    int32_t pme_order;        /* B-spline order of the mesh, 4..10 and <= pme_grid */
} bd_params;

typedef struct bd_plan bd_plan;

typedef struct {
    int32_t n3;               /* 3N                                               */
    int32_t ld;               /* leading dimension of D in elements               */
    int64_t d_bytes;          /* bytes of device memory D needs                   */
    int32_t n_kvec;           /* half-space k-vectors of the reciprocal sum       */
    int32_t precision;        /* bd_precision of the plan                          */
    int64_t scratch_bytes;    /* device scratch owned by the plan                 */
} bd_plan_info;

/* Device-resident statistics of one step (the caller reads them back when it
 * wants; bd_step writes them on the stream). */
typedef struct {
    double  d_min, d_max;     /* eigenvalue bounds used by the Chebyshev series   */
    double  ef_max;           /* max over Wiener columns of E_f (Sec. IV)           */
    int32_t n_cheb;           /* Chebyshev terms used                              */
    int32_t n_overstretched;  /* FENE springs with |Q|^2 >= b in the proposal      */
    int32_t accepted;         /* 1 if R was advanced, 0 if the step was rejected   */
    int32_t status;           /* bd_status of the device-side checks              */
} bd_step_stats;

/* Options of bd_step. */
typedef struct {
    int32_t m;                /* Wiener columns (1..max_rhs); column 0 advances R  */
    int32_t n_cheb;           /* Chebyshev terms N_Ch (2..max_cheb); 0 = adaptive  */
    int32_t lanczos_iters;    /* Lanczos steps for the bounds (4..128)            */
    double  bound_safety;     /* d_max = (1 + bound_safety) theta_max             */
    double  dmin_fraction;    /* d_min = dmin_fraction min(theta_min, theta_pair)
                                 (0 < f <= 1; see bd_eig_bounds)                   */
    uint64_t seed;            /* Philox key when dW == NULL                        */
    uint64_t step_index;      /* Philox counter high word when dW == NULL          */
    int32_t bounds_mode;      /* BD_BOUNDS_FRESH, _LAGGED, _FIXMAN_DILUTE or
                                 _FIXMAN_SEMIDILUTE (see bd_step)                  */
    int32_t flags;            /* BD_STEP_DEVICE_COUNTER | BD_STEP_MATRIX_FREE or 0  */
    double  ef_tol;           /* n_cheb == 0: adaptive N_Ch until E_f < ef_tol      */
    double  fixman_c;         /* BD_BOUNDS_FIXMAN_SEMIDILUTE: C of Eq. (fmin)       */
} bd_step_opts;

#define BD_STEP_MATRIX_FREE 2 /* never store D: every product recomputes D(R) X from R
                                 (bd_apply_D_matfree); D may be NULL.  Bounds come from
                                 fresh Lanczos or Fixman's estimates (not lagged)     */
#define BD_STEP_DEVICE_COUNTER 1  /* with dW == NULL: the Philox counter high word is
                                     the plan's device step counter (set by
                                     bd_plan_set_step_counter) and the step advances
                                     it, so a captured graph draws new noise on
                                     every replay; step_index is ignored           */

#define BD_BOUNDS_FRESH 0     /* lanczos_iters Lanczos products every step, d_min
                                 tightened by the pair estimate of this step's D
                                 (bd_eig_bounds; not on matrix-free steps)          */
#define BD_BOUNDS_FIXMAN_DILUTE 2     /* Eq. (lmax-lmin-dilute): lambda^F_max,min =
                                 U+-.D.U+- / 3N with U+ all ones and U- alternating
                                 +1, -1 (two extra columns of the first product);
                                 d_max = 2 lambda^F_max, d_min = lambda^F_min / 2  */
#define BD_BOUNDS_FIXMAN_SEMIDILUTE 3 /* Eqs. (fmax), (fmin): lambda_max = 0.35 N^0.6
                                 lambda^F_max, lambda_min = lambda_max / (C N^0.6)
                                 with C = fixman_c, N the number of beads;
                                 d_max = lambda_max, d_min = lambda_min            */
#define BD_BOUNDS_LAGGED 1    /* mixed plans: the Lanczos vector rides as one extra
                                 column of this step's products; its bounds serve
                                 the next step (the first step runs fresh), d_min
                                 tightened by the pair estimate of the current D,
                                 which the assembly computes on the fly           */

/* ---------------------------------------------------------------------------
 * Plan.  bd_plan_create validates the parameters, computes the reciprocal
 * table (k-vectors and M2(k), Eq. M2) in FP64 on the current device and
 * allocates the plan's scratch (Chebyshev and Lanczos vectors).
 * Errors: BD_ERR_INVALID for inconsistent parameters, BD_ERR_OOM when the
 * scratch cannot be allocated, BD_ERR_CUDA otherwise.  Synchronous.      */
bd_status bd_plan_create(const bd_params *params, bd_plan **out_plan);
/* Frees the plan and its scratch (synchronises the device first).  NULL ok. */
void bd_plan_destroy(bd_plan *plan);
/* Sizes and layout of the plan (host output). */
bd_status bd_plan_query(const bd_plan *plan, bd_plan_info *out_info);

/* ---------------------------------------------------------------------------
 * bd_forces -- non-hydrodynamic forces F_mu = F_spr + F_exv (Sec. II A).
 * Springs: F^c(Q_mu) - F^c(Q_{mu-1}) with Hookean F^c(Q) = Q or FENE
 * F^c(Q) = Q/(1 - |Q|^2/b).  Excluded volume: narrow-Gaussian
 * F = sum (z_star/d_star^5) r exp(-r^2/(2 d_star^2)) over all pairs and periodic images
 * with |r| <= r_ev.  The paper uses a WCA potential and does not define this
 * narrow-Gaussian form; U/kT = (z_star/d_star^3) exp(-r^2/(2 d_star^2)) is the
 * library's reading of the excluded volume the benchmarked systems switch on.
 *   R       dev, 3N doubles (input positions, unwrapped)
 *   F       dev, 3N doubles (output)
 *   n_bad   dev, one int32 (output, may be NULL): FENE springs with
 *           |Q|^2 >= b; their force is set to NaN.                      */
bd_status bd_forces(bd_plan *plan, const double *R, double *F, int32_t *n_bad, bd_stream stream);

/* ---------------------------------------------------------------------------
 * bd_build_D -- assemble the dense periodic diffusion matrix D(R), Eq.
 * (DFmodified): self term (1 - 6 a alpha/sqrt(pi) + 40 a^3 alpha^3/(3
 * sqrt(pi))) I on the diagonal blocks, the real-space sum of M1 (Eq. M1)
 * over periodic images with |r| <= r_c (n = 0 omitted for nu = mu), the
 * reciprocal sum of M2(k) cos(k.(r_nu - r_mu)) over 0 < |k|, n.n <= n2max
 * (Eq. M2), and, for the image of a pair nu != mu closer than 2a, the
 * overlap correction M* = Omega_B - Omega_A (Eq. cor5).
 * Mixed plans form the reciprocal sum as a tensor-core product U U^T of
 * 16-bit words where 4 n_kvec <= 1024 and k_max^2 a^2 < 3, else per pair in
 * FP32; FP64 plans per pair in FP64.  Positions may be any finite doubles:
 * unwrapped coordinates are reduced into [0, L) exactly (fmod) before use, so
 * chains may travel any number of box lengths.  A non-finite position makes
 * its own rows and columns of D non-finite and leaves the rest as for the
 * other beads alone (its pairs contribute no real-space images).
 *   R   dev, 3N doubles
 *   D   dev, bd_plan_info.d_bytes bytes (output; layout in the header
 *       comment).  Padding columns [3N, ld) are not written.            */
bd_status bd_build_D(bd_plan *plan, const double *R, void *D, bd_stream stream);

/* ---------------------------------------------------------------------------
 * bd_apply_D -- Y = D X, the drift product of Eq. (sde) (and any product of
 * Eqs. cheb2/cheb3).  X, Y: dev, 3N x m column-major doubles, 1 <= m <=
 * max_rhs, X and Y must not overlap.  FP64 plan: FP64 product.  Mixed plan:
 * tensor-core product of D16 with the columns of X scaled to 16 bits, FP32
 * accumulation; with flags & BD_APPLY_REFINE, followed by one FP64-residual
 * refinement step y += (D32 X - y) evaluated with the FP32 matrix and FP64
 * accumulation.                                                           */
#define BD_APPLY_REFINE 1
bd_status bd_apply_D(bd_plan *plan, const void *D, const double *X, int32_t m, double *Y,
                     int32_t flags, bd_stream stream);

/* ---------------------------------------------------------------------------
 * bd_eig_bounds -- bounds d_min <= lambda_min(D), d_max >= lambda_max(D)
 * required by the Chebyshev series (Sec. IV).  The paper estimates them from
 * Fixman's quadratic forms and empirical scalings (Eqs. lmax-lmin-dilute,
 * fmax, fmin); here they come from two upper estimates of the extreme
 * eigenvalues, widened:
 *   d_max = (1 + safety_max) theta_max,
 *   d_min = dmin_fraction min(theta_min, theta_pair).
 * theta_min, theta_max: the extreme Ritz values of `iters` Lanczos steps
 * (FP64 vectors and recurrence, start vector from a fixed Philox stream).
 * theta_max converges to lambda_max from below within a few tens of steps;
 * theta_min approaches lambda_min slowly.
 * theta_pair = d_s - max over pairs nu != mu of the spectral radius of the
 * 3x3 block D_{nu mu}, with d_s I the (common) diagonal block: the smallest
 * eigenvalue of the pair's 6x6 principal submatrix, >= lambda_min by Cauchy
 * interlacing.  In dense solutions the lowest modes of D are the relative
 * motions of the closest overlapping pairs, so theta_pair lies within a few
 * per cent of lambda_min (measured at N = 3000 and 8000, c/c* = 4).
 * theta_pair <= 0 proves D indefinite.  The pair estimate reads the
 * strictly upper 3x3 blocks of D (FP64, or D32 of a mixed plan) once; the
 * tridiagonal eigenvalues are found by bisection on the device; a Lanczos
 * breakdown (beta ~ 0) truncates the tridiagonal matrix.  1 <= iters <= 128
 * (clamped to 3N).
 *   bounds  dev, 2 doubles (output): {d_min, d_max}
 *   status  dev, one int32 (output, may be NULL): BD_ERR_NOT_PD when
 *           d_min <= 0 or d_max <= d_min, else BD_OK.                     */
bd_status bd_eig_bounds(bd_plan *plan, const void *D, int32_t iters, double safety_max,
                        double dmin_fraction, double *bounds, int32_t *status, bd_stream stream);

/* ---------------------------------------------------------------------------
 * bd_chebyshev_sqrt -- Fixman's Chebyshev approximation of the Brownian
 * term dS = sqrt(D) dW, Eqs. (cheb1)-(cheb3):
 *   dS = sum_{p<N_Ch} c_p V_p - (c_0/2) dW,  V_0 = dW, V_1 = Y V_0,
 *   V_p = 2 Y V_{p-1} - V_{p-2},  Y = (2 D - (d_max + d_min) I)/(d_max - d_min),
 * with c_p the coefficients of the Chebyshev interpolant of sqrt on
 * [d_min, d_max] (computed in FP64 on the device), and the error estimate
 * E_f = sqrt(|dS.dS - dW.D.dW| / dW.D.dW) per column (Sec. IV).
 *   bounds  dev, {d_min, d_max}
 *   n_cheb  N_Ch, 2 <= n_cheb <= max_cheb
 *   dW, dS  dev, 3N x m column-major doubles (dS output)
 *   Ef      dev, m doubles (output, may be NULL)                         */
bd_status bd_chebyshev_sqrt(bd_plan *plan, const void *D, const double *bounds, int32_t n_cheb,
                            const double *dW, int32_t m, double *dS, double *Ef,
                            bd_stream stream);

/* bd_chebyshev_sqrt_adaptive -- the same series with N_Ch chosen as in
 * Sec. IV: N_Ch starts at Eq. (nint), nint(sqrt(d_max / d_min)) + 1 (the
 * bounds stand in for the extreme eigenvalues), and grows by one term until
 * E_f < ef_tol in every column, at most to the plan's max_cheb.  The
 * recurrence vectors V_p are kept (they do not depend on N_Ch) and E_f of
 * each candidate N_Ch is evaluated from the Chebyshev moments dW.T_j(Y)dW,
 * so every V_p is computed once; dS is then formed with the coefficients of
 * the chosen N_Ch and Ef recomputed from it.  Synchronises the stream (the
 * host reads the bounds and one number per candidate; not for graph
 * capture).  The first call allocates (max_cheb - 1) x 3N x max_rhs doubles
 * of history.
 *   ef_tol  > 0
 *   n_used  host, one int32 (output, may be NULL): the N_Ch used
 * Returns BD_ERR_CHEB_NOCONV if E_f >= ef_tol at max_cheb terms; dS and Ef
 * then hold the max_cheb-term result.                                   */
bd_status bd_chebyshev_sqrt_adaptive(bd_plan *plan, const void *D, const double *bounds,
                                     double ef_tol, const double *dW, int32_t m, double *dS,
                                     double *Ef, int32_t *n_used, bd_stream stream);

/* bd_apply_D_matfree -- Y = D(R) X without storing D (the paper's LMA,
 * Sec. V): real-space images, overlap branch and self term are evaluated
 * per bead pair inside the product (every unordered pair twice, once per
 * row, so each row is summed in a fixed order), the reciprocal sum through
 * structure factors S_k = sum_mu (cos, sin)(k.r_mu) X_mu per half-space k.
 * Same D as bd_build_D (to rounding): FP64 arithmetic on FP64 plans, FP32
 * with FP64 output on mixed plans (no 16-bit rounding).  Cost O(N^2 images)
 * per call, memory O(N): the path for N whose D does not fit.
 * With pme_grid > 0 the product is the spectral one instead: the real-space
 * part over a neighbour table of the pairs within r_c (built from a cell
 * list on every call, and once per step in bd_step), the reciprocal sum on
 * the B-spline mesh; cost O(N) real space + O(K^3 log K) mesh per product,
 * memory O(N r_c^3 density) for the table.  This form synchronises the
 * stream once (sizing the neighbour table) and may return BD_ERR_OOM when
 * the table grows.
 *   R     dev, 3N positions
 *   X, Y  dev, 3N x m column-major doubles, 1 <= m <= max_rhs + 3      */
bd_status bd_apply_D_matfree(bd_plan *plan, const double *R, const double *X, int32_t m,
                             double *Y, bd_stream stream);

/* ---------------------------------------------------------------------------
 * bd_mesh_fft -- the 3-D mesh transforms of the spectral product (Sec. VIII:
 * the Fourier part of the Ewald sum by FFT), on their own.  B real meshes
 * [B][K][K][K] (row-major, last index fastest) <-> their half spectra
 * [B][K][K][K/2 + 1] of (re, im) pairs, unnormalised:
 *   forward (inverse = 0): out_k = sum_j in_j e^{-2 pi i j.k / K}
 *   inverse (inverse = 1): out_j = sum over the full spectrum of in_k
 *                          e^{+2 pi i j.k / K}, the missing half taken as the
 *                          Hermitian conjugate (so inverse(forward(x)) = K^3 x)
 *   K          even, 2..512, no prime factor above 5 (else BD_ERR_UNSUPPORTED)
 *   B          meshes, 1..65535 (BD_ERR_UNSUPPORTED above)
 *   precision  BD_FP64: doubles; BD_MIXED_F16 / BD_MIXED_BF16: floats
 *   in, out    dev, must not overlap; the inverse overwrites `in`
 * Forms its twiddle tables on every call and returns after the transform has
 * finished on `stream` (synchronous).  BD_ERR_INVALID for NULL pointers,
 * B < 1, an unknown precision or overlapping buffers; BD_ERR_OOM or
 * BD_ERR_CUDA from the device.                                            */
bd_status bd_mesh_fft(int32_t K, int32_t B, int32_t precision, int32_t inverse, void *in,
                      void *out, bd_stream stream);

/* ---------------------------------------------------------------------------
 * bd_step -- one Euler step of Eq. (sde) with kappa = 0:
 *   r(t+dt) = r + (dt/4) D.F + (1/sqrt 2) dS[:,0],
 * i.e. bd_forces, bd_build_D, bd_eig_bounds, the product D.[F, dW] and
 * bd_chebyshev_sqrt, then the update.  With opts->bounds_mode =
 * BD_BOUNDS_LAGGED on a mixed plan, the bounds of step t come from the
 * Lanczos recurrence run inside the products of step t-1 (the Lanczos vector
 * is one extra column of D.[F, dW] and of every Chebyshev product, so it costs
 * no extra pass over D; N_Ch - 1 Lanczos steps), widened by the same
 * margins; the plan keeps them between calls.  FP64 plans, the first step of
 * a plan, m + 2 > 32, n_cheb < 8 and n_cheb > 129 use fresh bounds.
 * opts->n_cheb == 0 selects the adaptive series of
 * bd_chebyshev_sqrt_adaptive with opts->ef_tol (fresh bounds; the call then
 * synchronises the stream); stats->n_cheb reports the N_Ch used and
 * stats->status = BD_ERR_CHEB_NOCONV if max_cheb terms did not reach ef_tol
 * (the step is still taken with them).  FENE systems reject a proposal with
 * any |Q|^2 >= b (Sec. VII): R is then left unchanged, stats->accepted = 0
 * and stats->status = BD_ERR_FENE_STRETCH.
 *   R      dev, 3N doubles, advanced in place (only if accepted)
 *   D      dev, bd_plan_info.d_bytes bytes of workspace for D (overwritten)
 *   dW     dev, 3N x m Wiener increments, or NULL to draw them on the device:
 *          element pair q from Philox4x32-10 with counter (q, step_index)
 *          and key seed, Box-Muller, scaled by sqrt(dt)
 *   DF, dS dev outputs (may be NULL): 3N drift D.F and 3N x m noise
 *   stats  dev, one bd_step_stats (output, may be NULL)                   */
bd_status bd_step(bd_plan *plan, double *R, void *D, const double *dW, const bd_step_opts *opts,
                  double *DF, double *dS, bd_step_stats *stats, bd_stream stream);

/* bd_step_capture / bd_step_replay -- the same step as one CUDA graph.
 * bd_step_capture records the launches of bd_step(plan, R, D, NULL, opts,
 * DF, dS, stats) by stream capture on a private stream (nothing runs; `stream`
 * is not used, the legacy default stream cannot be captured) with the Wiener
 * increments drawn from the plan's device step counter (BD_STEP_DEVICE_COUNTER
 * is added to opts->flags), instantiates the graph and keeps it in the plan,
 * replacing an earlier one; every bd_step_replay then launches that step on
 * `stream` -- new noise per replay, the pointers and options of the capture.
 * Steps that synchronise the host cannot be captured: adaptive N_Ch
 * (n_cheb == 0) and BD_STEP_MATRIX_FREE return BD_ERR_INVALID.  A lagged-bounds
 * step should be captured after one bd_step has run with the same options
 * (else the captured step recomputes fresh Lanczos bounds on every replay).
 * The plan's phase events and product timing are not recorded in the graph.
 * Errors: BD_ERR_INVALID as above, BD_ERR_CUDA if capture or instantiation
 * fails; bd_step_replay: BD_ERR_INVALID without a captured step.          */
bd_status bd_step_capture(bd_plan *plan, double *R, void *D, const bd_step_opts *opts,
                          double *DF, double *dS, bd_step_stats *stats, bd_stream stream);
bd_status bd_step_replay(bd_plan *plan, bd_stream stream);

/* ---------------------------------------------------------------------------
 * Reverse mode.  D(R) enters the step through D_{nu mu} = B(r_nu - r_mu)
 * (Eq. DFmodified); the derivative of each block is recomputed per pair from
 * R (image sum, overlap branch and reciprocal sum), nothing like dD/dR is
 * stored.  Bounds d_min, d_max and N_Ch are held fixed (their derivative is
 * not taken).  gR is overwritten (3N doubles).
 *
 * bd_apply_D_backward -- for L with dL/dY = gY, Y = D(R) F:
 *   gF = D gY (may be NULL; needs D, the matrix built from the same R),
 *   gR = dL/dR = sum_mu dB(d_{nu mu})/dd : (gY_nu F_mu^T + gY_mu F_nu^T).  */
bd_status bd_apply_D_backward(bd_plan *plan, const double *R, const void *D, const double *F,
                              const double *gY, double *gR, double *gF, bd_stream stream);
/* bd_chebyshev_backward -- for L with dL/ddS = gS, dS = P(D(R)) dW the
 * Chebyshev series of bd_chebyshev_sqrt (same bounds, n_cheb, dW, m):
 * replays the forward terms V_p, runs the adjoint recurrence
 *   U_{N-1} = c_{N-1} gS,  U_p = c_p gS + 2 Y U_{p+1} - U_{p+2},
 *   gdW = U_0 = (c_0/2) gS + Y U_1 - U_2   (equal to P(D) gS),
 * and contracts dL/dD = (2/(d_max - d_min)) (U_1 V_0^T + 2 sum_{p>=2} U_p V_{p-1}^T)
 * with the pair derivative of D(R) into gR.  gdW may be NULL.  The first
 * backward call on a plan allocates its history buffers (2 (max_cheb - 1)
 * max_rhs 3N doubles) and so synchronises; later calls do not allocate.   */
bd_status bd_chebyshev_backward(bd_plan *plan, const double *R, const void *D,
                                const double *bounds, int32_t n_cheb, const double *dW,
                                int32_t m, const double *gS, double *gR, double *gdW,
                                bd_stream stream);

/* Launch shapes of the mixed plans' tensor-core product Y = D16 X:
 *   1, 2  the stream-K kernel over all of D16 with 1 or 2 resident CTAs per
 *         SM (0, the default of a new plan, means 2);
 *   3     the symmetric kernel: only the 128 x 128 tiles on and above the
 *         diagonal are read, each serving D_IJ X_J and D_IJ^T X_I (D is
 *         symmetric, Eq. DF), with a second kernel summing the partials in a
 *         fixed order and running the epilogue.  With this shape set, the
 *         assembly (bd_build_D, bd_step) writes D32 and D16 only on and above
 *         the diagonal 128 x 128 tiles (the diagonal tiles whole) and the
 *         FP64-residual refinement of D.F reads that half too; the rest of
 *         the lower triangle is left as it was.  Set the shape before
 *         assembling the D that a product will read.
 *   5     row-streamed products for a few columns (plans with max_rhs <= 4):
 *         D16 is read row by row on the CUDA cores with the operand in FP32
 *         (no 16-bit quantisation of X), FP32 sums in an order fixed by the
 *         row, and a step's whole Chebyshev series (with the lagged Lanczos
 *         column) runs as one persistent cooperative launch.  Mixed batches
 *         (bd_batch_*) of such plans take this shape and run the series of
 *         all their replicas in that one launch.
 * Shapes 1-3 give the same product up to FP32 summation order.
 * Launch shapes of the FP64 plans' product Y = D X:
 *   0     (default) FP64 multiply-adds;
 *   4     double-float on the FP32 pipe: each FP64 entry of D and X is split
 *         into two FP32 words (hi = the leading 24 significant bits, lo the
 *         next 24), each product d x is formed from hi*hi exactly (FMA error
 *         term) plus the cross terms hi*lo + lo*hi, and the products are
 *         summed as an unevaluated FP32 pair (two-sum).  The result agrees
 *         with the FP64 product to about 1e-13 of sum_k |D_ik x_k| (FP32
 *         pair precision, 2^-46, times the growth of a 3N-term sum) and is
 *         returned in FP64.  D, X and the products d x must lie in the
 *         FP32 range: D entries below 2^-97 in magnitude count as zero,
 *         entries of 2^128 or more overflow to an infinity, products below
 *         about 2^-100 lose bits.  The D of a physical system in the plan's
 *         units has entries of order one.  On a GPU whose FP64 pipe is a
 *         small fraction of FP32 this is the faster shape.
 * The shapes of one precision are rejected on a plan of the other
 * (BD_ERR_INVALID for 4 on a mixed plan; an FP64 plan takes 1..3 as 0).   */
#define BD_SHAPE_SYMMETRIC 3
#define BD_SHAPE_F64_DOUBLE_FLOAT 4
#define BD_SHAPE_ROWS 5

/* Autotuner: for a mixed plan, times the product of max_rhs + 1 columns on D
 * (its contents do not matter) in shapes 1, 2, 3 and, when max_rhs <= 4, 5,
 * and keeps the fastest for all later products of this plan; returns the
 * choice in *split_out and the time per product (ms).  Synchronous.  FP64
 * plans: no-op (0).                                                       */
bd_status bd_plan_autotune(bd_plan *plan, void *D, int32_t *split_out, float *ms_out,
                           bd_stream stream);

/* Set the launch shape (0..5, above) of the plan's later products without
 * timing.  Shape 3 allocates its schedule and partial buffers on first use,
 * shape 4 its split operand (64 x 3N floats), shape 5 its FP32 operand and
 * work-queue tables, all synchronous and BD_ERR_OOM if they do not fit.
 * BD_ERR_INVALID outside 0..5, for 4 on a mixed plan and for 5 on a mixed
 * plan with max_rhs > 4; FP64 plans take 1..3 and 5 as 0 (FP64
 * multiply-adds).                                                         */
bd_status bd_plan_set_shape(bd_plan *plan, int32_t shape);

/* Test hook for the device-side failure path (the paper has no counterpart;
 * it exercises the bounded waits of the tensor-core kernels without a GPU
 * fault).  Arms a symmetric product that the plan launches or records (a
 * mixed plan in launch shape 3): the next one for term = 0, else the
 * term-th product of a Chebyshev series from now (term = 1: the series'
 * first product, the one that forms V_2; those products load their first D
 * tiles before the previous kernel's results are visible).  In that product,
 * CTA `cta` (0 <= cta < SM count) waits on an mbarrier that nothing
 * completes, gives up after a bounded spin as any wait that ran out does,
 * and takes the abort path: it records BD_ERR_TIMEOUT in the plan's status
 * word, lets its copies in flight land, frees its TMEM and returns.  That
 * product's output is invalid; a bd_step containing it rejects the proposal
 * (R unchanged, stats.status = BD_ERR_TIMEOUT, accepted = 0).  The hook
 * disarms itself after one product; cta < 0 disarms it.  BD_ERR_INVALID on
 * an FP64 plan, in another shape, for cta >= the SM count or term < 0.     */
bd_status bd_plan_test_stall(bd_plan *plan, int32_t cta, int32_t term);

/* Set the plan's device step counter used by BD_STEP_DEVICE_COUNTER (stream-
 * ordered write of one uint64). */
bd_status bd_plan_set_step_counter(bd_plan *plan, uint64_t value, bd_stream stream);

/* ---------------------------------------------------------------------------
 * Batched replicas.  A batch holds `count` independent systems (each with
 * its own bd_params: uneven N, box, spring model, ...), one plan per replica.
 * Positions are packed: replica i owns 3 N_i doubles at r_offset(i); the D
 * workspace is one caller-owned arena, replica i at d_offset(i) (each
 * offset 256-byte aligned).  bd_batch_step advances every replica by one
 * step (bd_step semantics per replica, Wiener increments drawn on the device
 * with replica i keyed by opts->seed + i).  The first call runs the steps
 * directly and primes lagged bounds; the second call records the whole
 * batched step into one CUDA graph (one branch per replica on its own stream,
 * forked from and joined back to `stream`), and every later call with the
 * same arguments is a single graph launch.  Changing R, D, opts or stats
 * pointers re-records the graph.  Mixed batches whose replicas have
 * max_rhs <= 4 put every plan in launch shape 5: each replica's step then
 * runs its front (forces, D, bounds, first product) on its branch, the
 * Chebyshev series of ALL replicas runs as one persistent launch over a work
 * queue of {replica, 64-row block} items (a bounded grid barrier between
 * terms), and each replica's back (E_f, lagged bounds, Euler update) follows
 * on its branch; a replica's results are bitwise those of its plan alone in
 * the same shape.  Not thread-safe per batch.                            */
typedef struct bd_batch bd_batch;
bd_status bd_batch_create(const bd_params *params, int32_t count, bd_batch **out_batch);
void bd_batch_destroy(bd_batch *batch);
/* sizes: total packed position doubles, total D arena bytes; per replica
 * (index >= 0) its plan info and offsets (doubles into R, bytes into D). */
bd_status bd_batch_query(const bd_batch *batch, int32_t index, bd_plan_info *info,
                         int64_t *r_offset, int64_t *d_offset, int64_t *r_total,
                         int64_t *d_total);
/* stats: dev, count bd_step_stats (may be NULL). */
bd_status bd_batch_step(bd_batch *batch, double *R, void *D, const bd_step_opts *opts,
                        bd_step_stats *stats, bd_stream stream);

/* ---------------------------------------------------------------------------
 * bd_wiener -- the device Wiener generator of bd_step on its own: count
 * N(0, dt) numbers (see bd_step for the counter layout).  out: dev doubles. */
bd_status bd_wiener(bd_plan *plan, uint64_t seed, uint64_t step_index, int64_t count,
                    double *out, bd_stream stream);

/* ---------------------------------------------------------------------------
 * Phase timing.  When `events` is non-NULL, subsequent bd_step calls on this
 * plan record the caller's CUDA events (cudaEvent_t values, created and
 * owned by the caller) on the step's stream at the phase boundaries:
 *   ev[0] start, ev[1] after the forces, ev[2] after the D assembly,
 *   ev[3] after the eigenvalue bounds, ev[4] after the first product
 *   D.[F, dW], ev[5] after the Chebyshev terms, ev[6] after the update.
 * count must be 7.  The array is copied; NULL disables recording.        */
#define BD_PHASE_EVENTS 7
bd_status bd_set_phase_events(bd_plan *plan, void *const *events, int32_t count);

/* Kernel timing of the Chebyshev products.  enable = 1: from now on the
 * plan records a pair of CUDA events on the launch stream around each
 * Chebyshev-product kernel (FP64 product or tensor-core product with the
 * recurrence epilogue), up to 1024 launches.  enable = 0: waits for the last
 * recorded event, returns the summed kernel time (ms) and the number of
 * launches timed, and stops recording.                                    */
bd_status bd_product_timing(bd_plan *plan, int32_t enable, float *total_ms, int32_t *launches);

/* Number of CUDA kernels this library has launched in the process so far
 * (host-side counter; lets a caller count the launches of a region). */
uint64_t bd_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * bd_eig_bounds_noalloc -- the Lanczos bounds of bd_eig_bounds for an FP64
 * matrix, for callers that must not allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the same computation.
 * bd_eig_bounds needs a plan, and creating a plan allocates; a caller whose
 * device memory belongs to someone else's allocator (a host framework that
 * reserved HBM for its own pool), or that runs in a latency-critical loop
 * where cudaMalloc's possible device synchronisation is not acceptable, can
 * call this instead.  It allocates nothing: its working vectors live in one
 * fixed file-scope device array of about 0.6 MB (3 x 24576 doubles plus the
 * tridiagonal matrix), which every GPU that loads the library holds until
 * the process exits.
 *   D        dev, FP64 matrix, row-major, n3 rows with leading dimension ld
 *            (the layout bd_build_D writes for a BD_FP64 plan), 8-byte aligned
 *   n3       3N, a multiple of 3, 3 <= n3 <= 24576 (8192 beads); larger
 *            sizes return BD_ERR_UNSUPPORTED before any work is enqueued
 *   iters, safety_max, dmin_fraction, bounds, status: as in bd_eig_bounds
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before starting any stream capture on the device.  Every call uses the same
 * array, which keeps the previous call's contents (each call re-initialises
 * what it reads first); calls whose work overlaps on the GPU race and must be
 * serialised by the caller.                                               */
bd_status bd_eig_bounds_noalloc(const double *D, int32_t n3, int32_t ld, int32_t iters,
                                double safety_max, double dmin_fraction, double *bounds,
                                int32_t *status, bd_stream stream);

/* Text of the last error on this thread ("" if none).  Never NULL. */
const char *bd_last_error(void);
/* Library version string. */
const char *bd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BD_H */
