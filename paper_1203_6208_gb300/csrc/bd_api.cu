// bd_api.cu -- the C ABI of libbdgb (include/bd.h): plan lifecycle, argument
// validation, error text, and the orchestration of the step on one stream.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "bd_internal.cuh"
#include "sym_gemm.cuh"
#include "tc_gemm.cuh"
#include "rows_gemm.cuh"
#include "adjoint.cuh"
#include "recip_tc.cuh"
#include "adaptive.cuh"
#include "spectral.cuh"

struct bd_plan {
    bd::Plan P;
};

namespace bd {

static thread_local char g_err[1024] = "";
static unsigned long long g_launches = 0;

void count_launches(int k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }

void prod_mark(Plan &P, int end, cudaStream_t s)
{
    if (!P.prod_on || P.prod_n >= P.prod_cap) return;
    cudaEventRecord(P.prod_ev[2 * P.prod_n + end], s);
    if (end) P.prod_n++;
}

bd_status set_error(bd_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

bd_status check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return BD_OK;
}


template <typename T>
static bd_status dmalloc(Plan &P, T **ptr, size_t count)
{
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return set_error(BD_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    P.scratch_bytes += (int64_t)bytes;
    return BD_OK;
}

static void free_plan(Plan &P)
{
    if (P.prod_ev) {
        for (int i = 0; i < 2 * P.prod_cap; i++) cudaEventDestroy(P.prod_ev[i]);
        delete[] P.prod_ev;
        P.prod_ev = nullptr;
    }
    void *ptrs[] = {P.d_kvec, P.d_km64, P.d_km32, P.d_xsplit, P.d_ewc, P.d_ew64, P.d_ew32,
                    P.d_pw64, P.d_pw32, P.d_tab, P.d_tab32, P.d_cos, P.d_sin, P.d_cos32, P.d_sin32, P.d_F, P.d_DF,
                    P.d_Rnew, P.d_V[0], P.d_V[1], P.d_V[2], P.d_X0, P.d_Y0, P.d_dS, P.d_dW,
                    P.d_coef, P.d_wdw, P.d_red, P.d_redpart, P.d_bounds, P.d_status, P.d_lq[0], P.d_lq[1],
                    P.d_lq[2], P.d_lab, P.d_x16, P.d_xscale, P.d_part, P.d_counters,
                    P.d_stats_scratch, P.d_y32, P.d_lag_bounds, P.d_pairw, P.d_step_ctr, P.d_vhist, P.d_xhist, P.d_ubuf[0], P.d_ubuf[1],
                    P.d_ubuf[2], P.d_ubuf[3], P.d_xdf, P.d_Uh, P.d_Ul, P.d_rtiles, P.d_kbasis, P.d_lanpart, P.d_mom, P.d_sfac, P.d_mfW, P.d_mfpart,
                    P.d_x32, P.d_rows_part, P.d_rows_rep, P.d_rows_items, P.d_rows_bar};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (P.h_est) cudaFreeHost(P.h_est);
    spectral_free(P);
    sym_plan_free(P);
    if (P.step_exec) cudaGraphExecDestroy(P.step_exec);
    if (P.step_graph) cudaGraphDestroy(P.step_graph);
    P.step_exec = nullptr;
    P.step_graph = nullptr;
}

static bd_status validate(const bd_params *p)
{
    if (!p) return set_error(BD_ERR_INVALID, "params is NULL");
    if (p->n_beads < 1) return set_error(BD_ERR_INVALID, "n_beads must be >= 1");
    if (p->beads_per_chain < 1 || p->n_beads % p->beads_per_chain != 0)
        return set_error(BD_ERR_INVALID, "n_beads must be a multiple of beads_per_chain >= 1");
    if ((int64_t)p->n_beads * 3 > (int64_t)1 << 20)
        return set_error(BD_ERR_UNSUPPORTED, "3N = %lld exceeds the library's limit 2^20",
                         (long long)p->n_beads * 3);
    if (!(p->box_L > 0.0)) return set_error(BD_ERR_INVALID, "box_L must be > 0");
    if (!(p->a >= 0.0) || !(2.0 * p->a < p->box_L))
        return set_error(BD_ERR_INVALID, "need 0 <= a and 2a < L (a=%g, L=%g)", p->a, p->box_L);
    if (!(p->alpha > 0.0)) return set_error(BD_ERR_INVALID, "alpha must be > 0");
    if (!(p->r_c > 0.0) || p->r_c / p->box_L > 64.0)
        return set_error(BD_ERR_INVALID, "r_c must satisfy 0 < r_c <= 64 L");
    if (p->n2max < 0 || p->n2max > (p->pme_grid > 0 ? (1 << 22) : 4096))
        return set_error(BD_ERR_INVALID, "n2max must be in [0, 4096] (2^22 with a mesh)");
    if (p->pme_grid < 0) return set_error(BD_ERR_INVALID, "pme_grid must be >= 0");
    if (p->pme_grid > 0) {
        int kmax = 0;
        while ((long)(kmax + 1) * (kmax + 1) <= p->n2max) kmax++;
        if (p->pme_grid % 8 != 0 || p->pme_grid > 512 || p->pme_grid < 2 * kmax + 2)
            return set_error(BD_ERR_INVALID, "pme_grid must be a multiple of 8, <= 512 and >= 2 "
                             "sqrt(n2max) + 2 = %d", 2 * kmax + 2);
        int r = p->pme_grid;
        for (int f : {2, 3, 5})
            while (r % f == 0) r /= f;
        if (r != 1)
            return set_error(BD_ERR_INVALID, "pme_grid must have no prime factor other than 2, 3, 5");
        if (p->pme_order < 4 || p->pme_order > 10 || p->pme_order > p->pme_grid)
            return set_error(BD_ERR_INVALID, "pme_order must be in [4, 10] and <= pme_grid");
        if (!(p->r_c < 0.5 * p->box_L))
            return set_error(BD_ERR_INVALID, "the spectral path needs r_c < L/2 (r_c=%g, L=%g)",
                             p->r_c, p->box_L);
    }
    if (p->spring != 0 && p->spring != 1)
        return set_error(BD_ERR_INVALID, "spring must be 0 (Hookean) or 1 (FENE)");
    if (p->spring == 1 && !(p->fene_b > 0.0))
        return set_error(BD_ERR_INVALID, "FENE needs fene_b > 0");
    if (p->ev_on && (!(p->d_star > 0.0) || !(p->r_ev >= 0.0) || p->r_ev / p->box_L > 64.0))
        return set_error(BD_ERR_INVALID, "excluded volume needs d_star > 0, 0 <= r_ev <= 64 L");
    if (p->precision < BD_FP64 || p->precision > BD_MIXED_BF16)
        return set_error(BD_ERR_INVALID, "unknown precision %d", p->precision);
    if (p->max_rhs < 1 || p->max_rhs > kMaxRhs)
        return set_error(BD_ERR_INVALID, "max_rhs must be in [1, %d]", kMaxRhs);
    if (p->max_cheb < 2 || p->max_cheb > kMaxCheb)
        return set_error(BD_ERR_INVALID, "max_cheb must be in [2, %d]", kMaxCheb);
    if (!(p->dt >= 0.0)) return set_error(BD_ERR_INVALID, "dt must be >= 0");
    return BD_OK;
}

}  // namespace bd

using namespace bd;

extern "C" {

const char *bd_last_error(void) { return g_err; }

const char *bd_version(void) { return "libbdgb 0.1 (sm_103a)"; }

uint64_t bd_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

bd_status bd_set_phase_events(bd_plan *plan, void *const *events, int32_t count)
{
    if (!plan) return set_error(BD_ERR_INVALID, "NULL plan");
    Plan &P = plan->P;
    if (!events) {
        P.phase_on = 0;
        return BD_OK;
    }
    if (count != BD_PHASE_EVENTS)
        return set_error(BD_ERR_INVALID, "phase events: count must be %d", BD_PHASE_EVENTS);
    for (int i = 0; i < BD_PHASE_EVENTS; i++) {
        if (!events[i]) return set_error(BD_ERR_INVALID, "phase event %d is NULL", i);
        P.phase_ev[i] = (cudaEvent_t)events[i];
    }
    P.phase_on = 1;
    return BD_OK;
}

bd_status bd_plan_create(const bd_params *params, bd_plan **out_plan)
{
    g_err[0] = 0;
    if (!out_plan) return set_error(BD_ERR_INVALID, "out_plan is NULL");
    *out_plan = nullptr;
    bd_status st = validate(params);
    if (st != BD_OK) return st;
    bd_plan *pl = new (std::nothrow) bd_plan();
    if (!pl) return set_error(BD_ERR_OOM, "host allocation failed");
    Plan &P = pl->P;
    memset(&P, 0, sizeof(P));
    P.p = *params;
    cudaGetDevice(&P.device);
    P.n = params->n_beads;
    P.n3 = 3 * P.n;
    P.ld = (P.n3 + kLdAlign - 1) / kLdAlign * kLdAlign;
    const size_t n3 = P.n3, R = params->max_rhs;
    const bool mixed = params->precision != BD_FP64;
#define TRY(x)                       \
    do {                             \
        st = (x);                    \
        if (st != BD_OK) goto fail;  \
    } while (0)
    TRY(dmalloc(P, &P.d_kvec, kMaxKvec));
    TRY(dmalloc(P, &P.d_km64, (size_t)12 * kMaxKvec));
    if (mixed) TRY(dmalloc(P, &P.d_km32, (size_t)12 * kMaxKvec));
    if (mixed) TRY(dmalloc(P, &P.d_xsplit, 2 * n3));
    TRY(dmalloc(P, &P.d_ewc, 1));
    TRY(dmalloc(P, &P.d_ew64, 1));
    if (mixed) TRY(dmalloc(P, &P.d_ew32, 1));
    TRY(dmalloc(P, &P.d_pw64, n3));
    if (mixed) TRY(dmalloc(P, &P.d_pw32, 2 * n3));
    m1_table_range(P.p, TabFmt<double>::BITS, &P.tab_i0, &P.ntab);
    m1_table_range(P.p, TabFmt<float>::BITS, &P.tab32_i0, &P.ntab32);
    if (P.ntab > kTabMax || (mixed && P.ntab32 > kTabMax)) {
        st = set_error(BD_ERR_UNSUPPORTED, "r_c/a ratio needs %d table intervals (limit %d)",
                       mixed ? P.ntab32 : P.ntab, kTabMax);
        goto fail;
    }
    TRY(dmalloc(P, &P.d_tab, (size_t)(P.ntab > 0 ? P.ntab : 1) * TabFmt<double>::STRIDE));
    if (mixed)
        TRY(dmalloc(P, &P.d_tab32, (size_t)(P.ntab32 > 0 ? P.ntab32 : 1) * TabFmt<float>::STRIDE));
    TRY(dmalloc(P, &P.d_F, n3));
    TRY(dmalloc(P, &P.d_DF, n3));
    TRY(dmalloc(P, &P.d_Rnew, n3));
    for (int i = 0; i < 3; i++) TRY(dmalloc(P, &P.d_V[i], n3 * R));
    TRY(dmalloc(P, &P.d_X0, n3 * (R + 3)));
    TRY(dmalloc(P, &P.d_Y0, n3 * (R + 3)));
    TRY(dmalloc(P, &P.d_lag_bounds, 2));
    TRY(dmalloc(P, &P.d_pairw, 2));
    TRY(dmalloc(P, &P.d_step_ctr, 1));
    TRY(dmalloc(P, &P.d_dS, n3 * R));
    TRY(dmalloc(P, &P.d_dW, n3 * R));
    TRY(dmalloc(P, &P.d_coef, kMaxCheb + 2));
    TRY(dmalloc(P, &P.d_wdw, kMaxRhs));
    TRY(dmalloc(P, &P.d_red, 4 * kMaxRhs));
    TRY(dmalloc(P, &P.d_redpart, (size_t)kRedBlocks * kMaxRhs));
    TRY(dmalloc(P, &P.d_bounds, 2));
    TRY(dmalloc(P, &P.d_status, 8));
    for (int i = 0; i < 3; i++) TRY(dmalloc(P, &P.d_lq[i], n3));
    TRY(dmalloc(P, &P.d_lab, 2 * kMaxLanczos));
    TRY(dmalloc(P, &P.d_stats_scratch, 1));
    {
        cudaStream_t s = 0;
        launch_kvec_table(P, s);
        if (P.nk > kMaxKvec && P.p.pme_grid > 0) {
            P.nk = 0;            // mesh plan with a k-sphere too large for the dense tables:
            P.dense_off = 1;     // only matrix-free (spectral) products
        }
        if (P.nk > kMaxKvec) {
            st = set_error(BD_ERR_UNSUPPORTED, "%d half-space k-vectors exceed the limit %d",
                           P.nk, kMaxKvec);
            goto fail;
        }
        TRY(check_launch("plan tables"));
        size_t nkn = (size_t)(P.nk > 0 ? P.nk : 1) * P.n;
        TRY(dmalloc(P, &P.d_cos, nkn));
        TRY(dmalloc(P, &P.d_sin, nkn));
        if (mixed) {
            TRY(dmalloc(P, &P.d_cos32, nkn));
            TRY(dmalloc(P, &P.d_sin32, nkn));
            TRY(tc_plan_init(P));
            TRY(recip_tc_init(P));
        }
        if (P.p.pme_grid > 0) TRY(spectral_init(P));
        cudaMemset(P.d_step_ctr, 0, sizeof(unsigned long long));
        if (cudaDeviceSynchronize() != cudaSuccess) {
            st = check_launch("plan creation");
            goto fail;
        }
    }
#undef TRY
    *out_plan = pl;
    return BD_OK;
fail:
    free_plan(P);
    delete pl;
    return st;
}

void bd_plan_destroy(bd_plan *plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan(plan->P);
    delete plan;
}

bd_status bd_plan_query(const bd_plan *plan, bd_plan_info *info)
{
    if (!plan || !info) return set_error(BD_ERR_INVALID, "NULL argument");
    const Plan &P = plan->P;
    info->n3 = P.n3;
    info->ld = P.ld;
    info->d_bytes = (int64_t)P.n3 * P.ld * (is_mixed(P) ? 6 : 8);
    info->n_kvec = P.nk;
    info->precision = P.p.precision;
    info->scratch_bytes = P.scratch_bytes;
    return BD_OK;
}

bd_status bd_forces(bd_plan *plan, const double *R, double *F, int32_t *n_bad, bd_stream stream)
{
    if (!plan || !R || !F) return set_error(BD_ERR_INVALID, "NULL argument");
    if (n_bad) cudaMemsetAsync(n_bad, 0, sizeof(int32_t), stream);
    launch_forces(plan->P, R, F, n_bad, stream);
    return check_launch("bd_forces");
}

static void split_mixed(const Plan &P, void *D, float **D32, void **D16)
{
    *D32 = (float *)D;
    *D16 = (void *)((char *)D + (size_t)P.n3 * P.ld * 4);
}

bd_status bd_build_D(bd_plan *plan, const double *R, void *D, bd_stream stream)
{
    if (!plan || !R || !D) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (P.dense_off)
        return set_error(BD_ERR_UNSUPPORTED, "this mesh plan's k-sphere exceeds the dense tables; "
                         "use matrix-free products");
    if (((uintptr_t)D & 255) != 0) return set_error(BD_ERR_INVALID, "D must be 256-byte aligned");
    if (!is_mixed(P)) {
        launch_build_D_f64(P, R, (double *)D, stream);
    } else {
        float *D32;
        void *D16;
        split_mixed(P, D, &D32, &D16);
        bd_status st = launch_build_D_f32(P, R, D32, D16, P.p.precision == BD_MIXED_BF16, stream);
        if (st != BD_OK) return st;
    }
    return check_launch("bd_build_D");
}

// Y = D X for the plan's precision (no refinement)
static bd_status apply_core(Plan &P, const void *D, const double *X, int m, double *Y,
                            int flags, cudaStream_t s)
{
    if (P.matfree_R) {        // inside a matrix-free step: recompute D(R) X (FP32 or FP64)
        (void)D;
        (void)flags;
        return matfree_product(P, X, m, Y, s);
    }
    if (!is_mixed(P)) {
        launch_gemm_f64(P, (const double *)D, X, m, Y, s);
        return check_launch("gemm_f64");
    }
    float *D32;
    void *D16;
    split_mixed(P, (void *)D, &D32, &D16);
    bd_status st = P.tc_split == kRowsShape && m <= kRowsMaxCols ? rows_apply(P, D16, X, m, Y, s)
                                                                   : tc_apply(P, D16, X, m, Y, s);
    if (st != BD_OK) return st;
    if (flags & BD_APPLY_REFINE) {
        launch_refine_f32(P, D32, X, m, Y, s);
        return check_launch("refine");
    }
    return BD_OK;
}

}  // extern "C"

namespace bd {
bd_status apply_dense(Plan &P, const void *D, const double *X, int m, double *Y, cudaStream_t s)
{
    return apply_core(P, D, X, m, Y, 0, s);
}
}  // namespace bd

extern "C" {

bd_status bd_apply_D(bd_plan *plan, const void *D, const double *X, int32_t m, double *Y,
                     int32_t flags, bd_stream stream)
{
    if (!plan || !D || !X || !Y) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (m < 1 || m > P.p.max_rhs) return set_error(BD_ERR_INVALID, "m=%d outside [1, max_rhs=%d]", m, P.p.max_rhs);
    const char *xb = (const char *)X, *yb = (const char *)Y;
    size_t bytes = (size_t)P.n3 * m * sizeof(double);
    if (xb < yb + bytes && yb < xb + bytes) return set_error(BD_ERR_INVALID, "X and Y overlap");
    return apply_core(P, D, X, m, Y, flags, stream);
}

// where the pair estimate of lambda_min comes from (pair_bound.cuh)
enum PairSource { kPairNone = 0, kPairFromBuild = 1, kPairScanD = 2 };

// Lanczos bounds, then d_min = min(d_min, f theta_pair) unless pair == kPairNone
static bd_status eig_bounds_core(Plan &P, const void *D, int iters, double smax, double fmin_,
                                 double *bounds, int32_t *status, cudaStream_t s,
                                 int pair = kPairScanD)
{
    int k = iters < P.n3 ? iters : P.n3;
    if (pair == kPairScanD) launch_pair_radius_scan(D, is_mixed(P), P.n, P.ld, P.d_pairw, s);
    launch_lanczos_init(P, s);
    for (int j = 0; j < k; j++) {
        bd_status st = apply_core(P, D, P.d_lq[1], 1, P.d_lq[2], 0, s);
        if (st != BD_OK) return st;
        launch_lanczos_update(P, j, s);
    }
    launch_lanczos_finish(P, k, smax, fmin_, bounds, status, s);
    if (pair != kPairNone) launch_bounds_pair(bounds, P.d_pairw, fmin_, status, s);
    return check_launch("bd_eig_bounds");
}

bd_status bd_eig_bounds(bd_plan *plan, const void *D, int32_t iters, double safety_max,
                        double dmin_fraction, double *bounds, int32_t *status, bd_stream stream)
{
    if (!plan || !D || !bounds) return set_error(BD_ERR_INVALID, "NULL argument");
    if (iters < 1 || iters > kMaxLanczos)
        return set_error(BD_ERR_INVALID, "iters must be in [1, %d]", kMaxLanczos);
    if (!(safety_max >= 0.0) || !(dmin_fraction > 0.0) || !(dmin_fraction <= 1.0))
        return set_error(BD_ERR_INVALID, "need safety_max >= 0 and 0 < dmin_fraction <= 1");
    return eig_bounds_core(plan->P, D, iters, safety_max, dmin_fraction, bounds, status, stream);
}

// parts of a Chebyshev series / of a step: the batch runs the front of every
// replica, then all replicas' loops in one launch, then the backs
enum StepPart { kPartAll = 0, kPartFront = 1, kPartBack = 2 };

// the plan's products run the whole loop in one launch (shape 5, dense D)
static bool rows_loop(const Plan &P) { return is_mixed(P) && !P.matfree_R && P.tc_split == kRowsShape; }

// Chebyshev recurrence given W = D dW; dS and E_f outputs.  kPartFront stops
// after V_1 (and, in shape 5, writes the loop's table entry to *slot);
// kPartBack runs only E_f.
static bd_status cheb_core(Plan &P, const void *D, const double *bounds, int nch,
                           const double *dW, const double *W, int m, double *dS, double *Ef,
                           bd_step_stats *stats, cudaStream_t s, int lanczos_from = -1,
                           int part = kPartAll, RowsRep *slot = nullptr, int item0 = 0)
{
    // lanczos_from >= 0: a Lanczos recurrence (its step lanczos_from already
    // taken) rides as an extra column of every product (mixed plans only)
    if (part == kPartBack) {
        launch_ef(P, dW, W, dS, m, Ef, stats, s);
        return check_launch("chebyshev");
    }
    launch_cheb_coeffs(P, bounds, nch, s);
    double *A = P.d_V[0], *B = P.d_V[1];
    launch_cheb_first(P, bounds, dW, W, m, A, B, dS, s);   // A = V0, B = V1
    if (rows_loop(P)) {
        float *D32;
        void *D16;
        split_mixed(P, (void *)D, &D32, &D16);
        const int lan = lanczos_from >= 0 ? 1 : 0;
        RowsRep rep = rows_rep(P, D16, P.d_coef, bounds, m, lan, dS);
        rep.item0 = item0;
        rows_cheb_prepare(P, rep, slot ? slot : (RowsRep *)P.d_rows_rep, B, lan, s);
        if (part == kPartFront) return check_launch("chebyshev");
        bd_status st = rows_cheb_launch((const RowsRep *)P.d_rows_rep, 1, P.d_rows_items,
                                        rep.nitems, m + lan, nch, lanczos_from, P.d_rows_bar,
                                        P.device, s);
        if (st != BD_OK) return st;
        launch_ef(P, dW, W, dS, m, Ef, stats, s);
        return check_launch("chebyshev");
    }
    double *prev2 = A, *prev1 = B;
    for (int p = 2; p < nch; p++) {
        if (P.matfree_R) {
            bd_status st = matfree_product(P, prev1, m, P.d_mfW, s);
            if (st != BD_OK) return st;
            launch_cheb_term(P, P.d_mfW, prev1, prev2, m, bounds, p, dS, s);
        } else if (!is_mixed(P)) {
            ChebEpi e{P.d_coef, bounds, p, prev2, prev1, dS};
            launch_gemm_f64_cheb(P, (const double *)D, m, e, s);
        } else {
            float *D32;
            void *D16;
            split_mixed(P, (void *)D, &D32, &D16);
            const int lan_step = lanczos_from >= 0 ? lanczos_from + (p - 1) : -1;
            bd_status st = tc_cheb(P, D16, m, P.d_coef, bounds, p, prev2, prev1, dS, s, lan_step);
            if (st != BD_OK) return st;
        }
        double *t = prev2;   // prev2 now holds V_p
        prev2 = prev1;
        prev1 = t;
    }
    launch_ef(P, dW, W, dS, m, Ef, stats, s);
    return check_launch("chebyshev");
}

bd_status bd_chebyshev_sqrt(bd_plan *plan, const void *D, const double *bounds, int32_t n_cheb,
                            const double *dW, int32_t m, double *dS, double *Ef,
                            bd_stream stream)
{
    if (!plan || !D || !bounds || !dW || !dS) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (m < 1 || m > P.p.max_rhs) return set_error(BD_ERR_INVALID, "m=%d outside [1, max_rhs=%d]", m, P.p.max_rhs);
    if (n_cheb < 2 || n_cheb > P.p.max_cheb)
        return set_error(BD_ERR_INVALID, "n_cheb=%d outside [2, max_cheb=%d]", n_cheb, P.p.max_cheb);
    bd_status st = apply_core(P, D, dW, m, P.d_V[2], 0, stream);
    if (st != BD_OK) return st;
    return cheb_core(P, D, bounds, n_cheb, dW, P.d_V[2], m, dS, Ef, nullptr, stream);
}

bd_status bd_chebyshev_sqrt_adaptive(bd_plan *plan, const void *D, const double *bounds,
                                     double ef_tol, const double *dW, int32_t m, double *dS,
                                     double *Ef, int32_t *n_used, bd_stream stream)
{
    if (!plan || !D || !bounds || !dW || !dS) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (m < 1 || m > P.p.max_rhs) return set_error(BD_ERR_INVALID, "m=%d outside [1, max_rhs=%d]", m, P.p.max_rhs);
    if (!(ef_tol > 0.0)) return set_error(BD_ERR_INVALID, "ef_tol must be > 0");
    if (P.p.max_cheb < 2) return set_error(BD_ERR_INVALID, "plan max_cheb < 2");
    bd_status st = apply_core(P, D, dW, m, P.d_V[2], 0, stream);
    if (st != BD_OK) return st;
    int N = 0, conv = 0;
    st = cheb_adaptive_core(P, D, bounds, ef_tol, dW, P.d_V[2], m, dS, Ef, nullptr, stream, &N,
                            &conv);
    if (n_used) *n_used = N;
    if (st != BD_OK) return st;
    if (!conv)
        return set_error(BD_ERR_CHEB_NOCONV, "E_f >= %g with max_cheb = %d terms", ef_tol, N);
    return BD_OK;
}

bd_status bd_apply_D_matfree(bd_plan *plan, const double *R, const double *X, int32_t m,
                             double *Y, bd_stream stream)
{
    if (!plan || !R || !X || !Y) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (m < 1 || m > P.p.max_rhs + 3)
        return set_error(BD_ERR_INVALID, "m=%d outside [1, max_rhs + 3 = %d]", m, P.p.max_rhs + 3);
    const char *xb = (const char *)X, *yb = (const char *)Y;
    const size_t bytes = (size_t)P.n3 * m * sizeof(double);
    if (xb < yb + bytes && yb < xb + bytes) return set_error(BD_ERR_INVALID, "X and Y overlap");
    bd_status st = matfree_init(P);
    if (st != BD_OK) return st;
    st = launch_matfree_tables(P, R, stream);
    if (st != BD_OK) return st;
    return matfree_product(P, X, m, Y, stream);
}

bd_status bd_product_timing(bd_plan *plan, int32_t enable, float *total_ms, int32_t *launches)
{
    if (!plan) return set_error(BD_ERR_INVALID, "NULL plan");
    Plan &P = plan->P;
    if (enable) {
        if (!P.prod_ev) {
            P.prod_cap = 1024;
            P.prod_ev = new (std::nothrow) cudaEvent_t[2 * P.prod_cap];
            if (!P.prod_ev) return set_error(BD_ERR_OOM, "host allocation failed");
            for (int i = 0; i < 2 * P.prod_cap; i++) cudaEventCreate(&P.prod_ev[i]);
        }
        P.prod_n = 0;
        P.prod_on = 1;
        return check_launch("bd_product_timing");
    }
    float tot = 0.f;
    int n = P.prod_on ? P.prod_n : 0;
    if (n > 0) {
        cudaEventSynchronize(P.prod_ev[2 * n - 1]);
        for (int i = 0; i < n; i++) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, P.prod_ev[2 * i], P.prod_ev[2 * i + 1]);
            tot += ms;
        }
    }
    P.prod_on = 0;
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    return check_launch("bd_product_timing");
}

bd_status bd_plan_autotune(bd_plan *plan, void *D, int32_t *split_out, float *ms_out,
                           bd_stream stream)
{
    if (!plan || !D) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (!is_mixed(P)) {
        if (split_out) *split_out = 0;
        if (ms_out) *ms_out = 0.f;
        return BD_OK;
    }
    float *D32;
    void *D16;
    split_mixed(P, D, &D32, &D16);
    int best = 0;
    float ms = 0.f;
    bd_status st = tc_autotune(P, D16, stream, &best, &ms);
    if (split_out) *split_out = best;
    if (ms_out) *ms_out = ms;
    return st;
}

bd_status bd_plan_set_shape(bd_plan *plan, int32_t shape)
{
    if (!plan) return set_error(BD_ERR_INVALID, "NULL plan");
    if (shape < 0 || shape > kRowsShape) return set_error(BD_ERR_INVALID, "shape %d outside 0..5", shape);
    Plan &P = plan->P;
    if (!is_mixed(P) && shape == kRowsShape) shape = 0;
    if (!is_mixed(P)) {
        // FP64 plans: 4 selects the double-float products, anything else DFMA
        if (shape == kF64DoubleFloat && !P.d_xdf) {
            bd_status st = dmalloc(P, &P.d_xdf, (size_t)2 * kMaxRhs * P.n3);   // a step's products carry up to kMaxRhs columns
            if (st != BD_OK) return st;
        }
        P.tc_split = shape == kF64DoubleFloat ? shape : 0;
        return BD_OK;
    }
    if (shape == kF64DoubleFloat) return set_error(BD_ERR_INVALID, "shape 4 is for FP64 plans");
    if (shape == kRowsShape) {
        // a step's first product carries m + 4 columns at most (F, the Lanczos
        // vector, Fixman's two vectors)
        if (P.p.max_rhs + 4 > kRowsMaxCols)
            return set_error(BD_ERR_INVALID, "shape 5 needs max_rhs <= %d", kRowsMaxCols - 4);
        bd_status st = rows_plan_init(P);
        if (st != BD_OK) return st;
    }
    if (shape == kSymShape) {
        bd_status st = sym_plan_init(P);
        if (st != BD_OK) return st;
    }
    P.tc_split = shape;
    return BD_OK;
}

bd_status bd_plan_test_stall(bd_plan *plan, int32_t cta, int32_t term)
{
    if (!plan) return set_error(BD_ERR_INVALID, "NULL plan");
    Plan &P = plan->P;
    if (cta < 0) {
        P.test_stall = 0;
        P.test_stall_term = 0;
        return BD_OK;
    }
    if (term < 0) return set_error(BD_ERR_INVALID, "term %d < 0", term);
    if (!is_mixed(P) || P.tc_split != kSymShape)
        return set_error(BD_ERR_INVALID, "the stall hook needs a mixed plan in the symmetric shape");
    if (cta >= P.num_sms) return set_error(BD_ERR_INVALID, "cta %d outside the product's grid", cta);
    P.test_stall = cta + 1;
    P.test_stall_term = term;
    return BD_OK;
}

bd_status bd_step_capture(bd_plan *plan, double *R, void *D, const bd_step_opts *opts,
                          double *DF, double *dS, bd_step_stats *stats, bd_stream stream)
{
    if (!plan || !opts) return set_error(BD_ERR_INVALID, "NULL argument");
    if (opts->n_cheb == 0)
        return set_error(BD_ERR_INVALID, "adaptive N_Ch synchronises the host: not capturable");
    if (opts->flags & BD_STEP_MATRIX_FREE)
        return set_error(BD_ERR_INVALID, "matrix-free steps synchronise the host: not capturable");
    Plan &P = plan->P;
    if (P.step_exec) cudaGraphExecDestroy(P.step_exec);
    if (P.step_graph) cudaGraphDestroy(P.step_graph);
    P.step_exec = nullptr;
    P.step_graph = nullptr;
    bd_step_opts o = *opts;
    o.flags |= BD_STEP_DEVICE_COUNTER;
    const int phase_on = P.phase_on, prod_on = P.prod_on;
    P.phase_on = 0;
    P.prod_on = 0;
    (void)stream;
    // recorded on a private stream (the legacy default stream cannot be
    // captured; nothing runs during a capture)
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        P.phase_on = phase_on;
        P.prod_on = prod_on;
        if (s) cudaStreamDestroy(s);
        cudaGetLastError();
        return set_error(BD_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    }
    bd_status st = bd_step(plan, R, D, nullptr, &o, DF, dS, stats, (bd_stream)s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    P.phase_on = phase_on;
    P.prod_on = prod_on;
    if (st != BD_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (st != BD_OK) return st;
        return set_error(BD_ERR_CUDA, "stream capture of the step: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return set_error(BD_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
    }
    P.step_graph = g;
    P.step_exec = x;
    return BD_OK;
}

bd_status bd_step_replay(bd_plan *plan, bd_stream stream)
{
    if (!plan) return set_error(BD_ERR_INVALID, "NULL plan");
    Plan &P = plan->P;
    if (!P.step_exec) return set_error(BD_ERR_INVALID, "no captured step (bd_step_capture)");
    cudaError_t e = cudaGraphLaunch(P.step_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(BD_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return BD_OK;
}

bd_status bd_plan_set_step_counter(bd_plan *plan, uint64_t value, bd_stream stream)
{
    if (!plan) return set_error(BD_ERR_INVALID, "NULL plan");
    static thread_local unsigned long long hv;
    hv = value;
    cudaMemcpyAsync(plan->P.d_step_ctr, &hv, sizeof(hv), cudaMemcpyHostToDevice, stream);
    cudaStreamSynchronize(stream);
    return check_launch("bd_plan_set_step_counter");
}

bd_status bd_wiener(bd_plan *plan, uint64_t seed, uint64_t step_index, int64_t count,
                    double *out, bd_stream stream)
{
    if (!plan || !out || count < 0) return set_error(BD_ERR_INVALID, "bad argument");
    if (count == 0) return BD_OK;
    launch_wiener(plan->P, seed, step_index, count, out, stream);
    return check_launch("bd_wiener");
}

}  // extern "C"

namespace bd {

// the end of a step after its Chebyshev series: the lagged Lanczos bounds of
// the next step, the Euler update with FENE rejection, the drift copy-out
static bd_status step_finish(Plan &P, const StepCtx &c, cudaStream_t s)
{
    if (c.lag) {             // N_Ch - 1 Lanczos steps -> bounds of the next step
        launch_lanczos_finish(P, c.nch - 1, c.bound_safety, c.dmin_fraction, P.d_lag_bounds,
                              nullptr, s);
        P.lag_valid = 1;
    }
    if (P.phase_on) cudaEventRecord(P.phase_ev[5], s);
    // (a8) Euler update with FENE rejection
    launch_euler(P, c.R, c.DFd, c.dSd, c.st_dev, s);
    if (P.phase_on) cudaEventRecord(P.phase_ev[6], s);
    if (c.DF) launch_copy_f64(c.DF, c.DFd, (size_t)P.n3, s);
    return check_launch("bd_step");
}

static bd_status step_run(bd_plan *plan, double *R, void *D, const double *dW,
                          const bd_step_opts *o, double *DF, double *dS, bd_step_stats *stats,
                          cudaStream_t stream, int part, RowsRep *slot, int item0);

bool step_batchable(bd_plan *plan, const bd_step_opts *o)
{
    const Plan &P = plan->P;
    return o && is_mixed(P) && P.tc_split == kRowsShape && o->n_cheb >= 3 &&
           !(o->flags & BD_STEP_MATRIX_FREE) && o->m >= 1 && o->m + 1 <= kRowsMaxCols;
}

int step_part_lag(bd_plan *plan) { return plan->P.step_ctx.lag; }
int step_part_items(bd_plan *plan) { return rows_items(plan->P.n3); }
int plan_device(bd_plan *plan) { return plan->P.device; }

bd_status step_part(bd_plan *plan, double *R, void *D, const bd_step_opts *o,
                    bd_step_stats *stats, cudaStream_t s, int part, RowsRep *slot, int item0)
{
    if (part == kPartBack) {
        Plan &P = plan->P;
        const StepCtx &c = P.step_ctx;
        bd_status st = cheb_core(P, c.D, P.d_bounds, c.nch, c.w, c.Wcols, c.m, c.dSd, nullptr,
                                 c.st_dev, s, c.lag ? 0 : -1, kPartBack);
        if (st != BD_OK) return st;
        return step_finish(P, c, s);
    }
    return step_run(plan, R, D, nullptr, o, nullptr, nullptr, stats, s, part, slot, item0);
}

}  // namespace bd

extern "C" {

bd_status bd_step(bd_plan *plan, double *R, void *D, const double *dW, const bd_step_opts *o,
                  double *DF, double *dS, bd_step_stats *stats, bd_stream stream)
{
    return step_run(plan, R, D, dW, o, DF, dS, stats, stream, kPartAll, nullptr, 0);
}

}  // extern "C"

namespace bd {

static bd_status step_run(bd_plan *plan, double *R, void *D, const double *dW,
                          const bd_step_opts *o, double *DF, double *dS, bd_step_stats *stats,
                          cudaStream_t stream, int part, RowsRep *slot, int item0)
{
    if (!plan || !R || !o) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    const bool matfree = (o->flags & BD_STEP_MATRIX_FREE) != 0;
    if (!D && !matfree) return set_error(BD_ERR_INVALID, "NULL D (needs BD_STEP_MATRIX_FREE)");
    const int m = o->m;
    if (m < 1 || m > P.p.max_rhs) return set_error(BD_ERR_INVALID, "m=%d outside [1, max_rhs=%d]", m, P.p.max_rhs);
    const bool adaptive = o->n_cheb == 0;
    if (!adaptive && (o->n_cheb < 2 || o->n_cheb > P.p.max_cheb))
        return set_error(BD_ERR_INVALID, "n_cheb outside [2, max_cheb] (0: adaptive)");
    if (adaptive && !(o->ef_tol > 0.0))
        return set_error(BD_ERR_INVALID, "adaptive N_Ch (n_cheb = 0) needs ef_tol > 0");
    const int fix = (o->bounds_mode == BD_BOUNDS_FIXMAN_DILUTE ||
                     o->bounds_mode == BD_BOUNDS_FIXMAN_SEMIDILUTE) ? o->bounds_mode : 0;
    if (o->bounds_mode < 0 || o->bounds_mode > BD_BOUNDS_FIXMAN_SEMIDILUTE)
        return set_error(BD_ERR_INVALID, "unknown bounds_mode %d", o->bounds_mode);
    if (fix == BD_BOUNDS_FIXMAN_SEMIDILUTE && !(o->fixman_c > 0.0))
        return set_error(BD_ERR_INVALID, "BD_BOUNDS_FIXMAN_SEMIDILUTE needs fixman_c > 0");
    if (o->lanczos_iters < 1 || o->lanczos_iters > kMaxLanczos)
        return set_error(BD_ERR_INVALID, "lanczos_iters outside [1, %d]", kMaxLanczos);
    if (!(o->bound_safety >= 0.0) || !(o->dmin_fraction > 0.0) || !(o->dmin_fraction <= 1.0))
        return set_error(BD_ERR_INVALID, "need bound_safety >= 0, 0 < dmin_fraction <= 1");
    if (!matfree && ((uintptr_t)D & 255) != 0)
        return set_error(BD_ERR_INVALID, "D must be 256-byte aligned");
    cudaStream_t s = stream;
    bd_step_stats *st_dev = stats ? stats : P.d_stats_scratch;
    if (matfree) {
        bd_status mst = matfree_init(P);
        if (mst != BD_OK) return mst;
    }
    // every product of a matrix-free step recomputes D(R) from the positions
    // at the start of the step (R changes only in the final update)
    struct MatfreeScope {
        Plan &P;
        MatfreeScope(Plan &p, const double *R, bool on) : P(p) { P.matfree_R = on ? R : nullptr; }
        ~MatfreeScope() { P.matfree_R = nullptr; }
    } mf_scope(P, R, matfree);
    const size_t n3 = P.n3;
    bd_status st;
#define PHASE(i) \
    do { if (P.phase_on) cudaEventRecord(P.phase_ev[i], s); } while (0)
    PHASE(0);
    launch_step_begin(st_dev, o->n_cheb, P.d_status, s);
    // (a1) forces; input over-stretch count in status word 2
    launch_forces(P, R, P.d_F, P.d_status + 2, s);
    PHASE(1);
    // (a2-a4) D(R), or the tables of the matrix-free products
    if (matfree) {
        st = launch_matfree_tables(P, R, s);
        if (st != BD_OK) return st;
        // the pair estimate of the bounds from D(R) (pair sums only; the
        // spectral path has no per-pair reciprocal tables)
        if (!P.pme && !fix) launch_pair_estimate(P, s);
    } else {
        st = bd_build_D(plan, R, D, s);
        if (st != BD_OK) return st;
    }
    PHASE(2);
    // (a6) bounds: fresh Lanczos, or the previous step's lagged recurrence
    const bool lag = !adaptive && !matfree && o->bounds_mode == BD_BOUNDS_LAGGED && is_mixed(P) &&
                     o->n_cheb >= 8 &&
                     o->n_cheb - 1 <= kMaxLanczos && m + 2 <= kMaxRhs;
    const bool lagged_now = lag && P.lag_valid;
    if (fix) {
        // Fixman's estimates come from the first product below
    } else if (lagged_now) {
        // the previous step's Lanczos bounds, d_min tightened by this step's
        // pair estimate (computed by the assembly above), and the statistics
        launch_bounds_lagged(P.d_bounds, P.d_lag_bounds, P.d_pairw, o->dmin_fraction,
                             P.d_status + 3, st_dev, s);
    } else {
        st = eig_bounds_core(P, D, o->lanczos_iters, o->bound_safety, o->dmin_fraction,
                             P.d_bounds, P.d_status + 3, s,
                             (matfree && P.pme) ? kPairNone : kPairFromBuild);
        if (st != BD_OK) return st;
    }
    if (!fix && !lagged_now) launch_stats_bounds(st_dev, P.d_bounds, P.d_status + 3, s);
    PHASE(3);
    // Wiener increments
    const double *w = dW;
    if (!w) {
        const bool dev_ctr = (o->flags & BD_STEP_DEVICE_COUNTER) != 0;
        launch_wiener(P, o->seed, o->step_index, (int64_t)n3 * m, P.d_dW, s,
                      dev_ctr ? P.d_step_ctr : nullptr);
        if (dev_ctr) launch_counter_add(P.d_step_ctr, s);
        w = P.d_dW;
    }
    // (a5) first product D [F, dW]  (one pass over D)
    double *Wcols;
    const int fcols = fix ? 2 : 0;         // Fixman's U+, U- ride along
    if (m + 1 + fcols <= kMaxRhs) {
        const int extra = lag ? 1 : 0;     // the Lanczos start vector q_1
        // X0 = [F, dW, q_1]
        if (lag) launch_lanczos_init(P, s);
        launch_copy3_f64(P.d_X0, P.d_F, n3, w, n3 * m, P.d_lq[1], lag ? n3 : 0, s);
        if (fix) launch_fixman_fill(P.d_X0 + n3 * (m + 1), n3, s);
        st = apply_core(P, D, P.d_X0, m + 1 + extra + fcols, P.d_Y0, 0, s);
        if (st != BD_OK) return st;
        Wcols = P.d_Y0 + n3;
        if (fix)
            launch_fixman_bounds(P, P.d_X0 + n3 * (m + 1), P.d_Y0 + n3 * (m + 1), fix,
                                 o->fixman_c, P.d_bounds, P.d_status + 3, s);
        if (is_mixed(P) && !matfree) {   // refine the drift column only
            launch_refine_f32(P, (const float *)D, P.d_F, 1, P.d_Y0, s);
        }
        if (lag)             // Lanczos step 0 from the product's last column (used in place)
            launch_lanczos_update(P, 0, s, P.d_Y0 + n3 * (m + 1));
    } else {
        st = apply_core(P, D, P.d_F, 1, P.d_Y0, BD_APPLY_REFINE, s);
        if (st != BD_OK) return st;
        st = apply_core(P, D, w, m, P.d_Y0 + n3, 0, s);
        if (st != BD_OK) return st;
        Wcols = P.d_Y0 + n3;
        if (fix) {
            double *X2 = P.d_X0 + n3 * (m + 1), *Y2 = P.d_Y0 + n3 * (m + 1);
            launch_fixman_fill(X2, n3, s);
            st = apply_core(P, D, X2, 2, Y2, 0, s);
            if (st != BD_OK) return st;
            launch_fixman_bounds(P, X2, Y2, fix, o->fixman_c, P.d_bounds, P.d_status + 3, s);
        }
    }
    if (fix) launch_stats_bounds(st_dev, P.d_bounds, P.d_status + 3, s);
    const double *DFd = P.d_Y0;
    PHASE(4);
    // (a7) Chebyshev
    double *dSd = dS ? dS : P.d_dS;
    StepCtx c{R, D, w, Wcols, dSd, st_dev, DFd, DF, m, o->n_cheb, lag ? 1 : 0, o->bound_safety,
              o->dmin_fraction};
#undef PHASE
    if (adaptive) {
        int N = 0, conv = 0;
        st = cheb_adaptive_core(P, D, P.d_bounds, o->ef_tol, w, Wcols, m, dSd, nullptr, st_dev, s,
                                &N, &conv);
    } else if (part == kPartFront) {
        // the batch runs every replica's loop in one launch, then the backs
        P.step_ctx = c;
        return cheb_core(P, D, P.d_bounds, o->n_cheb, w, Wcols, m, dSd, nullptr, st_dev, s,
                         lag ? 0 : -1, kPartFront, slot, item0);
    } else {
        st = cheb_core(P, D, P.d_bounds, o->n_cheb, w, Wcols, m, dSd, nullptr, st_dev, s,
                       lag ? 0 : -1);
    }
    if (st != BD_OK) return st;
    return step_finish(P, c, s);
}

}  // namespace bd

extern "C" {

static bd_status ensure_backward_scratch(Plan &P)
{
    // d_vhist may already exist (the adaptive Chebyshev series allocates it)
    size_t blk = (size_t)P.n3 * P.p.max_rhs;
    size_t hist = (size_t)(P.p.max_cheb - 1) * blk;
    bd_status st = BD_OK;
    if (!P.d_vhist) st = dmalloc(P, &P.d_vhist, hist);
    if (st == BD_OK && !P.d_xhist) st = dmalloc(P, &P.d_xhist, hist);
    for (int i = 0; i < 4 && st == BD_OK; i++)
        if (!P.d_ubuf[i]) st = dmalloc(P, &P.d_ubuf[i], blk);
    return st;
}

bd_status bd_apply_D_backward(bd_plan *plan, const double *R, const void *D, const double *F,
                              const double *gY, double *gR, double *gF, bd_stream stream)
{
    if (!plan || !R || !F || !gY || !gR) return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (gF) {
        if (!D) return set_error(BD_ERR_INVALID, "gF requested without D");
        bd_status st = apply_core(P, D, gY, 1, gF, BD_APPLY_REFINE, stream);
        if (st != BD_OK) return st;
    }
    launch_pair_adjoint(P, R, gY, F, 1, gR, stream);
    return check_launch("bd_apply_D_backward");
}

bd_status bd_chebyshev_backward(bd_plan *plan, const double *R, const void *D,
                                const double *bounds, int32_t n_cheb, const double *dW,
                                int32_t m, const double *gS, double *gR, double *gdW,
                                bd_stream stream)
{
    if (!plan || !R || !D || !bounds || !dW || !gS || !gR)
        return set_error(BD_ERR_INVALID, "NULL argument");
    Plan &P = plan->P;
    if (m < 1 || m > P.p.max_rhs) return set_error(BD_ERR_INVALID, "m=%d outside [1, max_rhs=%d]", m, P.p.max_rhs);
    if (n_cheb < 2 || n_cheb > P.p.max_cheb)
        return set_error(BD_ERR_INVALID, "n_cheb=%d outside [2, max_cheb=%d]", n_cheb, P.p.max_cheb);
    bd_status st = ensure_backward_scratch(P);
    if (st != BD_OK) return st;
    cudaStream_t s = stream;
    const long len = (long)P.n3 * m;
    const int N = n_cheb;
    double *W = P.d_ubuf[3];
    launch_cheb_coeffs(P, bounds, N, s);
    // forward history V_0 .. V_{N-2} (V_0 = dW, V_1 = Y V_0, V_p = 2 Y V_{p-1} - V_{p-2})
    double *Vh = P.d_vhist;
    cudaMemcpyAsync(Vh, dW, len * sizeof(double), cudaMemcpyDeviceToDevice, s);
    for (int p = 1; p <= N - 2; p++) {
        st = apply_core(P, D, Vh + (long)(p - 1) * len, m, W, 0, s);
        if (st != BD_OK) return st;
        launch_cheb_hist(W, Vh + (long)(p - 1) * len, p >= 2 ? Vh + (long)(p - 2) * len : nullptr,
                         len, bounds, p == 1 ? 1.0 : 2.0, 1.0, Vh + (long)p * len, s);
    }
    // adjoint recurrence: U_{N-1} = c_{N-1} h, U_p = c_p h + 2 Y U_{p+1} - U_{p+2},
    // X_{p-1} = (p == 1 ? 1 : 2) s U_p pairs with V_{p-1}
    double *Uq2 = nullptr, *Uq1 = nullptr;      // U_{p+2}, U_{p+1}
    double *bufs[3] = {P.d_ubuf[0], P.d_ubuf[1], P.d_ubuf[2]};
    for (int p = N - 1; p >= 1; p--) {
        double *Up = bufs[p % 3];
        if (p == N - 1) {
            launch_cheb_adj(gS, nullptr, nullptr, nullptr, len, bounds, P.d_coef, p, 0.0, 1.0, Up, s);
        } else {
            st = apply_core(P, D, Uq1, m, W, 0, s);
            if (st != BD_OK) return st;
            launch_cheb_adj(gS, W, Uq1, Uq2, len, bounds, P.d_coef, p, 2.0, 1.0, Up, s);
        }
        launch_scale_copy(Up, len, bounds, p == 1 ? 1.0 : 2.0, P.d_xhist + (long)(p - 1) * len, s);
        Uq2 = Uq1;
        Uq1 = Up;
    }
    if (gdW) {
        // U_0 = (c_0/2) h + Y U_1 - U_2
        st = apply_core(P, D, Uq1, m, W, 0, s);
        if (st != BD_OK) return st;
        launch_cheb_adj(gS, W, Uq1, Uq2, len, bounds, P.d_coef, 0, 1.0, 0.5, gdW, s);
    }
    launch_pair_adjoint(P, R, P.d_xhist, Vh, (N - 1) * m, gR, s);
    return check_launch("bd_chebyshev_backward");
}

}  // extern "C"
