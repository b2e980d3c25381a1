// adaptive.cuh -- Chebyshev series with an adaptive number of terms (Sec. IV).
#pragma once
#include "bd_internal.cuh"

namespace bd {

// Y = D X for the plan's precision (no refinement); defined in bd_api.cu
bd_status apply_dense(Plan &P, const void *D, const double *X, int m, double *Y, cudaStream_t s);

// dS = P_N(D) dW with N from Eq. (nint) grown until E_f < tol (at most
// max_cheb); W = D dW.  Synchronises the stream.  *n_used = N, *converged = 1
// if E_f < tol was reached.  Ef (optional, m values) and stats (optional) get
// the direct E_f of the returned dS.
bd_status cheb_adaptive_core(Plan &P, const void *D, const double *bounds, double tol,
                             const double *dW, const double *W, int m, double *dS, double *Ef,
                             bd_step_stats *stats, cudaStream_t s, int *n_used, int *converged);

}  // namespace bd
