// adjoint.cuh -- launchers of the reverse-mode kernels (adjoint.cu).
#pragma once
#include "bd_internal.cuh"

namespace bd {

// gR = dL/dR for dL/dD = sum_q X_q Y_q^T (X, Y: [Q][3N]); gR is overwritten
void launch_pair_adjoint(Plan &P, const double *R, const double *X, const double *Y, int Q,
                         double *gR, cudaStream_t s);
// out = a (s DV - t V1) - b V2 (V2 may be NULL)
void launch_cheb_hist(const double *DV, const double *V1, const double *V2, long len,
                      const double *bounds, double a, double b, double *out, cudaStream_t s);
// out = cscale c_p h + a (s DU - t U1) - U2 (DU, U2 may be NULL)
void launch_cheb_adj(const double *h, const double *DU, const double *U1, const double *U2,
                     long len, const double *bounds, const double *coef, int p, double a,
                     double cscale, double *out, cudaStream_t s);
// dst = k s src, s = 2/(d_max - d_min)
void launch_scale_copy(const double *src, long len, const double *bounds, double k, double *dst,
                       cudaStream_t s);

}  // namespace bd
