// tc_gemm.cuh -- tensor-core (tcgen05) products of the mixed-precision plans
// and the FP64-residual refinement of the drift product.
#pragma once
#include "bd_internal.cuh"

namespace bd {

// allocate the 16-bit operand scratch and stream-K workspace of a mixed plan
bd_status tc_plan_init(Plan &P);
// Y = D16 X (FP32 accumulation, FP64 output)
bd_status tc_apply(Plan &P, const void *D16, const double *X, int m, double *Y, cudaStream_t s);
// launch shape 3 of the product: the symmetric kernel over the upper triangle
constexpr int kSymShape = 3;
// measure the fastest launch shape of the product (1 or 2 CTAs per SM of the
// stream-K kernel, or the symmetric kernel) (synchronous)
bd_status tc_autotune(Plan &P, const void *D16, cudaStream_t s, int *best, float *ms);
// one Chebyshev term: V_p = 2 (s D16 V_{p-1} - t V_{p-1}) - V_{p-2} (in place
// over V_{p-2}), dS += c_p V_p
// lan_step >= 0: the Lanczos vector q_j (P.d_lq[1]) rides as column m of the
// operand; the product's epilogue writes w = D16 q_j and its row-block dot
// partials, and one kernel then takes Lanczos step j (alpha_j, beta_j, q_{j+1})
bd_status tc_cheb(Plan &P, const void *D16, int m, const double *coef, const double *bounds, int p,
                  double *Vprev2, const double *Vprev1, double *dS, cudaStream_t s,
                  int lan_step = -1);
// one step of FP64-residual refinement: Y += (D32 X - Y), with the residual
// accumulated in FP64 from the FP32 matrix
void launch_refine_f32(Plan &P, const float *D32, const double *X, int m, double *Y,
                       cudaStream_t s);

}  // namespace bd
