// sym_gemm.cuh -- the mixed-precision product Y = D16 X over the tiles on and
// above the diagonal of the symmetric 16-bit D.
#pragma once
#include "tc_common.cuh"

namespace bd {

// schedule and partial buffers of the symmetric product (plan scratch)
bd_status sym_plan_init(Plan &P);
void sym_plan_free(Plan &P);
// y += D32 x - y for one column from the FP32 D on and above the diagonal
// (x split into FP32 hi/lo words, xs[0 .. 3N) and xs[3N .. 6N))
bd_status sym_refine(Plan &P, const float *D32, const float *xs, double *y, cudaStream_t s);
// Y = D16 X16 with the epilogue e (plain store or Chebyshev term), from the
// tensor maps of D16 (128 x 64 boxes) and of X16 (64 x bn boxes); bn = 16 or 32
bd_status sym_launch(Plan &P, const CUtensorMap &mapD, const CUtensorMap &mapX, int bn,
                     const tc::Epi &e, cudaStream_t s);

}  // namespace bd
