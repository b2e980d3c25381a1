// recip_tc.cuh -- the reciprocal part of D as a tensor-core product (mixed
// plans): launchers.
#pragma once

#include <vector>

#include "bd_internal.cuh"

namespace bd {

// decides whether the plan can use the product (f(k) >= 0 on every k, a
// mixed plan with k-vectors) and allocates its operands; leaves P.recip_tc = 0
// otherwise
bd_status recip_tc_init(Plan &P);
// writes the reciprocal sum U U^T into the tiles of D32 on and above the
// diagonal (128 x 128 tiles); needs the trig tables of the current R
bd_status launch_recip_tc(Plan &P, float *D32, cudaStream_t s);

}  // namespace bd
