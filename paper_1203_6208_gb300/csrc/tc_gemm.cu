// tc_gemm.cu -- mixed-precision products (placeholder until the tcgen05
// kernel lands) and the FP64-residual refinement of D.F.
#include "tc_gemm.cuh"

namespace bd {

bd_status tc_plan_init(Plan &P)
{
    (void)P;
    return BD_OK;
}

bd_status tc_apply(Plan &P, const void *D16, const double *X, int m, double *Y, cudaStream_t s)
{
    (void)P; (void)D16; (void)X; (void)m; (void)Y; (void)s;
    return set_error(BD_ERR_UNSUPPORTED, "mixed-precision products are not built yet");
}

bd_status tc_cheb(Plan &P, const void *D16, int m, const double *coef, const double *bounds, int p,
                  double *Vprev2, const double *Vprev1, double *dS, cudaStream_t s)
{
    (void)P; (void)D16; (void)m; (void)coef; (void)bounds; (void)p; (void)Vprev2; (void)Vprev1;
    (void)dS; (void)s;
    return set_error(BD_ERR_UNSUPPORTED, "mixed-precision products are not built yet");
}

// one warp per row: r = sum_k D32[i][k] X[k][j] - Y[i][j] in FP64; Y += r
__global__ void k_refine(const float *__restrict__ D32, long ld, int n3,
                         const double *__restrict__ X, int m, double *__restrict__ Y)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n3) return;
    const float *row = D32 + (long)warp * ld;
    for (int j = 0; j < m; j++) {
        const double *x = X + (long)j * n3;
        double acc = 0.0;
        for (int k = lane; k < n3; k += 32) acc = fma((double)row[k], x[k], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            double y0 = Y[(long)j * n3 + warp];
            double r = acc - y0;
            Y[(long)j * n3 + warp] = y0 + r;
        }
    }
}

void launch_refine_f32(Plan &P, const float *D32, const double *X, int m, double *Y,
                       cudaStream_t s)
{
    long threads = (long)P.n3 * 32;
    k_refine<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(D32, P.ld, P.n3, X, m, Y);
    count_launches(1);
}

}  // namespace bd
