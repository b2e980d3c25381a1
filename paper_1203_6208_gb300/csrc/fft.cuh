// fft.cuh -- 3-D mesh transforms of the spectral product (fft.cu).
#pragma once
#include "bd_internal.cuh"

namespace bd {

constexpr int kFftMaxK = 512;     // mesh points per edge

struct FftPlan {
    int K;                        // mesh points per edge, 2^a 3^b 5^c
    unsigned code32, code64;      // radix passes, 5 bits each from the low end (FP32, FP64)
    void *d_tw64, *d_tw32;        // e^{-2 pi i t/K}, t < K (FP64 and FP32 pairs)
};

// factor K and form the twiddle tables (BD_ERR_UNSUPPORTED for other K)
bd_status fft_plan_init(FftPlan &f, int K);
void fft_free(FftPlan &f);
// B real meshes [B][K][K][K] -> half spectra [B][K][K][K/2 + 1] (complex
// pairs of T), forward, unnormalised
template <typename T>
bd_status fft3_r2c(const FftPlan &f, const T *in, void *out, int B, cudaStream_t s);
// half spectra -> real meshes, inverse, unnormalised; overwrites `in`
template <typename T>
bd_status fft3_c2r(const FftPlan &f, void *in, T *out, int B, cudaStream_t s);

}  // namespace bd
