// noalloc_bounds.cu -- bd_eig_bounds_noalloc: the Lanczos eigenvalue bounds
// of an FP64 diffusion matrix, for callers that cannot allocate device memory.
//
// bd_eig_bounds needs a plan, and creating a plan allocates (tables and
// scratch through cudaMalloc).  Some callers may not do that: a host
// framework that has already handed all of HBM to its own caching allocator
// and forbids raw cudaMalloc next to it, or a latency-critical loop where a
// cudaMalloc (which can synchronise the device) is not acceptable.  This
// entry point takes the matrix and its sizes directly and keeps its working
// vectors in a file-scope device array instead of allocating them.
//
// The array has a fixed size (kNoAllocMaxN3 rows, about 0.6 MB); every GPU
// that loads the library holds it until the process exits.  All calls share
// it and it keeps the last call's contents, so calls whose work overlaps on
// the GPU (different streams, or different host threads on one device) race
// and must be serialised by the caller.
#include <string.h>

#include <mutex>

#include "bd_internal.cuh"

namespace bd {

// largest 3N this entry point accepts (8192 beads)
constexpr int kNoAllocMaxN3 = 24576;
// q_{j-1}, q_j, w (3 x 3N), the tridiagonal alpha/beta (2 x kMaxLanczos), the
// reduction words (4 x kMaxRhs) and their per-block partials (kRedBlocks x
// kMaxRhs), laid out as in a plan, and one slot for the two pair-estimate words
constexpr size_t kNoAllocDoubles = 3 * (size_t)kNoAllocMaxN3 + 2 * kMaxLanczos + 4 * kMaxRhs +
                                   (size_t)kRedBlocks * kMaxRhs + 1;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// device address of the array per device (host code must not use the
// symbol's name as a device pointer: on the host it is only a stand-in)
static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[256];

static bd_status noalloc_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(BD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return set_error(BD_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(BD_ERR_CUDA, "cudaGetSymbolAddress(no-alloc scratch): %s",
                             cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return BD_OK;
}

}  // namespace bd

using namespace bd;

extern "C" bd_status bd_eig_bounds_noalloc(const double *D, int32_t n3, int32_t ld, int32_t iters,
                                           double safety_max, double dmin_fraction,
                                           double *bounds, int32_t *status, bd_stream stream)
{
    if (!D || !bounds) return set_error(BD_ERR_INVALID, "NULL argument");
    if (n3 < 3 || n3 % 3 != 0) return set_error(BD_ERR_INVALID, "n3=%d must be a positive multiple of 3", n3);
    if (n3 > kNoAllocMaxN3)
        return set_error(BD_ERR_UNSUPPORTED,
                         "n3=%d exceeds the no-allocation scratch limit of %d (8192 beads); "
                         "use bd_eig_bounds with a plan", n3, kNoAllocMaxN3);
    if (ld < n3) return set_error(BD_ERR_INVALID, "ld=%d < n3=%d", ld, n3);
    if (((uintptr_t)D & 7) != 0) return set_error(BD_ERR_INVALID, "D must be 8-byte aligned");
    if (iters < 1 || iters > kMaxLanczos)
        return set_error(BD_ERR_INVALID, "iters must be in [1, %d]", kMaxLanczos);
    if (!(safety_max >= 0.0) || !(dmin_fraction > 0.0) || !(dmin_fraction <= 1.0))
        return set_error(BD_ERR_INVALID, "need safety_max >= 0 and 0 < dmin_fraction <= 1");
    double *scr = nullptr;
    bd_status st = noalloc_scratch(&scr);
    if (st != BD_OK) return st;
    // a plan-shaped view onto the static array: only the sizes and the
    // Lanczos/reduction pointers are used by the launchers below
    Plan P;
    memset(&P, 0, sizeof(P));
    P.n3 = n3;
    P.n = n3 / 3;
    P.ld = ld;
    P.d_lq[0] = scr;
    P.d_lq[1] = scr + kNoAllocMaxN3;
    P.d_lq[2] = scr + 2 * (size_t)kNoAllocMaxN3;
    P.d_lab = scr + 3 * (size_t)kNoAllocMaxN3;
    P.d_red = P.d_lab + 2 * kMaxLanczos;
    P.d_redpart = P.d_red + 4 * kMaxRhs;
    unsigned *pair_word = (unsigned *)(scr + kNoAllocDoubles - 1);
    cudaStream_t s = stream;
    int k = iters < n3 ? iters : n3;
    // the pair estimate of lambda_min from D's blocks (clears its word first)
    launch_pair_radius_scan(D, 0, P.n, ld, pair_word, s);
    launch_lanczos_init(P, s);          // overwrites q and q_prev, clears its reduction word
    for (int j = 0; j < k; j++) {
        launch_gemm_f64(P, D, P.d_lq[1], 1, P.d_lq[2], s);
        launch_lanczos_update(P, j, s); // clears the words it accumulates into
    }
    launch_lanczos_finish(P, k, safety_max, dmin_fraction, bounds, status, s);
    launch_bounds_pair(bounds, pair_word, dmin_fraction, status, s);
    return check_launch("bd_eig_bounds_noalloc");
}
