// fft.cu -- the 3-D mesh transforms of the spectral product (Sec. VIII
// outlook: the Fourier part of the Ewald sum by FFT): a batch of real K^3
// meshes to their half spectra K x K x (K/2 + 1) and back, unnormalised
// (forward e^{-2 pi i jk/K}, inverse e^{+2 pi i jk/K}), K = 2^a 3^b 5^c.
//
// Each 1-D transform runs in shared memory as a Stockham (self-sorting)
// sequence of radix-4, 2, 3 and 5 passes: pass q with radix R and Ns = the
// product of the earlier radices reads R values K/R apart, turns them by the
// twiddles w^{r (j mod Ns) K/(Ns R)}, takes the R-point DFT and writes them Ns
// apart at (j div Ns) Ns R + (j mod Ns); the output is in natural order.
//   z (contiguous) : two real lines a, b form c = a + i b; after the complex
//                    transform A_k = (C_k + conj C_{-k})/2 and
//                    B_k = (C_k - conj C_{-k})/(2i), k = 0 .. K/2 (the inverse
//                    rebuilds C = A + i B from the Hermitian halves).
//   y, x (strided) : complex lines; a CTA takes 8 lines with consecutive k_z,
//                    so each of its loads covers 8 neighbouring complex values.
// Twiddles come from a per-mesh table e^{-2 pi i t/K}, t < K, formed once in
// FP64 with sincospi (an FP32 copy for mixed plans).
#include <math.h>

#include "fft.cuh"

namespace bd {

namespace ff {

constexpr int kThreads = 256;
// lines per CTA: complex values of 8 neighbouring lines make one 128-byte
// run in FP64, of 16 in FP32
template <typename T> __host__ __device__ constexpr int lines_per_cta() { return sizeof(T) == 8 ? 8 : 16; }

template <typename T> struct C2 { T x, y; };

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }
// multiply by sg * i
template <typename T> __device__ __forceinline__ C2<T> cmuli(C2<T> a, T sg) { return {-sg * a.y, sg * a.x}; }

// R-point DFTs, y_k = sum_t a_t e^{sg 2 pi i t k / R}
template <typename T, int R>
__device__ __forceinline__ void dft(C2<T> *a, T sg)
{
    if (R == 2) {
        const C2<T> t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    } else if (R == 4) {
        const C2<T> t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]), t2 = cadd(a[1], a[3]);
        const C2<T> t3 = cmuli(csub(a[1], a[3]), sg);
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    } else if (R == 3) {
        const T h3 = (T)0.86602540378443864676;             // sqrt(3)/2
        const C2<T> s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        const C2<T> h = {a[0].x - (T)0.5 * s.x, a[0].y - (T)0.5 * s.y};
        const C2<T> t = cmuli(C2<T>{h3 * d.x, h3 * d.y}, sg);
        a[0] = cadd(a[0], s);
        a[1] = cadd(h, t);
        a[2] = csub(h, t);
    } else {                                                 // R == 5
        const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;   // cos(2pi/5), cos(4pi/5)
        const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;    // sin(2pi/5), sin(4pi/5)
        const C2<T> b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
        const C2<T> d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
        const C2<T> r1 = {a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y};
        const C2<T> r2 = {a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y};
        const C2<T> i1 = cmuli(C2<T>{s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y}, sg);
        const C2<T> i2 = cmuli(C2<T>{s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y}, sg);
        a[0] = cadd(a[0], cadd(b1, b2));
        a[1] = cadd(r1, i1);
        a[4] = csub(r1, i1);
        a[2] = cadd(r2, i2);
        a[3] = csub(r2, i2);
    }
}

struct Radices {
    int n;
    int r[16];
};

// n / d and n % d for 0 <= n < 2^22 and a runtime d: the quotient from an
// FP32 reciprocal, corrected by one step either way (integer division would
// cost ~20 instructions per element in the load and store loops)
struct FastDiv {
    int d;
    float inv;
    __device__ explicit FastDiv(int d_) : d(d_), inv(1.0f / (float)d_) {}
    __device__ __forceinline__ int div(int n) const
    {
        int q = (int)((float)n * inv);
        const int r = n - q * d;
        q += r >= d ? 1 : (r < 0 ? -1 : 0);
        return q;
    }
};

// one Stockham pass of radix R over NL lines of length K (line stride K + 1
// in shared memory), src -> dst; consecutive threads take the same butterfly
// of consecutive lines (each thread keeps its line), so the padded stride
// spreads them over the banks.  Lines past nl compute on padding and are
// never written back.
template <typename T, int R, int NL>
__device__ __forceinline__ void fft_pass(const C2<T> *src, C2<T> *dst, const C2<T> *tw, int K,
                                         int Ns, T sg)
{
    const int nb = K / R;
    const int tstep = K / (Ns * R);
    const int KP = K + 1;
    const int line = threadIdx.x % NL;
    const C2<T> *s = src + (size_t)line * KP;
    C2<T> *dl = dst + (size_t)line * KP;
    // j = jd Ns + jm walked with an incremental (jd, jm): no division per butterfly
    int j = threadIdx.x / NL;
    constexpr int step = kThreads / NL;
    int jd = j / Ns, jm = j - jd * Ns;
    const int sd = step / Ns, sm = step - sd * Ns;
    for (; j < nb; j += step) {
        C2<T> a[R];
#pragma unroll
        for (int r = 0; r < R; r++) a[r] = s[j + r * nb];
        if (Ns > 1) {                     // the first pass has no twiddles
#pragma unroll
            for (int r = 1; r < R; r++) {
                C2<T> w = tw[r * jm * tstep];
                w.y *= -sg;               // the table holds e^{-2 pi i t/K}; sg = +1 conjugates
                a[r] = cmul(a[r], w);
            }
        }
        dft<T, R>(a, sg);
        C2<T> *d = dl + jd * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; r++) d[r * Ns] = a[r];
        jd += sd;
        jm += sm;
        if (jm >= Ns) {
            jm -= Ns;
            jd++;
        }
    }
}

// the transforms of the CTA's lines of length K held in buf0 ([line][K + 1]);
// returns the buffer that holds the result.  All threads of the CTA take part.
template <typename T>
__device__ C2<T> *fft_lines(C2<T> *buf0, C2<T> *buf1, const C2<T> *tw, int K,
                            const Radices &rd, T sg)
{
    constexpr int NL = lines_per_cta<T>();
    C2<T> *src = buf0, *dst = buf1;
    int Ns = 1;
    for (int q = 0; q < rd.n; q++) {
        const int R = rd.r[q];
        switch (R) {
        case 2: fft_pass<T, 2, NL>(src, dst, tw, K, Ns, sg); break;
        case 3: fft_pass<T, 3, NL>(src, dst, tw, K, Ns, sg); break;
        case 4: fft_pass<T, 4, NL>(src, dst, tw, K, Ns, sg); break;
        default: fft_pass<T, 5, NL>(src, dst, tw, K, Ns, sg); break;
        }
        __syncthreads();
        C2<T> *t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// forward z: pairs of real lines (2p, 2p + 1) -> their half spectra
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fft_z_r2c(const T *__restrict__ in, C2<T> *__restrict__ out, long npairs, int K,
            const C2<T> *__restrict__ twg, Radices rd)
{
    constexpr int kLines = lines_per_cta<T>();
    extern __shared__ __align__(16) unsigned char smem[];
    C2<T> *tw = (C2<T> *)smem;
    C2<T> *b0 = tw + K, *b1 = b0 + (size_t)kLines * (K + 1);
    const long p0 = (long)blockIdx.x * kLines;
    const int nl = (int)min((long)kLines, npairs - p0);
    const int H = K / 2 + 1;
    for (int t = threadIdx.x; t < K; t += blockDim.x) tw[t] = twg[t];
    const FastDiv dK(K), dH(H);
    // lines 2 p0 .. 2 (p0 + nl) - 1 are one contiguous run of reals
    const T *src = in + (size_t)2 * p0 * K;
    for (int e = threadIdx.x; e < 2 * nl * K; e += blockDim.x) {
        const int line = dK.div(e), k = e - line * K;
        const T v = src[e];
        C2<T> &c = b0[(size_t)(line >> 1) * (K + 1) + k];
        if (line & 1) c.y = v;
        else c.x = v;
    }
    __syncthreads();
    const C2<T> *res = fft_lines<T>(b0, b1, tw, K, rd, (T)-1);
    C2<T> *dst = out + (size_t)2 * p0 * H;
    for (int e = threadIdx.x; e < 2 * nl * H; e += blockDim.x) {
        const int line = dH.div(e), k = e - line * H;
        const C2<T> *c = res + (size_t)(line >> 1) * (K + 1);
        const C2<T> ck = c[k], cm = c[k ? K - k : 0];        // C_k, C_{-k}
        C2<T> v;
        if (line & 1) v = {(T)0.5 * (ck.y + cm.y), (T)-0.5 * (ck.x - cm.x)};   // (C_k - conj C_-k)/(2i)
        else v = {(T)0.5 * (ck.x + cm.x), (T)0.5 * (ck.y - cm.y)};             // (C_k + conj C_-k)/2
        dst[e] = v;
    }
}

// inverse z: pairs of half spectra -> their real lines (unnormalised)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fft_z_c2r(const C2<T> *__restrict__ in, T *__restrict__ out, long npairs, int K,
            const C2<T> *__restrict__ twg, Radices rd)
{
    constexpr int kLines = lines_per_cta<T>();
    extern __shared__ __align__(16) unsigned char smem[];
    C2<T> *tw = (C2<T> *)smem;
    C2<T> *b0 = tw + K, *b1 = b0 + (size_t)kLines * (K + 1);
    const long p0 = (long)blockIdx.x * kLines;
    const int nl = (int)min((long)kLines, npairs - p0);
    const int H = K / 2 + 1;
    for (int t = threadIdx.x; t < K; t += blockDim.x) tw[t] = twg[t];
    const FastDiv dK(K);
    const C2<T> *src = in + (size_t)2 * p0 * H;
    // C_k = A_k + i B_k over the whole line, the upper half from conjugates
    for (int e = threadIdx.x; e < nl * K; e += blockDim.x) {
        const int pr = dK.div(e), k = e - pr * K;
        const bool lo = k < H;
        const int kk = lo ? k : K - k;
        C2<T> a = src[(size_t)(2 * pr) * H + kk], b = src[(size_t)(2 * pr + 1) * H + kk];
        if (!lo) {
            a.y = -a.y;
            b.y = -b.y;
        }
        b0[(size_t)pr * (K + 1) + k] = {a.x - b.y, a.y + b.x};
    }
    __syncthreads();
    const C2<T> *res = fft_lines<T>(b0, b1, tw, K, rd, (T)1);
    T *dst = out + (size_t)2 * p0 * K;
    for (int e = threadIdx.x; e < 2 * nl * K; e += blockDim.x) {
        const int line = dK.div(e), k = e - line * K;
        const C2<T> c = res[(size_t)(line >> 1) * (K + 1) + k];
        dst[e] = (line & 1) ? c.y : c.x;
    }
}

// complex transforms along a strided axis, in place.  Line (o, z): element t
// at (o / q) A + (o % q) B + z + t S, z < H; a CTA takes kLines consecutive z
// of one o.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_fft_strided(C2<T> *__restrict__ data, int K, int H, int q, long A, long B, long S,
              const C2<T> *__restrict__ twg, Radices rd, T sg)
{
    constexpr int kLines = lines_per_cta<T>();
    extern __shared__ __align__(16) unsigned char smem[];
    C2<T> *tw = (C2<T> *)smem;
    C2<T> *b0 = tw + K, *b1 = b0 + (size_t)kLines * (K + 1);
    const int zt = (H + kLines - 1) / kLines;
    const long o = blockIdx.x / zt;
    const int z0 = (int)(blockIdx.x % zt) * kLines;
    const int nl = min(kLines, H - z0);
    C2<T> *base = data + (o / q) * A + (o % q) * B + z0;
    for (int t = threadIdx.x; t < K; t += blockDim.x) tw[t] = twg[t];
    for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
        const int t = e / kLines, l = e - t * kLines;
        if (l < nl) b0[(size_t)l * (K + 1) + t] = base[(size_t)t * S + l];
    }
    __syncthreads();
    const C2<T> *res = fft_lines<T>(b0, b1, tw, K, rd, sg);
    for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
        const int t = e / kLines, l = e - t * kLines;
        if (l < nl) base[(size_t)t * S + l] = res[(size_t)l * (K + 1) + t];
    }
}

__global__ void k_twiddles(int K, C2<double> *t64, C2<float> *t32)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    double s, c;
    sincospi(-2.0 * t / K, &s, &c);
    t64[t] = {c, s};
    t32[t] = {(float)c, (float)s};
}

template <typename T>
static size_t smem_bytes(int K) { return (size_t)(K + 2 * lines_per_cta<T>() * (K + 1)) * sizeof(C2<T>); }

}  // namespace ff

using namespace ff;

bd_status fft_plan_init(FftPlan &f, int K)
{
    f.K = K;
    int r = K, n = 0;
    while (r % 4 == 0 && n < 16) { f.rad[n++] = 4; r /= 4; }
    while (r % 2 == 0 && n < 16) { f.rad[n++] = 2; r /= 2; }
    while (r % 3 == 0 && n < 16) { f.rad[n++] = 3; r /= 3; }
    while (r % 5 == 0 && n < 16) { f.rad[n++] = 5; r /= 5; }
    if (r != 1 || K < 2 || K > kFftMaxK)
        return set_error(BD_ERR_UNSUPPORTED, "mesh size %d is not 2^a 3^b 5^c <= %d", K, kFftMaxK);
    f.nrad = n;
    cudaError_t e = cudaMalloc(&f.d_tw64, sizeof(C2<double>) * K);
    if (e == cudaSuccess) e = cudaMalloc(&f.d_tw32, sizeof(C2<float>) * K);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BD_ERR_OOM, "FFT twiddles: %s", cudaGetErrorString(e));
    }
    k_twiddles<<<(K + 127) / 128, 128>>>(K, (C2<double> *)f.d_tw64, (C2<float> *)f.d_tw32);
    count_launches(1);
    const size_t s64 = smem_bytes<double>(K), s32 = smem_bytes<float>(K);
    cudaError_t a[6] = {
        cudaFuncSetAttribute(k_fft_z_r2c<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64),
        cudaFuncSetAttribute(k_fft_z_c2r<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64),
        cudaFuncSetAttribute(k_fft_strided<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64),
        cudaFuncSetAttribute(k_fft_z_r2c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32),
        cudaFuncSetAttribute(k_fft_z_c2r<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32),
        cudaFuncSetAttribute(k_fft_strided<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32)};
    for (cudaError_t x : a)
        if (x != cudaSuccess) return set_error(BD_ERR_CUDA, "FFT smem attribute: %s", cudaGetErrorString(x));
    return check_launch("FFT plan");
}

void fft_free(FftPlan &f)
{
    if (f.d_tw64) cudaFree(f.d_tw64);
    if (f.d_tw32) cudaFree(f.d_tw32);
    f.d_tw64 = f.d_tw32 = nullptr;
}

template <typename T>
static void strided_passes(const FftPlan &f, C2<T> *q, int B, T sg, const C2<T> *tw,
                           const Radices &rd, cudaStream_t s, bool y_first)
{
    constexpr int kLines = lines_per_cta<T>();
    const int K = f.K, H = K / 2 + 1, zt = (H + kLines - 1) / kLines;
    const size_t sm = smem_bytes<T>(K);
    const long KH = (long)K * H;
    for (int pass = 0; pass < 2; pass++) {
        const bool ypass = (pass == 0) == y_first;
        if (ypass)   // lines (b, i0, z) along i1: stride H
            k_fft_strided<T><<<(unsigned)((long)B * K * zt), kThreads, sm, s>>>(q, K, H, 1, KH, 0, H, tw, rd, sg);
        else         // lines (b, i1, z) along i0: stride K H
            k_fft_strided<T><<<(unsigned)((long)B * K * zt), kThreads, sm, s>>>(q, K, H, K, K * KH, H, KH, tw, rd, sg);
    }
}

template <typename T>
bd_status fft3_r2c(const FftPlan &f, const T *in, void *out, int B, cudaStream_t s)
{
    Radices rd;
    rd.n = f.nrad;
    for (int i = 0; i < f.nrad; i++) rd.r[i] = f.rad[i];
    const int K = f.K;
    const C2<T> *tw = (const C2<T> *)(sizeof(T) == 8 ? f.d_tw64 : f.d_tw32);
    constexpr int kLines = lines_per_cta<T>();
    const long npairs = (long)B * K * K / 2;
    const size_t sm = smem_bytes<T>(K);
    k_fft_z_r2c<T><<<(unsigned)((npairs + kLines - 1) / kLines), kThreads, sm, s>>>(
        in, (C2<T> *)out, npairs, K, tw, rd);
    strided_passes<T>(f, (C2<T> *)out, B, (T)-1, tw, rd, s, true);
    count_launches(3);
    return check_launch("FFT forward");
}

template <typename T>
bd_status fft3_c2r(const FftPlan &f, void *in, T *out, int B, cudaStream_t s)
{
    Radices rd;
    rd.n = f.nrad;
    for (int i = 0; i < f.nrad; i++) rd.r[i] = f.rad[i];
    const int K = f.K;
    const C2<T> *tw = (const C2<T> *)(sizeof(T) == 8 ? f.d_tw64 : f.d_tw32);
    constexpr int kLines = lines_per_cta<T>();
    const long npairs = (long)B * K * K / 2;
    const size_t sm = smem_bytes<T>(K);
    strided_passes<T>(f, (C2<T> *)in, B, (T)1, tw, rd, s, false);
    k_fft_z_c2r<T><<<(unsigned)((npairs + kLines - 1) / kLines), kThreads, sm, s>>>(
        (const C2<T> *)in, out, npairs, K, tw, rd);
    count_launches(3);
    return check_launch("FFT inverse");
}

template bd_status fft3_r2c<double>(const FftPlan &, const double *, void *, int, cudaStream_t);
template bd_status fft3_r2c<float>(const FftPlan &, const float *, void *, int, cudaStream_t);
template bd_status fft3_c2r<double>(const FftPlan &, void *, double *, int, cudaStream_t);
template bd_status fft3_c2r<float>(const FftPlan &, void *, float *, int, cudaStream_t);

}  // namespace bd
