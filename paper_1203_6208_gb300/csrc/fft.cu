// fft.cu -- the 3-D mesh transforms of the spectral product (Sec. VIII
// outlook: the Fourier part of the Ewald sum by FFT): a batch of real K^3
// meshes to their half spectra K x K x (K/2 + 1) and back, unnormalised
// (forward e^{-2 pi i jk/K}, inverse e^{+2 pi i jk/K}), K an even
// 2^a 3^b 5^c <= 512.
//
// Each 1-D transform runs in shared memory as a Stockham (self-sorting)
// sequence of radix passes: pass q with radix R and Ns = the product of the
// earlier radices reads R values K/R apart, turns them by the twiddles
// w^{r (j mod Ns) K/(Ns R)}, takes the R-point DFT and writes them Ns apart
// at (j div Ns) Ns R + (j mod Ns); the output is in natural order.  The
// radices are 16 (FP32 only), 8, 4, 2, 9, 3 and 5, largest first; 8, 9 and
// 16 are one Cooley-Tukey split done in registers, so fewer passes go
// through shared memory (K = 144 = 16 9: two).
//   z (contiguous) : two real lines a, b form c = a + i b; after the complex
//                    transform A_k = (C_k + conj C_{-k})/2 and
//                    B_k = (C_k - conj C_{-k})/(2i), k = 0 .. K/2 (the inverse
//                    rebuilds C = A + i B from the Hermitian halves).
//   y, x (strided) : complex lines; a CTA takes 8 (FP64) or 16 (FP32) lines
//                    with consecutive k_z, so each mesh row it reads is one
//                    128-byte run.
// Every tile comes into shared memory by asynchronous copies issued all at
// once (cp.async), so a CTA has its whole tile in flight.
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

// resident CTAs a SM: five in FP32 (register cap 48, the 16-point butterfly
// still without spills), four in FP64
template <typename T> __host__ __device__ constexpr int kMinBlocks() { return sizeof(T) == 4 ? 5 : 4; }

// shared memory by 32-bit byte address: every index in the transforms is
// 32-bit arithmetic on these addresses
template <typename T> __device__ __forceinline__ C2<T> ld_s(uint32_t a);
template <> __device__ __forceinline__ C2<float> ld_s<float>(uint32_t a)
{
    C2<float> v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
template <> __device__ __forceinline__ C2<double> ld_s<double>(uint32_t a)
{
    C2<double> v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_s(uint32_t a, C2<float> v)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_s(uint32_t a, C2<double> v)
{
    asm volatile("st.shared.v2.f64 [%0], {%1, %2};\n" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// asynchronous global -> shared copies of B = 4, 8 or 16 bytes (both
// addresses B-aligned): a thread issues all of its copies of a tile before
// it waits, so every load of the tile is in flight at once
template <int B>
__device__ __forceinline__ void cp_async(uint32_t sdst, const void *gsrc)
{
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sdst), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }
// multiply by SG i (the direction SG = -1 forward, +1 inverse, fixed at compile time)
template <int SG, typename T> __device__ __forceinline__ C2<T> cmuli(C2<T> a)
{
    return SG > 0 ? C2<T>{-a.y, a.x} : C2<T>{a.y, -a.x};
}

// a (c + SG i s)
template <int SG, typename T>
__device__ __forceinline__ C2<T> rot(C2<T> a, T c, T s)
{
    return SG > 0 ? C2<T>{a.x * c - a.y * s, a.y * c + a.x * s} : C2<T>{a.x * c + a.y * s, a.y * c - a.x * s};
}

// R-point DFTs, y_k = sum_t a_t e^{SG 2 pi i t k / R}: radices 2, 3, 4 and 5
// directly, 8 = 2 x 4, 9 = 3 x 3 and 16 = 4 x 4 in registers by one
// Cooley-Tukey split R = R1 R2: with t = t1 + R1 t2 and k = R2 k1 + k2,
// y_{R2 k1 + k2} = sum_{t1} W_{R1}^{t1 k1} W_R^{t1 k2} b_{t1}[k2], b_{t1} the
// R2-point DFT of a_{t1}, a_{t1 + R1}, ...  (W_n = e^{SG 2 pi i/n})
template <typename T, int R, int SG>
__device__ __forceinline__ void dft(C2<T> *a)
{
    if (R == 8) {                                              // R1 = 2, R2 = 4
        const T h = (T)0.707106781186547524401;                // cos(pi/4)
        C2<T> e[4] = {a[0], a[2], a[4], a[6]}, o[4] = {a[1], a[3], a[5], a[7]};
        dft<T, 4, SG>(e);
        dft<T, 4, SG>(o);
        o[1] = rot<SG>(o[1], h, h);                            // W_8
        o[2] = cmuli<SG>(o[2]);                                // W_8^2
        o[3] = rot<SG>(o[3], -h, h);                           // W_8^3
#pragma unroll
        for (int k = 0; k < 4; k++) {
            a[k] = cadd(e[k], o[k]);
            a[k + 4] = csub(e[k], o[k]);
        }
    } else if (R == 9) {                                       // R1 = R2 = 3
        const T c1 = (T)0.766044443118978035202, s1 = (T)0.642787609686539326323;    // W_9
        const T c2 = (T)0.173648177666930348852, s2 = (T)0.984807753012208059367;    // W_9^2
        const T c4 = (T)-0.939692620785908384054, s4 = (T)0.342020143325668733044;   // W_9^4
        C2<T> b[3][3];
#pragma unroll
        for (int t1 = 0; t1 < 3; t1++) {
#pragma unroll
            for (int t2 = 0; t2 < 3; t2++) b[t1][t2] = a[t1 + 3 * t2];
            dft<T, 3, SG>(b[t1]);
        }
        b[1][1] = rot<SG>(b[1][1], c1, s1);
        b[1][2] = rot<SG>(b[1][2], c2, s2);
        b[2][1] = rot<SG>(b[2][1], c2, s2);
        b[2][2] = rot<SG>(b[2][2], c4, s4);
#pragma unroll
        for (int k2 = 0; k2 < 3; k2++) {
            C2<T> c[3] = {b[0][k2], b[1][k2], b[2][k2]};
            dft<T, 3, SG>(c);
#pragma unroll
            for (int k1 = 0; k1 < 3; k1++) a[3 * k1 + k2] = c[k1];
        }
    } else if (R == 16) {                                      // R1 = R2 = 4
        const T c = (T)0.923879532511286756128, s = (T)0.382683432365089771728;      // W_16
        const T h = (T)0.707106781186547524401;
        C2<T> b[4][4];
#pragma unroll
        for (int t1 = 0; t1 < 4; t1++) {
#pragma unroll
            for (int t2 = 0; t2 < 4; t2++) b[t1][t2] = a[t1 + 4 * t2];
            dft<T, 4, SG>(b[t1]);
        }
        b[1][1] = rot<SG>(b[1][1], c, s);                      // W_16
        b[1][2] = rot<SG>(b[1][2], h, h);                      // W_16^2
        b[1][3] = rot<SG>(b[1][3], s, c);                      // W_16^3
        b[2][1] = rot<SG>(b[2][1], h, h);                      // W_16^2
        b[2][2] = cmuli<SG>(b[2][2]);                          // W_16^4
        b[2][3] = rot<SG>(b[2][3], -h, h);                     // W_16^6
        b[3][1] = rot<SG>(b[3][1], s, c);                      // W_16^3
        b[3][2] = rot<SG>(b[3][2], -h, h);                     // W_16^6
        b[3][3] = rot<SG>(b[3][3], -c, -s);                    // W_16^9
#pragma unroll
        for (int k2 = 0; k2 < 4; k2++) {
            C2<T> e[4] = {b[0][k2], b[1][k2], b[2][k2], b[3][k2]};
            dft<T, 4, SG>(e);
#pragma unroll
            for (int k1 = 0; k1 < 4; k1++) a[4 * k1 + k2] = e[k1];
        }
    } else if (R == 2) {
        const C2<T> t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    } else if (R == 4) {
        const C2<T> t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]), t2 = cadd(a[1], a[3]);
        const C2<T> t3 = cmuli<SG>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    } else if (R == 3) {
        const T h3 = (T)0.86602540378443864676;             // sqrt(3)/2
        const C2<T> s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        const C2<T> h = {a[0].x - (T)0.5 * s.x, a[0].y - (T)0.5 * s.y};
        const C2<T> t = cmuli<SG>(C2<T>{h3 * d.x, h3 * d.y});
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
        const C2<T> i1 = cmuli<SG>(C2<T>{s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y});
        const C2<T> i2 = cmuli<SG>(C2<T>{s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y});
        a[0] = cadd(a[0], cadd(b1, b2));
        a[1] = cadd(r1, i1);
        a[4] = csub(r1, i1);
        a[2] = cadd(r2, i2);
        a[3] = csub(r2, i2);
    }
}

// the radix sequence, 5 bits a pass from the low end (at most 6 passes)
struct Radices {
    unsigned code;
};

// n div d for 0 <= n < 4096 and 1 <= d <= 1024 from the approximate
// reciprocal: (n + 1/2)/d lies at least 1/(2d) from an integer, and the
// product's error (a few ulp of n/d) stays far below that
__device__ __forceinline__ int small_div(int n, int d)
{
    return (int)(((float)n + 0.5f) * __fdividef(1.0f, (float)d));
}

// (e div d, e mod d) for e = e0, e0 + kThreads, ...: one division, then a
// step of (kThreads div d, kThreads mod d) with one carry
struct DivWalk {
    int q, r, dq, dr, d;
    __device__ DivWalk(int e0, int d_) : q(small_div(e0, d_)), r(e0 - q * d_), dq(small_div(kThreads, d_)),
                                          dr(kThreads - dq * d_), d(d_) {}
    __device__ __forceinline__ void next()
    {
        q += dq;
        r += dr;
        if (r >= d) {
            r -= d;
            q++;
        }
    }
};

// one Stockham pass of radix R over NL lines of length K (line stride K + 1
// in shared memory), src -> dst (byte addresses of line 0); consecutive
// threads take the same butterfly of consecutive lines (each thread keeps its
// line), so the padded stride spreads them over the banks.  Lines past nl
// compute on padding and are never written back.
template <typename T, int R, int NL, int SG>
__device__ __forceinline__ void fft_pass(uint32_t src, uint32_t dst, uint32_t tw, int K, int Ns)
{
    constexpr uint32_t E = sizeof(C2<T>);
    constexpr int step = kThreads / NL;
    const int nb = K / R;
    const uint32_t row = (uint32_t)(threadIdx.x % NL) * (uint32_t)(K + 1) * E;
    const uint32_t s0 = src + row, d0 = dst + row;
    const uint32_t nbE = (uint32_t)nb * E, NsE = (uint32_t)Ns * E;
    const uint32_t twE = (uint32_t)(K / (Ns * R)) * E;   // twiddle table step per unit of j mod Ns
    // jm = j mod Ns walked incrementally: no division per butterfly
    int j = threadIdx.x / NL;
    int jm = j - small_div(j, Ns) * Ns;
    const int sm = step - small_div(step, Ns) * Ns;
    for (; j < nb; j += step) {
        C2<T> a[R];
        const uint32_t pj = s0 + (uint32_t)j * E;
#pragma unroll
        for (int r = 0; r < R; r++) a[r] = ld_s<T>(pj + r * nbE);
        if (Ns > 1) {                     // the first pass has no twiddles
            const uint32_t q = (uint32_t)jm * twE;
#pragma unroll
            for (int r = 1; r < R; r++) {
                C2<T> w = ld_s<T>(tw + r * q);
                if (SG > 0) w.y = -w.y;   // the table holds e^{-2 pi i t/K}; the inverse conjugates
                a[r] = cmul(a[r], w);
            }
        }
        dft<T, R, SG>(a);
        const uint32_t o = d0 + (uint32_t)((j - jm) * R + jm) * E;
#pragma unroll
        for (int r = 0; r < R; r++) st_s(o + r * NsE, a[r]);
        jm += sm;
        if (jm >= Ns) jm -= Ns;
    }
}

// the transforms of the CTA's lines of length K held at buf0 ([line][K + 1]);
// returns the address of the buffer that holds the result.  All threads of
// the CTA take part.
template <typename T, int SG>
__device__ uint32_t fft_lines(uint32_t buf0, uint32_t buf1, uint32_t tw, int K, Radices rd)
{
    constexpr int NL = lines_per_cta<T>();
    uint32_t src = buf0, dst = buf1;
    int Ns = 1;
    for (unsigned code = rd.code; code; code >>= 5) {
        const int R = (int)(code & 31u);
        switch (R) {
        case 2: fft_pass<T, 2, NL, SG>(src, dst, tw, K, Ns); break;
        case 3: fft_pass<T, 3, NL, SG>(src, dst, tw, K, Ns); break;
        case 4: fft_pass<T, 4, NL, SG>(src, dst, tw, K, Ns); break;
        case 5: fft_pass<T, 5, NL, SG>(src, dst, tw, K, Ns); break;
        case 8: fft_pass<T, 8, NL, SG>(src, dst, tw, K, Ns); break;
        case 9: fft_pass<T, 9, NL, SG>(src, dst, tw, K, Ns); break;
        default:
            if constexpr (sizeof(T) == 4) fft_pass<T, 16, NL, SG>(src, dst, tw, K, Ns);
            break;
        }
        __syncthreads();
        const uint32_t t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// shared memory of a CTA: the twiddle table, then two line buffers
// ([kLines][K + 1] and, behind it, room for the inverse z kernel's staged
// half spectra)
template <typename T>
struct Smem {
    uint32_t tw, b0, b1;
    __device__ Smem(unsigned char *base, int K)
    {
        constexpr uint32_t E = sizeof(C2<T>);
        tw = smem_addr(base);
        b0 = tw + (uint32_t)K * E;
        b1 = b0 + (uint32_t)(lines_per_cta<T>() * (K + 1)) * E;
    }
};

template <typename T>
__device__ __forceinline__ void load_twiddles(uint32_t tw, const C2<T> *twg, int K)
{
    for (int t = threadIdx.x; t < K; t += kThreads) cp_async<sizeof(C2<T>)>(tw + t * (uint32_t)sizeof(C2<T>), &twg[t]);
}

// forward z: pairs of real lines (2p, 2p + 1) -> their half spectra
template <typename T>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T>())
k_fft_z_r2c(const T *__restrict__ in, C2<T> *__restrict__ out, long npairs, int K,
            const C2<T> *__restrict__ twg, Radices rd)
{
    constexpr int kLines = lines_per_cta<T>();
    constexpr uint32_t E = sizeof(C2<T>);
    extern __shared__ __align__(16) unsigned char smem[];
    const Smem<T> sh(smem, K);
    const long p0 = (long)blockIdx.x * kLines;
    const int nl = (int)min((long)kLines, npairs - p0);
    const int H = K / 2 + 1;
    load_twiddles<T>(sh.tw, twg, K);
    // lines 2 p0 .. 2 (p0 + nl) - 1 are one contiguous run of reals; element
    // (p, k) of the CTA takes line 2p to the real part of line p in shared
    // memory, line 2p + 1 to the imaginary part
    const T *src = in + (size_t)2 * p0 * K;
    DivWalk w(threadIdx.x, K);
    for (int e = threadIdx.x; e < nl * K; e += kThreads, w.next()) {
        const uint32_t a = sh.b0 + (uint32_t)(w.q * (K + 1) + w.r) * E;
        const T *g = src + 2 * w.q * K + w.r;
        cp_async<sizeof(T)>(a, g);
        cp_async<sizeof(T)>(a + (uint32_t)sizeof(T), g + K);
    }
    cp_async_wait_all();
    __syncthreads();
    const uint32_t res = fft_lines<T, -1>(sh.b0, sh.b1, sh.tw, K, rd);
    // element (p, k), k < H: A_k to half spectrum 2p, B_k to 2p + 1
    C2<T> *dst = out + (size_t)2 * p0 * H;
    DivWalk v(threadIdx.x, H);
    for (int e = threadIdx.x; e < nl * H; e += kThreads, v.next()) {
        const int k = v.r;
        const uint32_t c = res + (uint32_t)(v.q * (K + 1)) * E;
        const C2<T> ck = ld_s<T>(c + (uint32_t)k * E), cm = ld_s<T>(c + (uint32_t)(k ? K - k : 0) * E);   // C_k, C_{-k}
        C2<T> *d = dst + 2 * v.q * H + k;
        d[0] = {(T)0.5 * (ck.x + cm.x), (T)0.5 * (ck.y - cm.y)};              // (C_k + conj C_-k)/2
        d[H] = {(T)0.5 * (ck.y + cm.y), (T)-0.5 * (ck.x - cm.x)};             // (C_k - conj C_-k)/(2i)
    }
}

// inverse z: pairs of half spectra -> their real lines (unnormalised)
template <typename T>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T>())
k_fft_z_c2r(const C2<T> *__restrict__ in, T *__restrict__ out, long npairs, int K,
            const C2<T> *__restrict__ twg, Radices rd)
{
    constexpr int kLines = lines_per_cta<T>();
    constexpr uint32_t E = sizeof(C2<T>);
    extern __shared__ __align__(16) unsigned char smem[];
    const Smem<T> sh(smem, K);
    const long p0 = (long)blockIdx.x * kLines;
    const int nl = (int)min((long)kLines, npairs - p0);
    const int H = K / 2 + 1;
    load_twiddles<T>(sh.tw, twg, K);
    // the CTA's 2 nl half spectra are one contiguous run of 2 nl H E bytes
    // (a multiple of 16; start 16-byte aligned), staged at b1 in 16-byte
    // copies (2 H <= K + 2 values a line pair, kLines extra values allotted)
    const unsigned char *gsrc = (const unsigned char *)(in + (size_t)2 * p0 * H);
    for (int e = threadIdx.x; e < (int)(2 * nl * H * E / 16); e += kThreads)
        cp_async<16>(sh.b1 + (uint32_t)e * 16u, gsrc + (size_t)e * 16);
    cp_async_wait_all();
    __syncthreads();
    // C_k = A_k + i B_k over the whole line, the upper half from conjugates
    DivWalk w(threadIdx.x, K);
    for (int e = threadIdx.x; e < nl * K; e += kThreads, w.next()) {
        const int pr = w.q, k = w.r;
        const bool lo = k < H;
        const uint32_t kk = (uint32_t)(lo ? k : K - k);
        C2<T> a = ld_s<T>(sh.b1 + ((uint32_t)(2 * pr * H) + kk) * E);
        C2<T> b = ld_s<T>(sh.b1 + ((uint32_t)((2 * pr + 1) * H) + kk) * E);
        if (!lo) {
            a.y = -a.y;
            b.y = -b.y;
        }
        st_s(sh.b0 + (uint32_t)(pr * (K + 1) + k) * E, C2<T>{a.x - b.y, a.y + b.x});
    }
    __syncthreads();
    const uint32_t res = fft_lines<T, 1>(sh.b0, sh.b1, sh.tw, K, rd);
    // element (p, k): the real part to line 2p, the imaginary to 2p + 1
    T *dst = out + (size_t)2 * p0 * K;
    DivWalk v(threadIdx.x, K);
    for (int e = threadIdx.x; e < nl * K; e += kThreads, v.next()) {
        const C2<T> c = ld_s<T>(res + (uint32_t)(v.q * (K + 1) + v.r) * E);
        T *d = dst + 2 * v.q * K + v.r;
        d[0] = c.x;
        d[K] = c.y;
    }
}

// complex transforms along a strided axis, in place.  Line (b, i, z): element
// t at b A + i I + z + t S, z < H; CTA (z tile, i, b) takes kLines
// consecutive z.  Each thread keeps one z (its lane mod kLines) and walks t.
template <typename T, int SG>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T>())
k_fft_strided(C2<T> *__restrict__ data, int K, int H, long A, long I, long S,
              const C2<T> *__restrict__ twg, Radices rd)
{
    constexpr int kLines = lines_per_cta<T>();
    constexpr int tstep = kThreads / kLines;
    constexpr uint32_t E = sizeof(C2<T>);
    extern __shared__ __align__(16) unsigned char smem[];
    const Smem<T> sh(smem, K);
    const int z0 = (int)blockIdx.x * kLines;
    const int nl = min(kLines, H - z0);
    const int l = threadIdx.x % kLines, t0 = threadIdx.x / kLines;
    C2<T> *base = data + (long)blockIdx.z * A + (long)blockIdx.y * I + z0 + l;
    const long gs = (long)tstep * S;
    const uint32_t off = (uint32_t)(l * (K + 1) + t0) * E;
    load_twiddles<T>(sh.tw, twg, K);
    if (l < nl) {
        const C2<T> *g = base + (long)t0 * S;
        uint32_t a = sh.b0 + off;
        for (int t = t0; t < K; t += tstep, g += gs, a += tstep * E) cp_async<sizeof(C2<T>)>(a, g);
    }
    cp_async_wait_all();
    __syncthreads();
    const uint32_t res = fft_lines<T, SG>(sh.b0, sh.b1, sh.tw, K, rd);
    if (l < nl) {
        C2<T> *g = base + (long)t0 * S;
        uint32_t a = res + off;
        for (int t = t0; t < K; t += tstep, g += gs, a += tstep * E) *g = ld_s<T>(a);
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
static size_t smem_bytes(int K) { return (size_t)(K + 2 * lines_per_cta<T>() * (K + 2)) * sizeof(C2<T>); }

}  // namespace ff

using namespace ff;

// K's radix passes, largest radices first (the first pass has no twiddles):
// powers of two in 16s (FP32; 8s in FP64, whose 16-point butterfly would
// not fit the registers), 8, 4, 2, then 9, 3 and 5; false if K has another
// prime factor or takes more than 6 passes
static bool radix_code(int K, bool f64, unsigned &code)
{
    const int f32_list[7] = {16, 8, 4, 2, 9, 3, 5}, f64_list[6] = {8, 4, 2, 9, 3, 5};
    const int *list = f64 ? f64_list : f32_list, nl = f64 ? 6 : 7;
    int r = K, n = 0;
    code = 0;
    for (int i = 0; i < nl; i++)
        while (r % list[i] == 0 && n < 6) {
            code |= (unsigned)list[i] << (5 * n++);
            r /= list[i];
        }
    return r == 1;
}

bd_status fft_plan_init(FftPlan &f, int K)
{
    f.K = K;
    if (K < 2 || K % 2 || K > kFftMaxK || !radix_code(K, false, f.code32) || !radix_code(K, true, f.code64))
        return set_error(BD_ERR_UNSUPPORTED, "mesh size %d is not an even 2^a 3^b 5^c <= %d", K, kFftMaxK);
    cudaError_t e = cudaMalloc(&f.d_tw64, sizeof(C2<double>) * K);
    if (e == cudaSuccess) e = cudaMalloc(&f.d_tw32, sizeof(C2<float>) * K);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BD_ERR_OOM, "FFT twiddles: %s", cudaGetErrorString(e));
    }
    k_twiddles<<<(K + 127) / 128, 128>>>(K, (C2<double> *)f.d_tw64, (C2<float> *)f.d_tw32);
    count_launches(1);
    const int s64 = (int)smem_bytes<double>(K), s32 = (int)smem_bytes<float>(K);
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t a[8] = {
        cudaFuncSetAttribute(k_fft_z_r2c<double>, at, s64), cudaFuncSetAttribute(k_fft_z_c2r<double>, at, s64),
        cudaFuncSetAttribute(k_fft_strided<double, -1>, at, s64), cudaFuncSetAttribute(k_fft_strided<double, 1>, at, s64),
        cudaFuncSetAttribute(k_fft_z_r2c<float>, at, s32), cudaFuncSetAttribute(k_fft_z_c2r<float>, at, s32),
        cudaFuncSetAttribute(k_fft_strided<float, -1>, at, s32), cudaFuncSetAttribute(k_fft_strided<float, 1>, at, s32)};
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
static Radices radices(const FftPlan &f) { return Radices{sizeof(T) == 8 ? f.code64 : f.code32}; }

template <typename T, int SG>
static void strided_passes(const FftPlan &f, C2<T> *q, int B, const C2<T> *tw, const Radices &rd,
                           cudaStream_t s, bool y_first)
{
    constexpr int kLines = lines_per_cta<T>();
    const int K = f.K, H = K / 2 + 1;
    const dim3 grid((unsigned)((H + kLines - 1) / kLines), (unsigned)K, (unsigned)B);
    const size_t sm = smem_bytes<T>(K);
    const long KH = (long)K * H;
    for (int pass = 0; pass < 2; pass++) {
        if ((pass == 0) == y_first)   // lines (b, i0, z) along i1: stride H
            k_fft_strided<T, SG><<<grid, kThreads, sm, s>>>(q, K, H, K * KH, KH, H, tw, rd);
        else                          // lines (b, i1, z) along i0: stride K H
            k_fft_strided<T, SG><<<grid, kThreads, sm, s>>>(q, K, H, K * KH, H, KH, tw, rd);
    }
}

template <typename T>
bd_status fft3_r2c(const FftPlan &f, const T *in, void *out, int B, cudaStream_t s)
{
    const Radices rd = radices<T>(f);
    const int K = f.K;
    const C2<T> *tw = (const C2<T> *)(sizeof(T) == 8 ? f.d_tw64 : f.d_tw32);
    constexpr int kLines = lines_per_cta<T>();
    const long npairs = (long)B * K * K / 2;
    const size_t sm = smem_bytes<T>(K);
    k_fft_z_r2c<T><<<(unsigned)((npairs + kLines - 1) / kLines), kThreads, sm, s>>>(
        in, (C2<T> *)out, npairs, K, tw, rd);
    strided_passes<T, -1>(f, (C2<T> *)out, B, tw, rd, s, true);
    count_launches(3);
    return check_launch("FFT forward");
}

template <typename T>
bd_status fft3_c2r(const FftPlan &f, void *in, T *out, int B, cudaStream_t s)
{
    const Radices rd = radices<T>(f);
    const int K = f.K;
    const C2<T> *tw = (const C2<T> *)(sizeof(T) == 8 ? f.d_tw64 : f.d_tw32);
    constexpr int kLines = lines_per_cta<T>();
    const long npairs = (long)B * K * K / 2;
    const size_t sm = smem_bytes<T>(K);
    strided_passes<T, 1>(f, (C2<T> *)in, B, tw, rd, s, false);
    k_fft_z_c2r<T><<<(unsigned)((npairs + kLines - 1) / kLines), kThreads, sm, s>>>(
        (const C2<T> *)in, out, npairs, K, tw, rd);
    count_launches(3);
    return check_launch("FFT inverse");
}

extern "C" bd_status bd_mesh_fft(int32_t K, int32_t B, int32_t precision, int32_t inverse,
                                 void *in, void *out, bd_stream stream)
{
    if (!in || !out) return set_error(BD_ERR_INVALID, "NULL argument");
    if (B < 1) return set_error(BD_ERR_INVALID, "B=%d < 1", B);
    if (B > 65535) return set_error(BD_ERR_UNSUPPORTED, "B=%d > 65535 meshes in one call", B);
    if (precision != BD_FP64 && precision != BD_MIXED_F16 && precision != BD_MIXED_BF16)
        return set_error(BD_ERR_INVALID, "unknown precision %d", precision);
    if (K < 2 || K % 2) return set_error(BD_ERR_UNSUPPORTED, "mesh size %d is not even", K);
    const size_t w = precision == BD_FP64 ? sizeof(double) : sizeof(float);
    const size_t real_b = (size_t)B * K * K * K * w, half_b = (size_t)B * K * K * (K / 2 + 1) * 2 * w;
    const char *ib = (const char *)in, *ob = (const char *)out;
    const size_t ilen = inverse ? half_b : real_b, olen = inverse ? real_b : half_b;
    if (ib < ob + olen && ob < ib + ilen) return set_error(BD_ERR_INVALID, "in and out overlap");
    FftPlan f{};
    bd_status st = fft_plan_init(f, K);
    if (st == BD_OK && cudaDeviceSynchronize() != cudaSuccess) st = set_error(BD_ERR_CUDA, "FFT twiddles");
    if (st == BD_OK) {
        const cudaStream_t s = (cudaStream_t)stream;
        if (precision == BD_FP64)
            st = inverse ? fft3_c2r<double>(f, in, (double *)out, B, s) : fft3_r2c<double>(f, (const double *)in, out, B, s);
        else
            st = inverse ? fft3_c2r<float>(f, in, (float *)out, B, s) : fft3_r2c<float>(f, (const float *)in, out, B, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        if (st == BD_OK && e != cudaSuccess) st = set_error(BD_ERR_CUDA, "FFT: %s", cudaGetErrorString(e));
    }
    fft_free(f);
    return st;
}

template bd_status fft3_r2c<double>(const FftPlan &, const double *, void *, int, cudaStream_t);
template bd_status fft3_r2c<float>(const FftPlan &, const float *, void *, int, cudaStream_t);
template bd_status fft3_c2r<double>(const FftPlan &, void *, double *, int, cudaStream_t);
template bd_status fft3_c2r<float>(const FftPlan &, void *, float *, int, cudaStream_t);

}  // namespace bd
