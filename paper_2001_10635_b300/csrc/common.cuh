// common.cuh -- shared internals of libreach.so (device parameter blocks,
// status plumbing, launch bookkeeping).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "reach.h"

namespace reach {

enum Method : int { MM = 0, CGB = 1 };

// Per-kind parameters as the kernels see them: derived constants are
// computed on the host once per call, never per element.
struct TrafficK {
    double cap, v, w, xbar;
    double wxbar;        // w * xbar
    int v_pow2;          // v is 2^e exactly (e = v_exp), so v * x is an exponent shift
    int v_exp;
    long long v_add;     // e << 52, the shift as an addend to the bit pattern
    double d_lo, d_hi;   // MM inputs (p, ph)
    double d_c, d_r;     // CGB input center and half-width
    int local;           // CGB with the box-evaluated contraction matrix
    int sound;           // outward rounding
    double c6l, c6u;     // h / 6 rounded down and up (outward rounding)
    double one = 1.0;    // read at run time (fadd; the directed sums of the outward-rounded kernel)
    double pzero = 0.0, nzero = -0.0;   // read at run time (the outward-rounded kernel's directed products)
    // CGB radius in nested form (stencil.cu, traffic_radius_step): per stage
    // s the coefficient c_s in (h/4, h/3, h/2, h) and c_s v, c_s w
    double rc[4], rv[4], rw[4];
};

struct KsK {
    double a0, a1, a2;   // 5-point stencil of -g_2 u_xx - g_4 u_xxxx
    double k;            // g_nl / (2 dx)
    double one = 1.0, nzero = -0.0;   // read at run time (fadd / fmul)
};

struct OscK {
    double ka, kb, kc;
};

struct HeatK {
    double kh;           // alpha / dx^2 = alpha l^2
    int64_t l;
    int open;            // the face z = 0 sees an environment at zero
};

// v * y as an exponent shift when v = 2^e: exact whenever y and the result are
// normal numbers (then the product is a power-of-two scaling); scale_ok says
// whether that holds for y
__device__ __forceinline__ bool scale_ok(double y, int e) {
    const int ef = (int)((__double_as_longlong(y) >> 52) & 0x7ff);
    return ef != 0 && ef != 0x7ff && ef + e >= 1 && ef + e <= 0x7fe;
}
__device__ __forceinline__ double scale_pow2(double y, long long add) {
    return __longlong_as_double(__double_as_longlong(y) + add);
}

// Binary64 sum and product issued as fused multiply-adds: fma(a, 1, b) and
// fma(a, b, -0) are rounded once from the same exact value as a + b and a * b
// (signed zeros included), so the results are the same bit for bit, and the
// FP64 pipe of this GPU retires DFMA about 19% faster than DADD or DMUL
// (independent chains: 5.6e11 against 4.75e11 per second).  `one` and `nzero`
// must be run-time values (a kernel parameter), or the compiler turns the
// fused form back into the plain one.
__device__ __forceinline__ double fadd(double a, double b, double one) { return __fma_rn(a, one, b); }
__device__ __forceinline__ double fmul(double a, double b, double nzero) { return __fma_rn(a, b, nzero); }

// bit flags written by kernels into a per-call status word
enum : int {
    ST_NONFINITE = 1,   // a result became NaN / Inf
    ST_BADINPUT = 2,    // lo > hi or a non-finite input seen on the device
    ST_NEGRADIUS = 4,   // CGB radius went negative (cannot happen for valid C)
    ST_TIMEOUT = 8,     // a bounded wait ran out
};

// process-wide launch counter (bench bookkeeping); host side only
void count_launch(int64_t k = 1);

// map a cudaError_t into a status code
int cuda_fail(cudaError_t e, const char *where);

#define REACH_CUDA(call)                                               \
    do {                                                               \
        cudaError_t e__ = (call);                                      \
        if (e__ != cudaSuccess) return ::reach::cuda_fail(e__, #call); \
    } while (0)

#define REACH_LAUNCHED(where)                                          \
    do {                                                               \
        ::reach::count_launch();                                       \
        cudaError_t e__ = cudaPeekAtLastError();                       \
        if (e__ != cudaSuccess) return ::reach::cuda_fail(e__, where); \
    } while (0)

// Order-preserving integer key of a double: for non-NaN a, b,
// a < b  <=>  key(a) < key(b) as signed 64-bit integers.  Minimum, maximum and
// comparisons of doubles through these keys run on the integer pipe; the
// FP64 pipe of this GPU retires two operations per SM per clock and is kept
// for arithmetic.
__device__ __forceinline__ long long dkey(double x) {
    long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double kmin(double a, double b) { return dkey(b) < dkey(a) ? b : a; }
__device__ __forceinline__ double kmax(double a, double b) { return dkey(b) > dkey(a) ? b : a; }
__device__ __forceinline__ bool kle(double a, double b) { return dkey(a) <= dkey(b); }
__device__ __forceinline__ double kabs(double x) {
    return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool kfinite(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// periodic index of g on a grid of n points without integer division (which
// this GPU emulates partly on the FP64 pipe): one conditional wrap covers the
// rows a tile can reach when n is at least the tile, a bounded loop the rest
__device__ __forceinline__ int64_t wrap_index(int64_t g, int64_t n) {
    g = g < 0 ? g + n : g;
    g = g >= n ? g - n : g;
    if (g < 0 || g >= n) {
        while (g < 0) g += n;
        while (g >= n) g -= n;
    }
    return g;
}

// global nanosecond clock of the GPU
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the paper's
// definition: 10 rounds of (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)) with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t a = c[0], b = c[2];
        uint32_t hi_a = __umulhi(0xD2511F53u, a), lo_a = 0xD2511F53u * a;
        uint32_t hi_b = __umulhi(0xCD9E8D57u, b), lo_b = 0xCD9E8D57u * b;
        c[0] = hi_b ^ c[1] ^ k0;
        c[1] = lo_b;
        c[2] = hi_a ^ c[3] ^ k1;
        c[3] = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// uniform double in [0,1) for (sample j, component i, tag) under `seed`:
// counter (i, j, tag, 0), key (seed lo, seed hi), top 53 bits of w0:w1
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint32_t j, uint32_t i, uint32_t tag) {
    uint32_t c[4] = {i, j, tag, 0u};
    philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    uint64_t bits = ((uint64_t)c[0] << 32) | c[1];
    return (double)(bits >> 11) * 0x1.0p-53;
}

// sample lo + (hi - lo) U without contraction, exactly as the definition reads
__device__ __forceinline__ double box_sample(double lo, double hi, double u) {
    return __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), u));
}

}  // namespace reach
