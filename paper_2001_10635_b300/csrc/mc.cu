// mc.cu -- Monte Carlo reachability (Sec. 2.1, Algorithm 4).
//
// Samples are drawn on the device with Philox4x32-10 (common.cuh) and
// integrated with RK4 in binary64 or binary32.
//   mc_onchip : small n, one block = SB samples x the whole state, all N steps
//               in shared memory (SB = 32, or 8 or 2 when there are too few
//               samples for blocks of 32 to reach every SM); lane = sample,
//               minima / maxima over samples by warp shuffles.
//   mc_rows / mc_rows64 (the streaming defaults): large stencil systems, state
//               in HBM with each sample (binary64) or pair of samples (binary32)
//               a contiguous run of rows; a lane holds consecutive rows, so the
//               stencil crosses lanes by shuffles and no warp waits for
//               another; S RK4 steps per launch with a 4RS-row halo; sampling
//               fused into the first launch, minima / maxima over samples in a
//               final pass over the state.
//   mc_stream / mc_stream2 / mc_stream2p: the same systems in the
//               sample-fastest layout x[i * M + j] (lane = sample; blocks of
//               sample rows exchanging edge rows through shared memory), kept
//               as options.
//   mc_quad   : the quadrotor swarm, 32 samples of one agent per warp.
// Per-block partial minima / maxima are combined by mc_reduce (no atomics, so
// the result does not depend on scheduling).
#include <algorithm>
#include <cmath>

#include <atomic>
#include <type_traits>

#include <cuda.h>

#include "api_internal.cuh"
#include "quad.cuh"

namespace reach {

constexpr int MC_WARPS = 16;            // warps per block
constexpr int MC_THREADS = 32 * MC_WARPS;
constexpr int MC_Q = 8;                 // component rows per thread (on-chip)

// Precision-explicit helpers: a float trajectory must stay on the FP32 pipe
// (an overload that promotes to double would run the stage arithmetic and two
// conversions per operation on the FP64 pipe); minima of doubles use the
// integer pipe.
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return kmin(a, b); }
// minimum of three: one three-input instruction in binary32 (the traffic flux
// min(cap, v y, w (xbar - y')) is the kernels' only use of minima)
__device__ __forceinline__ float tmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ double tmin3(double a, double b, double c) { return kmin(a, kmin(b, c)); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }

// ------------------------------------------------------------------ plain f
// Y: rows of 32 samples (row c at Y + 32 c), P: input rows.  `g` is the
// global component of row c; rows c +- R exist in Y (halo or wrapped).
template <int SYS, class T>
struct Plain;

template <class T>
struct Plain<REACH_TRAFFIC, T> {
    static constexpr int R = 1;
    // flux out of global cell g given its row value y and right neighbour yr
    static __device__ __forceinline__ T flux(const T *q, T y, T yr, int64_t g, int64_t n, T d) {
        T cong = (g == n - 1) ? q[0] : tfma(-q[2], yr, q[3]);
        T f = tmin3(q[0], q[1] * y, cong);
        f = (g == -1) ? d : f;
        f = (g < -1 || g >= n) ? T(0) : f;
        return f;
    }
    template <class Row, class In>
    static __device__ __forceinline__ T rhs(const T *q, Row row, int c, int64_t g, int64_t n, In pin) {
        T d = pin(0);
        T fin = flux(q, row(c - 1), row(c), g - 1, n, d);
        T fout = flux(q, row(c), row(c + 1), g, n, d);
        return fin - fout;
    }
};

template <class T>
struct Plain<REACH_KS, T> {
    static constexpr int R = 2;
    template <class Row, class In>
    static __device__ __forceinline__ T rhs(const T *q, Row row, int c, int64_t, int64_t, In) {
        T um2 = row(c - 2), um1 = row(c - 1), u = row(c), up1 = row(c + 1), up2 = row(c + 2);
        // u (a0 - k (u_{i+1} - u_{i-1})) + a1 (u_{i-1} + u_{i+1}) + a2 (u_{i-2} + u_{i+2})
        return tfma(u, tfma(-q[3], up1 - um1, q[0]), tfma(q[1], um1 + up1, q[2] * (um2 + up2)));
    }
};

template <class T>
struct Plain<REACH_OSC, T> {
    static constexpr int R = 0;
    // whole state on chip: rows 0..m-1 positions, m..2m-1 velocities
    template <class Row, class In>
    static __device__ __forceinline__ T rhs(const T *q, Row row, int c, int64_t, int64_t n, In pin) {
        const int m = (int)(n >> 1);
        if (c < m) return row(m + c);
        const int j = c - m;
        T z = row(j);
        T xl = (j > 0) ? row(j - 1) : T(0), xr = (j < m - 1) ? row(j + 1) : T(0);
        // -(ka + 2kc + kb z^2) z + kc (xl + xr) + w
        T t = tfma(q[1], z * z, q[3]);
        T r = tfma(q[2], xl + xr, pin(j));
        return tfma(-t, z, r);
    }
};

template <class T>
struct Plain<REACH_HEAT3D, T> {
    static constexpr int R = 0;
    // whole grid on chip; q: kh, l, open face
    template <class Row, class In>
    static __device__ __forceinline__ T rhs(const T *q, Row row, int c, int64_t, int64_t, In) {
        const int l = (int)q[1], pl = l * l;
        const int x = c % l, y = (c / l) % l, z = c / pl;
        T s = (x > 0) ? row(c - 1) : T(0);
        s += (x + 1 < l) ? row(c + 1) : T(0);
        s += (y > 0) ? row(c - l) : T(0);
        s += (y + 1 < l) ? row(c + l) : T(0);
        s += (z > 0) ? row(c - pl) : T(0);
        s += (z + 1 < l) ? row(c + pl) : T(0);
        const int m = (x > 0) + (x + 1 < l) + (y > 0) + (y + 1 < l) + (z > 0 || q[2] != T(0)) + (z + 1 < l);
        return q[0] * tfma(-(T)m, row(c), s);
    }
};

template <class T>
struct Plain<REACH_LINEAR, T> {
    static constexpr int R = 0;
    template <class Row, class In>
    static __device__ __forceinline__ T rhs(const T *, Row row, int c, int64_t, int64_t n, In pin,
                                            const double *A) {
        T acc = T(0);
        const double *Ar = A + (int64_t)c * n;
#pragma unroll 1
        for (int j = 0; j < (int)n; ++j) acc = tfma((T)__ldg(Ar + j), row(j), acc);
        return acc + pin(c);
    }
};

template <int SYS, class T>
__device__ __forceinline__ void mc_consts(const double *prm, T (&q)[4]) {
    q[0] = q[1] = q[2] = q[3] = T(0);
    if (SYS == REACH_TRAFFIC) { q[0] = (T)prm[0]; q[1] = (T)prm[1]; q[2] = (T)prm[2]; q[3] = (T)(prm[2] * prm[3]); }
    if (SYS == REACH_KS) { q[0] = (T)prm[0]; q[1] = (T)prm[1]; q[2] = (T)prm[2]; q[3] = (T)prm[3]; }
    if (SYS == REACH_OSC || SYS == REACH_HEAT3D) { q[0] = (T)prm[0]; q[1] = (T)prm[1]; q[2] = (T)prm[2]; }
    if (SYS == REACH_OSC) q[3] = (T)(prm[0] + 2.0 * prm[2]);
}

// sample value rounded to the run precision (binary32 runs start from the
// binary64 sample rounded to nearest)
template <class T>
__device__ __forceinline__ T as_run(double v) { return (T)v; }

// warp min / max over the valid lanes of one component row, in the
// trajectory's own precision (no FP64 work for binary32 samples); lane 0
// writes the pair as binary64
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return kmax(a, b); }
__device__ __forceinline__ bool tfinite(float v) { return isfinite(v); }
__device__ __forceinline__ bool tfinite(double v) { return kfinite(v); }

template <class T>
__device__ __forceinline__ void warp_minmax(T v, bool valid, double *plo, double *phi, int *status) {
    const T inf = (T)INFINITY;
    T a = valid ? v : inf, b = valid ? v : -inf;
    const bool bad = valid && !tfinite(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = tmin(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = tmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
    if ((threadIdx.x & 31) == 0) { *plo = (double)a; *phi = (double)b; }
}

// the same over each group of SB consecutive lanes (SB = 2, 8 or 32), every
// lane taking part; the group's first lane writes.  `active`: the lane holds a
// row of the state.
template <int SB, class T>
__device__ __forceinline__ void group_minmax(T v, bool valid, bool active, double *plo, double *phi,
                                             int *status) {
    if (SB == 32) {
        if (active) warp_minmax<T>(v, valid, plo, phi, status);
        return;
    }
    const T inf = (T)INFINITY;
    T a = valid ? v : inf, b = valid ? v : -inf;
    const bool bad = active && valid && !tfinite(v);
#pragma unroll
    for (int o = SB / 2; o > 0; o >>= 1) {
        a = tmin(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = tmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    if (active && (threadIdx.x % SB) == 0) { *plo = (double)a; *phi = (double)b; }
}

struct McArgs {
    int64_t n, nw, m, N;
    double h;
    uint64_t seed;
    const double *xlo, *xhi, *wlo, *whi, *prm;
    double *plo, *phi;   // partials [block][n]
    int *status;
};

// ------------------------------------------------------------------ on-chip
// A block holds SB samples (smp = threadIdx % SB) of the whole state; its
// threads form G = blockDim / SB row groups, group g holding rows g, g + G, ...
// (at most Q <= MC_Q).  Sample j = block * SB + smp draws the same Philox numbers
// whatever SB is, so the box does not depend on the layout.
template <int SYS, class T, int SB, int Q>
__global__ void __launch_bounds__(MC_THREADS) mc_onchip(McArgs a) {
    extern __shared__ unsigned char smraw[];
    T *Y = (T *)smraw;                    // [n][SB]
    T *P = Y + a.n * SB;                  // [nw][SB]
    const int smp = (int)(threadIdx.x % SB), grp = (int)(threadIdx.x / SB), G = (int)(blockDim.x / SB);
    const int64_t j = (int64_t)blockIdx.x * SB + smp;   // sample
    const bool valid = j < a.m;
    const int n = (int)a.n;
    T q[4];
    mc_consts<SYS, T>(a.prm, q);
    int flags = 0;

    for (int k = grp; k < (int)a.nw; k += G) {
        double lo = a.wlo[k], hi = a.whi[k];
        if (smp == 0 && !(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
        P[k * SB + smp] = as_run<T>(box_sample(lo, hi, philox_uniform(a.seed, (uint32_t)j, (uint32_t)k, 1u)));
    }
    T z[Q], acc[Q], kk[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        int c = grp + s * G;
        z[s] = acc[s] = T(0);
        if (c < n) {
            double lo = a.xlo[c], hi = a.xhi[c];
            if (smp == 0 && !(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
            z[s] = as_run<T>(box_sample(lo, hi, philox_uniform(a.seed, (uint32_t)j, (uint32_t)c, 0u)));
            Y[c * SB + smp] = z[s];
        }
    }
    __syncthreads();
    const bool wrap = (SYS == REACH_KS);
    auto row = [&](int c) -> T {
        if (wrap) c = c < 0 ? c + n : (c >= n ? c - n : c);
        else if (c < 0 || c >= n) return T(0);
        return Y[c * SB + smp];
    };
    auto pin = [&](int k) -> T { return P[k * SB + smp]; };
    const T h = (T)a.h, hh = (T)(0.5 * a.h), h6 = (T)(a.h / 6.0);
    for (int64_t step = 0; step < a.N; ++step) {
#pragma unroll 1
        for (int stage = 0; stage < 4; ++stage) {
#pragma unroll
            for (int s = 0; s < Q; ++s) {
                int c = grp + s * G;
                if (c < n) {
                    if constexpr (SYS == REACH_LINEAR)
                        kk[s] = Plain<SYS, T>::rhs(q, row, c, c, a.n, pin, a.prm);
                    else
                        kk[s] = Plain<SYS, T>::rhs(q, row, c, c, a.n, pin);
                }
            }
            __syncthreads();
            const T cst = (stage == 2) ? h : hh;
#pragma unroll
            for (int s = 0; s < Q; ++s) {
                int c = grp + s * G;
                if (c < n) {
                    T y;
                    if (stage == 0) acc[s] = kk[s];
                    else if (stage < 3) acc[s] = tfma(T(2), kk[s], acc[s]);
                    else acc[s] += kk[s];
                    if (stage < 3) y = tfma(cst, kk[s], z[s]);
                    else { z[s] = tfma(h6, acc[s], z[s]); y = z[s]; }
                    Y[c * SB + smp] = y;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        // every lane of a group takes part in its shuffles (a group's lanes
        // share their row count, so no lane of a warp leaves early)
        const int c = grp + s * G;
        const int cc = c < n ? c : 0;
        group_minmax<SB, T>(z[s], valid, c < n, a.plo + blockIdx.x * a.n + cc, a.phi + blockIdx.x * a.n + cc,
                            a.status);
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ streaming
// Large stencil systems.  State in HBM, sample-fastest (x[i * M + j]); one
// launch advances S RK4 steps.  A block covers 32 samples (lane = sample) and
// WPB * MC_B consecutive components (rows); each warp owns MC_B rows in
// registers, so the stencil along the rows is register-local and only R edge
// rows per warp cross warps, through a small double-buffered shared-memory
// exchange (one barrier per stage).  The 4 R S halo rows at each end of the
// block are recomputed; the first launch draws the samples, the last one
// reduces them.
struct McStep {
    int64_t n, M, m;          // M: padded sample count (row stride)
    int64_t nM;               // n * M, the state size (computed on the host)
    int TC, H;                // owned rows per block, halo rows per side (4 R S)
    unsigned ntile;           // ceil(n / TC), computed on the host
    int S;                    // RK4 steps in this launch (0: only sample, t_final = 0)
    double h, hh, h6;         // h, h/2, h/6 (computed on the host)
    float hf[3];              // the same rounded to binary32, and the system
    float qf[4];              // constants as mc_consts forms them (host-rounded:
                              // a conversion would occupy the FP64 pipe)
    uint64_t seed;
    const double *xlo, *xhi;  // first launch: the initial box
    double dlo, dhi;          // traffic inflow box
    const void *in;           // state (T) of the previous launch
    void *out;
    double *plo, *phi;        // last launch: partials [sample block][n]
    int first, last;
    int *status;
};

constexpr int MC_B = 16;   // rows per warp

// the same for a cell with a right neighbour inside the chain (0 <= g < n - 1)
template <class T>
__device__ __forceinline__ T tr_flux_interior(const T (&q)[4], T y, T yr) {
    return tmin3(q[0], q[1] * y, tfma(-q[2], yr, q[3]));
}

// traffic flux out of global cell g from its value y and its right neighbour yr
template <class T>
__device__ __forceinline__ T tr_flux(const T (&q)[4], T y, T yr, int64_t g, int64_t n, T d) {
    T cong = (g == n - 1) ? q[0] : tfma(-q[2], yr, q[3]);
    T f = tmin3(q[0], q[1] * y, cong);
    f = (g == -1) ? d : f;
    return (g < -1 || g >= n) ? T(0) : f;
}

// Two blocks per SM for every variant: the traffic ones then spill a little
// (64 / 128 registers) and still run 5% (binary32) and 7% (binary64) faster
// than one block at 128 / 254 registers; KS binary64 fits 126 registers (+2%).
template <int SYS, class T, int WPB, int MINB = 2>
__global__ void __launch_bounds__(32 * WPB, MINB)
mc_stream(McStep a, const double *__restrict__ prm) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    constexpr int B = MC_B;
    __shared__ T edge[2][WPB][2 * R][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = a.n;
    const int64_t tile = blockIdx.x % a.ntile, sb = blockIdx.x / a.ntile;   // 32-bit division
    const int64_t j = sb * 32 + lane;
    const bool valid = j < a.m;
    const int64_t own0 = tile * a.TC;
    const int64_t row0 = own0 - a.H + (int64_t)warp * B;   // global row of this warp's first row
    T q[4];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = a.qf[i];
    } else {
        mc_consts<SYS, T>(prm, q);
    }
    int flags = 0;
    T d = T(0);
    if (SYS == REACH_TRAFFIC) d = as_run<T>(box_sample(a.dlo, a.dhi, philox_uniform(a.seed, (uint32_t)j, 0u, 1u)));
    // Row offsets advance by additions, and the few products are 32 x 32 -> 64
    // bit (n, M < 2^32): a 64-bit integer multiply would occupy this GPU's FP64
    // pipe, which an FP32 trajectory does not otherwise use.
    const int64_t nM = a.nM;
    const int64_t wr0 = (SYS == REACH_KS) ? wrap_index(row0, n) : row0;
    int64_t off = (int64_t)(int32_t)wr0 * (int32_t)a.M + j;
    int64_t gi = wr0;              // wrapped row index
    T z[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const int64_t g = row0 + r;
        bool in = true;
        if (SYS == REACH_KS) {
            if (off >= nM) { off -= nM; gi -= n; }
        } else {
            in = g >= 0 && g < n;
        }
        T v = T(0);
        if (in) {
            if (a.first) {
                double lo = a.xlo[gi], hi = a.xhi[gi];
                const bool owned = g >= own0 && g < own0 + a.TC;
                if (lane == 0 && owned && !(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
                v = as_run<T>(box_sample(lo, hi, philox_uniform(a.seed, (uint32_t)j, (uint32_t)gi, 0u)));
            } else {
                v = ((const T *)a.in)[off];
            }
        }
        z[r] = v;
        off += a.M;
        ++gi;
    }
    T h = (T)a.h, hh = (T)a.hh, h6 = (T)a.h6;
    if constexpr (sizeof(T) == 4) {
        h = a.hf[0];
        hh = a.hf[1];
        h6 = a.hf[2];
    }
    // A traffic warp whose fluxes are all between two cells of the chain (rows
    // row0 - 1 .. row0 + B - 1 inside [0, n - 1)) takes them without the
    // boundary selects, which cost issue slots in this issue-bound kernel.
    const bool interior = SYS != REACH_KS && row0 >= 1 && row0 + B <= n - 1;
    int buf = 0;
    auto steps = [&](auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;
        (void)IN;
        for (int s = 0; s < a.S; ++s) {
            // e[R + r] is the stage input of row r; e[0..R) and e[R+B..) hold the
            // neighbouring warps' edge rows
            T e[B + 2 * R], acc[B];
#pragma unroll
            for (int r = 0; r < B; ++r) e[R + r] = z[r];
#pragma unroll
            for (int stage = 0; stage < 4; ++stage) {
#pragma unroll
                for (int q2 = 0; q2 < R; ++q2) {
                    edge[buf][warp][q2][lane] = e[R + q2];
                    edge[buf][warp][R + q2][lane] = e[B + q2];
                }
                __syncthreads();
#pragma unroll
                for (int q2 = 0; q2 < R; ++q2) {
                    e[q2] = warp > 0 ? edge[buf][warp - 1][R + q2][lane] : T(0);
                    e[B + R + q2] = warp < WPB - 1 ? edge[buf][warp + 1][q2][lane] : T(0);
                }
                buf ^= 1;
                // derivative of row r, then the update of row r - R, whose stage
                // input row r was the last to read; only R + 1 derivatives are live
                T kring[R + 1];
                T fprev = T(0);
                (void)fprev;
                if constexpr (SYS != REACH_KS)   // flux into row 0
                    fprev = IN ? tr_flux_interior<T>(q, e[0], e[1]) : tr_flux<T>(q, e[0], e[1], row0 - 1, n, d);
#pragma unroll
                for (int r = 0; r < B + R; ++r) {
                    if (r < B) {
                        T kr;
                        if constexpr (SYS == REACH_KS) {
                            T um2 = e[r], um1 = e[r + 1], u = e[r + 2], up1 = e[r + 3], up2 = e[r + 4];
                            kr = tfma(u, tfma(-q[3], up1 - um1, q[0]), tfma(q[1], um1 + up1, q[2] * (um2 + up2)));
                        } else {
                            T fout = IN ? tr_flux_interior<T>(q, e[r + 1], e[r + 2])
                                        : tr_flux<T>(q, e[r + 1], e[r + 2], row0 + r, n, d);
                            kr = fprev - fout;
                            fprev = fout;
                        }
                        kring[r % (R + 1)] = kr;
                    }
                    if (r >= R) {
                        const int u = r - R;
                        const T k = kring[u % (R + 1)];
                        if (stage == 0) { acc[u] = k; e[R + u] = tfma(hh, k, z[u]); }
                        if (stage == 1) { acc[u] = tfma(T(2), k, acc[u]); e[R + u] = tfma(hh, k, z[u]); }
                        if (stage == 2) { acc[u] = tfma(T(2), k, acc[u]); e[R + u] = tfma(h, k, z[u]); }
                        if (stage == 3) { acc[u] += k; z[u] = tfma(h6, acc[u], z[u]); e[R + u] = z[u]; }
                    }
                }
            }
        }
    };
    if (interior) steps(std::true_type{});
    else steps(std::false_type{});
    int64_t oo = (int64_t)(int32_t)row0 * (int32_t)a.M + j;   // store offset of row 0 (owned rows are in range)
    const int64_t pb = (int64_t)((uint64_t)(uint32_t)sb * (uint32_t)n);
    double *plo = a.plo + pb + row0, *phi = a.phi + pb + row0;
#pragma unroll
    for (int r = 0; r < B; ++r, oo += a.M) {
        const int64_t g = row0 + r;
        if (g < own0 || g >= own0 + a.TC || g >= n) continue;   // warp-uniform
        if (a.last) warp_minmax<T>(z[r], valid, plo + r, phi + r, a.status);
        else ((T *)a.out)[oo] = z[r];
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ streaming, two samples per lane
// The binary32 streaming kernel is issue-bound: one sample per lane spends an
// issue slot on every FP32 operation.  Blackwell's packed FP32 instructions
// (__ffma2_rn, __fadd2_rn, __fmul2_rn: two IEEE binary32 operations, each
// rounded to nearest, in one issue) let a lane carry two adjacent samples
// j0 = 64 sb + 2 lane and j0 + 1 as a float2, halving the arithmetic
// instructions per sample and making every state access one 8-byte access per
// lane.  Each sample sees the same operations in the same order as in
// mc_stream, so the two kernels give the same box bit for bit.  Minima have no
// packed form and stay per sample (traffic only: one three-input minimum per
// flux and sample).  A block covers 64 samples and WPB * B rows; the state
// rows hold M samples, M a multiple of 64.
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 min3_2(float2 a, float2 b, float2 c) {
    return make_float2(tmin3(a.x, b.x, c.x), tmin3(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 sel2(bool p, float2 a, float2 b) { return p ? a : b; }

struct Q2 {
    float2 cap, v, nw, wxbar;   // traffic: cap, v, -w, w xbar
    float2 a0, a1, a2, nk;      // KS: a0, a1, a2, -k
};

__device__ __forceinline__ float2 tr_flux2_interior(const Q2 &q, float2 y, float2 yr) {
    return min3_2(q.cap, mul2(q.v, y), fma2(q.nw, yr, q.wxbar));
}

__device__ __forceinline__ float2 tr_flux2(const Q2 &q, float2 y, float2 yr, int64_t g, int64_t n, float2 d) {
    const float2 cong = (g == n - 1) ? q.cap : fma2(q.nw, yr, q.wxbar);
    float2 f = min3_2(q.cap, mul2(q.v, y), cong);
    f = sel2(g == -1, d, f);
    return sel2(g < -1 || g >= n, bc2(0.f), f);
}

// min / max of one component row over the warp's 64 samples (valid ones only)
__device__ __forceinline__ void warp_minmax2(float2 v, bool v0, bool v1, double *plo, double *phi, int *status) {
    float a = fminf(v0 ? v.x : INFINITY, v1 ? v.y : INFINITY);
    float b = fmaxf(v0 ? v.x : -INFINITY, v1 ? v.y : -INFINITY);
    const bool bad = (v0 && !isfinite(v.x)) || (v1 && !isfinite(v.y));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
    if ((threadIdx.x & 31) == 0) { *plo = (double)a; *phi = (double)b; }
}

template <int SYS, int WPB, int B, int MINB>
__global__ void __launch_bounds__(32 * WPB, MINB) mc_stream2(McStep a) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    __shared__ float2 edge[2][WPB][2 * R][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = a.n;
    const int64_t tile = blockIdx.x % a.ntile, sb = blockIdx.x / a.ntile;   // 32-bit division
    const int64_t j0 = sb * 64 + 2 * lane;
    const bool v0 = j0 < a.m, v1 = j0 + 1 < a.m;
    const int64_t own0 = tile * a.TC;
    const int64_t row0 = own0 - a.H + (int64_t)warp * B;
    Q2 q;
    q.cap = bc2(a.qf[0]); q.v = bc2(a.qf[1]); q.nw = bc2(-a.qf[2]); q.wxbar = bc2(a.qf[3]);
    q.a0 = bc2(a.qf[0]); q.a1 = bc2(a.qf[1]); q.a2 = bc2(a.qf[2]); q.nk = bc2(-a.qf[3]);
    int flags = 0;
    float2 d = bc2(0.f);
    if (SYS == REACH_TRAFFIC) {
        d.x = (float)box_sample(a.dlo, a.dhi, philox_uniform(a.seed, (uint32_t)j0, 0u, 1u));
        d.y = (float)box_sample(a.dlo, a.dhi, philox_uniform(a.seed, (uint32_t)(j0 + 1), 0u, 1u));
    }
    const int64_t nM = a.nM;
    const int64_t wr0 = (SYS == REACH_KS) ? wrap_index(row0, n) : row0;
    int64_t off = (int64_t)(int32_t)wr0 * (int32_t)a.M + j0;   // in floats; even
    int64_t gi = wr0;
    float2 z[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const int64_t g = row0 + r;
        bool in = true;
        if (SYS == REACH_KS) {
            if (off >= nM) { off -= nM; gi -= n; }
        } else {
            in = g >= 0 && g < n;
        }
        float2 v = bc2(0.f);
        if (in) {
            if (a.first) {
                const double lo = a.xlo[gi], hi = a.xhi[gi];
                const bool owned = g >= own0 && g < own0 + a.TC;
                if (lane == 0 && owned && !(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
                v.x = (float)box_sample(lo, hi, philox_uniform(a.seed, (uint32_t)j0, (uint32_t)gi, 0u));
                v.y = (float)box_sample(lo, hi, philox_uniform(a.seed, (uint32_t)(j0 + 1), (uint32_t)gi, 0u));
            } else {
                v = *reinterpret_cast<const float2 *>((const float *)a.in + off);
            }
        }
        z[r] = v;
        off += a.M;
        ++gi;
    }
    const float2 h = bc2(a.hf[0]), hh = bc2(a.hf[1]), h6 = bc2(a.hf[2]), two = bc2(2.f);
    const bool interior = SYS != REACH_KS && row0 >= 1 && row0 + B <= n - 1;
    int buf = 0;
    auto steps = [&](auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;
        (void)IN;
        for (int s = 0; s < a.S; ++s) {
            float2 e[B + 2 * R], acc[B];
#pragma unroll
            for (int r = 0; r < B; ++r) e[R + r] = z[r];
#pragma unroll
            for (int stage = 0; stage < 4; ++stage) {
#pragma unroll
                for (int q2 = 0; q2 < R; ++q2) {
                    edge[buf][warp][q2][lane] = e[R + q2];
                    edge[buf][warp][R + q2][lane] = e[B + q2];
                }
                __syncthreads();
#pragma unroll
                for (int q2 = 0; q2 < R; ++q2) {
                    e[q2] = warp > 0 ? edge[buf][warp - 1][R + q2][lane] : bc2(0.f);
                    e[B + R + q2] = warp < WPB - 1 ? edge[buf][warp + 1][q2][lane] : bc2(0.f);
                }
                buf ^= 1;
                float2 kring[R + 1];
                float2 fprev = bc2(0.f);
                (void)fprev;
                if constexpr (SYS != REACH_KS)
                    fprev = IN ? tr_flux2_interior(q, e[0], e[1]) : tr_flux2(q, e[0], e[1], row0 - 1, n, d);
#pragma unroll
                for (int r = 0; r < B + R; ++r) {
                    if (r < B) {
                        float2 kr;
                        if constexpr (SYS == REACH_KS) {
                            const float2 um2 = e[r], um1 = e[r + 1], u = e[r + 2], up1 = e[r + 3], up2 = e[r + 4];
                            kr = fma2(u, fma2(q.nk, sub2(up1, um1), q.a0),
                                      fma2(q.a1, add2(um1, up1), mul2(q.a2, add2(um2, up2))));
                        } else {
                            const float2 fout = IN ? tr_flux2_interior(q, e[r + 1], e[r + 2])
                                                   : tr_flux2(q, e[r + 1], e[r + 2], row0 + r, n, d);
                            kr = sub2(fprev, fout);
                            fprev = fout;
                        }
                        kring[r % (R + 1)] = kr;
                    }
                    if (r >= R) {
                        const int u = r - R;
                        const float2 k = kring[u % (R + 1)];
                        if (stage == 0) { acc[u] = k; e[R + u] = fma2(hh, k, z[u]); }
                        if (stage == 1) { acc[u] = fma2(two, k, acc[u]); e[R + u] = fma2(hh, k, z[u]); }
                        if (stage == 2) { acc[u] = fma2(two, k, acc[u]); e[R + u] = fma2(h, k, z[u]); }
                        if (stage == 3) { acc[u] = add2(acc[u], k); z[u] = fma2(h6, acc[u], z[u]); e[R + u] = z[u]; }
                    }
                }
            }
        }
    };
    if (interior) steps(std::true_type{});
    else steps(std::false_type{});
    int64_t oo = (int64_t)(int32_t)row0 * (int32_t)a.M + j0;
    const int64_t pb = (int64_t)((uint64_t)(uint32_t)sb * (uint32_t)n);
    double *plo = a.plo + pb + row0, *phi = a.phi + pb + row0;
#pragma unroll
    for (int r = 0; r < B; ++r, oo += a.M) {
        const int64_t g = row0 + r;
        if (g < own0 || g >= own0 + a.TC || g >= n) continue;   // warp-uniform
        if (a.last) warp_minmax2(z[r], v0, v1, plo + r, phi + r, a.status);
        else *reinterpret_cast<float2 *>((float *)a.out + oo) = z[r];
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ streaming, two samples per lane, prefetched
// mc_stream2 loads a block's state rows when the block starts, so with one
// block per SM the FP32 pipe waits out every tile's load.  Here the blocks
// are persistent and the next tiles' rows arrive ahead of time: one thread
// issues a bulk copy (cp.async.bulk, the TMA engine) of each 256-byte row
// segment (64 samples) into a double-buffered shared-memory tile, counted on
// an mbarrier; the warps wait on it, move their rows into registers, and the
// copy of the tile after next starts into the freed buffer while they
// compute.  Every wait on an mbarrier is bounded (ST_TIMEOUT).  Used for the
// launches after the first (the first draws the samples); the arithmetic is
// mc_stream2's, so the box is the same bit for bit.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}

// bounded wait for phase `parity` of an mbarrier (about 2 s); false on timeout
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(b, parity)) {
        if (global_ns() - t0 > 2000000000ULL) return false;
    }
    return true;
}

// one 2-D tensor copy (TMA) of a box of ROWS rows x 64 samples at (x, y) =
// (first sample, first row); rows outside the tensor arrive as zeros
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(b))
        : "memory");
}

template <int SYS, int WPB, int B>
__global__ void __launch_bounds__(32 * WPB, 1) mc_stream2p(McStep a, unsigned long long items,
                                                          const __grid_constant__ CUtensorMap map) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    constexpr int ROWS = WPB * B;
    extern __shared__ __align__(128) float2 tbuf[];   // [2][ROWS][32]
    __shared__ float2 edge[2][WPB][2 * R][32];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int ready;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = a.n;
    Q2 q;
    q.cap = bc2(a.qf[0]); q.v = bc2(a.qf[1]); q.nw = bc2(-a.qf[2]); q.wxbar = bc2(a.qf[3]);
    q.a0 = bc2(a.qf[0]); q.a1 = bc2(a.qf[1]); q.a2 = bc2(a.qf[2]); q.nk = bc2(-a.qf[3]);
    const float2 h = bc2(a.hf[0]), hh = bc2(a.hf[1]), h6 = bc2(a.hf[2]), two = bc2(2.f);
    const unsigned long long G = gridDim.x;

    // rows of item it: its tile's first halo row and sample block
    auto item_rows = [&](unsigned long long it, int64_t &row0b, int64_t &sb) {
        const int64_t tile = (int64_t)(it % a.ntile);
        sb = (int64_t)(it / a.ntile);
        row0b = tile * a.TC - a.H;
    };
    // warp 0: the copies of item it into buffer k.  One tensor copy of the
    // whole box (rows outside a traffic chain arrive as zeros); a KS box that
    // wraps around the periodic grid takes one row copy per lane in turn
    // (lane 0 announces the bytes first in both cases)
    auto issue = [&](unsigned long long it, int k) {
        int64_t row0b, sb;
        item_rows(it, row0b, sb);
        if (SYS != REACH_KS || (row0b >= 0 && row0b + ROWS <= n)) {
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bar[k], (uint32_t)(ROWS * 256));
                tma_load_2d(tbuf + (size_t)k * ROWS * 32, &map, (int)(sb * 64), (int)row0b, &bar[k]);
            }
            __syncwarp();
            return;
        }
        int64_t rows_in = ROWS;
        if (SYS != REACH_KS) {
            const int64_t lo = row0b > 0 ? row0b : 0, hi = row0b + ROWS < n ? row0b + ROWS : n;
            rows_in = hi > lo ? hi - lo : 0;
        }
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[k], (uint32_t)(rows_in * 256));
        }
        __syncwarp();
        const float *src = (const float *)a.in;
        for (int r = lane; r < ROWS; r += 32) {
            const int64_t g = row0b + r;
            int64_t gi = g;
            if (SYS == REACH_KS) gi = wrap_index(g, n);
            else if (g < 0 || g >= n) continue;
            bulk_g2s(tbuf + ((size_t)k * ROWS + r) * 32, src + gi * a.M + sb * 64, 256, &bar[k]);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        if (blockIdx.x < items) issue(blockIdx.x, 0);
        if (blockIdx.x + G < items) issue(blockIdx.x + G, 1);
    }
    uint32_t ph[2] = {0, 0};
    int flags = 0, buf = 0;
    bool timed_out = false;
    int k = 0;
    for (unsigned long long it = blockIdx.x; it < items; it += G, k ^= 1) {
        int64_t row0b, sb;
        item_rows(it, row0b, sb);
        const int64_t own0 = row0b + a.H;
        const int64_t j0 = sb * 64 + 2 * lane;
        const bool v0 = j0 < a.m, v1 = j0 + 1 < a.m;
        const int64_t row0 = row0b + (int64_t)warp * B;
        float2 d = bc2(0.f);
        if (SYS == REACH_TRAFFIC) {
            d.x = (float)box_sample(a.dlo, a.dhi, philox_uniform(a.seed, (uint32_t)j0, 0u, 1u));
            d.y = (float)box_sample(a.dlo, a.dhi, philox_uniform(a.seed, (uint32_t)(j0 + 1), 0u, 1u));
        }
        // thread 0 waits (bounded) and tells the block, so that a timeout
        // leaves the loop in every thread at the same point
        if (threadIdx.x == 0) ready = mbar_wait_bounded(&bar[k], ph[k]) ? 1 : 0;
        __syncthreads();
        if (!ready) {
            timed_out = true;
            break;
        }
        // the phase is complete: each thread's own wait returns at once and
        // makes the copied rows visible to it
        mbar_wait_bounded(&bar[k], ph[k]);
        ph[k] ^= 1;
        float2 z[B];
#pragma unroll
        for (int r = 0; r < B; ++r) {
            const int64_t g = row0 + r;
            const bool in = SYS == REACH_KS || (g >= 0 && g < n);
            z[r] = in ? tbuf[((size_t)k * ROWS + warp * B + r) * 32 + lane] : bc2(0.f);
        }
        __syncthreads();   // buffer k is free: the copy of the item after next starts
        if (warp == 0 && it + 2 * G < items) issue(it + 2 * G, k);
        const bool interior = SYS != REACH_KS && row0 >= 1 && row0 + B <= n - 1;
        auto steps = [&](auto in_tag) {
            constexpr bool IN = decltype(in_tag)::value;
            (void)IN;
            for (int s = 0; s < a.S; ++s) {
                float2 e[B + 2 * R], acc[B];
#pragma unroll
                for (int r = 0; r < B; ++r) e[R + r] = z[r];
#pragma unroll
                for (int stage = 0; stage < 4; ++stage) {
#pragma unroll
                    for (int q2 = 0; q2 < R; ++q2) {
                        edge[buf][warp][q2][lane] = e[R + q2];
                        edge[buf][warp][R + q2][lane] = e[B + q2];
                    }
                    __syncthreads();
#pragma unroll
                    for (int q2 = 0; q2 < R; ++q2) {
                        e[q2] = warp > 0 ? edge[buf][warp - 1][R + q2][lane] : bc2(0.f);
                        e[B + R + q2] = warp < WPB - 1 ? edge[buf][warp + 1][q2][lane] : bc2(0.f);
                    }
                    buf ^= 1;
                    float2 kring[R + 1];
                    float2 fprev = bc2(0.f);
                    (void)fprev;
                    if constexpr (SYS != REACH_KS)
                        fprev = IN ? tr_flux2_interior(q, e[0], e[1]) : tr_flux2(q, e[0], e[1], row0 - 1, n, d);
#pragma unroll
                    for (int r = 0; r < B + R; ++r) {
                        if (r < B) {
                            float2 kr;
                            if constexpr (SYS == REACH_KS) {
                                const float2 um2 = e[r], um1 = e[r + 1], u = e[r + 2], up1 = e[r + 3], up2 = e[r + 4];
                                kr = fma2(u, fma2(q.nk, sub2(up1, um1), q.a0),
                                          fma2(q.a1, add2(um1, up1), mul2(q.a2, add2(um2, up2))));
                            } else {
                                const float2 fout = IN ? tr_flux2_interior(q, e[r + 1], e[r + 2])
                                                       : tr_flux2(q, e[r + 1], e[r + 2], row0 + r, n, d);
                                kr = sub2(fprev, fout);
                                fprev = fout;
                            }
                            kring[r % (R + 1)] = kr;
                        }
                        if (r >= R) {
                            const int u = r - R;
                            const float2 kk = kring[u % (R + 1)];
                            if (stage == 0) { acc[u] = kk; e[R + u] = fma2(hh, kk, z[u]); }
                            if (stage == 1) { acc[u] = fma2(two, kk, acc[u]); e[R + u] = fma2(hh, kk, z[u]); }
                            if (stage == 2) { acc[u] = fma2(two, kk, acc[u]); e[R + u] = fma2(h, kk, z[u]); }
                            if (stage == 3) { acc[u] = add2(acc[u], kk); z[u] = fma2(h6, acc[u], z[u]); e[R + u] = z[u]; }
                        }
                    }
                }
            }
        };
        if (interior) steps(std::true_type{});
        else steps(std::false_type{});
        int64_t oo = (int64_t)(int32_t)row0 * (int32_t)a.M + j0;
        const int64_t pb = (int64_t)((uint64_t)(uint32_t)sb * (uint32_t)n);
        double *plo = a.plo + pb + row0, *phi = a.phi + pb + row0;
#pragma unroll
        for (int r = 0; r < B; ++r, oo += a.M) {
            const int64_t g = row0 + r;
            if (g < own0 || g >= own0 + a.TC || g >= n) continue;   // warp-uniform
            if (a.last) warp_minmax2(z[r], v0, v1, plo + r, phi + r, a.status);
            else *reinterpret_cast<float2 *>((float *)a.out + oo) = z[r];
        }
    }
    if (timed_out) {
        flags |= ST_TIMEOUT;
        // let copies still in flight land before the block's shared memory goes (bounded)
        if (threadIdx.x == 0)
            for (int kk = 0; kk < 2; ++kk) mbar_wait_bounded(&bar[kk], ph[kk]);
        __syncthreads();
    }
    if (flags && (threadIdx.x & 31) == 0) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ streaming, sample pairs along the rows
// State layout: sample pair p (samples 2p and 2p + 1) is a contiguous run of
// n float2 rows, x[p ns + i] (ns = n rounded up to even, so every run starts
// on 16 bytes).  A warp owns 32 KC consecutive rows of one pair, KC per lane
// in registers: stencil neighbours come from the adjacent lanes by shuffles,
// so a warp never waits for another one (no shared memory, no block barrier,
// against one barrier per stage in mc_stream2), and a warp tile longer than a
// lane-per-sample block keeps the recomputed halo of 4 R S rows per side a
// smaller share.  Persistent warps take (pair, tile) items; the first launch
// draws the samples, and the per-row minimum and maximum over the samples is
// one coalesced pass over the final state (mc_rows_reduce).  Each sample sees
// the operations of mc_stream2 in the same order, so the box is the same bit
// for bit.
struct RowStep {
    int64_t n, ns;            // rows, row stride of a pair's run (even)
    int64_t m;                // samples (drawn beyond m up to 2P, never reduced)
    unsigned P;               // sample pairs (binary64 kernel: samples)
    unsigned ntile;           // ceil(n / W)
    int W, H;                 // owned rows per warp tile, halo rows per side (4 R S)
    int S;                    // RK4 steps in this launch (0: only draw the samples)
    float hf[3];              // h, h/2, h/6 rounded to binary32 on the host
    float qf[4];              // system constants as mc_stream2 takes them
    double h, h6;             // binary64 kernel: h and h/6 (the host's)
    double one, nzero;        // binary64 kernel: 1 and -0 (fadd / fmul)
    uint64_t seed;
    const double *xlo, *xhi;  // first launch: the initial box
    double dlo, dhi;          // traffic inflow box
    const void *in;           // state of the previous launch (float2 pairs or doubles)
    void *out;
    int first;
    int *status;
    unsigned *ctr;            // mc_rows: two item counters; this launch takes ctr[slot]
    int slot;                 // and clears the other one for the next launch
};

// 16-byte global -> shared copy by the executing thread (cp.async, cached in
// L2 only); complete and visible to that thread after cp_async_wait_all
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// mc_rows copies the next item's rows ahead on the traffic chain (2^20 cells,
// 256 samples, 200 steps: 0.0599 s against 0.0613 s); on the KS grid, bound by
// the FP32 pipe, the copies cost more than they hide (1024 samples, 500 steps:
// 0.717 s against 0.699 s), so it loads each item's rows when it starts it
template <int SYS>
__host__ __device__ constexpr bool rows_prefetch() { return SYS == REACH_TRAFFIC; }
// dynamic shared memory of mc_rows: per warp two stage buffers of 32 KC / 2
// float4 (a lane's rows of one item, r-major so that a warp's accesses to row
// pair r are 512 contiguous bytes)
template <int SYS, int KC>
constexpr size_t rows_stage_bytes() { return rows_prefetch<SYS>() ? 8 * 2 * (KC / 2) * 32 * sizeof(float4) : 0; }

template <int SYS, int KC>
__global__ void __launch_bounds__(256, 2) mc_rows(RowStep a) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    constexpr bool PF = rows_prefetch<SYS>();
    extern __shared__ float4 rows_stage[];
    const unsigned lane = threadIdx.x & 31;
    float4 *stage = rows_stage + (threadIdx.x >> 5) * (2 * (KC / 2) * 32) + lane;
    const uint32_t items = a.ntile * a.P;   // items + 2 warps < 2^32 (checked on the host)
    const int64_t n = a.n;
    unsigned *ctr = a.ctr + a.slot;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctr[a.slot ^ 1] = 0u;   // the next launch's counter
    Q2 q;
    q.cap = bc2(a.qf[0]); q.v = bc2(a.qf[1]); q.nw = bc2(-a.qf[2]); q.wxbar = bc2(a.qf[3]);
    q.a0 = bc2(a.qf[0]); q.a1 = bc2(a.qf[1]); q.a2 = bc2(a.qf[2]); q.nk = bc2(-a.qf[3]);
    const float2 h = bc2(a.hf[0]), hh = bc2(a.hf[1]), h6 = bc2(a.hf[2]), two = bc2(2.f);
    int flags = 0;
    // Warps take items from the counter as they finish the previous one, so a
    // warp that the scheduler favours takes more of them (with a fixed stride
    // the favoured warps finish first and their SM runs the rest with fewer
    // warps).  Lane 0 asks for the next item before the warp works on the
    // current one.  With PF a warp knows its next item while it works on the
    // current one and copies the next item's rows into its other stage buffer
    // meanwhile (launches after the first, lanes whose run lies inside the
    // chain), and lane 0 asks for the item after that.  One lane's successive
    // requests are ordered, so a warp's items increase and it stops at the
    // first one past the end, having asked once (twice with PF) past the end:
    // the counter ends at items + warps (items + 2 warps).
    uint32_t req = 0, req2 = 0;
    if (lane == 0) {
        req = atomicAdd(ctr, 1u);
        if (PF) req2 = atomicAdd(ctr, 1u);
    }
    uint32_t it = __shfl_sync(0xffffffffu, req, 0);
    uint32_t nx = PF ? __shfl_sync(0xffffffffu, req2, 0) : 0u;
    bool staged = false;   // this lane's rows of item `it` are in stage buffer `sb`
    int sb = 0;
    while (it < items) {
        if (lane == 0) req = atomicAdd(ctr, 1u);
        const uint32_t p = it / a.ntile, t = it - p * a.ntile;
        const int64_t own0 = (int64_t)t * a.W;
        const int64_t g0 = own0 - a.H + (int64_t)(lane * KC);
        const int64_t base = (int64_t)((uint64_t)p * (uint64_t)a.ns);
        const uint32_t j0 = 2 * p;
        float2 d = bc2(0.f);
        if (SYS == REACH_TRAFFIC) {
            d.x = (float)box_sample(a.dlo, a.dhi, philox_uniform(a.seed, j0, 0u, 1u));
            d.y = (float)box_sample(a.dlo, a.dhi, philox_uniform(a.seed, j0 + 1, 0u, 1u));
        }
        float2 z[KC];
        const float2 *in = static_cast<const float2 *>(a.in);
        float2 *out = static_cast<float2 *>(a.out);
        const bool whole = g0 >= 0 && g0 + KC <= n;   // the lane's run lies inside [0, n)
        if (a.first) {
#pragma unroll
            for (int r = 0; r < KC; ++r) {
                int64_t g = g0 + r;
                bool ok = true;
                if (SYS == REACH_KS) g = wrap_index(g, n);
                else ok = g >= 0 && g < n;
                float2 v = bc2(0.f);
                if (ok) {
                    const double lo = a.xlo[g], hi = a.xhi[g];
                    const bool owned = p == 0 && g0 + r >= own0 && g0 + r < own0 + a.W;
                    if (owned && !(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
                    v.x = (float)box_sample(lo, hi, philox_uniform(a.seed, j0, (uint32_t)g, 0u));
                    v.y = (float)box_sample(lo, hi, philox_uniform(a.seed, j0 + 1, (uint32_t)g, 0u));
                }
                z[r] = v;
            }
        } else if (whole) {
            if (PF && staged) {
                cp_async_wait_all();
                const float4 *src = stage + sb * ((KC / 2) * 32);
#pragma unroll
                for (int r = 0; r < KC / 2; ++r) {
                    const float4 v = src[r * 32];
                    z[2 * r] = make_float2(v.x, v.y);
                    z[2 * r + 1] = make_float2(v.z, v.w);
                }
            } else {
                const float4 *src = reinterpret_cast<const float4 *>(in + base + g0);   // g0 and base even
#pragma unroll
                for (int r = 0; r < KC / 2; ++r) {
                    const float4 v = __ldcs(src + r);
                    z[2 * r] = make_float2(v.x, v.y);
                    z[2 * r + 1] = make_float2(v.z, v.w);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < KC; ++r) {
                int64_t g = g0 + r;
                bool ok = true;
                if (SYS == REACH_KS) g = wrap_index(g, n);
                else ok = g >= 0 && g < n;
                z[r] = ok ? __ldcs(in + base + g) : bc2(0.f);
            }
        }
        // the next item's rows into the other buffer while this one computes
        // (its g0 is even like this one's: W and H are even)
        sb ^= 1;
        staged = false;
        if (PF && !a.first && nx < items) {
            const uint32_t p2 = nx / a.ntile, t2 = nx - p2 * a.ntile;
            const int64_t g2 = (int64_t)t2 * a.W - a.H + (int64_t)(lane * KC);
            if (g2 >= 0 && g2 + KC <= n) {
                const float4 *src = reinterpret_cast<const float4 *>(in + (int64_t)((uint64_t)p2 * (uint64_t)a.ns) + g2);
                float4 *dst = stage + sb * ((KC / 2) * 32);
#pragma unroll
                for (int r = 0; r < KC / 2; ++r) cp_async16(dst + r * 32, src + r);
                cp_async_commit();
                staged = true;
            }
        }
        // every flux of the lane's run between two cells of the chain; the
        // choice is warp-uniform, since the stages shuffle across the warp
        const bool interior = SYS != REACH_KS && __all_sync(0xffffffffu, g0 >= 1 && g0 + KC <= n - 1);
        auto steps = [&](auto in_tag) {
            constexpr bool IN = decltype(in_tag)::value;
            (void)IN;
            for (int s = 0; s < a.S; ++s) {
                float2 e[KC + 2 * R], acc[KC];
#pragma unroll
                for (int r = 0; r < KC; ++r) e[R + r] = z[r];
#pragma unroll
                for (int stage = 0; stage < 4; ++stage) {
                    // the R rows on each side from the neighbouring lanes (the
                    // warp's outermost halo rows take garbage, which stays in
                    // the halo)
#pragma unroll
                    for (int q2 = 0; q2 < R; ++q2) {
                        const float2 lo_ = e[KC + q2], hi_ = e[R + q2];
                        e[q2].x = __shfl_up_sync(0xffffffffu, lo_.x, 1);
                        e[q2].y = __shfl_up_sync(0xffffffffu, lo_.y, 1);
                        e[R + KC + q2].x = __shfl_down_sync(0xffffffffu, hi_.x, 1);
                        e[R + KC + q2].y = __shfl_down_sync(0xffffffffu, hi_.y, 1);
                    }
                    float2 kring[R + 1];
                    float2 fprev = bc2(0.f);
                    (void)fprev;
                    if constexpr (SYS != REACH_KS)
                        fprev = IN ? tr_flux2_interior(q, e[0], e[1]) : tr_flux2(q, e[0], e[1], g0 - 1, n, d);
#pragma unroll
                    for (int r = 0; r < KC + R; ++r) {
                        if (r < KC) {
                            float2 kr;
                            if constexpr (SYS == REACH_KS) {
                                const float2 um2 = e[r], um1 = e[r + 1], u = e[r + 2], up1 = e[r + 3], up2 = e[r + 4];
                                kr = fma2(u, fma2(q.nk, sub2(up1, um1), q.a0),
                                          fma2(q.a1, add2(um1, up1), mul2(q.a2, add2(um2, up2))));
                            } else {
                                const float2 fout = IN ? tr_flux2_interior(q, e[r + 1], e[r + 2])
                                                       : tr_flux2(q, e[r + 1], e[r + 2], g0 + r, n, d);
                                kr = sub2(fprev, fout);
                                fprev = fout;
                            }
                            kring[r % (R + 1)] = kr;
                        }
                        if (r >= R) {
                            const int u = r - R;
                            const float2 kk = kring[u % (R + 1)];
                            if (stage == 0) { acc[u] = kk; e[R + u] = fma2(hh, kk, z[u]); }
                            if (stage == 1) { acc[u] = fma2(two, kk, acc[u]); e[R + u] = fma2(hh, kk, z[u]); }
                            if (stage == 2) { acc[u] = fma2(two, kk, acc[u]); e[R + u] = fma2(h, kk, z[u]); }
                            if (stage == 3) { acc[u] = add2(acc[u], kk); z[u] = fma2(h6, acc[u], z[u]); e[R + u] = z[u]; }
                        }
                    }
                }
            }
        };
        if (interior) steps(std::true_type{});
        else steps(std::false_type{});
        // the owned rows of the lane's run
        if (whole && g0 >= own0 && g0 + KC <= own0 + a.W) {
            float4 *dst = reinterpret_cast<float4 *>(out + base + g0);
#pragma unroll
            for (int r = 0; r < KC / 2; ++r) __stcs(dst + r, make_float4(z[2 * r].x, z[2 * r].y, z[2 * r + 1].x, z[2 * r + 1].y));
        } else {
#pragma unroll
            for (int r = 0; r < KC; ++r) {
                const int64_t g = g0 + r;
                if (g >= own0 && g < own0 + a.W && g >= 0 && g < n) __stcs(out + base + g, z[r]);
            }
        }
        if (PF) {
            it = nx;
            nx = __shfl_sync(0xffffffffu, req, 0);
        } else {
            it = __shfl_sync(0xffffffffu, req, 0);
        }
    }
    if (PF) cp_async_wait_all();   // nothing stays in flight (a copy is only made for an item the warp then takes)
    if (flags) atomicOr(a.status, flags);
}

// per-row minimum and maximum over the valid samples of the pair-row state,
// written as binary64 (each bound is one sample's value, so the order of the
// scan does not matter); a non-finite sample sets ST_NONFINITE
__global__ void mc_rows_reduce(const float2 *x, int64_t ns, int64_t n, unsigned P, int64_t m, double *lo,
                               double *hi, int *status) {
    int flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float a = INFINITY, b = -INFINITY;
        bool bad = false;
        const float2 *col = x + i;
        for (unsigned p = 0; p < P; ++p) {
            const float2 v = __ldcs(col + (int64_t)((uint64_t)p * (uint64_t)ns));
            const int64_t j = 2 * (int64_t)p;
            if (j < m) { a = fminf(a, v.x); b = fmaxf(b, v.x); bad |= !isfinite(v.x); }
            if (j + 1 < m) { a = fminf(a, v.y); b = fmaxf(b, v.y); bad |= !isfinite(v.y); }
        }
        lo[i] = (double)a;
        hi[i] = (double)b;
        if (bad) flags |= ST_NONFINITE;
    }
    if (flags) atomicOr(status, flags);
}

// ------------------------------------------------------------------ streaming binary64, samples along the rows
// The binary64 version of mc_rows: sample j is a contiguous run of n doubles,
// x[j ns + i], and a warp owns 32 KC consecutive rows of one sample (KC per
// lane), neighbours by shuffles, no barrier, the 4 R S halo rows recomputed.
// Each sample sees mc_stream's operations in the same order (sums and products
// in the fused forms, which round the same), so the box is the same bit for
// bit.
template <int SYS, int KC, int MINB>
__global__ void __launch_bounds__(256, MINB) mc_rows64(RowStep a, const double *__restrict__ prm) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    const unsigned lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    const uint32_t items = a.ntile * a.P;   // P = samples here; < 2^32 (checked on the host)
    const int64_t n = a.n;
    double q[4];
    mc_consts<SYS, double>(prm, q);
    const double one = a.one, nz = a.nzero;
    const double h = a.h, hh = 0.5 * a.h, h6 = a.h6;
    int flags = 0;
    for (uint64_t it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += nwarps) {
        const uint32_t j = (uint32_t)it / a.ntile, t = (uint32_t)it - j * a.ntile;   // 32-bit division
        const int64_t own0 = (int64_t)t * a.W;
        const int64_t g0 = own0 - a.H + (int64_t)(lane * KC);
        const int64_t base = (int64_t)((uint64_t)j * (uint64_t)a.ns);
        double d = 0.0;
        if (SYS == REACH_TRAFFIC) d = box_sample(a.dlo, a.dhi, philox_uniform(a.seed, j, 0u, 1u));
        double z[KC];
        const bool whole = g0 >= 0 && g0 + KC <= n;
        const double *in = static_cast<const double *>(a.in);
        if (a.first) {
#pragma unroll
            for (int r = 0; r < KC; ++r) {
                int64_t g = g0 + r;
                bool ok = true;
                if (SYS == REACH_KS) g = wrap_index(g, n);
                else ok = g >= 0 && g < n;
                double v = 0.0;
                if (ok) {
                    const double lo = a.xlo[g], hi = a.xhi[g];
                    const bool owned = j == 0 && g0 + r >= own0 && g0 + r < own0 + a.W;
                    if (owned && !(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
                    v = box_sample(lo, hi, philox_uniform(a.seed, j, (uint32_t)g, 0u));
                }
                z[r] = v;
            }
        } else if (whole) {
            const double2 *src = reinterpret_cast<const double2 *>(in + base + g0);   // g0 and base even
#pragma unroll
            for (int r = 0; r < KC / 2; ++r) {
                const double2 v = __ldcs(src + r);
                z[2 * r] = v.x;
                z[2 * r + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int r = 0; r < KC; ++r) {
                int64_t g = g0 + r;
                bool ok = true;
                if (SYS == REACH_KS) g = wrap_index(g, n);
                else ok = g >= 0 && g < n;
                z[r] = ok ? __ldcs(in + base + g) : 0.0;
            }
        }
        const bool interior = SYS != REACH_KS && __all_sync(0xffffffffu, g0 >= 1 && g0 + KC <= n - 1);
        auto steps = [&](auto in_tag) {
            constexpr bool IN = decltype(in_tag)::value;
            (void)IN;
            for (int s = 0; s < a.S; ++s) {
                double e[KC + 2 * R], acc[KC];
#pragma unroll
                for (int r = 0; r < KC; ++r) e[R + r] = z[r];
#pragma unroll
                for (int stage = 0; stage < 4; ++stage) {
#pragma unroll
                    for (int q2 = 0; q2 < R; ++q2) {
                        e[q2] = __shfl_up_sync(0xffffffffu, e[KC + q2], 1);
                        e[R + KC + q2] = __shfl_down_sync(0xffffffffu, e[R + q2], 1);
                    }
                    double kring[R + 1];
                    double fprev = 0.0;
                    (void)fprev;
                    if constexpr (SYS != REACH_KS)
                        fprev = IN ? tr_flux_interior<double>(q, e[0], e[1])
                                   : tr_flux<double>(q, e[0], e[1], g0 - 1, n, d);
#pragma unroll
                    for (int r = 0; r < KC + R; ++r) {
                        if (r < KC) {
                            double kr;
                            if constexpr (SYS == REACH_KS) {
                                const double um2 = e[r], um1 = e[r + 1], u = e[r + 2], up1 = e[r + 3], up2 = e[r + 4];
                                kr = fma(u, fma(-q[3], fadd(up1, -um1, one), q[0]),
                                         fma(q[1], fadd(um1, up1, one), fmul(q[2], fadd(um2, up2, one), nz)));
                            } else {
                                const double fout = IN ? tr_flux_interior<double>(q, e[r + 1], e[r + 2])
                                                       : tr_flux<double>(q, e[r + 1], e[r + 2], g0 + r, n, d);
                                kr = fadd(-fout, fprev, one);
                                fprev = fout;
                            }
                            kring[r % (R + 1)] = kr;
                        }
                        if (r >= R) {
                            const int u = r - R;
                            const double k = kring[u % (R + 1)];
                            if (stage == 0) { acc[u] = k; e[R + u] = fma(hh, k, z[u]); }
                            if (stage == 1) { acc[u] = fma(2.0, k, acc[u]); e[R + u] = fma(hh, k, z[u]); }
                            if (stage == 2) { acc[u] = fma(2.0, k, acc[u]); e[R + u] = fma(h, k, z[u]); }
                            if (stage == 3) { acc[u] = fadd(k, acc[u], one); z[u] = fma(h6, acc[u], z[u]); e[R + u] = z[u]; }
                        }
                    }
                }
            }
        };
        if (interior) steps(std::true_type{});
        else steps(std::false_type{});
        double *out = static_cast<double *>(a.out);
        if (whole && g0 >= own0 && g0 + KC <= own0 + a.W) {
            double2 *dst = reinterpret_cast<double2 *>(out + base + g0);
#pragma unroll
            for (int r = 0; r < KC / 2; ++r) __stcs(dst + r, make_double2(z[2 * r], z[2 * r + 1]));
        } else {
#pragma unroll
            for (int r = 0; r < KC; ++r) {
                const int64_t g = g0 + r;
                if (g >= own0 && g < own0 + a.W && g >= 0 && g < n) __stcs(out + base + g, z[r]);
            }
        }
    }
    if (flags) atomicOr(a.status, flags);
}

// per-row minimum and maximum over the samples of the binary64 row state
// (integer-key minima, as mc_stream's warp reduction takes them)
__global__ void mc_rows64_reduce(const double *x, int64_t ns, int64_t n, int64_t m, double *lo, double *hi,
                                 int *status) {
    int flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double a = INFINITY, b = -INFINITY;
        bool bad = false;
        for (int64_t j = 0; j < m; ++j) {
            const double v = __ldcs(x + (int64_t)((uint64_t)j * (uint64_t)ns) + i);
            a = kmin(a, v);
            b = kmax(b, v);
            bad |= !kfinite(v);
        }
        lo[i] = a;
        hi[i] = b;
        if (bad) flags |= ST_NONFINITE;
    }
    if (flags) atomicOr(status, flags);
}

// ------------------------------------------------------------------ reduce
__global__ void mc_reduce(const double *plo, const double *phi, int64_t nblk, int64_t n, double *lo,
                          double *hi) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double a = INFINITY, b = -INFINITY;
        for (int64_t k = 0; k < nblk; ++k) {
            a = fmin(a, plo[k * n + i]);
            b = fmax(b, phi[k * n + i]);
        }
        lo[i] = a;
        hi[i] = b;
    }
}

// ------------------------------------------------------------------ quadrotor swarm
// fused multiply-add in the kernel's precision
__device__ __forceinline__ float qfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double qfma(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ float qabs(float a) { return fabsf(a); }
__device__ __forceinline__ double qabs(double a) { return fabs(a); }

// sin d and cos d for any d by argument halving (scaling and squaring): d is
// halved k times into the range of the Maclaurin series, and the series'
// values are doubled back k times by the double-angle formulas, each of
// which about doubles the rounding error (k <= 3 for |d| <= 1/2); at most 40
// halvings, so that an infinite d ends as a non-finite result
template <class T>
__device__ __forceinline__ void halved_sincos(T d, T &s, T &c) {
    int k = 0;
    while (qabs(d) > T(Q_SMALL) && k < 40) {
        d = d * T(0.5);
        ++k;
    }
    small_sincos(d, s, c);
    for (int i = 0; i < k; ++i) {
        const T t = s + s;
        const T c2 = qfma(-t, s, T(1));
        s = t * c;
        c = c2;
    }
}

// The four stages of one RK4 step of a sample's chain, their accelerations
// summed into m.  (s0, c0): the sines and cosines of the step-start angles,
// replaced by those of the last stage, the next step's start.  The stages'
// sines and cosines follow by angle addition over the stage increments d_1 =
// (h/2) w and d_2 = (h/2) X, and d_3 = h X = 2 d_2 exactly (h = 2 (h/2)), so
// the last stage takes the double-angle formulas of d_2's sine and cosine.
// The increments' sines and cosines come from the Maclaurin series, or with
// FAR (an increment may pass Q_SMALL) from halved_sincos.  Neither copy calls
// sincos: with the calls in the loop, the compiler computed part of them at
// every stage (their conversions kept the FP64 pipe 87% busy: 44.1 against
// 37.2 ms for 10^6 agents x 32 samples x 200 steps).
template <class T, bool FAR>
__device__ __forceinline__ void quad_mc_stages(const QChain<T> &c, T h, T fa, T fg, T (&s0)[3], T (&c0)[3],
                                               QSums<T> &m) {
    T sd2[3], cd2[3];   // sine and cosine of d_2, for the last stage
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        T dq[3], sn[3], cs[3], acc[3];
        stage_deltas(c, st, h, dq);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (st == 0) {
                sn[d] = s0[d];
                cs[d] = c0[d];
                continue;
            }
            T sd, cd;
            if (st == 3) {
                const T t = sd2[d] + sd2[d];
                sd = t * cd2[d];
                cd = qfma(-t, sd2[d], T(1));
            } else {
                if (FAR) halved_sincos(dq[d], sd, cd);
                else small_sincos(dq[d], sd, cd);
                if (st == 2) {
                    sd2[d] = sd;
                    cd2[d] = cd;
                }
            }
            sn[d] = qfma(s0[d], cd, c0[d] * sd);
            cs[d] = qfma(c0[d], cd, -(s0[d] * sd));
            if (st == 3) {
                s0[d] = sn[d];
                c0[d] = cs[d];
            }
        }
        quad_acc_trig<T>(sn, cs, fa, fg, acc);
        add_stage(m, acc, st);
    }
}

// Lane = sample of one agent: a warp integrates 32 samples of agent k (blockIdx.x
// * 4 + warp) over the whole horizon in registers (the agents are independent)
// and reduces each of its 12 components over the samples; blockIdx.y is the
// 32-sample chunk, so the partials have the [chunk][n] layout of mc_reduce.
template <class T>
__global__ void __launch_bounds__(128) mc_quad(McArgs a, QuadK p) {
    const int lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (k >= a.n / 12) return;   // whole warps leave together
    const int64_t j = (int64_t)blockIdx.y * 32 + lane;
    const bool valid = j < a.m;
    const double J[3] = {p.Jx, p.Jy, p.Jz};
    QChain<T> c;
    int flags = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int64_t i = 12 * k + 3 * r + d;
            const double lo = a.xlo[i], hi = a.xhi[i];
            if (!(kle(lo, hi) && kfinite(lo) && kfinite(hi))) flags |= ST_BADINPUT;
            const T v = as_run<T>(box_sample(lo, hi, philox_uniform(a.seed, (uint32_t)j, (uint32_t)i, 0u)));
            if (r == 0) c.p[d] = v;
            else if (r == 1) c.v[d] = v;
            else if (r == 2) c.q[d] = v;
            else c.w[d] = v;
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int64_t i = 3 * k + d;
        const double lo = a.wlo[i], hi = a.whi[i];
        if (!(kle(lo, hi) && kfinite(lo) && kfinite(hi))) flags |= ST_BADINPUT;
        const T tau = as_run<T>(box_sample(lo, hi, philox_uniform(a.seed, (uint32_t)j, (uint32_t)i, 1u)));
        c.al[d] = tau / (T)J[d];
    }
    const T h = (T)a.h, fa = (T)p.a, fg = (T)p.g;
    // Sines and cosines at the step start: taken afresh every QUAD_ANCHOR
    // steps, and in between the previous step's last-stage values, those of
    // q + d_3, which is the new step-start angle up to the rounding of the
    // state update (quad_mc_stages).  A step whose stage increments d_1 or d_2
    // pass Q_SMALL takes the copy of the stages that halves them into the
    // series' range.
    T s0[3], c0[3];
    for (int64_t s = 0; s < a.N; ++s) {
        if (s % QUAD_ANCHOR == 0) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if constexpr (sizeof(T) == 4) sincosf(c.q[d], &s0[d], &c0[d]);
                else sincos(c.q[d], &s0[d], &c0[d]);
            }
        }
        T d1[3], d2[3];
        stage_deltas(c, 1, h, d1);
        stage_deltas(c, 2, h, d2);
        bool far = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) far = far || qabs(d1[d]) > T(Q_SMALL) || qabs(d2[d]) > T(Q_SMALL);
        QSums<T> m;
        if (far) quad_mc_stages<T, true>(c, h, fa, fg, s0, c0, m);
        else quad_mc_stages<T, false>(c, h, fa, fg, s0, c0, m);
        chain_update(c, m, h);
    }
    double *plo = a.plo + (int64_t)blockIdx.y * a.n + 12 * k, *phi = a.phi + (int64_t)blockIdx.y * a.n + 12 * k;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        warp_minmax<T>(c.p[d], valid, plo + d, phi + d, a.status);
        warp_minmax<T>(c.v[d], valid, plo + 3 + d, phi + 3 + d, a.status);
        warp_minmax<T>(c.q[d], valid, plo + 6 + d, phi + 6 + d, a.status);
        warp_minmax<T>(c.w[d], valid, plo + 9 + d, phi + 9 + d, a.status);
    }
    if (flags && lane == 0) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ host
// Samples per block of the on-chip kernel: blocks of 32 samples while there
// are enough of them for every SM, else 8 or 2, which spreads the same warps
// over more SMs (a few warps per SM instead of sixteen on a few SMs).
int mc_onchip_sb(int64_t m) {
    if (opt_mc_sb() > 0) return (int)opt_mc_sb();
    if ((m + 31) / 32 >= 148) return 32;
    if ((m + 7) / 8 >= 148) return 8;
    return 2;
}

template <int SYS, class T, int SB>
static int launch_onchip_sb(const McArgs &a, cudaStream_t st) {
    const int64_t nblk = (a.m + SB - 1) / SB;
    // row groups: 16 with 32 samples (16 warps); otherwise one row per thread
    // up to MC_THREADS threads, the count a multiple of 32 / SB so that whole
    // warps launch
    int64_t G = 16;
    if (SB < 32) {
        const int64_t unit = 32 / SB;
        G = (a.n + unit - 1) / unit * unit;
        if (G > MC_THREADS / SB) G = MC_THREADS / SB;
    }
    const int64_t rows = (a.n + G - 1) / G;
    if (rows > MC_Q) return REACH_EINVAL;   // more rows than a thread holds
    const size_t smem = (size_t)(a.n + a.nw) * SB * sizeof(T);
    // one row per thread runs a one-row loop: the eight-row one keeps the
    // absent rows' code in the stage loop
    static std::atomic<bool> attr1{false}, attr8{false};   // idempotent: a second setter is harmless
    if (rows == 1) {
        if (!attr1.load()) {
            int rc = allow_max_dynamic_smem((const void *)mc_onchip<SYS, T, SB, 1>);
            if (rc) return rc;
            attr1.store(true);
        }
        mc_onchip<SYS, T, SB, 1><<<(unsigned)nblk, (unsigned)(SB * G), smem, st>>>(a);
    } else {
        if (!attr8.load()) {
            int rc = allow_max_dynamic_smem((const void *)mc_onchip<SYS, T, SB, MC_Q>);
            if (rc) return rc;
            attr8.store(true);
        }
        mc_onchip<SYS, T, SB, MC_Q><<<(unsigned)nblk, (unsigned)(SB * G), smem, st>>>(a);
    }
    REACH_LAUNCHED("mc_onchip");
    return REACH_OK;
}

template <int SYS, class T>
static int launch_onchip(const McArgs &a, int sb, cudaStream_t st) {
    if (sb == 2) return launch_onchip_sb<SYS, T, 2>(a, st);
    if (sb == 8) return launch_onchip_sb<SYS, T, 8>(a, st);
    return launch_onchip_sb<SYS, T, 32>(a, st);
}

// warps per block of the streaming kernel: binary64 keeps 2x the registers
template <class T>
constexpr int mc_wpb() { return sizeof(T) == 4 ? 16 : 8; }

template <int SYS, class T, int WPB = mc_wpb<T>(), int MINB = 2>
static int launch_stream_v(McStep a, const double *prm, int64_t N, void *bufA, void *bufB, cudaStream_t st) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    // binary32 samples: two steps per launch halve the state traffic for a
    // 4R-row halo (measured +27% on the KS grid); binary64 is FP64-pipe bound
    int S = opt_steps() > 0 ? (int)opt_steps() : (sizeof(T) == 4 ? 2 : 1);
    while (S > 1 && 2 * 4 * R * S >= WPB * MC_B / 2) --S;   // keep the halo below half the block
    const int64_t L = N > 0 ? (N + S - 1) / S : 1;
    void *buf[2] = {bufA, bufB};
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        const int s = N > 0 ? (int)std::min<int64_t>(S, N - done) : 0;
        a.S = s;
        a.H = 4 * R * s;
        a.TC = WPB * MC_B - 2 * a.H;
        a.first = (q == 0);
        a.last = (q == L - 1);
        a.in = buf[q % 2];
        a.out = buf[(q + 1) % 2];
        const int64_t ntile = (a.n + a.TC - 1) / a.TC;
        const int64_t grid = ntile * (a.M / 32);
        if (grid > 0x7fffffffLL) return REACH_EINVAL;
        a.ntile = (unsigned)ntile;
        mc_stream<SYS, T, WPB, MINB><<<(unsigned)grid, 32 * WPB, 0, st>>>(a, prm);
        REACH_LAUNCHED("mc_stream");
        done += s;
    }
    return REACH_OK;
}

template <int SYS, class T>
static int launch_stream(McStep a, const double *prm, int64_t N, void *bufA, void *bufB, cudaStream_t st) {
    // binary64 in sample-row blocks (the row layout of mc_rows64 is the
    // default): one 16-warp block per SM halves the 16-row halo share of two
    // 8-warp blocks on KS grids (1024 samples of 2^20 points: 0.77 against
    // 0.74 of the FP64 peak); the traffic chain's one-row halo gains nothing
    // (2.26e10 against 2.33e10 comp-steps/s).  REACH_OPT_MC_LAYOUT 7 forces
    // the 16-warp block, 1..6 the 8-warp blocks.
    const int64_t lay = opt_mc_layout();
    if (sizeof(T) == 8 && lay == 7)
        return launch_stream_v<SYS, T, 16, 1>(a, prm, N, bufA, bufB, st);
    return launch_stream_v<SYS, T>(a, prm, N, bufA, bufB, st);
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link to
// the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static std::atomic<EncodeTiledFn> fn{nullptr};
    EncodeTiledFn f = fn.load();
    if (!f) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        f = (EncodeTiledFn)p;
        fn.store(f);
    }
    return f;
}

// the n x M binary32 state buffers as 2-D tensors (M samples per row, the
// inner dimension), boxes of `rows` rows x 64 samples
static int state_maps(const McStep &a, void *bufA, void *bufB, int rows, CUtensorMap (&maps)[2]) {
    EncodeTiledFn f = encode_tiled();
    if (!f) return REACH_ECUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)a.M, (cuuint64_t)a.n};
    const cuuint64_t strides[1] = {(cuuint64_t)a.M * sizeof(float)};
    const cuuint32_t box[2] = {64, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    void *bufs[2] = {bufA, bufB};
    for (int i = 0; i < 2; ++i)
        if (f(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, bufs[i], dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return REACH_ECUDA;
    return REACH_OK;
}

// binary32 streaming with two samples per lane: a block of WPB warps x B rows
// x 64 samples, at least MINB blocks per SM
template <int SYS, int WPB, int B, int MINB, bool PREFETCH = false>
static int launch_stream2_v(McStep a, int64_t N, void *bufA, void *bufB, int S_auto, cudaStream_t st) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    int S = opt_steps() > 0 ? (int)opt_steps() : S_auto;
    while (S > 1 && 2 * 4 * R * S >= WPB * B / 2) --S;   // keep the halo below half the block
    const int64_t L = N > 0 ? (N + S - 1) / S : 1;
    void *buf[2] = {bufA, bufB};
    // tensor maps of the two state buffers (rows of M binary32 samples), for
    // the launches that copy their tiles ahead
    CUtensorMap maps[2];
    bool maps_ok = false;
    if constexpr (PREFETCH) {
        if (L > 1 && bufA && bufB) maps_ok = state_maps(a, bufA, bufB, WPB * B, maps) == REACH_OK;
    }
    (void)maps_ok;
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        const int s = N > 0 ? (int)std::min<int64_t>(S, N - done) : 0;
        a.S = s;
        a.H = 4 * R * s;
        a.TC = WPB * B - 2 * a.H;
        a.first = (q == 0);
        a.last = (q == L - 1);
        a.in = buf[q % 2];
        a.out = buf[(q + 1) % 2];
        const int64_t ntile = (a.n + a.TC - 1) / a.TC;
        const int64_t grid = ntile * (a.M / 64);
        if (grid > 0x7fffffffLL) return REACH_EINVAL;
        a.ntile = (unsigned)ntile;
        bool prefetched = false;
        if constexpr (PREFETCH) {
          if (q > 0 && maps_ok) {
            // persistent blocks, one per SM, the next tiles' rows copied ahead
            static std::atomic<bool> attr_set{false};   // idempotent: a second setter is harmless
            if (!attr_set.load()) {
                int rc = allow_max_dynamic_smem((const void *)mc_stream2p<SYS, WPB, B>);
                if (rc) return rc;
                attr_set.store(true);
            }
            int dev = 0, sms = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const unsigned pgrid = (unsigned)std::min<int64_t>(grid, sms);
            const size_t smem = (size_t)2 * WPB * B * 32 * sizeof(float2);
            mc_stream2p<SYS, WPB, B><<<pgrid, 32 * WPB, smem, st>>>(a, (unsigned long long)grid, maps[q % 2]);
            REACH_LAUNCHED("mc_stream2p");
            prefetched = true;
          }
        }
        if (!prefetched) {
            mc_stream2<SYS, WPB, B, MINB><<<(unsigned)grid, 32 * WPB, 0, st>>>(a);
            REACH_LAUNCHED("mc_stream2");
        }
        done += s;
    }
    return REACH_OK;
}

// binary32 streaming on the pair-row layout: persistent mc_rows warps, KC
// rows per lane, S steps per launch, then the per-row reduction of the final
// state into (lo, hi)
template <int SYS, int KC>
static int launch_rows(RowStep a, int64_t N, float2 *bufA, float2 *bufB, double *lo, double *hi, cudaStream_t st) {
    REACH_CUDA(cudaMemsetAsync(a.ctr, 0, 2 * sizeof(unsigned), st));
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    int S = opt_steps() > 0 ? (int)opt_steps() : 3;
    while (S > 1 && 2 * 4 * R * S >= 32 * KC / 2) --S;   // keep the halo below half the warp tile
    const int64_t L = N > 0 ? (N + S - 1) / S : 1;
    float2 *buf[2] = {bufA, bufB};
    int dev = 0, sms = 148, per_sm = 2;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    constexpr size_t smem = rows_stage_bytes<SYS, KC>();
    REACH_CUDA(cudaFuncSetAttribute(mc_rows<SYS, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    REACH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mc_rows<SYS, KC>, 256, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        const int s = N > 0 ? (int)std::min<int64_t>(S, N - done) : 0;
        a.S = s;
        a.H = 4 * R * s;
        a.W = 32 * KC - 2 * a.H;
        a.first = (q == 0);
        a.in = buf[q % 2];
        a.out = buf[(q + 1) % 2];
        a.slot = (int)(q % 2);
        const int64_t ntile = (a.n + a.W - 1) / a.W;
        const int64_t items = ntile * (int64_t)a.P;
        const int64_t blocks = std::min<int64_t>((items + 7) / 8, (int64_t)sms * per_sm);
        if (items + 16 * blocks >= (1LL << 32)) return REACH_EINVAL;   // the 32-bit item counter
        a.ntile = (unsigned)ntile;
        mc_rows<SYS, KC><<<(unsigned)blocks, 256, smem, st>>>(a);
        REACH_LAUNCHED("mc_rows");
        done += s;
    }
    int64_t g = (a.n + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    mc_rows_reduce<<<(unsigned)g, 256, 0, st>>>(buf[L % 2], a.ns, a.n, a.P, a.m, lo, hi, a.status);
    REACH_LAUNCHED("mc_rows_reduce");
    return REACH_OK;
}

// binary64 streaming on the row layout: persistent mc_rows64 warps, KC rows
// per lane, S steps per launch (default 1: the kernel is bound by the FP64
// pipe), then the per-row reduction of the final state into (lo, hi)
template <int SYS, int KC, int MINB>
static int launch_rows64(RowStep a, const double *prm, int64_t N, double *bufA, double *bufB, double *lo,
                         double *hi, cudaStream_t st) {
    constexpr int R = (SYS == REACH_KS) ? 2 : 1;
    int S = opt_steps() > 0 ? (int)opt_steps() : 1;
    while (S > 1 && 2 * 4 * R * S >= 32 * KC / 2) --S;
    const int64_t L = N > 0 ? (N + S - 1) / S : 1;
    double *buf[2] = {bufA, bufB};
    int dev = 0, sms = 148, per_sm = MINB;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    REACH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mc_rows64<SYS, KC, MINB>, 256, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        const int s = N > 0 ? (int)std::min<int64_t>(S, N - done) : 0;
        a.S = s;
        a.H = 4 * R * s;
        a.W = 32 * KC - 2 * a.H;
        a.first = (q == 0);
        a.in = buf[q % 2];
        a.out = buf[(q + 1) % 2];
        const int64_t ntile = (a.n + a.W - 1) / a.W;
        if (ntile * (int64_t)a.P >= (1LL << 32)) return REACH_EINVAL;
        a.ntile = (unsigned)ntile;
        const int64_t items = ntile * (int64_t)a.P;
        const int64_t blocks = std::min<int64_t>((items + 7) / 8, (int64_t)sms * per_sm);
        mc_rows64<SYS, KC, MINB><<<(unsigned)blocks, 256, 0, st>>>(a, prm);
        REACH_LAUNCHED("mc_rows64");
        done += s;
    }
    int64_t g = (a.n + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    mc_rows64_reduce<<<(unsigned)g, 256, 0, st>>>(buf[L % 2], a.ns, a.n, a.m, lo, hi, a.status);
    REACH_LAUNCHED("mc_rows64_reduce");
    return REACH_OK;
}

// Block shapes of the sample-row layout (REACH_OPT_MC_LAYOUT 2..6; the
// pair-row kernel mc_rows is the default, see mc_dispatch), measured on 1024
// samples of the 2^20-point KS grid over 500 steps and 256 of the 2^20-cell
// chain over 200: the packed kernel is bound by the FP32 FMA pipe (a packed
// instruction holds it two cycles), so the shape that best hides each tile's
// load behind arithmetic wins.  KS: persistent 16-warp blocks whose next tiles
// arrive by tensor copies (layout 6) at three steps per launch, 0.87 s; the
// same shape loading at block start 0.96 s, two 8-warp blocks per SM 1.02 s
// (two steps), the one-sample kernel 1.05 s at its best.  Traffic: two 8-warp
// blocks per SM at three steps, 0.077 s (0.081 s prefetched, 0.098 s for the
// one-sample kernel).
template <int SYS>
static int launch_stream2(const McStep &a, int64_t N, void *bufA, void *bufB, cudaStream_t st) {
    int layout = (int)opt_mc_layout();
    const int S_auto = 3;
    switch (layout) {
    case 3: return launch_stream2_v<SYS, 32, 8, 1>(a, N, bufA, bufB, S_auto, st);
    case 4: return launch_stream2_v<SYS, 8, 16, 2>(a, N, bufA, bufB, S_auto, st);
    case 5: return launch_stream2_v<SYS, 16, 8, 2>(a, N, bufA, bufB, S_auto, st);
    case 6: return launch_stream2_v<SYS, 16, 16, 1, true>(a, N, bufA, bufB, S_auto, st);
    default: return launch_stream2_v<SYS, 16, 16, 1>(a, N, bufA, bufB, S_auto, st);
    }
}

int64_t mc_onchip_limit(int kind, int prec) {
    // rows per thread x warps, and shared memory for [n + nw][32]
    int64_t by_regs = (int64_t)MC_Q * MC_WARPS;
    int64_t elt = prec == 32 ? 4 : 8;
    int64_t smem = onchip_max_smem();
    int64_t by_smem = smem / (32 * elt);   // n + nw rows
    if (kind == REACH_OSC) by_smem = by_smem * 2 / 3;        // nw = n / 2
    if (kind == REACH_LINEAR || kind == REACH_TRAFFIC) by_smem = by_smem - 1;
    if (kind == REACH_LINEAR) by_smem /= 2;
    return by_regs < by_smem ? by_regs : by_smem;
}

}  // namespace reach

using namespace reach;

template <class T>
static int mc_dispatch(const reach_system *sys, Staging &sg, const McArgs &base, double *dlo, double *dhi,
                       double wl, double wh) {
    const int64_t n = sys->n;
    int rc;
    if (sys->kind == REACH_QUAD) {
        const int64_t nblk = (base.m + 31) / 32;
        if (nblk > 65535) return REACH_EINVAL;   // chunks run along the grid's y dimension
        McArgs a = base;
        if ((rc = sg.scratch(2 * nblk * n * sizeof(double), (void **)&a.plo))) return rc;
        a.phi = a.plo + nblk * n;
        QuadK p;
        p.a = sys->prm[0]; p.g = sys->prm[1]; p.Jx = sys->prm[2]; p.Jy = sys->prm[3]; p.Jz = sys->prm[4];
        const dim3 grid((unsigned)((n / 12 + 3) / 4), (unsigned)nblk);
        mc_quad<T><<<grid, 128, 0, sg.st>>>(a, p);
        REACH_LAUNCHED("mc_quad");
        int64_t g = (n + 255) / 256;
        if (g > 148 * 16) g = 148 * 16;
        mc_reduce<<<(unsigned)g, 256, 0, sg.st>>>(a.plo, a.phi, nblk, n, dlo, dhi);
        REACH_LAUNCHED("mc_reduce");
        return REACH_OK;
    }
    bool onchip = n <= mc_onchip_limit(sys->kind, sizeof(T) == 4 ? 32 : 64);
    if (opt_kernel() == 1 && (sys->kind == REACH_TRAFFIC || sys->kind == REACH_KS) && n >= 16) onchip = false;
    if (!onchip && !(sys->kind == REACH_TRAFFIC || sys->kind == REACH_KS)) return REACH_EINVAL;
    // binary32 samples on the streaming kernel go two per lane
    const bool pairs = !onchip && sizeof(T) == 4 && opt_mc_layout() != 1;
    const int64_t lay = opt_mc_layout();
    if (!onchip && sizeof(T) == 8 && (lay == 0 || lay >= 8)) {
        // binary64 on the row layout (mc_rows64, the default: 16 rows per lane
        // in one 8-warp block per SM at 190 registers; the option picks 8 or
        // 12 in two blocks per SM).  64 samples of the 2^20-point KS grid over
        // 100 steps: 0.419 s against 0.515 s for one 16-warp block per SM of
        // sample rows with a barrier per stage (0.93 against 0.77 of the FP64
        // peak), 0.431 s with 8 rows per lane; the 2^20-cell chain over 200
        // steps: 0.513 s against 0.573 s.
        if (n > INT32_MAX - 64) return REACH_EINVAL;
        RowStep r;
        memset(&r, 0, sizeof r);
        r.n = n;
        r.ns = (n + 1) & ~(int64_t)1;
        r.m = base.m;
        r.P = (unsigned)base.m;
        r.h = base.h;
        r.h6 = base.h / 6.0;
        r.one = 1.0;
        r.nzero = -0.0;
        r.seed = base.seed;
        r.xlo = base.xlo;
        r.xhi = base.xhi;
        r.dlo = wl;
        r.dhi = wh;
        r.status = base.status;
        double *bufA, *bufB;
        const size_t bytes = (size_t)r.ns * r.P * sizeof(double);
        if ((rc = sg.scratch(bytes, (void **)&bufA)) || (rc = sg.scratch(bytes, (void **)&bufB))) return rc;
        if (sys->kind == REACH_TRAFFIC) {
            if (lay == 8) return launch_rows64<REACH_TRAFFIC, 8, 2>(r, base.prm, base.N, bufA, bufB, dlo, dhi, sg.st);
            if (lay == 9) return launch_rows64<REACH_TRAFFIC, 12, 2>(r, base.prm, base.N, bufA, bufB, dlo, dhi, sg.st);
            return launch_rows64<REACH_TRAFFIC, 16, 1>(r, base.prm, base.N, bufA, bufB, dlo, dhi, sg.st);
        }
        if (lay == 8) return launch_rows64<REACH_KS, 8, 2>(r, base.prm, base.N, bufA, bufB, dlo, dhi, sg.st);
        if (lay == 9) return launch_rows64<REACH_KS, 12, 2>(r, base.prm, base.N, bufA, bufB, dlo, dhi, sg.st);
        return launch_rows64<REACH_KS, 16, 1>(r, base.prm, base.N, bufA, bufB, dlo, dhi, sg.st);
    }
    if (pairs && (lay == 0 || lay >= 8)) {
        // pair-row layout (mc_rows, the default): no per-block partials, the
        // reduction reads the final state.  1024 samples of the 2^20-point KS
        // grid over 500 steps: 0.689 s against 0.870 s for the best block
        // layout (6), 0.789 s with 8 rows per lane (halo 19% of the warp
        // tile), 0.699 s with 12, 0.720 s with 16; 256 samples of the 2^20-cell chain over 200 steps: 0.060 s
        // against 0.076 s (layout 4).  An L2 prefetch of each warp's next
        // item gained nothing on the KS grid (2% traffic).
        if (n > INT32_MAX - 64) return REACH_EINVAL;
        RowStep r;
        memset(&r, 0, sizeof r);
        r.n = n;
        r.ns = (n + 1) & ~(int64_t)1;
        r.m = base.m;
        r.P = (unsigned)((base.m + 1) / 2);
        r.hf[0] = (float)base.h;
        r.hf[1] = (float)(0.5 * base.h);
        r.hf[2] = (float)(base.h / 6.0);
        const double *pr = sys->prm;   // mc_stream2's binary32 constants
        const bool tr = sys->kind == REACH_TRAFFIC;
        r.qf[0] = (float)pr[0];
        r.qf[1] = (float)pr[1];
        r.qf[2] = (float)pr[2];
        r.qf[3] = tr ? (float)(pr[2] * pr[3]) : (float)pr[3];
        r.seed = base.seed;
        r.xlo = base.xlo;
        r.xhi = base.xhi;
        r.dlo = wl;
        r.dhi = wh;
        r.status = base.status;
        float2 *bufA, *bufB;
        const size_t bytes = (size_t)r.ns * r.P * sizeof(float2);
        if ((rc = sg.scratch(bytes, (void **)&bufA)) || (rc = sg.scratch(bytes, (void **)&bufB)) ||
            (rc = sg.scratch(2 * sizeof(unsigned), (void **)&r.ctr)))
            return rc;
        // rows per lane: the option's 8 / 12 / 16, else 14 on the KS grid
        // (0.689 s against 0.699 s with 12, same box) and 12 on the chain
        // (whose 14- and 16-row variants spill)
        const bool ks = sys->kind == REACH_KS;
        const int kc = lay == 8 ? 8 : lay == 9 ? 12 : lay == 10 ? 16 : (ks ? 14 : 12);
        if (!ks) {
            if (kc == 8) return launch_rows<REACH_TRAFFIC, 8>(r, base.N, bufA, bufB, dlo, dhi, sg.st);
            if (kc == 12) return launch_rows<REACH_TRAFFIC, 12>(r, base.N, bufA, bufB, dlo, dhi, sg.st);
            return launch_rows<REACH_TRAFFIC, 16>(r, base.N, bufA, bufB, dlo, dhi, sg.st);
        }
        if (kc == 8) return launch_rows<REACH_KS, 8>(r, base.N, bufA, bufB, dlo, dhi, sg.st);
        if (kc == 12) return launch_rows<REACH_KS, 12>(r, base.N, bufA, bufB, dlo, dhi, sg.st);
        if (kc == 14) return launch_rows<REACH_KS, 14>(r, base.N, bufA, bufB, dlo, dhi, sg.st);
        return launch_rows<REACH_KS, 16>(r, base.N, bufA, bufB, dlo, dhi, sg.st);
    }
    // partial minima / maxima per block of samples
    const int sb = onchip ? mc_onchip_sb(base.m) : (pairs ? 64 : 32);
    int64_t nblk = (base.m + sb - 1) / sb;
    McArgs a = base;
    if ((rc = sg.scratch(2 * nblk * n * sizeof(double), (void **)&a.plo))) return rc;
    a.phi = a.plo + nblk * n;
    if (onchip) {
        switch (sys->kind) {
        case REACH_TRAFFIC: rc = launch_onchip<REACH_TRAFFIC, T>(a, sb, sg.st); break;
        case REACH_KS: rc = launch_onchip<REACH_KS, T>(a, sb, sg.st); break;
        case REACH_OSC: rc = launch_onchip<REACH_OSC, T>(a, sb, sg.st); break;
        case REACH_HEAT3D: rc = launch_onchip<REACH_HEAT3D, T>(a, sb, sg.st); break;
        default: rc = launch_onchip<REACH_LINEAR, T>(a, sb, sg.st); break;
        }
    } else {
        McStep s;
        memset(&s, 0, sizeof s);
        // the kernel forms row offsets by 32 x 32 -> 64-bit products
        if (n > INT32_MAX - 64 || nblk * sb > INT32_MAX) return REACH_EINVAL;
        s.n = n;
        s.m = base.m;
        s.M = nblk * sb;
        s.nM = n * s.M;
        s.h = base.h;
        s.hh = 0.5 * base.h;
        s.h6 = base.h / 6.0;
        s.hf[0] = (float)s.h;
        s.hf[1] = (float)s.hh;
        s.hf[2] = (float)s.h6;
        {
            const double *pr = sys->prm;   // mc_consts's binary32 constants, rounded here
            const bool tr = sys->kind == REACH_TRAFFIC;
            s.qf[0] = (float)pr[0];
            s.qf[1] = (float)pr[1];
            s.qf[2] = (float)pr[2];
            s.qf[3] = tr ? (float)(pr[2] * pr[3]) : (float)pr[3];
        }
        s.seed = base.seed;
        s.xlo = base.xlo;
        s.xhi = base.xhi;
        s.dlo = wl;
        s.dhi = wh;
        s.plo = a.plo;
        s.phi = a.phi;
        s.status = base.status;
        void *bufA = nullptr, *bufB = nullptr;
        if (base.N > 1) {
            if ((rc = sg.scratch((size_t)n * s.M * sizeof(T), &bufA))) return rc;
            if ((rc = sg.scratch((size_t)n * s.M * sizeof(T), &bufB))) return rc;
        }
        if (pairs) {
            if (sys->kind == REACH_TRAFFIC) rc = launch_stream2<REACH_TRAFFIC>(s, base.N, bufA, bufB, sg.st);
            else rc = launch_stream2<REACH_KS>(s, base.N, bufA, bufB, sg.st);
        } else if (sys->kind == REACH_TRAFFIC) {
            rc = launch_stream<REACH_TRAFFIC, T>(s, base.prm, base.N, bufA, bufB, sg.st);
        } else {
            rc = launch_stream<REACH_KS, T>(s, base.prm, base.N, bufA, bufB, sg.st);
        }
    }
    if (rc) return rc;
    int64_t g = (n + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    mc_reduce<<<(unsigned)g, 256, 0, sg.st>>>(a.plo, a.phi, nblk, n, dlo, dhi);
    REACH_LAUNCHED("mc_reduce");
    return REACH_OK;
}

extern "C" int reach_mc(const reach_system *sys, const double *x0_lo, const double *x0_hi, const double *w_lo,
                        const double *w_hi, double t_final, double dt, int64_t m, uint64_t seed, int precision,
                        double *lo, double *hi, void *stream) {
    if (!sys || !x0_lo || !x0_hi || !lo || !hi) return REACH_EINVAL;
    if (sys->nw > 0 && (!w_lo || !w_hi)) return REACH_EINVAL;
    if (m < 1 || m >= (1LL << 32) || (precision != 32 && precision != 64)) return REACH_EINVAL;
    int64_t N;
    int rc = nsteps(t_final, dt, &N);
    if (rc) return rc;
    // the sampling kernels check the state box on the device
    if ((rc = check_host_box(w_lo, w_hi, sys->nw))) return rc;
    const int64_t n = sys->n;
    if (n >= (1LL << 32)) return REACH_EINVAL;

    Staging sg((cudaStream_t)stream);
    const double *dxlo, *dxhi, *dwlo = nullptr, *dwhi = nullptr;
    double *dlo, *dhi;
    if ((rc = sg.in(x0_lo, n, &dxlo)) || (rc = sg.in(x0_hi, n, &dxhi)) || (rc = sg.in(w_lo, sys->nw, &dwlo)) ||
        (rc = sg.in(w_hi, sys->nw, &dwhi)) || (rc = sg.out(lo, n, &dlo)) || (rc = sg.out(hi, n, &dhi)) ||
        (rc = sg.begin_status()))
        return rc;
    double wl = 0, wh = 0;
    if (sys->kind == REACH_TRAFFIC) {
        if (is_device_ptr(w_lo)) {
            REACH_CUDA(cudaMemcpyAsync(&wl, w_lo, sizeof(double), cudaMemcpyDeviceToHost, sg.st));
            REACH_CUDA(cudaMemcpyAsync(&wh, w_hi, sizeof(double), cudaMemcpyDeviceToHost, sg.st));
            REACH_CUDA(cudaStreamSynchronize(sg.st));
        } else {
            wl = w_lo[0];
            wh = w_hi[0];
        }
        if (!(wl <= wh) || !std::isfinite(wl) || !std::isfinite(wh)) return REACH_EINVAL;
    }
    McArgs a;
    a.n = n;
    a.nw = sys->nw;
    a.m = m;
    a.N = N;
    a.h = dt;
    a.seed = seed;
    a.xlo = dxlo; a.xhi = dxhi; a.wlo = dwlo; a.whi = dwhi;
    a.prm = sys->dprm;
    a.status = sg.status;
    a.plo = a.phi = nullptr;
    rc = (precision == 64) ? mc_dispatch<double>(sys, sg, a, dlo, dhi, wl, wh)
                           : mc_dispatch<float>(sys, sg, a, dlo, dhi, wl, wh);
    if (rc) return rc;
    return sg.finish();
}
