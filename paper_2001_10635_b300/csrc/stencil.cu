// stencil.cu -- streaming RK4 kernels for large stencil systems (traffic
// chain, periodic KS grid), mixed monotonicity and growth bound.
//
// Algorithm 1 of the paper runs the four RK4 stages as four parallel sections
// with a synchronisation (a kernel launch) between them and k0..k3, tmp in
// global memory.  Here one launch performs S whole RK4 steps: a warp owns a
// tile of 32*KC consecutive cells in registers, neighbour values cross lanes
// by warp shuffles, and the stencil halo of 4*R*S cells per side is
// recomputed instead of synchronised.  The state is read once and written
// once per launch (16 B per component-step at S = 1).
//
// These kernels are bound by the FP64 pipe (two operations per SM per clock
// on this GPU), so they spend it on arithmetic only: minima, maxima and
// comparisons of doubles go through integer keys (common.cuh), the four
// stages are unrolled so that no update form is selected at run time, and
// input terms enter through fused multiply-adds.
//
// State halves: MM  A = x (lower), B = xh (upper)        (Sec. 2.1, Alg. 3)
//               CGB A = c (center), B = r (half-width)    (Sec. 2.1, Alg. 2)
// The traffic halves are independent (the chain is cooperative, so MM's two
// halves are two trajectories; its contraction matrix is constant, so the
// radius does not depend on the center): each traffic warp owns one half,
// which halves its registers.  The KS halves are coupled and stay together.
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "api_internal.cuh"

namespace reach {

// cells per lane: a warp tile is 32 * KC cells.  Wide tiles (256 cells) keep
// the recomputed halo small; narrow ones (64 cells) give four times as many
// warps to grids too short to fill the GPU with wide ones.
constexpr int KC_WIDE = 8;
constexpr int KC_NARROW = 2;
constexpr int WARPS_PER_BLOCK = 8;
// The KS kernel holds both halves per warp: three 4-warp blocks per SM give it
// 168 registers (a few spilled) where two 8-warp blocks give 128 (more spilled);
// measured 1% faster (MM 1.263e10 against 1.248e10 comp-steps/s at n = 2^20).
constexpr int KS_WARPS_PER_BLOCK = 4;

struct StepArgs {
    const double *inA, *inB;   // state, or the input box on the first launch
    double *outA, *outB;
    int64_t n;
    int64_t W;                 // owned cells per tile = 32 KC - 2H
    int64_t ntiles;            // ceil(n / W), computed on the host
    int64_t tile0, tcount;     // the tiles this launch covers (traffic: a range, for overlapped copies)
    int H;                     // halo cells per side = 4 R S
    int S;                     // RK4 steps in this launch
    double h, hh, h6;          // h, h / 2 and h / 6, formed on the host (no FP64 division in the kernel)
    double one = 1.0, nzero = -0.0;   // read at run time (fadd / fmul in common.cuh); set again after a memset
    int first, last;           // convert the input box / emit the output box
    int vec;                   // every state pointer is 16-byte aligned: runs move as double2
    int *status;
};

// ------------------------------------------------------------------ helpers
// A lane's KC consecutive cells start at an even cell (tile starts and halos
// are even), so with 16-byte aligned arrays a run that lies inside [0, n)
// moves as KC/2 double2 loads or stores.
// COH: the data was written by other warps of the same launch, so it is read
// through L2 (the read-only path may hold a stale line)
template <int KC, bool COH = false>
__device__ __forceinline__ void load_run(const double *src, int64_t g0, int64_t n, bool vec, double (&v)[KC]) {
    if (vec && g0 >= 0 && g0 + KC <= n) {
        const double2 *p = reinterpret_cast<const double2 *>(src + g0);
#pragma unroll
        for (int j = 0; j < KC / 2; ++j) {
            const double2 t = COH ? __ldcg(p + j) : __ldg(p + j);
            v[2 * j] = t.x;
            v[2 * j + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            v[j] = (g >= 0 && g < n) ? (COH ? __ldcg(src + g) : __ldg(src + g)) : 0.0;
        }
    }
}
template <int R, int KC>
__device__ __forceinline__ void exchange(const double (&y)[KC], double (&e)[KC + 2 * R]) {
    // e[R + j] = y[j];  e[0..R-1] from lane-1, e[R+KC..] from lane+1
#pragma unroll
    for (int j = 0; j < KC; ++j) e[R + j] = y[j];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        e[q] = __shfl_up_sync(0xffffffffu, y[KC - R + q], 1);
        e[R + KC + q] = __shfl_down_sync(0xffffffffu, y[q], 1);
    }
}

// one RK4 stage update of a lane's cells (stage is a compile-time constant)
template <int STAGE, int KC>
__device__ __forceinline__ void rk4_update(double (&z)[KC], double (&y)[KC], double (&acc)[KC],
                                           const double (&k)[KC], const StepArgs &a) {
    const double h = a.h, hh = a.hh, h6 = a.h6;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        if (STAGE == 0) { acc[j] = k[j]; y[j] = fma(hh, k[j], z[j]); }
        if (STAGE == 1) { acc[j] = fma(2.0, k[j], acc[j]); y[j] = fma(hh, k[j], z[j]); }
        if (STAGE == 2) { acc[j] = fma(2.0, k[j], acc[j]); y[j] = fma(h, k[j], z[j]); }
        if (STAGE == 3) { acc[j] = fadd(k[j], acc[j], a.one); z[j] = fma(h6, acc[j], z[j]); y[j] = z[j]; }
    }
}

// ------------------------------------------------------------------ traffic
// k[j] = f_{g-1} - f_g: flux out of cell g is min(cap, v y_g, w (xbar - y_{g+1}))
// (min(cap, v y_g) for the last cell), the inflow of cell 0 is d, and cells
// outside [0, n) carry no flux.  IN: every flux of the tile is between two
// cells of the chain, so none of those cases arises and the tests are skipped.
template <bool POW2, int KC, bool IN = false>
__device__ __forceinline__ void traffic_rhs(const TrafficK &p, const double (&y)[KC], int64_t g0,
                                            int64_t n, double d, double (&k)[KC]) {
    double e[KC + 2];
    exchange<1>(y, e);
    double vy[KC];
    bool shifted = false;
    if (POW2) {
        // v = 2^e: free-flow flux by exponent shift on the integer pipe when
        // every lane's values allow it (a warp-uniform choice)
        bool ok = true;
#pragma unroll
        for (int j = 0; j < KC; ++j) ok = ok && scale_ok(e[1 + j], p.v_exp);
        if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
            for (int j = 0; j < KC; ++j) vy[j] = scale_pow2(e[1 + j], p.v_add);
            shifted = true;
        }
    }
    if (!shifted) {
#pragma unroll
        for (int j = 0; j < KC; ++j) vy[j] = p.v * e[1 + j];
    }
    double f[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        const int64_t g = g0 + j;
        double cong = fma(-p.w, e[2 + j], p.wxbar);
        if (!IN) cong = (g == n - 1) ? p.cap : cong;          // no congestion term at the outlet
        double fj = kmin(p.cap, kmin(vy[j], cong));
        if (!IN) {
            fj = (g == -1) ? d : fj;
            fj = (g < -1 || g >= n) ? 0.0 : fj;
        }
        f[j] = fj;
    }
    double fl = __shfl_up_sync(0xffffffffu, f[KC - 1], 1);
    if (!IN) fl = (g0 == 0) ? d : fl;
#pragma unroll
    for (int j = 0; j < KC; ++j) k[j] = fadd(-f[j], j == 0 ? fl : f[j - 1], p.one);
}

// CGB radius of the traffic chain, r' = C r + [p] with the constant C of
// reading R3 (v to the left neighbour, w to the right, the input half-width
// into cell 0): a linear system with a constant input, for which one classic
// RK4 step equals, in exact arithmetic, the nested form
//   y1 = r + (h/4) f(r), y2 = r + (h/3) f(y1), y3 = r + (h/2) f(y2), r+ = r + h f(y3)
// (both are r + h f + h^2/2 C f + h^3/6 C^2 f + h^4/24 C^3 f with f = f(r)).
// Each stage is two fused multiply-adds per cell, 8 per step against 15 for
// the stage form, and needs no accumulator.  The input enters cell 0 in the
// place of its missing left neighbour (coefficient c_s instead of c_s v).
// Cells outside the chain take part in the shuffles only: cell 0 never reads
// its left neighbour and cell n - 1 never its right one, so their values do
// not enter the chain.  IN: every cell of the tile lies in [1, n - 2].
template <int KC, bool IN>
__device__ __forceinline__ void traffic_radius_step(const TrafficK &p, double (&z)[KC], int64_t g0, int64_t n) {
    double y[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) y[j] = z[j];
#pragma unroll
    for (int stage = 0; stage < 4; ++stage) {
        double e[KC + 2];
        exchange<1>(y, e);
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            double cl = p.rv[stage], left = e[j], right = e[j + 2];
            if (!IN) {
                const int64_t g = g0 + j;
                cl = (g == 0) ? p.rc[stage] : cl;
                left = (g == 0) ? p.d_r : (g > 0 ? left : 0.0);
                right = (g < n - 1) ? right : 0.0;
            }
            y[j] = fma(cl, left, fma(p.rw[stage], right, z[j]));
        }
    }
#pragma unroll
    for (int j = 0; j < KC; ++j) z[j] = y[j];
}

// one traffic half per warp: HALF 0 = x / c, HALF 1 = xh (the CGB radius r
// takes traffic_radius_step instead)
template <int METHOD, int HALF, bool POW2, int KC, bool IN>
__device__ __forceinline__ void traffic_rhs_half(const TrafficK &p, const double (&y)[KC], int64_t g0,
                                                 int64_t n, double (&k)[KC]) {
    if (METHOD == MM) traffic_rhs<POW2, KC, IN>(p, y, g0, n, HALF ? p.d_hi : p.d_lo, k);
    else traffic_rhs<POW2, KC, IN>(p, y, g0, n, p.d_c, k);
}

template <int METHOD, int HALF, bool POW2, int KC, bool IN, bool COH = false>
__device__ __forceinline__ void traffic_tile(const StepArgs &a, const TrafficK &p, int64_t t, int lane,
                                             int &flags) {
    const int64_t n = a.n;
    const int64_t own0 = t * a.W;
    const int64_t g0 = own0 - a.H + (int64_t)lane * KC;
    double z[KC];
    if (a.first) {
        double lo[KC], hi[KC];
        load_run<KC, COH>(a.inA, g0, n, a.vec, lo);
        load_run<KC, COH>(a.inB, g0, n, a.vec, hi);
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            const bool owned = g >= own0 && g < own0 + a.W && g >= 0 && g < n;
            if (HALF == 0 && owned && !(kle(lo[j], hi[j]) && kfinite(lo[j]) && kfinite(hi[j]))) flags |= ST_BADINPUT;
            if (METHOD == MM) z[j] = HALF ? hi[j] : lo[j];
            else z[j] = HALF ? 0.5 * (hi[j] - lo[j]) : 0.5 * (lo[j] + hi[j]);
        }
    } else {
        load_run<KC, COH>(HALF ? a.inB : a.inA, g0, n, a.vec, z);
    }
    for (int s = 0; s < a.S; ++s) {
        if constexpr (METHOD == CGB && HALF == 1) {
            traffic_radius_step<KC, IN>(p, z, g0, n);
        } else {
            double y[KC], acc[KC], k[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) y[j] = z[j];
            traffic_rhs_half<METHOD, HALF, POW2, KC, IN>(p, y, g0, n, k);
            rk4_update<0>(z, y, acc, k, a);
            traffic_rhs_half<METHOD, HALF, POW2, KC, IN>(p, y, g0, n, k);
            rk4_update<1>(z, y, acc, k, a);
            traffic_rhs_half<METHOD, HALF, POW2, KC, IN>(p, y, g0, n, k);
            rk4_update<2>(z, y, acc, k, a);
            traffic_rhs_half<METHOD, HALF, POW2, KC, IN>(p, y, g0, n, k);
            rk4_update<3>(z, y, acc, k, a);
        }
    }
    double *out = HALF ? a.outB : a.outA;
    if (a.last && METHOD == MM) {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            if (g >= own0 && g < own0 + a.W && g < n && g >= 0 && !kfinite(z[j])) flags |= ST_NONFINITE;
        }
    }
    if (a.vec && g0 >= own0 && g0 + KC <= own0 + a.W && g0 + KC <= n) {
        double2 *p = reinterpret_cast<double2 *>(out + g0);
#pragma unroll
        for (int j = 0; j < KC / 2; ++j) p[j] = make_double2(z[2 * j], z[2 * j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            if (g >= own0 && g < own0 + a.W && g < n && g >= 0) out[g] = z[j];
        }
    }
}

template <int METHOD, bool POW2, int KC>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, 2) stencil_traffic_rk4(StepArgs a, TrafficK p) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t cnt = a.tcount;
    int flags = 0;
    for (int64_t t = warp; t < 2 * cnt; t += nwarps) {
        const int64_t tile = a.tile0 + (t < cnt ? t : t - cnt);
        // Inside the chain (every flux of the tile, cells own0 - H - 1 ..
        // own0 - H + 32 KC - 1, between two of its cells) the boundary tests are
        // skipped: MM 5% faster.
        const int64_t c0 = tile * a.W - a.H;
        const bool in = c0 >= 1 && c0 + 32 * KC <= a.n - 1;
        if (t < cnt) {
            if (in) traffic_tile<METHOD, 0, POW2, KC, true>(a, p, tile, lane, flags);
            else traffic_tile<METHOD, 0, POW2, KC, false>(a, p, tile, lane, flags);
        } else {
            if (in) traffic_tile<METHOD, 1, POW2, KC, true>(a, p, tile, lane, flags);
            else traffic_tile<METHOD, 1, POW2, KC, false>(a, p, tile, lane, flags);
        }
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ traffic, all steps in one launch
// The traffic chain's version of stencil_ks_flow (below): for grids of a few
// waves of warp tiles, one persistent launch runs every step, item (step,
// half, tile) starting once tiles t - 1, t, t + 1 of the same half have
// finished the previous step (the halves are independent: MM's two corner
// trajectories, CGB's center and its radius under a constant C).  Per-tile
// step counters with release / acquire ordering, state read through L2,
// bounded waits (ST_TIMEOUT); a tile's arithmetic is stencil_traffic_rk4's at
// one step per launch, so the box is the same bit for bit.
struct TrafficFlowArgs {
    StepArgs st;                   // n, W, H = 4, h, hh, h6, vec, status; ntiles
    const double *xlo, *xhi;
    double *bufA[2], *bufB[2];     // step s writes [(N - 1 - s) % 2]: [0] is the output (lo, hi)
    int64_t N;
    unsigned long long *next;      // item counter (zeroed before the launch)
    int *ready;                    // per half and tile: steps completed (zeroed before the launch)
    unsigned long long wait_ns;
};

__device__ __forceinline__ int ld_acquire_gpu_i(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu_i(int *p, int v) {
    asm volatile("st.release.gpu.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int METHOD, bool POW2, int KC>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, 2) stencil_traffic_flow(TrafficFlowArgs f, TrafficK p) {
    const int lane = threadIdx.x & 31;
    const uint32_t T = (uint32_t)f.st.ntiles, T2 = 2 * T;
    const unsigned long long total = (unsigned long long)f.N * T2;   // < 2^32 (checked on the host)
    int flags = 0;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(f.next, 1ULL);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= total) break;
        const uint32_t s = (uint32_t)i / T2, r = (uint32_t)i - s * T2;   // 32-bit division
        const uint32_t half = r >= T ? 1u : 0u, t = r - half * T;
        int *rd = f.ready + half * T;
        if (s > 0) {
            int late = 0;
            if (lane == 0) {
                const unsigned long long t0 = global_ns();
                unsigned ns = 64;
                while ((t > 0 && ld_acquire_gpu_i(rd + t - 1) < (int)s) || ld_acquire_gpu_i(rd + t) < (int)s ||
                       (t + 1 < T && ld_acquire_gpu_i(rd + t + 1) < (int)s)) {
                    if (global_ns() - t0 > f.wait_ns || (*(volatile int *)f.st.status & ST_TIMEOUT)) {
                        late = 1;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 1024) ns *= 2;
                }
            }
            if (__shfl_sync(0xffffffffu, late, 0)) {
                if (lane == 0) atomicOr(f.st.status, ST_TIMEOUT);
                return;
            }
        }
        StepArgs a = f.st;
        const int in = (int)((f.N - s) & 1), out = (int)((f.N - 1 - s) & 1);
        a.inA = s == 0 ? f.xlo : f.bufA[in];
        a.inB = s == 0 ? f.xhi : f.bufB[in];
        a.outA = f.bufA[out];
        a.outB = f.bufB[out];
        a.first = s == 0;
        a.last = (int64_t)s == f.N - 1;
        const int64_t c0 = (int64_t)t * a.W - a.H;
        const bool inner = c0 >= 1 && c0 + 32 * KC <= a.n - 1;
        if (half == 0) {
            if (inner) traffic_tile<METHOD, 0, POW2, KC, true, true>(a, p, t, lane, flags);
            else traffic_tile<METHOD, 0, POW2, KC, false, true>(a, p, t, lane, flags);
        } else {
            if (inner) traffic_tile<METHOD, 1, POW2, KC, true, true>(a, p, t, lane, flags);
            else traffic_tile<METHOD, 1, POW2, KC, false, true>(a, p, t, lane, flags);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_gpu_i(rd + t, (int)s + 1);
    }
    if (flags) atomicOr(f.st.status, flags);
}

// ------------------------------------------------------------------ traffic, box-evaluated C
// CGB radius with the contraction matrix taken over the stage box [c - r, c + r]
// (reading R14): C_{g,g-1} = v only if the free-flow branch of f_{g-1} can be
// the minimum in the box, C_{g,g+1} = w only if the congestion branch of f_g
// can, and C_gg = -v (-w) where the free-flow branch of f_g (congestion branch
// of f_{g-1}) is strictly the minimum everywhere.  The tests use the plain
// IEEE products w (xbar - x) and v x, so that they decide as a direct
// evaluation of those expressions would.
__device__ __forceinline__ bool klt(double a, double b) { return dkey(a) < dkey(b); }

template <int KC>
__device__ __forceinline__ void traffic_growth_local(const TrafficK &p, const double (&cc)[KC],
                                                     const double (&rr)[KC], int64_t g0, int64_t n,
                                                     double (&k)[KC]) {
    double C[KC + 2], Rr[KC + 2];
    exchange<1>(cc, C);
    exchange<1>(rr, Rr);
    double vlo[KC + 2], vhi[KC + 2], qlo[KC + 2], qhi[KC + 2];
#pragma unroll
    for (int m = 0; m < KC + 2; ++m) {
        const double lo = __dsub_rn(C[m], Rr[m]), hi = __dadd_rn(C[m], Rr[m]);
        vlo[m] = __dmul_rn(p.v, lo);
        vhi[m] = __dmul_rn(p.v, hi);
        qlo[m] = __dmul_rn(p.w, __dsub_rn(p.xbar, lo));   // congestion term of the cell to the left
        qhi[m] = __dmul_rn(p.w, __dsub_rn(p.xbar, hi));
    }
    // branch tests of the flux out of cell g0 - 1 + m, m = 0..KC
    bool ffp[KC + 1], ffc[KC + 1], cgp[KC + 1], cgc[KC + 1];
#pragma unroll
    for (int m = 0; m <= KC; ++m) {
        const bool last = g0 - 1 + m == n - 1;
        ffp[m] = kle(vlo[m], p.cap) && (last || kle(vlo[m], qlo[m + 1]));
        ffc[m] = klt(vhi[m], p.cap) && (last || klt(vhi[m], qhi[m + 1]));
        cgp[m] = !last && kle(qhi[m + 1], p.cap) && kle(qhi[m + 1], vhi[m]);
        cgc[m] = !last && klt(qlo[m + 1], p.cap) && klt(qlo[m + 1], vlo[m]);
    }
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        const int64_t g = g0 + j;
        const double cl = (g > 0 && ffp[j]) ? p.v : 0.0;
        const double cr = cgp[j + 1] ? p.w : 0.0;
        double cd = ffc[j + 1] ? -p.v : 0.0;
        cd = (g > 0 && cgc[j]) ? cd - p.w : cd;
        const double left = (g > 0) ? Rr[j] : 0.0;
        const double right = (g < n - 1) ? Rr[j + 2] : 0.0;
        const double add = (g == 0) ? p.d_r : 0.0;
        const double v = fma(cl, left, fma(cr, right, fma(cd, Rr[j + 1], add)));
        k[j] = (g < 0 || g >= n) ? 0.0 : v;
    }
}

// both halves per warp: the radius reads the center
template <bool POW2>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK) stencil_traffic_cgbl_rk4(StepArgs a, TrafficK p) {
    constexpr int KC = KC_WIDE;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t n = a.n;
    int flags = 0;
    for (int64_t t = warp; t < a.ntiles; t += nwarps) {
        const int64_t own0 = t * a.W;
        const int64_t g0 = own0 - a.H + (int64_t)lane * KC;
        double zc[KC], zr[KC];
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            const bool in = g >= 0 && g < n;
            double va = in ? __ldg(a.inA + g) : 0.0, vb = in ? __ldg(a.inB + g) : 0.0;
            if (a.first) {
                const bool owned = g >= own0 && g < own0 + a.W && in;
                if (owned && !(kle(va, vb) && kfinite(va) && kfinite(vb))) flags |= ST_BADINPUT;
                const double c = 0.5 * (va + vb), r = 0.5 * (vb - va);
                va = c;
                vb = r;
            }
            zc[j] = va;
            zr[j] = vb;
        }
        for (int s = 0; s < a.S; ++s) {
            double yc[KC], yr[KC], ac[KC], ar[KC], kc[KC], kr[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) { yc[j] = zc[j]; yr[j] = zr[j]; }
            traffic_rhs<POW2, KC>(p, yc, g0, n, p.d_c, kc);
            traffic_growth_local(p, yc, yr, g0, n, kr);
            rk4_update<0>(zc, yc, ac, kc, a);
            rk4_update<0>(zr, yr, ar, kr, a);
            traffic_rhs<POW2, KC>(p, yc, g0, n, p.d_c, kc);
            traffic_growth_local(p, yc, yr, g0, n, kr);
            rk4_update<1>(zc, yc, ac, kc, a);
            rk4_update<1>(zr, yr, ar, kr, a);
            traffic_rhs<POW2, KC>(p, yc, g0, n, p.d_c, kc);
            traffic_growth_local(p, yc, yr, g0, n, kr);
            rk4_update<2>(zc, yc, ac, kc, a);
            rk4_update<2>(zr, yr, ar, kr, a);
            traffic_rhs<POW2, KC>(p, yc, g0, n, p.d_c, kc);
            traffic_growth_local(p, yc, yr, g0, n, kr);
            rk4_update<3>(zc, yc, ac, kc, a);
            rk4_update<3>(zr, yr, ar, kr, a);
        }
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            if (!(g >= own0 && g < own0 + a.W && g < n && g >= 0)) continue;
            double oa = zc[j], ob = zr[j];
            if (a.last) {
                if (dkey(ob) < 0) flags |= ST_NEGRADIUS;
                const double lo = oa - ob, hi = oa + ob;
                oa = lo;
                ob = hi;
                if (!kfinite(oa) || !kfinite(ob)) flags |= ST_NONFINITE;
            }
            a.outA[g] = oa;
            a.outB[g] = ob;
        }
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ traffic, outward rounding
// Every operation rounded outward (reading R15): a warp carries one half as an
// interval [zl, zu] of binary64 numbers containing the exact-arithmetic value
// (MM halves, CGB center) or, for the CGB radius, only its upper end (all its
// terms are nonnegative).  The operations are the ones a plain evaluation
// takes, each rounded once in its direction: no product is fused into a sum,
// so that each result is the directed rounding of the exact one (a sum or a
// product alone is issued as a directed fused multiply-add with 1 or a signed
// zero, which rounds it identically: add_rd and the others below).
struct SoundArgs {
    const double *xlo, *xhi;
    const double *inL[2], *inU[2];   // interval state per half (previous launch)
    double *outL[2], *outU[2];
    double *lo, *hi;                 // MM: written by the last launch
    int64_t n, W, ntiles;
    int H, S;
    double h;
    int first, last;
    int *status;
};

// Directed-rounding sums and products issued as fused multiply-adds:
// fma_rd(a, 1, b) and fma_ru(a, 1, b) round a + b exactly as the plain
// directed sums do, and fma_rd(a, b, +0), fma_ru(a, b, -0) round a b exactly
// as the plain directed products do (an exactly zero product keeps its sign
// under that addend in that mode), so the box is the same bit for bit; the
// FP64 pipe retires the fused forms faster.  1, +0 and -0 come from the
// kernel parameters, or the compiler would fold the fused forms back.
__device__ __forceinline__ double add_rd(double a, double b, const TrafficK &p) { return __fma_rd(a, p.one, b); }
__device__ __forceinline__ double add_ru(double a, double b, const TrafficK &p) { return __fma_ru(a, p.one, b); }
__device__ __forceinline__ double mul_rd(double a, double b, const TrafficK &p) { return __fma_rd(a, b, p.pzero); }
__device__ __forceinline__ double mul_ru(double a, double b, const TrafficK &p) { return __fma_ru(a, b, p.nzero); }

// flux of R6 out of cell g, as an interval; y?n: the right neighbour
__device__ __forceinline__ void flux_iv(const TrafficK &p, double yl, double yu, double yln, double yun, int64_t g,
                                        int64_t n, double &fl, double &fu) {
    const double vl = mul_rd(p.v, yl, p), vu = mul_ru(p.v, yu, p);
    if (g == n - 1) {
        fl = kmin(p.cap, vl);
        fu = kmin(p.cap, vu);
    } else {
        fl = kmin(p.cap, kmin(vl, mul_rd(p.w, add_rd(p.xbar, -yun, p), p)));
        fu = kmin(p.cap, kmin(vu, mul_ru(p.w, add_ru(p.xbar, -yln, p), p)));
    }
}

template <int RADIUS, int KC>
__device__ __forceinline__ void sound_rhs(const TrafficK &p, const double (&yl)[KC], const double (&yu)[KC],
                                          int64_t g0, int64_t n, double dl, double du, double hp,
                                          double (&kl)[KC], double (&ku)[KC]) {
    double EU[KC + 2];
    exchange<1>(yu, EU);
    if (RADIUS) {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            double acc = (g == 0) ? hp : 0.0;
            if (g > 0) acc = add_ru(acc, mul_ru(p.v, EU[j], p), p);
            if (g < n - 1) acc = add_ru(acc, mul_ru(p.w, EU[j + 2], p), p);
            ku[j] = (g < 0 || g >= n) ? 0.0 : acc;
        }
        return;
    }
    double EL[KC + 2];
    exchange<1>(yl, EL);
    // fluxes out of cells g0 - 1 .. g0 + KC - 1
    double fl[KC + 1], fu[KC + 1];
#pragma unroll
    for (int m = 0; m <= KC; ++m) {
        const int64_t g = g0 - 1 + m;
        flux_iv(p, EL[m], EU[m], EL[m + 1], EU[m + 1], g, n, fl[m], fu[m]);
        if (g == -1) { fl[m] = dl; fu[m] = du; }   // inflow of cell 0
    }
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        const int64_t g = g0 + j;
        const double a = add_rd(fl[j], -fu[j + 1], p), b = add_ru(fu[j], -fl[j + 1], p);
        const bool in = g >= 0 && g < n;
        kl[j] = in ? a : 0.0;
        ku[j] = in ? b : 0.0;
    }
}

template <int METHOD, int HALF>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, 2) stencil_traffic_sound_rk4(SoundArgs a, TrafficK p) {
    constexpr int KC = KC_WIDE;
    constexpr int RADIUS = (METHOD == CGB && HALF == 1);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t n = a.n;
    int flags = 0;
    // inflow of this half: MM the corner's own input, CGB the center's interval
    double dl, du;
    if (METHOD == MM) { dl = du = HALF ? p.d_hi : p.d_lo; }
    else { dl = 0.5 * add_rd(p.d_lo, p.d_hi, p); du = 0.5 * add_ru(p.d_lo, p.d_hi, p); }
    const double hp = 0.5 * add_ru(p.d_hi, -p.d_lo, p);
    const double hh = 0.5 * a.h;
    for (int64_t t = warp; t < a.ntiles; t += nwarps) {
        const int64_t own0 = t * a.W;
        const int64_t g0 = own0 - a.H + (int64_t)lane * KC;
        double zl[KC], zu[KC];
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            const bool in = g >= 0 && g < n;
            if (a.first) {
                const double lo = in ? __ldg(a.xlo + g) : 0.0, hi = in ? __ldg(a.xhi + g) : 0.0;
                const bool owned = g >= own0 && g < own0 + a.W && in;
                if (HALF == 0 && owned && !(kle(lo, hi) && kfinite(lo) && kfinite(hi))) flags |= ST_BADINPUT;
                if (METHOD == MM) { zl[j] = zu[j] = HALF ? hi : lo; }
                else if (HALF == 0) { zl[j] = 0.5 * add_rd(lo, hi, p); zu[j] = 0.5 * add_ru(lo, hi, p); }
                else { zl[j] = 0.0; zu[j] = 0.5 * add_ru(hi, -lo, p); }
            } else {
                zl[j] = (in && !RADIUS) ? __ldg(a.inL[HALF] + g) : 0.0;
                zu[j] = in ? __ldg(a.inU[HALF] + g) : 0.0;
            }
        }
        for (int s = 0; s < a.S; ++s) {
            double yl[KC], yu[KC], al[KC], au[KC], kl[KC], ku[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) { yl[j] = zl[j]; yu[j] = zu[j]; }
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                sound_rhs<RADIUS>(p, yl, yu, g0, n, dl, du, hp, kl, ku);
                const double cs = (st == 2) ? a.h : hh;
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    if (st == 0) { au[j] = ku[j]; al[j] = kl[j]; }
                    else if (st == 3) { au[j] = add_ru(au[j], ku[j], p); al[j] = add_rd(al[j], kl[j], p); }
                    else { au[j] = add_ru(au[j], 2.0 * ku[j], p); al[j] = add_rd(al[j], 2.0 * kl[j], p); }
                    if (st < 3) {
                        yu[j] = add_ru(zu[j], mul_ru(cs, ku[j], p), p);
                        if (!RADIUS) yl[j] = add_rd(zl[j], mul_rd(cs, kl[j], p), p);
                    }
                }
            }
            // z + (h/6) acc with h/6 in [c6l, c6u]
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                const double ql = RADIUS ? au[j] : al[j];
                zu[j] = add_ru(zu[j], mul_ru(dkey(au[j]) >= 0 ? p.c6u : p.c6l, au[j], p), p);
                if (!RADIUS) zl[j] = add_rd(zl[j], mul_rd(dkey(ql) >= 0 ? p.c6l : p.c6u, ql, p), p);
            }
        }
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            if (!(g >= own0 && g < own0 + a.W && g < n && g >= 0)) continue;
            if (a.last && METHOD == MM) {
                const double v = HALF ? zu[j] : zl[j];
                if (!kfinite(v)) flags |= ST_NONFINITE;
                (HALF ? a.hi : a.lo)[g] = v;
            } else {
                if (!RADIUS) a.outL[HALF][g] = zl[j];
                a.outU[HALF][g] = zu[j];
            }
        }
    }
    if (flags) atomicOr(a.status, flags);
}

// CGB outward box: lo = (cl - ru) rounded down, hi = (cu + ru) rounded up
__global__ void sound_cgb_box(const double *cl, const double *cu, const double *ru, double *lo, double *hi, int64_t n,
                              int *status) {
    int flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = ru[i];
        if (dkey(r) < 0) flags |= ST_NEGRADIUS;
        const double l = __dadd_rd(cl[i], -r), u = __dadd_ru(cu[i], r);
        if (!kfinite(l) || !kfinite(u)) flags |= ST_NONFINITE;
        lo[i] = l;
        hi[i] = u;
    }
    if (flags) atomicOr(status, flags);
}

// CGB output box from the final center and radius: lo = c - r, hi = c + r
__global__ void cgb_box(double *c_lo, double *r_hi, int64_t n, int *status) {
    int flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double c = c_lo[i], r = r_hi[i];
        if (dkey(r) < 0) flags |= ST_NEGRADIUS;
        double lo = c - r, hi = c + r;
        if (!kfinite(lo) || !kfinite(hi)) flags |= ST_NONFINITE;
        c_lo[i] = lo;
        r_hi[i] = hi;
    }
    if (flags) atomicOr(status, flags);
}

// ------------------------------------------------------------------ KS
// MM embedding (the decomposition of R7): linear stencil split by coefficient
// sign, the product -g_nl u_i u_x bounded with u_i at its own argument over
// the interval of u_x spanned by the neighbours.  With q = -k u_i and the two
// candidate differences dL (at x_{i+1}, xh_{i-1}) and dH (at xh_{i+1}, x_{i-1}),
// the lower half takes min(q dL, q dH) when dL <= dH and the max otherwise;
// in both cases that is q times dL when q >= 0 and dH when q < 0 (the upper
// half likewise with the roles of dL and dH exchanged).  The sign of q is
// read from the sign bits of k and u_i (u_i = 0 makes the term vanish either
// way), and u_i (a0 - k d) + a1 l1 + a2 l2 takes four fused operations.
__device__ __forceinline__ bool sign_differs(double a, double b) {
    return (__double_as_longlong(a) ^ __double_as_longlong(b)) < 0;
}

template <int KC>
__device__ __forceinline__ void ks_mm_rhs(const KsK &p, const double (&x)[KC], const double (&xh)[KC],
                                          double (&kx)[KC], double (&kxh)[KC]) {
    double X[KC + 4], XH[KC + 4];
    exchange<2>(x, X);
    exchange<2>(xh, XH);
    const bool s1 = p.a1 >= 0.0, s2 = p.a2 >= 0.0;
    const double nk = -p.k, one = p.one, nz = p.nzero;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        const int c = j + 2;
        double l1 = fadd(s1 ? X[c - 1] : XH[c - 1], s1 ? X[c + 1] : XH[c + 1], one);
        double l2 = fadd(s2 ? X[c - 2] : XH[c - 2], s2 ? X[c + 2] : XH[c + 2], one);
        double u1 = fadd(s1 ? XH[c - 1] : X[c - 1], s1 ? XH[c + 1] : X[c + 1], one);
        double u2 = fadd(s2 ? XH[c - 2] : X[c - 2], s2 ? XH[c + 2] : X[c + 2], one);
        const double dL = fadd(X[c + 1], -XH[c - 1], one);   // 2dx * u_x at (x_{i+1}, xh_{i-1})
        const double dH = fadd(XH[c + 1], -X[c - 1], one);   // 2dx * u_x at (xh_{i+1}, x_{i-1})
        // -k u >= 0 exactly when the signs of k and u differ
        const double dl = sign_differs(p.k, X[c]) ? dL : dH;
        const double dh = sign_differs(p.k, XH[c]) ? dH : dL;
        kx[j] = fma(X[c], fma(nk, dl, p.a0), fma(p.a1, l1, fmul(p.a2, l2, nz)));
        kxh[j] = fma(XH[c], fma(nk, dh, p.a0), fma(p.a1, u1, fmul(p.a2, u2, nz)));
    }
}

// CGB: center f(c) and radius C(c, r) r with C the supremum of the Jacobian
// over the box [c - r, c + r] (R3): C_ii = a0 - k dc + |k| (r_{i+1} + r_{i-1}),
// C_{i,i+-1} = |a1 -+ k c_i| + |k| r_i, C_{i,i+-2} = |a2|; the two |k| r_i r_{i+-1}
// terms fold into the diagonal's factor
template <int KC>
__device__ __forceinline__ void ks_cgb_rhs(const KsK &p, const double (&cc)[KC], const double (&rr)[KC],
                                           double (&kc)[KC], double (&kr)[KC]) {
    double C[KC + 4], Rr[KC + 4];
    exchange<2>(cc, C);
    exchange<2>(rr, Rr);
    const double aa2 = kabs(p.a2), ak = kabs(p.k), nk = -p.k, one = p.one, nz = p.nzero;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        const int c = j + 2;
        const double dc = fadd(C[c + 1], -C[c - 1], one);
        const double t = fmul(p.k, C[c], nz);
        const double lin = fma(p.a2, fadd(C[c - 2], C[c + 2], one),
                               fma(p.a1, fadd(C[c - 1], C[c + 1], one), fmul(p.a0, C[c], nz)));
        kc[j] = fma(-t, dc, lin);
        // C_ii r_i + |k| r_i (r_{i+1} + r_{i-1}) = r_i (a0 - k dc + 2 |k| sr)
        const double sr = fadd(Rr[c + 1], Rr[c - 1], one);
        const double e = fma(2.0 * ak, sr, fma(nk, dc, p.a0));
        double acc = fma(aa2, fadd(Rr[c - 2], Rr[c + 2], one), fmul(e, Rr[c], nz));
        acc = fma(kabs(fadd(-t, p.a1, one)), Rr[c + 1], acc);
        kr[j] = fma(kabs(fadd(t, p.a1, one)), Rr[c - 1], acc);
    }
}

template <int METHOD, int KC>
__device__ __forceinline__ void ks_rhs(const KsK &p, const double (&a)[KC], const double (&b)[KC],
                                       double (&ka)[KC], double (&kb)[KC]) {
    if (METHOD == MM) ks_mm_rhs(p, a, b, ka, kb);
    else ks_cgb_rhs(p, a, b, ka, kb);
}

template <int METHOD, int KC>
__global__ void __launch_bounds__(32 * KS_WARPS_PER_BLOCK, 3) stencil_ks_rk4(StepArgs a, KsK p) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t n = a.n;
    const int64_t ntiles = a.ntiles;
    int flags = 0;

    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int64_t own0 = t * a.W;
        const int64_t g0 = own0 - a.H + (int64_t)lane * KC;
        double zA[KC], zB[KC];
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            const int64_t idx = wrap_index(g, n);   // periodic grid
            double va = __ldg(a.inA + idx), vb = __ldg(a.inB + idx);
            if (a.first) {
                const bool owned = g >= own0 && g < own0 + a.W && g < n && g >= 0;
                if (owned && !(kle(va, vb) && kfinite(va) && kfinite(vb))) flags |= ST_BADINPUT;
                if (METHOD == CGB) {
                    double c = 0.5 * (va + vb), r = 0.5 * (vb - va);
                    va = c;
                    vb = r;
                }
            }
            zA[j] = va;
            zB[j] = vb;
        }
        for (int s = 0; s < a.S; ++s) {
            double yA[KC], yB[KC], aA[KC], aB[KC], kA[KC], kB[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) { yA[j] = zA[j]; yB[j] = zB[j]; }
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<0>(zA, yA, aA, kA, a);
            rk4_update<0>(zB, yB, aB, kB, a);
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<1>(zA, yA, aA, kA, a);
            rk4_update<1>(zB, yB, aB, kB, a);
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<2>(zA, yA, aA, kA, a);
            rk4_update<2>(zB, yB, aB, kB, a);
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<3>(zA, yA, aA, kA, a);
            rk4_update<3>(zB, yB, aB, kB, a);
        }
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            if (!(g >= own0 && g < own0 + a.W && g < n && g >= 0)) continue;
            double oa = zA[j], ob = zB[j];
            if (a.last) {
                if (METHOD == CGB) {
                    if (dkey(ob) < 0) flags |= ST_NEGRADIUS;
                    double lo = oa - ob, hi = oa + ob;
                    oa = lo;
                    ob = hi;
                }
                if (!kfinite(oa) || !kfinite(ob)) flags |= ST_NONFINITE;
            }
            a.outA[g] = oa;
            a.outB[g] = ob;
        }
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ KS, all steps in one launch
// A KS grid of a few waves of warp tiles (2^20 points: 4370 tiles over 1776
// resident warps) loses the end of every launch: as the last tiles of a step
// finish, SMs hold fewer warps than keep the FP64 pipe busy, and the next
// step's launch waits for all of them.  Here one persistent launch runs every
// step: warps take (step, tile) items in step-major order from a counter, and
// item (s, t) starts as soon as tiles t - 1, t, t + 1 (the tiles its halo of
// 4R = 8 cells reaches) have finished step s - 1, so step s + 1 fills the SMs
// that step s leaves idle.  An item waits only for items handed out before it
// (to running warps), so no wait is circular; each wait is also bounded
// (wait_ns), after which the launch records ST_TIMEOUT and stops.  A tile's
// arithmetic is that of stencil_ks_rk4 at one step per launch, so the box is
// the same bit for bit.
struct FlowArgs {
    StepArgs st;                   // n, W, H = 8, h, hh, h6, status; ntiles
    const double *xlo, *xhi;       // the input box (step 0)
    double *bufA[2], *bufB[2];     // step s writes [(N - 1 - s) % 2]: [0] is the output (lo, hi)
    int64_t N;
    unsigned long long *next;      // item counter (zeroed before the launch)
    int *ready;                    // per tile: steps completed (zeroed before the launch)
    unsigned long long wait_ns;
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int METHOD, int KC>
__global__ void __launch_bounds__(32 * KS_WARPS_PER_BLOCK, 3) stencil_ks_flow(FlowArgs f, KsK p) {
    const StepArgs &a = f.st;
    const int lane = threadIdx.x & 31;
    const int64_t n = a.n;
    const uint32_t T = (uint32_t)a.ntiles;
    const unsigned long long total = (unsigned long long)f.N * T;   // < 2^32 (checked on the host)
    int flags = 0;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(f.next, 1ULL);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= total) break;
        const uint32_t s = (uint32_t)i / T, t = (uint32_t)i - s * T;   // 32-bit division
        if (s > 0) {
            // wait for the neighbouring tiles' previous step (bounded)
            int late = 0;
            if (lane == 0) {
                const uint32_t tl = t == 0 ? T - 1 : t - 1, tr = t == T - 1 ? 0 : t + 1;
                const unsigned long long t0 = global_ns();
                unsigned ns = 64;
                while (ld_acquire_gpu(f.ready + tl) < (int)s || ld_acquire_gpu(f.ready + t) < (int)s ||
                       ld_acquire_gpu(f.ready + tr) < (int)s) {
                    if (global_ns() - t0 > f.wait_ns || (*(volatile int *)a.status & ST_TIMEOUT)) {
                        late = 1;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 1024) ns *= 2;
                }
            }
            if (__shfl_sync(0xffffffffu, late, 0)) {
                if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
                return;
            }
        }
        const int64_t own0 = (int64_t)t * a.W;
        const int64_t g0 = own0 - a.H + (int64_t)lane * KC;
        const int in = (int)((f.N - s) & 1), out = (int)((f.N - 1 - s) & 1);
        const double *srcA = s == 0 ? f.xlo : f.bufA[in], *srcB = s == 0 ? f.xhi : f.bufB[in];
        double zA[KC], zB[KC];
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            const int64_t idx = wrap_index(g, n);
            // written by other warps during this launch: read through L2
            double va = __ldcg(srcA + idx), vb = __ldcg(srcB + idx);
            if (s == 0) {
                const bool owned = g >= own0 && g < own0 + a.W && g < n && g >= 0;
                if (owned && !(kle(va, vb) && kfinite(va) && kfinite(vb))) flags |= ST_BADINPUT;
                if (METHOD == CGB) {
                    double c = 0.5 * (va + vb), r = 0.5 * (vb - va);
                    va = c;
                    vb = r;
                }
            }
            zA[j] = va;
            zB[j] = vb;
        }
        {
            double yA[KC], yB[KC], aA[KC], aB[KC], kA[KC], kB[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) { yA[j] = zA[j]; yB[j] = zB[j]; }
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<0>(zA, yA, aA, kA, a);
            rk4_update<0>(zB, yB, aB, kB, a);
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<1>(zA, yA, aA, kA, a);
            rk4_update<1>(zB, yB, aB, kB, a);
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<2>(zA, yA, aA, kA, a);
            rk4_update<2>(zB, yB, aB, kB, a);
            ks_rhs<METHOD>(p, yA, yB, kA, kB);
            rk4_update<3>(zA, yA, aA, kA, a);
            rk4_update<3>(zB, yB, aB, kB, a);
        }
        const bool last = (int64_t)s == f.N - 1;
        double *outA = f.bufA[out], *outB = f.bufB[out];
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const int64_t g = g0 + j;
            if (!(g >= own0 && g < own0 + a.W && g < n && g >= 0)) continue;
            double oa = zA[j], ob = zB[j];
            if (last) {
                if (METHOD == CGB) {
                    if (dkey(ob) < 0) flags |= ST_NEGRADIUS;
                    double lo = oa - ob, hi = oa + ob;
                    oa = lo;
                    ob = hi;
                }
                if (!kfinite(oa) || !kfinite(ob)) flags |= ST_NONFINITE;
            }
            outA[g] = oa;
            outB[g] = ob;
        }
        // the tile's step s is visible before its flag says so
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_gpu(f.ready + t, (int)s + 1);
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ host
// Launch shape for a grid of warp tiles.  A tile is one warp's serial FP64
// work (a warp issues an FP64 instruction about every 68 clocks, and an SM's
// FP64 pipe keeps about four warps at that rate), so a launch with few tiles
// takes one tile's time only if its warps are spread over all SMs: below
// max_wpb warps per SM the blocks shrink to ceil(warps / 148) warps, one block
// per SM.
struct Shape {
    unsigned grid, threads;
};
static Shape shape_for(int64_t warps_needed, int64_t max_wpb = WARPS_PER_BLOCK) {
    int64_t wpb = (warps_needed + 147) / 148;
    if (wpb < 1) wpb = 1;
    if (wpb > max_wpb) wpb = max_wpb;
    int64_t blocks = (warps_needed + wpb - 1) / wpb;
    const int64_t cap = 148LL * 64;
    return Shape{(unsigned)(blocks > cap ? cap : blocks), (unsigned)(32 * wpb)};
}

// Cells per lane for an n-cell grid with a halo of H cells per tile side and
// `halves` warps per tile: the narrow tile when its estimated time is shorter,
// the time being the waves of warps over 592 full-rate warp slots (four per
// SM; at least one wave) times a warp's cells.  The narrow tile is taken only
// while its halo leaves it at least half its cells.
static int tile_kc(int64_t n, int H, int halves) {
    if (2 * H > 32 * KC_NARROW / 2) return KC_WIDE;
    if (opt_tile() > 0) return opt_tile() == KC_NARROW ? KC_NARROW : KC_WIDE;
    auto cost = [&](int kc) {
        const int64_t w = 32 * kc - 2 * H;
        const double warps = (double)halves * (double)((n + w - 1) / w);
        return (warps > 592.0 ? warps / 592.0 : 1.0) * kc;
    };
    return cost(KC_NARROW) < cost(KC_WIDE) ? KC_NARROW : KC_WIDE;
}

// A grid whose narrow tiles fit in one wave of warps (592, four per SM)
// takes its time from the fixed cost of each launch, not from
// the FP64 pipe: it runs the most steps per launch (up to 4) that keep it in
// one wave and leave the narrow tile half its cells.  Other grids: 1.
int stencil_short_steps(int R, int halves, int64_t n) {
    for (int S = 4; S > 1; S /= 2) {
        const int H = 4 * R * S;
        if (2 * H > 32 * KC_NARROW / 2) continue;
        const int64_t w = 32 * KC_NARROW - 2 * H;
        if ((int64_t)halves * ((n + w - 1) / w) <= 592) return S;
    }
    return 1;
}

template <int KC>
static void launch_traffic_rk4(int method, bool pw, const StepArgs &a, const TrafficK &p, cudaStream_t st) {
    const Shape g = shape_for(2 * a.tcount);
    if (method == MM && pw) stencil_traffic_rk4<MM, true, KC><<<g.grid, g.threads, 0, st>>>(a, p);
    else if (method == MM) stencil_traffic_rk4<MM, false, KC><<<g.grid, g.threads, 0, st>>>(a, p);
    else if (pw) stencil_traffic_rk4<CGB, true, KC><<<g.grid, g.threads, 0, st>>>(a, p);
    else stencil_traffic_rk4<CGB, false, KC><<<g.grid, g.threads, 0, st>>>(a, p);
}

// Integrate N steps with S steps per launch, ping-ponging between the output
// (lo, hi) and the scratch pair so that the last launch writes the output.
template <class LaunchFn>
static int run_steps(int R, int kc, int64_t n, const double *xlo, const double *xhi, double *lo, double *hi,
                     double *sA, double *sB, double h, int64_t N, int S, int *status, LaunchFn launch) {
    const int64_t L = (N + S - 1) / S;
    double *bufA[2] = {lo, sA}, *bufB[2] = {hi, sB};
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        const int s = (int)((N - done) < S ? (N - done) : S);
        StepArgs a;
        a.n = n;
        a.H = 4 * R * s;
        a.W = 32 * kc - 2 * a.H;
        a.ntiles = (n + a.W - 1) / a.W;
        a.tile0 = 0;
        a.tcount = a.ntiles;
        a.S = s;
        a.h = h;
        a.hh = 0.5 * h;
        a.h6 = h / 6.0;
        a.one = 1.0;
        a.nzero = -0.0;
        a.first = (q == 0);
        a.last = (q == L - 1);
        a.inA = (q == 0) ? xlo : bufA[(L - q) % 2];
        a.inB = (q == 0) ? xhi : bufB[(L - q) % 2];
        a.outA = bufA[(L - 1 - q) % 2];
        a.outB = bufB[(L - 1 - q) % 2];
        a.status = status;
        const double *ptrs[6] = {a.inA, a.inB, a.outA, a.outB, sA, sB};
        a.vec = 1;
        for (const double *ptr : ptrs)
            if (reinterpret_cast<uintptr_t>(ptr) % 16) a.vec = 0;
        int rc = launch(a);
        if (rc) return rc;
        done += s;
    }
    return REACH_OK;
}

// Whether stencil_traffic_flow runs an n-cell chain over N steps: the plain
// (not box-evaluated, not outward-rounded) kernel with wide tiles at one step
// per launch, N x 2 x tiles < 2^32, and by default at least 1.5 waves of the
// 2368 resident warps (two 8-warp blocks per SM).  Measured at one launch
// against one per step (fraction of the FP64 peak, MM / CGB): 2^19 cells
// 0.672 / 0.735 against 0.665 / 0.679, 2^20 0.856 / 0.881 against 0.722 /
// 0.746, 2^22 0.861 / 0.885 against 0.823 / 0.855, 2^26 0.862 / 0.885 against
// 0.859 / 0.883; at 2^18 (0.9 waves) 0.386 / 0.451 against 0.571 / 0.625.
bool traffic_flow_eligible(const TrafficK &p, int method, int64_t n, int64_t N) {
    if (opt_one_launch() == 1 || N < 2 || p.sound || (method == CGB && p.local)) return false;
    if (tile_kc(n, 4, 2) != KC_WIDE) return false;
    const int64_t W = 32 * KC_WIDE - 8, T = (n + W - 1) / W;
    if (T < 2 || (uint64_t)N * (uint64_t)(2 * T) >= (1ULL << 32)) return false;
    if (opt_one_launch() == 2) return true;
    return 2 * T >= 3 * 2368 / 2;
}

int64_t traffic_flow_work_bytes(int64_t n) {
    const int64_t W = 32 * KC_WIDE - 8, T = (n + W - 1) / W;
    return 16 + 8 * T;
}

// the per-call coefficients of traffic_radius_step for step h
static TrafficK with_radius_coeffs(TrafficK p, double h) {
    const double c[4] = {0.25 * h, h / 3.0, 0.5 * h, h};
    for (int s = 0; s < 4; ++s) {
        p.rc[s] = c[s];
        p.rv[s] = c[s] * p.v;
        p.rw[s] = c[s] * p.w;
    }
    return p;
}

int stencil_traffic_flow_run(int method, const TrafficK &p0, int64_t n, const double *xlo, const double *xhi,
                             double *lo, double *hi, double *sA, double *sB, double h, int64_t N, int *status,
                             void *work, cudaStream_t st) {
    const TrafficK p = with_radius_coeffs(p0, h);
    TrafficFlowArgs f;
    memset(&f, 0, sizeof f);
    StepArgs &a = f.st;
    a.n = n;
    a.H = 4;
    a.W = 32 * KC_WIDE - 2 * a.H;
    a.ntiles = (n + a.W - 1) / a.W;
    a.tile0 = 0;
    a.tcount = a.ntiles;
    a.S = 1;
    a.h = h;
    a.hh = 0.5 * h;
    a.h6 = h / 6.0;
    a.one = 1.0;
    a.nzero = -0.0;
    a.status = status;
    const double *ptrs[6] = {xlo, xhi, lo, hi, sA, sB};
    a.vec = 1;
    for (const double *ptr : ptrs)
        if (reinterpret_cast<uintptr_t>(ptr) % 16) a.vec = 0;
    f.xlo = xlo;
    f.xhi = xhi;
    f.bufA[0] = lo; f.bufB[0] = hi;
    f.bufA[1] = sA; f.bufB[1] = sB;
    f.N = N;
    f.next = (unsigned long long *)work;
    f.ready = (int *)((char *)work + 16);
    f.wait_ns = 2000000000ULL;   // 2 s: far beyond any tile's step
    REACH_CUDA(cudaMemsetAsync(work, 0, traffic_flow_work_bytes(n), st));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(2 * sms);   // two 8-warp blocks per SM: the kernel's launch bound
    const bool pw = p.v_pow2 != 0;
    const unsigned threads = 32 * WARPS_PER_BLOCK;
    if (method == MM && pw) stencil_traffic_flow<MM, true, KC_WIDE><<<grid, threads, 0, st>>>(f, p);
    else if (method == MM) stencil_traffic_flow<MM, false, KC_WIDE><<<grid, threads, 0, st>>>(f, p);
    else if (pw) stencil_traffic_flow<CGB, true, KC_WIDE><<<grid, threads, 0, st>>>(f, p);
    else stencil_traffic_flow<CGB, false, KC_WIDE><<<grid, threads, 0, st>>>(f, p);
    REACH_LAUNCHED("stencil_traffic_flow");
    if (method == CGB) {
        int64_t blocks = (n + 255) / 256;
        if (blocks > 148 * 16) blocks = 148 * 16;
        cgb_box<<<(unsigned)blocks, 256, 0, st>>>(lo, hi, n, status);
        REACH_LAUNCHED("cgb_box");
    }
    return REACH_OK;
}

int stencil_traffic(int method, const TrafficK &p0, int64_t n, const double *xlo, const double *xhi,
                    double *lo, double *hi, double *sA, double *sB, double h, int64_t N, int S,
                    int *status, cudaStream_t st) {
    const TrafficK p = with_radius_coeffs(p0, h);
    const bool local = method == CGB && p.local;
    // the box-evaluated C kernel holds both halves per warp: wide tiles only
    const int kc = local ? KC_WIDE : tile_kc(n, 4 * S, 2);
    int rc = run_steps(1, kc, n, xlo, xhi, lo, hi, sA, sB, h, N, S, status, [&](const StepArgs &a) {
        const int64_t ntiles = (n + a.W - 1) / a.W;
        const bool pw = p.v_pow2 != 0;
        if (local) {
            const Shape g = shape_for(ntiles);
            if (pw) stencil_traffic_cgbl_rk4<true><<<g.grid, g.threads, 0, st>>>(a, p);
            else stencil_traffic_cgbl_rk4<false><<<g.grid, g.threads, 0, st>>>(a, p);
            REACH_LAUNCHED("stencil_traffic_cgbl_rk4");
            return REACH_OK;
        }
        if (kc == KC_NARROW) launch_traffic_rk4<KC_NARROW>(method, pw, a, p, st);
        else launch_traffic_rk4<KC_WIDE>(method, pw, a, p, st);
        REACH_LAUNCHED("stencil_traffic_rk4");
        return REACH_OK;
    });
    if (rc || method != CGB || local) return rc;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    cgb_box<<<(unsigned)blocks, 256, 0, st>>>(lo, hi, n, status);
    REACH_LAUNCHED("cgb_box");
    return REACH_OK;
}

// Host buffers in and out: the input box goes to the device in chunks on a
// second stream, the first launch runs chunk by chunk behind those copies
// (chunk c waits for c + 1, which holds its right halo), and the last launch
// sends each chunk's result back while the next chunk computes, so the
// copies overlap the first and last RK4 steps instead of preceding and
// following the whole run.
namespace {
struct CopyLane {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[2 * OVERLAP_CHUNKS] = {};
    int nev = 0;
    ~CopyLane() {
        for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
        if (cs) cudaStreamDestroy(cs);
    }
};
}  // namespace

int stencil_traffic_overlap(int method, const TrafficK &p0, int64_t n, const double *hxlo, const double *hxhi,
                            double *hlo, double *hhi, double h, int64_t N, int S, Staging &sg) {
    const TrafficK p = with_radius_coeffs(p0, h);
    constexpr int C = OVERLAP_CHUNKS;
    double *buf;
    int rc;
    const int64_t np = (n + 1) & ~(int64_t)1;   // even stride: every vector starts on 16 bytes
    if ((rc = sg.scratch(6 * np * sizeof(double), (void **)&buf))) return rc;
    double *dxlo = buf, *dxhi = buf + np, *dlo = buf + 2 * np, *dhi = buf + 3 * np, *sA = buf + 4 * np,
           *sB = buf + 5 * np;
    CopyLane cl;
    REACH_CUDA(cudaStreamCreateWithFlags(&cl.cs, cudaStreamNonBlocking));
    for (int i = 0; i < 2 * C; ++i) {
        REACH_CUDA(cudaEventCreateWithFlags(&cl.ev[i], cudaEventDisableTiming));
        cl.nev = i + 1;
    }
    cudaEvent_t *ein = cl.ev, *eout = cl.ev + C;
    const cudaStream_t st = sg.st;
    // the copy stream starts after the work already queued on the call's stream
    REACH_CUDA(cudaEventRecord(eout[0], st));
    REACH_CUDA(cudaStreamWaitEvent(cl.cs, eout[0], 0));

    const int64_t L = (N + S - 1) / S;
    const bool pw = p.v_pow2 != 0;
    auto launch = [&](const StepArgs &b) {
        launch_traffic_rk4<KC_WIDE>(method, pw, b, p, st);
        REACH_LAUNCHED("stencil_traffic_rk4");
        return REACH_OK;
    };
    if (N % S == 0 && L >= 2 * C) {
        // Wavefront at both ends: the first C launches and the last C launches
        // run chunk by chunk, the launches between them whole.  Within an end,
        // launch q's chunk c reads chunks c - 1 .. c + 1 of launch q - 1's
        // output and is issued on diagonal q + c, earlier launches first within
        // a diagonal, so chunk c + 1 of launch q - 1 (same diagonal, smaller q)
        // precedes it; launch q + 1 overwrites chunk c of launch q's input on
        // diagonal q + c + 1, after all of its readers (launch q, chunks
        // c - 1 .. c + 1).  Everything is on one stream.  The input copies then
        // overlap the first diagonals, and chunk c of the last launch completes
        // early, its copy back overlapping the rest of the end.
        StepArgs a;
        a.n = n;
        a.H = 4 * S;
        a.W = 32 * KC_WIDE - 2 * a.H;
        a.ntiles = (n + a.W - 1) / a.W;
        a.S = S;
        a.h = h;
        a.hh = 0.5 * h;
        a.h6 = h / 6.0;
        a.one = 1.0;
        a.nzero = -0.0;
        a.status = sg.status;
        a.vec = (reinterpret_cast<uintptr_t>(buf) % 16) == 0;   // one allocation, even strides
        double *bufA[2] = {dlo, sA}, *bufB[2] = {dhi, sB};
        auto tile_at = [&](int c) { return a.ntiles * c / C; };
        auto args_for = [&](int64_t q) {
            StepArgs b = a;
            b.first = (q == 0);
            b.last = (q == L - 1);
            b.inA = (q == 0) ? dxlo : bufA[(L - q) % 2];
            b.inB = (q == 0) ? dxhi : bufB[(L - q) % 2];
            b.outA = bufA[(L - 1 - q) % 2];
            b.outB = bufB[(L - 1 - q) % 2];
            b.tile0 = 0;
            b.tcount = a.ntiles;
            return b;
        };
        for (int c = 0; c < C; ++c) {
            const int64_t c0 = tile_at(c) * a.W, c1 = std::min<int64_t>(tile_at(c + 1) * a.W, n);
            REACH_CUDA(cudaMemcpyAsync(dxlo + c0, hxlo + c0, (c1 - c0) * sizeof(double), cudaMemcpyHostToDevice,
                                       cl.cs));
            REACH_CUDA(cudaMemcpyAsync(dxhi + c0, hxhi + c0, (c1 - c0) * sizeof(double), cudaMemcpyHostToDevice,
                                       cl.cs));
            REACH_CUDA(cudaEventRecord(ein[c], cl.cs));
        }
        // launches [q0, q0 + C) in wavefront order
        auto wavefront = [&](int64_t q0) -> int {
            for (int64_t d = 0; d < 2 * C - 1; ++d) {
                const int64_t qlo = d - (C - 1) > 0 ? d - (C - 1) : 0, qhi = d < C - 1 ? d : C - 1;
                for (int64_t dq = qlo; dq <= qhi; ++dq) {
                    const int64_t q = q0 + dq;
                    const int c = (int)(d - dq);
                    StepArgs b = args_for(q);
                    b.tile0 = tile_at(c);
                    b.tcount = tile_at(c + 1) - b.tile0;
                    if (q == 0) REACH_CUDA(cudaStreamWaitEvent(st, ein[c + 1 < C ? c + 1 : C - 1], 0));
                    if ((rc = launch(b))) return rc;
                    if (q == L - 1) {
                        const int64_t c0 = b.tile0 * a.W, c1 = std::min<int64_t>((b.tile0 + b.tcount) * a.W, n);
                        if (method == CGB) {
                            int64_t blocks = (c1 - c0 + 255) / 256;
                            if (blocks > 148 * 16) blocks = 148 * 16;
                            cgb_box<<<(unsigned)blocks, 256, 0, st>>>(dlo + c0, dhi + c0, c1 - c0, sg.status);
                            REACH_LAUNCHED("cgb_box");
                        }
                        REACH_CUDA(cudaEventRecord(eout[c], st));
                        REACH_CUDA(cudaStreamWaitEvent(cl.cs, eout[c], 0));
                        REACH_CUDA(cudaMemcpyAsync(hlo + c0, dlo + c0, (c1 - c0) * sizeof(double),
                                                   cudaMemcpyDeviceToHost, cl.cs));
                        REACH_CUDA(cudaMemcpyAsync(hhi + c0, dhi + c0, (c1 - c0) * sizeof(double),
                                                   cudaMemcpyDeviceToHost, cl.cs));
                    }
                }
            }
            return REACH_OK;
        };
        if ((rc = wavefront(0))) return rc;
        for (int64_t q = C; q < L - C; ++q)
            if ((rc = launch(args_for(q)))) return rc;
        if ((rc = wavefront(L - C))) return rc;
        REACH_CUDA(cudaEventRecord(eout[0], cl.cs));
        REACH_CUDA(cudaStreamWaitEvent(st, eout[0], 0));
        REACH_CUDA(cudaStreamSynchronize(cl.cs));
        return REACH_OK;
    }
    // few launches, or launches of unequal length (N not a multiple of S): only
    // the first and the last launch run chunk by chunk
    double *bufA[2] = {dlo, sA}, *bufB[2] = {dhi, sB};
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        const int s = (int)((N - done) < S ? (N - done) : S);
        StepArgs a;
        a.n = n;
        a.H = 4 * s;
        a.W = 32 * KC_WIDE - 2 * a.H;
        a.ntiles = (n + a.W - 1) / a.W;
        a.tile0 = 0;
        a.tcount = a.ntiles;
        a.S = s;
        a.h = h;
        a.hh = 0.5 * h;
        a.h6 = h / 6.0;
        a.one = 1.0;
        a.nzero = -0.0;
        a.first = (q == 0);
        a.last = (q == L - 1);
        a.inA = (q == 0) ? dxlo : bufA[(L - q) % 2];
        a.inB = (q == 0) ? dxhi : bufB[(L - q) % 2];
        a.outA = bufA[(L - 1 - q) % 2];
        a.outB = bufB[(L - 1 - q) % 2];
        a.status = sg.status;
        a.vec = (reinterpret_cast<uintptr_t>(buf) % 16) == 0;   // one allocation, even strides
        if (!a.first && !a.last) {
            if ((rc = launch(a))) return rc;
            done += s;
            continue;
        }
        // chunk c: tiles [t0, t1), cells [t0 W, t1 W) of the output and of the input copy
        auto tile_at = [&](int c) { return a.ntiles * c / C; };
        if (a.first) {
            for (int c = 0; c < C; ++c) {
                const int64_t c0 = tile_at(c) * a.W, c1 = std::min<int64_t>(tile_at(c + 1) * a.W, n);
                if (c1 > c0) {
                    REACH_CUDA(cudaMemcpyAsync(dxlo + c0, hxlo + c0, (c1 - c0) * sizeof(double),
                                               cudaMemcpyHostToDevice, cl.cs));
                    REACH_CUDA(cudaMemcpyAsync(dxhi + c0, hxhi + c0, (c1 - c0) * sizeof(double),
                                               cudaMemcpyHostToDevice, cl.cs));
                }
                REACH_CUDA(cudaEventRecord(ein[c], cl.cs));
            }
        }
        for (int c = 0; c < C; ++c) {
            StepArgs b = a;
            b.tile0 = tile_at(c);
            b.tcount = tile_at(c + 1) - b.tile0;
            if (a.first) REACH_CUDA(cudaStreamWaitEvent(st, ein[c + 1 < C ? c + 1 : C - 1], 0));
            if (b.tcount > 0 && (rc = launch(b))) return rc;
            if (a.last) {
                const int64_t c0 = b.tile0 * a.W, c1 = std::min<int64_t>((b.tile0 + b.tcount) * a.W, n);
                if (c1 <= c0) continue;
                if (method == CGB) {
                    int64_t blocks = (c1 - c0 + 255) / 256;
                    if (blocks > 148 * 16) blocks = 148 * 16;
                    cgb_box<<<(unsigned)blocks, 256, 0, st>>>(dlo + c0, dhi + c0, c1 - c0, sg.status);
                    REACH_LAUNCHED("cgb_box");
                }
                REACH_CUDA(cudaEventRecord(eout[c], st));
                REACH_CUDA(cudaStreamWaitEvent(cl.cs, eout[c], 0));
                REACH_CUDA(cudaMemcpyAsync(hlo + c0, dlo + c0, (c1 - c0) * sizeof(double), cudaMemcpyDeviceToHost,
                                           cl.cs));
                REACH_CUDA(cudaMemcpyAsync(hhi + c0, dhi + c0, (c1 - c0) * sizeof(double), cudaMemcpyDeviceToHost,
                                           cl.cs));
            }
        }
        done += s;
    }
    // the call's stream waits for the copies back, so the caller's stream order holds
    REACH_CUDA(cudaEventRecord(eout[0], cl.cs));
    REACH_CUDA(cudaStreamWaitEvent(st, eout[0], 0));
    REACH_CUDA(cudaStreamSynchronize(cl.cs));
    return REACH_OK;
}

// h / 6 rounded down and up: q = fl(h / 6) and the exact remainder h - 6 q
static void sixth_bounds(double h, double *dn, double *up) {
    const double q = h / 6.0, e = std::fma(-q, 6.0, h);
    *dn = e < 0.0 ? std::nextafter(q, -INFINITY) : q;
    *up = e > 0.0 ? std::nextafter(q, INFINITY) : q;
}

int stencil_traffic_sound(int method, const TrafficK &p0, int64_t n, const double *xlo, const double *xhi,
                          double *lo, double *hi, double h, int64_t N, int S, Staging &sg) {
    TrafficK p = p0;
    sixth_bounds(h, &p.c6l, &p.c6u);
    // two sets of interval state (lower and upper end per half)
    double *buf;
    int rc;
    if ((rc = sg.scratch(8 * n * sizeof(double), (void **)&buf))) return rc;
    double *setL[2][2], *setU[2][2];
    for (int q = 0; q < 2; ++q)
        for (int half = 0; half < 2; ++half) {
            setL[q][half] = buf + (4 * q + 2 * half) * n;
            setU[q][half] = buf + (4 * q + 2 * half + 1) * n;
        }
    const int64_t L = (N + S - 1) / S;
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        const int s = (int)((N - done) < S ? (N - done) : S);
        SoundArgs a;
        a.xlo = xlo;
        a.xhi = xhi;
        for (int half = 0; half < 2; ++half) {
            a.inL[half] = setL[q % 2][half];
            a.inU[half] = setU[q % 2][half];
            a.outL[half] = setL[(q + 1) % 2][half];
            a.outU[half] = setU[(q + 1) % 2][half];
        }
        a.lo = lo;
        a.hi = hi;
        a.n = n;
        a.H = 4 * s;
        a.W = 32 * KC_WIDE - 2 * a.H;
        a.ntiles = (n + a.W - 1) / a.W;
        a.S = s;
        a.h = h;
        a.first = q == 0;
        a.last = q == L - 1;
        a.status = sg.status;
        const Shape g = shape_for(a.ntiles);
        if (method == MM) {
            stencil_traffic_sound_rk4<MM, 0><<<g.grid, g.threads, 0, sg.st>>>(a, p);
            stencil_traffic_sound_rk4<MM, 1><<<g.grid, g.threads, 0, sg.st>>>(a, p);
        } else {
            stencil_traffic_sound_rk4<CGB, 0><<<g.grid, g.threads, 0, sg.st>>>(a, p);
            stencil_traffic_sound_rk4<CGB, 1><<<g.grid, g.threads, 0, sg.st>>>(a, p);
        }
        REACH_LAUNCHED("stencil_traffic_sound_rk4");
        REACH_LAUNCHED("stencil_traffic_sound_rk4");
        done += s;
    }
    if (method == CGB) {
        const int fin = (int)(L % 2);   // the set the last launch wrote
        int64_t blocks = (n + 255) / 256;
        if (blocks > 148 * 16) blocks = 148 * 16;
        sound_cgb_box<<<(unsigned)blocks, 256, 0, sg.st>>>(setL[fin][0], setU[fin][0], setU[fin][1], lo, hi, n,
                                                          sg.status);
        REACH_LAUNCHED("sound_cgb_box");
    }
    return REACH_OK;
}

// Whether stencil_ks_flow runs an n-point KS grid over N steps: wide tiles at
// one step per launch, at least three tiles (a tile's two neighbours differ),
// N x tiles < 2^32, and by default two to eight waves of the 1776 resident
// warps (three 4-warp blocks per SM), where the end of each launch costs
// most: measured at one launch against one per step, 2^20 points MM 0.80
// against 0.74 of the FP64 pipe, CGB 0.83 against 0.75; 2^21 CGB 0.84 against
// 0.82, MM equal; from 2^22 equal; and at 2^18 (0.6 waves) 0.38 against 0.68,
// where warps waiting for their neighbours hold most of the resident slots.
bool ks_flow_eligible(int64_t n, int64_t N) {
    if (opt_one_launch() == 1 || N < 2) return false;
    if (tile_kc(n, 8, 1) != KC_WIDE) return false;
    const int64_t W = 32 * KC_WIDE - 16, T = (n + W - 1) / W;
    if (T < 3 || (uint64_t)N * (uint64_t)T >= (1ULL << 32)) return false;
    if (opt_one_launch() == 2) return true;
    return T >= 2 * 1776 && T <= 8 * 1776;
}

int stencil_ks_flow_run(int method, const KsK &p, int64_t n, const double *xlo, const double *xhi, double *lo,
                        double *hi, double *sA, double *sB, double h, int64_t N, int *status, void *work,
                        cudaStream_t st) {
    FlowArgs f;
    memset(&f, 0, sizeof f);
    StepArgs &a = f.st;
    a.n = n;
    a.H = 8;
    a.W = 32 * KC_WIDE - 2 * a.H;
    a.ntiles = (n + a.W - 1) / a.W;
    a.tile0 = 0;
    a.tcount = a.ntiles;
    a.S = 1;
    a.h = h;
    a.hh = 0.5 * h;
    a.h6 = h / 6.0;
    a.one = 1.0;
    a.nzero = -0.0;
    a.status = status;
    f.xlo = xlo;
    f.xhi = xhi;
    f.bufA[0] = lo; f.bufB[0] = hi;
    f.bufA[1] = sA; f.bufB[1] = sB;
    f.N = N;
    f.next = (unsigned long long *)work;
    f.ready = (int *)((char *)work + 16);
    f.wait_ns = 2000000000ULL;   // 2 s: far beyond any tile's step
    REACH_CUDA(cudaMemsetAsync(work, 0, ks_flow_work_bytes(n), st));
    // a resident grid: three 4-warp blocks per SM (the kernel's launch bound)
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(3 * sms);
    if (method == MM) stencil_ks_flow<MM, KC_WIDE><<<grid, 32 * KS_WARPS_PER_BLOCK, 0, st>>>(f, p);
    else stencil_ks_flow<CGB, KC_WIDE><<<grid, 32 * KS_WARPS_PER_BLOCK, 0, st>>>(f, p);
    REACH_LAUNCHED("stencil_ks_flow");
    return REACH_OK;
}

int64_t ks_flow_work_bytes(int64_t n) {
    const int64_t W = 32 * KC_WIDE - 16, T = (n + W - 1) / W;
    return 16 + 4 * T;
}

int stencil_ks(int method, const KsK &p, int64_t n, const double *xlo, const double *xhi, double *lo,
               double *hi, double *sA, double *sB, double h, int64_t N, int S, int *status,
               cudaStream_t st) {
    const int kc = tile_kc(n, 8 * S, 1);
    return run_steps(2, kc, n, xlo, xhi, lo, hi, sA, sB, h, N, S, status, [&](const StepArgs &a) {
        const Shape g = shape_for(a.ntiles, KS_WARPS_PER_BLOCK);
        if (method == MM && kc == KC_NARROW) stencil_ks_rk4<MM, KC_NARROW><<<g.grid, g.threads, 0, st>>>(a, p);
        else if (method == MM) stencil_ks_rk4<MM, KC_WIDE><<<g.grid, g.threads, 0, st>>>(a, p);
        else if (kc == KC_NARROW) stencil_ks_rk4<CGB, KC_NARROW><<<g.grid, g.threads, 0, st>>>(a, p);
        else stencil_ks_rk4<CGB, KC_WIDE><<<g.grid, g.threads, 0, st>>>(a, p);
        REACH_LAUNCHED("stencil_ks_rk4");
        return REACH_OK;
    });
}

}  // namespace reach
