// stencil.cu -- streaming RK4 kernel for large stencil systems (traffic
// chain, periodic KS grid), mixed monotonicity and growth bound.
//
// Algorithm 1 of the paper runs the four RK4 stages as four parallel sections
// with a synchronisation (a kernel launch) between them and k0..k3, tmp in
// global memory.  Here one launch performs S whole RK4 steps: every warp owns a
// tile of 32*KC consecutive cells of both state halves in registers, neighbour
// values cross lanes by warp shuffles, and the stencil halo of 4*R*S cells per
// side is recomputed redundantly instead of synchronised.  The state is read
// once and written once per launch (16 B per component-step at S = 1).
//
// State halves: MM  A = x (lower), B = xh (upper)        (Sec. 2.1, Alg. 3)
//               CGB A = c (center), B = r (half-width)    (Sec. 2.1, Alg. 2)
#include <stdint.h>

#include "common.cuh"

namespace reach {

constexpr int KC = 8;                 // cells per lane
constexpr int TILE = 32 * KC;         // cells per warp tile
constexpr int WARPS_PER_BLOCK = 8;

struct StepArgs {
    const double *inA, *inB;   // state (or the input box on the first launch)
    double *outA, *outB;
    int64_t n;
    int64_t W;                 // owned cells per tile = TILE - 2H
    int H;                     // halo cells per side = 4 R S
    int S;                     // RK4 steps in this launch
    double h;
    int first, last;           // convert the input box / emit the output box
    int *status;
};

// ------------------------------------------------------------------ helpers
template <int R>
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

// ------------------------------------------------------------------ traffic
// flux out of cell g (reading R6 of the oracle header: f_{-1} = d inflow,
// f_{n-1} = min(cap, v x), cells outside [0, n) carry no flux)
__device__ __forceinline__ double traffic_flux(const TrafficK &p, double y, double yr, int64_t g,
                                               int64_t n, double d) {
    double f = fmin(p.cap, fmin(p.v * y, fma(-p.w, yr, p.wxbar)));
    double flast = fmin(p.cap, p.v * y);
    f = (g == n - 1) ? flast : f;
    f = (g == -1) ? d : f;
    f = (g < -1 || g >= n) ? 0.0 : f;
    return f;
}

// k[j] = f_{g-1} - f_g for the KC cells of this lane
__device__ __forceinline__ void traffic_rhs(const TrafficK &p, const double (&y)[KC], int64_t g0,
                                            int64_t n, double d, double (&k)[KC]) {
    double e[KC + 2];
    exchange<1>(y, e);
    double f[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) f[j] = traffic_flux(p, e[1 + j], e[2 + j], g0 + j, n, d);
    double fl = __shfl_up_sync(0xffffffffu, f[KC - 1], 1);
    // the flux into the lane's first cell: computed by lane-1, except that the
    // domain inflow is known here without it
    fl = (g0 == 0) ? d : fl;
#pragma unroll
    for (int j = 0; j < KC; ++j) k[j] = (j == 0 ? fl : f[j - 1]) - f[j];
}

// radius dynamics (Mr)_g = v r_{g-1} + w r_{g+1} + [d] at g = 0
__device__ __forceinline__ void traffic_growth(const TrafficK &p, const double (&r)[KC], int64_t g0,
                                               int64_t n, double (&k)[KC]) {
    double e[KC + 2];
    exchange<1>(r, e);
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        int64_t g = g0 + j;
        double left = (g > 0) ? e[j] : 0.0;
        double right = (g < n - 1) ? e[2 + j] : 0.0;
        double v = fma(p.v, left, p.w * right);
        k[j] = (g == 0) ? v + p.d_r : v;
    }
}

// ------------------------------------------------------------------ KS
// MM embedding (oracle d_ks): linear stencil split by coefficient sign, the
// product -g_nl u_i u_x bounded with u_i at its own argument.
__device__ __forceinline__ void ks_mm_rhs(const KsK &p, const double (&x)[KC], const double (&xh)[KC],
                                          double (&kx)[KC], double (&kxh)[KC]) {
    double X[KC + 4], XH[KC + 4];
    exchange<2>(x, X);
    exchange<2>(xh, XH);
    const bool s1 = p.a1 >= 0.0, s2 = p.a2 >= 0.0;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        const int c = j + 2;
        // lower: nonnegative coefficients take x, negative ones xh
        double l1 = (s1 ? X[c - 1] : XH[c - 1]) + (s1 ? X[c + 1] : XH[c + 1]);
        double l2 = (s2 ? X[c - 2] : XH[c - 2]) + (s2 ? X[c + 2] : XH[c + 2]);
        double u1 = (s1 ? XH[c - 1] : X[c - 1]) + (s1 ? XH[c + 1] : X[c + 1]);
        double u2 = (s2 ? XH[c - 2] : X[c - 2]) + (s2 ? XH[c + 2] : X[c + 2]);
        double linl = fma(p.a2, l2, fma(p.a1, l1, p.a0 * X[c]));
        double linu = fma(p.a2, u2, fma(p.a1, u1, p.a0 * XH[c]));
        double dL = X[c + 1] - XH[c - 1];   // 2dx * D at (x_{i+1}, xh_{i-1})
        double dH = XH[c + 1] - X[c - 1];   // 2dx * D at (xh_{i+1}, x_{i-1})
        double ql = -p.k * X[c], qu = -p.k * XH[c];
        double ea = ql * dL, eb = ql * dH;
        double fa = qu * dH, fb = qu * dL;
        double nll = (dL <= dH) ? fmin(ea, eb) : fmax(ea, eb);
        double nlu = (dH <= dL) ? fmin(fa, fb) : fmax(fa, fb);
        kx[j] = linl + nll;
        kxh[j] = linu + nlu;
    }
}

// CGB: center f(c) and radius C(c, r) r with C the supremum of the Jacobian
// over the box [c - r, c + r] (reading R3 of the oracle header)
__device__ __forceinline__ void ks_cgb_rhs(const KsK &p, const double (&cc)[KC], const double (&rr)[KC],
                                           double (&kc)[KC], double (&kr)[KC]) {
    double C[KC + 4], Rr[KC + 4];
    exchange<2>(cc, C);
    exchange<2>(rr, Rr);
    const double aa2 = fabs(p.a2);
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        const int c = j + 2;
        double dc = C[c + 1] - C[c - 1];
        double lin = fma(p.a2, C[c - 2] + C[c + 2], fma(p.a1, C[c - 1] + C[c + 1], p.a0 * C[c]));
        kc[j] = fma(-p.k * C[c], dc, lin);
        double sr = Rr[c + 1] + Rr[c - 1];
        double cii = fmax(fma(-p.k, dc - sr, p.a0), fma(-p.k, dc + sr, p.a0));
        double t = p.k * C[c], u = fabs(p.k * Rr[c]);
        double cip = fabs(p.a1 - t) + u;   // sup |a1 - k u_i| over the box
        double cim = fabs(p.a1 + t) + u;   // sup |a1 + k u_i|
        kr[j] = fma(aa2, Rr[c - 2] + Rr[c + 2], fma(cip, Rr[c + 1], fma(cim, Rr[c - 1], cii * Rr[c])));
    }
}

// ------------------------------------------------------------------ kernel
template <int SYS, int METHOD>
struct SysTraits;
template <int METHOD>
struct SysTraits<REACH_TRAFFIC, METHOD> { static constexpr int R = 1; static constexpr bool periodic = false; using P = TrafficK; };
template <int METHOD>
struct SysTraits<REACH_KS, METHOD> { static constexpr int R = 2; static constexpr bool periodic = true; using P = KsK; };

template <int SYS, int METHOD>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK)
stencil_rk4(StepArgs a, typename SysTraits<SYS, METHOD>::P p) {
    constexpr bool periodic = SysTraits<SYS, METHOD>::periodic;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
    const int64_t n = a.n;
    const int64_t ntiles = (n + a.W - 1) / a.W;
    const double h = a.h, hh = 0.5 * a.h, h6 = a.h / 6.0;
    int flags = 0;

    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int64_t start = t * a.W - a.H;
        const int64_t g0 = start + (int64_t)lane * KC;
        double zA[KC], zB[KC];
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            int64_t g = g0 + j;
            bool in = g >= 0 && g < n;
            int64_t idx = g;
            if (periodic) { idx = ((g % n) + n) % n; in = true; }
            double va = in ? __ldg(a.inA + idx) : 0.0;
            double vb = in ? __ldg(a.inB + idx) : 0.0;
            if (a.first) {
                bool owned = g >= t * a.W && g < t * a.W + a.W && g < n && g >= 0;
                if (owned && !(va <= vb && isfinite(va) && isfinite(vb))) flags |= ST_BADINPUT;
                if (METHOD == CGB) {
                    double c = 0.5 * (va + vb), r = 0.5 * (vb - va);
                    va = c; vb = r;
                }
            }
            zA[j] = va;
            zB[j] = vb;
        }

        for (int s = 0; s < a.S; ++s) {
            double yA[KC], yB[KC], aA[KC], aB[KC];
#pragma unroll
            for (int j = 0; j < KC; ++j) { yA[j] = zA[j]; yB[j] = zB[j]; }
#pragma unroll 1
            for (int stage = 0; stage < 4; ++stage) {
                double kA[KC], kB[KC];
                if constexpr (SYS == REACH_TRAFFIC) {
                    if constexpr (METHOD == MM) {
                        traffic_rhs(p, yA, g0, n, p.d_lo, kA);
                        traffic_rhs(p, yB, g0, n, p.d_hi, kB);
                    } else {
                        traffic_rhs(p, yA, g0, n, p.d_c, kA);
                        traffic_growth(p, yB, g0, n, kB);
                    }
                } else {
                    if constexpr (METHOD == MM) ks_mm_rhs(p, yA, yB, kA, kB);
                    else ks_cgb_rhs(p, yA, yB, kA, kB);
                }
                const double cst = (stage == 2) ? h : hh;
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    if (stage == 0) { aA[j] = kA[j]; aB[j] = kB[j]; }
                    else if (stage < 3) { aA[j] = fma(2.0, kA[j], aA[j]); aB[j] = fma(2.0, kB[j], aB[j]); }
                    else { aA[j] += kA[j]; aB[j] += kB[j]; }
                    if (stage < 3) { yA[j] = fma(cst, kA[j], zA[j]); yB[j] = fma(cst, kB[j], zB[j]); }
                    else { zA[j] = fma(h6, aA[j], zA[j]); zB[j] = fma(h6, aB[j], zB[j]); }
                }
            }
        }
        (void)h;

#pragma unroll
        for (int j = 0; j < KC; ++j) {
            int64_t g = g0 + j;
            bool owned = g >= t * a.W && g < t * a.W + a.W && g < n && g >= 0;
            if (!owned) continue;
            double oa = zA[j], ob = zB[j];
            if (a.last) {
                if (METHOD == CGB) {
                    if (ob < 0.0) flags |= ST_NEGRADIUS;
                    double lo = oa - ob, hi = oa + ob;
                    oa = lo; ob = hi;
                }
                if (!isfinite(oa) || !isfinite(ob)) flags |= ST_NONFINITE;
            }
            a.outA[g] = oa;
            a.outB[g] = ob;
        }
    }
    if (flags) atomicOr(a.status, flags);
}

// ------------------------------------------------------------------ host
int stencil_tile_owned(int R, int S) { return TILE - 2 * 4 * R * S; }

template <int SYS, int METHOD, class P>
static int launch_one(const StepArgs &a, const P &p, cudaStream_t st) {
    int64_t ntiles = (a.n + a.W - 1) / a.W;
    int64_t blocks = (ntiles + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    int64_t cap = 148LL * 64;
    if (blocks > cap) blocks = cap;
    stencil_rk4<SYS, METHOD><<<(unsigned)blocks, 32 * WARPS_PER_BLOCK, 0, st>>>(a, p);
    REACH_LAUNCHED("stencil_rk4");
    return REACH_OK;
}

// Integrate N steps with S steps per launch.  in: the input box; out: the
// output box; scratch: 2n doubles (ping-pong partner of out).
template <int SYS, int METHOD, class P>
static int run_stencil(const P &p, int64_t n, const double *xlo, const double *xhi, double *lo,
                       double *hi, double *scratchA, double *scratchB, double h, int64_t N, int S,
                       int *status, cudaStream_t st) {
    constexpr int R = SysTraits<SYS, METHOD>::R;
    int64_t L = (N + S - 1) / S;
    double *bufA[2] = {lo, scratchA}, *bufB[2] = {hi, scratchB};
    int64_t done = 0;
    for (int64_t q = 0; q < L; ++q) {
        int s = (int)((N - done) < S ? (N - done) : S);
        StepArgs a;
        a.n = n;
        a.H = 4 * R * s;
        a.W = TILE - 2 * a.H;
        a.S = s;
        a.h = h;
        a.first = (q == 0);
        a.last = (q == L - 1);
        a.inA = (q == 0) ? xlo : bufA[(L - q) % 2];
        a.inB = (q == 0) ? xhi : bufB[(L - q) % 2];
        a.outA = bufA[(L - 1 - q) % 2];
        a.outB = bufB[(L - 1 - q) % 2];
        a.status = status;
        int rc = launch_one<SYS, METHOD>(a, p, st);
        if (rc) return rc;
        done += s;
    }
    return REACH_OK;
}

int stencil_traffic(int method, const TrafficK &p, int64_t n, const double *xlo, const double *xhi,
                    double *lo, double *hi, double *sA, double *sB, double h, int64_t N, int S,
                    int *status, cudaStream_t st) {
    if (method == MM) return run_stencil<REACH_TRAFFIC, MM>(p, n, xlo, xhi, lo, hi, sA, sB, h, N, S, status, st);
    return run_stencil<REACH_TRAFFIC, CGB>(p, n, xlo, xhi, lo, hi, sA, sB, h, N, S, status, st);
}

int stencil_ks(int method, const KsK &p, int64_t n, const double *xlo, const double *xhi, double *lo,
               double *hi, double *sA, double *sB, double h, int64_t N, int S, int *status,
               cudaStream_t st) {
    if (method == MM) return run_stencil<REACH_KS, MM>(p, n, xlo, xhi, lo, hi, sA, sB, h, N, S, status, st);
    return run_stencil<REACH_KS, CGB>(p, n, xlo, xhi, lo, hi, sA, sB, h, N, S, status, st);
}

}  // namespace reach
