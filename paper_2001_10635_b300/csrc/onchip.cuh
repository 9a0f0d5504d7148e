// onchip.cuh -- whole-horizon RK4 of one MM / CGB problem by one thread group
// with the stage vector in shared memory (small and medium n).
//
// The group's threads own components c = cbeg + gt, cbeg + gt + gs, ...; the
// RK4 state z and the stage accumulator live in their registers, the stage
// input y (both halves) in shared memory, and all N steps run without leaving
// the SM: two group barriers per stage (all k computed from y, then y
// rewritten), no global traffic between the first load and the final store.
// The same device code serves one problem per block (reach_mm / reach_cgb on
// small systems) and many problems per block in the batched persistent kernel.
#pragma once

#include "common.cuh"

namespace reach {

constexpr int QMAX = 16;   // components per thread

struct OnItem {
    int64_t n, nw;
    int kind, method;
    const double *xlo, *xhi, *wlo, *whi;
    double *lo, *hi;
    const double *prm;     // device parameters of the system (linear: A, n x n)
    int64_t N;
    double h;
    int *status;
    double one, nzero;     // 1 and -0, read at run time (fadd / fmul)
    double hh, h6;         // h / 2 and h / 6, formed on the host (no binary64 division per stage)
};

// group barrier: a warp syncs itself, a larger group uses a named barrier
struct GroupSync {
    int bar, nthreads;
    __device__ __forceinline__ void operator()() const {
        if (nthreads <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
    }
};

// ---- per-component right-hand sides.  yA / yB: the two halves of the
// embedding (MM: x, xh) or of the center/radius system (CGB: c, r); wA / wB:
// the inputs (MM: w_lo, w_hi; CGB: center, half-width of the input box).

__device__ __forceinline__ double tr_flux_out(const double *y, int64_t i, int64_t n, double cap,
                                              double v, double w, double wxbar, double nz) {
    double cong = (i == n - 1) ? cap : fma(-w, y[i + 1], wxbar);
    return kmin(cap, kmin(fmul(v, y[i], nz), cong));
}

template <int SYS, int METHOD>
__device__ __forceinline__ double onchip_rhs(int64_t c, int64_t n, const double *__restrict__ yA,
                                             const double *__restrict__ yB, const double *wA,
                                             const double *wB, const double *prm, const double (&q)[8]) {
    const bool upper = c >= n;
    const int64_t i = upper ? c - n : c;
    const double one = q[6], nz = q[7];   // 1 and -0 (fadd / fmul)
    if constexpr (SYS == REACH_TRAFFIC) {
        // q: cap, v, w, wxbar, box-evaluated C, xbar
        if (METHOD == CGB && upper && q[4] != 0.0) {
            // radius with C over the stage box [c - r, c + r] (reading R14)
            auto lo = [&](int64_t j) { return __dsub_rn(yA[j], yB[j]); };
            auto hi = [&](int64_t j) { return __dadd_rn(yA[j], yB[j]); };
            auto cong = [&](double x) { return __dmul_rn(q[2], __dsub_rn(q[5], x)); };
            auto ffp = [&](int64_t j) {
                const double f = __dmul_rn(q[1], lo(j));
                return dkey(f) <= dkey(q[0]) && (j == n - 1 || dkey(f) <= dkey(cong(lo(j + 1))));
            };
            auto ffc = [&](int64_t j) {
                const double f = __dmul_rn(q[1], hi(j));
                return dkey(f) < dkey(q[0]) && (j == n - 1 || dkey(f) < dkey(cong(hi(j + 1))));
            };
            auto cgp = [&](int64_t j) {
                if (j == n - 1) return false;
                const double c = cong(hi(j + 1));
                return dkey(c) <= dkey(q[0]) && dkey(c) <= dkey(__dmul_rn(q[1], hi(j)));
            };
            auto cgc = [&](int64_t j) {
                if (j == n - 1) return false;
                const double c = cong(lo(j + 1));
                return dkey(c) < dkey(q[0]) && dkey(c) < dkey(__dmul_rn(q[1], lo(j)));
            };
            const double cl = (i > 0 && ffp(i - 1)) ? q[1] : 0.0;
            const double cr = cgp(i) ? q[2] : 0.0;
            double cd = ffc(i) ? -q[1] : 0.0;
            cd = (i > 0 && cgc(i - 1)) ? cd - q[2] : cd;
            const double left = (i > 0) ? yB[i - 1] : 0.0, right = (i < n - 1) ? yB[i + 1] : 0.0;
            const double v = fma(cl, left, fma(cr, right, cd * yB[i]));
            return (i == 0) ? v + wB[0] : v;
        }
        if (METHOD == MM || !upper) {
            const double *y = upper ? yB : yA;
            double d = upper ? wB[0] : wA[0];
            double fin = (i == 0) ? d : tr_flux_out(y, i - 1, n, q[0], q[1], q[2], q[3], nz);
            return fadd(-tr_flux_out(y, i, n, q[0], q[1], q[2], q[3], nz), fin, one);
        } else {
            double left = (i > 0) ? yB[i - 1] : 0.0;
            double right = (i < n - 1) ? yB[i + 1] : 0.0;
            double v = fma(q[1], left, fmul(q[2], right, nz));
            return (i == 0) ? fadd(v, wB[0], one) : v;
        }
    } else if constexpr (SYS == REACH_KS) {
        // q: a0, a1, a2, k
        const int64_t im1 = i == 0 ? n - 1 : i - 1, ip1 = i == n - 1 ? 0 : i + 1;
        const int64_t im2 = i < 2 ? i + n - 2 : i - 2, ip2 = i >= n - 2 ? i + 2 - n : i + 2;
        const double a0 = q[0], a1 = q[1], a2 = q[2], k = q[3];
        if constexpr (METHOD == MM) {
            // the product term of R7 is q d with q = -k u_i and d the difference
            // at (own_{i+1}, other_{i-1}) when q >= 0, at (other_{i+1}, own_{i-1})
            // otherwise (the stencil kernel's form)
            const double *Y = upper ? yB : yA, *O = upper ? yA : yB;   // own / other half
            const bool s1 = a1 >= 0.0, s2 = a2 >= 0.0;
            double l1 = fadd(s1 ? Y[im1] : O[im1], s1 ? Y[ip1] : O[ip1], one);
            double l2 = fadd(s2 ? Y[im2] : O[im2], s2 ? Y[ip2] : O[ip2], one);
            const double da = fadd(Y[ip1], -O[im1], one), db = fadd(O[ip1], -Y[im1], one);
            const bool qpos = (__double_as_longlong(k) ^ __double_as_longlong(Y[i])) < 0;
            return fma(Y[i], fma(-k, qpos ? da : db, a0), fma(a1, l1, fmul(a2, l2, nz)));
        } else {
            double dc = fadd(yA[ip1], -yA[im1], one);
            const double t = fmul(k, yA[i], nz);
            if (!upper) {
                double lin = fma(a2, fadd(yA[im2], yA[ip2], one), fma(a1, fadd(yA[im1], yA[ip1], one), fmul(a0, yA[i], nz)));
                return fma(-t, dc, lin);
            }
            // C_ii r_i + |k| r_i (r_{i+1} + r_{i-1}) = r_i (a0 - k dc + 2 |k| sr)
            const double ak = kabs(k), sr = fadd(yB[ip1], yB[im1], one);
            const double e = fma(2.0 * ak, sr, fma(-k, dc, a0));
            double acc = fma(kabs(a2), fadd(yB[im2], yB[ip2], one), fmul(e, yB[i], nz));
            acc = fma(kabs(fadd(-t, a1, one)), yB[ip1], acc);
            return fma(kabs(fadd(t, a1, one)), yB[im1], acc);
        }
    } else if constexpr (SYS == REACH_OSC) {
        // q: ka, kb, kc, ka + 2 kc, 3 kb, |kc|;  state [x_1..x_m | v_1..v_m]
        const int64_t m = n >> 1;
        if constexpr (METHOD == MM) {
            const double *Y = upper ? yB : yA, *O = upper ? yA : yB;
            if (i < m) return Y[m + i];
            const int64_t j = i - m;
            double z = O[j];   // x_j enters the v_j row through the hatted argument
            double xl = (j > 0) ? Y[j - 1] : 0.0, xr = (j < m - 1) ? Y[j + 1] : 0.0;
            double w = upper ? wB[j] : wA[j];
            // -(ka + kb z^2) z + kc (xl - 2z + xr) + w = -(ka + 2kc + kb z^2) z + kc (xl + xr) + w
            double t = fma(q[1], fmul(z, z, nz), q[3]);
            double r = fma(q[2], fadd(xl, xr, one), w);
            return fma(-t, z, r);
        } else {
            if (!upper) {
                if (i < m) return yA[m + i];
                const int64_t j = i - m;
                double z = yA[j];
                double xl = (j > 0) ? yA[j - 1] : 0.0, xr = (j < m - 1) ? yA[j + 1] : 0.0;
                double t = fma(q[1], fmul(z, z, nz), q[3]);
                double r = fma(q[2], fadd(xl, xr, one), wA[j]);
                return fma(-t, z, r);
            }
            if (i < m) return yB[m + i];
            const int64_t j = i - m;
            double ax = fadd(kabs(yA[j]), yB[j], one);
            double cxx = fma(fmul(q[4], ax, nz), ax, q[3]);   // ka + 2kc + 3 kb (|c| + r)^2
            double rl = (j > 0) ? yB[j - 1] : 0.0, rr = (j < m - 1) ? yB[j + 1] : 0.0;
            return fma(cxx, yB[j], fma(q[5], fadd(rl, rr, one), wB[j]));
        }
    } else if constexpr (SYS == REACH_HEAT3D) {
        // q: kh, l (integer bits), open face;  both halves (MM: corners, CGB:
        // center and radius, C = A) evolve by the same Metzler operator
        const double *Y = upper ? yB : yA;
        const int l = (int)__double_as_longlong(q[1]), pl = l * l;
        const int ii = (int)i, x = ii % l, y = (ii / l) % l, z = ii / pl;
        double s = (x > 0) ? Y[i - 1] : 0.0;
        s = fadd((x + 1 < l) ? Y[i + 1] : 0.0, s, one);
        s = fadd((y > 0) ? Y[i - l] : 0.0, s, one);
        s = fadd((y + 1 < l) ? Y[i + l] : 0.0, s, one);
        s = fadd((z > 0) ? Y[i - pl] : 0.0, s, one);
        s = fadd((z + 1 < l) ? Y[i + pl] : 0.0, s, one);
        const int m = (x > 0) + (x + 1 < l) + (y > 0) + (y + 1 < l) + (z > 0 || q[2] != 0.0) + (z + 1 < l);
        return fmul(q[0], fma(-(double)m, Y[i], s), nz);
    } else {   // REACH_LINEAR, prm = A row-major
        const double *Arow = prm + i * n;
        double acc = 0.0;
        if constexpr (METHOD == MM) {
            const double *Y = upper ? yB : yA, *O = upper ? yA : yB;
#pragma unroll 1
            for (int64_t j = 0; j < n; ++j) {
                double a = __ldg(Arow + j);
                double v = (j == i || __double_as_longlong(a) >= 0) ? Y[j] : O[j];
                acc = fma(a, v, acc);
            }
            return fadd(acc, upper ? wB[i] : wA[i], one);
        } else {
            if (!upper) {
#pragma unroll 1
                for (int64_t j = 0; j < n; ++j) acc = fma(__ldg(Arow + j), yA[j], acc);
                return fadd(acc, wA[i], one);
            }
#pragma unroll 1
            for (int64_t j = 0; j < n; ++j) {
                double a = __ldg(Arow + j);
                acc = fma(j == i ? a : kabs(a), yB[j], acc);
            }
            return fadd(acc, wB[i], one);
        }
    }
}

template <int SYS>
__device__ __forceinline__ void load_consts(const double *prm, double (&q)[8]) {
#pragma unroll
    for (int t = 0; t < 8; ++t) q[t] = 0.0;
    if constexpr (SYS == REACH_TRAFFIC) {
        q[0] = prm[0]; q[1] = prm[1]; q[2] = prm[2]; q[3] = prm[2] * prm[3];
        q[4] = prm[4]; q[5] = prm[3];
    } else if constexpr (SYS == REACH_KS) {
        q[0] = prm[0]; q[1] = prm[1]; q[2] = prm[2]; q[3] = prm[3];
    } else if constexpr (SYS == REACH_OSC) {
        q[0] = prm[0]; q[1] = prm[1]; q[2] = prm[2];
        q[3] = prm[0] + 2.0 * prm[2]; q[4] = 3.0 * prm[1]; q[5] = kabs(prm[2]);
    } else if constexpr (SYS == REACH_HEAT3D) {
        q[0] = prm[0]; q[1] = __longlong_as_double((long long)prm[1]); q[2] = prm[2];
    }
}

// One RK4 stage of the group.  The stage vector is double-buffered: the
// derivatives are taken from (yA, yB) and the next stage input is written to
// (oA, oB) at once, so a stage needs one barrier and no derivative buffer.
template <int SYS, int METHOD, int STAGE, int Q, class Sync>
__device__ __forceinline__ void onchip_stage(const OnItem &it, const double *yA, const double *yB, double *oA,
                                             double *oB, const double *wA, const double *wB, int64_t cbeg,
                                             int64_t cend, int gt, int gs, const Sync &sync, const double (&q)[8],
                                             double (&z)[Q], double (&acc)[Q]) {
    const int64_t n = it.n;
    const double h = it.h;
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        int64_t c = cbeg + gt + (int64_t)s * gs;
        if (c < cend) {
            const double k = onchip_rhs<SYS, METHOD>(c, n, yA, yB, wA, wB, it.prm, q);
            double y;
            if (STAGE == 0) { acc[s] = k; y = fma(it.hh, k, z[s]); }
            if (STAGE == 1) { acc[s] = fma(2.0, k, acc[s]); y = fma(it.hh, k, z[s]); }
            if (STAGE == 2) { acc[s] = fma(2.0, k, acc[s]); y = fma(h, k, z[s]); }
            if (STAGE == 3) { acc[s] = fadd(k, acc[s], q[6]); z[s] = fma(it.h6, acc[s], z[s]); y = z[s]; }
            (c < n ? oA[c] : oB[c - n]) = y;
        }
    }
    sync();
}

// Integrate one problem.  (yA, yB) and (yA2, yB2): the two stage buffers, n
// doubles per half (the halves may live in different blocks of a cluster);
// wA, wB: nw doubles each.  The calling threads own components [cbeg, cend)
// with stride gs starting at cbeg + gt, at most Q each (Q is a template
// parameter so that small problems run a small loop: the code of a 16-slot
// loop does not fit a lone warp's instruction cache).  The final state is in
// (yA, yB).
template <int SYS, int METHOD, int Q, class Sync>
__device__ void onchip_run(const OnItem &it, double *yA, double *yB, double *yA2, double *yB2, double *wA,
                           double *wB, int64_t cbeg, int64_t cend, int gt, int gs, const Sync &sync) {
    const int64_t n = it.n;
    double q[8];
    load_consts<SYS>(it.prm, q);
    q[6] = it.one;
    q[7] = it.nzero;
    int flags = 0;

    // inputs: MM takes (w_lo, w_hi), CGB (center, half-width)
    if (cbeg == 0) {
        for (int64_t k = gt; k < it.nw; k += gs) {
            double lo = it.wlo[k], hi = it.whi[k];
            if (!(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
            wA[k] = (METHOD == CGB) ? 0.5 * (lo + hi) : lo;
        }
    }
    if (cend == 2 * n) {
        for (int64_t k = gt; k < it.nw; k += gs) {
            double lo = it.wlo[k], hi = it.whi[k];
            wB[k] = (METHOD == CGB) ? 0.5 * (hi - lo) : hi;
        }
    }

    double z[Q], acc[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        int64_t c = cbeg + gt + (int64_t)s * gs;
        z[s] = 0.0;
        acc[s] = 0.0;
        if (c < cend) {
            int64_t i = c < n ? c : c - n;
            double lo = it.xlo[i], hi = it.xhi[i];
            if (c < n && !(lo <= hi && isfinite(lo) && isfinite(hi))) flags |= ST_BADINPUT;
            double v;
            if (METHOD == CGB) v = (c < n) ? 0.5 * (lo + hi) : 0.5 * (hi - lo);
            else v = (c < n) ? lo : hi;
            z[s] = v;
            (c < n ? yA[c] : yB[c - n]) = v;
        }
    }
    sync();

    for (int64_t step = 0; step < it.N; ++step) {
        onchip_stage<SYS, METHOD, 0, Q>(it, yA, yB, yA2, yB2, wA, wB, cbeg, cend, gt, gs, sync, q, z, acc);
        onchip_stage<SYS, METHOD, 1, Q>(it, yA2, yB2, yA, yB, wA, wB, cbeg, cend, gt, gs, sync, q, z, acc);
        onchip_stage<SYS, METHOD, 2, Q>(it, yA, yB, yA2, yB2, wA, wB, cbeg, cend, gt, gs, sync, q, z, acc);
        onchip_stage<SYS, METHOD, 3, Q>(it, yA2, yB2, yA, yB, wA, wB, cbeg, cend, gt, gs, sync, q, z, acc);
    }

    // y holds the final state of both halves
    for (int64_t c = cbeg + gt; c < cend; c += gs) {
        if (c >= n) continue;
        double a = yA[c], b = yB[c];
        double lo = a, hi = b;
        if (METHOD == CGB) {
            if (dkey(b) < 0) flags |= ST_NEGRADIUS;
            lo = a - b;
            hi = a + b;
        }
        if (!kfinite(lo) || !kfinite(hi)) flags |= ST_NONFINITE;
        it.lo[c] = lo;
        it.hi[c] = hi;
    }
    if (flags) atomicOr(it.status, flags);
}

}  // namespace reach
