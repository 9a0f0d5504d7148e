// quad.cu -- MM and CGB boxes of the quadrotor swarm (Sec. 5.2).
//
// The agents are independent, so one thread integrates one agent's two
// chains (MM: lower and upper corner; CGB: center and radius) over the whole
// horizon in registers: one launch per call, HBM touched only to read the box
// and write the result.  The work is the trigonometric part of the
// accelerations (sines and cosines at each end of three angle intervals per
// stage: a sincos per angle at the step start, the stages by angle addition),
// which makes the kernel bound by the FP64 pipe.
#include "api_internal.cuh"
#include "quad.cuh"

namespace reach {

struct QuadArgs {
    const double *xlo, *xhi, *wlo, *whi;
    double *lo, *hi;
    int64_t K, N;
    double h;
    QuadK p;
    int *status;
};

template <int METHOD>
__global__ void __launch_bounds__(128) quad_box(QuadArgs A) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.K) return;
    const double *xl = A.xlo + 12 * k, *xh = A.xhi + 12 * k, *tl = A.wlo + 3 * k, *th = A.whi + 3 * k;
    const double J[3] = {A.p.Jx, A.p.Jy, A.p.Jz};
    QChain<double> c0, c1;
    int flags = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double l[4] = {xl[j], xl[3 + j], xl[6 + j], xl[9 + j]};
        double u[4] = {xh[j], xh[3 + j], xh[6 + j], xh[9 + j]};
        const double tlo = tl[j], thi = th[j];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (!(kle(l[r], u[r]) && kfinite(l[r]) && kfinite(u[r]))) flags |= ST_BADINPUT;
        if (!(kle(tlo, thi) && kfinite(tlo) && kfinite(thi))) flags |= ST_BADINPUT;
        if (METHOD == MM) {
            c0.p[j] = l[0]; c0.v[j] = l[1]; c0.q[j] = l[2]; c0.w[j] = l[3]; c0.al[j] = tlo / J[j];
            c1.p[j] = u[0]; c1.v[j] = u[1]; c1.q[j] = u[2]; c1.w[j] = u[3]; c1.al[j] = thi / J[j];
        } else {
            c0.p[j] = (l[0] + u[0]) / 2.0; c1.p[j] = (u[0] - l[0]) / 2.0;
            c0.v[j] = (l[1] + u[1]) / 2.0; c1.v[j] = (u[1] - l[1]) / 2.0;
            c0.q[j] = (l[2] + u[2]) / 2.0; c1.q[j] = (u[2] - l[2]) / 2.0;
            c0.w[j] = (l[3] + u[3]) / 2.0; c1.w[j] = (u[3] - l[3]) / 2.0;
            c0.al[j] = ((tlo + thi) / 2.0) / J[j];
            c1.al[j] = ((thi - tlo) / 2.0) / J[j];
        }
    }
    const double h = A.h;
    // sines and cosines at the step start: MM the two chains' attitudes; CGB
    // the center's and the two ends of the angle box.  A step moves each angle
    // by a small increment, so the next step's values follow by angle addition
    // (shifted_sincos); every QUAD_ANCHOR steps they are taken afresh, which
    // bounds the rounding carried from step to step to that many additions
    double sa[3], ca[3], sb[3], cb[3], sx[3], cx[3];
    double pa[3], pb[3], px[3];   // the angles those values belong to
    for (int64_t s = 0; s < A.N; ++s) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double na = METHOD == MM ? c0.q[j] : c0.q[j] - c1.q[j];
            const double nb = METHOD == MM ? c1.q[j] : c0.q[j] + c1.q[j];
            if (s % QUAD_ANCHOR == 0) {
                sincos(na, &sa[j], &ca[j]);
                sincos(nb, &sb[j], &cb[j]);
                if (METHOD == CGB) sincos(c0.q[j], &sx[j], &cx[j]);
            } else {
                double t0 = sa[j], t1 = ca[j];
                shifted_sincos(na, na - pa[j], t0, t1, sa[j], ca[j]);
                t0 = sb[j];
                t1 = cb[j];
                shifted_sincos(nb, nb - pb[j], t0, t1, sb[j], cb[j]);
                if (METHOD == CGB) {
                    t0 = sx[j];
                    t1 = cx[j];
                    shifted_sincos(c0.q[j], c0.q[j] - px[j], t0, t1, sx[j], cx[j]);
                }
            }
            pa[j] = na;
            pb[j] = nb;
            px[j] = c0.q[j];
        }
        QSums<double> m0, m1;
        // stages in a loop: the trigonometric code is large, and unrolling it
        // four times costs registers and instruction cache without adding ILP
#pragma unroll 1
        for (int st = 0; st < 4; ++st) {
            double q0[3], q1[3], d0[3], d1[3], a0[3], a1[3];
            stage_angles(c0, st, h, q0);
            stage_angles(c1, st, h, q1);
            stage_deltas(c0, st, h, d0);
            stage_deltas(c1, st, h, d1);
            double s_a[3], c_a[3], s_b[3], c_b[3];
            if (METHOD == MM) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    shifted_sincos(q0[j], d0[j], sa[j], ca[j], s_a[j], c_a[j]);
                    shifted_sincos(q1[j], d1[j], sb[j], cb[j], s_b[j], c_b[j]);
                }
                quad_acc_mm(q0, q1, s_a, c_a, s_b, c_b, A.p, a0, a1);
            } else {
                double s_x[3], c_x[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    shifted_sincos(q0[j], d0[j], sx[j], cx[j], s_x[j], c_x[j]);
                    shifted_sincos(q0[j] - q1[j], d0[j] - d1[j], sa[j], ca[j], s_a[j], c_a[j]);
                    shifted_sincos(q0[j] + q1[j], d0[j] + d1[j], sb[j], cb[j], s_b[j], c_b[j]);
                }
                quad_acc_cgb(q0, q1, s_x, c_x, s_a, c_a, s_b, c_b, A.p, a0, a1);
            }
            add_stage(m0, a0, st);
            add_stage(m1, a1, st);
        }
        chain_update(c0, m0, h);
        chain_update(c1, m1, h);
    }
    double *lo = A.lo + 12 * k, *hi = A.hi + 12 * k;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double x0[4] = {c0.p[j], c0.v[j], c0.q[j], c0.w[j]};
        const double x1[4] = {c1.p[j], c1.v[j], c1.q[j], c1.w[j]};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double l, u;
            if (METHOD == MM) {
                l = x0[r];
                u = x1[r];
            } else {
                if (dkey(x1[r]) < 0) flags |= ST_NEGRADIUS;
                l = x0[r] - x1[r];
                u = x0[r] + x1[r];
            }
            if (!kfinite(l) || !kfinite(u)) flags |= ST_NONFINITE;
            lo[3 * r + j] = l;
            hi[3 * r + j] = u;
        }
    }
    if (flags) atomicOr(A.status, flags);
}

int quad_run(int method, const QuadK &p, int64_t n, const double *xlo, const double *xhi, const double *wlo,
             const double *whi, double *lo, double *hi, double h, int64_t N, int *status, cudaStream_t st) {
    QuadArgs a;
    a.xlo = xlo; a.xhi = xhi; a.wlo = wlo; a.whi = whi;
    a.lo = lo; a.hi = hi;
    a.K = n / 12;
    a.N = N;
    a.h = h;
    a.p = p;
    a.status = status;
    const unsigned blocks = (unsigned)((a.K + 127) / 128);
    if (method == MM) quad_box<MM><<<blocks, 128, 0, st>>>(a);
    else quad_box<CGB><<<blocks, 128, 0, st>>>(a);
    REACH_LAUNCHED("quad_box");
    return REACH_OK;
}

}  // namespace reach
