// quad.cuh -- device code of the quadrotor swarm (Sec. 5.2): K independent
// agents of 12 states (p_n, p_e, h, dp_n, dp_e, dh, phi, theta, psi, dphi,
// dtheta, dpsi), torque inputs (tau_phi, tau_theta, tau_psi) per agent, thrust
// F a parameter.  Shared by the MM / CGB kernels (quad.cu) and the Monte Carlo
// kernel (mc.cu).
//
// RK4 of one agent in chain form.  Every row except the three translational
// accelerations is linear: dp = v, dq = w (angles q, rates w), dw = alpha =
// tau / J, constant over a call.  Classic RK4 (Sec. 3.1) of this structure
// needs the accelerations a_1..a_4 at the four stage angle triples
//   q_1 = q,  q_2 = q + h/2 w,  q_3 = q + h/2 (w + h/2 alpha),  q_4 = q + h (w + h/2 alpha),
// and then gives exactly (in exact arithmetic) the classic update
//   v+ = v + h/6 (a_1 + 2 a_2 + 2 a_3 + a_4),  p+ = p + h v + h^2/6 (a_1 + a_2 + a_3),
//   q+ = q + h w + h^2/2 alpha,  w+ = w + h alpha,
// so a step evaluates the trigonometric part four times and carries no stage
// vectors.  The CGB radius follows the same chain with C r_q in place of the
// accelerations and [p] / J in place of alpha.
#pragma once

#include "common.cuh"

namespace reach {

struct QuadK {
    double a;            // F / m
    double g;
    double Jx, Jy, Jz;
};

constexpr double Q_PI = 3.141592653589793;
constexpr double Q_HALF_PI = 1.5707963267948966;
constexpr double Q_TWO_PI = 6.283185307179586;
constexpr double Q_INV_TWO_PI = 0.15915494309189535;

struct Iv {
    double lo, hi;
};

__device__ __forceinline__ Iv iv_add(Iv a, Iv b) { return {a.lo + b.lo, a.hi + b.hi}; }
__device__ __forceinline__ Iv iv_neg(Iv a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ Iv iv_mul(Iv a, Iv b) {
    const double p1 = a.lo * b.lo, p2 = a.lo * b.hi, p3 = a.hi * b.lo, p4 = a.hi * b.hi;
    return {kmin(kmin(p1, p2), kmin(p3, p4)), kmax(kmax(p1, p2), kmax(p3, p4))};
}
// c >= 0 (F / m)
__device__ __forceinline__ Iv iv_scale(double c, Iv a) { return {c * a.lo, c * a.hi}; }
__device__ __forceinline__ double iv_mag(Iv a) { return kmax(kabs(a.lo), kabs(a.hi)); }

constexpr double Q_THREE_HALF_PI = 4.71238898038469;

// Does c + 2 pi k (c in [0, 2 pi)) lie in [a, b] for an integer k: with
// r = a - 2 pi floor(a / 2 pi), where a falls in [0, 2 pi), the first such
// point at or after a lies c - r beyond it (c + 2 pi - r when c < r).  r is
// shared by the four extrema of an interval; products and sums are kept
// separate (no contraction) so that each decision is the one a plain IEEE
// evaluation of the same expressions takes.
__device__ __forceinline__ double turn_position(double a) {
    const double k = floor(__dmul_rn(a, Q_INV_TWO_PI));
    return __dsub_rn(a, __dmul_rn(Q_TWO_PI, k));
}

template <int C_ID>
__device__ __forceinline__ bool holds_point(double r, double w) {
    constexpr double c = C_ID == 0 ? 0.0 : C_ID == 1 ? Q_HALF_PI : C_ID == 2 ? Q_PI : Q_THREE_HALF_PI;
    constexpr double c2 = c + Q_TWO_PI;
    const double d = (c >= r) ? __dsub_rn(c, r) : __dsub_rn(c2, r);
    return d <= w;
}

// ranges of sin and cos over [lo, hi] (lo <= hi) from the endpoint values
// (s0, c0 at lo; s1, c1 at hi), and +-1 where an extremum lies inside:
// sin peaks at pi/2 and 3 pi/2, cos at 0 and pi
__device__ __forceinline__ void iv_sincos_at(double lo, double hi, double s0, double c0, double s1, double c1,
                                             Iv &S, Iv &C) {
    const double w = hi - lo;
    if (w >= Q_TWO_PI) {
        S = {-1.0, 1.0};
        C = {-1.0, 1.0};
        return;
    }
    const double r = turn_position(lo);
    S.lo = holds_point<3>(r, w) ? -1.0 : kmin(s0, s1);
    S.hi = holds_point<1>(r, w) ? 1.0 : kmax(s0, s1);
    C.lo = holds_point<2>(r, w) ? -1.0 : kmin(c0, c1);
    C.hi = holds_point<0>(r, w) ? 1.0 : kmax(c0, c1);
}

// Sines and cosines at the stage angles.  The stage angle q_s = q + d_s lies
// within a small d_s = O(h |w|) of the step-start angle, so its sine and
// cosine follow from the step start's by the angle-addition formulas, with
// sin d and cos d from their Maclaurin series through d^9 and d^10 (for
// |d| <= 1/16 the first omitted terms are below 2e-21 and 1e-23, far under
// the rounding of the result); a larger d falls back to sincos.
constexpr double Q_SMALL = 0.0625;

// steps between fresh sines and cosines of the step-start angles; in between
// a step's values follow from the previous step's by angle addition, which
// bounds the rounding carried from step to step to that many additions
constexpr int64_t QUAD_ANCHOR = 32;

__device__ __forceinline__ void small_sincos(double d, double &s, double &c) {
    const double d2 = d * d;
    const double ps = fma(d2, fma(d2, fma(d2, 2.7557319223985893e-06, -0.0001984126984126984),
                                  0.008333333333333333), -0.16666666666666666);
    s = fma(d * d2, ps, d);
    const double pc = fma(d2, fma(d2, fma(d2, fma(d2, -2.755731922398589e-07, 2.48015873015873e-05),
                                          -0.001388888888888889), 0.041666666666666664), -0.5);
    c = fma(d2, pc, 1.0);
}

// sin and cos of a + d from s0 = sin a, c0 = cos a (ang = a + d as rounded)
__device__ __forceinline__ void shifted_sincos(double ang, double d, double s0, double c0, double &s, double &c) {
    if (kabs(d) <= Q_SMALL) {
        double sd, cd;
        small_sincos(d, sd, cd);
        s = fma(s0, cd, c0 * sd);
        c = fma(c0, cd, -(s0 * sd));
    } else {
        sincos(ang, &s, &c);
    }
}

// binary32: the same with the series through d^7 and d^6 (for |d| <= 1/16 the
// first omitted terms are below 2e-16 and 6e-15, under binary32 rounding)
__device__ __forceinline__ void small_sincos(float d, float &s, float &c) {
    const float d2 = d * d;
    s = fmaf(d * d2, fmaf(d2, fmaf(d2, -1.98412698e-4f, 8.33333333e-3f), -0.166666667f), d);
    c = fmaf(d2, fmaf(d2, fmaf(d2, -1.38888889e-3f, 4.16666667e-2f), -0.5f), 1.0f);
}

__device__ __forceinline__ void shifted_sincos(float ang, float d, float s0, float c0, float &s, float &c) {
    if (fabsf(d) <= (float)Q_SMALL) {
        float sd, cd;
        small_sincos(d, sd, cd);
        s = fmaf(s0, cd, c0 * sd);
        c = fmaf(c0, cd, -(s0 * sd));
    } else {
        sincosf(ang, &s, &c);
    }
}

// the plain accelerations from the sines and cosines of the attitude
template <class T>
__device__ __forceinline__ void quad_acc_trig(const T (&s)[3], const T (&c)[3], T a, T g, T (&acc)[3]) {
    const T cs = c[0] * s[1];
    acc[0] = a * (-(cs * c[2]) - s[0] * s[2]);
    acc[1] = a * (-(cs * s[2]) + s[0] * c[2]);
    acc[2] = g - a * (c[0] * c[1]);
}

// MM: natural interval extension of the accelerations over the hull of the
// two attitudes (ql, qh: the stage angles of the two chains; sl, cl, sh, ch:
// their sines and cosines); the lower chain takes the lower ends, the upper
// chain the upper ends
__device__ __forceinline__ void quad_acc_mm(const double (&ql)[3], const double (&qh)[3], const double (&sl)[3],
                                            const double (&cl)[3], const double (&sh)[3], const double (&ch)[3],
                                            const QuadK &p, double (&al)[3], double (&ah)[3]) {
    Iv S[3], C[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const bool ord = kle(ql[j], qh[j]);
        if (ord) iv_sincos_at(ql[j], qh[j], sl[j], cl[j], sh[j], ch[j], S[j], C[j]);
        else iv_sincos_at(qh[j], ql[j], sh[j], ch[j], sl[j], cl[j], S[j], C[j]);
    }
    const Iv &sf = S[0], &cf = C[0], &st = S[1], &ct = C[1], &sp = S[2], &cp = C[2];
    const Iv cs = iv_mul(cf, st);
    const Iv an = iv_scale(p.a, iv_add(iv_neg(iv_mul(cs, cp)), iv_neg(iv_mul(sf, sp))));
    const Iv ae = iv_scale(p.a, iv_add(iv_neg(iv_mul(cs, sp)), iv_mul(sf, cp)));
    const Iv ac = iv_scale(p.a, iv_mul(cf, ct));
    al[0] = an.lo; ah[0] = an.hi;
    al[1] = ae.lo; ah[1] = ae.hi;
    al[2] = p.g - ac.hi; ah[2] = p.g - ac.lo;
}

// CGB: the center's accelerations (sc, cc: sines and cosines of the center's
// attitude), and C r over the angle rows of the radius, C bounding
// |d acc / d angle| over the box [c - r, c + r] (slo, clo, shi, chi: sines
// and cosines at its ends)
__device__ __forceinline__ void quad_acc_cgb(const double (&qc)[3], const double (&qr)[3], const double (&sc)[3],
                                             const double (&cc)[3], const double (&slo)[3], const double (&clo)[3],
                                             const double (&shi)[3], const double (&chi)[3], const QuadK &p,
                                             double (&ac)[3], double (&ar)[3]) {
    quad_acc_trig<double>(sc, cc, p.a, p.g, ac);
    Iv S[3], C[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        iv_sincos_at(qc[j] - qr[j], qc[j] + qr[j], slo[j], clo[j], shi[j], chi[j], S[j], C[j]);
    const Iv &sf = S[0], &cf = C[0], &st = S[1], &ct = C[1], &sp = S[2], &cp = C[2];
    const Iv sfst = iv_mul(sf, st), cs = iv_mul(cf, st), ccx = iv_mul(cf, ct);
    const double n_f = p.a * iv_mag(iv_add(iv_mul(sfst, cp), iv_neg(iv_mul(cf, sp))));
    const double n_t = p.a * iv_mag(iv_mul(ccx, cp));
    const double n_p = p.a * iv_mag(iv_add(iv_mul(cs, sp), iv_neg(iv_mul(sf, cp))));
    const double e_f = p.a * iv_mag(iv_add(iv_mul(sfst, sp), iv_mul(cf, cp)));
    const double e_t = p.a * iv_mag(iv_mul(ccx, sp));
    const double e_p = p.a * iv_mag(iv_add(iv_neg(iv_mul(cs, cp)), iv_neg(iv_mul(sf, sp))));
    const double h_f = p.a * iv_mag(iv_mul(sf, ct));
    const double h_t = p.a * iv_mag(cs);
    ar[0] = fma(n_f, qr[0], fma(n_t, qr[1], n_p * qr[2]));
    ar[1] = fma(e_f, qr[0], fma(e_t, qr[1], e_p * qr[2]));
    ar[2] = fma(h_f, qr[0], h_t * qr[1]);
}

// one chain of an agent: positions, velocities, angles, rates, angular
// acceleration (constant)
template <class T>
struct QChain {
    T p[3], v[3], q[3], w[3], al[3];
};

// stage angle triple s (0..3) of a chain
template <class T>
__device__ __forceinline__ void stage_angles(const QChain<T> &c, int s, T h, T (&q)[3]) {
    const T hh = T(0.5) * h;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (s == 0) q[j] = c.q[j];
        else if (s == 1) q[j] = c.q[j] + hh * c.w[j];
        else if (s == 2) q[j] = c.q[j] + hh * (c.w[j] + hh * c.al[j]);
        else q[j] = c.q[j] + h * (c.w[j] + hh * c.al[j]);
    }
}

// increment d_s of the stage angles over the step-start angles (d_0 = 0)
template <class T>
__device__ __forceinline__ void stage_deltas(const QChain<T> &c, int s, T h, T (&d)[3]) {
    const T hh = T(0.5) * h;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (s == 0) d[j] = T(0);
        else if (s == 1) d[j] = hh * c.w[j];
        else if (s == 2) d[j] = hh * (c.w[j] + hh * c.al[j]);
        else d[j] = h * (c.w[j] + hh * c.al[j]);
    }
}

// running sums of the stage accelerations: a_1 + 2 a_2 + 2 a_3 + a_4 for the
// velocities and a_1 + a_2 + a_3 for the positions, so that a stage's
// accelerations are dead once added
template <class T>
struct QSums {
    T sv[3], sp[3];
};

template <class T>
__device__ __forceinline__ void add_stage(QSums<T> &m, const T (&a)[3], int s) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (s == 0) {
            m.sv[j] = a[j];
            m.sp[j] = a[j];
        } else if (s == 3) {
            m.sv[j] = m.sv[j] + a[j];
        } else {
            m.sv[j] = m.sv[j] + T(2) * a[j];
            m.sp[j] = m.sp[j] + a[j];
        }
    }
}

// the step update from the summed stage accelerations
template <class T>
__device__ __forceinline__ void chain_update(QChain<T> &c, const QSums<T> &m, T h) {
    const T h6 = h / T(6), hh = T(0.5) * h;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const T v0 = c.v[j];
        c.v[j] = v0 + h6 * m.sv[j];
        c.p[j] = c.p[j] + h * v0 + (h * h6) * m.sp[j];
        c.q[j] = c.q[j] + h * c.w[j] + (h * hh) * c.al[j];
        c.w[j] = c.w[j] + h * c.al[j];
    }
}

}  // namespace reach
