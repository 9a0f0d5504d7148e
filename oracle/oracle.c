/*
 * oracle.c -- plain, slow, single-threaded FP64 reference implementation of
 * the interval reachability methods of PIRK (Devonport, Khaled, Arcak, Zamani:
 * "PIRK: Scalable Interval Reachability Analysis for High-Dimensional
 * Nonlinear Systems", 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The CUDA library
 * neither links nor calls it, and the two share no source, header, table or
 * constant generator.  Build: gcc -O2 -ffp-contract=off -fPIC -shared (no
 * fast-math, no threads, no FMA contraction).
 *
 * Every function below names the passage of the paper it follows.  Where the
 * paper is silent, garbled or inconsistent the reading taken is stated next
 * to the code:
 *
 *  R1 (Sec. 3.1, Algorithm 1).  The printed listing is read as classic
 *     fourth-order Runge-Kutta: the third stage is evaluated at y + h*k3 (the
 *     listing writes h/2), the update carries the factor h, and the loop runs
 *     N = round((t1 - t0)/h) steps (the listing's time set has N+1 elements).
 *     Only this reading is fourth order, which the section title claims.
 *  R2 (Sec. 2.1, CGB; Algorithm 2).  Center and radius are integrated as one
 *     coupled 2n-dimensional system with the same RK4.  When the contraction
 *     matrix C is constant this equals the paper's two sequential runs; when C
 *     is evaluated on the current box (R3) it is the natural reading.
 *  R3 (Sec. 2.1, CGB).  The paper does not say over which domain C must bound
 *     the Jacobian.  Systems with globally valid constant bounds (traffic,
 *     linear) use a constant C; the KS grid and the oscillator chain use the
 *     supremum of the Jacobian over the current stage box [c - r, c + r].
 *  R4 (Sec. 2.1, MC).  The text samples the initial set and the input set;
 *     Algorithm 4 samples only x0.  The text is followed: inputs are sampled
 *     too, once per trajectory and constant in time (Sec. 2).
 *  R5 (Sec. 2.1, MC).  "log" in the sample bound is the natural logarithm.
 *  R6 (Sec. 5.1).  The printed traffic equations are garbled (the first cell
 *     lacks its outflow, indices disagree).  The chain is: cells 0..n-1,
 *     flux out of cell i  f_i = min(c, v x_i, w (xbar - x_{i+1})) for i<n-1,
 *     f_{n-1} = min(c, v x_{n-1}), inflow of cell 0 is the input d, and
 *     dx_i/dt = f_{i-1} - f_i (beta = T = 1).
 *  R7 (Sec. 2.1, MM).  The paper leaves the decomposition function to its
 *     references; each system below documents the one used.
 *  R12 (Sec. 5.4).  Heat diffusion in the unit cube on an l x l x l grid,
 *      spacing dx = 1/l, first-order differences: du_i/dt = alpha/dx^2 times the
 *      sum over the six neighbours of (u_nb - u_i).  Five faces are insulated (a
 *      missing neighbour contributes nothing); the face z = 0 exchanges heat with
 *      an environment at temperature zero (a missing neighbour at z = -1 counts
 *      as u_nb = 0).  The paper does not give alpha, the heated region or the
 *      initial box; they are inputs here.
 *  R14 (Sec. 2.1, CGB; Sec. 5.1).  Optional box-evaluated contraction matrix
 *      for the traffic chain (traffic parameter 5 nonzero): instead of the
 *      bounds valid for every state (C_{i,i-1} = v, C_{i,i+1} = w, C_ii = 0),
 *      C is taken over the current box [c - r, c + r] (as in R3): an
 *      off-diagonal entry keeps v (w) only if the free-flow (congestion)
 *      branch of the flux can be the minimum somewhere in the box, and the
 *      diagonal gets -v (-w) where the free-flow branch of f_i (the
 *      congestion branch of f_{i-1}) is strictly the minimum everywhere in it.
 *  R15 (Sec. 2.1, Sec. 3.1; optional).  Outward-rounded MM and CGB for the
 *      traffic chain (traffic parameter 6 nonzero): the computed box contains
 *      the box the same method (R1, R2, R6) yields in exact real arithmetic
 *      from the same binary64 inputs and step.  Each MM half and the CGB
 *      center are carried as intervals of binary64 numbers that contain the
 *      exact value, every operation rounded outward; the CGB radius has only
 *      nonnegative coefficients, so each of its operations is rounded up.
 *      Directed rounding is computed from round-to-nearest results and their
 *      exact errors (TwoSum: Knuth, TAOCP vol. 2, 4.2.2; the product error by
 *      one fused multiply-add), stepping to the adjacent binary64 number where
 *      the error shows the rounded result on the wrong side.
 *  R13 (Sec. 5.2).  Quadrotor swarm of K = n/12 independent agents.  Agent k
 *      holds x[12k + 0..11] = (p_n, p_e, h, dp_n, dp_e, dh, phi, theta, psi,
 *      dphi, dtheta, dpsi) and inputs p[3k + 0..2] = (tau_phi, tau_theta,
 *      tau_psi); the thrust F is a parameter (hover: F = m g), so the system
 *      is input-affine as CGB requires.  The paper gives no mass, inertia,
 *      thrust or sets; they are inputs here.  MM decomposition: the three
 *      translational accelerations are not monotone in the angles; each takes
 *      the lower end of its natural interval extension over the hull of the
 *      two angle triples when (phi, theta, psi) <= (phi^, theta^, psi^), the
 *      upper end otherwise; every other row is increasing in its argument and
 *      takes its own.  CGB: C bounds |J| over the current box by the natural
 *      interval extension of each partial derivative (R3); C_ii = 0.
 *
 * Random numbers of the MC method come from Philox4x32-10 (Salmon, Moraes,
 * Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3", SC'11),
 * implemented here from that definition.  Sample j, component i, stream tag t
 * uses counter (i, j, t, 0) and key (seed mod 2^32, seed div 2^32); the first
 * two output words w0, w1 give U = ((w0 << 32 | w1) >> 11) * 2^-53 in [0,1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_MM = 0, ORC_CGB = 1, ORC_MC = 2 };
enum { ORC_TRAFFIC = 0, ORC_KS = 1, ORC_OSC = 2, ORC_LINEAR = 3, ORC_HEAT = 4, ORC_QUAD = 5 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ENONFINITE = -4 };

/* ---------------------------------------------------------------------- */
/* System description                                                      */
/* ---------------------------------------------------------------------- */

typedef struct {
    int kind;
    int64_t n;          /* state dimension */
    int64_t nw;         /* input dimension */
    /* traffic (Sec. 5.1): capacity c, free-flow speed v, congestion wave
       speed w, jam density xbar */
    double cap, v, w, xbar;
    int tr_local;       /* CGB with the box-evaluated C (reading R14) */
    int tr_sound;       /* outward-rounded MM / CGB (reading R15) */
    /* KS grid: u_t = -g_nl u u_x - g_2 u_xx - g_4 u_xxxx, spacing dx */
    double dx, g_nl, g_2, g_4;
    double a0, a1, a2;  /* 5-point stencil of -g_2 u_xx - g_4 u_xxxx */
    /* oscillator chain: xdd_i = -ka x_i - kb x_i^3 + kc (x_{i-1} - 2 x_i + x_{i+1}) + w_i */
    double ka, kb, kc;
    /* linear: dx/dt = A x + p, A row-major n x n */
    const double *A;
    /* heat: grid side l, alpha / dx^2, whether the face z = 0 is open */
    int64_t l;
    double kh;
    int open;
    /* quadrotor swarm: mass, gravity, thrust, moments of inertia */
    double qm, qg, qF, Jx, Jy, Jz;
} orc_sys;

static int64_t input_dim(int kind, int64_t n)
{
    switch (kind) {
    case ORC_TRAFFIC: return 1;
    case ORC_KS: return 0;
    case ORC_OSC: return n / 2;
    case ORC_LINEAR: return n;
    case ORC_HEAT: return 0;
    case ORC_QUAD: return n % 12 ? -1 : n / 12 * 3;
    }
    return -1;
}

int64_t orc_input_dim(int kind, int64_t n) { return input_dim(kind, n); }

static int make_sys(orc_sys *s, int kind, const double *prm, const double *A, int64_t n)
{
    memset(s, 0, sizeof *s);
    s->kind = kind;
    s->n = n;
    s->nw = input_dim(kind, n);
    if (n < 1 || s->nw < 0) return ORC_EINVAL;
    switch (kind) {
    case ORC_TRAFFIC:
        s->cap = prm[0]; s->v = prm[1]; s->w = prm[2]; s->xbar = prm[3];
        s->tr_local = prm[4] != 0.0;
        s->tr_sound = prm[5] != 0.0;
        if (s->tr_local && s->tr_sound) return ORC_EINVAL;
        break;
    case ORC_KS: {
        double d2, d4;
        s->dx = prm[0]; s->g_nl = prm[1]; s->g_2 = prm[2]; s->g_4 = prm[3];
        d2 = 1.0 / (s->dx * s->dx);
        d4 = d2 * d2;
        /* -g_2 (u_{i+1} - 2u_i + u_{i-1})/dx^2
           -g_4 (u_{i+2} - 4u_{i+1} + 6u_i - 4u_{i-1} + u_{i-2})/dx^4 */
        s->a0 = 2.0 * s->g_2 * d2 - 6.0 * s->g_4 * d4;
        s->a1 = -s->g_2 * d2 + 4.0 * s->g_4 * d4;
        s->a2 = -s->g_4 * d4;
        break;
    }
    case ORC_OSC:
        if (n % 2) return ORC_EINVAL;
        s->ka = prm[0]; s->kb = prm[1]; s->kc = prm[2];
        break;
    case ORC_LINEAR:
        if (!A) return ORC_EINVAL;
        s->A = A;
        break;
    case ORC_HEAT: {
        /* prm: alpha, l, open (1: the face z = 0 exchanges with zero temperature) */
        double alpha = prm[0], dx;
        s->l = (int64_t)prm[1];
        s->open = prm[2] != 0.0;
        if (s->l < 1 || s->l * s->l * s->l != n) return ORC_EINVAL;
        dx = 1.0 / (double)s->l;
        s->kh = alpha / (dx * dx);
        break;
    }
    case ORC_QUAD:
        /* prm: m, g, F, Jx, Jy, Jz */
        s->qm = prm[0]; s->qg = prm[1]; s->qF = prm[2];
        s->Jx = prm[3]; s->Jy = prm[4]; s->Jz = prm[5];
        if (!(s->qm > 0.0) || !(s->qF >= 0.0) || !(s->Jx > 0.0) || !(s->Jy > 0.0) || !(s->Jz > 0.0))
            return ORC_EINVAL;
        break;
    default:
        return ORC_EINVAL;
    }
    return ORC_OK;
}

static double min2(double a, double b) { return a < b ? a : b; }
static double max2(double a, double b) { return a > b ? a : b; }
static double posp(double a) { return a > 0.0 ? a : 0.0; }
static double negp(double a) { return a < 0.0 ? a : 0.0; }

/* periodic index for the KS grid */
static int64_t wrap(int64_t i, int64_t n) { i %= n; return i < 0 ? i + n : i; }

/* ---------------------------------------------------------------------- */
/* Right-hand sides f(t, x, p)  (Sec. 2: dx/dt = f(t, x, p))               */
/* ---------------------------------------------------------------------- */

/* traffic flux out of cell i (reading R6) */
static double traffic_flux(const orc_sys *s, const double *x, int64_t i)
{
    if (i == s->n - 1) return min2(s->cap, s->v * x[i]);
    return min2(s->cap, min2(s->v * x[i], s->w * (s->xbar - x[i + 1])));
}

static void f_traffic(const orc_sys *s, const double *x, const double *p, double *dx)
{
    for (int64_t i = 0; i < s->n; ++i) {
        double in = (i == 0) ? p[0] : traffic_flux(s, x, i - 1);
        dx[i] = in - traffic_flux(s, x, i);
    }
}

/* KS, second-order central differences on a periodic grid */
static void f_ks(const orc_sys *s, const double *u, double *du)
{
    int64_t n = s->n;
    for (int64_t i = 0; i < n; ++i) {
        double um2 = u[wrap(i - 2, n)], um1 = u[wrap(i - 1, n)];
        double up1 = u[wrap(i + 1, n)], up2 = u[wrap(i + 2, n)];
        double lin = s->a0 * u[i] + s->a1 * (um1 + up1) + s->a2 * (um2 + up2);
        double ux = (up1 - um1) / (2.0 * s->dx);
        du[i] = lin - s->g_nl * u[i] * ux;
    }
}

/* oscillator chain, state [x_1..x_m | v_1..v_m], fixed ends x_0 = x_{m+1} = 0 */
static void f_osc(const orc_sys *s, const double *y, const double *w, double *dy)
{
    int64_t m = s->n / 2;
    const double *x = y, *v = y + m;
    for (int64_t i = 0; i < m; ++i) {
        double xl = (i > 0) ? x[i - 1] : 0.0;
        double xr = (i < m - 1) ? x[i + 1] : 0.0;
        dy[i] = v[i];
        dy[m + i] = -s->ka * x[i] - s->kb * x[i] * x[i] * x[i]
                    + s->kc * (xl - 2.0 * x[i] + xr) + w[i];
    }
}

static void f_linear(const orc_sys *s, const double *x, const double *p, double *dx)
{
    for (int64_t i = 0; i < s->n; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < s->n; ++j) acc += s->A[i * s->n + j] * x[j];
        dx[i] = acc + p[i];
    }
}

/* heat diffusion (reading R12): kh times the sum of (u_nb - u_i) over the
   neighbours that exist, the ghost below z = 0 at zero when the face is open */
static void f_heat(const orc_sys *s, const double *u, double *du)
{
    int64_t l = s->l;
    for (int64_t z = 0; z < l; ++z)
        for (int64_t y = 0; y < l; ++y)
            for (int64_t x = 0; x < l; ++x) {
                int64_t i = x + l * (y + l * z);
                double acc = 0.0;
                if (x > 0) acc += u[i - 1] - u[i];
                if (x < l - 1) acc += u[i + 1] - u[i];
                if (y > 0) acc += u[i - l] - u[i];
                if (y < l - 1) acc += u[i + l] - u[i];
                if (z > 0) acc += u[i - l * l] - u[i];
                else if (s->open) acc += 0.0 - u[i];
                if (z < l - 1) acc += u[i + l * l] - u[i];
                du[i] = s->kh * acc;
            }
}

/* quadrotor swarm (Sec. 5.2, reading R13): the translational accelerations
   of the paper's model, double integrators for position and angles, angular
   accelerations tau / J */
static void f_quad(const orc_sys *s, const double *x, const double *p, double *dx)
{
    double a = s->qF / s->qm;
    for (int64_t k = 0; k < s->n / 12; ++k) {
        const double *y = x + 12 * k, *tau = p + 3 * k;
        double *dy = dx + 12 * k;
        double sf = sin(y[6]), cf = cos(y[6]), st = sin(y[7]), ct = cos(y[7]);
        double sp = sin(y[8]), cp = cos(y[8]);
        dy[0] = y[3];
        dy[1] = y[4];
        dy[2] = y[5];
        dy[3] = a * (-(cf * st * cp) - sf * sp);
        dy[4] = a * (-(cf * st * sp) + sf * cp);
        dy[5] = s->qg - a * (cf * ct);
        dy[6] = y[9];
        dy[7] = y[10];
        dy[8] = y[11];
        dy[9] = tau[0] / s->Jx;
        dy[10] = tau[1] / s->Jy;
        dy[11] = tau[2] / s->Jz;
    }
}

static void f_sys(const orc_sys *s, const double *x, const double *p, double *dx)
{
    switch (s->kind) {
    case ORC_QUAD: f_quad(s, x, p, dx); break;
    case ORC_HEAT: f_heat(s, x, dx); break;
    case ORC_TRAFFIC: f_traffic(s, x, p, dx); break;
    case ORC_KS: f_ks(s, x, dx); break;
    case ORC_OSC: f_osc(s, x, p, dx); break;
    case ORC_LINEAR: f_linear(s, x, p, dx); break;
    }
}

/* ---------------------------------------------------------------------- */
/* Decomposition functions d(t, x, p, xh, ph)  (Sec. 2.1, MM)              */
/* d(x,p,x,p) = f(x,p); d_i nondecreasing in x_j (j != i) and p,           */
/* nonincreasing in xh_j (j != i) and ph.                                  */
/* ---------------------------------------------------------------------- */

/* Traffic is cooperative (every off-diagonal Jacobian entry is >= 0) and
   increasing in the inflow, so d(x, p, xh, ph) = f(x, p). */
static void d_traffic(const orc_sys *s, const double *x, const double *p,
                      const double *xh, const double *ph, double *dx)
{
    (void)xh; (void)ph;
    f_traffic(s, x, p, dx);
}

/* KS: the linear stencil is split by coefficient sign; the product
   -g_nl u_i D_i, D_i = (u_{i+1} - u_{i-1})/(2 dx), is bounded with u_i held at
   its own argument x_i and D_i ranging over the interval its neighbours span:
   Da = (x_{i+1} - xh_{i-1})/(2dx), Db = (xh_{i+1} - x_{i-1})/(2dx).  When x is
   the lower end (Da <= Db) the minimum over that interval is taken, otherwise
   the maximum: this is the tight decomposition of the product on ordered
   boxes, and it reduces to f when xh = x. */
static void d_ks(const orc_sys *s, const double *x, const double *xh, double *dx)
{
    int64_t n = s->n;
    double a1p = posp(s->a1), a1m = negp(s->a1), a2p = posp(s->a2), a2m = negp(s->a2);
    for (int64_t i = 0; i < n; ++i) {
        int64_t im2 = wrap(i - 2, n), im1 = wrap(i - 1, n);
        int64_t ip1 = wrap(i + 1, n), ip2 = wrap(i + 2, n);
        double lin = s->a0 * x[i]
                   + (a1p * x[im1] + a1m * xh[im1]) + (a1p * x[ip1] + a1m * xh[ip1])
                   + (a2p * x[im2] + a2m * xh[im2]) + (a2p * x[ip2] + a2m * xh[ip2]);
        double Da = (x[ip1] - xh[im1]) / (2.0 * s->dx);
        double Db = (xh[ip1] - x[im1]) / (2.0 * s->dx);
        double ea = -s->g_nl * x[i] * Da, eb = -s->g_nl * x[i] * Db;
        double nl = (Da <= Db) ? min2(ea, eb) : max2(ea, eb);
        dx[i] = lin + nl;
    }
}

/* Oscillator: dv_i/dt is decreasing in x_i (an off-diagonal entry for the
   v_i row, slope -ka - 2kc - 3kb x_i^2 < 0) and increasing in x_{i+-1}, v_i
   and w_i; so x_i enters through the hatted argument. */
static void d_osc(const orc_sys *s, const double *y, const double *w,
                  const double *yh, const double *wh, double *dy)
{
    int64_t m = s->n / 2;
    const double *x = y, *v = y + m, *xh = yh;
    (void)wh;
    for (int64_t i = 0; i < m; ++i) {
        double xl = (i > 0) ? x[i - 1] : 0.0;
        double xr = (i < m - 1) ? x[i + 1] : 0.0;
        double z = xh[i];
        dy[i] = v[i];
        dy[m + i] = -s->ka * z - s->kb * z * z * z + s->kc * (xl - 2.0 * z + xr) + w[i];
    }
}

/* Linear: off-diagonal entries split by sign, diagonal at its own argument. */
static void d_linear(const orc_sys *s, const double *x, const double *p,
                     const double *xh, double *dx)
{
    for (int64_t i = 0; i < s->n; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < s->n; ++j) {
            double a = s->A[i * s->n + j];
            if (j == i) acc += a * x[j];
            else acc += posp(a) * x[j] + negp(a) * xh[j];
        }
        dx[i] = acc + p[i];
    }
}

/* Natural interval extensions for the quadrotor (reading R13). */
typedef struct { double lo, hi; } ival;

#define ORC_PI 3.141592653589793
#define ORC_HALF_PI 1.5707963267948966
#define ORC_TWO_PI 6.283185307179586

static ival iv_hull(double a, double b) { ival r = {min2(a, b), max2(a, b)}; return r; }
static ival iv_add(ival a, ival b) { ival r = {a.lo + b.lo, a.hi + b.hi}; return r; }
static ival iv_neg(ival a) { ival r = {-a.hi, -a.lo}; return r; }
static ival iv_mul(ival a, ival b)
{
    double p1 = a.lo * b.lo, p2 = a.lo * b.hi, p3 = a.hi * b.lo, p4 = a.hi * b.hi;
    ival r = {min2(min2(p1, p2), min2(p3, p4)), max2(max2(p1, p2), max2(p3, p4))};
    return r;
}
static ival iv_scale(double c, ival a) { return iv_mul((ival){c, c}, a); }
static double iv_mag(ival a) { return max2(fabs(a.lo), fabs(a.hi)); }

/* does c + 2 pi k lie in [a, b] for some integer k: take the smallest k
   with c + 2 pi k >= a (the first such point at or after a) and test it
   against b.  The quotient only proposes k; the two loops make the
   definition hold for the computed points. */
static int holds_point(double a, double b, double c)
{
    double k = ceil((a - c) / ORC_TWO_PI);
    double p = c + ORC_TWO_PI * k;
    while (p < a) { k += 1.0; p = c + ORC_TWO_PI * k; }
    while (c + ORC_TWO_PI * (k - 1.0) >= a) { k -= 1.0; p = c + ORC_TWO_PI * k; }
    return p <= b;
}

/* range of sin over [a, b]: the endpoints, and +-1 where a maximum
   (pi/2 + 2 pi k) or minimum (-pi/2 + 2 pi k) lies inside */
static ival iv_sin(ival a)
{
    ival r = {-1.0, 1.0};
    double s0, s1;
    if (a.hi - a.lo >= ORC_TWO_PI) return r;
    s0 = sin(a.lo); s1 = sin(a.hi);
    r.lo = holds_point(a.lo, a.hi, -ORC_HALF_PI) ? -1.0 : min2(s0, s1);
    r.hi = holds_point(a.lo, a.hi, ORC_HALF_PI) ? 1.0 : max2(s0, s1);
    return r;
}

/* range of cos over [a, b]: maxima at 2 pi k, minima at pi + 2 pi k */
static ival iv_cos(ival a)
{
    ival r = {-1.0, 1.0};
    double c0, c1;
    if (a.hi - a.lo >= ORC_TWO_PI) return r;
    c0 = cos(a.lo); c1 = cos(a.hi);
    r.lo = holds_point(a.lo, a.hi, ORC_PI) ? -1.0 : min2(c0, c1);
    r.hi = holds_point(a.lo, a.hi, 0.0) ? 1.0 : max2(c0, c1);
    return r;
}

static void d_quad(const orc_sys *s, const double *x, const double *p,
                   const double *xh, const double *ph, double *dx)
{
    double a = s->qF / s->qm;
    (void)ph;
    for (int64_t k = 0; k < s->n / 12; ++k) {
        const double *y = x + 12 * k, *yh = xh + 12 * k, *tau = p + 3 * k;
        double *dy = dx + 12 * k;
        int lower = y[6] <= yh[6] && y[7] <= yh[7] && y[8] <= yh[8];
        ival F = iv_hull(y[6], yh[6]), T = iv_hull(y[7], yh[7]), P = iv_hull(y[8], yh[8]);
        ival sf = iv_sin(F), cf = iv_cos(F), st = iv_sin(T), ct = iv_cos(T);
        ival sp = iv_sin(P), cp = iv_cos(P);
        ival an = iv_scale(a, iv_add(iv_neg(iv_mul(iv_mul(cf, st), cp)), iv_neg(iv_mul(sf, sp))));
        ival ae = iv_scale(a, iv_add(iv_neg(iv_mul(iv_mul(cf, st), sp)), iv_mul(sf, cp)));
        ival ah = iv_add((ival){s->qg, s->qg}, iv_neg(iv_scale(a, iv_mul(cf, ct))));
        dy[0] = y[3];
        dy[1] = y[4];
        dy[2] = y[5];
        dy[3] = lower ? an.lo : an.hi;
        dy[4] = lower ? ae.lo : ae.hi;
        dy[5] = lower ? ah.lo : ah.hi;
        dy[6] = y[9];
        dy[7] = y[10];
        dy[8] = y[11];
        dy[9] = tau[0] / s->Jx;
        dy[10] = tau[1] / s->Jy;
        dy[11] = tau[2] / s->Jz;
    }
}

static void d_sys(const orc_sys *s, const double *x, const double *p,
                  const double *xh, const double *ph, double *dx)
{
    switch (s->kind) {
    case ORC_QUAD: d_quad(s, x, p, xh, ph, dx); break;
    /* heat is linear with nonnegative off-diagonal coefficients (cooperative):
       d(x, p, xh, ph) = f(x) */
    case ORC_HEAT: f_heat(s, x, dx); break;
    case ORC_TRAFFIC: d_traffic(s, x, p, xh, ph, dx); break;
    case ORC_KS: d_ks(s, x, xh, dx); break;
    case ORC_OSC: d_osc(s, x, p, xh, ph, dx); break;
    case ORC_LINEAR: d_linear(s, x, p, xh, dx); break;
    }
}

/* ---------------------------------------------------------------------- */
/* Growth dynamics g(r) = C r + [p]  (Sec. 2.1, CGB)                        */
/* C_ii >= J_ii and C_ij >= |J_ij| (i != j).  c is the current center and  */
/* r the current radius (used only by the box-evaluated bounds, R3).       */
/* ---------------------------------------------------------------------- */

static void g_traffic(const orc_sys *s, const double *c, const double *r,
                      const double *hp, double *dr)
{
    /* dx_i/dx_{i-1} in {0, v}, dx_i/dx_{i+1} in {0, w}, dx_i/dx_i in [-v-w, 0]:
       C_{i,i-1} = v, C_{i,i+1} = w, C_ii = 0, valid for every x.  The inflow
       enters cell 0 with coefficient 1. */
    (void)c;
    for (int64_t i = 0; i < s->n; ++i) {
        double acc = 0.0;
        if (i > 0) acc += s->v * r[i - 1];
        if (i < s->n - 1) acc += s->w * r[i + 1];
        dr[i] = acc + ((i == 0) ? hp[0] : 0.0);
    }
}

/* Reading R14: the traffic flux out of cell j is min(cap, v x_j, w (xbar -
   x_{j+1})) (the last cell has no congestion term).  Over the box
   [lo, hi] = [c - r, c + r], the free-flow branch v x_j can be the minimum
   somewhere iff it can at x_j = lo_j, x_{j+1} = lo_{j+1}, and is strictly the
   minimum everywhere iff it is at hi_j, hi_{j+1}; the congestion branch can
   be the minimum iff it can at hi_j, hi_{j+1}, and is strictly everywhere
   iff it is at lo_j, lo_{j+1}. */
static int tr_ff_possible(const orc_sys *s, const double *lo, int64_t j)
{
    double f = s->v * lo[j];
    if (!(f <= s->cap)) return 0;
    return j == s->n - 1 || f <= s->w * (s->xbar - lo[j + 1]);
}

static int tr_ff_certain(const orc_sys *s, const double *hi, int64_t j)
{
    double f = s->v * hi[j];
    if (!(f < s->cap)) return 0;
    return j == s->n - 1 || f < s->w * (s->xbar - hi[j + 1]);
}

static int tr_cong_possible(const orc_sys *s, const double *hi, int64_t j)
{
    double q;
    if (j == s->n - 1) return 0;
    q = s->w * (s->xbar - hi[j + 1]);
    return q <= s->cap && q <= s->v * hi[j];
}

static int tr_cong_certain(const orc_sys *s, const double *lo, int64_t j)
{
    double q;
    if (j == s->n - 1) return 0;
    q = s->w * (s->xbar - lo[j + 1]);
    return q < s->cap && q < s->v * lo[j];
}

static void g_traffic_local(const orc_sys *s, const double *c, const double *r,
                            const double *hp, double *dr)
{
    int64_t n = s->n;
    double *lo = malloc(sizeof(double) * n), *hi = malloc(sizeof(double) * n);
    if (!lo || !hi) { free(lo); free(hi); for (int64_t i = 0; i < n; ++i) dr[i] = NAN; return; }
    for (int64_t i = 0; i < n; ++i) { lo[i] = c[i] - r[i]; hi[i] = c[i] + r[i]; }
    for (int64_t i = 0; i < n; ++i) {
        double cl = (i > 0 && tr_ff_possible(s, lo, i - 1)) ? s->v : 0.0;
        double cr = tr_cong_possible(s, hi, i) ? s->w : 0.0;
        double cd = 0.0;
        double acc = 0.0;
        if (tr_ff_certain(s, hi, i)) cd -= s->v;
        if (i > 0 && tr_cong_certain(s, lo, i - 1)) cd -= s->w;
        if (i > 0) acc += cl * r[i - 1];
        acc += cd * r[i];
        if (i < n - 1) acc += cr * r[i + 1];
        dr[i] = acc + ((i == 0) ? hp[0] : 0.0);
    }
    free(lo);
    free(hi);
}

static void g_ks(const orc_sys *s, const double *c, const double *r, double *dr)
{
    /* J_ii = a0 - g_nl D_i,  J_{i,i+1} = a1 - g_nl u_i/(2dx),
       J_{i,i-1} = a1 + g_nl u_i/(2dx),  J_{i,i+-2} = a2.
       Suprema over the box u in [c - r, c + r]. */
    int64_t n = s->n;
    double k = s->g_nl / (2.0 * s->dx);
    for (int64_t i = 0; i < n; ++i) {
        int64_t im2 = wrap(i - 2, n), im1 = wrap(i - 1, n);
        int64_t ip1 = wrap(i + 1, n), ip2 = wrap(i + 2, n);
        double lo_i = c[i] - r[i], hi_i = c[i] + r[i];
        /* D_i ranges over [(lo_{i+1} - hi_{i-1}), (hi_{i+1} - lo_{i-1})]/(2dx) */
        double dmin = (c[ip1] - r[ip1]) - (c[im1] + r[im1]);
        double dmax = (c[ip1] + r[ip1]) - (c[im1] - r[im1]);
        double Cii = max2(s->a0 - k * dmin, s->a0 - k * dmax);
        double Cip = max2(fabs(s->a1 - k * lo_i), fabs(s->a1 - k * hi_i));
        double Cim = max2(fabs(s->a1 + k * lo_i), fabs(s->a1 + k * hi_i));
        double C2 = fabs(s->a2);
        dr[i] = Cii * r[i] + Cim * r[im1] + Cip * r[ip1] + C2 * (r[im2] + r[ip2]);
    }
}

static void g_osc(const orc_sys *s, const double *c, const double *r,
                  const double *hp, double *dr)
{
    /* rows x_i: J[x_i, v_i] = 1.  rows v_i: J[v_i, x_i] = -ka - 2kc - 3kb x_i^2,
       J[v_i, x_{i+-1}] = kc, diagonal entries 0. */
    int64_t m = s->n / 2;
    const double *cx = c, *rx = r, *rv = r + m;
    for (int64_t i = 0; i < m; ++i) {
        double amax = fabs(cx[i]) + rx[i];
        double cxx = s->ka + 2.0 * s->kc + 3.0 * s->kb * amax * amax;
        double rl = (i > 0) ? rx[i - 1] : 0.0;
        double rr = (i < m - 1) ? rx[i + 1] : 0.0;
        dr[i] = rv[i];
        dr[m + i] = cxx * rx[i] + fabs(s->kc) * (rl + rr) + hp[i];
    }
}

static void g_linear(const orc_sys *s, const double *r, const double *hp, double *dr)
{
    for (int64_t i = 0; i < s->n; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < s->n; ++j) {
            double a = s->A[i * s->n + j];
            acc += ((j == i) ? a : fabs(a)) * r[j];
        }
        dr[i] = acc + hp[i];
    }
}

/* Quadrotor (reading R13): the only state-dependent Jacobian entries are
   those of the translational accelerations with respect to the angles; each
   is bounded in magnitude over the box [c - r, c + r] by the natural
   interval extension of the partial derivative.  Rows of positions and angles
   have the entry 1 on their velocity; the angular accelerations depend on
   the inputs only, [p] entering as half-width / J. */
static void g_quad(const orc_sys *s, const double *c, const double *r,
                   const double *hp, double *dr)
{
    double a = s->qF / s->qm;
    for (int64_t k = 0; k < s->n / 12; ++k) {
        const double *cc = c + 12 * k, *rr = r + 12 * k, *hw = hp + 3 * k;
        double *d = dr + 12 * k;
        ival F = {cc[6] - rr[6], cc[6] + rr[6]}, T = {cc[7] - rr[7], cc[7] + rr[7]};
        ival P = {cc[8] - rr[8], cc[8] + rr[8]};
        ival sf = iv_sin(F), cf = iv_cos(F), st = iv_sin(T), ct = iv_cos(T);
        ival sp = iv_sin(P), cp = iv_cos(P);
        /* d/dphi, d/dtheta, d/dpsi of a(-cf st cp - sf sp) */
        double n_f = a * iv_mag(iv_add(iv_mul(iv_mul(sf, st), cp), iv_neg(iv_mul(cf, sp))));
        double n_t = a * iv_mag(iv_mul(iv_mul(cf, ct), cp));
        double n_p = a * iv_mag(iv_add(iv_mul(iv_mul(cf, st), sp), iv_neg(iv_mul(sf, cp))));
        /* of a(-cf st sp + sf cp) */
        double e_f = a * iv_mag(iv_add(iv_mul(iv_mul(sf, st), sp), iv_mul(cf, cp)));
        double e_t = a * iv_mag(iv_mul(iv_mul(cf, ct), sp));
        double e_p = a * iv_mag(iv_add(iv_neg(iv_mul(iv_mul(cf, st), cp)), iv_neg(iv_mul(sf, sp))));
        /* of g - a cf ct */
        double h_f = a * iv_mag(iv_mul(sf, ct));
        double h_t = a * iv_mag(iv_mul(cf, st));
        d[0] = rr[3];
        d[1] = rr[4];
        d[2] = rr[5];
        d[3] = n_f * rr[6] + n_t * rr[7] + n_p * rr[8];
        d[4] = e_f * rr[6] + e_t * rr[7] + e_p * rr[8];
        d[5] = h_f * rr[6] + h_t * rr[7];
        d[6] = rr[9];
        d[7] = rr[10];
        d[8] = rr[11];
        d[9] = hw[0] / s->Jx;
        d[10] = hw[1] / s->Jy;
        d[11] = hw[2] / s->Jz;
    }
}

static void g_sys(const orc_sys *s, const double *c, const double *r,
                  const double *hp, double *dr)
{
    switch (s->kind) {
    case ORC_QUAD: g_quad(s, c, r, hp, dr); break;
    /* heat: J = A is Metzler and constant, so C = A and g(r) = A r */
    case ORC_HEAT: (void)c; (void)hp; f_heat(s, r, dr); break;
    case ORC_TRAFFIC:
        if (s->tr_local) g_traffic_local(s, c, r, hp, dr);
        else g_traffic(s, c, r, hp, dr);
        break;
    case ORC_KS: g_ks(s, c, r, dr); break;
    case ORC_OSC: g_osc(s, c, r, hp, dr); break;
    case ORC_LINEAR: g_linear(s, r, hp, dr); break;
    }
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 (Sec. 3.1): fourth-order Runge-Kutta, reading R1           */
/* ---------------------------------------------------------------------- */

typedef void (*rhs_fn)(const void *ctx, double t, const double *y, double *dy);

static int rk4(rhs_fn F, const void *ctx, int64_t dim, double *y,
               double t0, double h, int64_t N)
{
    double *k1 = malloc(sizeof(double) * dim), *k2 = malloc(sizeof(double) * dim);
    double *k3 = malloc(sizeof(double) * dim), *k4 = malloc(sizeof(double) * dim);
    double *tmp = malloc(sizeof(double) * dim);
    if (!k1 || !k2 || !k3 || !k4 || !tmp) {
        free(k1); free(k2); free(k3); free(k4); free(tmp);
        return ORC_ENOMEM;
    }
    for (int64_t k = 0; k < N; ++k) {
        double t = t0 + (double)k * h;
        F(ctx, t, y, k1);
        for (int64_t i = 0; i < dim; ++i) tmp[i] = y[i] + (h / 2.0) * k1[i];
        F(ctx, t + h / 2.0, tmp, k2);
        for (int64_t i = 0; i < dim; ++i) tmp[i] = y[i] + (h / 2.0) * k2[i];
        F(ctx, t + h / 2.0, tmp, k3);
        for (int64_t i = 0; i < dim; ++i) tmp[i] = y[i] + h * k3[i];
        F(ctx, t + h, tmp, k4);
        for (int64_t i = 0; i < dim; ++i)
            y[i] = y[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    free(k1); free(k2); free(k3); free(k4); free(tmp);
    return ORC_OK;
}

/* number of RK4 steps for [0, t_final] with step dt (reading R1) */
int orc_nsteps(double t_final, double dt, int64_t *N)
{
    double q;
    if (!(dt > 0.0) || !(t_final >= 0.0) || !isfinite(dt) || !isfinite(t_final))
        return ORC_EINVAL;
    q = nearbyint(t_final / dt);
    if (fabs(q * dt - t_final) > 1e-9 * t_final) return ORC_EINVAL;
    *N = (int64_t)q;
    return ORC_OK;
}

/* ---- plain system:  dy/dt = f(y, p) ---- */
typedef struct { const orc_sys *s; const double *p; } flow_ctx;

static void flow_rhs(const void *ctx, double t, const double *y, double *dy)
{
    const flow_ctx *c = ctx;
    (void)t;
    f_sys(c->s, y, c->p, dy);
}

/* ---- embedding system (Sec. 2.1):  [x; xh]' = [d(x,p,xh,ph); d(xh,ph,x,p)] ---- */
typedef struct { const orc_sys *s; const double *p, *ph; } mm_ctx;

static void mm_rhs(const void *ctx, double t, const double *z, double *dz)
{
    const mm_ctx *c = ctx;
    int64_t n = c->s->n;
    (void)t;
    d_sys(c->s, z, c->p, z + n, c->ph, dz);
    d_sys(c->s, z + n, c->ph, z, c->p, dz + n);
}

/* ---- center/radius system (Sec. 2.1, R2):  [c; r]' = [f(c,p*); C r + [p]] ---- */
typedef struct { const orc_sys *s; const double *pc, *hp; } cgb_ctx;

static void cgb_rhs(const void *ctx, double t, const double *z, double *dz)
{
    const cgb_ctx *c = ctx;
    int64_t n = c->s->n;
    (void)t;
    f_sys(c->s, z, c->pc, dz);
    g_sys(c->s, z, z + n, c->hp, dz + n);
}

static int all_finite(const double *a, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) if (!isfinite(a[i])) return 0;
    return 1;
}

static int check_box(const double *lo, const double *hi, int64_t n)
{
    if (n > 0 && (!lo || !hi)) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(lo[i]) || !isfinite(hi[i]) || lo[i] > hi[i]) return ORC_EINVAL;
    return ORC_OK;
}

/* one trajectory of f from x0 under constant input p (Sec. 2: Phi(t1; t0, x0, p)) */
int orc_flow(int kind, const double *prm, const double *A, int64_t n,
             const double *x0, const double *p, double t_final, double dt, double *x1)
{
    orc_sys s;
    flow_ctx c;
    int64_t N;
    int rc = make_sys(&s, kind, prm, A, n);
    if (rc) return rc;
    if ((rc = orc_nsteps(t_final, dt, &N))) return rc;
    memcpy(x1, x0, sizeof(double) * n);
    c.s = &s; c.p = p;
    if ((rc = rk4(flow_rhs, &c, n, x1, 0.0, dt, N))) return rc;
    return all_finite(x1, n) ? ORC_OK : ORC_ENONFINITE;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 3: mixed monotonicity.  If pipe_lo is given, the box after    */
/* every `every` steps is written to row q of pipe_lo / pipe_hi (the reach */
/* pipe of Sec. 5.5); otherwise every == N.                                 */
/* ---------------------------------------------------------------------- */
static int reach_mm(const orc_sys *s, const double *xlo, const double *xhi,
                    const double *wlo, const double *whi, double h, int64_t N,
                    int64_t every, double *pipe_lo, double *pipe_hi,
                    double *lo, double *hi)
{
    int64_t n = s->n;
    mm_ctx c;
    int rc = ORC_OK;
    double *z = malloc(sizeof(double) * 2 * n);
    if (!z) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; ++i) { z[i] = xlo[i]; z[n + i] = xhi[i]; }
    c.s = s; c.p = wlo; c.ph = whi;
    for (int64_t done = 0, q = 0; done < N && !rc; done += every, ++q) {
        rc = rk4(mm_rhs, &c, 2 * n, z, (double)done * h, h, every);
        if (!rc && pipe_lo) {
            memcpy(pipe_lo + q * n, z, sizeof(double) * n);
            memcpy(pipe_hi + q * n, z + n, sizeof(double) * n);
        }
    }
    if (!rc) {
        for (int64_t i = 0; i < n; ++i) { lo[i] = z[i]; hi[i] = z[n + i]; }
        if (!all_finite(z, 2 * n)) rc = ORC_ENONFINITE;
    }
    free(z);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 2: contraction / growth bound (pipe output as in reach_mm)     */
/* ---------------------------------------------------------------------- */
static int reach_cgb(const orc_sys *s, const double *xlo, const double *xhi,
                     const double *wlo, const double *whi, double h, int64_t N,
                     int64_t every, double *pipe_lo, double *pipe_hi,
                     double *lo, double *hi)
{
    int64_t n = s->n, nw = s->nw;
    cgb_ctx c;
    int rc = ORC_OK;
    double *z = malloc(sizeof(double) * 2 * n);
    double *pc = malloc(sizeof(double) * (nw > 0 ? nw : 1));
    double *hp = malloc(sizeof(double) * (nw > 0 ? nw : 1));
    if (!z || !pc || !hp) { free(z); free(pc); free(hp); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        z[i] = (xlo[i] + xhi[i]) / 2.0;      /* center, Sec. 2 */
        z[n + i] = (xhi[i] - xlo[i]) / 2.0;  /* half-width */
    }
    for (int64_t k = 0; k < nw; ++k) {
        pc[k] = (wlo[k] + whi[k]) / 2.0;
        hp[k] = (whi[k] - wlo[k]) / 2.0;
    }
    c.s = s; c.pc = pc; c.hp = hp;
    for (int64_t done = 0, q = 0; done < N && !rc; done += every, ++q) {
        rc = rk4(cgb_rhs, &c, 2 * n, z, (double)done * h, h, every);
        if (!rc && pipe_lo) {
            for (int64_t i = 0; i < n; ++i) {
                pipe_lo[q * n + i] = z[i] - z[n + i];
                pipe_hi[q * n + i] = z[i] + z[n + i];
            }
        }
    }
    if (!rc) {
        for (int64_t i = 0; i < n; ++i) { lo[i] = z[i] - z[n + i]; hi[i] = z[i] + z[n + i]; }
        if (!all_finite(z, 2 * n)) rc = ORC_ENONFINITE;
    }
    free(z); free(pc); free(hp);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11)                                     */
/* ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform(uint64_t seed, int64_t j, int64_t i, uint32_t tag)
{
    uint32_t ctr[4] = { (uint32_t)i, (uint32_t)j, tag, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t o[4];
    uint64_t bits;
    orc_philox4x32_10(ctr, key, o);
    bits = ((uint64_t)o[0] << 32) | o[1];
    return (double)(bits >> 11) * 0x1.0p-53;
}

/* Sec. 2.1: m >= (2n/eps) log(2n/delta), natural log (reading R5) */
int64_t orc_mc_samples(int64_t n, double eps, double delta)
{
    double q = 2.0 * (double)n;
    return (int64_t)ceil((q / eps) * log(q / delta));
}

/* ---------------------------------------------------------------------- */
/* Algorithm 4: Monte Carlo.  prec == 32: each sample is rounded to FP32   */
/* (the value an FP32 trajectory starts from) and integrated in FP64.      */
/* finals (optional) receives every sample's final state, row j = sample j. */
/* ---------------------------------------------------------------------- */
static int reach_mc(const orc_sys *s, const double *xlo, const double *xhi,
                    const double *wlo, const double *whi, double h, int64_t N,
                    int64_t m, uint64_t seed, int prec,
                    double *lo, double *hi, double *finals)
{
    int64_t n = s->n, nw = s->nw;
    flow_ctx c;
    int rc = ORC_OK;
    double *x = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * (nw > 0 ? nw : 1));
    if (!x || !p) { free(x); free(p); return ORC_ENOMEM; }
    if (m < 1) { free(x); free(p); return ORC_EINVAL; }
    for (int64_t i = 0; i < n; ++i) { lo[i] = INFINITY; hi[i] = -INFINITY; }
    c.s = s; c.p = p;
    for (int64_t j = 0; j < m && !rc; ++j) {
        for (int64_t i = 0; i < n; ++i) {
            x[i] = xlo[i] + (xhi[i] - xlo[i]) * orc_uniform(seed, j, i, 0u);
            if (prec == 32) x[i] = (double)(float)x[i];
        }
        for (int64_t k = 0; k < nw; ++k) {
            p[k] = wlo[k] + (whi[k] - wlo[k]) * orc_uniform(seed, j, k, 1u);
            if (prec == 32) p[k] = (double)(float)p[k];
        }
        rc = rk4(flow_rhs, &c, n, x, 0.0, h, N);
        if (rc) break;
        if (!all_finite(x, n)) { rc = ORC_ENONFINITE; break; }
        for (int64_t i = 0; i < n; ++i) {
            lo[i] = min2(lo[i], x[i]);
            hi[i] = max2(hi[i], x[i]);
        }
        if (finals) memcpy(finals + j * n, x, sizeof(double) * n);
    }
    free(x); free(p);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Outward rounding (reading R15)                                           */
/* ---------------------------------------------------------------------- */

/* a + b rounded down / up: s = fl(a + b) and its exact error e (TwoSum) */
static double add_dn(double a, double b)
{
    double s = a + b, bb = s - a, e = (a - (s - bb)) + (b - bb);
    return e < 0.0 ? nextafter(s, -INFINITY) : s;
}

static double add_up(double a, double b)
{
    double s = a + b, bb = s - a, e = (a - (s - bb)) + (b - bb);
    return e > 0.0 ? nextafter(s, INFINITY) : s;
}

/* a * b rounded down / up: the error of p = fl(a b) is fma(a, b, -p), exact */
static double mul_dn(double a, double b)
{
    double p = a * b, e = fma(a, b, -p);
    return e < 0.0 ? nextafter(p, -INFINITY) : p;
}

static double mul_up(double a, double b)
{
    double p = a * b, e = fma(a, b, -p);
    return e > 0.0 ? nextafter(p, INFINITY) : p;
}

/* a / b (b > 0) rounded down / up: the remainder a - q b is fma(-q, b, a), exact */
static double div_dn(double a, double b)
{
    double q = a / b, e = fma(-q, b, a);
    return e < 0.0 ? nextafter(q, -INFINITY) : q;
}

static double div_up(double a, double b)
{
    double q = a / b, e = fma(-q, b, a);
    return e > 0.0 ? nextafter(q, INFINITY) : q;
}

/* the interval [ql, qu] times c, for the constant c in [cl, cu], cl >= 0 */
static void imul_pos(double cl, double cu, double ql, double qu, double *rl, double *ru)
{
    *rl = mul_dn(ql >= 0.0 ? cl : cu, ql);
    *ru = mul_up(qu >= 0.0 ? cu : cl, qu);
}

/* interval traffic right-hand side: the flux of R6 with every operation
   rounded outward, inflow [dl, du] */
static void tr_flux_iv(const orc_sys *s, const double *yl, const double *yu, int64_t i,
                       double *fl, double *fu)
{
    double vl = mul_dn(s->v, yl[i]), vu = mul_up(s->v, yu[i]);
    if (i == s->n - 1) {
        *fl = min2(s->cap, vl);
        *fu = min2(s->cap, vu);
        return;
    }
    /* w (xbar - y_{i+1}) is decreasing in y_{i+1} */
    *fl = min2(s->cap, min2(vl, mul_dn(s->w, add_dn(s->xbar, -yu[i + 1]))));
    *fu = min2(s->cap, min2(vu, mul_up(s->w, add_up(s->xbar, -yl[i + 1]))));
}

static void f_traffic_iv(const orc_sys *s, const double *yl, const double *yu, double dl, double du,
                         double *kl, double *ku)
{
    for (int64_t i = 0; i < s->n; ++i) {
        double inl = dl, inu = du, outl, outu;
        if (i > 0) tr_flux_iv(s, yl, yu, i - 1, &inl, &inu);
        tr_flux_iv(s, yl, yu, i, &outl, &outu);
        kl[i] = add_dn(inl, -outu);
        ku[i] = add_up(inu, -outl);
    }
}

/* upper bound of the CGB radius right-hand side C r + [p] (all terms >= 0) */
static void g_traffic_up(const orc_sys *s, const double *r, double hp, double *dr)
{
    for (int64_t i = 0; i < s->n; ++i) {
        double acc = (i == 0) ? hp : 0.0;
        if (i > 0) acc = add_up(acc, mul_up(s->v, r[i - 1]));
        if (i < s->n - 1) acc = add_up(acc, mul_up(s->w, r[i + 1]));
        dr[i] = acc;
    }
}

/* N classic RK4 steps (R1) of the traffic chain on the interval state
   [zl, zu] with inflow [dl, du], all rounded outward.  With zl == NULL only
   the upper end is carried and the right-hand side is the radius bound
   (every quantity nonnegative). */
static int rk4_sound(const orc_sys *s, double *zl, double *zu, double dl, double du, double hp,
                     double h, int64_t N)
{
    int64_t n = s->n;
    const int radius = zl == NULL;
    double hh = 0.5 * h, c6l = div_dn(h, 6.0), c6u = div_up(h, 6.0);
    double *b = malloc(sizeof(double) * 6 * n);
    double *yl, *yu, *kl, *ku, *al, *au;
    if (!b) return ORC_ENOMEM;
    yl = b; yu = b + n; kl = b + 2 * n; ku = b + 3 * n; al = b + 4 * n; au = b + 5 * n;
    for (int64_t step = 0; step < N; ++step) {
        for (int64_t i = 0; i < n; ++i) { yu[i] = zu[i]; if (!radius) yl[i] = zl[i]; }
        for (int stage = 0; stage < 4; ++stage) {
            /* stage weights 1, 2, 2, 1 and stage inputs y + h/2 k, y + h/2 k, y + h k */
            double cs = (stage == 2) ? h : hh;
            if (radius) g_traffic_up(s, yu, hp, ku);
            else f_traffic_iv(s, yl, yu, dl, du, kl, ku);
            for (int64_t i = 0; i < n; ++i) {
                double tl = 0.0, tu;
                if (radius) tu = ku[i];
                else { tl = kl[i]; tu = ku[i]; }
                if (stage == 0) { au[i] = tu; if (!radius) al[i] = tl; }
                else if (stage == 3) { au[i] = add_up(au[i], tu); if (!radius) al[i] = add_dn(al[i], tl); }
                else { au[i] = add_up(au[i], 2.0 * tu); if (!radius) al[i] = add_dn(al[i], 2.0 * tl); }
                if (stage < 3) {
                    yu[i] = add_up(zu[i], mul_up(cs, tu));
                    if (!radius) yl[i] = add_dn(zl[i], mul_dn(cs, tl));
                }
            }
        }
        for (int64_t i = 0; i < n; ++i) {
            double ql, qu;
            /* z + (h/6) acc with h/6 in [c6l, c6u] */
            imul_pos(c6l, c6u, radius ? au[i] : al[i], au[i], &ql, &qu);
            zu[i] = add_up(zu[i], qu);
            if (!radius) zl[i] = add_dn(zl[i], ql);
        }
    }
    free(b);
    return ORC_OK;
}

/* The pieces of R15 one by one, for the pins: a directed operation (op 0..5:
   add, mul, div, each down then up), the constant-interval product, and the
   interval right-hand sides of the traffic chain and of its radius. */
int orc_sound_op(int op, double a, double b, double *out)
{
    switch (op) {
    case 0: *out = add_dn(a, b); return ORC_OK;
    case 1: *out = add_up(a, b); return ORC_OK;
    case 2: *out = mul_dn(a, b); return ORC_OK;
    case 3: *out = mul_up(a, b); return ORC_OK;
    case 4: if (!(b > 0.0)) return ORC_EINVAL; *out = div_dn(a, b); return ORC_OK;
    case 5: if (!(b > 0.0)) return ORC_EINVAL; *out = div_up(a, b); return ORC_OK;
    }
    return ORC_EINVAL;
}

int orc_sound_mul_pos(double cl, double cu, double ql, double qu, double *rl, double *ru)
{
    if (!(cl >= 0.0) || !(cu >= cl)) return ORC_EINVAL;
    imul_pos(cl, cu, ql, qu, rl, ru);
    return ORC_OK;
}

int orc_traffic_sound_rhs(const double *prm, int64_t n, const double *yl, const double *yu,
                          double dl, double du, double *kl, double *ku)
{
    orc_sys s;
    int rc = make_sys(&s, ORC_TRAFFIC, prm, NULL, n);
    if (rc) return rc;
    f_traffic_iv(&s, yl, yu, dl, du, kl, ku);
    return ORC_OK;
}

int orc_traffic_sound_radius_rhs(const double *prm, int64_t n, const double *r, double hp, double *dr)
{
    orc_sys s;
    int rc = make_sys(&s, ORC_TRAFFIC, prm, NULL, n);
    if (rc) return rc;
    g_traffic_up(&s, r, hp, dr);
    return ORC_OK;
}

static int reach_sound(int method, const orc_sys *s, const double *xlo, const double *xhi,
                       const double *wlo, const double *whi, double h, int64_t N,
                       double *lo, double *hi)
{
    int64_t n = s->n;
    int rc = ORC_OK;
    double *z = malloc(sizeof(double) * 3 * n);
    if (!z) return ORC_ENOMEM;
    if (method == ORC_MM) {
        /* the two corner trajectories, each from a point */
        double *l = z, *u = z + n, *t = z + 2 * n;
        memcpy(l, xlo, sizeof(double) * n);
        memcpy(u, xlo, sizeof(double) * n);
        rc = rk4_sound(s, l, u, wlo[0], wlo[0], 0.0, h, N);
        if (!rc) {
            memcpy(lo, l, sizeof(double) * n);
            memcpy(u, xhi, sizeof(double) * n);
            memcpy(t, xhi, sizeof(double) * n);
            rc = rk4_sound(s, t, u, whi[0], whi[0], 0.0, h, N);
            if (!rc) memcpy(hi, u, sizeof(double) * n);
        }
    } else {
        /* center [cl, cu] and radius upper bound ru */
        double *cl = z, *cu = z + n, *ru = z + 2 * n;
        double dcl = 0.5 * add_dn(wlo[0], whi[0]), dcu = 0.5 * add_up(wlo[0], whi[0]);
        double hp = 0.5 * add_up(whi[0], -wlo[0]);
        for (int64_t i = 0; i < n; ++i) {
            cl[i] = 0.5 * add_dn(xlo[i], xhi[i]);
            cu[i] = 0.5 * add_up(xlo[i], xhi[i]);
            ru[i] = 0.5 * add_up(xhi[i], -xlo[i]);
        }
        rc = rk4_sound(s, cl, cu, dcl, dcu, 0.0, h, N);
        if (!rc) rc = rk4_sound(s, NULL, ru, 0.0, 0.0, hp, h, N);
        if (!rc) {
            for (int64_t i = 0; i < n; ++i) {
                lo[i] = add_dn(cl[i], -ru[i]);
                hi[i] = add_up(cu[i], ru[i]);
            }
        }
    }
    if (!rc && (!all_finite(lo, n) || !all_finite(hi, n))) rc = ORC_ENONFINITE;
    free(z);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Entry point                                                              */
/* ---------------------------------------------------------------------- */
int orc_reach(int method, int kind, const double *prm, const double *A, int64_t n,
              const double *x_lo, const double *x_hi,
              const double *w_lo, const double *w_hi,
              double t_final, double dt, int64_t m, uint64_t seed, int prec,
              double *lo, double *hi, double *finals)
{
    orc_sys s;
    int64_t N;
    int rc = make_sys(&s, kind, prm, A, n);
    if (rc) return rc;
    if ((rc = orc_nsteps(t_final, dt, &N))) return rc;
    if ((rc = check_box(x_lo, x_hi, n))) return rc;
    if ((rc = check_box(w_lo, w_hi, s.nw))) return rc;
    if (s.kind == ORC_TRAFFIC && s.tr_sound && (method == ORC_MM || method == ORC_CGB))
        return reach_sound(method, &s, x_lo, x_hi, w_lo, w_hi, dt, N, lo, hi);
    switch (method) {
    case ORC_MM: return reach_mm(&s, x_lo, x_hi, w_lo, w_hi, dt, N, N > 0 ? N : 1, NULL, NULL, lo, hi);
    case ORC_CGB: return reach_cgb(&s, x_lo, x_hi, w_lo, w_hi, dt, N, N > 0 ? N : 1, NULL, NULL, lo, hi);
    case ORC_MC:
        if (prec != 32 && prec != 64) return ORC_EINVAL;
        return reach_mc(&s, x_lo, x_hi, w_lo, w_hi, dt, N, m, seed, prec, lo, hi, finals);
    }
    return ORC_EINVAL;
}

/* The reach pipe (Sec. 5.5): the box after every `every` RK4 steps.
   pipe_lo / pipe_hi receive N/every rows of n values; lo / hi the final box. */
int orc_reach_pipe(int method, int kind, const double *prm, const double *A, int64_t n,
                   const double *x_lo, const double *x_hi,
                   const double *w_lo, const double *w_hi,
                   double t_final, double dt, int64_t every,
                   double *pipe_lo, double *pipe_hi, double *lo, double *hi)
{
    orc_sys s;
    int64_t N;
    int rc = make_sys(&s, kind, prm, A, n);
    if (rc) return rc;
    if ((rc = orc_nsteps(t_final, dt, &N))) return rc;
    if (every < 1 || N % every) return ORC_EINVAL;
    if (s.kind == ORC_TRAFFIC && s.tr_sound) return ORC_EINVAL;   /* R15 covers whole horizons only */
    if ((rc = check_box(x_lo, x_hi, n))) return rc;
    if ((rc = check_box(w_lo, w_hi, s.nw))) return rc;
    if (method == ORC_MM)
        return reach_mm(&s, x_lo, x_hi, w_lo, w_hi, dt, N, every, pipe_lo, pipe_hi, lo, hi);
    if (method == ORC_CGB)
        return reach_cgb(&s, x_lo, x_hi, w_lo, w_hi, dt, N, every, pipe_lo, pipe_hi, lo, hi);
    return ORC_EINVAL;
}

/* ---------------------------------------------------------------------- */
/* Single evaluations of f, d and g, so that tests can check the defining  */
/* properties of Sec. 2.1 (d(x,p,x,p) = f(x,p), monotonicity of d,         */
/* C_ii >= J_ii and C_ij >= |J_ij|) against f directly.                    */
/* ---------------------------------------------------------------------- */
int orc_rhs(int kind, const double *prm, const double *A, int64_t n,
            const double *x, const double *p, double *dx)
{
    orc_sys s;
    int rc = make_sys(&s, kind, prm, A, n);
    if (rc) return rc;
    f_sys(&s, x, p, dx);
    return ORC_OK;
}

int orc_decomp(int kind, const double *prm, const double *A, int64_t n,
               const double *x, const double *p, const double *xh, const double *ph,
               double *dx)
{
    orc_sys s;
    int rc = make_sys(&s, kind, prm, A, n);
    if (rc) return rc;
    d_sys(&s, x, p, xh, ph, dx);
    return ORC_OK;
}

int orc_growth(int kind, const double *prm, const double *A, int64_t n,
               const double *c, const double *r, const double *hp, double *dr)
{
    orc_sys s;
    int rc = make_sys(&s, kind, prm, A, n);
    if (rc) return rc;
    g_sys(&s, c, r, hp, dr);
    return ORC_OK;
}
