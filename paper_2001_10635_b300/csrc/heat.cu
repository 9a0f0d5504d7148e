// heat.cu -- RK4 of the 3-D heat-diffusion grid (Sec. 5.4) for MM and CGB.
//
// The system is linear with nonnegative off-diagonal coefficients, so MM's two
// halves (lower and upper corner) and CGB's two halves (center and radius,
// C = A) are each integrated with the same operator and do not interact.  For
// a linear autonomous system one classic RK4 step is the polynomial
//   x+ = (I + hA + (hA)^2/2 + (hA)^3/6 + (hA)^4/24) x,
// evaluated here in nested (Horner) form, y1 = x + (h/4) A x,
// y2 = x + (h/3) A y1, y3 = x + (h/2) A y2, x+ = x + h A y3: the same step in
// exact arithmetic, with four operator applications but no accumulator, so a
// step moves 11 state vectors instead of 17 and costs 28 FP64 operations per
// component instead of 31.  One launch applies one stage to both halves: the
// 7-point stencil is the sum of the present neighbours minus their count
// times the cell (an open face z = 0 adds one count for its zero-temperature
// ghost), scaled by alpha / dx^2, which is folded into the stage coefficient.
// Neighbour values come through L1/L2 (the planes above and below a block's
// plane were loaded by the blocks of the neighbouring planes).  The kernels
// are bound by the FP64 pipe; index arithmetic stays in 32-bit or
// 32 x 32 -> 64-bit products (wide integer multiplies and divisions use the
// FP64 pipe of this GPU).
#include "api_internal.cuh"

namespace reach {

// neighbour count m as a double, without an int -> double conversion
__constant__ double c_count[8] = {0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0};

struct HeatArgs {
    const double *in;    // stage input, both halves (2n)
    const double *x;     // state at the start of the step (2n)
    double *out;         // next stage input, or the new state after the last stage (2n)
    uint32_t l, plane;   // l, l * l
    int64_t n;
    double c;            // stage coefficient: kh h / 4, kh h / 3, kh h / 2, kh h
    int open;
};

// FIRST: the stage input is the state itself (no second read of x)
template <bool FIRST>
__global__ void __launch_bounds__(256) heat_stage(HeatArgs a) {
    const uint32_t x = blockIdx.x * 32 + threadIdx.x;
    const uint32_t y = blockIdx.y * 8 + threadIdx.y;
    const uint32_t zz = blockIdx.z;                 // plane of both halves: half * l + z
    const uint32_t half = zz >= a.l ? 1u : 0u;
    const uint32_t z = zz - half * a.l;
    if (x >= a.l || y >= a.l) return;
    const int64_t i = (half ? a.n : 0) + (int64_t)((uint64_t)z * a.plane) + (int64_t)(y * a.l + x);
    const double *u = a.in;
    const double ui = u[i];
    // neighbour sum: the first term is a select, so an interior cell takes
    // five FP64 additions
    double s = (x > 0) ? u[i - 1] : 0.0;
    int m = (x > 0) + (x + 1 < a.l) + (y > 0) + (y + 1 < a.l) + (z > 0 || a.open) + (z + 1 < a.l);
    s += (x + 1 < a.l) ? u[i + 1] : 0.0;
    s += (y > 0) ? u[i - a.l] : 0.0;
    s += (y + 1 < a.l) ? u[i + a.l] : 0.0;
    s += (z > 0) ? u[i - a.plane] : 0.0;          // z = 0 on an open face: ghost at temperature zero
    s += (z + 1 < a.l) ? u[i + a.plane] : 0.0;
    // (A u)_i / kh
    const double d = fma(-c_count[m], ui, s);
    a.out[i] = fma(a.c, d, FIRST ? ui : a.x[i]);
}

// the box to the state: MM (lo, hi); CGB ((lo + hi)/2, (hi - lo)/2)
__global__ void heat_init(const double *xlo, const double *xhi, double *z, int64_t n, int cgb, int *status) {
    int flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double lo = xlo[i], hi = xhi[i];
        if (!(kle(lo, hi) && kfinite(lo) && kfinite(hi))) flags |= ST_BADINPUT;
        z[i] = cgb ? 0.5 * (lo + hi) : lo;
        z[n + i] = cgb ? 0.5 * (hi - lo) : hi;
    }
    if (flags) atomicOr(status, flags);
}

// the state to the box
__global__ void heat_box(const double *z, double *lo, double *hi, int64_t n, int cgb, int *status) {
    int flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = z[i], b = z[n + i];
        if (cgb && dkey(b) < 0) flags |= ST_NEGRADIUS;
        const double l = cgb ? a - b : a, u = cgb ? a + b : b;
        if (!kfinite(l) || !kfinite(u)) flags |= ST_NONFINITE;
        lo[i] = l;
        hi[i] = u;
    }
    if (flags) atomicOr(status, flags);
}

int heat_run(int method, const HeatK &p, int64_t n, const double *xlo, const double *xhi, double *lo, double *hi,
             double h, int64_t N, Staging &sg) {
    if (p.l > 65535 / 2 && N > 0) return REACH_EINVAL;   // grid z holds both halves' planes
    double *X, *Y, *Y2;
    int rc;
    if ((rc = sg.scratch(6 * n * sizeof(double), (void **)&X))) return rc;
    Y = X + 2 * n;
    Y2 = Y + 2 * n;
    const int cgb = method == CGB;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    heat_init<<<(unsigned)blocks, 256, 0, sg.st>>>(xlo, xhi, X, n, cgb, sg.status);
    REACH_LAUNCHED("heat_init");
    HeatArgs a;
    a.l = (uint32_t)p.l;
    a.plane = (uint32_t)(p.l * p.l);
    a.n = n;
    a.open = p.open;
    a.x = X;
    const double kh_h = p.kh * h;
    const dim3 block(32, 8), grid((unsigned)((p.l + 31) / 32), (unsigned)((p.l + 7) / 8), (unsigned)(2 * p.l));
    for (int64_t s = 0; s < N; ++s) {
        a.in = X;  a.out = Y;  a.c = kh_h / 4.0;
        heat_stage<true><<<grid, block, 0, sg.st>>>(a);
        REACH_LAUNCHED("heat_stage");
        a.in = Y;  a.out = Y2; a.c = kh_h / 3.0;
        heat_stage<false><<<grid, block, 0, sg.st>>>(a);
        REACH_LAUNCHED("heat_stage");
        a.in = Y2; a.out = Y;  a.c = kh_h / 2.0;
        heat_stage<false><<<grid, block, 0, sg.st>>>(a);
        REACH_LAUNCHED("heat_stage");
        // the last stage overwrites x in place: each thread reads x[i] before
        // writing it, and no thread reads another's x (neighbours come from Y)
        a.in = Y;  a.out = X;  a.c = kh_h;
        heat_stage<false><<<grid, block, 0, sg.st>>>(a);
        REACH_LAUNCHED("heat_stage");
    }
    heat_box<<<(unsigned)blocks, 256, 0, sg.st>>>(X, lo, hi, n, cgb, sg.status);
    REACH_LAUNCHED("heat_box");
    return REACH_OK;
}

}  // namespace reach
