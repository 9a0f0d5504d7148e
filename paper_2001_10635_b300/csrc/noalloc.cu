// noalloc.cu -- reach_mm_noalloc: the mixed-monotonicity box of a streaming
// stencil system (traffic chain, KS grid) without any device allocation.
//
// Some callers cannot let a library allocate device memory: a process whose
// device memory is already reserved by another allocator (a framework's
// caching pool that holds nearly all of HBM, so cudaMalloc fails), or a
// latency-critical loop that must never enter the driver's allocator, which
// can take locks and synchronise.  For them this entry point runs the same
// streaming RK4 kernel as reach_mm, with the kernel's ping-pong state buffer
// and the status word in a fixed buffer that the library defines at file
// scope.  Every GPU that loads the library holds this buffer until the
// process exits.
#include "api_internal.cuh"

namespace reach {

// ping-pong partner of the output (2 * REACH_NOALLOC_MAX_N doubles) followed
// by the status word
static __device__ __align__(256) double g_noalloc_scratch[2 * REACH_NOALLOC_MAX_N + 32];

// Device address of the buffer on the current device, looked up on every
// call (the lookup allocates nothing and stays valid across a device reset,
// which reloads the module at another address).  The name g_noalloc_scratch
// is only a host-side stand-in: kernels must be given the address the runtime
// reports for the current device.
static int noalloc_buffer(double **out) {
    void *p = nullptr;
    REACH_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = (double *)p;
    return REACH_OK;
}

}  // namespace reach

using namespace reach;

extern "C" int reach_mm_noalloc(const reach_system *sys, const double *x0_lo, const double *x0_hi,
                                const double *w_lo, const double *w_hi, double t_final, double dt,
                                double *lo, double *hi, void *stream) {
    if (!sys || !x0_lo || !x0_hi || !lo || !hi) return REACH_EINVAL;
    if (sys->kind != REACH_TRAFFIC && sys->kind != REACH_KS) return REACH_EINVAL;
    if (sys->kind == REACH_TRAFFIC && sys->prm[5] != 0.0) return REACH_EINVAL;   // no outward-rounded kernel here
    if (sys->n > REACH_NOALLOC_MAX_N) return REACH_EINVAL;   // larger than the fixed buffer
    if (sys->nw > 0 && (!w_lo || !w_hi)) return REACH_EINVAL;
    // no staging copies: the state vectors must already be on the device
    if (!is_device_ptr(x0_lo) || !is_device_ptr(x0_hi) || !is_device_ptr(lo) || !is_device_ptr(hi))
        return REACH_EINVAL;
    int64_t N;
    int rc = nsteps(t_final, dt, &N);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = sys->n;

    double *buf;
    if ((rc = noalloc_buffer(&buf))) return rc;
    double *sA = buf, *sB = buf + n;
    int *status = (int *)(buf + 2 * REACH_NOALLOC_MAX_N);
    // the buffer keeps the previous call's contents: the status word must start at zero
    REACH_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));

    if (N == 0) {
        REACH_CUDA(cudaMemcpyAsync(lo, x0_lo, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        REACH_CUDA(cudaMemcpyAsync(hi, x0_hi, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else if (sys->kind == REACH_TRAFFIC) {
        double wl = 0, wh = 0;
        if (is_device_ptr(w_lo)) {
            REACH_CUDA(cudaMemcpyAsync(&wl, w_lo, sizeof(double), cudaMemcpyDeviceToHost, st));
            REACH_CUDA(cudaMemcpyAsync(&wh, w_hi, sizeof(double), cudaMemcpyDeviceToHost, st));
            REACH_CUDA(cudaStreamSynchronize(st));
        } else {
            wl = w_lo[0];
            wh = w_hi[0];
        }
        if (!(wl <= wh) || !std::isfinite(wl) || !std::isfinite(wh)) return REACH_EINVAL;
        TrafficK p = make_traffic_k(sys->prm, wl, wh);
        // the launch schedule of reach_mm: several RK4 steps per launch for
        // grids too short to fill the GPU (the ping-pong buffer is the same)
        const int S = opt_steps() > 0 ? (int)opt_steps() : stencil_short_steps(1, 2, n);
        rc = stencil_traffic(MM, p, n, x0_lo, x0_hi, lo, hi, sA, sB, dt, N, S, status, st);
    } else {
        KsK p;
        p.a0 = sys->prm[0]; p.a1 = sys->prm[1]; p.a2 = sys->prm[2]; p.k = sys->prm[3];
        const int S = opt_steps() > 0 ? (int)opt_steps() : stencil_short_steps(2, 1, n);
        rc = stencil_ks(MM, p, n, x0_lo, x0_hi, lo, hi, sA, sB, dt, N, S, status, st);
    }
    if (rc) return rc;
    int host_status = 0;
    REACH_CUDA(cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    REACH_CUDA(cudaStreamSynchronize(st));
    if (host_status & ST_BADINPUT) return REACH_EINVAL;
    if (host_status & (ST_NONFINITE | ST_NEGRADIUS)) return REACH_ENONFINITE;
    return REACH_OK;
}
