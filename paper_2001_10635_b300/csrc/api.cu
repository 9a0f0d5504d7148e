// api.cu -- the C ABI of libreach.so (include/reach.h): systems, argument
// checking, host/device staging, kernel dispatch and status reporting.
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>

#include "api_internal.cuh"

namespace reach {

static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t k) { g_launches += k; }

int cuda_fail(cudaError_t e, const char *where) {
    if (getenv("REACH_DEBUG")) fprintf(stderr, "libreach: %s failed: %s\n", where, cudaGetErrorString(e));
    cudaGetLastError();   // clear a sticky-free error so the next call starts clean
    if (e == cudaErrorMemoryAllocation) return REACH_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return REACH_ENODEV;
    return REACH_ECUDA;
}

// process-wide options; read by calls on any thread
static std::atomic<int64_t> g_opt_kernel{0}, g_opt_steps{0}, g_opt_block{0}, g_opt_batch_cpt{0}, g_opt_tile{0},
    g_opt_mc_sb{0}, g_opt_mc_layout{0}, g_opt_serve_queue_blocks{64}, g_opt_serve_queue_n{512},
    g_opt_serve_max_wide{0}, g_opt_batch_cluster_from{0}, g_opt_one_launch{0},
    g_opt_serve_priority{0}, g_opt_serve_wide_exclusive{1},
    g_opt_serve_light{1 << 15};

// ---------------------------------------------------------------- memory
static std::atomic<bool> g_pool_ready[64];

// (setting the attribute twice from two threads is harmless)
int pool_init() {
    int dev = 0;
    REACH_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !g_pool_ready[dev].load()) {
        cudaMemPool_t pool;
        REACH_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
        uint64_t thr = UINT64_MAX;   // keep freed blocks cached for the next call
        REACH_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pool_ready[dev].store(true);
    }
    return REACH_OK;
}

int dalloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    return REACH_OK;
}

void dfree(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stage a caller vector on the device: device pointers are used in place,
// host vectors are copied into a pool buffer.
int Staging::in(const double *src, int64_t count, const double **dev) {
    if (count == 0 || !src) { *dev = src; return REACH_OK; }
    if (is_device_ptr(src)) { *dev = src; return REACH_OK; }
    void *p;
    int rc = dalloc(&p, count * sizeof(double), st);
    if (rc) return rc;
    owned[nowned++] = p;
    REACH_CUDA(cudaMemcpyAsync(p, src, count * sizeof(double), cudaMemcpyHostToDevice, st));
    *dev = (const double *)p;
    return REACH_OK;
}

int Staging::out(double *dst, int64_t count, double **dev) {
    if (is_device_ptr(dst)) { *dev = dst; return REACH_OK; }
    void *p;
    int rc = dalloc(&p, count * sizeof(double), st);
    if (rc) return rc;
    owned[nowned++] = p;
    back_dst[nback] = dst;
    back_src[nback] = (double *)p;
    back_n[nback++] = count;
    *dev = (double *)p;
    return REACH_OK;
}

int Staging::scratch(size_t bytes, void **dev) {
    void *p;
    int rc = dalloc(&p, bytes, st);
    if (rc) return rc;
    owned[nowned++] = p;
    *dev = p;
    return REACH_OK;
}

int Staging::begin_status() {
    int rc = scratch(sizeof(int), (void **)&status);
    if (rc) return rc;
    REACH_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    return REACH_OK;
}

// copy outputs back, wait for the stream, translate the status word
int Staging::finish() {
    for (int i = 0; i < nback; ++i)
        REACH_CUDA(cudaMemcpyAsync(back_dst[i], back_src[i], back_n[i] * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    int host_status = 0;
    if (status) REACH_CUDA(cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    release();
    REACH_CUDA(cudaStreamSynchronize(st));
    if (host_status & ST_BADINPUT) return REACH_EINVAL;
    if (host_status & ST_TIMEOUT) return REACH_ETIMEOUT;
    if (host_status & (ST_NONFINITE | ST_NEGRADIUS)) return REACH_ENONFINITE;
    return REACH_OK;
}

void Staging::release() {
    for (int i = 0; i < nowned; ++i) dfree(owned[i], st);
    nowned = 0;
    status = nullptr;
}

Staging::~Staging() {
    if (nowned) {
        release();
        cudaStreamSynchronize(st);
    }
}

// ---------------------------------------------------------------- checks
int nsteps(double t_final, double dt, int64_t *N) {
    if (!(dt > 0.0) || !std::isfinite(dt) || !(t_final >= 0.0) || !std::isfinite(t_final)) return REACH_EINVAL;
    double q = std::nearbyint(t_final / dt);
    if (std::fabs(q * dt - t_final) > 1e-9 * t_final) return REACH_EINVAL;
    if (q > 9.0e15) return REACH_EINVAL;
    *N = (int64_t)q;
    return REACH_OK;
}

// host-side box check when the data is on the host (device data is checked
// by the kernels as they load it)
int check_host_box(const double *lo, const double *hi, int64_t count) {
    if (count == 0) return REACH_OK;
    if (!lo || !hi) return REACH_EINVAL;
    if (is_device_ptr(lo) || is_device_ptr(hi)) return REACH_OK;
    for (int64_t i = 0; i < count; ++i)
        if (!(lo[i] <= hi[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i])) return REACH_EINVAL;
    return REACH_OK;
}

TrafficK make_traffic_k(const double *prm, double wl, double wh) {
    TrafficK p;
    p.cap = prm[0];
    p.v = prm[1];
    p.w = prm[2];
    p.xbar = prm[3];
    p.wxbar = p.w * p.xbar;
    int e = 0;
    const double m = std::frexp(p.v, &e);   // v = m 2^e, m in [0.5, 1)
    p.v_pow2 = (p.v > 0.0 && m == 0.5) ? 1 : 0;
    p.v_exp = e - 1;
    p.v_add = p.v_exp >= 0 ? ((long long)p.v_exp << 52) : -((long long)(-p.v_exp) << 52);
    p.d_lo = wl;
    p.d_hi = wh;
    p.d_c = 0.5 * (wl + wh);
    p.d_r = 0.5 * (wh - wl);
    p.local = prm[4] != 0.0;
    p.sound = prm[5] != 0.0;
    // h / 6 rounded down and up (set per call by the caller when sound)
    p.c6l = p.c6u = 0.0;
    p.one = 1.0;
    p.pzero = 0.0;
    p.nzero = -0.0;
    return p;
}

int64_t opt_kernel() { return g_opt_kernel; }
int64_t opt_steps() { return g_opt_steps; }
int64_t opt_block() { return g_opt_block; }
int64_t opt_batch_cpt() { return g_opt_batch_cpt; }
int64_t opt_tile() { return g_opt_tile; }
int64_t opt_mc_sb() { return g_opt_mc_sb; }
int64_t opt_mc_layout() { return g_opt_mc_layout; }
int64_t opt_batch_cluster_from() { return g_opt_batch_cluster_from; }
int64_t opt_one_launch() { return g_opt_one_launch; }

}  // namespace reach

using namespace reach;

// ================================================================ systems
extern "C" int reach_system_create(int kind, int64_t n, const void *params, size_t params_bytes,
                                   reach_system **out) {
    if (!out) return REACH_EINVAL;
    *out = nullptr;
    if (n < 1) return REACH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return REACH_ENODEV;
    }
    reach_system s;
    memset(&s, 0, sizeof s);
    s.kind = kind;
    s.n = n;
    double host[8] = {0};
    switch (kind) {
    case REACH_TRAFFIC: {
        reach_traffic_params p{40.0, 0.5, 1.0 / 6.0, 320.0, 0, 0};
        if (params) {
            // the four doubles alone are accepted too
            const size_t base = offsetof(reach_traffic_params, cgb_local);
            if (params_bytes != sizeof p && params_bytes != base) return REACH_EINVAL;
            memcpy(&p, params, params_bytes);
        }
        if (p.cgb_local && p.sound) return REACH_EINVAL;
        if (!std::isfinite(p.cap) || !std::isfinite(p.v) || !std::isfinite(p.w) || !std::isfinite(p.xbar) ||
            p.v < 0 || p.w < 0)
            return REACH_EINVAL;
        s.nw = 1;
        host[0] = p.cap; host[1] = p.v; host[2] = p.w; host[3] = p.xbar;
        host[4] = p.cgb_local ? 1.0 : 0.0;
        host[5] = p.sound ? 1.0 : 0.0;
        break;
    }
    case REACH_KS: {
        reach_ks_params p{M_PI / 4.0, 1.0, 1.0, 1.0};
        if (params) {
            if (params_bytes != sizeof p) return REACH_EINVAL;
            memcpy(&p, params, sizeof p);
        }
        if (!(p.dx > 0) || !std::isfinite(p.dx) || !std::isfinite(p.g_nl) || !std::isfinite(p.g_2) ||
            !std::isfinite(p.g_4) || n < 5)
            return REACH_EINVAL;
        s.nw = 0;
        // -g_2 u_xx - g_4 u_xxxx by central differences: coefficients of
        // u_i, u_{i+-1}, u_{i+-2}
        double d2 = 1.0 / (p.dx * p.dx), d4 = d2 * d2;
        host[0] = 2.0 * p.g_2 * d2 - 6.0 * p.g_4 * d4;
        host[1] = -p.g_2 * d2 + 4.0 * p.g_4 * d4;
        host[2] = -p.g_4 * d4;
        host[3] = p.g_nl / (2.0 * p.dx);
        break;
    }
    case REACH_OSC: {
        reach_osc_params p{1.0, 0.1, 0.5};
        if (params) {
            if (params_bytes != sizeof p) return REACH_EINVAL;
            memcpy(&p, params, sizeof p);
        }
        if (n % 2 || !std::isfinite(p.ka) || !std::isfinite(p.kb) || !std::isfinite(p.kc) || p.kb < 0)
            return REACH_EINVAL;
        s.nw = n / 2;
        host[0] = p.ka; host[1] = p.kb; host[2] = p.kc;
        break;
    }
    case REACH_LINEAR: {
        if (!params || params_bytes != sizeof(reach_linear_params) || n > 256) return REACH_EINVAL;
        s.nw = n;
        break;
    }
    case REACH_HEAT3D: {
        reach_heat_params p{8e-6, (int64_t)std::llround(std::cbrt((double)n)), 1};
        if (params) {
            if (params_bytes != sizeof p) return REACH_EINVAL;
            memcpy(&p, params, sizeof p);
        }
        if (p.l < 1 || p.l > 2097151 || p.l * p.l * p.l != n || !std::isfinite(p.alpha) || p.alpha < 0)
            return REACH_EINVAL;
        s.nw = 0;
        host[0] = p.alpha * (double)p.l * (double)p.l;   // alpha / dx^2
        host[1] = (double)p.l;
        host[2] = p.open_face ? 1.0 : 0.0;
        break;
    }
    case REACH_QUAD: {
        reach_quad_params p{1.4, 9.81, 1.4 * 9.81, 0.054, 0.054, 0.104};
        if (params) {
            if (params_bytes != sizeof p) return REACH_EINVAL;
            memcpy(&p, params, sizeof p);
        }
        if (n % 12 || !(p.m > 0) || !(p.F >= 0) || !(p.Jx > 0) || !(p.Jy > 0) || !(p.Jz > 0) ||
            !std::isfinite(p.m) || !std::isfinite(p.g) || !std::isfinite(p.F) || !std::isfinite(p.Jx) ||
            !std::isfinite(p.Jy) || !std::isfinite(p.Jz))
            return REACH_EINVAL;
        s.nw = n / 12 * 3;
        host[0] = p.F / p.m; host[1] = p.g; host[2] = p.Jx; host[3] = p.Jy; host[4] = p.Jz;
        break;
    }
    default:
        return REACH_EINVAL;
    }
    if (pool_init()) return REACH_ECUDA;
    memcpy(s.prm, host, sizeof host);
    if (kind == REACH_LINEAR) {
        const double *A = ((const reach_linear_params *)params)->A;
        if (!A) return REACH_EINVAL;
        REACH_CUDA(cudaMalloc(&s.dprm, n * n * sizeof(double)));
        cudaError_t e = cudaMemcpy(s.dprm, A, n * n * sizeof(double), cudaMemcpyDefault);
        if (e != cudaSuccess) { cudaFree(s.dprm); return cuda_fail(e, "cudaMemcpy A"); }
        if (!is_device_ptr(A)) {
            for (int64_t i = 0; i < n * n; ++i)
                if (!std::isfinite(A[i])) { cudaFree(s.dprm); return REACH_EINVAL; }
        }
    } else {
        REACH_CUDA(cudaMalloc(&s.dprm, 8 * sizeof(double)));
        cudaError_t e = cudaMemcpy(s.dprm, host, 8 * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(s.dprm); return cuda_fail(e, "cudaMemcpy params"); }
    }
    reach_system *p = new (std::nothrow) reach_system(s);
    if (!p) { cudaFree(s.dprm); return REACH_ENOMEM; }
    *out = p;
    return REACH_OK;
}

extern "C" int reach_system_destroy(reach_system *sys) {
    if (!sys) return REACH_EINVAL;
    if (sys->dprm) cudaFree(sys->dprm);
    delete sys;
    return REACH_OK;
}

extern "C" int64_t reach_system_dim(const reach_system *sys) { return sys ? sys->n : REACH_EINVAL; }
extern "C" int64_t reach_input_dim(const reach_system *sys) { return sys ? sys->nw : REACH_EINVAL; }

// ================================================================ MM / CGB
namespace reach {

// the on-chip kernels hold a problem in one block (2n <= QMAX * 512) or in a
// cluster of two blocks (2n <= 2 * QMAX * 512)
static bool onchip_fits(const reach_system *s) {
    const int64_t cap = (int64_t)QMAX * 512;
    if (2 * s->n <= cap) return onchip_smem_bytes(s->n, s->nw) <= onchip_max_smem();
    return 2 * s->n <= 2 * cap && cluster_smem_bytes(s->n, s->nw) <= onchip_max_smem();
}

bool use_onchip(const reach_system *s) {
    if (s->kind == REACH_QUAD) return false;   // one thread per agent at every size
    if (s->kind == REACH_TRAFFIC && s->prm[5] != 0.0) return false;   // outward rounding: streaming kernel only
    int64_t k = opt_kernel();
    bool fits = onchip_fits(s);
    if (k == 2) return fits;
    if (k == 1) return s->kind == REACH_OSC || s->kind == REACH_LINEAR;
    if (s->kind == REACH_OSC || s->kind == REACH_LINEAR) return true;
    if (s->kind == REACH_HEAT3D) return 2 * s->n <= 1024;
    return 2 * s->n <= 1024 || (s->kind == REACH_KS && s->n < 256);
}

int onchip_threads(int64_t n) {
    int64_t b = opt_block();
    if (b > 0) return (int)b;
    int64_t t = (2 * n + QMAX - 1) / QMAX;   // at most QMAX components per thread
    t = (t + 31) / 32 * 32;
    if (t < 128) t = (2 * n < 128) ? ((2 * n + 31) / 32 * 32) : 128;
    if (t > 512) t = 512;
    return (int)t;
}

static int reach_box(int method, const reach_system *sys, const double *x0_lo, const double *x0_hi,
                     const double *w_lo, const double *w_hi, double t_final, double dt, double *lo,
                     double *hi, void *stream) {
    if (!sys || !x0_lo || !x0_hi || !lo || !hi) return REACH_EINVAL;
    if (sys->nw > 0 && (!w_lo || !w_hi)) return REACH_EINVAL;
    int64_t N;
    int rc = nsteps(t_final, dt, &N);
    if (rc) return rc;
    // with N > 0 the first launch of every kernel checks the box on the device
    // (REACH_EINVAL through the status word), so a host box is not read twice
    if (N == 0 && (rc = check_host_box(x0_lo, x0_hi, sys->n))) return rc;
    if ((rc = check_host_box(w_lo, w_hi, sys->nw))) return rc;
    const int64_t n = sys->n;
    bool onchip = use_onchip(sys);
    if (onchip && !onchip_fits(sys))
        return REACH_EINVAL;   // too large for the on-chip kernels and no streaming kernel for this kind

    // the traffic streaming kernel with host buffers in and out: copies in
    // chunks that overlap the first and last steps (the input checks run on
    // the device as for every launch)
    if (sys->kind == REACH_TRAFFIC && !onchip && N > 0 && sys->prm[4] == 0.0 && sys->prm[5] == 0.0 &&
        n >= OVERLAP_MIN_CELLS && !is_device_ptr(x0_lo) && !is_device_ptr(x0_hi) && !is_device_ptr(lo) &&
        !is_device_ptr(hi) && !is_device_ptr(w_lo)) {
        const double wl = w_lo[0], wh = w_hi[0];
        if (!(wl <= wh) || !std::isfinite(wl) || !std::isfinite(wh)) return REACH_EINVAL;
        Staging sg((cudaStream_t)stream);
        if ((rc = sg.begin_status())) return rc;
        const TrafficK p = make_traffic_k(sys->prm, wl, wh);
        const int S = opt_steps() > 0 ? (int)opt_steps() : 1;
        if ((rc = stencil_traffic_overlap(method, p, n, x0_lo, x0_hi, lo, hi, dt, N, S, sg))) return rc;
        return sg.finish();
    }

    Staging sg((cudaStream_t)stream);
    const double *dxlo, *dxhi, *dwlo = nullptr, *dwhi = nullptr;
    double *dlo, *dhi;
    if ((rc = sg.in(x0_lo, n, &dxlo)) || (rc = sg.in(x0_hi, n, &dxhi)) || (rc = sg.in(w_lo, sys->nw, &dwlo)) ||
        (rc = sg.in(w_hi, sys->nw, &dwhi)) || (rc = sg.out(lo, n, &dlo)) || (rc = sg.out(hi, n, &dhi)) ||
        (rc = sg.begin_status()))
        return rc;

    // host copies of the (scalar) traffic input for the streaming kernel
    double wl_host = 0, wh_host = 0;
    if (!onchip && sys->kind == REACH_TRAFFIC) {
        if (is_device_ptr(w_lo)) {
            REACH_CUDA(cudaMemcpyAsync(&wl_host, w_lo, sizeof(double), cudaMemcpyDeviceToHost, sg.st));
            REACH_CUDA(cudaMemcpyAsync(&wh_host, w_hi, sizeof(double), cudaMemcpyDeviceToHost, sg.st));
            REACH_CUDA(cudaStreamSynchronize(sg.st));
        } else {
            wl_host = w_lo[0];
            wh_host = w_hi[0];
        }
        if (!(wl_host <= wh_host) || !std::isfinite(wl_host) || !std::isfinite(wh_host)) return REACH_EINVAL;
    }

    if (N == 0) {
        // the box itself (Algorithms 2 and 3 with no step)
        REACH_CUDA(cudaMemcpyAsync(dlo, dxlo, n * sizeof(double), cudaMemcpyDeviceToDevice, sg.st));
        REACH_CUDA(cudaMemcpyAsync(dhi, dxhi, n * sizeof(double), cudaMemcpyDeviceToDevice, sg.st));
        return sg.finish();
    }

    if (onchip) {
        OnItem it;
        it.n = n;
        it.nw = sys->nw;
        it.kind = sys->kind;
        it.method = method;
        it.xlo = dxlo; it.xhi = dxhi; it.wlo = dwlo; it.whi = dwhi;
        it.lo = dlo; it.hi = dhi;
        it.prm = sys->dprm;
        it.N = N;
        it.h = dt;
        it.status = sg.status;
        it.one = 1.0;
        it.nzero = -0.0;
        it.hh = 0.5 * dt;
        it.h6 = dt / 6.0;
        if (2 * n <= (int64_t)QMAX * 512) rc = onchip_launch_single(it, onchip_threads(n), sg.st);
        else rc = onchip_launch_cluster(it, sg.st);
        if (rc) return rc;
        return sg.finish();
    }

    if (sys->kind == REACH_QUAD) {
        QuadK p;
        p.a = sys->prm[0]; p.g = sys->prm[1]; p.Jx = sys->prm[2]; p.Jy = sys->prm[3]; p.Jz = sys->prm[4];
        rc = quad_run(method, p, n, dxlo, dxhi, dwlo, dwhi, dlo, dhi, dt, N, sg.status, sg.st);
    } else if (sys->kind == REACH_HEAT3D) {
        HeatK p;
        p.kh = sys->prm[0];
        p.l = (int64_t)sys->prm[1];
        p.open = sys->prm[2] != 0.0;
        rc = heat_run(method, p, n, dxlo, dxhi, dlo, dhi, dt, N, sg);
    } else {
        // ping-pong partner of the output for the fused stencil kernels
        double *sA, *sB;
        if ((rc = sg.scratch(2 * n * sizeof(double), (void **)&sA))) return rc;
        sB = sA + n;
        // FP64 stencil kernels are bound by the FP64 pipe: recomputing a wider
        // halo costs more than the HBM traffic it saves, so one step per launch
        // unless the grid is too short to fill the GPU
        int S = opt_steps() > 0 ? (int)opt_steps() : 1;
        if (sys->kind == REACH_TRAFFIC) {
            TrafficK p = make_traffic_k(sys->prm, wl_host, wh_host);
            if (opt_steps() == 0 && !p.sound && !(method == CGB && p.local)) S = stencil_short_steps(1, 2, n);
            if (p.sound) {
                rc = stencil_traffic_sound(method, p, n, dxlo, dxhi, dlo, dhi, dt, N, S, sg);
            } else if (S == 1 && traffic_flow_eligible(p, method, n, N)) {
                void *work;
                if ((rc = sg.scratch((size_t)traffic_flow_work_bytes(n), &work))) return rc;
                rc = stencil_traffic_flow_run(method, p, n, dxlo, dxhi, dlo, dhi, sA, sB, dt, N, sg.status, work,
                                              sg.st);
            } else {
                rc = stencil_traffic(method, p, n, dxlo, dxhi, dlo, dhi, sA, sB, dt, N, S, sg.status, sg.st);
            }
        } else {
            KsK p;
            p.a0 = sys->prm[0]; p.a1 = sys->prm[1]; p.a2 = sys->prm[2]; p.k = sys->prm[3];
            if (opt_steps() == 0) S = stencil_short_steps(2, 1, n);
            if (S == 1 && ks_flow_eligible(n, N)) {
                void *work;
                if ((rc = sg.scratch((size_t)ks_flow_work_bytes(n), &work))) return rc;
                rc = stencil_ks_flow_run(method, p, n, dxlo, dxhi, dlo, dhi, sA, sB, dt, N, sg.status, work, sg.st);
            } else {
                rc = stencil_ks(method, p, n, dxlo, dxhi, dlo, dhi, sA, sB, dt, N, S, sg.status, sg.st);
            }
        }
    }
    if (rc) return rc;
    return sg.finish();
}

}  // namespace reach

extern "C" int reach_mm(const reach_system *sys, const double *x0_lo, const double *x0_hi, const double *w_lo,
                        const double *w_hi, double t_final, double dt, double *lo, double *hi, void *stream) {
    return reach_box(MM, sys, x0_lo, x0_hi, w_lo, w_hi, t_final, dt, lo, hi, stream);
}

extern "C" int reach_cgb(const reach_system *sys, const double *x0_lo, const double *x0_hi, const double *w_lo,
                         const double *w_hi, double t_final, double dt, double *lo, double *hi, void *stream) {
    return reach_box(CGB, sys, x0_lo, x0_hi, w_lo, w_hi, t_final, dt, lo, hi, stream);
}

extern "C" int64_t reach_mc_samples(int64_t n, double eps, double delta) {
    if (n < 1 || !(eps > 0 && eps < 1) || !(delta > 0 && delta < 1)) return REACH_EINVAL;
    double q = 2.0 * (double)n;
    return (int64_t)std::ceil((q / eps) * std::log(q / delta));
}

extern "C" int reach_set_option(int key, int64_t value) {
    switch (key) {
    case REACH_OPT_KERNEL:
        if (value < 0 || value > 2) return REACH_EINVAL;
        g_opt_kernel = value;
        return REACH_OK;
    case REACH_OPT_STEPS_PER_LAUNCH:
        if (value < 0 || value > 8) return REACH_EINVAL;
        g_opt_steps = value;
        return REACH_OK;
    case REACH_OPT_BLOCK:
        if (value != 0 && (value < 32 || value > 512 || value % 32)) return REACH_EINVAL;
        g_opt_block = value;
        return REACH_OK;
    case REACH_OPT_BATCH_CPT:
        if (value != 0 && value != 2 && value != 4 && value != 8 && value != 16) return REACH_EINVAL;
        g_opt_batch_cpt = value;
        return REACH_OK;
    case REACH_OPT_TILE:
        if (value != 0 && value != 2 && value != 8) return REACH_EINVAL;
        g_opt_tile = value;
        return REACH_OK;
    case REACH_OPT_MC_SB:
        if (value != 0 && value != 2 && value != 8 && value != 32) return REACH_EINVAL;
        g_opt_mc_sb = value;
        return REACH_OK;
    case REACH_OPT_MC_LAYOUT:
        if (value < 0 || value > 10) return REACH_EINVAL;
        g_opt_mc_layout = value;
        return REACH_OK;
    case REACH_OPT_SERVE_QUEUE_BLOCKS:
        if (value < 0 || value > 4096) return REACH_EINVAL;
        g_opt_serve_queue_blocks = value;
        return REACH_OK;
    case REACH_OPT_SERVE_QUEUE_N:
        if (value < 0 || value > REACH_QUEUE_MAX_N) return REACH_EINVAL;
        g_opt_serve_queue_n = value;
        return REACH_OK;
    case REACH_OPT_SERVE_MAX_WIDE:
        if (value < 0 || value > 256) return REACH_EINVAL;
        g_opt_serve_max_wide = value;
        return REACH_OK;
    case REACH_OPT_BATCH_CLUSTER_FROM:
        if (value < 0 || value > 16384) return REACH_EINVAL;
        g_opt_batch_cluster_from = value;
        return REACH_OK;
    case REACH_OPT_ONE_LAUNCH:
        if (value < 0 || value > 2) return REACH_EINVAL;
        g_opt_one_launch = value;
        return REACH_OK;
    case REACH_OPT_SERVE_PRIORITY:
        if (value < 0 || value > 3) return REACH_EINVAL;
        g_opt_serve_priority = value;
        return REACH_OK;
    case REACH_OPT_SERVE_WIDE_EXCLUSIVE:
        if (value < 0 || value > 1) return REACH_EINVAL;
        g_opt_serve_wide_exclusive = value;
        return REACH_OK;
    case REACH_OPT_SERVE_LIGHT:
        if (value < 0 || value > ((int64_t)1 << 40)) return REACH_EINVAL;
        g_opt_serve_light = value;
        return REACH_OK;
    }
    return REACH_EINVAL;
}

extern "C" int64_t reach_get_option(int key) {
    switch (key) {
    case REACH_OPT_KERNEL: return g_opt_kernel;
    case REACH_OPT_STEPS_PER_LAUNCH: return g_opt_steps;
    case REACH_OPT_BLOCK: return g_opt_block;
    case REACH_OPT_BATCH_CPT: return g_opt_batch_cpt;
    case REACH_OPT_TILE: return g_opt_tile;
    case REACH_OPT_MC_SB: return g_opt_mc_sb;
    case REACH_OPT_MC_LAYOUT: return g_opt_mc_layout;
    case REACH_OPT_SERVE_QUEUE_BLOCKS: return g_opt_serve_queue_blocks;
    case REACH_OPT_SERVE_QUEUE_N: return g_opt_serve_queue_n;
    case REACH_OPT_SERVE_MAX_WIDE: return g_opt_serve_max_wide;
    case REACH_OPT_BATCH_CLUSTER_FROM: return g_opt_batch_cluster_from;
    case REACH_OPT_ONE_LAUNCH: return g_opt_one_launch;
    case REACH_OPT_SERVE_PRIORITY: return g_opt_serve_priority;
    case REACH_OPT_SERVE_WIDE_EXCLUSIVE: return g_opt_serve_wide_exclusive;
    case REACH_OPT_SERVE_LIGHT: return g_opt_serve_light;
    }
    return REACH_EINVAL;
}

extern "C" const char *reach_strerror(int code) {
    switch (code) {
    case REACH_OK: return "ok";
    case REACH_EINVAL: return "invalid argument";
    case REACH_ENOMEM: return "out of device memory";
    case REACH_EADMIT: return "query exceeds the device memory budget";
    case REACH_ENONFINITE: return "result is not finite";
    case REACH_ETIMEOUT: return "bounded wait timed out";
    case REACH_ECUDA: return "CUDA runtime error";
    case REACH_ENODEV: return "no CUDA device";
    }
    return "unknown status";
}

extern "C" int64_t reach_kernel_launches(void) { return g_launches.load(); }

// ================================================================ reach pipe
// Boxes after every `every` steps (the reach pipe of Sec. 5.5).  Each segment
// integrates `every` steps from the previous box into the next pipe row on the
// device.  The MM state is the box, so segments continue the integration
// exactly; a CGB segment restarts from c = (lo + hi)/2, r = (hi - lo)/2 of the
// previous row, which recovers the center and radius up to one rounding.
extern "C" int reach_pipe(const reach_system *sys, int method, const double *x0_lo, const double *x0_hi,
                          const double *w_lo, const double *w_hi, double t_final, double dt, int64_t every,
                          double *pipe_lo, double *pipe_hi, void *stream) {
    if (!sys || !x0_lo || !x0_hi || !pipe_lo || !pipe_hi || (method != MM && method != CGB) || every < 1)
        return REACH_EINVAL;
    if (sys->kind == REACH_TRAFFIC && sys->prm[5] != 0.0) return REACH_EINVAL;   // outward rounding: whole horizons
    if (sys->nw > 0 && (!w_lo || !w_hi)) return REACH_EINVAL;
    int64_t N;
    int rc = nsteps(t_final, dt, &N);
    if (rc) return rc;
    if (N % every) return REACH_EINVAL;
    if ((rc = check_host_box(x0_lo, x0_hi, sys->n))) return rc;
    if ((rc = check_host_box(w_lo, w_hi, sys->nw))) return rc;
    const int64_t n = sys->n, rows = N / every;
    if (rows == 0) return REACH_OK;
    Staging sg((cudaStream_t)stream);
    const double *dxlo, *dxhi, *dwlo = nullptr, *dwhi = nullptr;
    double *plo, *phi;
    if ((rc = sg.in(x0_lo, n, &dxlo)) || (rc = sg.in(x0_hi, n, &dxhi)) || (rc = sg.in(w_lo, sys->nw, &dwlo)) ||
        (rc = sg.in(w_hi, sys->nw, &dwhi)) || (rc = sg.out(pipe_lo, rows * n, &plo)) ||
        (rc = sg.out(pipe_hi, rows * n, &phi)))
        return rc;
    const double T = dt * (double)every;
    for (int64_t q = 0; q < rows && !rc; ++q) {
        const double *alo = q ? plo + (q - 1) * n : dxlo, *ahi = q ? phi + (q - 1) * n : dxhi;
        rc = reach_box(method, sys, alo, ahi, dwlo, dwhi, T, dt, plo + q * n, phi + q * n, stream);
    }
    if (rc) return rc;
    return sg.finish();
}
