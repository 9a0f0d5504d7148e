// api_internal.cuh -- host-side internals shared by the ABI translation units.
#pragma once

#include "common.cuh"
#include "onchip.cuh"
#include "quad.cuh"

struct reach_system {
    int kind;
    int64_t n, nw;
    double prm[8];    // host copy of the device parameter block (not for linear)
    double *dprm;     // device parameters (linear: A, n x n)
};

namespace reach {

// per-call device staging: input copies, output buffers, scratch, status word
struct Staging {
    cudaStream_t st;
    void *owned[16];
    int nowned = 0;
    double *back_dst[4];
    double *back_src[4];
    int64_t back_n[4];
    int nback = 0;
    int *status = nullptr;

    explicit Staging(cudaStream_t s) : st(s) {}
    ~Staging();
    int in(const double *src, int64_t count, const double **dev);
    int out(double *dst, int64_t count, double **dev);
    int scratch(size_t bytes, void **dev);
    int begin_status();
    int finish();
    void release();
};

int pool_init();
int dalloc(void **p, size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);
bool is_device_ptr(const void *p);
int nsteps(double t_final, double dt, int64_t *N);
int check_host_box(const double *lo, const double *hi, int64_t count);
int64_t opt_kernel();
int64_t opt_steps();
int64_t opt_block();
int64_t opt_batch_cpt();
int64_t opt_tile();
int64_t opt_mc_sb();
int64_t opt_mc_layout();
int64_t opt_batch_cluster_from();
int64_t opt_one_launch();
// samples per block of the on-chip MC kernel for m samples (2, 8 or 32)
int mc_onchip_sb(int64_t m);

// traffic parameters as the streaming kernel sees them (inputs d in [wl, wh])
TrafficK make_traffic_k(const double *prm, double wl, double wh);

// device work queue: whether a query of this system and method can be queued
bool queue_accepts(const reach_system *s, int method);

// kernels
constexpr int BATCH_THREADS = 512;   // threads per block of the batched kernel
int64_t onchip_smem_bytes(int64_t n, int64_t nw);
int onchip_max_smem();
// raise a kernel's dynamic shared-memory limit to what the device allows
// beside the kernel's own static shared memory
int allow_max_dynamic_smem(const void *fn);
int onchip_launch_single(const OnItem &it, int threads, cudaStream_t st);
int64_t cluster_smem_bytes(int64_t n, int64_t nw);
int onchip_launch_cluster(const OnItem &it, cudaStream_t st);
int onchip_launch_batch(int kind, int method, int q, const void *items, const void *slots, const void *bins,
                        const void *tasks, int ntasks, int *counter, uint64_t *done, int clusters, size_t smem,
                        cudaStream_t st);
int onchip_launch_stamp(uint64_t *t0, cudaStream_t st);
int onchip_batch_threads();

// host mirrors of the batch kernel's work-list records (onchip.cu)
struct BatchSlot {
    int item, warp0, nwarps, bar;
    int64_t off;
};
struct BatchBin {
    int slot0, nslots;
};
struct BatchTask {
    int big;
    int bin[2];
};
// RK4 steps per launch of the streaming stencil kernels for an n-cell grid of
// stencil radius R and `halves` warps per tile
int stencil_short_steps(int R, int halves, int64_t n);
int stencil_traffic(int method, const TrafficK &p, int64_t n, const double *xlo, const double *xhi,
                    double *lo, double *hi, double *sA, double *sB, double h, int64_t N, int S,
                    int *status, cudaStream_t st);
int quad_run(int method, const QuadK &p, int64_t n, const double *xlo, const double *xhi, const double *wlo,
             const double *whi, double *lo, double *hi, double h, int64_t N, int *status, cudaStream_t st);
// the host-buffer path of the traffic kernel overlaps its copies in this many
// chunks, for chains long enough that the copies outweigh a second stream,
// sixteen events and the chunked launches (2^20 cells: 8 MiB per vector)
constexpr int OVERLAP_CHUNKS = 8;
constexpr int64_t OVERLAP_MIN_CELLS = (int64_t)1 << 20;
int stencil_traffic_overlap(int method, const TrafficK &p, int64_t n, const double *hxlo, const double *hxhi,
                            double *hlo, double *hhi, double h, int64_t N, int S, Staging &sg);
int stencil_traffic_sound(int method, const TrafficK &p, int64_t n, const double *xlo, const double *xhi,
                          double *lo, double *hi, double h, int64_t N, int S, Staging &sg);
int heat_run(int method, const HeatK &p, int64_t n, const double *xlo, const double *xhi, double *lo,
             double *hi, double h, int64_t N, Staging &sg);
// traffic MM / CGB with every step in one persistent launch (stencil_traffic_flow)
bool traffic_flow_eligible(const TrafficK &p, int method, int64_t n, int64_t N);
int64_t traffic_flow_work_bytes(int64_t n);
int stencil_traffic_flow_run(int method, const TrafficK &p, int64_t n, const double *xlo, const double *xhi,
                             double *lo, double *hi, double *sA, double *sB, double h, int64_t N, int *status,
                             void *work, cudaStream_t st);
// KS MM / CGB with every step in one persistent launch (stencil_ks_flow):
// whether it runs this grid, its scratch (an item counter and one word per
// tile), and the call
bool ks_flow_eligible(int64_t n, int64_t N);
int64_t ks_flow_work_bytes(int64_t n);
int stencil_ks_flow_run(int method, const KsK &p, int64_t n, const double *xlo, const double *xhi, double *lo,
                        double *hi, double *sA, double *sB, double h, int64_t N, int *status, void *work,
                        cudaStream_t st);
int stencil_ks(int method, const KsK &p, int64_t n, const double *xlo, const double *xhi, double *lo,
               double *hi, double *sA, double *sB, double h, int64_t N, int S, int *status,
               cudaStream_t st);

}  // namespace reach
