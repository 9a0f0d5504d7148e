// onchip.cu -- host side of the on-chip path: shared-memory sizing, kernel
// attributes, and dispatch to the per-kind instantiations (onchip_<kind>.cu).
#include "api_internal.cuh"

namespace reach {

// shared memory of one problem: y (2n), inputs (2 nw), stage derivatives (2n)
int64_t onchip_smem_bytes(int64_t n, int64_t nw) { return (4 * n + 2 * nw) * (int64_t)sizeof(double); }

int allow_max_dynamic_smem(const void *fn) {
    cudaFuncAttributes fa;
    REACH_CUDA(cudaFuncGetAttributes(&fa, fn));
    int cap = onchip_max_smem() - (int)fa.sharedSizeBytes;
    REACH_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    return REACH_OK;
}

int onchip_max_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// shared memory of one cluster block: its half of y, its inputs, its derivatives
int64_t cluster_smem_bytes(int64_t n, int64_t nw) { return (2 * n + nw) * (int64_t)sizeof(double); }

__global__ void stamp_start(uint64_t *t0) { *t0 = global_ns(); }

int onchip_launch_stamp(uint64_t *t0, cudaStream_t st) {
    stamp_start<<<1, 1, 0, st>>>(t0);
    REACH_LAUNCHED("stamp_start");
    return REACH_OK;
}

int onchip_batch_threads() { return BATCH_THREADS; }

template <int SYS> int onchip_single_k(const OnItem &, int, cudaStream_t);
template <int SYS> int onchip_cluster_k(const OnItem &, cudaStream_t);
template <int SYS>
int onchip_batch_k(int, int, const void *, const void *, const void *, const void *, int, int *, uint64_t *, int,
                   size_t, cudaStream_t);

int onchip_launch_single(const OnItem &it, int threads, cudaStream_t st) {
    switch (it.kind) {
    case REACH_TRAFFIC: return onchip_single_k<REACH_TRAFFIC>(it, threads, st);
    case REACH_KS: return onchip_single_k<REACH_KS>(it, threads, st);
    case REACH_OSC: return onchip_single_k<REACH_OSC>(it, threads, st);
    case REACH_LINEAR: return onchip_single_k<REACH_LINEAR>(it, threads, st);
    case REACH_HEAT3D: return onchip_single_k<REACH_HEAT3D>(it, threads, st);
    }
    return REACH_EINVAL;
}

int onchip_launch_cluster(const OnItem &it, cudaStream_t st) {
    switch (it.kind) {
    case REACH_TRAFFIC: return onchip_cluster_k<REACH_TRAFFIC>(it, st);
    case REACH_KS: return onchip_cluster_k<REACH_KS>(it, st);
    case REACH_OSC: return onchip_cluster_k<REACH_OSC>(it, st);
    case REACH_LINEAR: return onchip_cluster_k<REACH_LINEAR>(it, st);
    case REACH_HEAT3D: return onchip_cluster_k<REACH_HEAT3D>(it, st);
    }
    return REACH_EINVAL;
}

int onchip_launch_batch(int kind, int method, int q, const void *items, const void *slots, const void *bins,
                        const void *tasks, int ntasks, int *counter, uint64_t *done, int clusters, size_t smem,
                        cudaStream_t st) {
    switch (kind) {
    case REACH_TRAFFIC: return onchip_batch_k<REACH_TRAFFIC>(method, q, items, slots, bins, tasks, ntasks, counter, done, clusters, smem, st);
    case REACH_KS: return onchip_batch_k<REACH_KS>(method, q, items, slots, bins, tasks, ntasks, counter, done, clusters, smem, st);
    case REACH_OSC: return onchip_batch_k<REACH_OSC>(method, q, items, slots, bins, tasks, ntasks, counter, done, clusters, smem, st);
    case REACH_LINEAR: return onchip_batch_k<REACH_LINEAR>(method, q, items, slots, bins, tasks, ntasks, counter, done, clusters, smem, st);
    case REACH_HEAT3D: return onchip_batch_k<REACH_HEAT3D>(method, q, items, slots, bins, tasks, ntasks, counter, done, clusters, smem, st);
    }
    return REACH_EINVAL;
}

}  // namespace reach
