// onchip.cu -- kernels built on onchip_run: one problem per block, and the
// batched persistent kernel that runs many uneven problems in one launch.
#include "api_internal.cuh"

namespace reach {

// ---------------------------------------------------------------- one problem
template <int SYS, int METHOD>
__global__ void __launch_bounds__(512) onchip_single(OnItem it) {
    extern __shared__ double sm[];
    const int64_t n = it.n;
    GroupSync sync{0, (int)blockDim.x};
    onchip_run<SYS, METHOD>(it, sm, sm + n, sm + 2 * n, sm + 2 * n + it.nw, sm + 2 * n + 2 * it.nw, 0,
                            2 * n, (int)threadIdx.x, (int)blockDim.x, sync);
}

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

template <int SYS, int METHOD>
static int launch_single_t(const OnItem &it, int threads, cudaStream_t st) {
    int64_t smem = onchip_smem_bytes(it.n, it.nw);
    static bool attr_set = false;
    if (!attr_set) {
        int rc = allow_max_dynamic_smem((const void *)onchip_single<SYS, METHOD>);
        if (rc) return rc;
        attr_set = true;
    }
    onchip_single<SYS, METHOD><<<1, threads, (size_t)smem, st>>>(it);
    REACH_LAUNCHED("onchip_single");
    return REACH_OK;
}

int onchip_launch_single(const OnItem &it, int threads, cudaStream_t st) {
    switch (it.kind * 2 + it.method) {
    case REACH_TRAFFIC * 2 + MM: return launch_single_t<REACH_TRAFFIC, MM>(it, threads, st);
    case REACH_TRAFFIC * 2 + CGB: return launch_single_t<REACH_TRAFFIC, CGB>(it, threads, st);
    case REACH_KS * 2 + MM: return launch_single_t<REACH_KS, MM>(it, threads, st);
    case REACH_KS * 2 + CGB: return launch_single_t<REACH_KS, CGB>(it, threads, st);
    case REACH_OSC * 2 + MM: return launch_single_t<REACH_OSC, MM>(it, threads, st);
    case REACH_OSC * 2 + CGB: return launch_single_t<REACH_OSC, CGB>(it, threads, st);
    case REACH_LINEAR * 2 + MM: return launch_single_t<REACH_LINEAR, MM>(it, threads, st);
    case REACH_LINEAR * 2 + CGB: return launch_single_t<REACH_LINEAR, CGB>(it, threads, st);
    }
    return REACH_EINVAL;
}

// ---------------------------------------------------------------- batch
// A bin is the work of one block: up to 16 slots, each a problem run by a
// contiguous range of warps with its own named barrier and shared-memory
// region.  Blocks take bins from a global counter, largest first.
struct Slot {
    int item, warp0, nwarps, bar;
    int64_t off;   // shared-memory offset (doubles)
};
struct Bin {
    int slot0, nslots;
};

constexpr int BATCH_THREADS = 512;

template <int SYS>
__global__ void __launch_bounds__(BATCH_THREADS) onchip_batch(const OnItem *__restrict__ items,
                                                              const Slot *__restrict__ slots,
                                                              const Bin *__restrict__ bins, int nbins,
                                                              int *counter) {
    extern __shared__ double sm[];
    __shared__ int cur;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int b = cur;
        __syncthreads();
        if (b >= nbins) break;
        const Bin bn = bins[b];
        for (int s = bn.slot0; s < bn.slot0 + bn.nslots; ++s) {
            const Slot sl = slots[s];
            if (warp < sl.warp0 || warp >= sl.warp0 + sl.nwarps) continue;
            const OnItem &it = items[sl.item];
            double *y = sm + sl.off;
            const int64_t n = it.n;
            GroupSync sync{sl.bar, sl.nwarps * 32};
            const int gt = (int)threadIdx.x - sl.warp0 * 32, gs = sl.nwarps * 32;
            double *w = y + 2 * n, *kb = w + 2 * it.nw;
            if (it.method == MM)
                onchip_run<SYS, MM>(it, y, y + n, w, w + it.nw, kb, 0, 2 * n, gt, gs, sync);
            else
                onchip_run<SYS, CGB>(it, y, y + n, w, w + it.nw, kb, 0, 2 * n, gt, gs, sync);
            break;
        }
        __syncthreads();   // every slot of this bin is done before its memory is reused
    }
}

template <int SYS>
static int launch_batch_t(const OnItem *items, const Slot *slots, const Bin *bins, int nbins, int *counter,
                          int grid, size_t smem, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        int rc = allow_max_dynamic_smem((const void *)onchip_batch<SYS>);
        if (rc) return rc;
        attr_set = true;
    }
    onchip_batch<SYS><<<grid, BATCH_THREADS, smem, st>>>(items, slots, bins, nbins, counter);
    REACH_LAUNCHED("onchip_batch");
    return REACH_OK;
}

int onchip_launch_batch(int kind, const void *items, const void *slots, const void *bins, int nbins,
                        int *counter, int grid, size_t smem, cudaStream_t st) {
    const OnItem *it = (const OnItem *)items;
    const Slot *sl = (const Slot *)slots;
    const Bin *bn = (const Bin *)bins;
    switch (kind) {
    case REACH_TRAFFIC: return launch_batch_t<REACH_TRAFFIC>(it, sl, bn, nbins, counter, grid, smem, st);
    case REACH_KS: return launch_batch_t<REACH_KS>(it, sl, bn, nbins, counter, grid, smem, st);
    case REACH_OSC: return launch_batch_t<REACH_OSC>(it, sl, bn, nbins, counter, grid, smem, st);
    case REACH_LINEAR: return launch_batch_t<REACH_LINEAR>(it, sl, bn, nbins, counter, grid, smem, st);
    }
    return REACH_EINVAL;
}

int onchip_batch_threads() { return BATCH_THREADS; }
size_t onchip_slot_bytes() { return sizeof(Slot); }
size_t onchip_bin_bytes() { return sizeof(Bin); }
size_t onchip_item_bytes() { return sizeof(OnItem); }

}  // namespace reach
