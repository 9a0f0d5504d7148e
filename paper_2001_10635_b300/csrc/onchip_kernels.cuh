// onchip_kernels.cuh -- kernel templates of the on-chip path (one problem per
// block, one problem per two-block cluster, batched persistent kernel).  Each
// onchip_<kind>.cu instantiates them for one system kind.
#pragma once

#include <cooperative_groups.h>

#include <atomic>

#include "api_internal.cuh"
#include "queue.cuh"

namespace reach {

// ---------------------------------------------------------------- one problem
template <int SYS, int METHOD, int Q>
__global__ void __launch_bounds__(512) onchip_single(OnItem it) {
    extern __shared__ double sm[];
    const int64_t n = it.n;
    GroupSync sync{0, (int)blockDim.x};
    // [yA | yB | yA2 | yB2 | wA | wB]
    onchip_run<SYS, METHOD, Q>(it, sm, sm + n, sm + 2 * n, sm + 3 * n, sm + 4 * n, sm + 4 * n + it.nw, 0, 2 * n,
                               (int)threadIdx.x, (int)blockDim.x, sync);
}

template <int SYS, int METHOD, int Q>
static int launch_single_q(const OnItem &it, int threads, cudaStream_t st) {
    int64_t smem = onchip_smem_bytes(it.n, it.nw);
    static std::atomic<bool> attr_set{false};   // idempotent: a second setter is harmless
    if (!attr_set.load()) {
        int rc = allow_max_dynamic_smem((const void *)onchip_single<SYS, METHOD, Q>);
        if (rc) return rc;
        attr_set.store(true);
    }
    onchip_single<SYS, METHOD, Q><<<1, threads, (size_t)smem, st>>>(it);
    REACH_LAUNCHED("onchip_single");
    return REACH_OK;
}

// the smallest components-per-thread loop that covers 2n components
template <int SYS, int METHOD>
static int launch_single_t(const OnItem &it, int threads, cudaStream_t st) {
    const int64_t per = (2 * it.n + threads - 1) / threads;
    if (per <= 1) return launch_single_q<SYS, METHOD, 1>(it, threads, st);
    if (per <= 2) return launch_single_q<SYS, METHOD, 2>(it, threads, st);
    if (per <= 4) return launch_single_q<SYS, METHOD, 4>(it, threads, st);
    if (per <= 8) return launch_single_q<SYS, METHOD, 8>(it, threads, st);
    return launch_single_q<SYS, METHOD, QMAX>(it, threads, st);
}

template <int SYS>
int onchip_single_k(const OnItem &it, int threads, cudaStream_t st) {
    return it.method == MM ? launch_single_t<SYS, MM>(it, threads, st) : launch_single_t<SYS, CGB>(it, threads, st);
}

// ---------------------------------------------------------------- clusters
// Problems with 2n > QMAX * 512 components do not fit one block: a cluster of
// two blocks runs them, block r holding half r of the state (and its inputs
// and derivatives) in its own shared memory and reading the other half
// through distributed shared memory; barriers are cluster barriers.
namespace cg = cooperative_groups;

struct ClusterSync {
    __device__ __forceinline__ void operator()() const { cg::this_cluster().sync(); }
};


// one problem on the calling cluster of two blocks (all threads of both)
template <int SYS, int METHOD>
__device__ __forceinline__ void cluster_item(const OnItem &it, double *sm) {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    const int64_t n = it.n;
    // per block [y | y2 | w]: this block's half in both stage buffers
    double *y = sm, *y2 = sm + n, *w = sm + 2 * n;
    double *other = cl.map_shared_rank(y, rank ^ 1u), *other2 = cl.map_shared_rank(y2, rank ^ 1u);
    double *yA = rank == 0 ? y : other, *yB = rank == 0 ? other : y;
    double *yA2 = rank == 0 ? y2 : other2, *yB2 = rank == 0 ? other2 : y2;
    // the lower / center block uses wA, the upper / radius block wB
    onchip_run<SYS, METHOD, QMAX>(it, yA, yB, yA2, yB2, w, w, rank * n, (rank + 1) * n, (int)threadIdx.x,
                                  (int)blockDim.x, ClusterSync{});
}


template <int SYS, int METHOD>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512, 1) onchip_single_cluster(OnItem it) {
    extern __shared__ double sm[];
    cluster_item<SYS, METHOD>(it, sm);
    cg::this_cluster().sync();   // no block leaves while the other may still read its memory
}

template <int SYS, int METHOD>
static int launch_cluster_t(const OnItem &it, cudaStream_t st) {
    static std::atomic<bool> attr_set{false};   // idempotent: a second setter is harmless
    if (!attr_set.load()) {
        int rc = allow_max_dynamic_smem((const void *)onchip_single_cluster<SYS, METHOD>);
        if (rc) return rc;
        attr_set.store(true);
    }
    onchip_single_cluster<SYS, METHOD><<<2, 512, (size_t)cluster_smem_bytes(it.n, it.nw), st>>>(it);
    REACH_LAUNCHED("onchip_single_cluster");
    return REACH_OK;
}

template <int SYS>
int onchip_cluster_k(const OnItem &it, cudaStream_t st) {
    return it.method == MM ? launch_cluster_t<SYS, MM>(it, st) : launch_cluster_t<SYS, CGB>(it, st);
}

// ---------------------------------------------------------------- batch
// The batched persistent kernel runs on clusters of two blocks of 512
// threads.  Its work list is a sequence of tasks, largest first, taken from a
// global counter: a task is either one large problem spanning the cluster, or
// one bin per block.  A bin is up to 16 slots, each a problem run by a
// contiguous range of warps with its own named barrier and shared-memory
// region.  Each problem records the global time at which it completed.
struct Slot {
    int item, warp0, nwarps, bar;
    int64_t off;   // shared-memory offset (doubles)
};
struct Bin {
    int slot0, nslots;
};
struct Task {
    int big;          // >= 0: item index run by the whole cluster
    int bin[2];       // otherwise: bin of block 0 / block 1 (-1: none)
};


template <int SYS, int METHOD, int Q>
__device__ __forceinline__ void run_bin(const OnItem *__restrict__ items, const Slot *__restrict__ slots,
                                        const Bin &bn, double *sm, uint64_t *done) {
    const int warp = threadIdx.x >> 5;
    for (int s = bn.slot0; s < bn.slot0 + bn.nslots; ++s) {
        const Slot sl = slots[s];
        if (warp < sl.warp0 || warp >= sl.warp0 + sl.nwarps) continue;
        const OnItem &it = items[sl.item];
        double *y = sm + sl.off;
        const int64_t n = it.n;
        GroupSync sync{sl.bar, sl.nwarps * 32};
        const int gt = (int)threadIdx.x - sl.warp0 * 32, gs = sl.nwarps * 32;
        // [yA | yB | wA | wB | yA2 | yB2]
        double *w = y + 2 * n, *y2 = w + 2 * it.nw;
        onchip_run<SYS, METHOD, Q>(it, y, y + n, y2, y2 + n, w, w + it.nw, 0, 2 * n, gt, gs, sync);
        if (gt == 0) done[sl.item] = global_ns();
        break;
    }
}

template <int SYS, int METHOD, int Q>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(BATCH_THREADS, 1)
onchip_batch(const OnItem *__restrict__ items, const Slot *__restrict__ slots, const Bin *__restrict__ bins,
             const Task *__restrict__ tasks, int ntasks, int *counter, uint64_t *done) {
    extern __shared__ double sm[];
    __shared__ int cur;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) cur = atomicAdd(counter, 1);
        cl.sync();
        const int t = *cl.map_shared_rank(&cur, 0u);
        cl.sync();   // both blocks hold t before block 0 may take the next task
        if (t >= ntasks) break;
        const Task tk = tasks[t];
        if (tk.big >= 0) {
            cluster_item<SYS, METHOD>(items[tk.big], sm);
            if (rank == 0 && threadIdx.x == 0) done[tk.big] = global_ns();
        } else if (tk.bin[rank] >= 0) {
            run_bin<SYS, METHOD, Q>(items, slots, bins[tk.bin[rank]], sm, done);
        }
        cl.sync();   // the task is over in both blocks before either reuses memory
    }
}

template <int SYS, int METHOD, int Q>
static int launch_batch_t(const void *items, const void *slots, const void *bins, const void *tasks, int ntasks,
                          int *counter, uint64_t *done, int clusters, size_t smem, cudaStream_t st) {
    static std::atomic<bool> attr_set{false};   // idempotent: a second setter is harmless
    if (!attr_set.load()) {
        int rc = allow_max_dynamic_smem((const void *)onchip_batch<SYS, METHOD, Q>);
        if (rc) return rc;
        attr_set.store(true);
    }
    onchip_batch<SYS, METHOD, Q><<<2 * clusters, BATCH_THREADS, smem, st>>>((const OnItem *)items, (const Slot *)slots,
                                                                 (const Bin *)bins, (const Task *)tasks, ntasks,
                                                                 counter, done);
    REACH_LAUNCHED("onchip_batch");
    return REACH_OK;
}

// Q: the batch's components-per-thread target (the autotuned layout), which
// bounds the components each thread of a bin slot holds
template <int SYS>
int onchip_batch_k(int method, int q, const void *items, const void *slots, const void *bins, const void *tasks,
                   int ntasks, int *counter, uint64_t *done, int clusters, size_t smem, cudaStream_t st) {
#define REACH_BQ(Q)                                                                                             \
    if (q <= Q)                                                                                                 \
        return method == MM                                                                                     \
                   ? launch_batch_t<SYS, MM, Q>(items, slots, bins, tasks, ntasks, counter, done, clusters, smem, st) \
                   : launch_batch_t<SYS, CGB, Q>(items, slots, bins, tasks, ntasks, counter, done, clusters, smem, st);
    REACH_BQ(2)
    REACH_BQ(4)
    REACH_BQ(8)
    REACH_BQ(QMAX)
#undef REACH_BQ
    return REACH_EINVAL;
}


// ---------------------------------------------------------------- device work queue
// Persistent kernel of the work queue (queue.cuh, queue.cu): each block claims
// one published item at a time from the kind's ring (a compare-and-swap on
// the device head, so no item is claimed twice and none is lost), runs it
// with the same whole-horizon device code as onchip_single, and signals its
// completion in mapped host memory.  Every wait is bounded: a block with no
// item for idle_ns leaves (exit word QEXIT_IDLE), and one asked to stop
// leaves at its next idle poll (QEXIT_STOPPED).

// load at system scope with acquire semantics: the host writes an item before
// it advances the tail past it
__device__ __forceinline__ long long ld_acquire_sys(const long long *p) {
    long long v;
    asm volatile("ld.acquire.sys.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <int SYS, int METHOD>
__device__ __forceinline__ void queue_run(const OnItem &it, double *sm, int active) {
    const int64_t n = it.n;
    double *yA = sm, *yB = sm + n, *yA2 = sm + 2 * n, *yB2 = sm + 3 * n, *wA = sm + 4 * n, *wB = wA + it.nw;
    // the first `active` threads run the item: barrier 1 over them (a warp
    // syncs itself), so that the other warps wait at the block barrier
    GroupSync sync{1, active};
    const int64_t comps = 2 * n;
    const int t = (int)threadIdx.x;
    if (comps <= active) onchip_run<SYS, METHOD, 1>(it, yA, yB, yA2, yB2, wA, wB, 0, comps, t, active, sync);
    else if (comps <= 4 * active) onchip_run<SYS, METHOD, 4>(it, yA, yB, yA2, yB2, wA, wB, 0, comps, t, active, sync);
    else onchip_run<SYS, METHOD, QMAX>(it, yA, yB, yA2, yB2, wA, wB, 0, comps, t, active, sync);
}

template <int SYS>
__global__ void __launch_bounds__(QUEUE_THREADS, 1) queue_kernel(QueueArgs a) {
    extern __shared__ double sm[];
    __shared__ long long claimed;
    __shared__ QueueItem cur;
    unsigned long long since = global_ns();
    int code = QEXIT_IDLE;
    for (;;) {
        if (threadIdx.x == 0) {
            long long c = -1;
            unsigned ns = 256;
            for (;;) {
                const long long t = ld_acquire_sys(a.tail);
                const unsigned long long h = *(volatile unsigned long long *)a.head;
                if ((long long)h < t) {
                    if (atomicCAS(a.head, h, h + 1) == h) { c = (long long)h; break; }
                    continue;   // another block took item h: try the next one at once
                }
                if (*(volatile const int *)a.stop) { c = -QEXIT_STOPPED; break; }
                if (global_ns() - since > a.idle_ns) { c = -QEXIT_IDLE; break; }
                __nanosleep(ns);
                if (ns < 8192) ns *= 2;
            }
            if (c >= 0) {
                const int slot = (int)(c % a.cap);
                cur = a.ring[slot];
                a.dstatus[slot] = 0;
                __threadfence();
            }
            claimed = c;
        }
        __syncthreads();
        const long long c = claimed;
        if (c < 0) {
            code = (int)-c;
            break;
        }
        const int slot = (int)(c % a.cap);
        OnItem it = cur.it;
        it.status = a.dstatus + slot;
        const int64_t comps = 2 * it.n;
        const int active = comps < QUEUE_THREADS ? (int)((comps + 31) / 32 * 32) : QUEUE_THREADS;
        if ((int)threadIdx.x < active) {
            if (it.method == MM) queue_run<SYS, MM>(it, sm, active);
            else queue_run<SYS, CGB>(it, sm, active);
        }
        // each thread's results reach host memory before the block signals
        __threadfence_system();
        __syncthreads();
        if (threadIdx.x == 0) {
            a.hstatus[slot] = atomicOr(a.dstatus + slot, 0);
            __threadfence_system();
            *(volatile long long *)(a.done + slot) = cur.ticket;
        }
        since = global_ns();
    }
    if (threadIdx.x == 0) {
        __threadfence_system();
        *(volatile int *)(a.exited + blockIdx.x) = code;
    }
}

template <int SYS>
int queue_launch_k(const QueueArgs &a, int blocks, size_t smem, cudaStream_t st) {
    static std::atomic<bool> attr_set{false};   // idempotent: a second setter is harmless
    if (!attr_set.load()) {
        int rc = allow_max_dynamic_smem((const void *)queue_kernel<SYS>);
        if (rc) return rc;
        attr_set.store(true);
    }
    queue_kernel<SYS><<<blocks, QUEUE_THREADS, smem, st>>>(a);
    REACH_LAUNCHED("queue_kernel");
    return REACH_OK;
}

}  // namespace reach
