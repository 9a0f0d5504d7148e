// batch.cu -- many uneven MM / CGB queries in one graph launch of persistent
// kernels (reach_batch_*), with the work layout chosen by a small autotuner.
//
// Planning.  Every query becomes an item of 2n components.  An item that fits
// one block (<= 16 components per thread at 512 threads, shared memory for y,
// inputs and derivatives) is given a warp group of ceil(2n / (32 cpt)) warps,
// cpt being the tuned components-per-thread target; items are sorted by their
// critical path (components per thread x RK4 steps) and packed, largest first,
// into bins of at most 16 warps and one block's shared memory.  Larger items
// (up to twice that) run on a two-block cluster.  A task is one cluster item
// or two bins (one per block of the cluster); tasks are handed out largest
// first by an atomic counter (longest-processing-time order).
//
// Autotuning.  cpt in {2, 4, 8, 16} trades parallelism inside an item against
// the number of items running at once; then, with the best cpt, mid-size
// items (from 4096 or from 2048 components) may run on a two-block cluster
// instead of a bin slot (shorter critical path, fewer items at once).  Each
// candidate layout is timed on the real batch with every horizon cut to a few
// steps, and the fastest is kept.
//
// Graph.  Input copies (for host-resident queries), counter and status resets,
// a start stamp, one persistent kernel per (system kind, method) present, and
// the copies of outputs, statuses and completion stamps back are captured once
// into a CUDA graph that reach_batch_run replays.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.cuh"

namespace reach {

constexpr int BIN_WARPS = 16;                 // 512 threads per block
constexpr int64_t ITEM_MAX_BLOCK = (int64_t)QMAX * 512;   // components of a one-block item
constexpr int MAX_NAMED_BARRIERS = 15;        // ids 1..15 (0 is __syncthreads)

struct HostCopy {
    double *user;
    int64_t off, count;   // offset in the pinned / arena buffers (doubles)
};

struct Group {
    int kind, method;
    std::vector<int> items;   // query indices
    void *d_items = nullptr, *d_slots = nullptr, *d_bins = nullptr, *d_tasks = nullptr;
    int ntasks = 0, clusters = 0;
    size_t smem = 0;
};

}  // namespace reach

using namespace reach;

struct reach_batch {
    int64_t count = 0;
    std::vector<reach_query> q;
    std::vector<int64_t> N;
    std::vector<OnItem> items;          // one per query
    std::vector<Group> groups;
    double *d_arena = nullptr, *h_pinned = nullptr;
    int64_t arena = 0;
    std::vector<HostCopy> ins, outs;
    int *d_status = nullptr, *h_status = nullptr;
    int *d_counters = nullptr;
    uint64_t *d_done = nullptr, *h_done = nullptr;   // h_done[count] holds the start stamp
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    int nkernels = 0;
    int cpt = 0;
    int plan_cpt = 16;   // the layout currently planned (tuning tries several)
    int64_t cluster_from = 0;   // tuned: items of this many components or more run on a cluster (0: only too-large ones)
    double tune_ms[6] = {0, 0, 0, 0, 0, 0};
    double create_s = 0;
};

namespace reach {

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static int plan_group(reach_batch *b, Group &g, int cpt, int64_t cluster_from, int64_t n_override,
                      std::vector<char> &dev_mem_keep) {
    (void)dev_mem_keep;
    const int smem_cap = onchip_max_smem() - 64;
    struct Small { int item, warps; int64_t smem, cost; };
    std::vector<Small> small;
    struct Big { int item; int64_t smem, cost; };
    std::vector<Big> big;
    for (int qi : g.items) {
        const OnItem &it = b->items[qi];
        const int64_t comps = 2 * it.n;
        const int64_t N = n_override > 0 ? std::min<int64_t>(n_override, it.N) : it.N;
        const int64_t sm1 = onchip_smem_bytes(it.n, it.nw);
        // a bin slot holds at most cpt components per thread (the kernel is
        // instantiated for that loop length) and at most one block of warps;
        // items from cluster_from components take a cluster when they fit one
        const bool to_cluster = cluster_from > 0 && comps >= cluster_from && comps <= 2 * ITEM_MAX_BLOCK &&
                                cluster_smem_bytes(it.n, it.nw) <= smem_cap;
        if (!to_cluster && comps <= (int64_t)BIN_WARPS * 32 * cpt && sm1 <= smem_cap) {
            const int64_t w = std::max<int64_t>(1, ceil_div(comps, 32LL * cpt));
            small.push_back({qi, (int)w, sm1, ceil_div(comps, 32 * w) * N});
        } else if (comps <= 2 * ITEM_MAX_BLOCK && cluster_smem_bytes(it.n, it.nw) <= smem_cap) {
            big.push_back({qi, cluster_smem_bytes(it.n, it.nw), ceil_div(it.n, 512) * N});
        } else {
            return REACH_EINVAL;   // too large for an on-chip item
        }
    }
    std::sort(small.begin(), small.end(), [](const Small &a, const Small &c) { return a.cost > c.cost; });
    std::vector<BatchSlot> slots;
    std::vector<BatchBin> bins;
    std::vector<int64_t> bin_cost;
    size_t smem = 0;
    {
        int used_w = 0, bars = 0;
        int64_t used_sm = 0, cost = 0;
        BatchBin cur{0, 0};
        for (const Small &s : small) {
            const int need_bar = s.warps > 1 ? 1 : 0;
            if (cur.nslots > 0 && (used_w + s.warps > BIN_WARPS || used_sm + s.smem > smem_cap ||
                                   bars + need_bar > MAX_NAMED_BARRIERS)) {
                bins.push_back(cur);
                bin_cost.push_back(cost);
                smem = std::max(smem, (size_t)used_sm);
                cur = BatchBin{(int)slots.size(), 0};
                used_w = bars = 0;
                used_sm = cost = 0;
            }
            BatchSlot sl;
            sl.item = s.item;
            sl.warp0 = used_w;
            sl.nwarps = s.warps;
            sl.bar = need_bar ? 1 + bars : 0;
            sl.off = used_sm / (int64_t)sizeof(double);
            slots.push_back(sl);
            cur.nslots++;
            used_w += s.warps;
            bars += need_bar;
            used_sm += (s.smem + 255) / 256 * 256;
            cost = std::max(cost, s.cost);
        }
        if (cur.nslots > 0) {
            bins.push_back(cur);
            bin_cost.push_back(cost);
            smem = std::max(smem, (size_t)used_sm);
        }
    }
    // tasks: cluster items, and bins paired in cost order, largest first
    struct T { BatchTask t; int64_t cost; };
    std::vector<T> tasks;
    for (const Big &x : big) {
        tasks.push_back({BatchTask{x.item, {-1, -1}}, x.cost});
        smem = std::max(smem, (size_t)x.smem);
    }
    for (size_t i = 0; i < bins.size(); i += 2) {
        BatchTask t{-1, {(int)i, i + 1 < bins.size() ? (int)(i + 1) : -1}};
        tasks.push_back({t, bin_cost[i]});
    }
    std::stable_sort(tasks.begin(), tasks.end(), [](const T &a, const T &c) { return a.cost > c.cost; });
    std::vector<BatchTask> flat;
    for (const T &t : tasks) flat.push_back(t.t);

    // the big-item field of a task and the slot's item refer to the group's
    // item table, which lists the queries in order
    std::vector<OnItem> its;
    its.reserve(b->items.size());
    for (const OnItem &it : b->items) {
        OnItem c = it;
        if (n_override > 0) c.N = std::min<int64_t>(n_override, it.N);
        its.push_back(c);
    }
    g.ntasks = (int)flat.size();
    g.clusters = (int)std::max<int64_t>(1, std::min<int64_t>(74, g.ntasks));
    g.smem = std::max<size_t>(smem, 16);
    size_t bi = its.size() * sizeof(OnItem), bs = std::max<size_t>(1, slots.size()) * sizeof(BatchSlot);
    size_t bb = std::max<size_t>(1, bins.size()) * sizeof(BatchBin), bt = std::max<size_t>(1, flat.size()) * sizeof(BatchTask);
    char *d = nullptr;
    REACH_CUDA(cudaMalloc(&d, bi + bs + bb + bt));
    g.d_items = d;
    g.d_slots = d + bi;
    g.d_bins = d + bi + bs;
    g.d_tasks = d + bi + bs + bb;
    REACH_CUDA(cudaMemcpy(g.d_items, its.data(), bi, cudaMemcpyHostToDevice));
    if (!slots.empty()) REACH_CUDA(cudaMemcpy(g.d_slots, slots.data(), slots.size() * sizeof(BatchSlot), cudaMemcpyHostToDevice));
    if (!bins.empty()) REACH_CUDA(cudaMemcpy(g.d_bins, bins.data(), bins.size() * sizeof(BatchBin), cudaMemcpyHostToDevice));
    if (!flat.empty()) REACH_CUDA(cudaMemcpy(g.d_tasks, flat.data(), flat.size() * sizeof(BatchTask), cudaMemcpyHostToDevice));
    return REACH_OK;
}

static void free_groups(reach_batch *b) {
    for (Group &g : b->groups) {
        if (g.d_items) cudaFree(g.d_items);
        g.d_items = g.d_slots = g.d_bins = g.d_tasks = nullptr;
    }
}

static int plan_all(reach_batch *b, int cpt, int64_t cluster_from, int64_t n_override) {
    free_groups(b);
    b->plan_cpt = cpt;
    std::vector<char> keep;
    for (Group &g : b->groups) {
        int rc = plan_group(b, g, cpt, cluster_from, n_override, keep);
        if (rc) return rc;
    }
    return REACH_OK;
}

// enqueue one execution of the planned batch on `st`
static int enqueue(reach_batch *b, cudaStream_t st, bool with_copies) {
    int rc;
    if (with_copies) {
        for (const HostCopy &c : b->ins)
            REACH_CUDA(cudaMemcpyAsync(b->d_arena + c.off, b->h_pinned + c.off, c.count * sizeof(double),
                                       cudaMemcpyHostToDevice, st));
    }
    REACH_CUDA(cudaMemsetAsync(b->d_counters, 0, b->groups.size() * sizeof(int), st));
    REACH_CUDA(cudaMemsetAsync(b->d_status, 0, b->count * sizeof(int), st));
    if ((rc = onchip_launch_stamp(b->d_done + b->count, st))) return rc;
    for (size_t k = 0; k < b->groups.size(); ++k) {
        Group &g = b->groups[k];
        if ((rc = onchip_launch_batch(g.kind, g.method, b->plan_cpt, g.d_items, g.d_slots, g.d_bins, g.d_tasks, g.ntasks,
                                      b->d_counters + k, b->d_done, g.clusters, g.smem, st)))
            return rc;
    }
    if (with_copies) {
        for (const HostCopy &c : b->outs)
            REACH_CUDA(cudaMemcpyAsync(b->h_pinned + c.off, b->d_arena + c.off, c.count * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
        REACH_CUDA(cudaMemcpyAsync(b->h_status, b->d_status, b->count * sizeof(int), cudaMemcpyDeviceToHost, st));
        REACH_CUDA(cudaMemcpyAsync(b->h_done, b->d_done, (b->count + 1) * sizeof(uint64_t),
                                   cudaMemcpyDeviceToHost, st));
    }
    return REACH_OK;
}

static void destroy(reach_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    free_groups(b);
    if (b->d_arena) cudaFree(b->d_arena);
    if (b->h_pinned) cudaFreeHost(b->h_pinned);
    if (b->d_status) cudaFree(b->d_status);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->d_done) cudaFree(b->d_done);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->h_done) cudaFreeHost(b->h_done);
    delete b;
}

}  // namespace reach

extern "C" int reach_batch_create(const reach_query *queries, int64_t count, int flags, reach_batch **out) {
    if (!out || !queries || count < 1 || count > (1 << 24)) return REACH_EINVAL;
    const auto created0 = std::chrono::steady_clock::now();
    *out = nullptr;
    reach_batch *b = new (std::nothrow) reach_batch();
    if (!b) return REACH_ENOMEM;
    b->count = count;
    b->q.assign(queries, queries + count);
    int rc = REACH_OK;
    b->items.resize(count);
    b->N.resize(count);
    for (int64_t i = 0; i < count; ++i) {
        const reach_query &q = queries[i];
        if (!q.sys || q.sys->kind == REACH_QUAD || (q.sys->kind == REACH_TRAFFIC && q.sys->prm[5] != 0.0) || (q.method != MM && q.method != CGB) || !q.x0_lo || !q.x0_hi || !q.lo || !q.hi ||
            (q.sys->nw > 0 && (!q.w_lo || !q.w_hi))) {
            destroy(b);
            return REACH_EINVAL;
        }
        int64_t N;
        if ((rc = nsteps(q.t_final, q.dt, &N)) || (rc = check_host_box(q.x0_lo, q.x0_hi, q.sys->n)) ||
            (rc = check_host_box(q.w_lo, q.w_hi, q.sys->nw)) || N < 1) {
            destroy(b);
            return rc ? rc : REACH_EINVAL;
        }
        b->N[i] = N;
    }
    // pass 1: arena offsets of host-resident vectors (32-double aligned)
    struct Where { int64_t off; bool host; };
    std::vector<Where> where(6 * count);
    for (int64_t i = 0; i < count; ++i) {
        const reach_query &q = queries[i];
        const double *p[6] = {q.x0_lo, q.x0_hi, q.w_lo, q.w_hi, q.lo, q.hi};
        const int64_t cnt[6] = {q.sys->n, q.sys->n, q.sys->nw, q.sys->nw, q.sys->n, q.sys->n};
        for (int k = 0; k < 6; ++k) {
            Where &w = where[6 * i + k];
            w.host = cnt[k] > 0 && p[k] && !is_device_ptr(p[k]);
            w.off = b->arena;
            if (w.host) {
                (k < 4 ? b->ins : b->outs).push_back(HostCopy{(double *)p[k], b->arena, cnt[k]});
                b->arena += (cnt[k] + 31) / 32 * 32;
            }
        }
    }
    if (pool_init() || cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        destroy(b);
        return REACH_ECUDA;
    }
    cudaError_t e = cudaSuccess;
    if (b->arena > 0) {
        e = cudaMalloc(&b->d_arena, b->arena * sizeof(double));
        if (e == cudaSuccess) e = cudaMallocHost(&b->h_pinned, b->arena * sizeof(double));
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, count * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_done, (count + 1) * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, count * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_done, (count + 1) * sizeof(uint64_t));
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "reach_batch_create");
        destroy(b);
        return rc;
    }
    // pass 2: item records with device addresses
    for (int64_t i = 0; i < count; ++i) {
        const reach_query &q = queries[i];
        const double *p[6] = {q.x0_lo, q.x0_hi, q.w_lo, q.w_hi, q.lo, q.hi};
        const double *d[6];
        for (int k = 0; k < 6; ++k) d[k] = where[6 * i + k].host ? b->d_arena + where[6 * i + k].off : p[k];
        OnItem &it = b->items[i];
        it.n = q.sys->n;
        it.nw = q.sys->nw;
        it.kind = q.sys->kind;
        it.method = q.method;
        it.prm = q.sys->dprm;
        it.N = b->N[i];
        it.h = q.dt;
        it.one = 1.0;
        it.nzero = -0.0;
        it.hh = 0.5 * q.dt;
        it.h6 = q.dt / 6.0;
        it.xlo = d[0]; it.xhi = d[1]; it.wlo = d[2]; it.whi = d[3];
        it.lo = (double *)d[4]; it.hi = (double *)d[5];
        it.status = b->d_status + i;
    }
    // the inputs go to the device once now, so that tuning runs on real data
    for (const HostCopy &c : b->ins) memcpy(b->h_pinned + c.off, c.user, c.count * sizeof(double));
    for (const HostCopy &c : b->ins)
        if (cudaMemcpyAsync(b->d_arena + c.off, b->h_pinned + c.off, c.count * sizeof(double),
                            cudaMemcpyHostToDevice, b->cap) != cudaSuccess) {
            destroy(b);
            return REACH_ECUDA;
        }
    // groups by (kind, method)
    for (int64_t i = 0; i < count; ++i) {
        const OnItem &it = b->items[i];
        Group *g = nullptr;
        for (Group &x : b->groups) if (x.kind == it.kind && x.method == it.method) g = &x;
        if (!g) {
            b->groups.push_back(Group{});
            g = &b->groups.back();
            g->kind = it.kind;
            g->method = it.method;
        }
        g->items.push_back((int)i);
    }
    if (cudaMalloc(&b->d_counters, b->groups.size() * sizeof(int)) != cudaSuccess) {
        destroy(b);
        return REACH_ENOMEM;
    }

    // autotune the layout on short horizons: first the components-per-thread
    // target, then, with it, whether mid-size items (from 2048 or 4096
    // components) run on a two-block cluster instead of a bin slot
    const int cands[4] = {2, 4, 8, 16};
    const int64_t cfrom[2] = {4096, 2048};
    int best = (int)(opt_batch_cpt() > 0 ? opt_batch_cpt() : 8);
    int64_t best_from = opt_batch_cluster_from();
    if (!(flags & REACH_BATCH_NO_AUTOTUNE) && opt_batch_cpt() == 0) {
        int64_t maxN = *std::max_element(b->N.begin(), b->N.end());
        int64_t nshort = std::max<int64_t>(1, std::min<int64_t>(maxN, 24));
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        double best_ms = 1e300;
        auto time_layout = [&](int cpt, int64_t from, double *ms_out) -> int {
            int r = plan_all(b, cpt, from, nshort);
            if (r) return r;
            // warm once, then time
            if ((r = enqueue(b, b->cap, false))) return r;
            cudaEventRecord(e0, b->cap);
            if ((r = enqueue(b, b->cap, false))) return r;
            cudaEventRecord(e1, b->cap);
            if (cudaEventSynchronize(e1) != cudaSuccess) return REACH_ECUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            *ms_out = ms;
            return REACH_OK;
        };
        for (int c = 0; c < 4 && !rc; ++c) {
            rc = time_layout(cands[c], 0, &b->tune_ms[c]);
            if (!rc && b->tune_ms[c] < best_ms) { best_ms = b->tune_ms[c]; best = cands[c]; }
        }
        // only if some item lies in a candidate's range
        int64_t max_small = 0;
        for (const OnItem &it : b->items)
            if (2 * it.n <= (int64_t)BIN_WARPS * 32 * best) max_small = std::max<int64_t>(max_small, 2 * it.n);
        for (int c = 0; c < 2 && !rc && opt_batch_cluster_from() == 0; ++c) {
            if (max_small < cfrom[c]) continue;
            rc = time_layout(best, cfrom[c], &b->tune_ms[4 + c]);
            if (!rc && b->tune_ms[4 + c] < best_ms) { best_ms = b->tune_ms[4 + c]; best_from = cfrom[c]; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) { destroy(b); return rc; }
    }
    b->cpt = best;
    b->cluster_from = best_from;
    if ((rc = plan_all(b, best, best_from, 0))) { destroy(b); return rc; }

    // capture the whole run once
    cudaGraph_t graph = nullptr;
    int64_t launches_before = reach_kernel_launches();
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        destroy(b);
        return REACH_ECUDA;
    }
    rc = enqueue(b, b->cap, true);
    cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
    b->nkernels = (int)(reach_kernel_launches() - launches_before);
    count_launch(-b->nkernels);   // captured, not launched
    if (rc || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        destroy(b);
        return rc ? rc : cuda_fail(ce, "capture");
    }
    ce = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        destroy(b);
        return cuda_fail(ce, "cudaGraphInstantiate");
    }
    b->create_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - created0).count();
    *out = b;
    return REACH_OK;
}

extern "C" int reach_batch_run(reach_batch *b, void *stream, int *status, double *finish_s) {
    if (!b) return REACH_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    for (const HostCopy &c : b->ins) memcpy(b->h_pinned + c.off, c.user, c.count * sizeof(double));
    REACH_CUDA(cudaGraphLaunch(b->exec, st));
    count_launch(b->nkernels);
    REACH_CUDA(cudaStreamSynchronize(st));
    for (const HostCopy &c : b->outs) memcpy(c.user, b->h_pinned + c.off, c.count * sizeof(double));
    int worst = REACH_OK;
    for (int64_t i = 0; i < b->count; ++i) {
        int s = b->h_status[i];
        int code = (s & ST_BADINPUT) ? REACH_EINVAL
                   : (s & ST_TIMEOUT) ? REACH_ETIMEOUT
                   : (s & (ST_NONFINITE | ST_NEGRADIUS)) ? REACH_ENONFINITE : REACH_OK;
        if (status) status[i] = code;
        if (code && !worst) worst = code;
        if (finish_s) finish_s[i] = (double)(int64_t)(b->h_done[i] - b->h_done[b->count]) * 1e-9;
    }
    return worst;
}

extern "C" int reach_batch_info(const reach_batch *b, int64_t *cpt, int64_t *kernels, double *tune_ms) {
    if (!b) return REACH_EINVAL;
    if (cpt) *cpt = b->cpt;
    if (kernels) *kernels = b->nkernels;
    if (tune_ms) for (int i = 0; i < 4; ++i) tune_ms[i] = b->tune_ms[i];
    return REACH_OK;
}

extern "C" int reach_batch_layout(const reach_batch *b, int64_t *cpt, int64_t *cluster_from, double *create_s,
                                  double *tune_ms) {
    if (!b) return REACH_EINVAL;
    if (cpt) *cpt = b->cpt;
    if (cluster_from) *cluster_from = b->cluster_from;
    if (create_s) *create_s = b->create_s;
    if (tune_ms) for (int i = 0; i < 6; ++i) tune_ms[i] = b->tune_ms[i];
    return REACH_OK;
}

extern "C" int reach_batch_destroy(reach_batch *b) {
    if (!b) return REACH_EINVAL;
    cudaStreamSynchronize(b->cap);
    destroy(b);
    return REACH_OK;
}
