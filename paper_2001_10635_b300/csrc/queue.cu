// queue.cu -- the device work queue (reach_queue_*): MM / CGB queries small
// enough for one block, run by a persistent kernel as they arrive.
//
// Host side of the protocol (the kernel is queue_kernel, onchip_kernels.cuh):
//   submit   stages host vectors in a page-locked arena the GPU reads and
//            writes directly (no copy calls, no stream synchronisation), writes
//            the item into the kind's ring and publishes it by advancing the
//            ring's tail (a release store; the kernel loads the tail with
//            acquire semantics); then makes sure enough blocks are running
//   blocks   the controller launches the kind's persistent kernel with as many
//            blocks as there are published items without a block to run them,
//            up to the queue's block limit over all kinds; blocks that find no
//            work for the idle limit leave by themselves
//   wait     polls the item's done word in page-locked memory (bounded by the
//            caller's limit), then copies a staged result to the caller
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.cuh"
#include "queue.cuh"

namespace reach {

template <int SYS>
int queue_launch_k(const QueueArgs &, int, size_t, cudaStream_t);

constexpr int QKINDS = 5;            // traffic, KS, oscillator, linear, heat (the reach_kind values 0..4)
constexpr int QCAP = 2048;           // ring slots per kind: items in flight at once
constexpr int QLAUNCHES = 32;        // launches of the persistent kernel alive at once
constexpr int QMAX_BLOCKS = 256;     // blocks of one launch

using QClock = std::chrono::steady_clock;

// per-kind ring in mapped page-locked memory
struct QRingHost {
    QueueItem ring[QCAP];
    long long done[QCAP];
    int hstatus[QCAP];
    long long tail;
    long long pad[7];
};
struct QHost {
    QRingHost k[QKINDS];
    int stop;
    int pad[15];
    int exited[QLAUNCHES][QMAX_BLOCKS];
};
struct QDev {
    unsigned long long head[QKINDS];
    int dstatus[QKINDS][QCAP];
};

struct QLaunch {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int kind = -1, blocks = 0;
    bool busy = false;   // launched and not yet seen finished
};

struct QPending {
    int kind;
    int slot;
    int64_t seq;
    int64_t n;
    int64_t arena_off = -1, arena_len = 0;
    double *user_lo = nullptr, *user_hi = nullptr;   // host outputs to fill from the arena
    const double *st_lo = nullptr, *st_hi = nullptr;
};

// first-fit allocator over the arena (units: doubles)
struct Arena {
    std::map<int64_t, int64_t> free_;   // offset -> length
    void init(int64_t len) { free_.clear(); if (len > 0) free_[0] = len; }
    int64_t take(int64_t len) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < len) continue;
            const int64_t off = it->first, rest = it->second - len;
            free_.erase(it);
            if (rest > 0) free_[off + len] = rest;
            return off;
        }
        return -1;
    }
    void give(int64_t off, int64_t len) {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace reach

using namespace reach;

struct reach_queue {
    int device = 0;
    int max_blocks = 0;
    unsigned long long idle_ns = 0;
    std::mutex mu;
    QHost *hh = nullptr, *hd = nullptr;     // mapped control block: host and device addresses
    QDev *dev = nullptr;
    double *arena_h = nullptr, *arena_d = nullptr;
    int64_t arena_len = 0;
    Arena arena;
    QLaunch launches[QLAUNCHES];
    int64_t published[QKINDS] = {0, 0, 0, 0, 0};
    std::vector<int64_t> inflight[QKINDS];  // tickets of published items not yet waited for
    std::unordered_map<int64_t, QPending> pending;
    int64_t next_ticket = 1;
    int last_exit = REACH_OK;               // how the most recently finished launch ended
    int64_t launched_blocks = 0;
};

namespace reach {

static int64_t r32(int64_t v) { return (v + 31) / 32 * 32; }

bool queue_accepts(const reach_system *s, int method) {
    if (!s || (method != MM && method != CGB)) return false;
    if (s->kind < 0 || s->kind >= QKINDS) return false;
    if (s->kind == REACH_TRAFFIC && s->prm[5] != 0.0) return false;   // outward rounding: streaming kernel only
    if (2 * s->n > QUEUE_MAX_COMPONENTS) return false;
    return onchip_smem_bytes(s->n, s->nw) <= onchip_max_smem() - 1024;
}

// shared memory of a kind's launch: its largest accepted item
static size_t queue_smem(int kind) {
    const int64_t n = QUEUE_MAX_COMPONENTS / 2;
    int64_t b = 0;
    switch (kind) {
    case REACH_TRAFFIC: b = onchip_smem_bytes(n, 1); break;
    case REACH_OSC: b = onchip_smem_bytes(n, n / 2); break;
    case REACH_LINEAR: b = onchip_smem_bytes(256, 256); break;
    default: b = onchip_smem_bytes(n, 0); break;
    }
    return (size_t)std::min<int64_t>(b, onchip_max_smem() - 1024);
}

static int launch_kind(reach_queue *q, QLaunch &L, int kind, int blocks) {
    QueueArgs a;
    a.ring = q->hd->k[kind].ring;
    a.tail = &q->hd->k[kind].tail;
    a.stop = &q->hd->stop;
    a.done = q->hd->k[kind].done;
    a.hstatus = q->hd->k[kind].hstatus;
    const int li = (int)(&L - q->launches);
    for (int b = 0; b < blocks; ++b) ((volatile int *)q->hh->exited[li])[b] = QEXIT_RUNNING;
    a.exited = q->hd->exited[li];
    a.head = q->dev->head + kind;
    a.dstatus = q->dev->dstatus[kind];
    a.cap = QCAP;
    a.idle_ns = q->idle_ns;
    const size_t smem = queue_smem(kind);
    int rc;
    switch (kind) {
    case REACH_TRAFFIC: rc = queue_launch_k<REACH_TRAFFIC>(a, blocks, smem, L.st); break;
    case REACH_KS: rc = queue_launch_k<REACH_KS>(a, blocks, smem, L.st); break;
    case REACH_OSC: rc = queue_launch_k<REACH_OSC>(a, blocks, smem, L.st); break;
    case REACH_LINEAR: rc = queue_launch_k<REACH_LINEAR>(a, blocks, smem, L.st); break;
    default: rc = queue_launch_k<REACH_HEAT3D>(a, blocks, smem, L.st); break;
    }
    if (rc) return rc;
    REACH_CUDA(cudaEventRecord(L.ev, L.st));
    L.kind = kind;
    L.blocks = blocks;
    L.busy = true;
    q->launched_blocks += blocks;
    return REACH_OK;
}

// blocks of a launch that have not left yet
static int alive_blocks(reach_queue *q, const QLaunch &L) {
    const int li = (int)(&L - q->launches);
    int alive = 0;
    for (int b = 0; b < L.blocks; ++b) alive += ((volatile int *)q->hh->exited[li])[b] == QEXIT_RUNNING;
    return alive;
}

// notice finished launches (caller holds mu)
static void reap(reach_queue *q) {
    for (QLaunch &L : q->launches) {
        if (!L.busy) continue;
        cudaError_t e = cudaEventQuery(L.ev);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) cudaGetLastError();
        const int li = (int)(&L - q->launches);
        int code = QEXIT_STOPPED;
        for (int b = 0; b < L.blocks; ++b)
            if (((volatile int *)q->hh->exited[li])[b] == QEXIT_IDLE) code = QEXIT_IDLE;
        q->last_exit = (e != cudaSuccess) ? REACH_ECUDA : (code == QEXIT_IDLE ? REACH_ETIMEOUT : REACH_OK);
        L.busy = false;
    }
}

// Launch blocks for published items that no running block can take: one
// block per such item, up to the block limit over all kinds (caller holds mu).
static int control(reach_queue *q) {
    reap(q);
    int alive[QKINDS] = {0, 0, 0, 0, 0}, total = 0;
    for (QLaunch &L : q->launches)
        if (L.busy) {
            const int a = alive_blocks(q, L);
            alive[L.kind] += a;
            total += a;
        }
    for (int k = 0; k < QKINDS; ++k) {
        int waiting = 0;
        const QRingHost &R = q->hh->k[k];
        for (int64_t t : q->inflight[k]) {
            const QPending &p = q->pending[t];
            if (((volatile const long long *)R.done)[p.slot] != t) ++waiting;
        }
        int want = std::min(waiting - alive[k], q->max_blocks - total);
        while (want > 0) {
            QLaunch *free_l = nullptr;
            for (QLaunch &L : q->launches)
                if (!L.busy) { free_l = &L; break; }
            if (!free_l) return REACH_OK;   // every launch record in use: later
            const int b = std::min(want, QMAX_BLOCKS);
            int rc = launch_kind(q, *free_l, k, b);
            if (rc) return rc;
            want -= b;
            total += b;
        }
    }
    return REACH_OK;
}

// every published item has raised its done word (caller holds mu)
static bool all_done(reach_queue *q) {
    for (int k = 0; k < QKINDS; ++k)
        for (int64_t t : q->inflight[k])
            if (((volatile const long long *)q->hh->k[k].done)[q->pending[t].slot] != t) return false;
    return true;
}

static void destroy_queue(reach_queue *q) {
    if (!q) return;
    if (q->hh) {
        // submitted queries run to their end first (blocks are relaunched for
        // them if the idle ones have left)
        for (;;) {
            {
                std::lock_guard<std::mutex> lk(q->mu);
                if (all_done(q) || control(q) != REACH_OK) break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
        ((volatile int *)&q->hh->stop)[0] = 1;
    }
    for (QLaunch &L : q->launches) {
        if (L.st) {
            cudaStreamSynchronize(L.st);
            cudaStreamDestroy(L.st);
        }
        if (L.ev) cudaEventDestroy(L.ev);
    }
    if (q->dev) cudaFree(q->dev);
    if (q->hh) cudaFreeHost(q->hh);
    if (q->arena_h) cudaFreeHost(q->arena_h);
    delete q;
}

static int map_status(int bits) {
    if (bits & ST_BADINPUT) return REACH_EINVAL;
    if (bits & ST_TIMEOUT) return REACH_ETIMEOUT;
    if (bits & (ST_NONFINITE | ST_NEGRADIUS)) return REACH_ENONFINITE;
    return REACH_OK;
}

}  // namespace reach

extern "C" int reach_queue_create(int max_blocks, double idle_s, int64_t arena_bytes, reach_queue **out) {
    if (!out) return REACH_EINVAL;
    *out = nullptr;
    if (max_blocks < 1 || max_blocks > QLAUNCHES * QMAX_BLOCKS || !(idle_s > 0.0) || idle_s > 3600.0 ||
        arena_bytes < 0)
        return REACH_EINVAL;
    reach_queue *q = new (std::nothrow) reach_queue();
    if (!q) return REACH_ENOMEM;
    if (cudaGetDevice(&q->device) != cudaSuccess) {
        cudaGetLastError();
        delete q;
        return REACH_ENODEV;
    }
    q->max_blocks = max_blocks;
    q->idle_ns = (unsigned long long)(idle_s * 1e9);
    cudaError_t e = cudaHostAlloc((void **)&q->hh, sizeof(QHost), cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
        memset((void *)q->hh, 0, sizeof(QHost));
        e = cudaHostGetDevicePointer((void **)&q->hd, q->hh, 0);
    }
    q->arena_len = arena_bytes / (int64_t)sizeof(double) / 32 * 32;
    if (e == cudaSuccess && q->arena_len > 0) {
        e = cudaHostAlloc((void **)&q->arena_h, q->arena_len * sizeof(double),
                          cudaHostAllocMapped | cudaHostAllocPortable);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&q->arena_d, q->arena_h, 0);
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&q->dev, sizeof(QDev));
    if (e == cudaSuccess) e = cudaMemset(q->dev, 0, sizeof(QDev));
    int least = 0, greatest = 0;
    if (e == cudaSuccess && cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        greatest = 0;
    }
    // the queue's blocks get SMs ahead of other streams' blocks as they free up
    for (int i = 0; e == cudaSuccess && i < QLAUNCHES; ++i) {
        e = cudaStreamCreateWithPriority(&q->launches[i].st, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->launches[i].ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "reach_queue_create");
        destroy_queue(q);
        return rc;
    }
    q->arena.init(q->arena_len);
    for (int k = 0; k < QKINDS; ++k) q->inflight[k].reserve(QCAP);
    *out = q;
    return REACH_OK;
}

extern "C" int reach_queue_submit(reach_queue *q, const reach_query *qu, int64_t *ticket) {
    if (!q || !qu || !ticket || !qu->sys || !qu->x0_lo || !qu->x0_hi || !qu->lo || !qu->hi) return REACH_EINVAL;
    const reach_system *s = qu->sys;
    if (!queue_accepts(s, qu->method)) return REACH_EINVAL;
    if (s->nw > 0 && (!qu->w_lo || !qu->w_hi)) return REACH_EINVAL;
    int64_t N;
    int rc = nsteps(qu->t_final, qu->dt, &N);
    if (rc) return rc;
    if (N < 1) return REACH_EINVAL;   // a zero horizon is the box itself: nothing to queue
    if ((rc = check_host_box(qu->x0_lo, qu->x0_hi, s->n)) || (rc = check_host_box(qu->w_lo, qu->w_hi, s->nw)))
        return rc;
    const int64_t n = s->n, nw = s->nw;
    const double *src[4] = {qu->x0_lo, qu->x0_hi, qu->w_lo, qu->w_hi};
    const int64_t cnt[4] = {n, n, nw, nw};
    bool host_in[4], host_out[2];
    int64_t need = 0;
    for (int i = 0; i < 4; ++i) {
        host_in[i] = cnt[i] > 0 && !is_device_ptr(src[i]);
        if (host_in[i]) need += r32(cnt[i]);
    }
    host_out[0] = !is_device_ptr(qu->lo);
    host_out[1] = !is_device_ptr(qu->hi);
    for (int i = 0; i < 2; ++i)
        if (host_out[i]) need += r32(n);

    std::lock_guard<std::mutex> lk(q->mu);
    const int kind = s->kind;
    if ((int64_t)q->inflight[kind].size() >= QCAP) return REACH_EADMIT;   // ring full: wait for results first
    QPending p;
    p.kind = kind;
    p.n = n;
    if (need > 0) {
        p.arena_off = q->arena.take(need);
        if (p.arena_off < 0) return REACH_EADMIT;   // no staging space now
        p.arena_len = need;
    }
    int64_t off = p.arena_off;
    const double *dsrc[4];
    for (int i = 0; i < 4; ++i) {
        dsrc[i] = src[i];
        if (host_in[i]) {
            memcpy(q->arena_h + off, src[i], cnt[i] * sizeof(double));
            dsrc[i] = q->arena_d + off;
            off += r32(cnt[i]);
        }
    }
    double *dout[2] = {qu->lo, qu->hi};
    for (int i = 0; i < 2; ++i) {
        if (host_out[i]) {
            (i ? p.user_hi : p.user_lo) = i ? qu->hi : qu->lo;
            (i ? p.st_hi : p.st_lo) = q->arena_h + off;
            dout[i] = q->arena_d + off;
            off += r32(n);
        }
    }
    const int64_t t = q->next_ticket++;
    p.seq = q->published[kind];
    p.slot = (int)(p.seq % QCAP);
    QRingHost &R = q->hh->k[kind];
    QueueItem &item = R.ring[p.slot];
    OnItem &it = item.it;
    it.n = n;
    it.nw = nw;
    it.kind = kind;
    it.method = qu->method;
    it.xlo = dsrc[0]; it.xhi = dsrc[1]; it.wlo = dsrc[2]; it.whi = dsrc[3];
    it.lo = dout[0]; it.hi = dout[1];
    it.prm = s->dprm;
    it.N = N;
    it.h = qu->dt;
    it.one = 1.0;
    it.nzero = -0.0;
    it.hh = 0.5 * qu->dt;
    it.h6 = qu->dt / 6.0;
    it.status = nullptr;
    item.ticket = t;
    // publish: the item and the staged inputs are written before the tail
    std::atomic_thread_fence(std::memory_order_release);
    ((volatile long long *)&R.tail)[0] = p.seq + 1;
    q->published[kind]++;
    q->pending.emplace(t, p);
    q->inflight[kind].push_back(t);
    *ticket = t;
    return control(q);
}

extern "C" int reach_queue_wait(reach_queue *q, int64_t ticket, double timeout_s, int *status) {
    if (!q) return REACH_EINVAL;
    QPending p;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        auto it = q->pending.find(ticket);
        if (it == q->pending.end()) return REACH_EINVAL;
        p = it->second;
    }
    const volatile long long *done = q->hh->k[p.kind].done + p.slot;
    const auto t0 = QClock::now();
    auto last_control = t0;
    const double limit = timeout_s < 0 ? 0.0 : timeout_s;
    for (int spin = 0; *done != ticket; ++spin) {
        const auto now = QClock::now();
        if (std::chrono::duration<double>(now - t0).count() >= limit) return REACH_ETIMEOUT;
        // a block may have left between the publication and its last poll:
        // look again every millisecond
        if (now - last_control > std::chrono::milliseconds(1)) {
            std::lock_guard<std::mutex> lk(q->mu);
            int rc = control(q);
            if (rc) return rc;
            last_control = now;
        }
        if (spin < 2000) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    const int bits = ((volatile const int *)q->hh->k[p.kind].hstatus)[p.slot];
    if (p.user_lo) memcpy(p.user_lo, p.st_lo, p.n * sizeof(double));
    if (p.user_hi) memcpy(p.user_hi, p.st_hi, p.n * sizeof(double));
    {
        std::lock_guard<std::mutex> lk(q->mu);
        if (p.arena_off >= 0) q->arena.give(p.arena_off, p.arena_len);
        std::vector<int64_t> &v = q->inflight[p.kind];
        v.erase(std::find(v.begin(), v.end(), ticket));
        q->pending.erase(ticket);
    }
    if (status) *status = map_status(bits);
    return REACH_OK;
}

extern "C" int reach_queue_start(reach_queue *q, int kind, int blocks) {
    if (!q || kind < 0 || kind >= QKINDS || blocks < 1 || blocks > QMAX_BLOCKS) return REACH_EINVAL;
    std::lock_guard<std::mutex> lk(q->mu);
    reap(q);
    for (QLaunch &L : q->launches)
        if (!L.busy) return launch_kind(q, L, kind, blocks);
    return REACH_EADMIT;
}

extern "C" int reach_queue_join(reach_queue *q, double timeout_s, int *exit_status) {
    if (!q) return REACH_EINVAL;
    const auto t0 = QClock::now();
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(q->mu);
            reap(q);
            bool any = false;
            for (QLaunch &L : q->launches) any |= L.busy;
            if (!any) {
                if (exit_status) *exit_status = q->last_exit;
                return REACH_OK;
            }
        }
        if (std::chrono::duration<double>(QClock::now() - t0).count() >= timeout_s) return REACH_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

extern "C" int reach_queue_stats(reach_queue *q, int64_t *in_flight, int64_t *alive_blocks_out,
                                 int64_t *launched_blocks) {
    if (!q) return REACH_EINVAL;
    std::lock_guard<std::mutex> lk(q->mu);
    reap(q);
    int64_t f = 0, a = 0;
    for (int k = 0; k < QKINDS; ++k) f += (int64_t)q->inflight[k].size();
    for (QLaunch &L : q->launches)
        if (L.busy) a += alive_blocks(q, L);
    if (in_flight) *in_flight = f;
    if (alive_blocks_out) *alive_blocks_out = a;
    if (launched_blocks) *launched_blocks = q->launched_blocks;
    return REACH_OK;
}

extern "C" int reach_queue_destroy(reach_queue *q) {
    if (!q) return REACH_EINVAL;
    destroy_queue(q);
    return REACH_OK;
}
