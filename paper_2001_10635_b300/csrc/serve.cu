// serve.cu -- continuous-batching request loop (reach_server_*).
//
// The paper serves reachability problems to remote tools (Sec. 1, the
// pFaces REST interface); here that purpose becomes an in-process server:
// requests of any kind, size, method and horizon are submitted as they
// arrive, admitted as capacity frees up, and run concurrently.
//
//   submit     appends the request to the waiting list (never blocks on GPU work)
//   dispatch   whenever a request arrives or one finishes, the waiting list is
//              scanned in arrival order and every request that can start does:
//   queue      an MM / CGB request small enough for one block (2n <= 8192) joins
//              the server's device work queue (queue.cu): the blocks of a
//              persistent kernel take it as soon as it is published, beside
//              whatever else runs, with no launch, copy call or synchronisation
//              of its own; requests join while others are on the GPU
//              (continuous batching).  Requests up to REACH_OPT_SERVE_QUEUE_N
//              cells (default 512) go there: beyond that one block takes
//              longer per RK4 step than a streaming kernel spread over every SM
//   slots      every other request needs a free slot and its device footprint
//              must fit in what is left of the budget (first fit, so small
//              requests pass a large one that waits for memory); a slot is a
//              worker thread with its own CUDA streams that copies the
//              request's host vectors to the device, runs it through the
//              ordinary entry points and copies the box back, so copies and
//              kernels of different requests overlap
//   gate       a wide request (2^20 or more state components per step) fills
//              the GPU alone; by default it computes alone, since sharing the
//              GPU finishes both requests late: it passes the compute gate
//              when no other slot request computes (light ones included), and
//              none passes beside it except light ones (REACH_OPT_SERVE_LIGHT
//              components per step or fewer, on the least stream priority, so
//              their blocks only fill SMs the wide request leaves free) that
//              reach the gate while it computes and no other wide request
//              waits; waiters pass in arrival order.  So no request waits for
//              one that reached the gate after it: a light request that
//              backfills is never passed by a later wide one, and one that
//              arrives while a wide request waits queues behind it.
//              REACH_OPT_SERVE_MAX_WIDE can also cap wide requests at
//              admission.
//   priority   otherwise a slot request runs on a stream whose priority falls
//              with its work (components per step x steps: the greatest below
//              2^30 component updates, one level lower per factor 4 above):
//              the block scheduler hands SMs freed by a large request's short
//              blocks to a small request first
//   wait       bounded: returns REACH_ETIMEOUT when the request has not finished
//              within the caller's limit
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.cuh"

using Clock = std::chrono::steady_clock;

namespace reach {

struct Job {
    int64_t ticket;
    reach_request r;
    int64_t bytes;
    int level = 0;   // stream priority level, 0 = greatest
    Clock::time_point submitted, started, finished;
    int status = REACH_OK;
    bool done = false;
    bool queue_ok = false;   // may run on the device work queue
    bool wide = false;       // its kernels fill the GPU alone
    bool light = false;      // its kernels hold few SMs: it may backfill beside a wide request
    bool in_queue = false;   // submitted to it: qticket is its ticket there
    int64_t qticket = 0;
};

}  // namespace reach

using namespace reach;

struct reach_server {
    int device = 0;
    int64_t budget = 0, in_use = 0, peak = 0;
    int64_t next_ticket = 1;
    int nslots = 0, idle = 0;
    int nlevels = 1;   // stream priority levels (greatest first)
    int prio_mode = 0;  // 0: by work (small first), 1: by arrival, 2: one level, 3: by work (large first)
    int next_level = 0; // arrival order: the level of the next request to start
    int prio_greatest = 0;
    bool stopping = false;
    std::mutex mu;
    std::condition_variable work_cv, done_cv;
    std::deque<Job *> waiting;      // arrival order
    std::deque<Job *> admitted;     // ready for a slot
    std::unordered_map<int64_t, Job *> jobs;
    std::vector<std::thread> workers;
    int64_t n_admitted = 0, n_done = 0, n_rejected = 0;
    reach_queue *queue = nullptr;   // device work queue of small MM / CGB requests (null: none)
    int64_t queue_n = 0;            // cells up to which a request always takes the queue
    int64_t n_queued = 0;           // requests that went to the queue
    int queue_running = 0;          // requests on the queue and not yet finished
    int slot_running = 0;           // requests running on slots
    int wide_running = 0;           // wide requests admitted and not finished
    int max_wide = 0;               // wide requests at once (0: no limit)
    bool wide_exclusive = true;     // a wide request computes with no other slot request
    int64_t light_components = 0;   // requests of at most this many components per step backfill
    int computing = 0, wide_computing = 0;   // slot requests past the compute gate
    int wide_waiting = 0;           // wide requests waiting at the compute gate
    std::set<int64_t> gate;         // tickets of slot requests staged and waiting to compute
    std::condition_variable gate_cv;
};

namespace reach {

static int64_t mc_footprint(const reach_system *s, int64_t m, int prec) {
    // the sample-row streaming kernels pad the samples to blocks of 64
    // (binary32, two per lane) or 32, the on-chip one uses blocks of 2 to 32;
    // the row-layout defaults (mc_rows, mc_rows64) hold the same two state
    // buffers with rows padded to an even count and no partials, which the
    // partials term below more than covers
    const bool stream_kernel = (s->kind == REACH_TRAFFIC || s->kind == REACH_KS) && s->n > 128;
    const int64_t ss = prec == 32 ? 64 : 32, M = (m + ss - 1) / ss * ss, elt = prec == 32 ? 4 : 8, n = s->n;
    // partial minima / maxima: one row per block of samples
    const int64_t sb = mc_onchip_sb(m), blocks = std::max(M / 32, (m + sb - 1) / sb);
    int64_t partials = 2 * blocks * n * 8;
    return partials + (stream_kernel ? 2 * n * M * elt : 0);
}

int64_t footprint(const reach_request *r) {
    const reach_system *s = r->sys;
    const int64_t n = s->n, nw = s->nw;
    // staged inputs and outputs (the worst case: host buffers), the status word
    int64_t b = (4 * n + 2 * nw) * 8 + 256;
    if (r->method == 2) return b + mc_footprint(s, r->m, r->precision);
    // MM / CGB: the stencil kernels keep a 2n ping-pong buffer; the heat
    // stage kernels keep the state and two stage vectors (6n)
    if (s->kind == REACH_QUAD) return b;   // registers only
    if (s->kind == REACH_TRAFFIC && s->prm[5] != 0.0) return b + 8 * n * 8;   // interval halves, ping-pong
    return b + (s->kind == REACH_HEAT3D ? 6 : 2) * n * 8;
}

// Device copies of a slot request's host vectors, made before it computes
// (while other requests run) and copied back after, so that its own kernels
// start at once and the next request's copies overlap them.
struct Staged {
    reach_request r;     // the request with device pointers
    void *buf = nullptr;
    double *user_out[2] = {nullptr, nullptr};
    double *dev_out[2] = {nullptr, nullptr};
    int64_t n = 0;
};

static int stage_in(const Job *j, cudaStream_t st, Staged &g) {
    const reach_request &r = j->r;
    g.r = r;
    g.n = r.sys->n;
    const int64_t n = r.sys->n, nw = r.sys->nw;
    const double *in[4] = {r.x0_lo, r.x0_hi, r.w_lo, r.w_hi};
    const int64_t cnt[4] = {n, n, nw, nw};
    bool host_in[4], host_out[2];
    int64_t total = 0;
    for (int i = 0; i < 4; ++i) {
        host_in[i] = cnt[i] > 0 && in[i] && !is_device_ptr(in[i]);
        if (host_in[i]) total += (cnt[i] + 31) / 32 * 32;
    }
    double *out[2] = {r.lo, r.hi};
    for (int i = 0; i < 2; ++i) {
        host_out[i] = out[i] && !is_device_ptr(out[i]);
        if (host_out[i]) total += (n + 31) / 32 * 32;
    }
    if (total == 0) return REACH_OK;
    int rc = dalloc(&g.buf, (size_t)total * sizeof(double), st);
    if (rc) return rc;
    double *p = (double *)g.buf;
    const double **din[4] = {&g.r.x0_lo, &g.r.x0_hi, &g.r.w_lo, &g.r.w_hi};
    for (int i = 0; i < 4; ++i) {
        if (!host_in[i]) continue;
        REACH_CUDA(cudaMemcpyAsync(p, in[i], cnt[i] * sizeof(double), cudaMemcpyHostToDevice, st));
        *din[i] = p;
        p += (cnt[i] + 31) / 32 * 32;
    }
    double **dout[2] = {&g.r.lo, &g.r.hi};
    for (int i = 0; i < 2; ++i) {
        if (!host_out[i]) continue;
        g.user_out[i] = out[i];
        g.dev_out[i] = p;
        *dout[i] = p;
        p += (n + 31) / 32 * 32;
    }
    REACH_CUDA(cudaStreamSynchronize(st));
    return REACH_OK;
}

static int stage_out(Staged &g, cudaStream_t st, bool copy) {
    int rc = REACH_OK;
    for (int i = 0; i < 2 && copy; ++i)
        if (g.user_out[i]) {
            cudaError_t e = cudaMemcpyAsync(g.user_out[i], g.dev_out[i], g.n * sizeof(double),
                                            cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess && !rc) rc = cuda_fail(e, "stage_out");
        }
    if (g.buf) dfree(g.buf, st);
    g.buf = nullptr;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && !rc) rc = cuda_fail(e, "stage_out");
    return rc;
}

static void run_job(Job *j, const reach_request &r, cudaStream_t st) {
    if (r.method == 0)
        j->status = reach_mm(r.sys, r.x0_lo, r.x0_hi, r.w_lo, r.w_hi, r.t_final, r.dt, r.lo, r.hi, st);
    else if (r.method == 1)
        j->status = reach_cgb(r.sys, r.x0_lo, r.x0_hi, r.w_lo, r.w_hi, r.t_final, r.dt, r.lo, r.hi, st);
    else
        j->status = reach_mc(r.sys, r.x0_lo, r.x0_hi, r.w_lo, r.w_hi, r.t_final, r.dt, r.m, r.seed, r.precision,
                             r.lo, r.hi, st);
}

// a request the device work queue can run: MM / CGB of a small system with
// at least one step
static bool queue_eligible(const reach_request *r) {
    if (r->method != MM && r->method != CGB) return false;
    if (!queue_accepts(r->sys, r->method)) return false;
    int64_t N;
    return nsteps(r->t_final, r->dt, &N) == REACH_OK && N >= 1;
}

static void finish_locked(reach_server *s, Job *j, int status) {
    j->status = status;
    j->finished = Clock::now();
    j->done = true;
    s->n_done++;
    s->done_cv.notify_all();
}

// hand a waiting request to the device work queue; false if the queue cannot
// take it now (ring or staging arena full) and it must keep waiting
static bool to_queue_locked(reach_server *s, Job *j) {
    const reach_request &r = j->r;
    reach_query q{r.sys, r.method, r.x0_lo, r.x0_hi, r.w_lo, r.w_hi, r.t_final, r.dt, r.lo, r.hi};
    j->started = Clock::now();
    const int rc = reach_queue_submit(s->queue, &q, &j->qticket);
    if (rc == REACH_EADMIT) return false;
    s->n_admitted++;
    if (rc != REACH_OK) {
        finish_locked(s, j, rc);
        return true;
    }
    j->in_queue = true;
    s->n_queued++;
    s->queue_running++;
    s->done_cv.notify_all();   // its waiter continues on the queue
    return true;
}

// admit every waiting request that can start, in arrival order (caller holds mu)
static void dispatch_locked(reach_server *s) {
    int free_slots = s->idle - (int)s->admitted.size();
    for (auto it = s->waiting.begin(); it != s->waiting.end();) {
        Job *j = *it;
        // small requests go to the queue (up to queue_n cells: beyond about 500
        // cells one block takes longer per step than a streaming kernel spread
        // over the GPU, e.g. a KS CGB request of 4096 points and 14902 steps
        // 1.74 s queued against 0.68 s on a slot)
        if (j->queue_ok && j->r.sys->n <= s->queue_n) {
            if (to_queue_locked(s, j)) it = s->waiting.erase(it);
            else ++it;
            continue;
        }
        if (free_slots <= 0 || (j->wide && s->max_wide > 0 && s->wide_running >= s->max_wide)) {
            ++it;
            continue;
        }
        if (s->in_use + j->bytes <= s->budget) {
            if (j->wide) s->wide_running++;
            s->in_use += j->bytes;
            s->peak = std::max(s->peak, s->in_use);
            s->admitted.push_back(j);
            s->n_admitted++;
            --free_slots;
            it = s->waiting.erase(it);
        } else {
            ++it;
        }
    }
    if (!s->admitted.empty()) s->work_cv.notify_all();
}

// priority level of a request: 0 below 2^30 component updates, one more per
// factor 4 of work above, the largest requests sharing the least priority
static int work_level(const reach_request *r, int nlevels) {
    const int64_t n = r->sys->n;
    const double per_step = r->method == 2 ? (double)n * (double)std::max<int64_t>(r->m, 1) : 2.0 * (double)n;
    const double steps = r->dt > 0 ? std::ceil(r->t_final / r->dt) : 1.0;
    const double work = per_step * std::max(steps, 1.0);
    int level = 0;
    for (double t = (double)(1LL << 30); work >= t && level < nlevels - 1; t *= 4) ++level;
    return level;
}

static void worker_main(reach_server *s) {
    cudaSetDevice(s->device);
    std::vector<cudaStream_t> st(s->nlevels, nullptr);
    for (int k = 0; k < s->nlevels; ++k)
        if (cudaStreamCreateWithPriority(&st[k], cudaStreamNonBlocking, s->prio_greatest + k) != cudaSuccess) {
            cudaGetLastError();
            st[k] = k > 0 ? st[k - 1] : nullptr;
        }
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->idle++;
        dispatch_locked(s);
        s->work_cv.wait(lk, [&] { return s->stopping || !s->admitted.empty(); });
        s->idle--;
        if (s->admitted.empty()) {
            if (s->stopping) break;
            continue;
        }
        Job *j = s->admitted.front();
        s->admitted.pop_front();
        j->started = Clock::now();
        if (s->prio_mode == 1) {
            // arrival order: a request never outranks one that started before
            // it and still runs; the levels start over when the slots drain
            if (s->slot_running == 0) s->next_level = 0;
            j->level = s->next_level;
            s->next_level = std::min(s->next_level + 1, s->nlevels - 1);
        } else if (s->prio_mode == 2) {
            j->level = 0;
        } else if (s->prio_mode == 3) {
            j->level = s->nlevels - 1 - j->level;   // largest work first
        }
        s->slot_running++;
        cudaStream_t js = st[j->level];
        lk.unlock();
        Staged g;
        int rc = stage_in(j, js, g);
        lk.lock();
        if (!rc) {
            // the compute gate: with exclusive wide requests a wide one computes
            // alone (after everything that passed before it, light requests
            // included), and only light requests that arrive while it computes
            // pass beside it; waiters pass in arrival order
            const bool backfill = s->wide_exclusive && j->light && s->wide_computing > 0 && s->wide_waiting == 0;
            if (!backfill) {
                s->gate.insert(j->ticket);
                if (j->wide) s->wide_waiting++;
                s->gate_cv.wait(lk, [&] {
                    if (!s->wide_exclusive) return true;
                    if (*s->gate.begin() != j->ticket) return false;
                    return j->wide ? s->computing == 0 : s->wide_computing == 0;
                });
                if (j->wide) s->wide_waiting--;
                s->gate.erase(j->ticket);
            } else {
                // a light request passes the gate at the least priority: its
                // blocks take only SMs that the wide request's blocks leave free
                js = st[s->nlevels - 1];
            }
            if (s->wide_exclusive && j->wide) js = st[0];
            s->computing++;
            if (j->wide) s->wide_computing++;
            s->gate_cv.notify_all();
            lk.unlock();
            run_job(j, g.r, js);
            lk.lock();
            s->computing--;
            if (j->wide) s->wide_computing--;
            s->gate_cv.notify_all();
            rc = j->status;
        }
        lk.unlock();
        const int rc_out = stage_out(g, js, rc == REACH_OK);
        lk.lock();
        if (!rc && rc_out) rc = rc_out;
        s->slot_running--;
        if (j->wide) s->wide_running--;
        s->in_use -= j->bytes;
        finish_locked(s, j, rc);
    }
    for (int k = 0; k < s->nlevels; ++k)
        if (st[k] && (k == 0 || st[k] != st[k - 1])) cudaStreamDestroy(st[k]);
}

}  // namespace reach

extern "C" int64_t reach_request_footprint(const reach_request *r) {
    if (!r || !r->sys) return REACH_EINVAL;
    return footprint(r);
}

extern "C" int reach_server_create(int slots, int64_t hbm_budget_bytes, reach_server **out) {
    if (!out || slots < 1 || slots > 256 || hbm_budget_bytes <= 0) return REACH_EINVAL;
    *out = nullptr;
    reach_server *s = new (std::nothrow) reach_server();
    if (!s) return REACH_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return REACH_ENODEV;
    }
    if (pool_init()) {
        delete s;
        return REACH_ECUDA;
    }
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    // numerically lower is greater priority
    s->prio_greatest = greatest;
    s->nlevels = std::min(8, std::max(1, least - greatest + 1));
    s->budget = hbm_budget_bytes;
    s->nslots = slots;
    const int64_t qblocks = reach_get_option(REACH_OPT_SERVE_QUEUE_BLOCKS);
    s->queue_n = reach_get_option(REACH_OPT_SERVE_QUEUE_N);
    s->max_wide = (int)reach_get_option(REACH_OPT_SERVE_MAX_WIDE);
    s->prio_mode = (int)reach_get_option(REACH_OPT_SERVE_PRIORITY);
    s->wide_exclusive = reach_get_option(REACH_OPT_SERVE_WIDE_EXCLUSIVE) != 0;
    s->light_components = reach_get_option(REACH_OPT_SERVE_LIGHT);
    if (qblocks > 0) {
        int rc = reach_queue_create((int)qblocks, 0.005, (int64_t)256 << 20, &s->queue);
        if (rc) {
            delete s;
            return rc;
        }
    }
    for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return REACH_OK;
}

extern "C" int reach_server_submit(reach_server *s, const reach_request *r, int64_t *ticket) {
    if (!s || !r || !ticket || !r->sys || r->method < 0 || r->method > 2) return REACH_EINVAL;
    const int64_t bytes = footprint(r);
    std::lock_guard<std::mutex> lk(s->mu);
    if (bytes > s->budget) {   // can never be admitted
        s->n_rejected++;
        return REACH_EADMIT;
    }
    Job *j = new (std::nothrow) Job();
    if (!j) return REACH_ENOMEM;
    j->ticket = s->next_ticket++;
    j->r = *r;
    j->bytes = bytes;
    j->level = work_level(r, s->nlevels);
    j->queue_ok = s->queue && queue_eligible(r);
    // wide: state components per step enough to fill every SM (2^20)
    const double per_step = r->method == 2 ? (double)r->sys->n * (double)std::max<int64_t>(r->m, 1)
                                           : 2.0 * (double)r->sys->n;
    j->wide = per_step >= (double)(1 << 20);
    j->light = per_step <= (double)s->light_components;
    j->submitted = Clock::now();
    s->jobs[j->ticket] = j;
    s->waiting.push_back(j);
    dispatch_locked(s);
    *ticket = j->ticket;
    return REACH_OK;
}

extern "C" int reach_server_wait(reach_server *s, int64_t ticket, double timeout_s, int *status, double *queue_s,
                                 double *run_s) {
    if (!s) return REACH_EINVAL;
    const auto t0 = Clock::now();
    auto limit = std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return REACH_EINVAL;
    Job *j = it->second;
    if (!s->done_cv.wait_for(lk, limit, [&] { return j->done || j->in_queue; })) return REACH_ETIMEOUT;
    if (!j->done) {
        // on the device work queue: wait there without holding the lock
        const double left = std::max(0.0, timeout_s - std::chrono::duration<double>(Clock::now() - t0).count());
        const int64_t qt = j->qticket;
        lk.unlock();
        int st = REACH_OK;
        const int rc = reach_queue_wait(s->queue, qt, left, &st);
        lk.lock();
        if (rc == REACH_ETIMEOUT) return REACH_ETIMEOUT;
        j->in_queue = false;
        s->queue_running--;
        finish_locked(s, j, rc ? rc : st);
        dispatch_locked(s);
    }
    if (status) *status = j->status;
    if (queue_s) *queue_s = std::chrono::duration<double>(j->started - j->submitted).count();
    if (run_s) *run_s = std::chrono::duration<double>(j->finished - j->started).count();
    s->jobs.erase(it);
    delete j;
    return REACH_OK;
}

extern "C" int reach_server_stats(reach_server *s, int64_t *waiting, int64_t *running, int64_t *done,
                                  int64_t *bytes_in_use, int64_t *bytes_peak) {
    if (!s) return REACH_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (waiting) *waiting = (int64_t)s->waiting.size();
    if (running) *running = s->n_admitted - s->n_done;
    if (done) *done = s->n_done;
    if (bytes_in_use) *bytes_in_use = s->in_use;
    if (bytes_peak) *bytes_peak = s->peak;
    return REACH_OK;
}

extern "C" int64_t reach_server_queued(reach_server *s) {
    if (!s) return REACH_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->n_queued;
}

extern "C" int reach_server_destroy(reach_server *s) {
    if (!s) return REACH_EINVAL;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // admitted and waiting requests are finished first; requests on the
        // queue are collected there (their staged results copied out)
        for (;;) {
            Job *qj = nullptr;
            for (auto &kv : s->jobs)
                if (kv.second->in_queue) { qj = kv.second; break; }
            if (qj) {
                const int64_t qt = qj->qticket;
                lk.unlock();
                int st = REACH_OK;
                const int rc = reach_queue_wait(s->queue, qt, 3600.0, &st);
                lk.lock();
                qj->in_queue = false;
                s->queue_running--;
                finish_locked(s, qj, rc ? rc : st);
                dispatch_locked(s);
                continue;
            }
            if (s->admitted.empty() && s->slot_running == 0) {
                if (s->waiting.empty()) break;
                dispatch_locked(s);
                bool started = !s->admitted.empty() || s->slot_running > 0;
                for (auto &kv : s->jobs) started |= kv.second->in_queue;
                if (!started) break;   // nothing left can start
                continue;
            }
            s->done_cv.wait_for(lk, std::chrono::milliseconds(50));
        }
        s->stopping = true;
        s->work_cv.notify_all();
    }
    for (std::thread &t : s->workers) t.join();
    if (s->queue) reach_queue_destroy(s->queue);
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
    return REACH_OK;
}
