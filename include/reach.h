/*
 * reach.h -- C ABI of libreach.so, interval reachability on one B300 GPU.
 *
 * The library computes interval over-approximations (MM, CGB) and sampled
 * approximations (MC) of the finite-time reachable set of dx/dt = f(x, p):
 *
 *     R = { Phi(t1; 0, x0, p) : x0 in [x0_lo, x0_hi], p in [w_lo, w_hi] }
 *
 * (Devonport, Khaled, Arcak, Zamani, "PIRK", 2020: Sec. 2 for the problem,
 * Sec. 2.1 for the three methods, Algorithms 1-4 for their parallel form).
 * Integration is fixed-step classic fourth-order Runge-Kutta (Algorithm 1
 * read as RK4: stages at t, t+h/2, t+h/2, t+h with weights 1,2,2,1 / 6) with
 * N = round(t_final/dt) steps of size dt from t0 = 0.  All arithmetic of MM
 * and CGB is IEEE binary64; MC trajectories run in binary64 or binary32.
 *
 * Conventions shared by every entry point
 *   - Every pointer argument may be host memory (pageable or pinned) or CUDA
 *     device memory of the current device; the library asks the driver which
 *     (cudaPointerGetAttributes).  Host data is copied in and out by the
 *     call.  All buffers stay owned by the caller.
 *   - Vectors are dense, contiguous binary64 arrays.  A state vector has the
 *     system's dimension n, an input vector its input dimension nw
 *     (reach_input_dim).  Inputs are constant in time (Sec. 2).
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Work is
 *     ordered on that stream, and every computing reach_* call returns only
 *     after its results are complete (it synchronises the stream), so that
 *     it can report data-dependent errors.
 *   - Return value: REACH_OK (0) or a negative REACH_E* code.  No C++
 *     exception crosses the ABI.  On error the outputs are unspecified.
 *   - Scratch memory comes from the device's stream-ordered memory pool
 *     (cudaMallocAsync) and is returned before the call ends.
 */
#ifndef REACH_H
#define REACH_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define REACH_API __attribute__((visibility("default")))
#else
#define REACH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define REACH_OK 0
#define REACH_EINVAL (-1)     /* bad argument: size, lo > hi, non-finite input,
                                 dt <= 0, t_final/dt not an integer (within
                                 1e-9 t_final), unknown kind or method */
#define REACH_ENOMEM (-2)     /* device allocation failed */
#define REACH_EADMIT (-3)     /* serving: query can never fit the HBM budget */
#define REACH_ENONFINITE (-4) /* a result (or an MC sample) became NaN or Inf */
#define REACH_ETIMEOUT (-5)   /* a bounded device or host wait ran out */
#define REACH_ECUDA (-6)      /* a CUDA runtime call failed */
#define REACH_ENODEV (-7)     /* no usable CUDA device */

/* ---- built-in systems ---- */
typedef enum {
    /* Cell-transmission traffic chain (Sec. 5.1).  Cells i = 0..n-1, flux out
       of cell i  f_i = min(cap, v x_i, w (xbar - x_{i+1})) for i < n-1,
       f_{n-1} = min(cap, v x_{n-1}); inflow of cell 0 is the input d (nw = 1);
       dx_i/dt = f_{i-1} - f_i.  Params: reach_traffic_params. */
    REACH_TRAFFIC = 0,
    /* Kuramoto-Sivashinsky u_t = -g_nl u u_x - g_2 u_xx - g_4 u_xxxx on a
       periodic grid of n >= 5 points with spacing dx, second-order central
       differences (3-point u_x, u_xx; 5-point u_xxxx).  nw = 0.
       Params: reach_ks_params. */
    REACH_KS = 1,
    /* Chain of m = n/2 nonlinear oscillators, state [x_1..x_m | v_1..v_m]:
       dx_i/dt = v_i, dv_i/dt = -ka x_i - kb x_i^3 + kc (x_{i-1} - 2 x_i +
       x_{i+1}) + w_i with x_0 = x_{m+1} = 0.  nw = m.
       Params: reach_osc_params. */
    REACH_OSC = 2,
    /* Dense linear test system dx/dt = A x + p, nw = n, n <= 256.
       Params: reach_linear_params. */
    REACH_LINEAR = 3,
    /* Heat diffusion in the unit cube (Sec. 5.4) on an l x l x l grid
       (n = l^3, index x + l (y + l z)), spacing 1/l, first-order differences:
       du_i/dt = alpha l^2 sum over the six neighbours of (u_nb - u_i); missing
       neighbours of five faces contribute nothing (insulated), and with
       open_face set the face z = 0 sees an environment at temperature zero.
       nw = 0.  Params: reach_heat_params. */
    REACH_HEAT3D = 4,
    /* Quadrotor swarm (Sec. 5.2): K = n / 12 independent agents; agent k holds
       x[12k + 0..11] = (p_n, p_e, h, dp_n, dp_e, dh, phi, theta, psi, dphi,
       dtheta, dpsi) and inputs p[3k + 0..2] = (tau_phi, tau_theta, tau_psi):
         ddp_n = F/m (-cos phi sin theta cos psi - sin phi sin psi)
         ddp_e = F/m (-cos phi sin theta sin psi + sin phi cos psi)
         ddh   = g - F/m cos phi cos theta
         ddphi = tau_phi / Jx, ddtheta = tau_theta / Jy, ddpsi = tau_psi / Jz,
       with the thrust F a parameter (so the system is input-affine).  MM uses
       the natural interval extension of the accelerations over the angle box;
       CGB bounds |J| over the current box the same way.  nw = 3 K.
       Params: reach_quad_params.  Not accepted by reach_batch_create (one
       call already runs every agent in one launch). */
    REACH_QUAD = 5
} reach_kind;

/* cgb_local != 0: CGB takes the contraction matrix over the current box
   [c - r, c + r] (free-flow / congestion branches that can be, or are
   everywhere, the minimum of the flux) instead of the bounds valid for every
   state.  sound != 0: MM and CGB round every operation outward, so that the
   box contains the one the same method gives in exact real arithmetic from
   the same binary64 inputs and step (the MM halves and the CGB center are
   carried as intervals, the CGB radius rounded up); not with cgb_local, not
   with reach_pipe, reach_mm_noalloc or batches, and MC ignores it.  A struct
   of only the four doubles (params_bytes = 32) is accepted and means 0, 0. */
typedef struct { double cap, v, w, xbar; int cgb_local; int sound; } reach_traffic_params; /* 40, 0.5, 1/6, 320, 0, 0 */
typedef struct { double dx, g_nl, g_2, g_4; } reach_ks_params;     /* pi/4, 1, 1, 1 */
typedef struct { double ka, kb, kc; } reach_osc_params;            /* 1, 0.1, 0.5 */
typedef struct { const double *A; } reach_linear_params;           /* n x n, row-major */
typedef struct { double alpha; int64_t l; int open_face; } reach_heat_params; /* 8e-6, cbrt(n), 1 */
typedef struct { double m, g, F, Jx, Jy, Jz; } reach_quad_params; /* 1.4, 9.81, m g, 0.054, 0.054, 0.104 */

typedef struct reach_system reach_system;   /* opaque; parameters live on the device */

/* Create a system of dimension n.  `params` points to the kind's parameter
   struct (params_bytes = its sizeof), or is NULL for the defaults noted
   above (REACH_LINEAR requires params).  The parameters, including A, are
   copied to the current device; the caller's buffers may be freed
   afterwards.  REACH_EINVAL for n < 1, odd n with REACH_OSC, n < 5 with
   REACH_KS, n > 256 with REACH_LINEAR, n != l^3 with REACH_HEAT3D, n not a multiple of 12 with
   REACH_QUAD, a wrong params_bytes or non-finite params (traffic additionally needs v, w >= 0; KS
   dx > 0; osc kb >= 0; quad m, Jx, Jy, Jz > 0 and F >= 0). */
REACH_API int reach_system_create(int kind, int64_t n, const void *params, size_t params_bytes,
                        reach_system **out);
REACH_API int reach_system_destroy(reach_system *sys);
REACH_API int64_t reach_system_dim(const reach_system *sys);
REACH_API int64_t reach_input_dim(const reach_system *sys);

/* Mixed monotonicity (Sec. 2.1, Algorithm 3).  Integrates the embedding
   system [x; xh]' = [d(x, p, xh, ph); d(xh, ph, x, p)] from
   [x0_lo; x0_hi] with p = w_lo, ph = w_hi and returns [lo, hi] = [x(T), xh(T)].
   The decomposition function d of each built-in system is the tight one:
   cooperative traffic and heat use d = f; KS splits the linear stencil by
   coefficient sign and bounds u_i u_x with u_i held at its own argument; the
   oscillator feeds x_i into the v_i row through the hatted argument; linear
   splits off-diagonal entries of A by sign; the quadrotor bounds its
   accelerations by their natural interval extension over the angle box.
   x0_lo, x0_hi, lo, hi: n values.  w_lo, w_hi: nw values (may be NULL if
   nw = 0).  lo/hi may not alias x0_lo/x0_hi. */
REACH_API int reach_mm(const reach_system *sys, const double *x0_lo, const double *x0_hi,
             const double *w_lo, const double *w_hi, double t_final, double dt,
             double *lo, double *hi, void *stream);

/* Contraction / growth bound (Sec. 2.1, Algorithm 2).  Integrates the
   center c' = f(c, p*) and the radius r' = C(c, r) r + [p] as one coupled
   2n-dimensional system from c = (x0_lo + x0_hi)/2, r = (x0_hi - x0_lo)/2,
   p* = (w_lo + w_hi)/2, [p] = (w_hi - w_lo)/2 (entering as the input enters
   f), and returns [lo, hi] = [c(T) - r(T), c(T) + r(T)].  C satisfies
   C_ii >= J_ii and C_ij >= |J_ij|: a constant bound valid for every state
   (traffic by default, linear, heat with C = A) or a bound over the current
   stage box [c - r, c + r] (KS and oscillator: the supremum of the Jacobian;
   quadrotor: its natural interval extension; traffic with cgb_local).
   Arguments as reach_mm. */
REACH_API int reach_cgb(const reach_system *sys, const double *x0_lo, const double *x0_hi,
              const double *w_lo, const double *w_hi, double t_final, double dt,
              double *lo, double *hi, void *stream);

/* Monte Carlo (Sec. 2.1, Algorithm 4).  Draws m initial states and m input
   vectors uniformly from the boxes with Philox4x32-10 (Salmon et al., SC'11):
   for sample j and component i, counter (i, j, tag, 0) with tag 0 for the
   state and 1 for the input, key (seed mod 2^32, seed div 2^32), and
   U = ((w0 << 32 | w1) >> 11) 2^-53; x0_i = lo_i + (hi_i - lo_i) U computed in
   binary64.  Each sample is integrated with RK4 in binary64 (precision = 64)
   or, after rounding the sample to binary32, in binary32 (precision = 32).
   Returns the elementwise minimum and maximum over the samples of the
   final states, as binary64.  REACH_ENONFINITE if any sample trajectory
   ends NaN or Inf.  1 <= m < 2^32. */
REACH_API int reach_mc(const reach_system *sys, const double *x0_lo, const double *x0_hi,
             const double *w_lo, const double *w_hi, double t_final, double dt,
             int64_t m, uint64_t seed, int precision,
             double *lo, double *hi, void *stream);

/* The reach pipe (Sec. 5.5): the MM (method 0) or CGB (method 1) box after
   every `every` RK4 steps.  pipe_lo / pipe_hi receive N/every rows of n values
   (row q = the box after (q+1) every steps, row-major); N must be a multiple
   of every.  Each segment starts from the previous box: exact continuation
   for MM, and for CGB a restart from its center and radius, equal to one
   continuous integration up to one rounding of c and r per segment. */
REACH_API int reach_pipe(const reach_system *sys, int method, const double *x0_lo, const double *x0_hi,
                         const double *w_lo, const double *w_hi, double t_final, double dt, int64_t every,
                         double *pipe_lo, double *pipe_hi, void *stream);

/* Sample count for an (eps, delta) guarantee (Sec. 2.1):
   m = ceil((2n/eps) ln(2n/delta)).  Returns REACH_EINVAL for n < 1 or
   eps, delta outside (0, 1). */
REACH_API int64_t reach_mc_samples(int64_t n, double eps, double delta);

/* reach_mm for callers that cannot let a library allocate device memory
   (the paper has no counterpart): a process whose device memory is held by
   another allocator, such as a framework's caching pool that reserves nearly
   all of HBM, or a latency-critical loop that must not enter the driver's
   allocator, which can lock and synchronise.  It runs the same streaming RK4
   kernel as reach_mm for REACH_TRAFFIC and REACH_KS systems, and it allocates
   nothing: the kernel's ping-pong state buffer and the status word live in a
   fixed device buffer of the library (16 MiB + 256 B, held on every GPU that
   loads the library until the process exits).
     - n <= REACH_NOALLOC_MAX_N, else REACH_EINVAL; other kinds, and traffic
       systems created with outward rounding (sound), give REACH_EINVAL.
     - x0_lo, x0_hi, lo, hi must be device pointers (REACH_EINVAL otherwise);
       w_lo, w_hi (traffic inflow) may be host or device.
     - Every call looks up the buffer's device address on the current
       device (cudaGetSymbolAddress, which allocates nothing).
     - No call can be captured into a CUDA graph: each synchronises its
       stream and copies the status word to the host before it returns.
       Do not call it while its stream is being captured.
     - All calls share the buffer: calls whose work overlaps on the GPU (on
       different streams, or from several threads) race and give wrong
       results.  Each call clears the status word before use.
   Otherwise as reach_mm: same arguments, results, status codes, and the call
   returns after its results are complete. */
#define REACH_NOALLOC_MAX_N 1048576
REACH_API int reach_mm_noalloc(const reach_system *sys, const double *x0_lo, const double *x0_hi,
                               const double *w_lo, const double *w_hi, double t_final, double dt,
                               double *lo, double *hi, void *stream);

/* ---- batches: many uneven queries in one persistent launch ----
   Algorithms 2 and 3 applied to many independent queries at once (the paper
   runs one query per call; this batching is new).  A batch is planned once:
   every query becomes an on-chip problem (2n <= 16384 components; the
   streaming kernels are not used), problems are packed into the blocks of a
   persistent kernel (one per system kind and method present) largest first,
   the components-per-thread target is tuned by timing the candidate layouts
   on the batch itself with shortened horizons, and the whole run (input
   copies for host-resident queries, the kernels, output copies) is captured
   into a CUDA graph.  reach_batch_run replays it: it reads the query buffers
   given at creation (update their contents in place between runs), and
   returns after all results are written. */
typedef struct {
    const reach_system *sys;
    int method;                                  /* 0 = MM, 1 = CGB */
    const double *x0_lo, *x0_hi, *w_lo, *w_hi;   /* host or device, as reach_mm */
    double t_final, dt;
    double *lo, *hi;                             /* host or device */
} reach_query;

typedef struct reach_batch reach_batch;

#define REACH_BATCH_NO_AUTOTUNE 1   /* flag: use REACH_OPT_BATCH_CPT (default 8) */

/* REACH_EINVAL for an invalid query (as reach_mm), a zero horizon, or a
   query larger than the on-chip kernels hold. */
REACH_API int reach_batch_create(const reach_query *queries, int64_t count, int flags, reach_batch **out);
/* status (optional, count ints): each query's status; finish_s (optional,
   count doubles): seconds from the start of the kernels to the completion of
   each query.  Returns the first non-OK query status, or REACH_OK. */
REACH_API int reach_batch_run(reach_batch *b, void *stream, int *status, double *finish_s);
/* the tuned components-per-thread target, the kernels per run, and the
   timings (ms) of the four tuning candidates 2, 4, 8, 16 */
REACH_API int reach_batch_info(const reach_batch *b, int64_t *cpt, int64_t *kernels, double *tune_ms);
/* the tuned layout: the components-per-thread target, the item size (state
   components) from which items run on a two-block cluster instead of a bin
   slot (0: only items too large for one block), the seconds reach_batch_create
   spent (planning, tuning, graph capture), and the timings (ms) of the
   candidates tried: cpt 2, 4, 8, 16, then cluster thresholds 4096 and 2048
   components with the best cpt (0 where not tried) */
REACH_API int reach_batch_layout(const reach_batch *b, int64_t *cpt, int64_t *cluster_from, double *create_s,
                                 double *tune_ms);
REACH_API int reach_batch_destroy(reach_batch *b);

/* ---- device work queue: small queries run as they arrive ----
   Algorithms 2 and 3 for queries that arrive one by one while other work
   runs (the paper runs one query per call; this queue is new).  A query whose
   2n components fit one block (n <= REACH_QUEUE_MAX_N, and its stage vectors
   in shared memory) is appended to a ring in page-locked host memory that the
   GPU reads directly; the blocks of a persistent kernel take the published
   queries one at a time and integrate each whole horizon on chip, so a queued
   query costs no kernel launch, no copy call and no stream synchronisation.
   The queue launches blocks as queries arrive (one per query without a free
   block, at most max_blocks over all system kinds); a block that finds no
   query for idle_s seconds leaves by itself, so an idle queue holds no SM
   (a cudaDeviceSynchronize meanwhile waits up to idle_s for those blocks).
   Host vectors are staged in a page-locked arena of arena_bytes; the caller's
   input buffers may be reused when reach_queue_submit returns, its output
   buffers must stay valid until reach_queue_wait returns for the ticket.
   The four functions are thread-safe. */
#define REACH_QUEUE_MAX_N 4096
typedef struct reach_queue reach_queue;
REACH_API int reach_queue_create(int max_blocks, double idle_s, int64_t arena_bytes, reach_queue **out);
/* Queues one MM or CGB query (a reach_query, as for batches).  REACH_EINVAL
   for an invalid query, a zero horizon, a kind the queue does not run (the
   quadrotor, outward-rounded traffic) or n above REACH_QUEUE_MAX_N;
   REACH_EADMIT when 2048 queries of its kind are in flight or the staging
   arena is full (wait for results first). */
REACH_API int reach_queue_submit(reach_queue *q, const reach_query *query, int64_t *ticket);
/* Waits at most timeout_s seconds for a ticket: REACH_ETIMEOUT if it has not
   finished (it keeps running; wait again).  Otherwise copies staged outputs to
   the caller's host buffers, sets *status (REACH_OK, REACH_EINVAL for an
   inverted or non-finite box seen on the device, REACH_ENONFINITE) and
   forgets the ticket. */
REACH_API int reach_queue_wait(reach_queue *q, int64_t ticket, double timeout_s, int *status);
/* Launches `blocks` blocks of kind's persistent kernel now (they also start by
   themselves when queries are submitted). */
REACH_API int reach_queue_start(reach_queue *q, int kind, int blocks);
/* Waits at most timeout_s seconds for every block of the queue to leave:
   REACH_ETIMEOUT if some are still running.  Otherwise *exit_status tells how
   the last launch ended: REACH_ETIMEOUT when its blocks left because no query
   came within idle_s (their bounded wait ran out), REACH_OK when asked to stop. */
REACH_API int reach_queue_join(reach_queue *q, double timeout_s, int *exit_status);
/* queries submitted and not yet waited for, blocks running now, blocks launched so far */
REACH_API int reach_queue_stats(reach_queue *q, int64_t *in_flight, int64_t *alive_blocks, int64_t *launched_blocks);
/* runs every submitted query to its end, then frees the queue */
REACH_API int reach_queue_destroy(reach_queue *q);

/* ---- serving: a continuous-batching request loop ----
   The paper serves reachability problems to other tools over a network
   interface (Sec. 1); here that purpose is an in-process server.  Requests of
   any system, size, method and horizon are submitted as they arrive and
   start, in arrival order, as capacity frees up:
     - MM / CGB requests of up to REACH_OPT_SERVE_QUEUE_N cells (at most
       REACH_QUEUE_MAX_N; default 512, beyond which one block takes longer per
       RK4 step than a streaming kernel spread over every SM) join the
       server's device work queue (above), whose persistent blocks take them
       while other work runs;
     - every other request needs one of the server's slots and its
       device-memory footprint (reach_request_footprint) must fit in what is
       left of the budget (first fit).  Each slot is a worker thread that
       copies the request's host vectors to the device, runs it through
       reach_mm / reach_cgb / reach_mc on its own CUDA streams and copies the
       box back, so copies and kernels of different requests overlap.
     - By default a wide request (2^20 or more state components per step: it
       fills the GPU alone) computes alone: it starts computing when no other
       slot request computes (light ones included), and no other starts
       beside it except light ones (REACH_OPT_SERVE_LIGHT components per step
       or fewer) that arrive while it computes and no other wide request
       waits; they take the least stream priority so that their blocks only
       fill SMs the wide request leaves free.  Waiting requests start
       computing in arrival order, and no request waits for one that arrived
       after it.  Sharing the GPU with a wide request would finish both late
       (REACH_OPT_SERVE_WIDE_EXCLUSIVE = 0 lets them share).  Otherwise a
       stream's priority falls with the request's work (state components per
       step x steps; greatest below 2^30, one level lower per factor 4
       above), so the blocks of small requests are scheduled first.
   A request's buffers must stay valid until reach_server_wait has returned
   its result. */
typedef struct {
    const reach_system *sys;
    int method;                                  /* 0 = MM, 1 = CGB, 2 = MC */
    const double *x0_lo, *x0_hi, *w_lo, *w_hi;   /* host or device, as reach_mm */
    double t_final, dt;
    int64_t m;                                   /* MC: samples */
    uint64_t seed;                               /* MC */
    int precision;                               /* MC: 32 or 64 */
    double *lo, *hi;                             /* host or device */
} reach_request;

typedef struct reach_server reach_server;

/* device bytes a request may hold while it runs (staged inputs and outputs,
   ping-pong state, MC sample state and partial minima / maxima) */
REACH_API int64_t reach_request_footprint(const reach_request *r);
/* slots: concurrent requests (1..256); hbm_budget_bytes: admission budget */
REACH_API int reach_server_create(int slots, int64_t hbm_budget_bytes, reach_server **out);
/* REACH_EADMIT if the footprint alone exceeds the budget (never admitted) */
REACH_API int reach_server_submit(reach_server *s, const reach_request *r, int64_t *ticket);
/* Waits at most timeout_s seconds: REACH_ETIMEOUT if the request has not
   finished (it keeps running; wait again).  On success fills the request's
   status, its time from submission to start (queue_s) and its run time (run_s),
   and forgets the ticket. */
REACH_API int reach_server_wait(reach_server *s, int64_t ticket, double timeout_s, int *status, double *queue_s,
                                double *run_s);
REACH_API int reach_server_stats(reach_server *s, int64_t *waiting, int64_t *running, int64_t *done,
                                 int64_t *bytes_in_use, int64_t *bytes_peak);
/* requests that went to the server's device work queue so far */
REACH_API int64_t reach_server_queued(reach_server *s);
/* finishes every submitted request, then stops the slots */
REACH_API int reach_server_destroy(reach_server *s);

/* ---- tuning knobs (process-wide; used by tests, the autotuner, bench) ---- */
#define REACH_OPT_KERNEL 1           /* 0 auto, 1 streaming stencil, 2 on-chip */
#define REACH_OPT_STEPS_PER_LAUNCH 2 /* streaming kernels: RK4 steps per launch, 1..8; 0 = auto (FP64 1, FP32 MC
                                        3) */
#define REACH_OPT_BLOCK 3            /* threads per block of the on-chip kernel (0 auto) */
#define REACH_OPT_BATCH_CPT 4        /* batches: components per thread, 0 = autotune, or 2/4/8/16 */
#define REACH_OPT_TILE 5             /* streaming traffic / KS MM and CGB: cells per lane, 0 = auto, 2 (64-cell
                                        warp tiles, taken only while the halo leaves half the tile) or 8 (256) */
#define REACH_OPT_MC_SB 6            /* on-chip MC: samples per block, 0 = auto (32 from 4736 samples, 8 from 1184,
                                        else 2), or 2 / 8 / 32 */
#define REACH_OPT_MC_LAYOUT 7         /* streaming binary32 MC: 0 auto (two samples per lane, packed FP32
                                        arithmetic, along the rows of a sample pair with 14 rows per lane
                                        on the KS grid, 12 on the traffic chain), 1 one sample per lane; 2..6 block shapes of the two-sample
                                        kernel on sample rows (warps x rows x blocks per SM: 16x16x1,
                                        32x8x1, 8x16x2, 16x8x2, and 16x16x1 persistent with the next tiles
                                        copied ahead by the TMA engine); 8 / 9 / 10 along sample-pair
                                        rows with 8 / 12 / 16 rows per lane; all give the same box bit for
                                        bit.  Binary64: 0 auto (along the rows of one sample, 16 rows per
                                        lane: as 10), 8 / 9 / 10 along the rows with 8 / 12 / 16 rows per
                                        lane, 7 sample-row blocks of 16 warps, other values blocks of 8
                                        warps; all give the same box bit for bit */
#define REACH_OPT_SERVE_QUEUE_BLOCKS 8 /* servers created afterwards: blocks of their device work queue, 0 = no
                                         queue (default 64) */
#define REACH_OPT_SERVE_QUEUE_N 9      /* servers created afterwards: MM / CGB requests up to this many cells
                                         take the device work queue (default 512, at most REACH_QUEUE_MAX_N) */
#define REACH_OPT_SERVE_MAX_WIDE 10    /* servers created afterwards: requests with 2^20 or more state components
                                         per step (they fill the GPU alone) running at once, 0 = no limit
                                         (default) */
#define REACH_OPT_BATCH_CLUSTER_FROM 11 /* batches: items of this many state components or more run on a
                                          two-block cluster; 0 = tuned (untuned batches: only items too large
                                          for one block) */
#define REACH_OPT_ONE_LAUNCH 12       /* KS and traffic MM / CGB: 0 auto (every step in one persistent launch:
                                         KS grids of two to eight waves of warp tiles, 0.85e6 to 3.4e6 points;
                                         traffic chains from 1.5 waves, 4.4e5 cells), 1 one launch per step,
                                         2 one launch for every grid it can run */
#define REACH_OPT_SERVE_PRIORITY 13    /* servers created afterwards: stream priority of slot requests, 0 by
                                         work (smaller first), 1 by arrival (earlier first), 2 none, 3 by work
                                         (larger first) */
#define REACH_OPT_SERVE_WIDE_EXCLUSIVE 14 /* servers created afterwards: 1 (default) = a wide request computes
                                            only when no other slot request computes and none starts computing
                                            beside it, except light ones (queued requests still run); 0 = off */
#define REACH_OPT_SERVE_LIGHT 15       /* servers created afterwards, with exclusive wide requests: requests of at
                                         most this many state components per step compute beside a wide one,
                                         at the least stream priority (default 2^15; 0 = none) */
REACH_API int reach_set_option(int key, int64_t value);
REACH_API int64_t reach_get_option(int key);

/* Human-readable name of a status code. */
REACH_API const char *reach_strerror(int code);

/* Number of kernels this library has launched in the process (benchmark
   bookkeeping; a graph launch counts each kernel node it runs). */
REACH_API int64_t reach_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* REACH_H */
