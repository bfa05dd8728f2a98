/*
 * lb_rd.h -- C ABI of the GB300 (sm_103a) lattice-Boltzmann reaction-diffusion
 * library.
 *
 * The method is the multi-species lattice BGK scheme of Ayodele, Varnik and
 * Raabe, "Lattice Boltzmann study of pattern formation in reaction-diffusion
 * systems" (arXiv 1007.3109), Sec. II.A:
 *
 *   f_i,s(x + e_i, t + 1) = f_i,s(x, t) + (w_i rho_s - f_i,s(x, t)) / tau_s
 *                           + w_i R_s(rho_1, ..., rho_S)          (Eq. relax)
 *   rho_s = sum_i f_i,s,   f_i,s^eq = w_i rho_s                  (Eq. equili)
 *   D_s = c_s^2 (tau_s - 1/2),  c_s^2 = 1/3   (end of Sec. II.A, Eq. app22)
 *
 * on a periodic nx x ny lattice (Sec. II.B, Sec. IV) with the D2Q9 velocity
 * set of Eq. Weights (or D2Q5), and the reactions of Sec. II.B (transformation
 * A -> B, Eq. reac_diff3) and Sec. III (Gray-Scott, Eqs. reac_diff10/11 in
 * Pearson's (F, k) form).
 *
 * Conventions for every entry point:
 *  - Every function returns an lb_rd_status; LB_RD_OK is 0.  On failure the
 *    message of the calling thread's last error is in lb_rd_last_error().
 *  - Densities are FP64, row-major [s][y][x] (x fastest), S * ny * nx values.
 *  - A host pointer is any pageable or pinned host address; a device pointer
 *    is a CUDA device address on the current device (e.g. a torch tensor's
 *    data_ptr()).  is_device selects which one a pointer argument is.
 *  - Handles own all the device memory they allocate; callers own their
 *    buffers.  A device buffer passed in must stay alive until the call that
 *    reads or writes it has returned and, for asynchronous calls, until the
 *    handle's stream has been synchronised.
 *  - Work is enqueued on the handle's stream (lb_rd_config.stream).  Calls
 *    that return data to the host synchronise that stream.
 *  - A handle is not thread safe: one thread at a time may use it.  The
 *    server (lb_rd_server_*) is thread safe for submit and poll.
 *  - No entry point falls back to the CPU: without a usable CUDA device the
 *    calls that need one return LB_RD_ECUDA.
 */
#ifndef LB_RD_H
#define LB_RD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LB_RD_API __attribute__((visibility("default")))
#else
#define LB_RD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
    LB_RD_OK = 0,
    LB_RD_EINVAL = 1,   /* bad argument: tau <= 1/2, unknown enum, size < 1, NULL pointer */
    LB_RD_ENOMEM = 2,   /* a device allocation or the server's memory budget failed */
    LB_RD_ECUDA = 3,    /* a CUDA call failed (no device, launch error, ...) */
    LB_RD_EPENDING = 4, /* server request not finished yet */
    LB_RD_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    LB_RD_EBUSY = 6,    /* server full: request not admitted yet */
    LB_RD_ENOTFOUND = 7 /* unknown or already collected server ticket */
} lb_rd_status;

/* Velocity sets.  D2Q9: e = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
 * (-1,-1),(1,-1) with w = 4/9, 1/9 x4, 1/36 x4 (Eq. Weights).  D2Q5: the
 * first five velocities with w = 1/3, 1/6 x4 (not in the paper; the same
 * c_s^2 = 1/3, so the same tau <-> D map). */
typedef enum { LB_RD_D2Q9 = 0, LB_RD_D2Q5 = 1 } lb_rd_lattice;

/* Storage and arithmetic of the distributions.
 *  FP64:        f in double, double arithmetic without FMA contraction, in
 *               the operation order of Eq. relax (bit-reproducible).
 *  FP32:        f in float, float arithmetic.
 *  FP32_BF16DEV / FP32_FP16DEV: float arithmetic; per species and site the
 *               post-collision mass rho* = rho + R in float and the Q - 1
 *               deviations g_i = (1 - 1/tau)(f_i - w_i rho), i >= 1, in bf16
 *               or fp16 (g_0 = -sum g_i is implied); f*_i = w_i rho* + g_i. */
typedef enum {
    LB_RD_FP64 = 0,
    LB_RD_FP32 = 1,
    LB_RD_FP32_BF16DEV = 2,
    LB_RD_FP32_FP16DEV = 3
} lb_rd_precision;

/* Species and reaction-step capacity of one simulation. */
#define LB_RD_MAX_SPECIES 4
#define LB_RD_MAX_REACTIONS 16

/* Reactions R_s(rho).
 *  NONE:        R = 0 (pure diffusion).
 *  LINEAR:      transformation A -> B at rate kappa (Sec. II.B):
 *               R_A = -kappa rho_A; with a second species R_B = +kappa rho_A.
 *               1 or 2 species.
 *  GRAY_SCOTT:  2 species u = A, v = B, Eqs. reac_diff10/11 with
 *               A0 = k1 = 1, k_f = k_0 = F, k_2 = k:
 *               R_u = -u v^2 + F (1 - u),  R_v = u v^2 - (F + k) v.
 *  MASS_ACTION: a network of nreactions reaction steps among the species
 *               (Eq. reac_diff1 is written for N species; the paper's systems
 *               are built from such steps, e.g. U + 2V -> 3V, V -> P): step r
 *               proceeds at rate_r = rate[r] prod_j rho_j^order[r][j] and
 *               changes species s by change[r][s] per event, so
 *               R_s = sum_r change[r][s] rate_r.  FP64 evaluates
 *               p = rate[r], p = p * rho_j (order[r][j] times, j ascending),
 *               R_s = R_s + change[r][s] * p (steps in order, zero changes
 *               skipped), every operation rounded on its own. */
typedef enum {
    LB_RD_REACTION_NONE = 0,
    LB_RD_REACTION_LINEAR = 1,
    LB_RD_REACTION_GRAY_SCOTT = 2,
    LB_RD_REACTION_MASS_ACTION = 3
} lb_rd_reaction_kind;

typedef struct {
    int32_t kind;       /* lb_rd_reaction_kind */
    double kappa;       /* LINEAR rate */
    double F;           /* GRAY_SCOTT feed rate */
    double k;           /* GRAY_SCOTT kill rate */
    int32_t nreactions; /* MASS_ACTION: number of steps, 1 .. LB_RD_MAX_REACTIONS */
    double rate[LB_RD_MAX_REACTIONS];                      /* rate constants, finite, >= 0 */
    int8_t order[LB_RD_MAX_REACTIONS][LB_RD_MAX_SPECIES];  /* reactant exponents, 0 .. 3 */
    int8_t change[LB_RD_MAX_REACTIONS][LB_RD_MAX_SPECIES]; /* net change per event, -4 .. 4 */
} lb_rd_reaction;

/* Storage of the state.
 *  PINGPONG: two copies; each step pulls f*(t) from one into the other.
 *  INPLACE:  one copy (half the device memory): steps alternate between
 *            reading neighbours and writing the swapped slots back to them
 *            (t even) and reading and writing a site's own slots (t odd), the
 *            "AA" pattern; the same bits as PINGPONG.  FP64 and FP32 storage;
 *            FP32 launch variants; the last step of every lb_rd_step call
 *            also writes rho.  Batches and servers take in-place FP32
 *            instances (one copy each); not for lb_rd_step_noalloc. */
typedef enum { LB_RD_STREAM_PINGPONG = 0, LB_RD_STREAM_INPLACE = 1 } lb_rd_streaming;

/* One simulation: the paper's statement of the problem. */
typedef struct {
    int32_t lattice;         /* lb_rd_lattice */
    int32_t nspecies;        /* 1 .. LB_RD_MAX_SPECIES (GRAY_SCOTT needs 2, LINEAR at most 2) */
    int64_t nx, ny;          /* periodic grid, 1 .. 65535 each */
    double tau[LB_RD_MAX_SPECIES]; /* relaxation time per species, > 1/2 (D = (tau - 1/2)/3) */
    lb_rd_reaction reaction;
    int32_t precision;       /* lb_rd_precision */
    int32_t track_mass;      /* nonzero: every step also reduces sum_x rho_s in FP64 */
    int32_t streaming;       /* lb_rd_streaming */
    void *stream;            /* cudaStream_t for all work; NULL = legacy default stream */
    int32_t tb_depth;        /* time steps per launch (temporal blocking): 0 = the autotuner's cached choice
                                (else one step per launch); 1 = one; 2 .. 8 = a depth-K variant of that
                                many steps (FP32 or 16-bit deviation storage with two state copies and
                                at most two species only, else EINVAL; lb_rd_create also fails with
                                EINVAL when no variant of that depth fits the grid).  Batches take
                                cfgs[0].tb_depth as their steps per launch when it is nonzero; servers
                                and lb_rd_step_noalloc ignore it. */
} lb_rd_config;

typedef struct lb_rd_handle lb_rd_handle;

/* Message of the calling thread's last failure ("" if none).  Valid until the
 * thread's next lb_rd call. */
LB_RD_API const char *lb_rd_last_error(void);

/* Library version string, e.g. "lb_rd 1.0 sm_103a". */
LB_RD_API const char *lb_rd_version(void);

/* tau = D / c_s^2 + 1/2 = 3 D + 1/2 (end of Sec. II.A).  Pure arithmetic. */
LB_RD_API double lb_rd_tau_from_diffusion(double D);

/* Validate cfg without touching the GPU; *bytes (if not NULL) receives the
 * device memory lb_rd_create will allocate.  EINVAL names the bad field. */
LB_RD_API int lb_rd_check_config(const lb_rd_config *cfg, size_t *bytes);

/* Allocate a simulation on the current device.  The state is undefined until
 * lb_rd_init.  ENOMEM if the device allocation fails. */
LB_RD_API int lb_rd_create(const lb_rd_config *cfg, lb_rd_handle **out);

/* Synchronise the handle's stream and free everything the handle owns.
 * NULL is accepted. */
LB_RD_API int lb_rd_destroy(lb_rd_handle *h);

/* Set time t = 0 with f_i,s = w_i rho0_s at every site (equilibrium; the
 * paper does not state its initial distributions).  rho0: [S][ny][nx] FP64,
 * host (copied before return) or device (read asynchronously). */
LB_RD_API int lb_rd_init(lb_rd_handle *h, const double *rho0, int is_device);

/* Advance nsteps >= 0 time steps of Eq. relax (collide, then stream with
 * periodic wrap).  Asynchronous on the handle's stream.  Each step is the
 * fused update: pull-stream, rho_s = sum_i f_i,s, R_s, BGK + source, store;
 * one launch runs one step, or K steps with a temporal-blocking variant (see
 * lb_rd_autotune).  With a depth-K variant the call runs K steps per launch
 * and splits its last steps into launches of fewer steps (chosen from the
 * autotuner's times per depth to finish soonest); a last launch of two or more
 * steps also writes the densities rho(t), so that no single-step launch is
 * needed to leave them available. */
LB_RD_API int lb_rd_step(lb_rd_handle *h, int64_t nsteps);

/* Current time step t of the handle. */
LB_RD_API int lb_rd_get_time(const lb_rd_handle *h, int64_t *t);

/* Densities rho_s(x, t) = sum_i f_i,s(x, t) at the current time (pre-collision,
 * i.e. after t streams; t = 0 gives sum_i w_i rho0).  rho_out: [S][ny][nx]
 * FP64 or NULL; mass_out: S doubles, sum over all sites of rho_s, reduced in
 * FP64, or NULL.  Synchronises the handle's stream. */
LB_RD_API int lb_rd_moments(lb_rd_handle *h, double *rho_out, double *mass_out, int is_device);

/* Post-collision distributions f*_i,s(x, t) (the values about to be streamed
 * from x in step t -> t + 1), FP64 [s][i][y][x], Q planes per species.
 * Synchronises. */
LB_RD_API int lb_rd_get_distributions(lb_rd_handle *h, double *f_out, int is_device);

/* Checkpoint: raw device state (distributions, densities, time) to a host
 * buffer of lb_rd_state_size() bytes, and back.  Restore needs a handle
 * created with the same config; the resumed run is bitwise identical to an
 * uninterrupted one.  Both synchronise. */
LB_RD_API int lb_rd_state_size(const lb_rd_handle *h, size_t *bytes);
LB_RD_API int lb_rd_save(lb_rd_handle *h, void *host_buf, size_t bytes);
LB_RD_API int lb_rd_restore(lb_rd_handle *h, const void *host_buf, size_t bytes);

/* Device time of the step kernels.  When enabled, lb_rd_step brackets every
 * step kernel with CUDA events on the handle's stream; lb_rd_kernel_time
 * synchronises and returns the summed duration and launch count since the
 * last reset (enable = 1 also resets). */
LB_RD_API int lb_rd_set_timing(lb_rd_handle *h, int enable);
LB_RD_API int lb_rd_kernel_time(lb_rd_handle *h, double *total_ms, int64_t *launches);
/* The same events launch by launch: launch i of the timed step kernels (in
 * order, since the last lb_rd_set_timing) took ms[i] milliseconds, advanced
 * steps[i] time steps and ran launch variant variant[i] (lb_rd_handle_variant_name).
 * At most max entries are written (any array may be NULL); *count (may be
 * NULL) receives the number of timed launches.  Synchronises. */
LB_RD_API int lb_rd_launch_times(lb_rd_handle *h, double *ms, int32_t *steps, int32_t *variant, int64_t max,
                                 int64_t *count);

/* Number of kernels this handle has launched since creation. */
LB_RD_API int lb_rd_launch_count(const lb_rd_handle *h, int64_t *launches);

/* Launch variants and the autotuner.  The step kernel of a precision comes in
 * several launch variants (tile shape, register budget, cache policy, TMA
 * bulk-copy staging, temporal blocking of K = 2 .. 8 steps per launch:
 * FP32 variants named tb2*_ (two steps) and deep<K>*_ (K steps, the deep1_
 * form one step; deep<K>vw*_ with two columns per lane), 16-bit deviation
 * variants hdeep<K>_ and hpair<K>_ (K steps; hpair: two columns per lane, nx
 * a multiple of 8); see lb_rd_variant_name).  lb_rd_autotune times every
 * variant that fits the grid on the handle's own state -- reading the current
 * state and writing the spare copy, so the simulation is unchanged -- with
 * one warm-up launch and `iters` timed launches each, and selects the fastest
 * single-step variant and, if faster per step, a multi-step variant, and
 * records the fastest depth-K variant of every depth with its time; the
 * choice is cached per (device, precision, lattice, species, nx, ny) and
 * handles created later with the same shape start from it.  With a K-step
 * variant lb_rd_step advances K steps per launch; with a depth-K variant its
 * last r + K min(q, 4) steps (nsteps = q K + r) go in launches of 1 .. K
 * steps, fastest total by the recorded times (untuned: a fixed relative
 * table), the last one writing rho; with a two-step variant the last step is
 * single.  times_ms (may be NULL) receives the mean time per time step of
 * each variant (-1 for a variant that does not fit), at most max_times
 * entries; *best the variant used for the bulk of the steps.  Synchronises.
 * lb_rd_set_variant forces a variant (a multi-step one is used together with
 * the current single-step variant and the recorded or default depth-K
 * variants of fewer steps; -1 restores the cached or default choice);
 * lb_rd_get_variant returns the variant used for the bulk of the steps. */
LB_RD_API int lb_rd_variant_count(int32_t precision, int32_t *count);
LB_RD_API const char *lb_rd_variant_name(int32_t precision, int32_t variant);
/* The variants of one handle's configuration: configurations with more than
 * two species or a mass-action network run the general kernel, whose FP32
 * variants update 1, 2 or 4 consecutive sites per thread (nx a multiple of
 * that) and whose FP64 form has one variant.  Bitwise-equal results. */
LB_RD_API int lb_rd_handle_variant_count(const lb_rd_handle *h, int32_t *count);
LB_RD_API const char *lb_rd_handle_variant_name(const lb_rd_handle *h, int32_t variant);
LB_RD_API int lb_rd_autotune(lb_rd_handle *h, int32_t iters, int32_t *best, double *times_ms, int32_t max_times);
LB_RD_API int lb_rd_set_variant(lb_rd_handle *h, int32_t variant);
LB_RD_API int lb_rd_get_variant(const lb_rd_handle *h, int32_t *variant);

/* Test switch for the error path of the bounded device-side waits (not part
 * of the method).  When enabled, the next step launch of a TMA-staged variant
 * (bulk-copy or two-step) makes block 0 wait for 16 bytes that are never
 * copied; the wait gives up after about one second, the kernel records
 * LB_RD_ETIMEOUT in the handle's status word, waits (bounded) for its copies
 * in flight and returns.  The next lb_rd_moments returns LB_RD_ETIMEOUT; the
 * state is then invalid until lb_rd_init, which clears the status.  Nothing
 * faults, traps or hangs: the CUDA context stays usable.  One-shot. */
LB_RD_API int lb_rd_debug_inject_wait_timeout(lb_rd_handle *h, int32_t enable);

/* ---- Batched simulations ------------------------------------------------
 * n independent simulations advanced together, e.g. a phase-diagram sweep of
 * Gray-Scott (F, k) pairs or a set of diffusion-rescaled runs (Sec. IV).  All
 * share lattice, species count, precision and stream (taken from cfgs[0]);
 * grid size, tau and reaction constants may differ per instance.  Each time
 * step is ONE launch of a persistent kernel that walks the combined
 * (instance x tile) work list; lb_rd_batch_step replays the steps as CUDA
 * graphs.  Every instance computes exactly what a single handle with its
 * config computes (bitwise: same kernel body, same arithmetic).  Every
 * precision is supported (FP64 runs the FP64 per-site update, e.g. for a
 * point-source convergence sweep over D and kappa, Sec. II.B). */
typedef struct lb_rd_batch lb_rd_batch;

/* Allocate n >= 1 instances (two state copies each plus density caches).
 * EINVAL if the configs disagree on lattice, nspecies or precision. */
LB_RD_API int lb_rd_batch_create(const lb_rd_config *cfgs, int32_t n, lb_rd_batch **out);
LB_RD_API int lb_rd_batch_destroy(lb_rd_batch *b);

/* Initialise instance idx at equilibrium with rho0 ([S][ny][nx] FP64, host or
 * device), as lb_rd_init.  Every instance must be initialised before the
 * first lb_rd_batch_step.  Allowed only while the batch time is 0. */
LB_RD_API int lb_rd_batch_init(lb_rd_batch *b, int32_t idx, const double *rho0, int is_device);

/* Advance every instance by nsteps >= 0 steps (asynchronous).  The last
 * launch also writes each instance's densities: with depth-K launches
 * (lb_rd_batch_set_steps_per_launch) the call runs nsteps / K launches of K
 * steps and one launch of the nsteps % K steps left (a single step if one is
 * left), otherwise its last step is a single step. */
LB_RD_API int lb_rd_batch_step(lb_rd_batch *b, int64_t nsteps);

/* Steps per captured CUDA graph (an even number >= 2), or 0 to launch every
 * step directly.  Default 64. */
LB_RD_API int lb_rd_batch_set_graph(lb_rd_batch *b, int32_t steps_per_graph);

/* Time steps per launch, 1 .. 8: 2 runs the two-step (temporal blocking)
 * kernel over all instances, bitwise the same as two single steps, when the
 * instances are FP32 with two state copies and nx a multiple of 256; other
 * values >= 2 (and 2 otherwise) run the depth-K kernel over the (band, strip)
 * units of all instances (FP32, two state copies, any nx; bitwise the same as
 * K single steps; for K <= 5 (D2Q9) or 6 (D2Q5) its form with two columns per
 * lane; the default for such batches: 5 for D2Q9, 6 for D2Q5); 16-bit
 * deviation storage runs its own depth-K kernels, K = 2 .. 5 (the
 * two-column form when every nx is a multiple of 8, default 5; else default
 * 4).
 * EINVAL if neither applies.  1: one step per launch (the default for other
 * batches).  The graphs of lb_rd_batch_set_graph hold steps_per_graph / K
 * launches.  Synchronises the batch's stream. */
LB_RD_API int lb_rd_batch_set_steps_per_launch(lb_rd_batch *b, int32_t k);

/* Densities and FP64 mass of instance idx at the batch's current time (as
 * lb_rd_moments).  Synchronises. */
LB_RD_API int lb_rd_batch_moments(lb_rd_batch *b, int32_t idx, double *rho_out, double *mass_out, int is_device);

/* Batch time (steps taken) and kernels launched since creation. */
LB_RD_API int lb_rd_batch_get_time(const lb_rd_batch *b, int64_t *t, int64_t *launches);

/* ---- Serving: continuous batching of simulation requests -----------------
 * A server owns a worker thread and a CUDA stream.  Requests (a config, host
 * rho0 and a step count) are queued on submit and admitted first-in first-out
 * while the number of resident requests is below max_slots and their device
 * memory (two state copies plus the density cache) fits hbm_budget_bytes.
 * Resident requests advance together, steps_per_tick steps at a time (fewer
 * when a request finishes sooner), by launches of the batched kernels over
 * all of them: for FP32 and 16-bit deviation requests with two state copies,
 * tick / K launches of the depth-K kernel (K as the batches' default: 5 for
 * D2Q9 and 6 for D2Q5 in FP32; 5 or 4 in 16-bit storage) and one launch of the
 * tick % K
 * steps left (a single step if one is left), otherwise one launch per step;
 * the last launch of a tick also writes the densities.  Requests that arrive
 * meanwhile are admitted between ticks
 * as slots and memory free up.  A finished request's densities and mass are
 * copied to host memory and its device memory is released.  Each result is
 * bitwise what a single handle with the same config computes.  Any
 * precision; all requests of a server share lattice, species count and
 * precision (given in the server config).  submit and poll are thread
 * safe. */
typedef struct {
    size_t hbm_budget_bytes;  /* device memory the resident requests may hold */
    int32_t max_slots;        /* resident requests at most, >= 1 */
    int32_t steps_per_tick;   /* steps between admission points, >= 1 */
    int32_t lattice, nspecies, precision;
    void *stream;             /* NULL: the server creates its own stream */
    int64_t tick_sites;       /* 0: every resident request advances in every tick (processor sharing);
                                 > 0: a tick advances the resident requests with the least remaining work
                                 (sites x steps left) first, as many as make up at least tick_sites sites
                                 together (all if fewer), the others waiting for a later tick: short
                                 requests finish sooner, a long one can wait while shorter ones keep
                                 arriving */
} lb_rd_server_config;

typedef struct {
    int64_t arrival_ns;  /* submit time (steady clock) */
    int64_t start_ns;    /* admission time */
    int64_t end_ns;      /* results on the host */
    int64_t steps;
    int32_t status;      /* final status of the request */
} lb_rd_request_stats;

typedef struct lb_rd_server lb_rd_server;

LB_RD_API int lb_rd_server_create(const lb_rd_server_config *cfg, lb_rd_server **out);
/* Stops admitting, finishes nothing further, frees everything. */
LB_RD_API int lb_rd_server_destroy(lb_rd_server *srv);
/* Queue a request; rho0 ([S][ny][nx] FP64 host) is copied before return.
 * EINVAL for a bad config or one that does not match the server's lattice,
 * species or precision.  A request larger than the whole budget is accepted
 * and then fails with ENOMEM (see poll). */
LB_RD_API int lb_rd_submit(lb_rd_server *srv, const lb_rd_config *cfg, const double *rho0, int64_t nsteps,
                           uint64_t *ticket);
/* LB_RD_EPENDING while queued or running; otherwise the request's final
 * status (LB_RD_OK, LB_RD_ENOMEM, ...), after which the ticket is released.
 * On OK, rho_out ([S][ny][nx] FP64 host) and mass_out (S doubles) receive the
 * results if not NULL.  stats (may be NULL) is filled in every case.
 * ENOTFOUND for an unknown or already collected ticket. */
LB_RD_API int lb_rd_poll(lb_rd_server *srv, uint64_t ticket, double *rho_out, double *mass_out,
                         lb_rd_request_stats *stats);
/* Block until every submitted request has finished or timeout_ms elapses
 * (LB_RD_ETIMEOUT). */
LB_RD_API int lb_rd_server_drain(lb_rd_server *srv, int64_t timeout_ms);
/* Counters: batched step launches, ticks, requests finished. */
LB_RD_API int lb_rd_server_stats(const lb_rd_server *srv, int64_t *launches, int64_t *ticks, int64_t *finished);

/* Allocation-free fused step.  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory, such as a real-time loop whose
 * memory was all reserved at start-up or a plugin that may only use the
 * buffers its host application hands it.  It never calls cudaMalloc,
 * cudaFree or any allocating library routine.
 *
 * One time step t -> t + 1 of cfg (the same fused kernel as lb_rd_step) from
 * state_in to state_out, and mass_out[s] = sum_x rho_s(t + 1), reduced in
 * FP64.  All three pointers are device memory owned by the caller; state_in
 * and state_out must not overlap.  Work goes on cfg->stream; the call returns
 * without synchronising.
 *
 * State layout: the post-collision distributions f*(t) exactly as they follow
 * the 56-byte header of an lb_rd_save buffer (lb_rd_save's payload up to the
 * density cache).  Rows have a pitch of nx rounded up to a multiple of 32
 * elements.  FP64 / FP32: S * Q planes [s][i][y][pitch] of double / float.
 * 16-bit deviation storage: per species one float plane of rho* followed by
 * Q - 1 planes of 16-bit deviations.
 *
 * Scratch: the reduction's per-block partial sums and its arrival counter
 * live in a static device array of 65536 doubles plus 256 bytes (512 KiB),
 * held by every GPU that loads the library until the process exits.  One
 * block runs per tile (256 x 2 sites in FP32 and 16-bit storage, 32 x 4
 * sites in FP64), and the grid's tiles times S may not exceed 65536: for two
 * species that is up to 16.7 million FP32 sites (4096 x 4096) or 4.2 million
 * FP64 sites (2048 x 2048).  Larger grids return LB_RD_EINVAL with the
 * counts in the message.
 *
 * The first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) and caches it by device
 * ordinal; make that first call before any stream capture.  Only the CUDA
 * runtime's primary context is supported: after cudaDeviceReset (or under
 * another context) the cached address is stale and the entry point must not
 * be called again in that process.  Every call clears the counter on
 * its stream before the kernel.  All calls share the one array, which keeps
 * the last call's contents: calls whose work overlaps on the GPU (different
 * streams, or several host threads) race on it and must be serialised by the
 * caller. */
LB_RD_API int lb_rd_step_noalloc(const lb_rd_config *cfg, const void *state_in, void *state_out, double *mass_out);

#ifdef __cplusplus
}
#endif

#endif /* LB_RD_H */
