/*
 * d4orm.h -- C ABI of the GB300 (sm_103a) D4orm denoising library.
 *
 * D4orm (Zhang et al., IROS 2025) plans collision-free multi-robot
 * trajectories by diffusion-style denoising of a control deformation:
 * each denoising step draws N Monte Carlo deformation samples around the
 * current one (Eq. (12)), rolls every sample's robot team out through the
 * dynamics (Sec. III Eq. (1), Sec. V), scores it with the team reward
 * (Eq. (3)-(5)), and replaces the deformation by a softmax-weighted mean of
 * the samples (Eq. (6), Eq. (13), Algorithm 1).  Algorithm 2 repeats the
 * schedule as an anytime loop around a fixed base trajectory.
 *
 * Conventions (all entry points):
 *  - Plain C types only.  "_dev" pointers are CUDA device pointers owned by
 *    the caller; "_host" pointers are host memory owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is stream-ordered and asynchronous unless stated.
 *  - Argument errors are detected on the host before any launch and return
 *    D4ORM_ERR_INVALID_ARG / D4ORM_ERR_UNSUPPORTED; nothing is launched.
 *    CUDA failures return D4ORM_ERR_CUDA; d4orm_last_error() gives the
 *    message of the calling thread's last failure.  Nothing throws across
 *    the ABI and there is no CPU fallback: without a usable GPU every
 *    compute call returns D4ORM_ERR_CUDA.
 *  - Layouts: controls and deformations are float[T][n][d_u] (time-major,
 *    robots contiguous); states are float[T+1][n][d_x] with states[0] = S.
 *  - A problem handle carries device workspace (allocated on first use,
 *    grown when N grows); calls that use one handle must not overlap in
 *    time (issue them on one stream, or synchronise between streams).
 *
 * Dimensions per dynamics model (Sec. V, plus the unicycle):
 *   HOLO2D     x=[px,py,vx,vy]          u=[ax,ay]        d_x=4 d_u=2
 *   HOLO3D     x=[px,py,pz,vx,vy,vz]    u=[ax,ay,az]     d_x=6 d_u=3
 *   UNICYCLE   x=[px,py,theta]          u=[v,omega]      d_x=3 d_u=2
 *   DIFFDRIVE4 x=[px,py,theta,v]        u=[omega,a]      d_x=4 d_u=2
 */
#ifndef D4ORM_H
#define D4ORM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    D4ORM_OK = 0,
    D4ORM_ERR_INVALID_ARG = 1,  /* null pointer, size out of range, bad enum  */
    D4ORM_ERR_UNSUPPORTED = 2,  /* valid but beyond the library's limits     */
    D4ORM_ERR_OOM = 3,          /* device or pinned allocation failed         */
    D4ORM_ERR_CUDA = 4,         /* a CUDA call failed (see d4orm_last_error)  */
    D4ORM_ERR_TIMEOUT = 5,      /* a bounded device wait expired              */
    D4ORM_ERR_CANCELLED = 6     /* cancelled by the caller                    */
} d4orm_status;

typedef enum {
    D4ORM_DYN_HOLO2D = 0,
    D4ORM_DYN_HOLO3D = 1,
    D4ORM_DYN_UNICYCLE = 2,
    D4ORM_DYN_DIFFDRIVE4 = 3
} d4orm_dynamics;

typedef enum {
    D4ORM_INT_EULER = 0,        /* x += dt f(x, u)                           */
    D4ORM_INT_RK4 = 1           /* classical RK4, control held over the step */
} d4orm_integrator;

#define D4ORM_MAX_ROBOTS 32         /* robots share one warp                   */
#define D4ORM_MAX_ITERS 4096        /* iteration index fits 12 counter bits    */
#define D4ORM_MAX_TAG ((1u << 20) - 1)
#define D4ORM_MAX_CTRL 49152        /* T * n * d_u (mean controls in shared memory) */
#define D4ORM_MAX_OBSTACLES 16

typedef struct d4orm_problem d4orm_problem;

/* Problem of Sec. III: n robots of radius R_a, dynamics f_dyn, horizon T
 * (the paper's H; T controls per robot, states x_0..x_T), start S and
 * terminal state (goal; positions are what the terminal test uses). */
typedef struct {
    int n_robots;               /* 1..32                                      */
    int T;                      /* >= 1                                       */
    int dyn;                    /* d4orm_dynamics                             */
    int integ;                  /* d4orm_integrator                           */
    float dt;                   /* > 0                                        */
    float radius;               /* R_a > 0                                    */
    float eps_margin;           /* epsilon of Eq. (5), >= 0                   */
    float goal_tol;             /* terminal-condition tolerance [m], >= 0     */
    float v_max;                /* per-axis speed bound (holonomic; the speed
                                   state of DIFFDRIVE4); <= 0 means none      */
    const float *start;         /* host [n][d_x], copied at create            */
    const float *goal;          /* host [n][d_x], copied at create            */
    const float *u_lo;          /* host [d_u] control box, copied; NULL = the
                                   model's default box                        */
    const float *u_hi;          /* host [d_u]                                 */
    int n_obstacles;            /* 0..D4ORM_MAX_OBSTACLES static spherical
                                   obstacles (Appendix): each robot-step
                                   inside radius + R_a + eps costs w in
                                   Eq. (3); safety needs > radius + R_a     */
    const float *obstacles;     /* host [n_obstacles][4]: centre x, y, z
                                   (z ignored in 2D), radius > 0; copied     */
} d4orm_problem_desc;

/* Update rules.  DENOISE is the method (Eq. (12)-(13)): samples
 * dU_i / sqrt(abar_i) + sqrt(1/abar_i - 1) eps, new deformation
 * sqrt(abar_{i-1}) * (weighted mean).  MPPI is the softmax update the paper
 * contrasts its schedule with (Sec. IV-B; Williams et al.): samples
 * dU + mppi_sigma * eps around the current deformation and the new
 * deformation is their weighted mean, the same at every step (no
 * schedule; beta0/beta1 unused).  Both use the same sampling, rollout,
 * Eq. (3) fitness, Sec. IV-C normalisation and Eq. (6) weights. */
#define D4ORM_UPDATE_DENOISE 0
#define D4ORM_UPDATE_MPPI 1

/* Denoising parameters (Algorithm 1, Sec. IV-B/C). */
typedef struct {
    int n_samples;              /* N (the paper's M), >= 1                    */
    int n_steps;                /* K (the paper's N), 1..(1<<24)-1            */
    float temperature;          /* lambda of Eq. (6), > 0                     */
    float w_safe;               /* w of Eq. (3)                               */
    float beta0, beta1;         /* linear noise schedule, 0 < beta < 1        */
    uint64_t seed;              /* Philox key                                 */
    uint32_t instance_tag;      /* <= D4ORM_MAX_TAG; separates instances      */
    int update_rule;            /* D4ORM_UPDATE_DENOISE (0) or _MPPI (1)      */
    float mppi_sigma;           /* MPPI sample standard deviation, > 0 when
                                   update_rule is MPPI; unused otherwise     */
} d4orm_params;

/* Anytime budget of Algorithm 2. */
typedef struct {
    int max_iters;              /* 1..D4ORM_MAX_ITERS                         */
    double deadline_ms;         /* <= 0: none; else stop after the iteration
                                   during which it passed (host clock)       */
    int stop_on_success;        /* stop after the first collision-free,
                                   goal-reaching iteration                   */
    int start_step;             /* with du_init: first iteration runs steps
                                   start_step..1 from dU = du_init           */
} d4orm_budget;

/* Eq. (1)/(2) evaluation of one plan. */
typedef struct {
    int collision_free;         /* |p_k - p_l| > 2 R_a for all t in 0..T, and
                                   clear of every obstacle (radius + R_a)   */
    int goal_reached;           /* |p_k[T] - goal_k| <= goal_tol for all k    */
    float reward;               /* Eq. (3)                                    */
    float objective;            /* Eq. (2): fraction of (k, t>=1) at goal     */
    float min_pair_dist;        /* over t in 0..T (1e30 for one robot)        */
} d4orm_verdict;

typedef struct {
    d4orm_verdict verdict;      /* of the returned plan                       */
    int iters_run;              /* completed iterations                       */
    int first_success_iter;     /* -1 if none                                 */
    double ms_to_success;       /* host wall clock from call entry; -1 if none*/
    double ms_total;            /* host wall clock of the whole call          */
    int stop_reason;            /* D4ORM_STOP_BUDGET (max_iters or success),
                                   D4ORM_STOP_DEADLINE or D4ORM_STOP_CANCELLED */
} d4orm_result;

#define D4ORM_STOP_BUDGET 0
#define D4ORM_STOP_DEADLINE 1
#define D4ORM_STOP_CANCELLED 2

/* Create a problem (Sec. III).  Copies every host array; allocates no
 * device memory (device workspace is allocated on first compute call).
 * Errors: INVALID_ARG for null desc/out/start/goal, n/T/dt/radius out of
 * range, bad enums, u_lo > u_hi, obstacles with radius <= 0 or a null
 * array; UNSUPPORTED for n > 32, T * n * d_u > D4ORM_MAX_CTRL or more than
 * D4ORM_MAX_OBSTACLES obstacles.  *out is NULL on error. */
d4orm_status d4orm_problem_create(const d4orm_problem_desc *desc, d4orm_problem **out);

/* Frees the handle and its device workspace (synchronises the device work
 * the handle issued).  NULL is a no-op. */
void d4orm_problem_destroy(d4orm_problem *problem);

/* Rollout + fitness kernel used by the denoising steps of a problem.
 * REGISTER: one warp holds 32/SEG samples (SEG = next power of two >= n),
 * robots in lanes, state in registers over the whole horizon, pair terms by
 * shuffles.  PAIRED: the same with two robots per lane (32/(SEG/2) samples
 * per warp), the two robots' state sharing 64-bit registers so that their
 * arithmetic issues as packed f32x2 instructions.  PIPELINE: one rollout
 * warp per 32/SEG samples plus helper warps that generate the noise of the
 * next time chunk and score the previous one (for batches too small to
 * fill the GPU with the register kernel).  AUTO picks PAIRED for 2D/3D
 * holonomic teams of n >= 5 when the paired kernel has at least 6 warps per
 * SM (12 with obstacles), else PIPELINE when the register kernel would have
 * fewer than 2.5 warps per SM, else REGISTER (the pipelined kernel also
 * needs its shared memory to fit in 200 KB); the thresholds are measured
 * crossovers on GB300.  All compute the same fitness (summation order
 * aside). */
typedef enum {
    D4ORM_ROLLOUT_AUTO = 0,
    D4ORM_ROLLOUT_REGISTER = 1,
    D4ORM_ROLLOUT_PIPELINE = 2,
    D4ORM_ROLLOUT_PAIRED = 3
} d4orm_rollout_kernel;

/* Choose the rollout kernel of a problem (default AUTO).  Host only.
 * Errors: INVALID_ARG for a null problem or an unknown kind. */
d4orm_status d4orm_problem_set_rollout_kernel(d4orm_problem *problem, int kernel);

/* The kernel (REGISTER, PIPELINE or PAIRED) the problem's steps use for
 * n_samples samples on the current device; -1 on error. */
int d4orm_problem_rollout_kernel(const d4orm_problem *problem, int n_samples);

/* How many iteration graphs d4orm_solve has captured on this handle so far
 * (a diagnostic: a timed solve whose iteration shapes were all seen twice
 * before replays graphs and captures none); -1 for a null handle.  The
 * paper has no counterpart. */
long long d4orm_problem_graph_captures(const d4orm_problem *problem);

/* Rollout of one plan (Sec. IV-C; Algorithm 1 final line, Algorithm 2
 * update): controls u_dev[T][n][d_u] are held to the control box and
 * integrated from S.  states_dev (nullable) receives float[T+1][n][d_x].
 * verdict_host (nullable) receives the Eq. (1)/(2) verdict with the reward
 * weight of `params` (nullable: w_safe = 5); when it is given, the call
 * synchronises `stream` before returning. */
d4orm_status d4orm_rollout(d4orm_problem *problem, const d4orm_params *params, const float *u_dev,
                           float *states_dev, d4orm_verdict *verdict_host, void *stream);

/* One denoising step i (Algorithm 1 body, on deformations per Algorithm 2):
 *   samples   dU_j = dU_i / sqrt(abar_i) + sqrt(1/abar_i - 1) eps_j  (Eq. (12))
 *   fitness   r_j  = Eq. (3) of rollout(S, clip(u_base + dU_j))
 *   weights   w_j  = softmax(zscore(r) / lambda)                     (Eq. (6))
 *   update    dU_{i-1} = sqrt(abar_{i-1}) * sum_j w_j dU_j          (Eq. (13))
 * eps_j is regenerated from Philox4x32-10 (never stored), indexed by
 * (iter, step_i, j, robot, element): see d4orm_sample_noise.
 * u_base_dev, du_in_dev: [T][n][d_u]; du_out_dev: [T][n][d_u] (must not
 * alias du_in_dev); fitness_dev: nullable float[N] receiving r_j.
 * Errors: INVALID_ARG for null pointers, step_i not in 1..K, iter not in
 * 0..D4ORM_MAX_ITERS-1, bad params; OOM if the workspace cannot grow. */
d4orm_status d4orm_denoise_step(d4orm_problem *problem, const d4orm_params *params, int iter, int step_i,
                                const float *u_base_dev, const float *du_in_dev, float *du_out_dev,
                                float *fitness_dev, void *stream);

/* The first half of denoising step i on its own: the N samples of Eq. (12),
 * their rollouts and their Eq. (3) fitness r_j (Algorithm 1, sampling,
 * rollout and reward lines), with no weights and no update.  The values
 * are those d4orm_denoise_step writes to fitness_dev for the same
 * arguments.  u_base_dev, du_in_dev: [T][n][d_u]; fitness_dev: float[N]
 * (required).  The call allocates nothing after the problem's first step
 * of this N and makes no synchronising call, so it can be captured in a
 * CUDA graph.  Errors: as d4orm_denoise_step. */
d4orm_status d4orm_sample_fitness(d4orm_problem *problem, const d4orm_params *params, int iter, int step_i,
                                  const float *u_base_dev, const float *du_in_dev, float *fitness_dev,
                                  void *stream);

/* d4orm_denoise_step with a CUDA event recorded on `stream` between its
 * kernels; synchronises and writes the device time of each kernel, in ms,
 * to kernel_ms_host[3]: {rollout+fitness, softmax weights, weighted noise
 * sum with the Eq. (13) update}.  A ~200 us sleep kernel runs first so that the events
 * bracket device time, not host submission.
 * Results are identical to d4orm_denoise_step. */
d4orm_status d4orm_denoise_step_timed(d4orm_problem *problem, const d4orm_params *params, int iter, int step_i,
                                      const float *u_base_dev, const float *du_in_dev, float *du_out_dev,
                                      float *fitness_dev, float *kernel_ms_host, void *stream);

/* Allocation-free denoising step.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- a planner inside a
 * robot's real-time control loop, where cudaMalloc may synchronise the
 * device and has no latency bound, or a host application that reserves all
 * device memory in its own pool up front and forbids allocations by
 * libraries.  It computes exactly what d4orm_denoise_step computes (same
 * kernels, same launch shapes), but its scratch (weights, fitness when
 * fitness_dev is NULL, batch statistics) lives in a fixed 2 MiB array
 * inside the library's device image instead of the problem's workspace, so
 * the call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.  (d4orm_problem_create allocates no device memory.)
 * The caller still passes every input and output buffer.
 *  - Limits: n_samples <= D4ORM_NOALLOC_MAX_SAMPLES (the scratch, 3 floats
 *    per sample plus 64, then fits in D4ORM_NOALLOC_SCRATCH_FLOATS); beyond
 *    it the call returns D4ORM_ERR_UNSUPPORTED before launching anything.
 *  - Each call looks up the array's device address with the calling
 *    thread's device current (the host-side name of the array is only a
 *    stand-in) and sets the problem's rollout-kernel attributes; the first
 *    call on a device also reads its SM count.  A changed address (the
 *    context was re-created, e.g. after cudaDeviceReset) renews that
 *    cached set-up.  Make the first call on a device, and the first after
 *    a reset, before any stream capture.
 *  - Every call on a device shares the one array, which keeps the last
 *    call's contents (nothing in it needs to start at zero: each call writes
 *    all it reads).  Calls whose GPU work overlaps -- on different streams or
 *    from different host threads -- race on it; serialise them.
 *  - Arguments and errors as d4orm_denoise_step. */
#define D4ORM_NOALLOC_SCRATCH_FLOATS (1 << 19)
#define D4ORM_NOALLOC_MAX_SAMPLES 65536
d4orm_status d4orm_denoise_step_noalloc(const d4orm_problem *problem, const d4orm_params *params, int iter,
                                        int step_i, const float *u_base_dev, const float *du_in_dev,
                                        float *du_out_dev, float *fitness_dev, void *stream);

/* Algorithm 2 with an anytime budget.  tau.u starts at zero.  Each
 * iteration runs steps K..1 from dU_K = 0 (Sec. IV-D), or, in the first
 * iteration when du_init_dev is given, steps start_step..1 from
 * dU = du_init_dev; then tau.u <- clip(tau.u + dU_0) and the plan is rolled
 * out and judged.  u_out_dev [T][n][d_u] receives the final tau.u;
 * out_host (nullable) the result.  Synchronises `stream`.  Steps of one
 * iteration are replayed from a CUDA graph cached in the handle. */
d4orm_status d4orm_solve(d4orm_problem *problem, const d4orm_params *params, const d4orm_budget *budget,
                         const float *du_init_dev, float *u_out_dev, d4orm_result *out_host, void *stream);

/* Ask the running (or the next) d4orm_solve of this problem to stop before
 * its next iteration: it returns D4ORM_ERR_CANCELLED with the plan of the
 * iterations already completed (stop_reason D4ORM_STOP_CANCELLED).  The
 * request is consumed by that solve.  A solve without stop_on_success and
 * without a deadline enqueues its iterations without waiting for them, so
 * a request arriving during it stops only the iterations not yet enqueued.
 * Thread-safe.  The paper has no counterpart (a host control). */
d4orm_status d4orm_problem_cancel(d4orm_problem *problem);

/* ---------------------------------------------------------------------------
 * Batched persistent solve.  Many independent problems -- any mix of robot
 * counts, horizons and dynamics -- solved by Algorithm 2 in ONE persistent
 * kernel launch replayed from a CUDA graph.  Each CTA takes problems from
 * an atomic work queue (longest first) and runs every step and iteration of
 * one problem with block-level synchronisation only; CTAs never wait on
 * each other.  Problem b draws its noise with instance tag
 * params->instance_tag + b, so it reproduces d4orm_solve of that problem
 * with that tag (up to the order of floating-point reductions).
 * ------------------------------------------------------------------------- */
typedef struct d4orm_batch d4orm_batch;

#define D4ORM_BATCH_MAX_SAMPLES 8192

/* Build a batch over problems[0..count-1] (handles must outlive the batch)
 * with one set of denoising parameters.  Uploads descriptors and allocates
 * per-problem workspace.  autotune != 0 times the persistent kernel at 128,
 * 256 and 512 threads per CTA, each at the maximum resident CTAs per SM,
 * half of it and one, on a 2-step pilot over the whole batch, and keeps
 * the fastest (see d4orm_batch_info, d4orm_batch_tuning), then at that
 * shape chooses the robot-lane packing per bucket of problems (see
 * d4orm_batch_packing); otherwise 512 threads, one CTA per SM, two robots
 * per lane wherever the kernel has that rollout.
 * Errors: INVALID_ARG (null arguments, bad params, tags beyond
 * D4ORM_MAX_TAG), UNSUPPORTED (n_samples > D4ORM_BATCH_MAX_SAMPLES, or
 * shared memory above 200 KB: 4 bytes per control of the largest problem,
 * 12 per sample, and 24 KB of per-warp position buffers), OOM, CUDA. */
d4orm_status d4orm_batch_create(d4orm_problem *const *problems, int count, const d4orm_params *params,
                                int autotune, d4orm_batch **out);

/* Solve every problem of the batch.  u_out_dev: host array [count] of
 * device pointers, each [T_b][n_b][d_u_b] (final tau.u).  du_init_dev:
 * nullable host array [count] of device pointers: warm-start deformations
 * entering the first iteration at budget->start_step.  out_host (nullable):
 * [count] results; ms_to_success / ms_total are device-clock times of each
 * problem's own solve (from when its CTA picked it up).
 * Anytime stops (Sec. IV-D: the plan of the last completed iteration is
 * always a valid answer), checked by every CTA before each denoising step:
 *  - budget->deadline_ms > 0: device clock since the launch; a problem
 *    whose deadline passes keeps the plan of its completed iterations
 *    (stop_reason D4ORM_STOP_DEADLINE) and problems not yet started get
 *    none (iters_run 0).
 *  - d4orm_batch_cancel from any host thread (or before the call): the
 *    same, with stop_reason D4ORM_STOP_CANCELLED.
 * Returns D4ORM_ERR_CANCELLED if the solve was cancelled, D4ORM_ERR_TIMEOUT
 * if the deadline left some problem without any completed iteration, else
 * OK; plans and results are written in every case.  Synchronises the
 * device before and `stream` after the launch. */
d4orm_status d4orm_batch_solve(d4orm_batch *batch, const d4orm_budget *budget, const float *const *du_init_dev,
                               float *const *u_out_dev, d4orm_result *out_host, void *stream);

/* Launch shape the batch uses and the autotuner's best pilot time (ms, -1
 * when a width was not tried) for 128 / 256 / 512 threads per CTA. */
d4orm_status d4orm_batch_info(const d4orm_batch *batch, int *threads_per_cta, int *ctas, float *tuned_ms);

/* Every pilot the autotuner ran (0 without autotuning): *count entries of
 * (threads per CTA, resident CTAs per SM, pilot ms), at most `capacity`
 * written to the nullable host arrays.  The autotuner tries widths 128,
 * 256 and 512 at the maximum resident CTAs per SM, half of it and one. */
d4orm_status d4orm_batch_tuning(const d4orm_batch *batch, int capacity, int *count, int *threads_per_cta,
                                int *ctas_per_sm, float *pilot_ms);

/* Robot-lane packing of the batched solver's sample rollouts.  SINGLE: one
 * robot per lane.  PAIRED: two robots per lane, their pair tests and goal
 * terms (and, for holonomic teams, their integration) issued as packed
 * f32x2 arithmetic; the kernel has this rollout for teams of 5..16 robots,
 * and other problems keep one robot per lane.  Both give the same rewards
 * up to the order of float sums. */
enum { D4ORM_PACK_SINGLE = 0, D4ORM_PACK_PAIRED = 1 };

/* Set the packing of every problem of the batch (overrides the
 * autotuner's per-bucket choice; takes effect at the next solve).
 * Synchronises the device.  Errors: INVALID_ARG (null batch, unknown
 * mode), CUDA. */
d4orm_status d4orm_batch_set_packing(d4orm_batch *batch, int mode);

/* The packing each problem uses: paired[b] = 1 for two robots per lane (at
 * most `capacity` entries, nullable).  bucket_ns (nullable, 16 entries):
 * the autotuner's packing pilots, summed device ns of the problems of each
 * bucket with one and then two robots per lane, buckets in the order
 * (dynamics d, 5..8 robots), (d, 9..16 robots) for d = D4ORM_DYN_HOLO2D,
 * HOLO3D, UNICYCLE, DIFFDRIVE4; zeros without autotuning.  With
 * autotuning a bucket is packed when its paired sum is the smaller;
 * without it, every packable problem is. */
d4orm_status d4orm_batch_packing(const d4orm_batch *batch, int capacity, int *paired, long long *bucket_ns);

/* Request that the running (or the next) d4orm_batch_solve of this batch
 * stop at the next denoising-step boundary of every CTA.  Thread-safe; sets
 * a flag in host memory mapped into the device, which the solve clears
 * when it returns.  The paper has no counterpart (a host control). */
d4orm_status d4orm_batch_cancel(d4orm_batch *batch);

/* Free a batch (synchronises the device).  NULL is a no-op. */
void d4orm_batch_destroy(d4orm_batch *batch);

/* One-shot convenience: create (no autotuning), solve, destroy. */
d4orm_status d4orm_solve_batched(d4orm_problem *const *problems, int count, const d4orm_params *params,
                                 const d4orm_budget *budget, float *const *u_out_dev, d4orm_result *out_host,
                                 void *stream);

/* ---------------------------------------------------------------------------
 * Learned warm start (not part of the paper, whose method has no learning
 * component): a set-MLP that maps a team's starts and goals to a control
 * plan, trained on plans the method itself produced, used to seed the
 * deformation so that denoising can start at an intermediate step; the
 * plain method stays the fallback.
 *
 * Network, per team (robots padded to n_max, padded rows masked):
 *   x_k (16 features: start/scale, goal/scale, (goal-start)/scale,
 *        |goal-start|/scale, 1, zero padding; 3 slots per vector, z = 0 in 2D)
 *   H1 = relu(x W1' + b1), H2 = relu(H1 W2' + b2), H3 = relu(H2 W3' + b3)
 *   Pbar = masked mean of H3 over robots
 *   H4 = relu([H3, Pbar] W4' + b4), H5 = relu(H4 W5' + b5), Y = H5 W6' + b6
 *   (Y_k = robot k's controls, T * d_u values ordered t-major)
 * Loss: masked mean squared error against the target plans.  GEMMs run on
 * the tensor cores in BF16 with FP32 accumulation; parameters are FP32
 * masters (flat vector: W1, b1, W2, b2, ..., W6, b6; W_l row-major
 * [out][in]) with BF16 copies; AdamW updates the masters.
 * ------------------------------------------------------------------------- */
typedef struct d4orm_warmstart d4orm_warmstart;

typedef struct {
    int n_max;          /* robots per team (padded), 1..32                    */
    int T, d_u;         /* plan shape predicted per robot                     */
    int width;          /* hidden width (multiple of 16, <= 1024)             */
    int max_batch;      /* teams per forward/training batch                   */
    uint64_t seed;      /* initialisation (uniform +-1/sqrt(fan_in), zero bias) */
    float lr, beta1, beta2, eps, weight_decay;   /* AdamW                     */
    float pos_scale;    /* metres per unit of the position features          */
} d4orm_warmstart_desc;

/* Create a network with seeded initial weights.  Errors: INVALID_ARG for
 * shapes out of range; OOM; CUDA. */
d4orm_status d4orm_warmstart_create(const d4orm_warmstart_desc *desc, d4orm_warmstart **out);
void d4orm_warmstart_destroy(d4orm_warmstart *ws);

/* Number of FP32 parameters (-1 for NULL). */
int d4orm_warmstart_param_count(const d4orm_warmstart *ws);

/* Copy the FP32 master parameters to / from host memory (count must equal
 * the parameter count).  set_params also resets the AdamW state. */
d4orm_status d4orm_warmstart_get_params(const d4orm_warmstart *ws, float *host, int count);
d4orm_status d4orm_warmstart_set_params(d4orm_warmstart *ws, const float *host, int count);

/* Forward pass of B teams: x_dev [B][n_max][16], mask_dev [B][n_max],
 * y_dev [B][n_max][T*d_u].  Asynchronous on `stream`. */
d4orm_status d4orm_warmstart_forward(d4orm_warmstart *ws, const float *x_dev, const float *mask_dev, int B,
                                     float *y_dev, void *stream);

/* Forward + masked MSE against y_dev + backward, without updating.
 * loss_host (nullable; synchronises), grad_dev (nullable) receives the flat
 * FP32 gradient (parameter layout). */
d4orm_status d4orm_warmstart_loss_grad(d4orm_warmstart *ws, const float *x_dev, const float *mask_dev,
                                       const float *y_dev, int B, float *loss_host, float *grad_dev, void *stream);

/* One AdamW training step on B teams.  With idx_dev (int[B]) the teams are
 * gathered from a dataset x_all [*][n_max][16], mask_all [*][n_max],
 * y_all [*][n_max][T*d_u]; with idx_dev NULL the first B teams are used.
 * loss_host (nullable; synchronises) receives the loss before the update. */
d4orm_status d4orm_warmstart_train_step(d4orm_warmstart *ws, const float *x_all, const float *mask_all,
                                        const float *y_all, const int *idx_dev, int B, float *loss_host,
                                        void *stream);

/* Input features of one problem (host): x_host [n_max][16], mask_host [n_max]. */
d4orm_status d4orm_warmstart_features(const d4orm_problem *problem, int n_max, float pos_scale, float *x_host,
                                      float *mask_host);

/* Seed for d4orm_solve / d4orm_batch_solve: du_seed_dev [T][n][d_u] =
 * sqrt(abar_{start_step}) * Y (the network's plan for the problem), so the
 * first sampled mean at start_step is the predicted plan itself (base plan
 * zero).  Synchronises `stream`. */
d4orm_status d4orm_warmstart_predict(d4orm_warmstart *ws, const d4orm_problem *problem, const d4orm_params *params,
                                     int start_step, float *du_seed_dev, void *stream);

/* The sample noise eps of Eq. (12) exactly as the step kernels regenerate
 * it: eps_dev[count][T][n][d_u] for samples j0..j0+count-1 of (iter,
 * step_i).  Element e = t*d_u + d of robot k's stream, quad q = e/4, takes
 * word e%4 of Philox4x32-10 with counter (q, j, (k & 0xff) | (step_i << 8),
 * iter | (tag << 12)) and key (seed lo, seed hi), through Box-Muller on
 * word pairs (0,1) and (2,3).  Used by parity tests. */
d4orm_status d4orm_sample_noise(d4orm_problem *problem, const d4orm_params *params, int iter, int step_i,
                                int j0, int count, float *eps_dev, void *stream);

/* Raw Philox4x32-10 (Salmon et al., SC'11): out_dev[i][0..3] =
 * Philox(ctr_dev[i][0..3], key = (key0, key1)) for i < count. */
d4orm_status d4orm_philox4x32_10(const uint32_t *ctr_dev, uint32_t key0, uint32_t key1, int count,
                                 uint32_t *out_dev, void *stream);

/* Measured FP32 peak, the denominator the rollout kernel's FP32 fraction is
 * also quoted against (the paper has no counterpart: this is a roofline
 * instrument).  Launches `blocks` x `threads` threads, each running eight
 * independent chains of `iters` fused multiply-adds, i.e.
 * blocks * threads * iters * 16 FLOPs; time it with events on `stream`.
 * out_dev (device, caller-owned) receives blocks * threads floats.
 * threads must be a multiple of 32 in 32..1024; asynchronous. */
d4orm_status d4orm_fp32_fma_probe(float *out_dev, int blocks, int threads, int iters, void *stream);

/* Static string for a status code. */
const char *d4orm_status_string(d4orm_status status);

/* Message of the calling thread's last failed call ("" if none). */
const char *d4orm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* D4ORM_H */
