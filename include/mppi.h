/*
 * mppi.h -- C ABI of the GB300 MPPI library (libmppi_gb300.so).
 *
 * One call solves one MPPI optimisation step of "Model Predictive Path
 * Integral Control for Agile Unmanned Aerial Vehicles" (arXiv 2407.09812):
 * sample K perturbed control sequences (Sec. III-A, Eq. rollout_computation),
 * roll each out through the quadrotor model with its motor constraints over
 * N steps (Sec. III-B), score it with the tracking / input / obstacle cost
 * (Sec. IV-C, Sec. IV-D), weight the samples by the softmin of Eq. cost_2
 * and return the updated nominal sequence of Eq. u_update together with the
 * command sent to the low-level controller and the shifted warm start
 * (Alg. 1).
 *
 * Layouts (all float32, row major, no padding):
 *   state     x[13]      = p(3) [m], q(4) = (w, x, y, z) unit quaternion
 *                          rotating body to world, v(3) [m/s], omega(3)
 *                          body rates [rad/s]; world z up, gravity -z.
 *   control   u[4]       = F_t [N], omega_d(3) [rad/s] desired body rates.
 *   reference ref[N+1][13]  x_ref_0 .. x_ref_N, same layout as a state.
 *   nominal   u_nom[N][4]
 *   obstacle  obs[M][4]  = (cx, cy, cz, r); r >= 0 a sphere of radius r,
 *                          r < 0 a vertical infinite cylinder of radius |r|
 *                          (cz unused).  The pointer must be 16-byte
 *                          aligned (it is staged with bulk copies).
 *
 * Ownership: the caller owns every buffer it passes; the library never
 * keeps a caller pointer beyond the call (synchronous entry points) or
 * beyond completion of the work enqueued on the given stream
 * (asynchronous entry points), except the occupancy grid of mppi_set_grid
 * and the counter of mppi_set_counters, which a handle uses until they are
 * replaced or removed.  A handle owns its device workspace.
 *
 * Errors: every entry point returns MPPI_OK (0) or a negative code.
 * Arguments are validated on the host before any device work is queued;
 * on MPPI_EINVAL nothing is written.  Handles are not thread safe; a
 * server (mppi_server_*) is.  No entry point throws or aborts.
 */
#ifndef MPPI_GB300_H
#define MPPI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPPI_OK 0
#define MPPI_EINVAL (-1)     /* bad size, pointer, alignment or parameter   */
#define MPPI_ENOMEM (-2)     /* device memory or admission budget exceeded  */
#define MPPI_ECUDA (-3)      /* a CUDA runtime call failed                  */
#define MPPI_ETIMEOUT (-4)   /* a bounded device-side wait gave up          */
#define MPPI_ENONFINITE (-5) /* every rollout cost was non-finite           */
#define MPPI_EAGAIN (-6)     /* queue full / nothing ready; retry later     */
#define MPPI_ENOTFOUND (-7)  /* unknown vehicle or request id               */

#define MPPI_N_MAX 1024      /* largest horizon N                            */
#define MPPI_M_MAX 8192      /* largest obstacle count M per instance        */
#define MPPI_K_MAX (1 << 24) /* largest sample count K per instance          */

/* Vehicle model and input limits (Table I of the paper; Sec. III-B). */
typedef struct {
    float mass;        /* m [kg]                                            */
    float g;           /* |g| [m/s^2]                                       */
    float arm_l;       /* arm length l [m] (allocation matrix Gamma)        */
    float c_tf;        /* rotor torque constant c_tf [m]                    */
    float J[3];        /* diagonal inertia [kg m^2]                         */
    float T_min;       /* per-rotor thrust limits [N] (Eq. clipping)        */
    float T_max;
    int32_t motor_clip;/* 1: clip rotor thrusts; 0: no rotor limits        */
    float F_min;       /* box on the desired collective thrust [N]          */
    float F_max;
    float w_max[3];    /* box on the desired body rates [rad/s] (Sec. IV)   */
} mppi_model;

/* Optimiser and cost parameters (Table II; Sec. IV-C, IV-D). */
typedef struct {
    int32_t K;         /* rollouts                                          */
    int32_t N;         /* prediction steps                                  */
    float dt;          /* prediction time step [s]                          */
    float lambda;      /* temperature of Eq. cost_2, > 0                    */
    float sigma[4];    /* noise standard deviation per control component    */
    float c_p, c_q, c_v, c_w;  /* Eq. rho_ref weights                       */
    float R[4];        /* input weight diagonal (Eq. cost)                  */
    float Rd[4];       /* input-change weight diagonal (Eq. cost)           */
    float c_obs;       /* collision indicator weight (Sec. IV-D)            */
    float c_bar;       /* exponential barrier weight                        */
    float beta;        /* barrier rate [1/m^2]: c_bar exp(-beta max(gap,0)),
                          a term below 2^-48 c_bar counts as 0               */
    float r_uav;       /* vehicle radius added to every obstacle [m]        */
    int32_t quat_metric; /* 0: 1-<q,q_ref>^2 (Eq. quat_approx);
                            1: acos(2<q,q_ref>^2-1) (Eq. quat_angle)        */
    int32_t tail_mode; /* warm start tail: 0 hover u_init, 1 repeat last    */
    float shift_alpha; /* 1: shift by one step (Alg. 1); in (0,1): linear
                          interpolation alpha steps later (Sec. IV-B)       */
    float delay;       /* >= 0 [s]: start the rollouts from x_hat predicted
                          `delay` ahead (delay compensation, Sec. IV-E)     */
    uint64_t seed;     /* Philox key (with stream_id)                       */
    uint32_t stream_id;
    int32_t reserved;  /* must be 0                                         */
} mppi_params;

/* Capacity a handle's device workspace is allocated for at creation (a
 * call that needs more grows it; sizing it up front keeps allocation out of
 * later calls). */
typedef struct {
    int32_t max_instances; /* instances per batched launch (>= 1)           */
    int64_t max_samples;   /* sum of K over one batched launch              */
    int32_t N_max;         /* largest N of any instance                     */
    int32_t M_max;         /* largest M of any instance                     */
} mppi_capacity;

typedef struct mppi_ctx* mppi_handle;

/* Library version and the error string of a code (static storage; the
 * paper has no counterpart).  mppi_strerror never returns NULL: unknown
 * codes give a generic string. */
const char* mppi_version(void);
const char* mppi_strerror(int code);

/* Creates a handle for one vehicle model (Table I, Sec. III-B) and one
 * parameter set (the MPPI settings of Table II and the cost of Sec. IV-C/D)
 * on the current CUDA device; allocates its device workspace for `cap`
 * (NULL: one instance of params->K, params->N, MPPI_M_MAX obstacles).
 * *out is set to NULL on any error.
 * Returns MPPI_EINVAL for non-finite or out-of-range values, MPPI_ENOMEM
 * or MPPI_ECUDA if the workspace cannot be allocated. */
int mppi_create(const mppi_model* model, const mppi_params* params, const mppi_capacity* cap,
                mppi_handle* out);

/* Frees the handle and its workspace (synchronises its device work; the
 * paper has no counterpart).  NULL is ignored. */
void mppi_destroy(mppi_handle h);

/* Replaces the parameter set (Table II settings and cost weights).  Takes
 * effect for calls made afterwards; cached graphs are dropped, and the
 * workspace grows on the next call if K or N exceed what it holds.
 * MPPI_EINVAL (nothing changed) for invalid values. */
int mppi_set_params(mppi_handle h, const mppi_params* params);

/* Grid-based collision module (Sec. IV-D names occupancy maps as one way
 * to test set membership): a dense occupancy grid in DEVICE memory,
 * grid[(iz * ny + iy) * nx + ix] != 0 marking an occupied voxel that spans
 * origin + voxel * ([ix, ix+1) x [iy, iy+1) x [iz, iz+1)); positions outside
 * the grid are free.  A state inside an occupied voxel counts toward the
 * same once-per-state collision indicator as the obstacles (c_obs).  The
 * grid applies to every later solve of the handle (single and batched)
 * and must stay valid and unchanged while they run; grid == NULL removes
 * it.  MPPI_EINVAL for non-positive sizes or voxel, or non-finite origin. */
int mppi_set_grid(mppi_handle h, const uint8_t* grid, int32_t nx, int32_t ny, int32_t nz, const float* origin,
                  float voxel);

/* One MPPI step with HOST buffers, synchronous (Alg. 1, body of the loop).
 * The inputs and `iter` are packed into one pinned block, copied in, solved
 * and copied out on the handle's stream; from the second call with the same
 * sizes and launch shape on, the three are replayed from a CUDA graph.
 *   x_hat[13]          state estimate x^ (host).
 *   ref[(N+1)*13]      reference x_ref_0..x_ref_N (host).
 *   obstacles[M*4]     obstacle set (host, may be NULL when M == 0).
 *   u_nom[N*4]         nominal sequence before the update (host).
 *   iter               Philox counter word of this step (advance per step).
 * Outputs (host, each may be NULL):
 *   u_out[N*4]   updated nominal u_nom_j + sum_k w_k delta u_j^k (Eq. u_update),
 *                before the shift;
 *   u_cmd[4]     [F_clip, omega_clip] from x_hat and u_out_0 (Sec. III-B);
 *   u_next[N*4]  warm start for the next step (shift / interpolation);
 *   x_next[13]   x_hat advanced by the applied command over shift_alpha*dt;
 *   costs[K]     per-sample cost S_k.
 * Returns MPPI_OK, MPPI_EINVAL, MPPI_ECUDA, MPPI_ETIMEOUT, or
 * MPPI_ENONFINITE (every S_k non-finite: u_out = u_nom).  On MPPI_ETIMEOUT
 * (a bounded device wait gave up) the outputs are written but hold
 * unspecified values; on MPPI_EINVAL and MPPI_ECUDA they are not written. */
int mppi_solve(mppi_handle h, const float* x_hat, const float* ref, const float* obstacles, int32_t M,
               const float* u_nom, uint64_t iter, float* u_out, float* u_cmd, float* u_next,
               float* x_next, float* costs);

/* The same step (Alg. 1, body of the loop) with DEVICE buffers, enqueued
 * on `stream` (a cudaStream_t; NULL = legacy default stream); returns
 * after enqueueing.  Buffer sizes and layouts as for mppi_solve; x_hat,
 * ref, u_nom, the outputs and costs must be 4-byte aligned and obstacles
 * 16-byte aligned (MPPI_EINVAL otherwise).  `status`
 * (device int32, may be NULL) receives the step's result code.  All input
 * buffers must stay valid and unchanged until the stream reaches the end
 * of the step.  Graph capture of the stream is allowed. */
int mppi_solve_async(mppi_handle h, const float* x_hat, const float* ref, const float* obstacles,
                     int32_t M, const float* u_nom, uint64_t iter, float* u_out, float* u_cmd,
                     float* u_next, float* x_next, float* costs, int32_t* status, void* stream);

/* One instance of a batched launch.  Pointers are DEVICE pointers with the
 * layouts above; outputs may be NULL.  The model and the cost weights and
 * options (c_*, R, Rd, beta, r_uav, quat_metric, tail_mode, shift_alpha,
 * delay) come from the handle's parameter set; the fields below are per
 * instance. */
typedef struct {
    const float* x_hat;
    const float* ref;
    const float* obstacles;
    const float* u_nom;
    float* u_out;
    float* u_cmd;
    float* u_next;
    float* x_next;
    float* costs;
    int32_t* status;
    uint64_t* iter_dev; /* optional device counter: when non-NULL the step
                           uses *iter_dev and increments it on completion  */
    uint64_t iter;      /* used when iter_dev is NULL                       */
    int32_t K, N, M;
    float dt, lambda;
    float sigma[4];
    uint64_t seed;
    uint32_t stream_id;
    int32_t reserved;   /* must be 0                                        */
} mppi_instance;

/* Many independent MPPI steps (Alg. 1, one per vehicle) of uneven
 * (K, N, M) in one persistent launch on `stream` (the batched form of
 * mppi_solve_async; batching is this library's, not the paper's).  `instances` is a
 * HOST array of n descriptors (copied before return).  The launch shape
 * (block size, samples per warp) is taken from the handle's tuning table
 * (mppi_autotune) or the default for the batch's total K, largest N and
 * largest M (mppi_get_shape).  Every instance's result equals what
 * mppi_solve_async returns for it alone with the same launch shape. */
int mppi_solve_batch(mppi_handle h, const mppi_instance* instances, int32_t n, void* stream);

/* Same as mppi_solve_batch, replayed from a CUDA graph captured once per
 * (capacity bucket, launch shape) and cached in the handle; descriptors
 * are updated in place between replays. */
int mppi_solve_batch_graph(mppi_handle h, const mppi_instance* instances, int32_t n, void* stream);

/* The batched step with HOST buffers, synchronous (the batched form of
 * mppi_solve; Alg. 1, one step per vehicle).  `instances` is a HOST array of
 * n descriptors whose pointers are all HOST pointers; iter_dev must be NULL
 * (the counter is `iter`).  The inputs of all instances are packed, in
 * instance order, into one pinned block of 16-byte aligned segments per
 * instance (x_hat[13] padded to 16, ref[(N+1)*13] padded to a multiple of 4,
 * obstacles[M*4], u_nom[N*4]) and copied in with one copy; the launch is
 * that of mppi_solve_batch_graph; the outputs (per instance u_out[N*4],
 * u_cmd[4], u_next[N*4], x_next[13] padded to 16, status padded to 4, then
 * costs[K] padded to a multiple of 4 when costs != NULL) come back with one
 * copy and are written to the non-NULL output pointers.  An output buffer
 * may be an input buffer (u_next == u_nom for an in-place warm start).
 * Returns MPPI_EINVAL (nothing written), MPPI_ENOMEM, MPPI_ECUDA, or the
 * first non-OK per-instance status in instance order (each instance's
 * `status`, when non-NULL, receives its own). */
int mppi_solve_batch_host(mppi_handle h, const mppi_instance* instances, int32_t n);

/* Measurement hook (the paper has no counterpart): with a DEVICE counter
 * set, every later launch of the handle adds to counters[0] the number of
 * (rollout state, obstacle) pairs it evaluated after its exact culling
 * (pairs whose barrier term is below its floor, 2^-48 of c_bar, where it
 * counts as zero, and that cannot be in collision are skipped).  Used to state the roofline in work actually
 * required.  NULL turns it off.  The counter must be 8-byte aligned. */
int mppi_set_counters(mppi_handle h, uint64_t* counters);

/* Measured throughput of the pipes the step is bound by (the paper has no
 * counterpart): FP32 fused multiply-add and the multi-function unit, each
 * the best of a few launches of a micro-benchmark that fills every SM. */
typedef struct {
    int32_t sm_count;   /* SMs of the current device                      */
    int32_t reserved;
    double fp32_flops;  /* FFMA rate, 2 flop per FMA [flop/s]             */
    double fp32_ms;     /* duration of the timed FFMA launch [ms]         */
    double ex2_ops;     /* ex2.approx results per second                  */
    double lg2_ops;     /* lg2.approx                                     */
    double rsqrt_ops;   /* rsqrt.approx                                   */
    double sin_ops;     /* sin.approx                                     */
    double cos_ops;     /* cos.approx                                     */
} mppi_peaks;

/* Runs the micro-benchmark on the current device and `stream`
 * (synchronous, about 30 ms; allocates a small scratch buffer).  Used to
 * state the roofline against rates measured on the GPU itself. */
int mppi_measure_peaks(mppi_peaks* out, void* stream);

/* The sampling step of Sec. III-A (Eq. rollout_computation: delta u_{k,j}
 * ~ N(0, Sigma), Sigma = diag(sigma^2)) by itself, exactly as the rollouts
 * of a solve with these parameters and iteration count draw it:
 * Philox4x32-10 on the counter (k, j, iter) under the key (seed,
 * stream_id), Box-Muller, times sigma.  Writes delta for samples
 * k0 .. k0 + K - 1 and steps 0 .. N - 1 to out[((k - k0) N + j) 4 + c]
 * (device pointer, 16-byte aligned, K N 4 floats), asynchronously on
 * `stream`.  The paper has no call of its own for this; it exposes the
 * noise so that it can be compared with an independent implementation
 * element by element.  Of params only sigma, seed and stream_id are used
 * (the whole struct is validated).  Returns MPPI_EINVAL for a NULL or
 * misaligned pointer, invalid params, K or N < 1, K > MPPI_K_MAX,
 * N > MPPI_N_MAX or k0 + K > 2^32; MPPI_ECUDA if the launch fails. */
int mppi_sample_noise(const mppi_params* params, uint64_t iter, uint32_t k0, int32_t K, int32_t N,
                      float* out, void* stream);

/* Failure-path hook (the paper has no counterpart).  Every device-side wait
 * of the kernel (the obstacle staging copy, the pipelined form's state
 * ring) is a bounded poll of an mbarrier; polls sets that bound for this
 * handle's later launches (0: the default, about a second of polling).
 * stall_obstacle_copy != 0 makes the launches skip the staging copy of the
 * obstacle list, so that its wait runs out without any fault: every
 * instance with M > 0 then returns MPPI_ETIMEOUT, its outputs unspecified,
 * and the context stays usable.  Used by tests of the timeout path; keep
 * both 0 otherwise.  Returns MPPI_EINVAL for a NULL handle or polls < 0. */
int mppi_set_wait_limit(mppi_handle h, int64_t polls, int32_t stall_obstacle_copy);

/* Launch shape of the rollout kernel. */
typedef struct {
    int32_t block;          /* threads per block: 64, 128, 256 or 512; for
                               the pipelined forms a multiple of
                               32 (pipelined + lanes) up to 512             */
    int32_t lanes;          /* lanes per sample: 1 (one thread per sample),
                               2, 4, 8 or 32 (warp split of the obstacle
                               loop; 32: one sample per warp)               */
    int32_t pipelined;      /* 1 (with lanes 1 or 2): each sample has a
                               dynamics thread and `lanes` cost threads in
                               separate warps, handing states over through
                               shared-memory rings (block / (1 + lanes)
                               samples per block); 2: in addition a noise
                               thread per sample in its own warp that draws
                               the noise ahead of the dynamics thread
                               (block / (2 + lanes) samples per block); 3:
                               in addition the dynamics split over two
                               threads in separate warps, one for the
                               constraint pipeline and the attitude part of
                               RK4, one for velocity, position and the
                               tracking cost, the noise thread forming the
                               clamped control (block / (3 + lanes)
                               samples per block); the per-sample costs of
                               forms 1-3 are bitwise equal                  */
    float list_margin;      /* obstacle tiling: a warp's kept-obstacle list
                               covers the box of its positions grown by
                               this many metres and is reused while they
                               stay inside (0: the default, 1 m, or 0.5 m
                               for the pipelined form; results do not
                               depend on it beyond FP32 rounding)           */
    int32_t samples_per_thread; /* 1 (0 reads as 1), or 2 with pipelined 0,
                               lanes 1 and blocks of 64 or 128 threads:
                               each thread rolls out samples tid and
                               block + tid of its tile, the arithmetic
                               packed across the two (FP32x2); per-sample
                               results equal those of one sample per
                               thread to FP32 rounding                      */
} mppi_shape;

/* Forces a launch shape for subsequent calls on the handle (both 0: back
 * to the tuned/default choice; the paper has no counterpart).
 * MPPI_EINVAL for an unsupported shape or margin. */
int mppi_set_shape(mppi_handle h, const mppi_shape* shape);

/* Project autotuner (the paper has no counterpart): times every candidate shape (block size, samples per
 * warp or two samples per thread, pipelined forms 1-3, then the obstacle
 * tiling of the fastest) on a
 * synthetic problem of size (K, N, M) on `stream`, stores the fastest in
 * the handle's table for that size bucket and returns it in *best (may be
 * NULL).  Synchronous. */
int mppi_autotune(mppi_handle h, int32_t K, int32_t N, int32_t M, mppi_shape* best, void* stream);

/* The same tuning on one of the caller's own problems (DEVICE buffers, as
 * for mppi_solve_batch; validated the same way).  Its outputs are not
 * written and its Philox counter is not advanced.  Preferred over the
 * synthetic problem: the best shape depends on how the obstacles lie
 * relative to the rollouts, which a synthetic problem does not reproduce. */
int mppi_autotune_instance(mppi_handle h, const mppi_instance* instance, mppi_shape* best, void* stream);

/* The same tuning on a whole batch of the caller's instances (DEVICE
 * buffers, as for mppi_solve_batch; the paper has no counterpart): every
 * candidate shape, then the obstacle tiling of the fastest, is timed as
 * one persistent batched launch of these instances (outputs not written,
 * Philox counters not advanced), and the fastest is stored for the key a
 * batch of these instances is looked up under (its mean K, largest N and
 * largest M).  Synchronous. */
int mppi_autotune_batch(mppi_handle h, const mppi_instance* instances, int32_t n, mppi_shape* best,
                        void* stream);

/* Looks up the shape the handle uses for a problem of size (K, N, M)
 * (the paper has no counterpart): the forced shape, else the tuned one
 * for the size bucket, else the default for a launch of K samples on this
 * GPU's S multiprocessors:
 *   K <= 128 S: pipelined form 3 with the smallest tile of 32, 64 or 128
 *     samples (block 128, 256 or 512) that keeps one tile per
 *     multiprocessor, when its shared memory fits;
 *   K <= 256 S and M >= 16: pipelined form 1, block 256 (128 samples);
 *   K > 256 (S - 1): two samples per thread in blocks of 128, unless the
 *     busiest multiprocessor gets more than 8 % more samples with
 *     256-sample tiles than with 128-sample tiles;
 *   otherwise one thread per sample in blocks of 128.
 * For a batch the default takes its total K (the tuning table its mean K),
 * largest N and largest M. */
int mppi_get_shape(mppi_handle h, int32_t K, int32_t N, int32_t M, mppi_shape* shape);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of solve requests from many vehicles.
 * Each vehicle's nominal sequence and Philox counter stay on the device
 * between its requests (warm start: the step's shifted nominal replaces
 * the stored one, Alg. 1).  A dispatcher thread forms a batch from the
 * queued requests whenever one of `slots` launch slots is free, so
 * requests that arrive while earlier batches run are admitted as slots
 * free up and their work overlaps on the device.  A vehicle has at most
 * one request in flight; its later requests wait in the queue.  Vehicles
 * are admitted against a device-memory budget that also covers the slots'
 * workspaces.  All server entry points are thread safe.
 * ------------------------------------------------------------------- */
typedef struct mppi_server mppi_server;

typedef struct {
    int32_t max_vehicles;
    int32_t slots;             /* batches in flight at once (one stream each) */
    int32_t max_batch;         /* instances per batch                         */
    int32_t N_max, M_max;      /* largest N and M of any vehicle              */
    int32_t queue_capacity;    /* queued requests before MPPI_EAGAIN          */
    int64_t max_batch_samples; /* sum of K per batch                          */
    int64_t hbm_budget_bytes;  /* device bytes for vehicle state + slots      */
    int32_t block, lanes;      /* launch shape; 0, 0: automatic               */
} mppi_server_cfg;

typedef struct {
    uint64_t request_id;
    int32_t vehicle;
    int32_t status;            /* MPPI_OK or the step's error code            */
    float u_cmd[4];            /* [F_clip, omega_clip] to the flight controller */
    float u0[4];               /* updated nominal u_out_0                     */
    double t_submit_us;        /* host steady clock, microseconds             */
    double t_done_us;          /* when the dispatcher saw the batch complete  */
    int32_t batch_size;        /* instances in the batch that served it       */
    int32_t reserved;
} mppi_result;

typedef struct {
    int64_t submitted, completed, rejected, batches, instances;
    int64_t bytes_in_use, bytes_budget;
    double busy_us;            /* sum over batches of launch-to-completion time */
} mppi_server_stats;

/* Serving (the paper runs one controller per vehicle; continuous batching
 * of many vehicles' solves is this library's).  Every request is one
 * Alg. 1 step of its vehicle with the warm start and Philox counter kept
 * on the device.
 *
 * Creates a server on the current device for one vehicle model and one set
 * of cost weights and options (params' K, N, dt, lambda, sigma, seed are
 * unused: they are per vehicle).  MPPI_ENOMEM if the slots' workspaces do
 * not fit the budget. */
int mppi_server_create(const mppi_model* model, const mppi_params* params, const mppi_server_cfg* cfg,
                       mppi_server** out);

/* Registers a vehicle: sizes, temperature and noise, its obstacle set
 * (host M*4, copied to the device), initial nominal (host N*4; NULL:
 * hover) and Philox seed/stream.  MPPI_ENOMEM when its device state does
 * not fit the remaining budget, MPPI_EINVAL for sizes beyond the config. */
int mppi_server_add_vehicle(mppi_server* s, int32_t K, int32_t N, float dt, float lambda, const float* sigma,
                            const float* obstacles, int32_t M, const float* u_init, uint64_t seed,
                            uint32_t stream_id, int32_t* vehicle_id);

/* Releases a vehicle and its device state once its requests are done:
 * blocks until the requests already queued or in flight for it complete
 * (their results stay available to mppi_server_poll).  From the call on,
 * submissions, exports, imports and removals for the vehicle return
 * MPPI_ENOTFOUND. */
int mppi_server_remove_vehicle(mppi_server* s, int32_t vehicle_id);

/* Queues one solve request: state estimate x_hat[13] and reference window
 * ref[(N+1)*13] (host, copied before return).  MPPI_EAGAIN when the queue
 * is full, MPPI_ENOTFOUND for an unknown vehicle. */
int mppi_server_submit(mppi_server* s, int32_t vehicle_id, const float* x_hat, const float* ref,
                       uint64_t* request_id);

/* Moves up to `max` completed results into out[] (caller-owned, room for
 * `max`) and sets *n; MPPI_EINVAL for a NULL n or a NULL out with max > 0. */
int mppi_server_poll(mppi_server* s, mppi_result* out, int32_t max, int32_t* n);

/* Waits until no request is queued or in flight (timeout_ms < 0: no
 * limit); MPPI_ETIMEOUT if that did not happen in time. */
int mppi_server_drain(mppi_server* s, int32_t timeout_ms);

/* Copies a vehicle's device state (nominal N*4, Philox counter) to the
 * host, or replaces it from the host (migration, checkpoint and resume).
 * Both wait until the vehicle has nothing in flight. */
int mppi_server_export_vehicle(mppi_server* s, int32_t vehicle_id, float* u_nom, uint64_t* iter);
int mppi_server_import_vehicle(mppi_server* s, int32_t vehicle_id, const float* u_nom, uint64_t iter);

/* Copies the server's counters (submitted, completed, rejected, batches,
 * device bytes in use and budgeted, busy time) into *st. */
int mppi_server_get_stats(mppi_server* s, mppi_server_stats* st);

/* Stops the dispatcher after draining and frees everything. */
int mppi_server_destroy(mppi_server* s);

/* One MPPI step that allocates no memory (the paper has no counterpart:
 * this is an interface for callers that cannot call cudaMalloc, such as a
 * real-time control loop that forbids allocation after start-up, or a
 * plug-in whose host framework owns all device memory).  Same arguments
 * and results as mppi_solve_async, with the model and parameters passed
 * directly instead of a handle; all buffers are DEVICE buffers supplied by
 * the caller.  The scratch it needs lives in a fixed array compiled into
 * the library (about 1 MiB, held by every GPU that loads the library until
 * the process exits), so sizes are limited to K <= 32768 and N <= 256
 * (MPPI_EINVAL beyond).  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  The
 * address is kept for the life of the process: do not call this entry
 * point again after cudaDeviceReset (or any other teardown of the device's
 * primary context), which would leave it stale.  All calls share the
 * array: calls whose work overlaps on the GPU race, so order them on one
 * stream.  Pointers must be aligned as for mppi_solve_async (MPPI_EINVAL
 * otherwise).  Launch shape: 128 threads, one per sample. */
int mppi_solve_noalloc(const mppi_model* model, const mppi_params* params, const float* x_hat,
                       const float* ref, const float* obstacles, int32_t M, const float* u_nom, uint64_t iter,
                       float* u_out, float* u_cmd, float* u_next, float* x_next, float* costs, int32_t* status,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPPI_GB300_H */
