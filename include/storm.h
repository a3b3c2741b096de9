/*
 * storm.h -- C ABI of the B300 (sm_103a) STORM control-step library.
 *
 * The library runs the data-parallel hot path of joint-space sampling-based MPC
 * (Bhardwaj et al., arXiv 2104.13542, Algorithm 1): shift, then K iterations of
 * sample_controls -> generate_rollouts -> update_distribution, then
 * next_command.  All of it runs in hand-written CUDA kernels on one GPU.
 *
 * Conventions
 *  - Every entry point returns an int status: 0 = STORM_OK, < 0 = error,
 *    > 0 = warning.  No C++ exception crosses this boundary.  After an error
 *    storm_last_error() describes it.
 *  - The handle owns all device memory it allocates.  Pointers passed to
 *    storm_create are deep-copied; the caller may free them after the call.
 *  - Model parameters (robot, world, params) are double precision at the
 *    boundary and rounded once to float on the device.  Per-step data (state,
 *    goal, command, distribution) are float.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the device that was current at storm_create.  Device
 *    work is enqueued on the handle's stream (the one given to storm_create,
 *    or a private non-blocking stream when NULL was given).
 *  - A handle may be used by one host thread at a time.
 *
 * Array layouts are row-major (C order):
 *    state    3 x dof  (theta, theta_dot, theta_ddot)               Sec. 3 / Eq. 7
 *    goal     7        (x, y, z, qw, qx, qy, qz) goal pose X_g      Eq. 9
 *    mean     H x dof  mean control sequence mu (joint accel.)      Sec. 4, Eq. 4
 *    sigma    dof      per-joint standard deviation                 Sec. 4.3, Eq. 5
 *    u        N x H x dof sampled controls                          Algorithm 1
 *    ee       N x H x 12  end-effector pose as row-major 3x4 [R | p] Eq. 8
 *    terms    N x H x 8   unweighted cost terms, order:
 *                         pos, rot, stop, joint, manip, self, world, smooth
 *    cost     N x H       weighted running cost c_hat             Eq. 15
 *    Ctot     N           discounted total C_hat                  Eq. 2
 */
#ifndef STORM_H
#define STORM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STORM_MAX_DOF 7
#define STORM_MAX_H 64
#define STORM_MAX_SPHERES 64
#define STORM_MAX_PAIRS 2048
#define STORM_MAX_OBSTACLES 64 /* per kind: boxes, spheres */
#define STORM_MAX_N 16384
/* Cost terms reported per (particle, step): pos, rot, stop, joint, manip, self,
 * world, smooth, ee speed, ee acceleration, ball. */
#define STORM_NTERMS 11

typedef struct storm_handle storm_handle;

enum storm_status {
    STORM_OK = 0,
    STORM_WARN_DEGENERATE = 1, /* an iteration had no finite total cost; mu, sigma kept */
    STORM_ERR_INVALID_ARG = -1,
    STORM_ERR_CUDA = -2,
    STORM_ERR_OOM = -3,
    STORM_ERR_NONFINITE = -4, /* a non-finite value in the state or goal input */
    STORM_ERR_TIMEOUT = -5,
    STORM_ERR_STATE = -6 /* a checkpoint blob that does not match this handle */
};

enum storm_sampler { STORM_SAMPLER_PHILOX = 0, STORM_SAMPLER_HALTON = 1 };
enum storm_rot_mode { STORM_ROT_QUAT = 0, STORM_ROT_FROBENIUS = 1 };
enum storm_filter { STORM_FILTER_DEFAULT = 0, STORM_FILTER_COMB = 1, STORM_FILTER_MIXED = 2 };

/* Serial revolute chain in modified Denavit-Hartenberg form (Craig), with link
 * spheres for collision (Sec. 3.1 kinematic model, Eq. 8; Eqs. 13-14 with the
 * learned checks replaced by exact sphere geometry). */
typedef struct {
    int dof;                  /* d, 1..STORM_MAX_DOF */
    const double* dh;         /* d x 4: a_{i-1}, alpha_{i-1}, d_i, theta_offset_i */
    const double* q_min;      /* d joint limits (Eq. 11) */
    const double* q_max;      /* d */
    int n_spheres;            /* M, 0..STORM_MAX_SPHERES */
    const int* sphere_link;   /* M: frame 0..d the sphere is fixed to (0 = base) */
    const double* spheres;    /* M x 4: centre in that frame, radius */
    int n_pairs;              /* P, 0..STORM_MAX_PAIRS */
    const int* pairs;         /* P x 2 sphere indices checked for self-collision */
} storm_robot;

/* Obstacles: axis-aligned boxes and spheres in the world frame. */
typedef struct {
    int n_boxes;              /* 0..STORM_MAX_OBSTACLES */
    const double* boxes;      /* B x 6: cx, cy, cz, hx, hy, hz (half extents) */
    int n_spheres;            /* 0..STORM_MAX_OBSTACLES */
    const double* spheres;    /* S x 4: cx, cy, cz, r */
} storm_world;

typedef struct {
    int N;                    /* particles, 1..STORM_MAX_N */
    int H;                    /* horizon, 1..STORM_MAX_H */
    int K;                    /* optimisation iterations per step, 1..255 */
    int n_knots;              /* 0: no smoothing; else 4..H cubic B-spline knots (Sec. 4.3) */
    int sampler;              /* storm_sampler (Sec. 4.3) */
    int n_null;               /* particles 0..n_null-1 are zero-acceleration ("null") */
    const double* dt;         /* H time steps (Eq. 7) */
    double beta;              /* temperature (Eq. 6); 0 selects the argmin particle */
    double gamma;             /* discount (Eq. 2) */
    double alpha_mu;          /* mean step size (Eq. 4) */
    double alpha_sigma;       /* covariance step size (Eq. 5) */
    double sigma_init;        /* initial per-joint sigma */
    double sigma_min;         /* floor on sigma after each update */
    double w_pos, w_rot, w_stop, w_joint, w_manip, w_coll, w_smooth; /* Eq. 15 weights */
    double pos_axis_w[3];     /* alpha_2 of Eq. 9: goal-frame position axis weights */
    double rot_axis_w[3];     /* alpha_1 of Eq. 9 (STORM_ROT_FROBENIUS only) */
    int rot_mode;             /* storm_rot_mode */
    double k_jl;              /* joint-limit safety ratio (Eq. 11) */
    double k_m;               /* manipulability threshold (Eq. 12) */
    double qdd_max;           /* max acceleration of the stop cost (Eq. 10) */
    uint64_t seed;            /* Philox key */
    uint32_t instance;        /* Philox stream id (< 2^24) */
    int grad_steps;           /* gradient refinement steps after the K iterations (0..64);
                                 requires the default filter and w_ee_vel = w_ee_acc = w_ball = 0 */
    double grad_eta;          /* their step size: mu <- mu - grad_eta * dJ/dmu */
    /* Noise smoothing along the horizon (Sec. 4.3), storm_filter:
     *   STORM_FILTER_DEFAULT  cubic B-spline through n_knots samples when n_knots > 0, else
     *                         one raw sample per step;
     *   STORM_FILTER_COMB     one sample per step through the comb filter
     *                         y_h = comb[0] e_h + comb[1] y_{h-1} + comb[2] y_{h-2} (y_{<0} = 0);
     *   STORM_FILTER_MIXED    one sample per step; the first round(mix_bspline (N - n_null))
     *                         non-null particles take the B-spline through their first
     *                         n_knots samples (n_knots >= 4 required), the rest the comb. */
    int filter;
    double comb[3];
    double mix_bspline;       /* in [0, 1] */
    /* Task-space limits on Eq. 8's end-effector linear speed |X_dot| and acceleration
     * |X_ddot| (theta_ddot = u): terms max(0, |.| - max), weights >= 0.  Added terms. */
    double w_ee_vel, w_ee_acc, ee_vel_max, ee_acc_max;
    /* Ball on a tray held by the end effector (appendix, ball balancing): the ball's
     * in-plane distance from tray_center (end-effector frame) along the horizon, the
     * ball rolling under the in-plane part of gravity (world frame).  The ball state
     * is an input of each step (storm_set_ball); batches take w_ball = 0. */
    double w_ball;
    double gravity[3];
    double tray_center[3];
    /* STORM_SAMPLER_HALTON only: 1 scrambles the digits linearly, dimension k (base p_k)
     * mapping digit a to (f_k a) mod p_k with f_k = 1 + (Philox4x32-10 of counter
     * (k, 0, 0, 3) under the seed's key, first word) mod (p_k - 1) (generalised Halton;
     * plain Halton points in many prime dimensions are strongly correlated); 0 plain. */
    int halton_scramble;
} storm_params;

typedef struct {
    float best_cost;          /* min C_hat of the last iteration */
    float mean_weighted_cost; /* sum_n w_n C_hat_n of the last iteration */
    int status;               /* storm_status of the step */
    uint32_t step;            /* index of the step just taken */
} storm_step_info;

/* ---------------------------------------------------------------- lifetime */

/* Validate and upload robot / world / params, build the device tables
 * (B-spline basis, discounts, stop-velocity limits, Halton noise) and set
 * mu = 0, sigma = sigma_init, step = 0.  `cuda_stream` is a cudaStream_t or
 * NULL.  On error *out is NULL.  Errors: INVALID_ARG (sizes out of range,
 * NULL required pointer, bad sphere link / pair index), CUDA, OOM. */
int storm_create(const storm_robot* robot, const storm_world* world,
                 const storm_params* params, void* cuda_stream, storm_handle** out);

/* Release every resource of the handle (NULL is a no-op).  The controller of
 * Algorithm 1 has no explicit teardown; this ends the lifetime storm_create
 * began. */
void storm_destroy(storm_handle* h);

/* Static text of a storm_status value (never NULL).  The paper has no
 * counterpart: status codes are this library's error reporting. */
const char* storm_status_string(int status);
/* Message of the last error on this handle (never NULL). */
const char* storm_last_error(const storm_handle* h);

/* mu = 0, sigma = sigma_init, step counter = 0. */
int storm_reset(storm_handle* h);

/* ---------------------------------------------------------------- control step */

/* One control step of Algorithm 1 from host buffers: state (3 x dof, host),
 * goal (7, host) -> cmd (dof, host) = first action of the optimised mean
 * (next_command).  The inputs go in through pinned staging; the step's last
 * kernel writes the command and the step record into pinned memory itself
 * (its step counter last), and the call returns as soon as they are there —
 * the handle's stream may still be retiring that kernel, which every later
 * call on the handle is ordered after (with gradient refinement the outputs
 * are copied out and the call waits for the stream).  `info` may be NULL.
 * Errors: INVALID_ARG, NONFINITE (state or goal), CUDA; returns
 * WARN_DEGENERATE when an iteration had no finite total cost. */
int storm_step(storm_handle* h, const float* state, const float* goal, float* cmd,
               storm_step_info* info);

/* The same step on device buffers, enqueued on the handle's stream without
 * waiting: state_dev (3 x dof), goal_dev (7), cmd_dev (dof).  Passing the
 * pointers from storm_device_io() avoids two device-to-device copies.  Call
 * storm_sync() to wait and read the step's status. */
int storm_step_async(storm_handle* h, const float* state_dev, const float* goal_dev,
                     float* cmd_dev);

/* Wait for the handle's stream; `info` (nullable) receives the last step's info. */
int storm_sync(storm_handle* h, storm_step_info* info);

/* The handle's own device input/output buffers (state 3 x dof, goal 7, cmd dof). */
int storm_device_io(storm_handle* h, float** state_dev, float** goal_dev, float** cmd_dev);

/* ---------------------------------------------------------------- stages */

/* shift (Algorithm 1): mu_h <- mu_{h+1}, mu_{H-1} <- 0; sigma unchanged. */
int storm_shift(storm_handle* h);

/* The standard-normal noise of sample_controls (Sec. 4.3, Algorithm 1) for
 * iteration `iter` of control step `step`, before smoothing and scaling:
 * eps_dev (device, N x S x dof with S = n_knots, or H without smoothing).
 * Philox sampler: element e is lane e % 4 of Philox4x32-10 block e / 4 with
 * counter (e / 4, step, instance << 8 | iter, 0) and key (seed lo, seed hi),
 * lanes (0, 1) and (2, 3) Box-Muller pairs of 23-bit centred uniforms.
 * Halton sampler: the table drawn at storm_create.  Enqueued (no wait). */
int storm_sample_noise(storm_handle* h, uint32_t step, int iter, float* eps_dev);

/* The raw 32-bit words of that Philox noise stream, for checking the integer
 * stream bit for bit: block first_block + i (i < count) of the counter
 * (block, step, instance << 8 | iter, 0) under key (seed lo, seed hi) into
 * words_dev[4 i .. 4 i + 3] (device, 16-byte aligned, count x 4 uint32).
 * Philox4x32-10 is Salmon et al., SC'11; the paper samples with a
 * pseudo-random generator it does not name (Sec. 4.3).  Enqueued (no wait).
 * Errors: INVALID_ARG (NULL, bad iter, count outside 1..2^24, misaligned). */
int storm_philox_words(storm_handle* h, uint32_t step, int iter, uint32_t first_block, int count,
                       uint32_t* words_dev);

/* sample_controls + generate_rollouts (Algorithm 1; Eqs. 2, 7-15) for
 * iteration `iter` of control step `step` on the current distribution, from
 * device state_dev / goal_dev, with the handle's self-collision network when
 * one is set (storm_set_surrogate, storm_set_surrogate_cost).  The noise is the Philox stream of (step, iter)
 * or the Halton table.  Outputs are device buffers in the layouts above; any
 * of them may be NULL except that u_dev and Ctot_dev are always written when
 * given.  Enqueued on the handle's stream (no wait). */
int storm_generate_rollouts(storm_handle* h, const float* state_dev, const float* goal_dev,
                            uint32_t step, int iter, float* u_dev, float* theta_dev,
                            float* theta_dot_dev, float* ee_dev, float* terms_dev,
                            float* cost_dev, float* Ctot_dev);

/* update_distribution (Eqs. 4-6) of the handle's mu, sigma from device totals
 * Ctot_dev (N) and controls u_dev (N x H x dof).  weights_dev (N, nullable)
 * receives the normalised weights.  Enqueued (no wait); a degenerate update
 * is reported by the next storm_sync / storm_step. */
int storm_update_distribution(storm_handle* h, const float* Ctot_dev, const float* u_dev,
                              float* weights_dev);

/* Adjoint of the rollout cost (the paper has no counterpart; it samples
 * only): J(mu) = (1/N) sum_n C_hat_n(mu + sigma o eps~_n) (Eq. 2) with the
 * noise of (step, iter) and the handle's sigma fixed, and dJ/dmu (H x dof)
 * back through the running cost (Eqs. 9-15), the FK / Jacobian (Eq. 8) and
 * the integration scan (Eq. 7).  Null particles contribute to J but not to
 * the gradient.  Subgradients: 0 at a norm's or hinge's kink; the collision
 * minimum follows its minimising pair; the manipulability indicator is
 * differentiated only where m < k_m.  Device buffers: mean_dev (H x dof, in),
 * grad_dev (H x dof, out), J_dev (1, out), Ctot_dev (N, out, nullable).
 * Enqueued (no wait).  With params.grad_steps > 0 every control step ends
 * with that many refinement steps mu <- mu - grad_eta dJ/dmu, the noise of
 * step s being iteration K + s. */
int storm_cost_grad(storm_handle* h, const float* state_dev, const float* goal_dev,
                    const float* mean_dev, uint32_t step, int iter, float* grad_dev,
                    float* J_dev, float* Ctot_dev);

/* Host copies of mu (H x dof) and sigma (dof); either may be NULL.  Waits. */
int storm_get_distribution(storm_handle* h, float* mean, float* sigma);
int storm_set_distribution(storm_handle* h, const float* mean, const float* sigma);

/* Replace the obstacles of the world-collision term (Eq. 14), with counts
 * within the STORM_MAX_OBSTACLES limits.  The paper builds its scene once per
 * run and leaves moving scenes to future work (appendix, State Estimation and
 * Perception); this call lets the obstacles change between control steps.
 * Takes effect from the next step; waits for the copies.  Errors: INVALID_ARG
 * (NULL, counts out of range, non-finite values), CUDA. */
int storm_set_world(storm_handle* h, const storm_world* world);

/* Batched forward kinematics (Eq. 8) on device buffers: theta_dev (count x dof)
 * -> ee_dev (count x 12, row-major [R | p]).  Enqueued (no wait). */
int storm_forward_kinematics(storm_handle* h, const float* theta_dev, int count, float* ee_dev);

/* Batched end-effector velocity and acceleration (Eq. 8) on device buffers:
 * theta, theta_dot, theta_ddot (count x dof each) -> xd_dev, xdd_dev (count x 6,
 * [linear; angular] at the end-effector point, world frame).  Enqueued (no
 * wait). */
int storm_ee_twist(storm_handle* h, const float* theta_dev, const float* theta_dot_dev,
                   const float* theta_ddot_dev, int count, float* xd_dev, float* xdd_dev);

/* Ball state for the next steps (ball-on-tray cost): position and velocity in
 * the world frame (host, 6 floats), as measured at the current robot state.
 * Copied on the handle's stream, ordered with the steps.  Errors: INVALID_ARG
 * for NULL or non-finite values. */
int storm_set_ball(storm_handle* h, const float* ball_pos_vel);

/* ---------------------------------------------------------------- launch shape */

/* Rollout work mappings.  All compute bitwise the same results; they differ
 * only in how the (particle, step) items are spread over threads:
 *   STORM_MAP_CTA   a CTA takes a group of particles and runs each phase
 *                   (noise, controls, integration, FK and costs, world and
 *                   self collision, discounting) across all its threads,
 *                   with a CTA barrier between phases;
 *   STORM_MAP_WARP  a warp takes one particle (or 2 / 4 of them when H <= 16
 *                   / 8), one lane per step (two steps per lane when H > 32),
 *                   with warp-level synchronisation only;
 *   STORM_MAP_WARP_PAIR  the same with two warps per particle group: one for
 *                   the controls, the cost terms and world collision, one
 *                   for self collision, meeting once per step slot (the
 *                   default, one pair per CTA);
 *   STORM_MAP_WARP_QUAD  four warps per particle group: the controls and the
 *                   pose / joint / end-effector terms; world collision and
 *                   manipulability; two halves of self collision. */
#define STORM_MAP_CTA 0
#define STORM_MAP_WARP 1
#define STORM_MAP_WARP_PAIR 2
#define STORM_MAP_WARP_QUAD 3

/* CTA mapping and its shape: particles per CTA (1..N) and threads per CTA (a
 * multiple of 32 in 64..512).  Re-captures the step graph.  Errors:
 * INVALID_ARG when out of range or when the shape's shared-memory plan does not
 * fit a CTA. */
int storm_set_launch(storm_handle* h, int particles_per_cta, int threads_per_cta);
/* Warp mapping with 1..8 warps per CTA.  Re-captures the step graph.  Errors:
 * INVALID_ARG when out of range or when the plan does not fit a CTA. */
int storm_set_launch_warp(storm_handle* h, int warps_per_cta);
/* Warp-pair mapping with 1..4 pairs per CTA.  Errors as storm_set_launch_warp. */
int storm_set_launch_warp_pair(storm_handle* h, int pairs_per_cta);
/* Warp-quad mapping with 1..2 groups of four warps per CTA.  Errors as
 * storm_set_launch_warp. */
int storm_set_launch_warp_quad(storm_handle* h, int groups_per_cta);
/* Shape of the active mapping: particles and threads per CTA. */
int storm_get_launch(const storm_handle* h, int* particles_per_cta, int* threads_per_cta);
/* STORM_MAP_CTA, STORM_MAP_WARP, STORM_MAP_WARP_PAIR or STORM_MAP_WARP_QUAD;
 * INVALID_ARG for a NULL handle. */
int storm_get_launch_mapping(const storm_handle* h);

/* Dependent launch in the step graph (on = 1; off = 0, the default): every
 * rollout and distribution update is launched as a programmatic dependent of
 * the kernel before it, so its CTAs start while that kernel finishes and the
 * rollout draws its noise (a function of seed, step and iteration only) before
 * waiting for the previous update's mu and sigma.  Results are bitwise the same
 * either way; only the step graph uses it (the single-stage calls launch
 * ordinarily).  Off by default: on the 500 x 30 workload the early CTAs cost
 * more (the rollout's phases after the wait run slower) than the overlap
 * saves.  Re-captures the step graph; waits.  Errors: INVALID_ARG for a NULL
 * handle or on not 0 / 1.  storm_get_dependent_launch: 1, 0 or INVALID_ARG. */
int storm_set_dependent_launch(storm_handle* h, int on);
int storm_get_dependent_launch(const storm_handle* h);

/* Tracing: with trace_dev (device, 7 x uint64) set, thread 0 of rollout CTA 0
 * writes %globaltimer (ns) at the phase boundaries of every rollout launch:
 * [0] start, [1] tables + noise staged, [2] controls + integration, [3] FK,
 * Jacobian and non-collision costs, [4] world collision, [5] self collision,
 * [6] end (under the warp mapping, the timeline of warp 0; with two steps per
 * lane, [3]..[5] are those of the second).  NULL turns it off.  Re-captures
 * the step graph. */
int storm_set_trace(storm_handle* h, unsigned long long* trace_dev);

/* Collision broad phase (on by default): each link's spheres are enclosed in
 * one bounding sphere (fixed in the link frame, padded by 1e-4 m) and in one
 * capsule (a segment between two of its sphere centres and a radius, padded
 * by 1 mm), and the exact sphere-obstacle and sphere-pair tests run only where
 * two such bounds, or a bound and an obstacle, overlap (self collision under
 * the warp mappings: the bounding spheres, then the capsules, then each
 * first-link sphere against the second link's capsule).  The costs are
 * identical either way; off runs every exact test (brute force).  Re-captures
 * the step graph. */
int storm_set_broadphase(storm_handle* h, int on);

/* Autotuner: times this handle's rollout kernel (sample_controls +
 * generate_rollouts) with CUDA events on its stream for every candidate shape
 * -- CTA mapping with particles per CTA 1, 2, 3, 4, 6, 8, 12, 16 (at most N
 * and 512/H) x threads 128, 256, 512, warp mapping with 1, 2, 4, 8 warps per
 * CTA, pair mapping with 1, 2, 4 pairs per CTA, quad mapping with 1, 2 quads
 * per CTA -- on the state and goal of the handle's input buffers (call it
 * after a first step), keeps the fastest, except that the fastest pair shape
 * is kept when it is within 5 % of the fastest (one state is not every state:
 * the pair mapping shares collision-heavy items between its two warps); among
 * pair shapes one whose grid has fewer CTAs than the device has SMs must be
 * 5 % faster.  Then it re-captures the step graph.  best_us (nullable) receives the median time of
 * the chosen shape.  Waits. */
int storm_autotune(storm_handle* h, float* best_us);

/* ---------------------------------------------------------------- batched instances */

/* Many independent controllers of uneven sizes (particles, horizon, joints,
 * obstacles) stepped together, each one the control step of Algorithm 1
 * (shift, K x (sample_controls, generate_rollouts with Eqs. 2 and 7-15,
 * update_distribution with Eqs. 4-6), next_command): every kernel of a
 * control step is launched once for the whole batch, with the rollout work cut into tiles that
 * persistent CTAs deal out across the GPU.  The paper runs one controller;
 * batching is an added capability.  Instance i computes exactly what a
 * handle created from robots[i], worlds[i], params[i] computes (its Philox
 * stream is params[i].seed / params[i].instance). */
typedef struct storm_batch storm_batch;

#define STORM_MAX_BATCH 4096

/* count in 1..STORM_MAX_BATCH; arrays of `count` descriptions, validated as in
 * storm_create.  Errors: INVALID_ARG (with the failing instance in
 * storm_batch_last_error of a NULL batch being unavailable, the message goes
 * to stderr), CUDA, OOM. */
int storm_batch_create(int count, const storm_robot* robots, const storm_world* worlds,
                       const storm_params* params, void* cuda_stream, storm_batch** out);
void storm_batch_destroy(storm_batch* b);
const char* storm_batch_last_error(const storm_batch* b);

/* Sizes of the concatenated per-instance buffers: states (sum 3 dof_i floats),
 * goals (7 count floats), commands (sum dof_i floats). */
int storm_batch_sizes(const storm_batch* b, int* state_floats, int* cmd_floats);

/* One control step of every instance from host buffers: states = concatenation
 * of each instance's 3 x dof_i state, goals = count x 7, cmds (out) =
 * concatenation of the dof_i commands, statuses (out, nullable) = count
 * storm_status values.  Waits.  Errors: INVALID_ARG, NONFINITE, CUDA. */
int storm_batch_step(storm_batch* b, const float* states, const float* goals, float* cmds,
                     int* statuses);

/* The same step on the inputs already in the batch's device buffers (the last
 * storm_batch_step's, or written through storm_batch_device_io); enqueued, no
 * copies, no wait. */
int storm_batch_step_resident(storm_batch* b);
int storm_batch_device_io(storm_batch* b, float** states_dev, float** goals_dev, float** cmds_dev);
int storm_batch_sync(storm_batch* b);

/* Host copies of instance i's mu (H_i x dof_i) and sigma (dof_i); waits. */
int storm_batch_get_distribution(storm_batch* b, int i, float* mean, float* sigma);
int storm_batch_set_distribution(storm_batch* b, int i, const float* mean, const float* sigma);

/* Work mapping of the batched rollout, as for a single handle: the CTA-wide
 * mapping deals tiles of (particle, step) items to persistent CTAs; the warp
 * mapping (the default, 4 warps per CTA) deals (instance, particle group)
 * tasks to warps, each running the single-handle warp rollout on its
 * instance.  Both give every instance's results bitwise.
 *
 * storm_batch_set_launch: CTA mapping, items_per_tile >= 1 (rounded down to
 * whole particles, at least one), threads in 32..512, a multiple of 32.
 * storm_batch_set_launch_warp: warp mapping, warps_per_cta in 1..8.  Both
 * rebuild the task list and re-capture the step graph; wait.  Errors:
 * INVALID_ARG (also when the shape does not fit in shared memory), CUDA.
 *
 * Autotuner: every CTA shape of 32, 48, 64, 96, 128 items per tile x 128 /
 * 256 / 512 threads and every warp shape of 1, 2, 4, 8 warps per CTA, each
 * timed with CUDA events on the batch's inputs; keeps the fastest and
 * re-captures the step graph.  Waits.
 *
 * storm_batch_get_launch: items per tile and threads of the CTA mapping, or
 * 32 x warps per CTA for both on the warp mapping.
 * storm_batch_get_launch_mapping: STORM_MAP_CTA or STORM_MAP_WARP. */
int storm_batch_set_launch(storm_batch* b, int items_per_tile, int threads);
int storm_batch_set_launch_warp(storm_batch* b, int warps_per_cta);
int storm_batch_autotune(storm_batch* b, float* best_us);
int storm_batch_get_launch(const storm_batch* b, int* items_per_tile, int* threads);
int storm_batch_get_launch_mapping(const storm_batch* b);

/* ---------------------------------------------------------------- learned self-collision */

/* The paper replaces its exact self-collision check by a learned link-distance
 * network (Sec. 4.2, Eq. 13).  Here the network is an MLP: 16 encoded inputs
 * (x_j = theta_j / 3 for the joints, x_7 = 1, others 0) -> 256 -> 256 -> 256
 * -> 1 with ReLU, predicting the minimum signed distance (positive apart)
 * over the robot's self-collision pairs.  BF16 weights and activations, FP32
 * accumulation, every matrix product on tcgen05 tensor cores.  Parameters are
 * a flat FP32 vector (row-major, out x in): W1 256x16 | W2 256x256 | b2 256 |
 * W3 256x256 | b3 256 | w4 256 | b4 1. */
typedef struct storm_mlp storm_mlp;

#define STORM_MLP_PARAMS 135937
#define STORM_MLP_MAX_ROWS (1 << 22)

/* Architectures: STORM_MLP_DISTANCE is the network above; STORM_MLP_JOINTNERF
 * is the paper's jointNERF (Sec. 4.2): positional encoding x_j = sin theta_j,
 * x_{7+j} = cos theta_j, x_14 = 1, then 256 -> 128 -> 64 -> 1 with ReLU, the
 * same flat layout with those widths (45313 parameters). */
#define STORM_MLP_DISTANCE 0
#define STORM_MLP_JOINTNERF 1

/* He-uniform initial weights from the Philox stream of `seed`. */
int storm_mlp_create(uint64_t seed, void* cuda_stream, storm_mlp** out); /* STORM_MLP_DISTANCE */
int storm_mlp_create_arch(uint64_t seed, int arch, void* cuda_stream, storm_mlp** out);
/* Number of FP32 parameters of the network (INVALID_ARG for NULL). */
int storm_mlp_param_count(const storm_mlp* m);
void storm_mlp_destroy(storm_mlp* m);
const char* storm_mlp_last_error(const storm_mlp* m);
/* Host copies of the FP32 parameters (storm_mlp_param_count floats). */
int storm_mlp_get_params(storm_mlp* m, float* params);
int storm_mlp_set_params(storm_mlp* m, const float* params);
/* Predicted distances for theta_dev (count x dof, dof <= 7) into out_dev
 * (count); device buffers, waits.  count <= STORM_MLP_MAX_ROWS.  One kernel
 * runs the whole network per 128-row tile with the activations on chip
 * (weights streamed through shared memory by bulk asynchronous copies); the
 * result is bitwise that of storm_mlp_predict_layers. */
int storm_mlp_predict(storm_mlp* m, const float* theta_dev, int count, int dof, float* out_dev);
/* storm_mlp_predict enqueued on the network's stream without waiting (for
 * pipelined callers and timing); a tensor-core wait that ran out is reported by
 * the network's next waiting call.  Errors: INVALID_ARG, CUDA. */
int storm_mlp_predict_async(storm_mlp* m, const float* theta_dev, int count, int dof, float* out_dev);
/* The same predictions through the layer-by-layer tensor-core kernels of the
 * training forward pass (each layer's BF16 activations written to and read
 * back from global memory).  Same arguments, errors and waiting. */
int storm_mlp_predict_layers(storm_mlp* m, const float* theta_dev, int count, int dof, float* out_dev);
/* Mean squared error against target_dev (count) and its gradient (host,
 * storm_mlp_param_count floats, nullable); waits. */
int storm_mlp_loss_grad(storm_mlp* m, const float* theta_dev, const float* target_dev, int count,
                        int dof, float* loss, float* grad);
/* Adam training over `epochs` passes of shuffled minibatches of `batch`
 * (a multiple of 128) samples; epoch_loss (host, epochs, nullable) gets each
 * epoch's mean minibatch loss.  Waits.  STORM_ERR_TIMEOUT if a tensor-core
 * wait ran out (the network is then left as it was before the failing step). */
int storm_mlp_train(storm_mlp* m, const float* theta_dev, const float* target_dev, int count,
                    int dof, int batch, int epochs, float lr, uint64_t seed, float* epoch_loss);

/* Failure-path check of the tensor-core kernels' bounded waits (the paper has
 * no counterpart: this is the library's own failure detection).  Runs one
 * CTA that takes tensor memory and waits, with the routine every tensor-core
 * kernel uses, on an mbarrier that nothing ever completes, giving up after
 * limit_us microseconds (1..1,000,000) instead of the kernels' 1 s.  It then
 * flags the timeout, frees its tensor memory and ends, so the call returns
 * STORM_ERR_TIMEOUT with the network, its stream and the context still usable
 * (the flag is cleared on the way out).  Waits.  Errors: INVALID_ARG, CUDA. */
int storm_mlp_wait_probe(storm_mlp* m, unsigned int limit_us);

/* Exact self-collision label of the handle's robot: the minimum signed
 * distance over its self pairs for each configuration of theta_dev
 * (count x dof) into sd_dev (count).  Device buffers, enqueued. */
int storm_self_distance(storm_handle* h, const float* theta_dev, int count, float* sd_dev);

/* Use `mlp` (NULL: stop using it) in this handle's rollouts (the steps and
 * storm_generate_rollouts): the rollout kernel evaluates the network on every
 * (particle, step) configuration on the tensor cores, between the integration
 * and the costs, and runs the exact self-collision check only where the
 * prediction is below `margin` metres (elsewhere the self term is 0).  The
 * rollout then takes four particle groups per CTA of six warps (whatever
 * launch shape was set).  If a tensor-core wait of that kernel runs out, its
 * CTA falls back to the exact check for all its items and sets the network's
 * error flag (reported by the network's next call).  The network must live on
 * the handle's device, outlive its use and not be trained while this handle
 * steps; its weights are read at each step.  Allocates nothing.  Waits.
 * Errors: INVALID_ARG (NaN margin, another device, a problem whose fused
 * shared-memory plan exceeds a CTA), CUDA.  The adjoint (storm_cost_grad)
 * always differentiates the exact self-collision term. */
int storm_set_surrogate(storm_handle* h, storm_mlp* mlp, double margin);

/* The paper's own use of the network (Eq. 13): the self-collision term of each
 * (particle, step) is max(0, mlp(theta)) with the network predicting the
 * penetration depth (positive when colliding), and no exact self check runs.
 * NULL stops it.  Same kernel, rules and errors as storm_set_surrogate. */
int storm_set_surrogate_cost(storm_handle* h, storm_mlp* mlp);

/* ---------------------------------------------------------------- checkpoint */

/* Serialise the controller's state between steps -- the sampling
 * distribution (mean mu and per-joint sigma of Eqs. 4-5, Sec. 4.3) and the step
 * counter that indexes the noise (the Philox key is fixed by the params) -- so
 * that a resumed handle reproduces the same steps bit for bit.  The paper has no
 * checkpoint; the distribution is the state Algorithm 1 carries from one step
 * to the next.
 * With buf == NULL, *len receives the size needed.  Errors: INVALID_ARG when
 * *len is too small; STATE when a blob does not match the handle's shape. */
int storm_get_state(storm_handle* h, void* buf, size_t* len);
int storm_set_state(storm_handle* h, const void* buf, size_t len);

/* ---------------------------------------------------------------- measurement */

/* The FP32 fused multiply-add rate of the current device in TFLOP/s (the paper
 * has no counterpart: this is the peak the rollout kernel's ALU roofline is
 * quoted against).  Every thread of 8 x 256 threads per SM runs sixteen
 * independent FMA chains of `iters` steps on registers; tflops_scalar with one
 * FMA per instruction, tflops_paired with the paired FP32 FMA (two per
 * instruction); each the best of five timed launches after a warm-up, with CUDA
 * events on a private stream.  Allocates a few bytes; waits.  Errors:
 * INVALID_ARG (iters outside 1..2^24, NULL), CUDA. */
int storm_fp32_peak(int iters, float* tflops_scalar, float* tflops_paired);

/* ---------------------------------------------------------------- without allocation */

/* Size of the library's static device scratch used by the entry point below. */
#define STORM_NOALLOC_SCRATCH_BYTES (8u << 20)

/* generate_rollouts for callers that cannot allocate device memory.  The paper
 * has no counterpart: this exists for code embedded in a host that owns the
 * whole GPU memory budget -- a robot runtime or simulator that hands out fixed
 * buffers at start-up and forbids cudaMalloc afterwards, because an allocation
 * can synchronise the device and stall a hard-real-time control loop, or can
 * fail under a fixed memory cap.  Such a caller cannot create a handle
 * (storm_create allocates), so this call takes the model directly.
 *
 * It computes what storm_generate_rollouts computes for Ctot: the discounted
 * total cost (Eq. 2) of each of the N rollouts sampled from mean_dev / sigma_dev
 * for iteration `iter` of control step `step`.  It calls no cudaMalloc,
 * cudaFree or allocating library routine: the derived model tables and the
 * N x H x dof control batch live in one file-scope static device array of
 * STORM_NOALLOC_SCRATCH_BYTES (8 MiB), which every GPU that loads the library
 * holds until the process exits.
 *
 *   robot, world, params   host structs, as for storm_create (validated the same way)
 *   state_dev (3 x dof), goal_dev (7), mean_dev (H x dof), sigma_dev (dof)
 *                          device inputs, not modified
 *   Ctot_dev (N)           device output
 *   cuda_stream            cudaStream_t to enqueue on (NULL = legacy default stream)
 *
 * The first call on a device looks up the scratch array's device address with
 * cudaGetSymbolAddress (with that device current) and raises the rollout
 * kernel's shared-memory limit.  Every call builds the model tables on the host
 * exactly as storm_create does (spheres sorted by link, link-pair blocks, link
 * bounding spheres, collision broad phase on), copies them into the scratch and
 * rewrites every table the kernel reads, so no earlier contents are relied on;
 * the rollout runs the CTA mapping of storm_set_launch (bitwise the totals of
 * every other mapping).  Those copies come from pageable host memory, so each
 * call blocks the calling thread until its host tables have been staged for
 * the copy engine (not until the rollout ends), and a stream that is being
 * captured into a graph is refused (INVALID_ARG): the host memory the copies
 * read is freed when the call returns.
 * All calls share the one array: calls whose GPU work overlaps (other streams,
 * other host threads) race on it and must be serialised by the caller.
 * Errors: INVALID_ARG (as storm_create, NULL device pointer, bad iter, a
 * capturing stream, or a problem whose tables plus controls exceed the
 * scratch), CUDA.  The scratch holds, each rounded up to 256 bytes: about
 * 40 KB of model tables; with STORM_SAMPLER_HALTON the Halton noise,
 * 4*N*S*dof bytes (S = n_knots, or H without smoothing); and the controls,
 * 4*N*H*dof bytes -- e.g. N*H <= ~270,000 at dof 7 with the Philox sampler. */
int storm_rollout_costs_noalloc(const storm_robot* robot, const storm_world* world,
                                const storm_params* params, const float* state_dev,
                                const float* goal_dev, const float* mean_dev,
                                const float* sigma_dev, uint32_t step, int iter,
                                float* Ctot_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* STORM_H */
