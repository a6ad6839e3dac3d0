/*
 * crgb.h -- C ABI of the GB300 (sm_103a) library for batched collision-free
 * trajectory optimisation after "cuRobo: Parallelized Collision-Free
 * Minimum-Jerk Robot Motion Generation" (arXiv 2310.17274).
 *
 * The library evaluates, for every seed x timestep of a batch of joint-space
 * trajectories, forward kinematics of a serial revolute chain to collision
 * spheres, sphere-vs-oriented-box signed distance with the swept check and the
 * speed metric, self-collision, five-point-stencil smoothness, joint-limit and
 * goal-pose costs, and the backward pass to joint gradients (Sec. 2-3,
 * App. A); it runs the L-BFGS two-loop step and the parallel noisy line search
 * on the device (Sec. 4.1, Alg. 1).
 *
 * Conventions
 *  - Every function is `extern "C"`, returns a cr_status and never throws.
 *    On failure the thread-local message of cr_last_error() says why.
 *  - "host" pointers are read during the call only (descriptors are copied);
 *    "device" pointers are CUDA device memory owned by the caller, who keeps
 *    it alive until the stream has finished the call's work.
 *  - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) and is complete when that stream is; calls return before the GPU
 *    finishes unless stated.
 *  - Arrays are dense, row-major, float32 unless stated.
 *  - Sizes: 1 <= dof <= 16, 1 <= spheres <= 1024, pairs <= 65535,
 *    boxes <= 4096 per world, 1 <= horizon <= 128, history <= 16,
 *    1 <= n_alpha <= 16.  Anything else returns CR_EINVAL.
 */
#ifndef CRGB_H
#define CRGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cr_status;
#define CR_OK 0
#define CR_EINVAL 1    /* bad argument or size */
#define CR_ENOMEM 2    /* device or host allocation failed */
#define CR_ECUDA 3     /* a CUDA call failed (message has the CUDA error) */
#define CR_ETIMEOUT 4  /* cr_server_wait: the request did not finish within the time limit */
#define CR_EBUSY 5     /* cr_server_submit / cr_server_restore: the server's queue is full */
#define CR_ENAN 6      /* device status word (cr_result.status, cr_server_poll): a seed's cost is
                          not finite; NaN never wins the best seed */

#define CR_MAX_DOF 16
#define CR_MAX_ALPHA 16
#define CR_MAX_HISTORY 16
#define CR_N_TERMS 5   /* world, self, bound, smoothness, goal */

/* flags of cr_params.flags */
#define CR_SWEPT 1u          /* continuous (swept) collision check, Sec. 3.4 */
#define CR_SPEED 2u          /* speed metric on the world term, Sec. 3.3 / Eq. 11 */
#define CR_SELF 4u           /* self-collision term, Eq. 9 */
#define CR_WOLFE 8u          /* Wolfe condition in the line search, Alg. 1 */
#define CR_STRONG_WOLFE 16u  /* strong Wolfe instead of weak */
#define CR_IK_MODE 32u       /* single-state problems: no stencil terms, no sweep, no speed */
#define CR_VEL_COST 64u      /* velocity log-cosh term of Eq. 16 on every sample */
#define CR_CSPACE_GOAL 128u  /* joint-space goal cost of Eq. 15 (problems with goal_q) */
#define CR_NO_SELF_CHECK 256u /* IK mode without CR_SELF: the collision-free flag leaves out self-collision
                                 (IK without collision checking, Sec. 6); EINVAL in any other mode */

/* FP32 fused-multiply-add throughput of the current device (no counterpart
 * in the paper: the peak the evaluation kernel's roofline is reported
 * against).  Runs `iters` rounds of 128 independent FMAs per thread on a grid
 * of resident CTAs covering every SM, timed with CUDA events on `stream`;
 * writes TFLOP/s (an FMA counts as 2 FLOP) and the kernel time.  Synchronous;
 * allocates a few KB of device memory. */
cr_status cr_measure_ffma(int32_t iters, float* tflops, float* ms, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* cr_last_error(void);
/* Library version string. */
const char* cr_version(void);

/* ------------------------------------------------------------------------- */
/* Robot: serial revolute chain + sphere model (Sec. 3.1; App. E.1 "kinematics
 * data").  All pointers are host memory, copied to the device at creation.   */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t dof;
  const float* fixed_tf;      /* [dof+1][12] row-major 3x4 [R|p]: F_0..F_{dof-1}, then F_ee */
  const int32_t* axis;        /* [dof] revolute axis of each joint: 0 = x, 1 = y, 2 = z */
  const float* q_lo;          /* [dof] position limits (q_lo < q_hi) */
  const float* q_hi;          /* [dof] */
  const float* v_max;         /* [dof] symmetric velocity limit (> 0) */
  const float* a_max;         /* [dof] symmetric acceleration limit (> 0) */
  const float* j_max;         /* [dof] symmetric jerk limit (> 0) */
  int32_t n_spheres;
  const float* spheres;       /* [M][4] centre in its link frame, radius; radius < 0 disables it */
  const int32_t* sphere_link; /* [M] link (= joint) index 0..dof-1 the sphere rides on */
  int32_t n_pairs;
  const int32_t* pairs;       /* [P][2] self-collision pair set S of Eq. 9, i != j */
} cr_robot_desc;

typedef struct cr_robot cr_robot;
/* Copies the description to the device (synchronous).  *out is owned by the
 * caller and released with cr_robot_destroy. */
cr_status cr_robot_create(const cr_robot_desc* desc, cr_robot** out);
void cr_robot_destroy(cr_robot* robot);

/* ------------------------------------------------------------------------- */
/* World: oriented boxes (Sec. 3.5 "Oriented Bounding Box").                  */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t n;                  /* number of boxes, 0..4096 */
  const float* pose;          /* [n][7] host: centre xyz, quaternion wxyz (normalised on input) */
  const float* half_ext;      /* [n][3] host: half extents, each > 0 */
} cr_world_desc;

typedef struct cr_world cr_world;
/* Packs the boxes for the device (synchronous copy). */
cr_status cr_world_create(const cr_world_desc* desc, cr_world** out);
void cr_world_destroy(cr_world* world);

/* ------------------------------------------------------------------------- */
/* Parameters (App. A.1-A.3, App. B.3, Sec. 7.3).                              */
/* ------------------------------------------------------------------------- */
typedef struct {
  float w_goal_pos, w_goal_rot;  /* alpha_0, alpha_1 of Eq. 14 */
  float k_goal_pos, k_goal_rot;  /* alpha_2, alpha_3 of Eq. 14 */
  float w_coll;                  /* beta_2 of Eq. 11 */
  float w_self;                  /* beta_1 of Eq. 9 */
  float w_bound;                 /* weight of the Eq. 17 terms */
  float w_acc, w_jerk;           /* alpha_8, alpha_9 of Eq. 16 */
  float w_vel, k_vel;            /* alpha_6, alpha_7 of Eq. 16 (with CR_VEL_COST) */
  float eta;                     /* activation distance of Eq. 10 [m] */
  float eta_bound;               /* eta_2 of Eq. 17 */
  float dt;                      /* time step [s] */
  int32_t sweep_steps;           /* samples per side of the sweep, Sec. 3.4 */
  int32_t history;               /* L-BFGS memory m, 1..16 */
  int32_t n_alpha;               /* number of line-search step sizes, 1..16 */
  float alpha[CR_MAX_ALPHA];     /* step sizes; alpha[0] is the fallback "noisy" step */
  float armijo_c1, wolfe_c2;
  uint32_t flags;                /* CR_* flags above */
  float w_cspace, k_cspace;      /* alpha_4, alpha_5 of Eq. 15 (with CR_CSPACE_GOAL) */
} cr_params;

/* Defaults: the paper's weights and constants (App. A.1-A.3, App. B.3:
 * alpha_4 = 5000, alpha_5 = 50 for Eq. 15;
 * eta = 2.5 cm, weight 5000 for soft constraints; Sec. 7.3 step sizes
 * 0.01, 0.3, 0.7, 1.0), dt = 0.05, sweep_steps = 4, history = 6,
 * c1 = 1e-4, c2 = 0.9, flags = SWEPT|SPEED|SELF|WOLFE. */
void cr_params_default(cr_params* p);

/* One planning problem (Sec. 2): start configuration, goal pose, world. */
typedef struct {
  const cr_world* world;
  const float* q_start;       /* [dof] host */
  const float* goal;          /* [7] host: goal position xyz, quaternion wxyz */
  int32_t n_seeds;            /* B */
  int32_t horizon;            /* H free timesteps theta_1..theta_H */
  const float* seeds;         /* [B][H][dof] host initial trajectories (cr_solve only) */
  const float* goal_q;        /* [dof] host goal configuration for Eq. 15, or NULL */
} cr_problem;

/* ------------------------------------------------------------------------- */
/* Hot-path primitives                                                        */
/* ------------------------------------------------------------------------- */

/* Forward kinematics (Sec. 3.1; App. E.1 Table "Joint Transformation
 * matrices"): for N configurations theta (device [N][dof]) writes the sphere
 * centres and radii in the world (device [N][M][4], or NULL), the end-effector
 * pose as a 3x4 [R|p] (device [N][12], or NULL) and the link transforms
 * T_0..T_{dof-1} (device [N][dof][12], or NULL). */
cr_status cr_fk(const cr_robot* robot, const float* theta, int32_t n, float* spheres, float* ee,
                float* link_tf, void* stream);

/* Cost and gradient of B trajectories of one problem (Eq. 1 with every
 * constraint as a weighted soft cost: Eq. 9, 11, 14, 16, 17).
 *   theta  device [B][H][dof], H = problem->horizon (problem->seeds unused)
 *   cost   device [B] total cost
 *   grad   device [B][H][dof] d cost / d theta, or NULL
 *   cfree  device [B] uint8: 1 when every waypoint is clear of every box and
 *          every pair of S is separated (discrete check), or NULL
 *   terms  device [B][5] world, self, bound, smoothness, goal, or NULL
 *   state_terms  device [B][H][2] the world cost (Eq. 11 summed over the
 *          spheres) and the self cost (Eq. 9, weighted) of every state, or
 *          NULL; they add up to terms[0] and terms[1] (up to FP32 rounding
 *          order)
 * One fused kernel launch; link transforms stay on chip between the forward
 * and backward passes.  Deterministic: a trajectory's results do not depend
 * on B or on the other trajectories. */
cr_status cr_eval(const cr_robot* robot, const cr_problem* problem, const cr_params* params,
                  const float* theta, int32_t B, float* cost, float* grad, uint8_t* cfree,
                  float* terms, float* state_terms, void* stream);

/* Device-resident optimiser state of B seeds with n = H*dof variables each
 * (Sec. 4.1, App. A.7).  Every pointer is device memory owned by the caller.
 * The history (s, y, rho) is a ring of m slots: the pair appended by the
 * cr_opt_propose call that finds iter = k > 0 goes to slot (k-1) mod m, so
 * with iter = k the i-th of the m most recent pairs (i = 0 oldest, m-1
 * newest) is in slot (k-1+i) mod m.  Zeroed buffers with rho = 0 are inert.  cand* hold the n_alpha line-search candidates of each
 * seed, seed-major ([B][n_alpha][...]). */
typedef struct {
  int32_t n_seeds, horizon;
  float* x;             /* [B][n] current iterate */
  float* g;             /* [B][n] its gradient */
  float* c;             /* [B] its cost */
  float* x_prev;        /* [B][n] */
  float* g_prev;        /* [B][n] */
  float* s;             /* [B][m][n] */
  float* y;             /* [B][m][n] */
  float* rho;           /* [B][m] */
  int32_t* iter;        /* [B] iterations taken (0 = no previous iterate) */
  float* dir;           /* [B][n] last direction */
  float* cand;          /* [B][n_alpha][n] */
  float* cand_cost;     /* [B][n_alpha] */
  float* cand_grad;     /* [B][n_alpha][n] */
  uint8_t* cand_cfree;  /* [B][n_alpha] */
  float* best_x;        /* [B][n] best iterate so far */
  float* best_c;        /* [B] */
  uint8_t* best_cfree;  /* [B] */
  int32_t* ls_index;    /* [B] index chosen by the last line search */
} cr_opt_state;

/* L-BFGS step (App. A.7 "L-BFGS Step Update"): if iter > 0 append the pair
 * (x - x_prev, g - g_prev) with rho = 1/(y^T s) when y^T s > 1e-8 else 0,
 * dropping the oldest; store x_prev = x, g_prev = g; two-loop recursion with
 * H^0 = gamma I (gamma = s^T y / y^T y of the newest pair with rho > 0, else
 * 1) gives dir = -H g; then the candidates of Alg. 1,
 * cand[l] = clip(x + alpha_l dir, q_lo, q_hi).  One CTA per seed. */
cr_status cr_opt_propose(const cr_robot* robot, const cr_params* params, const cr_opt_state* st,
                         void* stream);

/* Line search selection of Alg. 1 over evaluated candidates: Armijo
 * c_l <= c + c1 alpha_l g^T dir (and, with CR_WOLFE, g_l^T dir >= c2 g^T dir,
 * or |g_l^T dir| <= c2 |g^T dir| with CR_STRONG_WOLFE); the largest passing
 * index, else 0, becomes (x, g, c); the best iterate is updated when c falls
 * below best_c (Sec. 4.1).  One CTA per seed. */
cr_status cr_opt_select(const cr_robot* robot, const cr_params* params, const cr_opt_state* st,
                        void* stream);

/* Particle-based optimisation (Sec. 4.2, Eq. 12-13, Alg. "Particle-Based
 * Optimization"): one iteration for n_seeds seeds of one problem, run before
 * L-BFGS to move seeds into a better basin.
 *   SAMPLE  particles = mu + sqrt(sigma) * eps (no clipping to the limits;
 *           the bound cost of Eq. 17 penalises what leaves them)
 *   COST    cr_eval of every particle (cost only)
 *   UPDATE  w_i = e^{c_i} / sum_j e^{c_j} with c = -cost / beta (computed
 *           after subtracting the smallest cost, which leaves w unchanged);
 *           mu <- (1 - k_mu) mu + k_mu sum_i w_i theta_i (Eq. 12);
 *           sigma <- (1 - k_sigma) sigma + k_sigma sum_i w_i (theta_i - mu)^2
 *           with the previous mu (Eq. 13 is garbled as printed; this reading
 *           makes sigma the weighted second moment of the particles)
 *   mu, sigma   device [n_seeds][H][dof] mean and diagonal covariance,
 *               updated in place (sigma >= 0)
 *   eps         device [n_seeds][n_particles][H][dof] zero-mean unit Gaussian
 *               samples drawn by the caller (the library draws no random numbers)
 *   particles   device [n_seeds][n_particles][H][dof] scratch; holds the
 *               samples on return
 *   cost        device [n_seeds][n_particles] scratch; their costs on return
 *   beta > 0, k_mu and k_sigma in [0, 1]: the paper gives no values.
 * Three launches on `stream`; deterministic (fixed summation orders). */
cr_status cr_particle_step(const cr_robot* robot, const cr_problem* problem, const cr_params* params,
                           int32_t n_seeds, int32_t n_particles, float* mu, float* sigma,
                           const float* eps, float* particles, float* cost, float beta, float k_mu,
                           float k_sigma, void* stream);

/* Parallel steering (Sec. 5, Alg. "Parallel Steering"), the edge check of
 * the paper's geometric planner on the same kinematics and distance code:
 * each edge e = [theta_0, theta_1] is discretised into n + 1 samples
 * l_i = theta_0 + (i / n)(theta_1 - theta_0), i = 0..n (the algorithm's
 * n = floor(max |theta_1 - theta_0| / r) + 1 is the caller's choice), every
 * sample is checked as cr_eval's collision-free flag checks a state (every
 * sphere clear of every box, every pair of S separated), and per edge:
 *   last   device [E] int32: the last valid sample before the first invalid
 *          one; n when all are valid, -1 when sample 0 is invalid
 *   v_new  device [E][dof]: that sample (theta_0 when last = -1)
 *   dist   device [E]: |v_new - theta_0| in joint space
 *   edges  device [E][2][dof]; samples device [E][n+1][dof], valid device
 *          [E][n+1] (uint8) and cost device [E][n+1] are scratch that hold
 *          the samples, their flags and their single-state costs on return.
 * Three launches on `stream`. */
cr_status cr_steer(const cr_robot* robot, const cr_world* world, int32_t n_edges, const float* edges,
                   int32_t n, float* samples, uint8_t* valid, float* cost, int32_t* last, float* v_new,
                   float* dist, void* stream);

/* Retiming of App. "Time-step Discretization" (Alg. "Time Discretization"):
 * for B trajectories theta (device [B][H][dof], H = problem->horizon, start
 * problem->q_start) writes dt (device [B]), the time step that puts each at
 * the robot's velocity, acceleration or jerk limit: the App. A.5 stencils at
 * dt = 1 give v1, a1, j1 and dt = max over samples and joints of
 * |v1|/v_max, sqrt(|a1|/a_max), cbrt(|j1|/j_max).  One launch on `stream`. */
cr_status cr_retime(const cr_robot* robot, const cr_problem* problem, int32_t B, const float* theta,
                    float* dt, void* stream);

/* Choosing among the seeds of a solve (App. "Solver details": IK returns the
 * valid solution with the lowest weighted sum of pose error and distance to
 * the current configuration; trajectory optimisation the valid seed with the
 * lowest blend of pose error, largest jerk and motion time).  With e_pose =
 * |p - p_g| + d_q at the last state (d_q = (3 - tr(R_g^T R)) / 4 of Eq. 14):
 *   params->flags & CR_IK_MODE:  score = w_pose e_pose + w_dist |theta_H - q_start|
 *   otherwise:                   score = w_pose e_pose + w_jerk max|jerk| + w_time H dt_b
 * the jerk being App. A.5's five-point stencil at dt_b (dt[b], or params->dt
 * when dt is NULL) over every sample and joint, H dt_b the motion time of the
 * H + 1 waypoints.  The paper gives no weights; they are the caller's.
 *   theta  device [B][H][dof] (H = problem->horizon), cfree device [B] (uint8)
 *   dt     device [B] per-seed time steps, or NULL
 *   score  device [B] out; best device [1] out: the lowest score among seeds
 *          with cfree != 0 (the lowest index on ties; NaN never wins), or -1.
 * Two launches on `stream`. */
cr_status cr_rank_seeds(const cr_robot* robot, const cr_problem* problem, const cr_params* params,
                        int32_t B, const float* theta, const uint8_t* cfree, const float* dt, float w_pose,
                        float w_jerk, float w_time, float w_dist, float* score, int32_t* best, void* stream);

/* ------------------------------------------------------------------------- */
/* Runtime: context, batched solve                                            */
/* ------------------------------------------------------------------------- */
typedef struct cr_ctx cr_ctx;

/* A context on CUDA device `device` owns the solver workspace (grown on
 * demand, capped by mem_budget bytes; 0 = no cap), the captured CUDA graphs
 * and the autotune table.  Not thread-safe: one host thread per context. */
cr_status cr_context_create(int device, size_t mem_budget, cr_ctx** out);
void cr_context_destroy(cr_ctx* ctx);

/* Output of one problem: device buffers owned by the caller (any may be NULL). */
typedef struct {
  float* traj;     /* [B][H][dof] best iterate of every seed */
  float* cost;     /* [B] its cost */
  uint8_t* cfree;  /* [B] its collision-free flag */
  int32_t* best;   /* [1] index of the lowest-cost collision-free seed, else of the lowest-cost seed */
  int32_t* status; /* [1] device status word, written on the stream with the results: CR_OK, or
                      CR_ENAN when a seed's best cost is not finite (a seed with a NaN or infinite
                      value, or an overflow); the other seeds' results stay valid */
} cr_result;

#define CR_SOLVE_GRAPH 1u       /* capture the whole solve as one CUDA graph, replayed on later calls */
#define CR_SOLVE_PERSISTENT 2u  /* evaluation launches sized to the GPU, tiles taken from a device counter */
#define CR_SOLVE_DEVICE_SEEDS 4u /* problems[p].seeds point to device memory instead of host memory */

/* Solve n_problems problems (each with its own world, start, goal, seed
 * count and horizon) together (Sec. 4.1): evaluate the seeds, then `iters`
 * iterations of L-BFGS step -> parallel noisy line search over all
 * candidates of all problems in one evaluation launch -> selection and
 * best-iterate update, then the per-problem result.  Seeds are host memory
 * (problems[p].seeds, [B][H][dof]; device memory with CR_SOLVE_DEVICE_SEEDS)
 * and are copied on `stream`; results are written on `stream`.  A problem's
 * results are identical whether it is solved alone or with others.  The call
 * waits until the previous call's small table upload has left its pinned
 * staging buffer before reusing it. */
cr_status cr_solve(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                   const cr_params* params, int32_t iters, uint32_t solve_flags,
                   const cr_result* results, void* stream);

/* cr_solve with particle-based optimisation of every seed first (Sec. 4.2,
 * Eq. 12-13; App. B.3 runs 2 iterations before L-BFGS for IK and trajectory
 * optimisation): each seed is the mean of its particles, sigma0 their
 * initial variance; an iteration samples particles = mean + sqrt(variance) x
 * eps, evaluates their cost (one launch over every particle of every
 * problem) and updates mean and variance exactly as cr_particle_step does
 * (bit for bit); the means then start the L-BFGS iterations.  eps (device)
 * holds iters x n_particles x V zero-mean unit Gaussian samples (V = sum over
 * problems of B_p H_p dof): for iteration k, problem after problem, the
 * block [B_p][n_particles][H_p][dof] of cr_particle_step's layout.  The
 * library draws no random numbers. */
typedef struct {
  int32_t iters;        /* particle iterations before L-BFGS */
  int32_t n_particles;  /* particles per seed, 1..4096 */
  float beta, k_mu, k_sigma;  /* as cr_particle_step */
  float sigma0;         /* initial variance of every variable (>= 0) */
  const float* eps;     /* device samples, see above */
} cr_particle_config;

cr_status cr_solve_particles(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                             const cr_params* params, int32_t iters, uint32_t solve_flags,
                             const cr_particle_config* particles, const cr_result* results, void* stream);

/* Alg. "Time Discretization" (App. "Time-step Discretization"): the
 * trajectory is first optimised at a coarse step without the jerk term, then
 * re-timed to the robot's limits and optimised again at that step.  Per
 * problem, entirely on the device (no host round trip between the stages):
 *   1. iters1 iterations (as cr_solve) at dt_init, the derivative weights
 *      scaled to dt_init and the jerk weight 0;
 *   2. the best seed of 1 (lowest-cost collision-free, else lowest-cost) is
 *      retimed (cr_retime): dt_opt = max(its step, dt_min); the weight on the
 *      square of the k-th derivative becomes w_k (dt_opt / dt)^(2k) with the
 *      params' own dt and weights (the reading of "scale the weights by the
 *      new dt": it keeps each term's value for the same waypoints), jerk on;
 *   3. iters2 iterations at dt_opt from the best iterates of every seed of 1;
 *   4. every seed of 3 is retimed and scored as cr_rank_seeds does with the
 *      weights below; the chosen seed is the lowest score among the
 *      collision-free seeds, else the solve's best.
 * `results` receive the second solve's output as cr_solve writes it; tres
 * (device buffers per problem, any may be NULL) the stages' outputs.
 * Trajectory problems only (CR_IK_MODE is refused).  solve_flags as cr_solve
 * (with CR_SOLVE_GRAPH the whole algorithm is one CUDA graph). */
typedef struct {
  float dt_init;     /* time step of the first solve [s] (the paper's coarse step: 0.25) */
  float dt_min;      /* floor of the retimed step [s] */
  int32_t iters1, iters2;
  float w_pose, w_jerk, w_time;  /* seed-choice weights of cr_rank_seeds */
} cr_timeopt_config;

typedef struct {
  float* first;    /* [H][dof] best trajectory of the first solve */
  float* stage;    /* [8] dt, w_vel, w_acc, w_jerk used by the first solve, then by the second */
  float* dt;       /* [B] each seed's retimed step after the second solve */
  float* score;    /* [B] its seed-choice score */
  int32_t* chosen; /* [1] the chosen seed */
} cr_timeopt_result;

cr_status cr_solve_timeopt(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                           const cr_params* params, const cr_timeopt_config* cfg, uint32_t solve_flags,
                           const cr_result* results, const cr_timeopt_result* tres, void* stream);

/* Autotuner: time cr_solve of this batch (`iters` iterations) for each tile
 * shape -- CTA size 256 or 512 threads; when a horizon is below 32, 8, 16,
 * 32 or 64 states per tile; sphere positions cached in shared memory or
 * recomputed (a smaller tile, so more CTAs share an SM) -- and keep the
 * fastest in the context for every problem shape of the batch (spheres, box
 * count rounded up to a power of two, horizon); later cr_solve calls on those
 * shapes use it.  Results do not depend on the tile shape.  Synchronous.
 * Writes the choice and its time (any output may be NULL). */
cr_status cr_autotune(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                      const cr_params* params, int32_t iters, int32_t* block, int32_t* short_tile,
                      int32_t* no_cache, float* ms);
/* Set the tile shape of one problem shape by hand: block 256 or 512;
 * no_cache = 1 recomputes sphere positions instead of caching them in shared
 * memory and bounds registers so two 512-thread CTAs share an SM, 0 caches
 * them (one CTA per SM), -1 takes 1 when two such CTAs fit, else 0 (the
 * default for shapes never tuned, and for cr_eval). */
cr_status cr_tune_set(cr_ctx* ctx, int32_t n_spheres, int32_t n_boxes, int32_t horizon, int32_t block,
                      int32_t short_tile, int32_t no_cache);

/* ------------------------------------------------------------------------- */
/* Serving: continuous batching of motion-generation and IK requests          */
/* ------------------------------------------------------------------------- */
typedef struct cr_server cr_server;

/* Request kinds: 0 = trajectory optimisation (motion generation), 1 = IK.
 * A request brings its own seed count and horizon (IK: horizon 1); the kind
 * fixes its parameters and iteration count.  Requests of one kind and one
 * shape share a pool of device slots with its own stream. */
typedef struct {
  int32_t kind_iters[2];      /* L-BFGS iterations per request of each kind, multiples of chunk */
  cr_params kind_params[2];   /* parameters per kind (kind 1 needs CR_IK_MODE) */
  int32_t chunk;              /* iterations a pool runs per round for each of its active requests */
  int32_t max_active;         /* cap on active requests per pool (0 = memory decides) */
  size_t reserve_bytes;       /* free device memory never given to request state */
  int32_t max_queued;         /* submit / restore return CR_EBUSY while this many requests wait for a
                                 slot (0 = no limit) */
} cr_server_config;

/* A server keeps the optimiser state of every active request on the device
 * (Sec. 4.1 state: iterate, gradient, history, candidates, best iterate).
 * Not thread-safe: one host thread per server. */
cr_status cr_server_create(cr_ctx* ctx, const cr_robot* robot, const cr_server_config* cfg,
                           cr_server** out);
/* Waits for the server's running rounds, then frees it. */
void cr_server_destroy(cr_server* server);
/* Queue a request (host inputs copied; problem->seeds [B][H][dof] host,
 * problem->goal_q optional).  It is admitted by a later step once a slot and
 * free device memory allow.  CR_EBUSY (nothing queued) when max_queued
 * requests already wait. */
cr_status cr_server_submit(cr_server* server, int32_t kind, const cr_problem* problem,
                           uint64_t* ticket);
/* One step.  It does not wait for the device, except while a pool grows or
 * a table buffer is enlarged: the live slots are copied into the new arrays
 * and the old ones freed, and freeing device memory can wait for the device
 * (a pool at its working size never does this).  For every pool: if its last round
 * has finished, the requests that retired in it become done (results already
 * in pinned host memory) and their slots free; queued requests are admitted
 * into free slots of idle pools (first come, first served per pool), a pool
 * growing while free device memory minus the reserve allows; every idle pool
 * with active requests starts a round: the initial evaluation and first
 * L-BFGS step of its new requests, `chunk` iterations for all (one
 * evaluation launch over all their line-search candidates, one selection +
 * L-BFGS launch), the results of those reaching their iteration count copied
 * to the host.  A request that arrives while its pool runs is admitted when
 * that round ends; other pools are not held up.  Work follows `stream`.
 * Each request's result equals cr_solve of that request alone with its
 * kind's parameters and iterations, bit for bit. */
cr_status cr_server_step(cr_server* server, void* stream);
/* Results of a finished request into host buffers (any may be NULL):
 * traj [B][H][dof], cost [B], cfree [B], best seed index, device status word
 * (CR_OK or CR_ENAN).  *done = 0 while pending. */
cr_status cr_server_poll(cr_server* server, uint64_t ticket, int32_t* done, float* traj,
                         float* cost, uint8_t* cfree, int32_t* best, int32_t* status);
/* Step until the request is done; CR_ETIMEOUT after timeout_ms milliseconds
 * (negative: no limit).  Blocks the host. */
cr_status cr_server_wait(cr_server* server, uint64_t ticket, int32_t timeout_ms);
/* Copy a pending request out of the server: its inputs and, once admitted,
 * its whole device optimiser state (iterate, gradient, previous iterate and
 * gradient, history ring, direction, line-search candidates, best iterate,
 * iteration count) after its last round (waits for a running round; a
 * request that finishes in it is no longer pending: CR_EINVAL).  With
 * buf = NULL writes the size needed to *bytes; else *bytes is the buffer's
 * size (CR_EINVAL, and the size needed, when too small).  The request keeps
 * running in this server.  Host memory, opaque, valid for cr_server_restore
 * on a server of the same robot and the same parameters for its kind. */
cr_status cr_server_snapshot(cr_server* server, uint64_t ticket, void* buf, size_t* bytes);
/* Queue a request from a snapshot (world: the handle of its world in this
 * process).  Admitted like a new request, it continues from the saved state:
 * its result is bit-identical to the original request's.  CR_EINVAL when the
 * snapshot is malformed, of another robot, or of other parameters or
 * iteration counts; CR_EBUSY as cr_server_submit. */
cr_status cr_server_restore(cr_server* server, const void* buf, size_t bytes, const cr_world* world,
                            uint64_t* ticket);
/* Active and queued requests, device bytes held by request state. */
cr_status cr_server_stats(cr_server* server, int32_t* active, int32_t* queued, size_t* pool_bytes);

/* ------------------------------------------------------------------------- */
/* Evaluation without allocation                                              */
/* ------------------------------------------------------------------------- */
#define CR_NOALLOC_MAX_PROBLEMS 256
#define CR_NOALLOC_MAX_TILES 32768

/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot let a library allocate device memory: a controller's real-time loop
 * that must not call cudaMalloc/cudaFree once running (those calls can take
 * unbounded time and synchronise the device), or an application whose own
 * pool owns all device memory.  It evaluates cost, gradient, flags and terms
 * (as cr_eval) of the trajectories of n_problems problems in one persistent
 * launch and allocates nothing: its scratch (problem and tile tables and a
 * work counter) is one fixed device array of about 0.6 MB inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   n_traj  host [n_problems]: trajectories of each problem (problems[p].seeds
 *           and n_seeds are unused)
 *   theta   device: each problem's block [n_traj[p]][H_p][dof], problem
 *           after problem
 *   cost, cfree, terms  device, per trajectory in the same order; grad like theta
 * At most CR_NOALLOC_MAX_PROBLEMS problems and CR_NOALLOC_MAX_TILES tiles (one
 * tile per trajectory when H >= 32, ceil(32/H) trajectories per tile below);
 * larger batches return CR_EINVAL.  The first call on a device looks up the
 * array's device address (a one-time set-up with that device current).  The
 * problem and tile tables are staged from host memory that exists only during
 * the call, with cudaMemcpyAsync from pageable memory: the call may block the
 * host until `stream` reaches those copies, and while `stream` is being
 * captured it returns CR_EINVAL and enqueues nothing.  Every call shares the
 * one array, so calls whose work overlaps on the GPU (different streams, or
 * different host threads) race: order them on one stream.  Results equal
 * those of cr_eval on each problem, bit for bit. */
cr_status cr_eval_batch_noalloc(const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                                const cr_params* params, const int32_t* n_traj, const float* theta,
                                float* cost, float* grad, uint8_t* cfree, float* terms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CRGB_H */
