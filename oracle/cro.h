/*
 * cro.h -- FP64 CPU oracle for the batched cost-and-gradient evaluation, the
 * L-BFGS two-loop step and the parallel noisy line search of
 * "cuRobo: Parallelized Collision-Free Minimum-Jerk Robot Motion Generation"
 * (arXiv 2310.17274).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded reference
 * written from the paper's equations.  It shares no code, header, table or
 * constant with the CUDA library (include/crgb.h); only tests/, the smoke check
 * and the bench's CPU-baseline leg may load it.
 *
 * Every function states the passage of the paper it follows.  Readings of
 * passages that are silent or garbled are listed beside the function that
 * takes them.
 */
#ifndef CRO_H
#define CRO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRO_MAX_DOF 16
#define CRO_MAX_ALPHA 16
#define CRO_MAX_HISTORY 16

/* flags (same meaning as the library's, defined independently) */
#define CRO_SWEPT        1u   /* continuous collision sweep, Sec. 3.4 */
#define CRO_SPEED        2u   /* speed metric, Sec. 3.3 */
#define CRO_SELF         4u   /* self-collision term, Eq. 9 */
#define CRO_WOLFE        8u   /* Wolfe test in Alg. 1 */
#define CRO_STRONG_WOLFE 16u  /* strong variant of the Wolfe test */
#define CRO_IK_MODE      32u  /* single-state problem: no stencil terms, no sweep, no speed */
#define CRO_VEL_COST     64u  /* velocity logcosh of Eq. 16 over all samples (Q = all) */
#define CRO_CSPACE_GOAL  128u /* Eq. 15 joint-space goal cost (needs goal_q) */
#define CRO_NO_SELF_CHECK 256u /* IK mode without CRO_SELF: no self-collision in the validity flag */

/* Robot: serial revolute chain + sphere model (Sec. 3.1, App. E.1 kinematics data). */
typedef struct {
  int32_t dof;
  const double* fixed_tf;     /* [dof+1][12] row-major 3x4: F_0..F_{dof-1}, F_ee */
  const int32_t* axis;        /* [dof]  0 = x, 1 = y, 2 = z (revolute) */
  const double* q_lo;         /* [dof] position limits */
  const double* q_hi;
  const double* v_max;        /* [dof] symmetric velocity / acceleration / jerk limits */
  const double* a_max;
  const double* j_max;
  int32_t n_spheres;
  const double* spheres;      /* [M][4] centre in link frame, radius (r < 0 disables) */
  const int32_t* sphere_link; /* [M] link index 0..dof-1 */
  int32_t n_pairs;
  const int32_t* pairs;       /* [P][2] self-collision set S of Eq. 9 */
} cro_robot;

/* World: oriented boxes (Sec. 3.5 "Oriented Bounding Box"). */
typedef struct {
  int32_t n;
  const double* pose;         /* [n][7] centre xyz, quaternion wxyz */
  const double* half_ext;     /* [n][3] */
} cro_world;

typedef struct {
  double w_goal_pos, w_goal_rot, k_goal_pos, k_goal_rot;  /* alpha_0, alpha_1, alpha_2, alpha_3 (Eq. 14) */
  double w_coll;              /* beta_2 (Eq. 11) */
  double w_self;              /* beta_1 (Eq. 9) */
  double w_bound;             /* weight of Eq. 17 terms */
  double w_acc, w_jerk;       /* alpha_8, alpha_9 (Eq. 16) */
  double w_vel, k_vel;        /* alpha_6, alpha_7 (Eq. 16) */
  double eta;                 /* collision activation distance (Eq. 10) */
  double eta_bound;           /* eta_2 (Eq. 17) */
  double dt;
  int32_t sweep_steps;
  int32_t history;            /* L-BFGS memory m */
  int32_t n_alpha;
  double alpha[CRO_MAX_ALPHA];
  double armijo_c1, wolfe_c2;
  uint32_t flags;
  double w_cspace, k_cspace;  /* alpha_4, alpha_5 (Eq. 15, with CRO_CSPACE_GOAL) */
} cro_params;

void cro_params_default(cro_params* p);

/* ---- pieces, exposed for the pins ---------------------------------------- */

/* 3x4 link transforms T_0..T_{dof-1} (after each joint rotation), sphere
 * centres+radii in the world, and the end-effector 3x4 pose.  Any output may be NULL. */
void cro_fk(const cro_robot* rb, const double* theta, double* link_tf, double* spheres,
            double* ee);

/* Signed distance from point x to a box (centre c, rotation from quaternion
 * wxyz, half extents h) and its gradient in the world frame (grad may be NULL). */
double cro_box_sdf(const double* pose7, const double* half_ext, const double* x, double* grad);

/* Eq. 10: smoothed collision distance d_c(d) of a penetration depth d and its slope. */
double cro_smooth_distance(double d, double eta, double* slope);

/* Eq. 17: bound cost of value q against [lo, hi] and its slope. */
double cro_bound_cost(double q, double lo, double hi, double eta2, double* slope);

/* Sweep of one sphere (radius r) against one box for the waypoint x1 with
 * neighbours x0, x2 (Sec. 3.4).  Returns the summed smoothed distance S and
 * writes dS/dx1 (surrogate gradient) into g1.  x0 / x2 may be NULL (no sweep
 * on that side).  If `margin` is non-NULL it receives the smallest distance of
 * any branch decision taken from its threshold (diagnostic only). */
double cro_sweep_box(const double* pose7, const double* half_ext, double r, const double* x0,
                     const double* x1, const double* x2, double eta, int32_t steps, double* g1,
                     double* margin);

/* Eq. 9 for one state: returns the (unweighted) largest pair penetration,
 * writes the argmax pair index (or -1) and the gradient w.r.t. the sphere
 * centres ([M][3], may be NULL, unweighted). */
double cro_self_penetration(const cro_robot* rb, const double* spheres_world, int32_t* argmax,
                            double* grad_x);

/* Five-point stencils of App. A.5 at ext indices 2..H+2 of the padded
 * sequence ext = [q0,q0,q0, theta_1..theta_H, theta_H, theta_H].
 * vel/acc/jerk: [H+1][dof]. */
void cro_stencil(int32_t H, int32_t dof, const double* q0, const double* theta, double dt,
                 double* vel, double* acc, double* jerk);

/* Eq. 14 pose cost of an end-effector 3x4 pose against goal (xyz + wxyz).
 * Writes dC/dp (3) and dC/dR (9, row-major) if non-NULL. */
double cro_goal_cost(const cro_params* prm, const double* ee, const double* goal7, double* dp,
                     double* dR);

/* ---- the whole evaluation ------------------------------------------------ */

/* terms per trajectory: [0] world (Eq. 11), [1] self (Eq. 9), [2] bound (Eq. 17),
 * [3] smoothness (Eq. 16), [4] goal (Eq. 14). */
#define CRO_N_TERMS 5

/* Cost and gradient of B trajectories theta [B][H][dof] of one problem.
 * cost [B]; grad [B][H][dof] (may be NULL); cfree [B] (may be NULL);
 * terms [B][5] (may be NULL); margin [B] (may be NULL): smallest distance of
 * any discrete decision from its threshold, for tolerance bookkeeping. */
void cro_eval(const cro_robot* rb, const cro_world* w, const double* q_start, const double* goal7,
              const double* goal_q,
              const cro_params* prm, int32_t H, const double* theta, int32_t B, double* cost,
              double* grad, uint8_t* cfree, double* terms, double* margin);

/* cro_eval with per-state outputs, for parity checks that skip single
 * states instead of whole trajectories (any output may be NULL):
 *   state_terms  [B][H][2]: the world cost (Eq. 11, summed over spheres) and
 *                the self cost (Eq. 9, weighted) of each state theta_t;
 *   state_margin [B][H]: the smallest distance from its threshold of any
 *                decision that sets that state's world or self cost or its
 *                gradient (sweep activation and stop tests, face and pair
 *                argmax, the zero of max(0, .) in Eq. 9); a decision of state
 *                t reaches the gradient rows t-1, t, t+1 (speed metric);
 *   state_clear  [B][H]: the smallest discrete clearance of the state (every
 *                sphere against every box, every pair of S unless the self
 *                check is off); the state is collision-free when it is > 0. */
void cro_eval_states(const cro_robot* rb, const cro_world* w, const double* q_start,
                     const double* goal7, const double* goal_q, const cro_params* prm, int32_t H,
                     const double* theta, int32_t B, double* cost, double* grad, uint8_t* cfree,
                     double* terms, double* margin, double* state_terms, double* state_margin,
                     double* state_clear);

/* ---- optimiser (Sec. 4.1, Alg. 1, App. A.7 L-BFGS step update) ----------- */

/* Per-seed optimiser state.  All arrays are caller-owned. */
typedef struct {
  int32_t n;         /* variables per seed = H*dof */
  int32_t m;         /* history length */
  double* x;         /* [n] current iterate */
  double* g;         /* [n] its gradient */
  double* c;         /* [1] its cost */
  double* x_prev;    /* [n] */
  double* g_prev;    /* [n] */
  double* s;         /* [m][n], newest last */
  double* y;         /* [m][n] */
  double* rho;       /* [m] */
  int32_t* iter;     /* [1] iterations taken (0 = no previous iterate) */
} cro_lbfgs;

/* Update the history with the step to the current iterate and compute the
 * L-BFGS direction d = -H g by the two-loop recursion.  Writes d [n]. */
void cro_lbfgs_direction(cro_lbfgs* st, double* d);

/* Candidates of Alg. 1: cand[l] = clip(x + alpha_l d) for l < n_alpha.
 * lo/hi are per-joint limits, dof the row length of x. */
void cro_ls_candidates(const cro_params* prm, int32_t n, int32_t dof, const double* q_lo,
                       const double* q_hi, const double* x, const double* d, double* cand);

/* Selection of Alg. 1: returns the largest index passing Armijo (and Wolfe
 * when enabled), else 0.  `margin` (may be NULL) receives the smallest
 * distance of any test from its threshold. */
int32_t cro_ls_select(const cro_params* prm, int32_t n, double c0, const double* g0,
                      const double* d, const double* cand_cost, const double* cand_grad,
                      double* margin);

/* Full solve of one problem: iters L-BFGS iterations with the noisy line
 * search and best-iterate tracking (Sec. 4.1).  seeds [B][H][dof].
 * best_x [B][H][dof], best_c [B], best_cfree [B]. */
void cro_solve(const cro_robot* rb, const cro_world* w, const double* q_start,
               const double* goal7, const double* goal_q, const cro_params* prm, int32_t H, int32_t B,
               const double* seeds, int32_t iters, double* best_x, double* best_c,
               uint8_t* best_cfree);

/* ------------------------------------------------------------------------ */
/* Sec. 4.2 particle-based optimisation (Eq. 12, Eq. 13, Alg. "Particle-Based */
/* Optimization"), one seed: mean mu [n] and diagonal covariance sigma [n].  */
/* ------------------------------------------------------------------------ */

/* SAMPLE: particles [n_p][n] = mu + sqrt(sigma) * eps, eps [n_p][n] the
 * zero-mean unit Gaussian samples (drawn by the caller). */
void cro_particle_sample(int32_t n, int32_t n_p, const double* mu, const double* sigma,
                         const double* eps, double* particles);

/* UPDATE: exponential utility w_i = e^{c_i} / sum_j e^{c_j}, c = -cost / beta
 * (evaluated after subtracting the smallest cost, which leaves w unchanged);
 * mu <- (1 - k_mu) mu + k_mu sum_i w_i theta_i (Eq. 12);
 * sigma <- (1 - k_sigma) sigma + k_sigma sum_i w_i (theta_i - mu_prev)^2
 * (Eq. 13 as read: the printed update is garbled).  Writes w [n_p] if not
 * NULL; mu and sigma are updated in place. */
void cro_particle_update(int32_t n, int32_t n_p, const double* cost, const double* particles,
                         double beta, double k_mu, double k_sigma, double* mu, double* sigma,
                         double* w);

/* ------------------------------------------------------------------------ */
/* Sec. 5 Alg. "Parallel Steering": discretise each edge e = [theta_0,        */
/* theta_1] into n + 1 samples l_i = theta_0 + (i / n)(theta_1 - theta_0),    */
/* i = 0..n, check every sample (mask_samples: the discrete clearance test of */
/* the evaluation, every sphere clear of every box and every pair of S        */
/* separated), and keep the last valid sample before the first invalid one.   */
/* ------------------------------------------------------------------------ */

/* n of the algorithm: the largest joint displacement of any edge over the
 * resolution r, floored, plus one.  edges [E][2][dof]. */
int32_t cro_steer_steps(int32_t E, int32_t dof, const double* edges, double r);

/* For each edge: last [E] = index of the last valid sample before the first
 * invalid one (n when every sample is valid, -1 when sample 0 is invalid);
 * v_new [E][dof] = that sample (theta_0 when last = -1); dist [E] = its
 * Euclidean joint-space distance from theta_0. */
void cro_steer(const cro_robot* rb, const cro_world* w, int32_t E, const double* edges, int32_t n,
               int32_t* last, double* v_new, double* dist);

/* ------------------------------------------------------------------------ */
/* App. "Time-step Discretization" (Alg. "Time Discretization"): retime       */
/* ------------------------------------------------------------------------ */

/* The time step that puts a trajectory at the robot's limits: the App. A.5
 * derivatives scale as 1/dt, 1/dt^2, 1/dt^3, so with v1, a1, j1 the stencils
 * at dt = 1 the smallest dt keeping every sample within the limits is
 * max over samples and joints of |v1|/v_max, sqrt(|a1|/a_max), cbrt(|j1|/j_max).
 * theta [H][dof] (one trajectory), q0 the start configuration. */
double cro_retime(const cro_robot* rb, int32_t H, const double* q0, const double* theta);

/* ------------------------------------------------------------------------ */
/* App. "Solver details": choosing among the seeds of a solve                 */
/* ------------------------------------------------------------------------ */

/* Pose error of a configuration's end effector against goal7 (xyz + quat
 * wxyz): |p - p_g| + d_q with d_q = (3 - tr(R_g^T R)) / 4 of Eq. 14. */
double cro_pose_error(const cro_robot* rb, const double* q, const double* goal7);

/* Score of each of B seeds (theta [B][H][dof], start q0):
 *   ik != 0:  w_pose * e_pose(theta_H) + w_dist * |theta_H - q0|
 *   ik == 0:  w_pose * e_pose(theta_H) + w_jerk * max |jerk| + w_time * H * dt_b
 * with the jerk of App. A.5's five-point stencil at dt_b (dt[b], or dt_all
 * when dt is NULL) over every sample and joint.  Returns the index of the
 * lowest score among seeds with cfree[b] != 0 (the lowest index on ties; a
 * NaN score never wins), or -1 when there is none. */
int32_t cro_rank_seeds(const cro_robot* rb, int32_t H, int32_t B, const double* q0, const double* goal7,
                       const double* theta, const uint8_t* cfree, const double* dt, double dt_all,
                       int32_t ik, double w_pose, double w_jerk, double w_time, double w_dist, double* score);

/* ------------------------------------------------------------------------ */
/* Alg. "Time Discretization" (App. "Time-step Discretization")               */
/* ------------------------------------------------------------------------ */

/* The parameters for step dt: prm with dt replaced and the weight on the
 * square of the k-th derivative (velocity k = 1, acceleration 2, jerk 3)
 * multiplied by (dt / prm->dt)^(2k) (reading of "scale the weights by the
 * new dt": the smoothness of the same waypoints keeps its value); jerk = 0
 * sets the jerk weight to zero. */
void cro_time_scaled_params(const cro_params* prm, double dt, int32_t jerk, cro_params* out);

/* The whole algorithm for one problem, in its order:
 *   1. cro_solve (iters1) with cro_time_scaled_params(prm, dt_init, no jerk);
 *   2. the best seed of 1 (lowest-cost collision-free, else lowest-cost),
 *      dt_opt = max(cro_retime(that seed), dt_min);
 *   3. cro_solve (iters2) from every seed's best iterate of 1 with
 *      cro_time_scaled_params(prm, dt_opt, jerk on);
 *   4. dt[b] = cro_retime of every seed of 3; cro_rank_seeds with those steps
 *      and the weights w_pose, w_jerk, w_time (App. "Solver details").
 * Writes first [H][dof] (best of 1), stage [8] (dt and the velocity,
 * acceleration and jerk weights of 1, then of 3), traj [B][H][dof], cost [B]
 * and cfree [B] (the best iterates of 3), dt [B], score [B]; returns the
 * chosen seed: the lowest score among the collision-free seeds, else the
 * best seed of 3 by the rule of step 2. */
int32_t cro_time_discretized_solve(const cro_robot* rb, const cro_world* w, const double* q_start,
                                   const double* goal7, const double* goal_q, const cro_params* prm,
                                   int32_t H, int32_t B, const double* seeds, int32_t iters1, int32_t iters2,
                                   double dt_init, double dt_min, double w_pose, double w_jerk, double w_time,
                                   double* first, double* stage, double* traj, double* cost, uint8_t* cfree,
                                   double* dt, double* score);

#ifdef __cplusplus
}
#endif
#endif
