// crgb_internal.cuh -- device-side views and launch helpers shared by the
// library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/crgb.h"
#include "fastdiv.h"

namespace crgb {

constexpr int kMaxDof = CR_MAX_DOF;
constexpr int kMaxSpheres = 1024;
constexpr int kMaxPairs = 65535;
constexpr int kPairTableSpheres = 64;  // robots up to this size get the pair table
constexpr int kMaxBoxes = 4096;
constexpr int kMaxHorizon = 128;
constexpr int kBoxChunk = 64;  // boxes staged in shared memory at a time
constexpr int kEvalBlock = 512; // threads of an evaluation CTA

// Programmatic dependent launch: the evaluation and optimiser kernels are
// launched so that the next one may start while the previous one finishes.
// Each waits (griddepcontrol.wait) before it touches anything the previous
// grid writes, then lets its own dependent start (launch_dependents); without
// a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename Kern, typename... Args>
inline cudaError_t launch_pdl(Kern kern, int grid, int block, size_t smem, cudaStream_t stream,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Robot as the kernels see it (device pointers into one allocation).
struct RobotView {
  int dof, n_spheres, n_pairs, n_groups;
  const float* fixed_tf;    // [(dof+1)*12]
  const int* axis;          // [dof]
  const float* lim;         // [5][dof]: q_lo, q_hi, v_max, a_max, j_max
  const float4* spheres;    // [M] centre (link frame), radius
  const int* sphere_link;   // [M]
  const float* sphere_off;  // [M] distance of the centre from its link's bounding-sphere centre
  const float4* link_bs;    // [dof] bounding sphere of each link's spheres (link frame centre,
                            //       radius; radius < 0 when the link has no enabled sphere)
  const float* link_dmax;   // [dof] largest sphere_off of each link
  const uint32_t* pairs;    // [P] i | (j << 16), grouped by link pair
  const int* pair_orig;     // [P] position of each pair in the caller's list (ties: first wins)
  const int4* groups;       // [G] (link a, link b, first pair, pair count)
  const int* link_start;    // [dof+1] spheres of link l are link_sph[link_start[l] .. link_start[l+1])
  const int* link_sph;      // [M] sphere indices ordered by link
  const float4* link_sph4;  // [M] the same spheres' centres and radii, in that order
  int max_link_spheres;     // largest sphere count of a link
  const int16_t* pair_at;   // [M][M] grouped index of the pair {i, j} (caller's first when listed
                            //   twice) or -1; robots of up to kPairTableSpheres spheres, else nullptr
  // dividers of work-item indices (set on the host): dof, spheres, link-pair
  // groups, largest sphere count of a link
  FastDiv fd_dof, fd_sph, fd_grp, fd_lsph;
};

// One box packed as five float4 rows: (R^T row k, t_k) for k = 0..2 so that
// u = R^T x + t is the point in the box frame, then (half extents, |h|), then
// (centre in the world frame, |h|), the box's bounding sphere.
struct BoxRows {
  float4 r0, r1, r2, h, c;
};

// One problem of a batch.
struct ProblemView {
  const BoxRows* boxes;
  int n_boxes;
  int horizon;
  int n_traj;          // trajectories of this problem in the evaluated batch
  int traj_base;       // index of its first trajectory in cost/cfree/terms
  long long var_base;  // float offset of its first trajectory in theta/grad
  float q_start[kMaxDof];
  float goal_p[3];
  float goal_R[9];     // row-major
  float goal_q[kMaxDof];  // Eq. 15 goal configuration when has_goal_q
  int has_goal_q;
  // time step and the weights of the derivative terms of Eq. 16 for this
  // problem (the parameters' values, or those a time-discretised solve sets
  // on the device between its two solves)
  float dt, w_vel, w_acc, w_jerk;
  // dividers of work-item indices (set on the host): horizon, stencil
  // samples of a trajectory times dof ((horizon + 1) dof)
  FastDiv fd_h, fd_hd;
};

// Arguments of the fused evaluation kernel.
struct EvalArgs {
  RobotView rb;
  cr_params prm;
  ProblemView prob0;             // single-problem launch
  const ProblemView* problems;   // batched launch: device table, or nullptr
  const int4* tiles;             // batched launch: (problem, first traj, n traj, -)
  int n_tiles;
  int* queue;                    // persistent launch: work counter (zeroed before launch), or nullptr
  int store_x;                   // set by the launcher: keep sphere positions in shared memory
  int no_store_x;                // tile option: 1 = never keep them, at most 64 registers a
                                 // thread (two 512-thread CTAs per SM); 0 = one CTA per SM,
                                 // positions kept when they fit; -1 = 1 when two CTAs fit
  int traj_per_tile;             // single-problem launch: trajectories per CTA
  int max_traj;                  // largest trajectory count of a tile
  int max_states;                // largest (trajectories x horizon) of a tile
  int max_horizon;
  const float* theta;
  float* cost;
  float* grad;
  uint8_t* cfree;
  float* terms;
  float* state_terms;            // [states][2] world and self cost of each state, or nullptr
};

// Shared-memory carve-up of the evaluation kernel (host and device agree).
// With store_x the world positions of every sphere of every state of the
// tile are kept (read by all later passes); without, they are recomputed
// from the link transforms (long horizons that would not fit).
struct EvalSmem {
  int off_fix, off_lim, off_sph, off_link, off_soff, off_lbs, off_ldm, off_lst, off_lsp, off_pairs, off_grp, off_th,
      off_lt, off_sc, off_x, off_sg, off_nz, off_rho, off_lm, off_mask, off_gmask, off_stw,
      off_sts, off_sta, off_gth, off_wsph, off_box, off_ee, off_sten, off_pb, off_db, off_sm, off_goal,
      off_free, bytes;
  __host__ __device__ static int align16(int x) { return (x + 15) & ~15; }
  __host__ __device__ void build(int dof, int M, int P, int G, int max_traj, int max_states,
                                 int n_warps, bool store_x) {
    int o = 0;
    auto take = [&](int nbytes) { int r = o; o = align16(o + nbytes); return r; };
    off_fix = take((dof + 1) * 12 * 4);
    off_lim = take(5 * dof * 4);
    off_sph = take(M * 16);
    off_link = take(M * 4);
    off_soff = take(M * 4);
    off_lbs = take(dof * 16);
    off_ldm = take(dof * 4);
    off_lst = take((dof + 1) * 4);
    off_lsp = take(M * 4);
    off_pairs = take(P * 4);
    off_grp = take(G * 16);
    off_th = take(max_states * dof * 4);
    off_lt = take((1 + max_states) * dof * 12 * 4);
    off_sc = take((1 + max_states) * dof * 8);
    off_x = take(store_x ? (1 + max_states) * M * 16 : 0);
    off_sg = take(max_states * M * 16);
    off_nz = take(max_states * ((M + 31) / 32) * 4);
    off_rho = take(max_states * dof * 16);
    off_lm = take(max_states * dof * 4);
    off_mask = take(max_states * dof * 8);  // 64 box bits per (state, link)
    off_gmask = take(max_states * ((G + 31) / 32) * 4);
    off_stw = take(max_states * 4);
    off_sts = take(max_states * 4);
    off_sta = take(max_states * 4);
    {  // joint gradients of the backward pass; before it, one bit per
       // (state, sphere) marking the items whose gradient can be non-zero
      const int mw = (M + 31) / 32;
      off_gth = take(max_states * (dof > mw ? dof : mw) * 4);
    }
    {  // per-warp sphere positions of the self term (without the cache), then
       // the world cost of each (state, sphere) in backward passes 1-2
      const int wsph = store_x ? 0 : n_warps * M * 16, wc = max_states * M * 4;
      off_wsph = take(wsph > wc ? wsph : wc);
    }
    off_box = take(kBoxChunk * (int)sizeof(BoxRows));
    off_ee = take(max_traj * 48);
    // stencil samples of a tile: nt (H + 1) <= max_states + max_traj
    const int n_samples = (max_states + max_traj) * dof;
    off_sten = take(n_samples * 3 * 4);
    off_pb = take(max_states * dof * 4);
    off_db = take(n_samples * 4);
    off_sm = take(n_samples * 4);
    off_goal = take(max_traj * 4);
    off_free = take(max_traj * 4);
    bytes = o;
  }
};

// Arguments of the optimiser kernels (one CTA per seed).
struct OptArgs {
  cr_params prm;
  const float* q_lo;   // device [dof]
  const float* q_hi;
  int dof;
  int n_seeds;
  int horizon;         // uniform horizon (single problem), or 0 with seed table
  const int4* seed_tab;  // batched: per listed seed (n vars, var offset, seed index, problem), or nullptr
  cr_opt_state st;
  int do_select;
  int do_propose;
  int init_best;       // first call after the initial evaluation: best := current
  int* reset_queue;    // the next evaluation's work counter, zeroed here (or nullptr)
  int early_loads;     // the previous grid is a candidate evaluation, which writes only
                       // cand_cost / cand_grad / cand_cfree: everything else may be
                       // loaded before that grid has finished
};

// Per-problem output pointers of the finishing kernel (runtime.cu).
struct ResultView {
  float* traj;
  float* cost;
  uint8_t* cfree;
  int* best;
  int* status;  // CR_OK, or CR_ENAN when a seed's best cost is not finite
  int n_seeds, n, seed_base, var_base;
};

// Per-problem outputs of the time-discretised solve (runtime.cu, k_time.cu);
// any may be nullptr.
struct TimeoptView {
  float* first;   // [H][dof] best trajectory of the first solve
  float* stage;   // [8] dt, w_vel, w_acc, w_jerk of the first, then of the second solve
  float* dt;      // [B] each seed's retimed step after the second solve
  float* score;   // [B] seed-choice score
  int* chosen;    // [1] chosen seed
};

// Reading of "scale the weights by the new dt" (Alg. "Time Discretization"):
// the weight on the square of the k-th derivative times (dt / dt0)^(2k).
struct TimeScale {
  float dt0, w_vel0, w_acc0, w_jerk0;  // the parameters' own step and weights
  float dt_min;                        // floor of the retimed step
  float rank_pose, rank_jerk, rank_time;  // seed-choice weights (App. "Solver details")
};

// launch helpers (k_eval.cu / k_opt.cu / runtime.cu)
cudaError_t launch_finish(const ResultView* res, int n_problems, const float* best_x,
                          const float* best_c, const uint8_t* best_cfree, cudaStream_t s);
cr_status check_params(const cr_params* p);
cr_status fill_problem(const cr_robot* rb, const cr_problem* pr, ProblemView* pv,
                       const cr_params* prm);
cudaError_t launch_fk(const RobotView& rb, const float* theta, int n, float* spheres, float* ee,
                      float* link_tf, cudaStream_t stream);
cudaError_t launch_eval(const EvalArgs& a, int grid, int block, cudaStream_t stream);
int eval_smem_bytes(const EvalArgs& a, int block);
int eval_blocks_per_sm(const EvalArgs& a, int block);
int eval_smem_limit();  // largest dynamic shared memory a tile may use
// IK mode (no sweep, speed or stencils): one thread per trajectory; launch_eval
// and the two queries above route IK-mode arguments here
cudaError_t launch_eval_ik(const EvalArgs& a, cudaStream_t stream);
int eval_ik_smem_bytes(int dof);
int eval_ik_blocks_per_sm(int dof);
cudaError_t launch_opt(const OptArgs& a, int n_max, cudaStream_t stream);
// particle-based optimisation over the seeds of a batch (k_particle.cu):
// phase 0 samples, phase 1 updates mean and covariance from the costs
cudaError_t launch_particle_batch(const int4* seed_tab, int n_seeds, int n_p, int phase, const float* eps,
                                  float* mu, float* sigma, float* particles, const float* cost, float beta,
                                  float k_mu, float k_sigma, cudaStream_t s);
cudaError_t launch_fill(float* p, long long n, float v, cudaStream_t s);
// time-discretised solve, between the two solves and after the second:
// k_time.cu (one CTA per problem)
cudaError_t launch_timeopt_mid(ProblemView* px, ProblemView* pc, int n_problems, const TimeoptView* tv,
                               const RobotView& rb, const float* best_x, const float* best_c,
                               const uint8_t* best_cfree, float* x, const TimeScale& sc, cudaStream_t s);
cudaError_t launch_timeopt_final(const ProblemView* px, int n_problems, const TimeoptView* tv,
                                 const RobotView& rb, const float* best_x, const float* best_c,
                                 const uint8_t* best_cfree, float* ws_dt, float* ws_score,
                                 const TimeScale& sc, cudaStream_t s);
// the time step and weights the scale gives for dt (jerk on or off); the same
// arithmetic on the host (first solve) and the device (second solve)
__host__ __device__ inline void time_scaled(const TimeScale& sc, float dt, bool jerk, float* out4) {
  const float r = dt / sc.dt0;
  const float r2 = r * r;
  out4[0] = dt;
  out4[1] = sc.w_vel0 * r2;
  out4[2] = sc.w_acc0 * (r2 * r2);
  out4[3] = jerk ? sc.w_jerk0 * (r2 * r2 * r2) : 0.f;
}
int opt_smem_bytes(int history, int n_max);

cr_status set_error(cr_status code, const char* msg);

}  // namespace crgb

// Handle types of the public ABI (opaque to callers).
struct cr_robot {
  int dof = 0, n_spheres = 0, n_pairs = 0;
  void* dev = nullptr;
  crgb::RobotView view{};
  float q_lo[CR_MAX_DOF], q_hi[CR_MAX_DOF];
};

struct cr_world {
  int n = 0;
  crgb::BoxRows* dev = nullptr;
};
