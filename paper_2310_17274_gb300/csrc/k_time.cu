// k_time.cu -- the device steps of Alg. "Time Discretization" (App.
// "Time-step Discretization") between and after the two solves of a
// time-discretised solve, so that the whole algorithm runs on the device
// without a host round trip:
//   mid:   per problem, the best seed of the first solve (the lowest-cost
//          collision-free seed, else the lowest-cost one), its retimed step
//          dt_opt = max(retime, dt_min), the derivative weights scaled to
//          dt_opt with the jerk term on, written into the problem tables the
//          second solve's kernels read; every seed's best iterate becomes a
//          seed of the second solve;
//   final: per problem, every seed of the second solve retimed and scored
//          (App. "Solver details"), and the chosen seed: the lowest score
//          among the collision-free seeds, else the solve's own best.
// One CTA per problem; maxima and the choice are order-free, so results do
// not depend on the launch.
#include <cuda_runtime.h>
#include <math.h>

#include "crgb_internal.cuh"
#include "k_time.cuh"

namespace crgb {

namespace {

constexpr int kTimeThreads = 256;

// the solve's best seed of a problem: lowest-cost collision-free, else
// lowest-cost (first index on ties; a NaN cost never wins)
__device__ int best_seed(const float* best_c, const uint8_t* best_cfree, int base, int B) {
  int bi = 0, bf = -1;
  float bc = INFINITY, fc = INFINITY;
  for (int b = 0; b < B; ++b) {
    const float c = best_c[base + b];
    if (c < bc) {
      bc = c;
      bi = b;
    }
    if (best_cfree[base + b] && (bf < 0 || c < fc)) {
      fc = c;
      bf = b;
    }
  }
  return bf >= 0 ? bf : bi;
}

__device__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  __syncthreads();
  return m;
}

__global__ void __launch_bounds__(kTimeThreads) k_timeopt_mid(ProblemView* px, ProblemView* pc, int P,
                                                              const TimeoptView* tv, RobotView rb,
                                                              const float* best_x, const float* best_c,
                                                              const uint8_t* best_cfree, float* x,
                                                              TimeScale sc) {
  __shared__ float red[32];
  __shared__ int s_best;
  __shared__ float s_q0[kMaxDof];
  const int p = blockIdx.x;
  if (p >= P) return;
  const int D = rb.dof;
  const int H = px[p].horizon, B = px[p].n_traj, base = px[p].traj_base;
  const long long vb = px[p].var_base, n = (long long)H * D;
  if (threadIdx.x < D) s_q0[threadIdx.x] = px[p].q_start[threadIdx.x];
  if (threadIdx.x == 0) s_best = best_seed(best_c, best_cfree, base, B);
  __syncthreads();
  const float* th = best_x + vb + s_best * n;
  const float dt = block_max(retime_part(th, s_q0, rb.lim, H, D, threadIdx.x, blockDim.x), red);
  if (threadIdx.x == 0) {
    float w1[4], w2[4];
    w1[0] = px[p].dt;
    w1[1] = px[p].w_vel;
    w1[2] = px[p].w_acc;
    w1[3] = px[p].w_jerk;
    time_scaled(sc, fmaxf(dt, sc.dt_min), true, w2);
    px[p].dt = pc[p].dt = w2[0];
    px[p].w_vel = pc[p].w_vel = w2[1];
    px[p].w_acc = pc[p].w_acc = w2[2];
    px[p].w_jerk = pc[p].w_jerk = w2[3];
    if (tv && tv[p].stage)
      for (int k = 0; k < 4; ++k) {
        tv[p].stage[k] = w1[k];
        tv[p].stage[4 + k] = w2[k];
      }
  }
  // every seed's best iterate seeds the second solve
  for (long long k = threadIdx.x; k < B * n; k += blockDim.x) x[vb + k] = best_x[vb + k];
  if (tv && tv[p].first)
    for (long long k = threadIdx.x; k < n; k += blockDim.x) tv[p].first[k] = th[k];
}

__global__ void __launch_bounds__(kTimeThreads) k_timeopt_final(const ProblemView* px, int P,
                                                                const TimeoptView* tv, RobotView rb,
                                                                const float* best_x, const float* best_c,
                                                                const uint8_t* best_cfree, float* ws_dt,
                                                                float* ws_score, TimeScale sc) {
  __shared__ float s_fix[(kMaxDof + 1) * 12];
  __shared__ int s_axis[kMaxDof];
  __shared__ ProblemView s_pv;
  const int p = blockIdx.x;
  if (p >= P) return;
  const int D = rb.dof;
  for (int k = threadIdx.x; k < (D + 1) * 12; k += blockDim.x) s_fix[k] = rb.fixed_tf[k];
  for (int k = threadIdx.x; k < D; k += blockDim.x) s_axis[k] = rb.axis[k];
  {
    const int* src = reinterpret_cast<const int*>(px + p);
    int* dst = reinterpret_cast<int*>(&s_pv);
    for (int k = threadIdx.x; k < (int)(sizeof(ProblemView) / 4); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const int H = s_pv.horizon, B = s_pv.n_traj, base = s_pv.traj_base;
  const long long vb = s_pv.var_base, n = (long long)H * D;
  // every seed retimed, a warp each
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = warp; b < B; b += nw) {
    float dt = retime_part(best_x + vb + b * n, s_pv.q_start, rb.lim, H, D, lane, 32);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dt = fmaxf(dt, __shfl_xor_sync(0xffffffffu, dt, o));
    if (lane == 0) {
      ws_dt[base + b] = dt;
      if (tv && tv[p].dt) tv[p].dt[b] = dt;
    }
  }
  __syncthreads();
  // scores at each seed's own step
  const RankWeights w{sc.rank_pose, sc.rank_jerk, sc.rank_time, 0.f};
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float s = seed_score(s_fix, s_axis, D, s_pv, best_x + vb + b * n, ws_dt[base + b], 0, w);
    ws_score[base + b] = s;
    if (tv && tv[p].score) tv[p].score[b] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0 && tv && tv[p].chosen) {
    float bs = INFINITY;
    int bi = -1;
    for (int b = 0; b < B; ++b)
      if (best_cfree[base + b] && score_better(ws_score[base + b], b, bs, bi)) {
        bs = ws_score[base + b];
        bi = b;
      }
    *tv[p].chosen = bi >= 0 ? bi : best_seed(best_c, best_cfree, base, B);
  }
}

}  // namespace

cudaError_t launch_timeopt_mid(ProblemView* px, ProblemView* pc, int n_problems, const TimeoptView* tv,
                               const RobotView& rb, const float* best_x, const float* best_c,
                               const uint8_t* best_cfree, float* x, const TimeScale& sc, cudaStream_t s) {
  if (n_problems <= 0) return cudaSuccess;
  k_timeopt_mid<<<n_problems, kTimeThreads, 0, s>>>(px, pc, n_problems, tv, rb, best_x, best_c, best_cfree,
                                                      x, sc);
  return cudaGetLastError();
}

cudaError_t launch_timeopt_final(const ProblemView* px, int n_problems, const TimeoptView* tv,
                                 const RobotView& rb, const float* best_x, const float* best_c,
                                 const uint8_t* best_cfree, float* ws_dt, float* ws_score,
                                 const TimeScale& sc, cudaStream_t s) {
  if (n_problems <= 0) return cudaSuccess;
  k_timeopt_final<<<n_problems, kTimeThreads, 0, s>>>(px, n_problems, tv, rb, best_x, best_c, best_cfree,
                                                        ws_dt, ws_score, sc);
  return cudaGetLastError();
}

}  // namespace crgb
